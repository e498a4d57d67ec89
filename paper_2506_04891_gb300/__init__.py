"""GB300-native layered QML state-vector simulator (arXiv 2506.04891 hot path).

Importing the package is cheap; the CUDA library is loaded on first use of
``paper_2506_04891_gb300.qlayer`` and fails loudly when it is missing.
"""
__all__ = ["qlayer", "workloads"]


def __getattr__(name):
    if name in ("qlayer", "workloads", "serving", "torch_fn", "tune", "dist"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
