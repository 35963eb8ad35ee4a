"""GB300-native fast multipole BEM operator for 3-D Helmholtz collocation
problems (single and double layer on flat triangles, centroid collocation).

The compute path lives in the CUDA shared library built from ``csrc/``;
``_lib`` is its thin ctypes binding and ``operator`` the PyTorch-facing
wrapper.  Importing this package does not load the CUDA library; the first
use of ``Operator`` does, and fails loudly if it is missing.
"""
__all__ = ["Operator"]


def __getattr__(name):
    if name == "Operator":
        import importlib
        return importlib.import_module(".operator", __name__).Operator
    raise AttributeError(name)
