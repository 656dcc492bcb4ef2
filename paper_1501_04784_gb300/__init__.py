"""GB300-native global stiffness-matrix construction (3D Poisson, Hex8 / Tet4).

The compute path is the CUDA library ``_build/libfem.so`` (sources in
``csrc/``, C ABI in ``include/fem.h``); ``fem`` is its torch binding and
``autograd`` wraps the build and its backward pass as a ``torch.autograd.Function``.
"""
from . import abi  # noqa: F401
from ._build import build  # noqa: F401


def __getattr__(name):
    # the torch-facing modules load lazily so that building needs no GPU
    if name in ("fem", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
