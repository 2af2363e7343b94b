"""GB300-native FDTD/PIC time step of the MITHRA full-wave FEL method
(arXiv 1612.03310): NSFD potential update with Mur boundaries, E/B from the
potentials, trilinear gather, Boris push through the boosted undulator field
and charge/current deposition, as hand-written CUDA for sm_103a behind the
C ABI declared in include/mithra.h.

The CUDA library is loaded on first use; when it is missing the binding
raises instead of falling back to any CPU path.
"""
from . import inputs  # noqa: F401  (seeded synthetic inputs; no method arithmetic)

__all__ = ["inputs", "mithra"]


def __getattr__(name):
    if name == "mithra":
        import importlib
        return importlib.import_module(__name__ + ".mithra")
    raise AttributeError(name)
