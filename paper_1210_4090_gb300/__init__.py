"""GB300-native solver for the fully discrete Lax--Oleinik scheme.

Bouillard, Faou & Zavidovique, "Fast weak-KAM integrators for separable
Hamiltonian systems": one time step is a min-plus convolution of u with the
convex kernel h*L(d*dx/h) along each axis (eq. eqconvol, Remark rk28) followed
by the potential term -h*V.  The compute path is the C-ABI library built from
``csrc/`` (hand-written sm_103a kernels); ``hjlo`` is its Python binding.
Submodules are imported lazily so that ``workloads`` can be used without the
compiled library.
"""
import importlib

__all__ = ["hjlo", "workloads", "dist", "autograd"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
