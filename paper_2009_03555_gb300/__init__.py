"""GB300-native Hartree-Fock exchange construction (screened contracted-Gaussian
ERIs contracted with a sparse density matrix), after the method of
arXiv 2009.03555 (Sec. 2-3).  The compute path is the CUDA library libhfx.so
(C ABI in include/hfx.h); ``hfx`` is its thin Python binding."""
from . import hfx  # noqa: F401
from .hfx import Basis, HFXError, Quartets, make_opts  # noqa: F401
