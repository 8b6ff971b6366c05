"""GB300 (sm_103a) library for the two-component regularised colour-gradient
lattice Boltzmann step of direct-writing printing (Monteferrante et al.,
arXiv 2102.02655): CUDA kernels behind the C ABI of include/lbm.h, with a
thin ctypes binding (``lbm``) and seeded synthetic inputs (``inputs``)."""
from . import inputs  # noqa: F401
