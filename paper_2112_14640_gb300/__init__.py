"""GB300-native multi-RHS Wilson, Brillouin and staggered Dirac operators and
their Krylov solvers (Duerr, arXiv:2112.14640), as hand-written sm_103a CUDA
behind a C ABI (``include/dirac.h``) with a thin ctypes binding."""
