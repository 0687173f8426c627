"""GB300-native (sm_103a) hot path of subquadratic network reconstruction
(Peixoto, arXiv:2401.01404): exact pair gains, NNDescent/FindBest best-pair
search and greedy coordinate descent, as a C-ABI CUDA library (``librecon.so``)
with a thin ctypes binding in :mod:`.recon`.

Importing the package loads nothing; :mod:`.recon` loads the library and
fails loudly if it has not been built.
"""
__all__ = ["recon", "inputs"]
