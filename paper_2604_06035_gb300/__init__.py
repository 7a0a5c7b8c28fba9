"""GB300-native level-by-level multigrid Poisson solve on RAMSES oct grids
(cuRAMSES, arXiv 2604.06035): a C-ABI CUDA library (libcmg.so) for sm_103a and
a thin ctypes binding.  Importing the package loads nothing; the binding in
``cmg`` loads the library on first use and raises if it is missing."""
__all__ = ["cmg", "inputs"]
