"""GB300-native relativistic lattice Boltzmann update (arXiv 2205.04658).

The compute path is the CUDA library ``librlbm.so`` built from ``csrc/``;
``rlbm`` is its thin ctypes binding.  Importing the package loads nothing;
the library is loaded on first use and its absence is an error.
"""
