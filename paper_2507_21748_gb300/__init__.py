"""GB300-native semi-implicit Fourier-spectral Cahn-Hilliard solver (evoxels method).

The compute path is the CUDA library ``libevx.so`` (C-ABI declared in
``include/evx.h``); ``paper_2507_21748_gb300.evx`` is its thin ctypes binding.
Importing the package does not load the library; importing ``.evx`` does, and
fails loudly if it has not been built.
"""
