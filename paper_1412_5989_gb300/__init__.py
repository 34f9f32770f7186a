"""GB300-native construction of the half-stored M-scheme CI Hamiltonian.

The compute path lives in the CUDA library ``libcih.so`` (C ABI, declared in
``include/cih.h``); ``paper_1412_5989_gb300.cih`` is its thin ctypes binding.
Importing this package does not load the library; the binding does, and it
raises if the library has not been built.
"""
