"""GB300-native thick-restart Lanczos for Hermitian J-symmetric matrices (TRLAN-JSYM).

The compute path lives in ``libjtrlan.so`` (hand-written CUDA for sm_103a behind a
C ABI, declared in ``include/jtrlan.h``); ``binding`` is a thin ctypes layer over it.
Importing this package does not load the library; ``binding.load()`` does, and it
raises if the library has not been built.
"""
