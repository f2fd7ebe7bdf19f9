"""GB300-native relational operator library (arxiv 2506.09226 hot path).

The operators run as hand-written CUDA kernels for sm_103a inside ``libqe.so``
behind a C ABI (``include/qe.h``); ``qe`` is the thin ctypes binding.  Import
of this package does not load the library; the binding loads it on first use
and raises if it is missing.
"""
