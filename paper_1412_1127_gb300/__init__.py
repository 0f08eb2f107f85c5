"""GB300-native runtime for the device side of an OpenACC accelerator region
(IPMACC, arXiv 1412.1127): `loop independent` work sharing with the
`reduction(op:var)` clause, the row nest, and the Listing-1 matrix nest.

The compute path is the C-ABI library ``libaccr.so`` (hand-written CUDA for
sm_103a, declared in ``include/accr.h``); ``paper_1412_1127_gb300.api`` is a
thin ctypes binding with the same function names.  The library is loaded on
first use, so the input generators (``inputs``) and the build script
(``build``) work on machines without a GPU.
"""
