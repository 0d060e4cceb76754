"""GB300-native SALE staggered-grid hydro cycle (ScalSALE, arXiv 2209.01983).

The compute path is the C-ABI library ``libsale_gb300.so`` (hand-written
sm_103a CUDA kernels); ``paper_2209_01983_gb300.sale`` is its thin ctypes
binding and ``paper_2209_01983_gb300.inputs`` builds seeded synthetic inputs.
Importing the package loads neither.
"""
