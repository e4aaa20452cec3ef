"""GB300-native multiscale fit with compactly supported Wendland kernels.

The compute path lives in ``libms.so`` (hand-written CUDA for sm_103a behind a C ABI);
``paper_2503_04914_gb300.ms`` is the thin ctypes binding with the same names.
Importing the package does not load the library; ``inputs`` holds the seeded
workload generators.
"""
