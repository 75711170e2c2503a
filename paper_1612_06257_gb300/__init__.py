"""Batched HighwayHash (arXiv:1612.06257) for NVIDIA GB300, behind a C ABI.

``paper_1612_06257_gb300.hh`` is the ctypes binding of libhh (include/hh.h),
which also hashes with the paper's SipTreeHash (Section 3);
``workloads`` builds the seeded synthetic batches; ``serve`` is the
continuous-batching request server; ``build`` compiles libhh.so with nvcc
for sm_103a.
"""
