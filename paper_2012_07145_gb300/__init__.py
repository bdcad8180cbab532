"""Fused image-pipeline kernels for GB300 (sm_103a).

Multi-stage image pipelines -- DAGs of point-wise, 2-D stencil, pyramid
down/upsample and histogram stages -- run as fused, overlapped-tile CUDA
kernels behind the C ABI of include/hp.h.  This package holds the CUDA sources
(csrc/), the in-tree build (build.py), the ctypes binding (hp.py), pipeline
builders for the evaluated apps (pipelines.py) and seeded input generators
(synth.py).  Nothing here computes on the CPU: calls fail if libhp.so is absent.
"""
