"""cxbwt: multi-string BWT construction for short DNA reads on GB300 (sm_103a).

The compute path is the CUDA library ``libcxbwt.so`` (built from ``csrc/``)
behind the C ABI in ``include/cxbwt.h``; ``binding`` is a thin ctypes layer
over it.  ``synth`` holds the seeded workload generators.
"""
