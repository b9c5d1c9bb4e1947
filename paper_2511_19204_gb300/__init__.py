"""GB300-native Hermite-spline MPPI hot path (arXiv 2511.19204, Sec. III).

The compute path lives in the CUDA library ``libmppi.so`` behind the C ABI declared in
``include/mppi.h``; ``paper_2511_19204_gb300.mppi`` binds it with the same names.
``paper_2511_19204_gb300.synth`` holds the seeded synthetic robots and workloads.
Importing the package loads nothing; the library loads on first use of ``mppi``.
"""
