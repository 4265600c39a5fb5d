"""FP64 CPU oracle of the anchor-Gaussian rendering path.

Test infrastructure only: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it; the CUDA package never imports it.
"""
