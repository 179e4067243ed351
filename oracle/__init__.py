"""FP64 reference implementation of the MAGPIE sweep (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package; the CUDA library and its binding never do.
"""
