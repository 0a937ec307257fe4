"""FP64 CPU oracle of the PIBM coupled step: test infrastructure only.

Nothing in the CUDA library imports this package; the tests, the smoke check
and the benchmark's CPU baseline leg are its only users.
"""
