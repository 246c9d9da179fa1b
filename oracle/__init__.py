"""Plain FP64 CPU oracle of the BTDF-IB / D2Q9 LBM step.

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU baseline of
the benchmark import this package.
"""
