"""CPU oracle of the hybrid LU-QR solver.

Test infrastructure only: the test suite, the smoke check and the benchmark's CPU
baseline leg use it; the GPU library never does.
"""
