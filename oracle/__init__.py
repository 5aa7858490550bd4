"""CPU oracle of the finite-volume Euler solver: TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The GPU path never imports, links or calls it.
"""
