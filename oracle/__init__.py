"""CPU oracle of the multi-receiver RF Gaussian renderer.

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` use it; the product library never does.
"""
