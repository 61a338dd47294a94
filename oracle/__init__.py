"""CPU FP64 oracle of the BoxMG V-cycle -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library never does.
"""
