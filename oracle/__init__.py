"""FP64 CPU oracle of the mDPD hot path -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package; the CUDA product path never does.
"""
