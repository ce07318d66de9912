"""FP64 CPU oracle of the GATE TE iteration -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package; the CUDA product path never
does.
"""
