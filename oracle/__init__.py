"""FP64 CPU oracle of the free-energy LB time step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline/reference leg
may import this package; the CUDA product path never does.
"""
