"""CPU oracle of the HFDIB steady-RANS SIMPLE sweep (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
arm may import this package.  The product path never does.
"""
