"""GB300 (sm_103a) implementation of the HFDIB steady-RANS SIMPLE sweep.

Submodules:
    geometry  seeded synthetic inputs (grids, lambda, wall distance, cases)
    hfdib     ctypes binding of the C-ABI library libhfdib.so
"""
