"""Test infrastructure: the FP64 CPU oracle (plain C, see ohm_oracle.c) and its ctypes wrapper.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.
"""
