"""FP64 CPU oracle of the rotating IMEX-DG hot path.

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py, never by the product package.
"""
