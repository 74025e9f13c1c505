"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no arithmetic of the eigensolver itself: it discretises the
test PDE into a DIA pencil (A, B), draws the random starting block, and reads
the stored workload definitions (disk centre/radius, orders p, q, block k), and
places the disks of the seeded batch workload.
"""
from .generator import (  # noqa: F401
    Pencil, make_pencil, random_block, orthonormal_random_block, load_workload,
    workload_names, closed_form_spectrum, batch_problems, batch_workload_names, BATCH_GRIDS,
)
