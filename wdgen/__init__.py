"""Seeded synthetic input generators (inputs only; no solver arithmetic)."""
from .haar import (Basis, Kernel, Workload, compressed_pattern, compressed_values, fwt,
                   haar_basis, haar_workload, level_side, rhs, workload_1d, workload_2d,
                   workload_autograd)

__all__ = ["Basis", "Kernel", "Workload", "compressed_pattern", "compressed_values", "fwt",
           "haar_basis", "haar_workload", "level_side", "rhs", "workload_1d", "workload_2d",
           "workload_autograd"]
