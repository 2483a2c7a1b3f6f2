"""Seeded synthetic input generators (inputs only; no solver arithmetic)."""
from .haar import (BATCH_LEVELS, Basis, BatchWorkload, Kernel, Workload, batch_instances,
                   batch_workload, compressed_pattern, compressed_pattern_two_term, compressed_values,
                   compressed_values_nonsym,
                   cutoff_parameters, fwt, haar_basis,
                   haar_workload, level_side, mass_matrix, own_pattern, rhs, workload_1d, workload_2d, workload_autograd)

__all__ = ["BATCH_LEVELS", "BatchWorkload", "batch_instances", "batch_workload", "Basis", "Kernel", "Workload", "compressed_pattern", "compressed_pattern_two_term", "compressed_values",
           "compressed_values_nonsym",
           "cutoff_parameters", "fwt",
           "haar_basis", "haar_workload", "level_side", "mass_matrix", "own_pattern", "rhs", "workload_1d", "workload_2d",
           "workload_autograd"]
