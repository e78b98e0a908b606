"""GB300-native state-vector simulator for dynamic circuits (mid-circuit
measurement, reset, if/else on classical predicates, bounded loops), after
arXiv 2604.11599.  The compute path is the CUDA library ``libsv`` (C-ABI in
``include/sv.h``); this package holds its Python binding, the IR builder and
the seeded workload generators.  Importing the package does not load the
CUDA library; ``paper_2604_11599_gb300.sv`` does."""

__all__ = ["ir", "workloads"]
