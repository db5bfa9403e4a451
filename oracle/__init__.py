"""Plain FP64 CPU oracle for the f(R) FAS multigrid solver (test infrastructure only)."""
