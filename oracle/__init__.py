"""FP64 CPU oracle of the implicit-complementarity IPM (test infrastructure only)."""
