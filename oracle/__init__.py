"""Plain FP64 CPU oracle of the SGS-PFP solver (test infrastructure only)."""
