"""SGS-PFP steady Boltzmann solver for GB300 (sm_103a): C-ABI CUDA library + thin binding."""
