"""FP64 CPU oracle for the cubic Klein-Gordon spectral scheme (test infrastructure only)."""
