"""FP64 CPU oracle for VDAMP -- test infrastructure only (see vdamp_oracle)."""
