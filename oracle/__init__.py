"""FP64 CPU oracle (test infrastructure only; see os3d_oracle)."""
