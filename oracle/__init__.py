"""FP64 CPU oracle (test infrastructure only; see cfust_oracle's module docstring)."""
