"""CPU oracle (test infrastructure only; see dmr_oracle's module docstring)."""
