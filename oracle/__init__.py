"""FP64 CPU oracle (test infrastructure only; see ptycho_oracle's docstring)."""
