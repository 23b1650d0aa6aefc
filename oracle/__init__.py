"""FP64 CPU oracle (test infrastructure only; see fastgraspd_oracle)."""
