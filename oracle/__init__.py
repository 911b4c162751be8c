"""CPU FP64 oracle (test infrastructure only; see qsel_oracle)."""
