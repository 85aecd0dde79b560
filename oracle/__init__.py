"""CPU FP64 oracle (test infrastructure only; see tca_oracle.py)."""
