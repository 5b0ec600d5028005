"""CPU FP64 oracle (test infrastructure only; see ch_oracle.py)."""
