"""CPU FP64 oracle (test infrastructure only; see sbd_oracle.py)."""
