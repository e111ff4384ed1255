"""FP64 CPU oracle (test infrastructure only; see trd_oracle.py)."""
