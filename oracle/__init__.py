"""FP64 CPU oracle (test infrastructure only; see inla_oracle.py)."""
