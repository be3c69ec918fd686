"""FP64 CPU oracle (test infrastructure only; see mdp_oracle.py)."""
