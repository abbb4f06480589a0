"""Plain FP64 CPU oracle of the HOSC scheme (test infrastructure only; see hosc_oracle.py)."""
