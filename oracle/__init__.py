"""FP64 CPU oracle of the MTP hot path (test infrastructure; see oracle.py)."""
