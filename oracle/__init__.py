"""FP64 CPU oracle of the S-BKI map update (test infrastructure only)."""
