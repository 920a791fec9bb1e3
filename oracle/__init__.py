"""FP64 CPU oracle of the HWENO-GR scheme (test infrastructure only)."""
