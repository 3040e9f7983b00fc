"""CPU oracle for numerical entanglement (test infrastructure only)."""
