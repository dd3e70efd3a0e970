"""CPU checker for the rule path (test infrastructure only; never imported by the library)."""
