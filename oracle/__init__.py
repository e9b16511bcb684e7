"""FP64 CPU oracle for CoR-UTV: test infrastructure, never the product path."""
