"""CPU oracle (test infrastructure): complex128 statement of the NLINV hot path.  Not part of the library."""
