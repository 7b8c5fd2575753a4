"""FP64 CPU oracle for the SSSP marcher: test infrastructure only (see sssp_oracle.py)."""
