"""The oracle: a plain, serial, FP64 CPU implementation of the paper's event
generator (LO matrix element, Sudakov veto-algorithm dipole shower, Durham /
thrust / heavy-jet-mass observables).  Test infrastructure: only the tests, the
smoke check and the benchmark's CPU-baseline leg may use it.  It shares no code
with the CUDA library."""
