"""CPU FP64 oracle of the multiscale fit.  Test infrastructure only: imported by the
tests, the package smoke check and the benchmark's CPU-baseline leg, never by the
library itself."""
