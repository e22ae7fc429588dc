"""CPU oracle (test infrastructure only): a plain FP64 statement of the
adaptive s-step GMRES, used by the tests, the smoke check and the CPU
baseline of the benchmark.  The library never imports it."""
