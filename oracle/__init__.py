"""FP64 CPU oracle of the TreeCode method (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package; the library never does.
"""
