"""CPU oracle for the FLD radiation substep (test infrastructure only).

Imported by the tests, the smoke check and the benchmark's CPU-baseline leg;
never by the library.
"""
