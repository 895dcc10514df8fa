"""CPU oracle for the FLD radiation substep (test infrastructure only).

Imported by the tests, the smoke check and the benchmark's CPU-baseline leg;
never by the library.

* ``fld``: the substep (limiter, backward-Euler diffusion, exchange), its explicit
  coupling terms and the opacity laws (constant, power law, table);
* ``dispersion``: the linear RMHD modes of Appendix B;
* ``rmhd1d``: the 1D radiation-MHD wave step of the linear-wave tests;
* ``cfld`` (with ``cfld.c``): a plain C restatement of the substep (limiter, V-cycle or
  Jacobi-PCG solve, exchange) with OpenMP loops, the timed CPU baseline, pinned to ``fld``;
* ``write_linmode_eigen``: writes the fast-mode amplitudes the 3D linear-mode recipe reads.
"""
