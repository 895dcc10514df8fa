"""The bounds-checked build (the library compiled with FLD_DEBUG): every computed index of
the stencil, gradient, residual, sweep and transfer kernels is checked, and an index
outside its array raises a flag instead of being dereferenced. Here the debug library is
built and a set of the parity tests runs against it in a child process; the autouse
fixture of conftest.py requires that no test leaves a flag raised, and the tests' own
comparisons with the oracle still hold."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# z-marching sweeps and transfers (3D, tuned and untuned shapes), the FP64, mixed and
# recursive residuals, 1D/2D levels, truncated V-cycles, the limiter's gradient with every
# wall kind, the whole step
TESTS = [
    "tests/test_gpu_step.py",
    "tests/test_gpu_limiter.py",
    "tests/test_gpu_diffuse.py::test_fused_sweep_matches_half_sweeps_and_oracle",
    "tests/test_gpu_tuned.py::test_inner_cycles_zmarch_graph_box",
    "tests/test_gpu_face_mean.py::test_diffuse_harmonic_matches_oracle",
    # the recursive refinement residual and the truncated V-cycle's coarse sweeps
    "tests/test_gpu_resid_update.py::test_recursive_residual_bounds_the_true_residual",
    "tests/test_gpu_truncate.py::test_truncated_vcycle_solves_the_same_system",
]


@pytest.mark.gpu
def test_debug_build_raises_no_flag_on_the_parity_tests():
    from paper_2503_02764_gb300 import build, fld
    lib = build.build(debug=True)
    env = dict(os.environ, FLD_LIBRARY=lib)
    p = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                        "-p", "no:cacheprovider", *TESTS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = "\n".join((p.stdout + p.stderr).splitlines()[-15:])
    assert p.returncode == 0, tail
    assert " passed" in tail, tail
    # the normal build carries no checks
    assert fld.fld_debug_flags() == -1
