"""The index-checked build (librfa_check.so, compiled with -DRFA_CHECK).

Its kernels test every global and shared-memory access range against the
array it indexes; an access outside records a status bit (reported as
RFA_E_INTERNAL) and is skipped instead of touching memory.  It stands in for a
memory checker, which this environment does not provide.  The ragged,
degenerate and blocked-kernel parity cases run against it in a child process
(the library is chosen when the package loads): they must pass unchanged,
which they cannot if a check fires or if the checks changed a result."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    "tests/test_gpu_parity.py::test_ragged_phantoms_with_damage",
    "tests/test_gpu_parity.py::test_param_precisions",
    "tests/test_gpu_parity.py::test_point_source_at_tile_corner",
    "tests/test_gpu_parity.py::test_paper_fixed_tip_through_place_needle",
    "tests/test_gpu_parity.py::test_fixed_tip_moves_and_is_removed",
    "tests/test_gpu_degenerate.py",
    "tests/test_gpu_tb.py::test_blocked_equals_one_step",
    "tests/test_gpu_tb.py::test_blocked_parity_with_oracle",
    "tests/test_gpu_batch.py::test_batch_equals_members_stepped_alone",
    "tests/test_zz_no_alloc.py::test_noalloc_reduction_matches_necrosis_mask_and_oracle_on_two_calls",
    # the model-option step and the adjoint step read every neighbour at a clamped
    # address (no branch): ragged grids, both face kinds, both state precisions
    "tests/test_gpu_cond.py::test_conservative_step_matches_oracle",
    "tests/test_gpu_alpha.py::test_coupled_perfusion_matches_oracle",
    "tests/test_gpu_adjoint.py::test_adjoint_matches_oracle_small",
    "tests/test_gpu_adjoint.py::test_adjoint_recorded_in_chunks_and_blocked_forward",
    "tests/test_gpu_cond.py::test_model_step_rows_across_thread_blocks",
    "tests/test_gpu_adjoint.py::test_adjoint_rows_across_thread_blocks",
]


def test_parity_cases_pass_on_the_checked_build():
    from paper_1907_05709_b300 import build
    lib = build.build(checked=True)
    assert os.path.basename(lib) == "librfa_check.so"
    env = dict(os.environ, RFA_CHECKED_BUILD="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider", *CASES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "failed" not in r.stdout, tail
