"""The bounds-checked build (GABP_DEBUG): kernels test the indices they compute
or read and report a failed test through the status word (no trap, no access
outside an array).  This runs a subset of the GPU parity tests (single sweeps
and trajectories against the oracle on the stencil, CSR and parity-class
layouts, line GaBP sweeps and solves, fused and separate multigrid cycles,
batched solves) in a child process on the checked library: every one must
pass with no index check failing, i.e. the release kernels' indices are in
range on those cases."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_subset_on_bounds_checked_build():
    sys.path.insert(0, ROOT)
    from paper_1904_04093_gb300 import build
    lib = build.build(debug=True)
    assert os.path.exists(lib)
    env = dict(os.environ, GABP_DEBUG="1")
    probe = subprocess.run(
        [sys.executable, "-c",
         "import paper_1904_04093_gb300 as g; L = g.load(); print(g.library_path(), L.gabp_debug_build())"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr
    assert probe.stdout.strip().endswith(" 1") and "libgabp_debug.so" in probe.stdout
    sel = ("single_sweep or trajectory or first_update or vcycle or fused or batch_equals "
           "or colored or residual_2norm or line_sweeps or line_solve_matches or line_frozen_precision "
           "or line_tiny or natural_columns or line_transposed")
    run = subprocess.run(
        [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-k", sel,
         "tests/test_gpu_parity.py", "tests/test_gpu_csr.py", "tests/test_gpu_mg_fused.py",
         "tests/test_gpu_batch.py", "tests/test_gpu_lines.py"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (run.stdout + run.stderr)[-3000:]
    assert run.returncode == 0, tail
    assert " passed" in run.stdout, tail
