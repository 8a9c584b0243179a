"""The checks build (-DROIBIN_CHECKS), which stands in for a device memory
checker: device bounds checks on the stores into output buffers and
offset-computed scratch record a failure instead of trapping, and guard bands
(0xA5 bytes) separate the sections of every context's scratch.  The library
reports both through roibin_ctx_debug_status, and roibin_ctx_destroy (so
Context.close) fails with ROIBIN_ERR_CHECK when either was hit.

Each test runs in a child process with ROIBIN_CHECKS=1, which makes the
package load libroibin_checks.so instead of libroibin.so."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code_or_args, timeout=1500):
    env = dict(os.environ, ROIBIN_CHECKS="1")
    args = code_or_args if isinstance(code_or_args, list) else [sys.executable, "-c", textwrap.dedent(code_or_args)]
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    return r.stdout


@pytest.fixture(scope="module", autouse=True)
def _checks_library():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    subprocess.run([sys.executable, "-c", "from paper_2206_11297_gb300 import _build; _build.build(checks=True)"],
                   cwd=ROOT, check=True, timeout=1500)


@pytest.mark.gpu
def test_checks_build_reports_clean_runs_and_an_overwritten_guard():
    out = _run("""
        import sys
        sys.path.insert(0, "tests")
        import numpy as np, torch
        import paper_2206_11297_gb300 as rb
        from synthetic import FrameRecipe, make_frame
        assert rb.library()._name.endswith("libroibin_checks.so")
        geom = (4, 37, 52)
        r = FrameRecipe(geom, peaks=("uniform", 2, 10), seed=5)
        f = torch.from_numpy(np.stack([make_frame(r, k) for k in range(3)])).cuda()
        ctx = rb.Context(geom, rb.default_params(atot_thr=300.0), max_frames=3)
        for path in (rb.PATH_PLAIN, rb.PATH_FUSED):
            ctx.set_path(path)
            out, nb, st = ctx.compress(f)
            torch.cuda.synchronize()
            assert (st.cpu() == 0).all()
        st, cb, first, failed, bad = ctx.debug_status()
        assert (st, cb, first, failed) == (rb.OK, True, 0, 0) and bad == 2**64 - 1
        ctx.debug_poke_guard(3)
        st, cb, first, failed, bad = ctx.debug_status()
        assert st == rb.ERR_CHECK and first == 0 and failed == 0 and bad < ctx.scratch_bytes
        try:
            ctx.close()
            raise SystemExit("close did not report the overwritten guard")
        except rb.RoibinError as e:
            assert e.code == rb.ERR_CHECK
        print("checks-ok")
    """)
    assert "checks-ok" in out


@pytest.mark.gpu
def test_gpu_parity_suites_pass_under_the_checks_build():
    """The parity suites on small cases, every context checked when it closes."""
    out = _run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                "tests/test_gpu_parity.py", "tests/test_roi_coder.py", "tests/test_chunks.py",
                "tests/test_graph.py", "tests/test_timeout.py", "tests/test_lorenzo_dims.py"])
    assert " passed" in out and "failed" not in out
