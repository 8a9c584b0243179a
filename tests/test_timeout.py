"""Failure detection on the fused path without a GPU fault: every flag wait of
the persistent kernel is bounded, and a wait that runs out reaches the caller as
ROIBIN_ERR_TIMEOUT in the frame status.  The test makes the waits run out by
setting the context's poll limit to 0 (roibin_ctx_set_wait_limit), so no wait
polls at all: nothing spins, nothing faults, the launch ends as usual.  The
next call at the default limit must write the oracle's bytes again."""
import numpy as np
import pytest

import paper_2206_11297_gb300 as rb
from synthetic import FrameRecipe, make_frame

from gpu_util import oparams
import oracle


def _frames(geom, n, seed):
    r = FrameRecipe(geom, peaks=("uniform", 2, 12), seed=seed)
    return np.stack([make_frame(r, k) for k in range(n)])


def test_wait_limit_argument_checks():
    lib = rb.library()
    assert lib.roibin_ctx_set_wait_limit(None, 0) == rb.ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("dense", [False, True])
def test_flag_wait_timeout_reaches_the_caller(dense):
    import torch
    geom = (6, 40, 64)
    frames = _frames(geom, 5, seed=21)
    params = rb.default_params(atot_thr=300.0)
    op = oparams(params)
    with rb.Context(geom, params, max_frames=len(frames)) as ctx:
        ctx.set_path(rb.PATH_FUSED)
        ctx.set_fused_dense_peaks(dense)
        d = torch.from_numpy(frames).cuda()
        ctx.set_wait_limit(0)
        out, nb, st = ctx.compress(d)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == rb.ERR_TIMEOUT).all(), st.cpu().numpy()
        assert (nb.cpu().numpy() == 0).all()
        # the default limit again: the context is usable and writes the oracle's bytes
        ctx.set_wait_limit(-1)
        out, nb, st = ctx.compress(d)
        torch.cuda.synchronize()
        out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
    for k in range(len(frames)):
        ost, ref = oracle.compress_frame(frames[k], op)
        assert ost == oracle.OK and st[k] == rb.OK
        assert nb[k] == len(ref) and np.array_equal(out[k, :nb[k]], ref), f"frame {k}"


@pytest.mark.gpu
def test_wait_limit_leaves_the_plain_path_alone():
    """The plain path has no flag waits: the hook does not touch it."""
    import torch
    geom = (3, 30, 44)
    frames = _frames(geom, 3, seed=22)
    params = rb.default_params(atot_thr=300.0)
    op = oparams(params)
    with rb.Context(geom, params, max_frames=len(frames)) as ctx:
        ctx.set_path(rb.PATH_PLAIN)
        ctx.set_wait_limit(0)
        out, nb, st = ctx.compress(torch.from_numpy(frames).cuda())
        torch.cuda.synchronize()
        out, nb, st = out.cpu().numpy(), nb.cpu().numpy(), st.cpu().numpy()
    for k in range(len(frames)):
        ost, ref = oracle.compress_frame(frames[k], op)
        assert st[k] == rb.OK and np.array_equal(out[k, :nb[k]], ref)
