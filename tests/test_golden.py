"""The oracle still writes the stored streams (format version 1) for the stored
frames; see tests/golden/make_golden.py, which wrote them from the oracle."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _cases():
    with open(os.path.join(HERE, "oracle_streams.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name", sorted(_cases()))
def test_oracle_reproduces_stored_stream(name):
    case = _cases()[name]
    frame = np.load(os.path.join(HERE, "oracle_inputs.npz"))[name]
    assert list(frame.shape) == case["geometry"]
    params = dict(oracle.DEFAULTS)
    params.update(case["params"])
    st, stream = oracle.compress_frame(frame, oracle.make_params(**params))
    assert st == 0 and len(stream) == case["stream_bytes"]
    assert hashlib.sha256(np.asarray(stream).tobytes()).hexdigest() == case["stream_sha256"]
    dst, rec = oracle.decompress_frame(stream, tuple(case["geometry"]))
    assert dst == 0
    assert hashlib.sha256(rec.astype(np.float32).tobytes()).hexdigest() == case["reconstruction_sha256"]


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(_cases()))
def test_gpu_writes_stored_stream(name):
    """Both compression paths write the stored bytes for the stored frames."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_11297_gb300 as rb
    case = _cases()[name]
    frame = np.load(os.path.join(HERE, "oracle_inputs.npz"))[name]
    params = rb.default_params(**case["params"])
    with rb.Context(tuple(case["geometry"]), params, max_frames=1) as ctx:
        for path in (rb.PATH_PLAIN, rb.PATH_AUTO):
            ctx.set_path(path)
            out, nb, st = ctx.compress(torch.from_numpy(frame[None]).cuda())
            torch.cuda.synchronize()
            assert int(st[0]) == 0 and int(nb[0]) == case["stream_bytes"]
            got = out[0, :int(nb[0])].cpu().numpy()
            assert hashlib.sha256(got.tobytes()).hexdigest() == case["stream_sha256"], path
