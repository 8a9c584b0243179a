"""Writes tests/golden/oracle_inputs.npz (a few small seeded frames) and
tests/golden/oracle_streams.json: for each frame, the oracle's stream (length
and SHA-256) and reconstruction (SHA-256).  The frames are stored so that the
check depends on the oracle alone, not on the generator's floating point.

These are not the paper's numbers (it prints no worked example).  They pin
format version 1 as the oracle writes it today, so that an unintended change
to the stream layout or to any arithmetic step shows up as a failing test.
Only oracle/ and the seeded generators are called.  Run from the repository
root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), "..", ".."))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synthetic import FrameRecipe, make_frame  # noqa: E402

# (name, geometry, recipe keywords, parameter overrides)
CASES = [
    ("cspad_like_small", (2, 37, 52), {"peaks": ("uniform", 3, 8), "seed": 101}, {"atot_thr": 300.0}),
    ("odd_panels_bin3", (3, 23, 31), {"peaks": ("fixed", 4), "seed": 102}, {"bin_h": 3, "bin_w": 3}),
    ("hot_pixels_eb1", (2, 40, 48), {"bg_mean": 30.0, "bg_sd": 8.0, "hot_fraction": 0.01,
                                     "peaks": ("fixed", 3), "seed": 103}, {"abs_eb": 1.0, "max_peaks": 512}),
    ("small_radius", (1, 64, 64), {"peaks": ("fixed", 6), "seed": 104}, {"quant_radius": 16, "abs_eb": 2.0}),
    ("lorenzo_run_1d", (3, 25, 29), {"peaks": ("fixed", 3), "seed": 105}, {"lorenzo_dims": 1, "abs_eb": 4.0}),
    ("lorenzo_stack_3d", (4, 30, 36), {"peaks": ("uniform", 2, 6), "seed": 106},
     {"lorenzo_dims": 3, "atot_thr": 300.0}),
    # the lossless ROI coder: windows of hot-pixel pairs, and of Bragg spots
    ("roi_coded_hot", (2, 40, 48), {"bg_mean": 30.0, "bg_sd": 8.0, "hot_fraction": 0.01,
                                    "peaks": ("fixed", 3), "seed": 107}, {"roi_coder": 1, "max_peaks": 512}),
    ("roi_coded_spots", (3, 37, 52), {"peaks": ("uniform", 4, 8), "seed": 108},
     {"roi_coder": 1, "atot_thr": 300.0, "npix_max": 49}),
]


def frames():
    return {name: make_frame(FrameRecipe(geom, **rkw), 0) for name, geom, rkw, _ in CASES}


def compute(inputs):
    out = {}
    for name, geom, rkw, pkw in CASES:
        frame = inputs[name]
        params = dict(oracle.DEFAULTS)
        params.update(pkw)
        st, stream = oracle.compress_frame(frame, oracle.make_params(**params))
        assert st == 0, (name, st)
        dst, rec = oracle.decompress_frame(stream, geom)
        assert dst == 0, (name, dst)
        out[name] = {"geometry": list(geom), "recipe": {k: list(v) if isinstance(v, tuple) else v
                                                        for k, v in rkw.items()},
                     "params": pkw, "stream_bytes": len(stream),
                     "stream_sha256": hashlib.sha256(np.asarray(stream).tobytes()).hexdigest(),
                     "reconstruction_sha256": hashlib.sha256(rec.astype(np.float32).tobytes()).hexdigest()}
    return out


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    inputs = frames()
    np.savez_compressed(os.path.join(here, "oracle_inputs.npz"), **inputs)
    with open(os.path.join(here, "oracle_streams.json"), "w") as f:
        json.dump(compute(inputs), f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", here)
