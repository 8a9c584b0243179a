"""Pins for the CPU oracle: checks against what the paper and the mathematics fix.

Each pin is a function that raises AssertionError when the oracle is wrong.
None of them recomputes the oracle's formula the oracle's way: they use brute
force written differently, closed forms, special cases whose answer is fixed by
construction, invariants (exact inverses, Kraft equality, optimal Huffman cost),
and an independent decoder.  tests/test_oracle_pins.py runs them on the oracle;
tests/test_oracle_mutants.py runs them on copies of the oracle with planted
mistakes and requires each mistake to be caught.
"""
from __future__ import annotations

import heapq
import math
from fractions import Fraction

import numpy as np

import oracle as O


# ------------------------------------------------------------------ helpers
def brute_candidates(panel: np.ndarray, rank: int, amax: float):
    """Local maxima by slicing the clipped window and comparing against the
    flattened pixels before / after the centre (row-major tie rule)."""
    H, W = panel.shape
    out = []
    for r in range(H):
        for c in range(W):
            v = panel[r, c]
            if not v >= amax:
                continue
            r0, r1 = max(r - rank, 0), min(r + rank + 1, H)
            c0, c1 = max(c - rank, 0), min(c + rank + 1, W)
            flat = panel[r0:r1, c0:c1].ravel()
            k = (r - r0) * (c1 - c0) + (c - c0)
            if np.all(v > flat[:k]) and np.all(v >= flat[k + 1:]):
                out.append((r, c))
    return out


def brute_accept(panel: np.ndarray, r: int, c: int, p) -> bool:
    """Candidate evaluation with exact rational arithmetic for the background."""
    H, W = panel.shape
    ii, jj = np.mgrid[0:H, 0:W]
    d2 = (ii - r) ** 2 + (jj - c) ** 2
    ring = (d2 >= p.ring_r0 ** 2) & (d2 < (p.ring_r0 + p.ring_dr) ** 2)
    vals = [Fraction(float(x)) for x in panel[ring]]
    if vals:
        bkg = sum(vals) / len(vals)
        var = sum((v - bkg) ** 2 for v in vals) / len(vals)
    else:
        bkg, var = Fraction(0), Fraction(0)
    sigma = math.sqrt(float(var))
    win = (np.abs(ii - r) <= p.rank) & (np.abs(jj - c) <= p.rank)
    dev = [Fraction(float(x)) - bkg for x in panel[win]]
    thr = p.pix_nsigma * sigma
    sel = [d for d in dev if float(d) > thr]
    npix = len(sel)
    atot = float(sum(sel)) if sel else 0.0
    return (p.npix_min <= npix <= p.npix_max and atot > p.atot_thr
            and atot > p.son_min * sigma * math.sqrt(npix))


def heap_huffman_cost(freqs) -> int:
    """Total bits of an optimal prefix code: the sum of all merged weights."""
    f = [int(x) for x in freqs if x > 0]
    if len(f) == 1:
        return f[0]
    heapq.heapify(f)
    cost = 0
    while len(f) > 1:
        a, b = heapq.heappop(f), heapq.heappop(f)
        cost += a + b
        heapq.heappush(f, a + b)
    return cost


def decode_stream(stream: np.ndarray, lengths=None):
    """Independent decoder: walks the container with the header counts, builds a
    {(length, codeword): symbol} map from the canonical rule and reads each chunk
    bit by bit.  Returns dict with codes, lorenzo, prequant, peaks, roi.
    `lengths`: the code lengths of a stream that keeps none (its chunk head's)."""
    h = O.parse_header(stream)
    o = O.section_offsets(h)
    nsym = 2 * h["quant_radius"]
    if lengths is None:
        lengths = stream[o["lengths"]:o["lengths"] + nsym].astype(int)
    order = sorted((l, s) for s, l in enumerate(lengths) if l > 0)
    table, code, prev = {}, 0, None
    for l, s in order:
        if prev is not None:
            code = (code + 1) << (l - prev)
        table[(l, code)] = s
        prev = l
    words = stream[o["bitstream"]:o["bitstream"] + 4 * h["n_words"]].view("<u4")
    cidx = stream[o["chunk_index"]:o["chunk_index"] + 4 * h["n_chunks"]].view("<u4")
    m = h["n_symbols"]
    codes = np.zeros(m, np.uint16)
    for k in range(h["n_chunks"]):
        pos = int(cidx[k]) * 32
        for i in range(k * O.CHUNK_SYMBOLS, min(m, (k + 1) * O.CHUNK_SYMBOLS)):
            l, cw = 0, 0
            while True:
                w = int(words[pos // 32])
                cw = (cw << 1) | ((w >> (31 - pos % 32)) & 1)
                pos += 1
                l += 1
                if (l, cw) in table:
                    codes[i] = table[(l, cw)]
                    break
                assert l <= 32, "undecodable bit pattern"
    lo = stream[o["lorenzo"]:o["lorenzo"] + 8 * h["n_lorenzo"]].view("<u4").reshape(-1, 2)
    pq = stream[o["prequant"]:o["prequant"] + 8 * h["n_prequant"]].view("<u4").reshape(-1, 2)
    peaks = stream[o["peaks"]:o["peaks"] + 6 * h["n_peaks"]].view("<u2").reshape(-1, 3)
    n_roi = h["n_peaks"] * h["roi_h"] * h["roi_w"]
    if h["roi_coding"] == 0:
        roi = stream[o["roi"]:o["roi"] + 4 * n_roi].view("<f4").reshape(-1, h["roi_h"], h["roi_w"])
    elif h["roi_coding"] == 2:
        roi = stream[o["roi_section"]:o["roi_section"] + 4 * n_roi].view("<f4").reshape(-1, h["roi_h"], h["roi_w"])
    else:
        roi = decode_roi_section(stream[o["roi_section"]:o["end"]], h["n_peaks"], h["roi_h"], h["roi_w"],
                                 h["roi_words"])[1]
    return dict(header=h, codes=codes, lengths=lengths, lorenzo=lo, prequant=pq, peaks=peaks, roi=roi)


def tiny_frame(seed=0, shape=(2, 12, 13)):
    rng = np.random.default_rng(seed)
    f = rng.normal(20, 5, shape).clip(0)
    # planted: an isolated peak, a plateau pair, an edge peak, a corner peak and a hot pixel
    f[0, 5, 6] = 900
    f[0, 4:7, 5:8] += np.array([[60, 120, 60], [120, 0, 120], [60, 120, 60]])
    f[1, 3, 3] = f[1, 3, 4] = 700
    f[1, 2:5, 2:6] += 80
    f[1, 3, 3] = f[1, 3, 4] = 700
    f[0, 0, 12] = 650
    f[0, 1, 12] = 260
    f[1, 11, 0] = 800
    f[1, 10, 0] = 400
    f[1, 11, 1] = 380
    f[1, 9, 10] = 5000
    return f.astype(np.float32)


# ------------------------------------------------------------------ peak pins
def pin_candidates_brute_force():
    for seed in range(6):
        f = tiny_frame(seed)
        if seed >= 3:
            # heavier: many candidates, ties from clipping
            f = np.round(f / 40) * 40
            f[f >= 40] += 300
        for pn in range(f.shape[0]):
            for rank in (1, 2, 3):
                got = [(r, c) for r in range(f.shape[1]) for c in range(f.shape[2])
                       if O.is_peak_candidate(f[pn], r, c, rank, 300.0)]
                assert got == brute_candidates(f[pn], rank, 300.0), (seed, pn, rank)


def pin_candidate_special_cases():
    flat = np.full((15, 15), 20.0, np.float32)
    a = flat.copy()
    a[7, 7] = 300.0
    assert O.is_peak_candidate(a, 7, 7, 3, 300.0), "a maximum equal to amax is kept"
    a[7, 7] = np.nextafter(np.float32(300.0), np.float32(0))
    assert not O.is_peak_candidate(a, 7, 7, 3, 300.0), "a maximum below amax is rejected"
    b = flat.copy()
    b[7, 7] = b[7, 9] = 500.0
    assert O.is_peak_candidate(b, 7, 7, 3, 300.0) and not O.is_peak_candidate(b, 7, 9, 3, 300.0), \
        "plateau: only the first pixel in row-major order"
    b2 = flat.copy()
    b2[7, 7] = b2[9, 5] = 500.0
    assert O.is_peak_candidate(b2, 7, 7, 3, 300.0) and not O.is_peak_candidate(b2, 9, 5, 3, 300.0)
    c = flat.copy()
    c[7, 7], c[7, 10] = 500.0, 600.0
    assert not O.is_peak_candidate(c, 7, 7, 3, 300.0), "a larger pixel 3 px away suppresses"
    c[7, 11] = c[7, 10]
    c[7, 10] = 20.0
    assert O.is_peak_candidate(c, 7, 7, 3, 300.0), "4 px away is outside the 7x7 window"
    d = flat.copy()
    d[0, 0] = 400.0
    d[14, 14] = 400.0
    assert O.is_peak_candidate(d, 0, 0, 3, 300.0) and O.is_peak_candidate(d, 14, 14, 3, 300.0)
    e = flat.copy()
    e[7, 7] = 500.0
    e[6, 8] = np.nan
    assert not O.is_peak_candidate(e, 7, 7, 3, 300.0), "NaN in the window fails the test"


def pin_evaluation_special_cases():
    p = O.make_params(pix_nsigma=3.0)
    base = np.full((25, 25), 20.0, np.float32)  # flat ring: sigma = 0, threshold 0 above bkg

    def accept(fr):
        return O.evaluate_peak(fr, 12, 12, p)

    a = base.copy()
    a[12, 12] = 5000.0
    assert not accept(a), "hot single pixel: npix = 1 < 2"
    a[12, 13] = 500.0
    assert accept(a), "two pixels, atot well above 600"
    b = base.copy()
    b[12, 12], b[12, 13] = 330.0, 310.0   # atot = 310 + 290 = 600: not > 600
    assert not accept(b)
    b[12, 13] = 311.0                     # atot = 601
    assert accept(b)
    c = base.copy()
    c[12, 12] = 500.0
    cells = [(i, j) for i in range(9, 16) for j in range(9, 16) if (i, j) != (12, 12)]
    for i, j in cells[:29]:
        c[i, j] = 400.0
    assert accept(c), "npix = 30 is allowed"
    c[cells[29]] = 400.0
    assert not accept(c), "npix = 31 is rejected"
    # a noisy ring: +-s around 20 makes sigma = s exactly (equal counts, see below)
    d = base.copy()
    ii, jj = np.mgrid[0:25, 0:25]
    d2 = (ii - 12) ** 2 + (jj - 12) ** 2
    ring = (d2 >= 25) & (d2 < 49)
    idx = np.argwhere(ring)
    assert len(idx) % 2 == 0
    for k, (i, j) in enumerate(idx):
        d[i, j] = 20.0 + (8.0 if k % 2 == 0 else -8.0)  # mean 20, sigma 8, thr 24
    d[12, 12], d[12, 13] = 300.0 + 20.0, 60.0 + 20.0  # devs 300 (>24) and 60 (>24); atot = 360
    assert not accept(d), "atot 360 < 600"
    d[12, 12] = 900.0 + 20.0                         # atot = 960; SNR = 960 / (8 sqrt 2) = 84.9
    assert accept(d)
    d[12, 13] = 20.0 + 20.0                          # dev 20 < 24: not a peak pixel -> npix 1
    assert not accept(d)
    # SNR boundary: sigma 8, npix 2, need atot > 10 * 8 * sqrt(2) = 113.1 (and > 600 -> relax)
    p2 = O.make_params(pix_nsigma=3.0, atot_thr=0.0)
    d[12, 12], d[12, 13] = 20.0 + 80.0, 20.0 + 30.0  # atot 110 < 113.1
    assert not O.evaluate_peak(d, 12, 12, p2)
    d[12, 12] = 20.0 + 85.0                          # atot 115 > 113.1
    assert O.evaluate_peak(d, 12, 12, p2)


def pin_evaluation_brute_force():
    rng = np.random.default_rng(7)
    p = O.make_params(pix_nsigma=2.0, atot_thr=600.0, son_min=10.0, npix_max=9)
    n_acc = n_rej = 0
    for t in range(60):
        fr = rng.normal(20, 5, (20, 21)).astype(np.float32)
        r, c = int(rng.integers(0, 20)), int(rng.integers(0, 21))
        fr[max(r - 1, 0):r + 2, max(c - 1, 0):c + 2] += rng.uniform(0, 120)
        fr[r, c] += rng.uniform(100, 400)
        got = O.evaluate_peak(fr, r, c, p)
        assert got == brute_accept(fr, r, c, p), (t, r, c)
        n_acc += got
        n_rej += not got
    assert n_acc > 5 and n_rej > 5


def pin_find_peaks_frame():
    p = O.make_params(atot_thr=300.0)
    for seed in range(3):
        f = tiny_frame(seed)
        st, peaks, n = O.find_peaks(f, p)
        assert st == O.OK
        expect = []
        for pn in range(f.shape[0]):
            for r, c in brute_candidates(f[pn], p.rank, p.amax_thr):
                if brute_accept(f[pn], r, c, p):
                    expect.append((pn, r, c))
        assert [tuple(x) for x in peaks.tolist()] == expect, seed
    # capacity: more peaks than max_peaks is an error, never a silent cut
    f = tiny_frame(0)
    st, _, n = O.find_peaks(f, O.make_params(atot_thr=300.0, max_peaks=1))
    assert n >= 2 and st == O.ERR_CAPACITY


# ------------------------------------------------------------------ ROI pins
def pin_roi():
    f = np.arange(2 * 30 * 31, dtype=np.float32).reshape(2, 30, 31)
    p = O.make_params()
    peaks = np.array([[1, 15, 15], [0, 0, 0], [1, 29, 30], [0, 3, 20]], np.uint16)
    roi = O.roi_extract(f, p, peaks)
    assert np.array_equal(roi[0], f[1, 7:24, 7:24]), "centred 17x17 window"
    assert np.all(roi[1][:8, :] == 0) and np.all(roi[1][:, :8] == 0), "fill past the edge is 0"
    assert np.array_equal(roi[1][8:, 8:], f[0, 0:9, 0:9])
    assert np.array_equal(roi[2][:9, :9], f[1, 21:30, 22:31]) and np.all(roi[2][9:, :] == 0)
    assert np.array_equal(roi[3][5:, :], f[0, 0:12, 12:29])
    m = O.roi_mask(f.shape, p, peaks)
    assert m[1, 7:24, 7:24].all() and m[1].sum() == 17 * 17 + 9 * 9 - 3 * 2  # 6 shared pixels
    assert m[0].sum() == len(np.unique(np.concatenate([
        np.ravel_multi_index(np.mgrid[0:9, 0:9].reshape(2, -1), (30, 31)),
        np.ravel_multi_index(np.mgrid[0:12, 12:29].reshape(2, -1), (30, 31))])))


# ------------------------------------------------------------------ binning pins
def pin_binning():
    rng = np.random.default_rng(1)
    # equal values -> that value
    f = np.full((2, 6, 8), 3.7, np.float32)
    assert np.all(O.bin_frame(f, 2, 2) == np.float32(3.7))
    # 1x1 is the identity, bit for bit
    g = rng.normal(0, 100, (3, 7, 9)).astype(np.float32)
    assert np.array_equal(O.bin_frame(g, 1, 1).view(np.uint32), g.view(np.uint32))
    # integers (exact sums): mean = exact sum / count rounded once; edge bins use in-panel count
    for bh, bw in ((2, 2), (3, 3), (2, 3), (4, 1)):
        h = rng.integers(-1000, 1000, (2, 7, 11)).astype(np.float32)
        got = O.bin_frame(h, bh, bw)
        P, Hb, Wb = got.shape
        for pn in range(P):
            for i in range(Hb):
                for j in range(Wb):
                    blk = h[pn, i * bh:(i + 1) * bh, j * bw:(j + 1) * bw].astype(np.float64)
                    exp = np.float32(blk.sum()) / np.float32(blk.size)
                    assert got[pn, i, j] == exp, (bh, bw, pn, i, j)
    # summation order: row-major, sequential in float32
    o = np.array([[[1e8, 1.0], [-1e8, 1.0]]], np.float32)
    assert O.bin_frame(o, 2, 2)[0, 0, 0] == np.float32(0.25)


# ------------------------------------------------------------------ quantisation pins
def pin_prequantize():
    # eb = 0.5: 2 eb = 1 and 1/(2 eb) = 1 exactly, so q = rint(b)
    b = np.array([2.5, 3.5, -2.5, 0.5, -0.5, 1.49, 7.0, 2 ** 28, 2 ** 28 - 16], np.float32)
    q, pq = O.prequantize(b, 0.5)
    assert q[:7].tolist() == [2, 4, -2, 0, 0, 1, 7], "round half to even"
    assert pq[:7].sum() == 0, "|b - q| = 0.5 = eb is within the bound"
    assert pq[7] == 1 and q[7] == 0, "|q| >= 2^28 is an outlier"
    assert pq[8] == 0 and q[8] == 2 ** 28 - 16
    nf = np.array([np.nan, np.inf, -np.inf, 3e38], np.float32)
    q, pq = O.prequantize(nf, 10.0)
    assert pq.tolist() == [1, 1, 1, 1] and q.tolist() == [0, 0, 0, 0]
    # the bound holds on every non-outlier, for many error bounds
    rng = np.random.default_rng(3)
    for eb in (1e-3, 0.3, 1.0, 10.0, 90.0, 1234.5):
        x = (rng.standard_cauchy(20000) * 50).astype(np.float32)
        q, pq = O.prequantize(x, eb)
        xh = q.astype(np.float32) * np.float32(2 * np.float32(eb))
        ok = pq == 0
        assert np.all(np.abs(x[ok].astype(np.float64) - xh[ok].astype(np.float64)) <= np.float32(eb))
        assert np.all(q[~ok] == 0)
        assert ok.mean() > 0.9


def pin_lorenzo():
    rng = np.random.default_rng(4)
    q = rng.integers(-2 ** 27, 2 ** 27, (3, 9, 11)).astype(np.int32)
    d = O.lorenzo(q)
    rebuilt = np.cumsum(np.cumsum(d.astype(np.int64), axis=1), axis=2)
    assert np.array_equal(rebuilt, q), "2-D prefix sum inverts the predictor"
    ramp = (5 * np.arange(6)[:, None] - 3 * np.arange(7)[None, :] + 11).astype(np.int32)[None]
    d = O.lorenzo(ramp)
    assert d[0, 0, 0] == 11 and np.all(d[0, 0, 1:] == -3) and np.all(d[0, 1:, 0] == 5)
    assert np.all(d[0, 1:, 1:] == 0), "a plane is predicted exactly"
    const = np.full((2, 4, 5), 9, np.int32)
    d = O.lorenzo(const)
    assert np.all(d[:, 0, 0] == 9) and np.count_nonzero(d) == 2, "per-panel, no cross-panel neighbour"


def pin_lorenzo_dims():
    """Dimension 1, 2 and 3 (the row of pixels, the panel, the panel stack):
    each is the zero-padded backward difference along its axes, a separable
    form the oracle does not use, and a prefix sum along the same axes
    inverts it."""
    rng = np.random.default_rng(14)
    q = rng.integers(-2 ** 27, 2 ** 27, (4, 7, 9)).astype(np.int32)
    q64 = q.astype(np.int64)
    d1 = O.lorenzo(q, dims=1)
    assert np.array_equal(d1.ravel(), np.diff(q64.ravel(), prepend=0)), "1-D: one run over the frame"
    d3 = O.lorenzo(q, dims=3)
    want = q64
    for ax in range(3):
        want = np.diff(want, axis=ax, prepend=0)
    assert np.array_equal(d3, want), "3-D: backward differences along panel, row and column"
    assert np.array_equal(O.lorenzo(q[:1], dims=3), O.lorenzo(q[:1], dims=2)), "one panel: 3-D is 2-D"
    rebuilt = d3.astype(np.int64)
    for ax in range(3):
        rebuilt = np.cumsum(rebuilt, axis=ax)
    assert np.array_equal(rebuilt, q64)
    # the 3-D predictor is exact on any sum of terms that each skip one axis
    P, H, W = 5, 6, 8
    g = rng.integers(-1000, 1000, (1, H, W))
    h = rng.integers(-1000, 1000, (P, 1, W))
    k = rng.integers(-1000, 1000, (P, H, 1))
    field = (g + h + k).astype(np.int32)
    d = O.lorenzo(field, dims=3)
    assert np.all(d[1:, 1:, 1:] == 0) and np.any(d[0] != 0)
    const = np.full((2, 3, 4), 7, np.int32)
    assert np.count_nonzero(O.lorenzo(const, dims=1)) == 1, "1-D: a constant frame is one delta"
    assert np.count_nonzero(O.lorenzo(const, dims=3)) == 1, "3-D: a constant stack is one delta"


def pin_lorenzo_dims_roundtrip():
    """Streams in dimension 1 and 3 decode within eb, name their dimension in
    the header, and carry the codes of that predictor."""
    f = tiny_frame(6, shape=(3, 21, 27))
    streams = {}
    for dims in (1, 2, 3):
        p = O.make_params(atot_thr=300.0, lorenzo_dims=dims)
        s, dec, rec = _roundtrip(f, p)
        streams[dims] = s
        assert dec["header"]["lorenzo_dims"] == dims
        assert int(s[72:76].view(np.uint32)[0]) == (0 if dims == 2 else dims)
        b = O.bin_frame(f, 2, 2)
        up = np.repeat(np.repeat(b, 2, axis=1), 2, axis=2)[:, :f.shape[1], :f.shape[2]]
        mask = O.roi_mask(f.shape, p, dec["peaks"])
        err = np.abs(rec.astype(np.float64) - up.astype(np.float64))
        assert np.all(err[mask == 0] <= p.abs_eb), dims
        assert np.array_equal(rec[mask == 1], f[mask == 1])
        q, pq = O.prequantize(b, p.abs_eb)
        dq = q.astype(np.int64)
        axes = {1: None, 2: (1, 2), 3: (0, 1, 2)}[dims]
        if axes is None:
            d = np.diff(dq.ravel(), prepend=0)
        else:
            d = dq
            for ax in axes:
                d = np.diff(d, axis=ax, prepend=0)
        d = d.astype(np.int32).ravel()
        codes = np.where(np.abs(d) < p.quant_radius, d + p.quant_radius, 0)
        assert np.array_equal(dec["codes"], codes), dims
        lo_idx = np.flatnonzero(codes == 0)
        assert np.array_equal(dec["lorenzo"][:, 1].view(np.int32), d[lo_idx])
    assert len({bytes(v) for v in streams.values()}) == 3
    for code in (2, 4):
        bad = streams[3].copy()
        bad[72:76] = np.array([code], np.uint32).view(np.uint8)
        assert O.decompress_frame(bad, f.shape)[0] == O.ERR_CORRUPT_STREAM, code
    st, _ = O.compress_frame(f, O.make_params(lorenzo_dims=4))
    assert st == O.ERR_INVALID_ARG


def pin_codes_histogram():
    R = 512
    d = np.array([0, 1, -1, R - 1, -(R - 1), R, -R, 10 ** 6, -(10 ** 6)], np.int32)
    c = O.quant_codes(d, R)
    assert c.tolist() == [R, R + 1, R - 1, 2 * R - 1, 1, 0, 0, 0, 0]
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 2 * R, 10000).astype(np.uint16)
    h = O.histogram(codes, 2 * R)
    assert h.sum() == codes.size and np.array_equal(h, np.bincount(codes, minlength=2 * R))


# ------------------------------------------------------------------ Huffman pins
def pin_huffman_small():
    # two symbols -> 1 bit each; one symbol -> 1 bit
    st, L = O.huffman_lengths([0, 5, 0, 9])
    assert st == O.OK and L.tolist() == [0, 1, 0, 1]
    st, L = O.huffman_lengths([0, 0, 7, 0])
    assert L.tolist() == [0, 0, 1, 0]
    # (1, 1, 2, 2): merge a+b -> 2; the two leaves of weight 2 go before the
    # internal node of weight 2 (leaf first on ties) -> all lengths 2.
    st, L = O.huffman_lengths([1, 1, 2, 2])
    assert L.tolist() == [2, 2, 2, 2]
    # (1, 1, 1, 3): a+b -> 2; c(1)+n(2) -> 3; d(3) leaf before n(3) -> d,c,a,b = 1,2,3,3
    st, L = O.huffman_lengths([1, 1, 1, 3])
    assert L.tolist() == [3, 3, 2, 1]
    # equal counts: ties broken by symbol, deeper codes on the smaller symbols
    st, L = O.huffman_lengths([4, 4, 4])
    assert L.tolist() == [2, 2, 1]
    # Fibonacci counts give the longest possible code: n - 1 bits
    fib = [1, 1]
    while len(fib) < 20:
        fib.append(fib[-1] + fib[-2])
    st, L = O.huffman_lengths(fib)
    assert max(L) == len(fib) - 1
    # canonical codes for lengths (2, 1, 3, 3): B=0, A=10, C=110, D=111
    cw = O.canonical_codes([2, 1, 3, 3])
    assert cw.tolist() == [0b10, 0b0, 0b110, 0b111]


def pin_huffman_optimal():
    rng = np.random.default_rng(6)
    for t in range(40):
        n = int(rng.integers(2, 300))
        h = np.zeros(1024, np.uint64)
        syms = rng.choice(1024, n, replace=False)
        h[syms] = rng.integers(1, [10, 1000, 10 ** 6][t % 3], n)
        st, L = O.huffman_lengths(h)
        assert st == O.OK
        used = L[h > 0].astype(np.int64)
        assert np.all(L[h == 0] == 0) and np.all(used >= 1)
        assert sum(Fraction(1, 2 ** int(l)) for l in used) == 1, "Kraft equality"
        assert int((h[h > 0].astype(object) * used.astype(object)).sum()) == heap_huffman_cost(h)
        cw = O.canonical_codes(L)
        words = sorted((int(L[s]), int(cw[s])) for s in np.flatnonzero(h))
        strs = [format(c, f"0{l}b") for l, c in words]
        assert all(int(c) < 2 ** l for l, c in words)
        for a, b in zip(strs, strs[1:]):
            assert not b.startswith(a), "prefix-free"
        # canonical order: sorted by (length, symbol) gives increasing codes
        order = sorted(np.flatnonzero(h), key=lambda s: (L[s], s))
        vals = [int(cw[s]) << (32 - int(L[s])) for s in order]
        assert vals == sorted(vals) and len(set(vals)) == len(vals)


# ------------------------------------------------------------------ stream pins
def pin_pack_decode():
    rng = np.random.default_rng(8)
    codes = np.clip(np.round(rng.normal(512, 3, 3 * 4096 + 777)), 0, 1023).astype(np.uint16)
    codes[::97] = 0
    h = O.histogram(codes, 1024)
    st, L = O.huffman_lengths(h)
    cw = O.canonical_codes(L)
    idx, words = O.pack_chunks(codes, L, cw)
    bits = [int(L[c]) for c in codes]
    starts = [0]
    for k in range(len(idx) - 1):
        nb = sum(bits[k * 4096:(k + 1) * 4096])
        starts.append(starts[-1] + (nb + 31) // 32)
    assert idx.tolist() == starts, "each chunk starts on a word boundary"
    # independent bit reader
    inv = {(int(L[s]), int(cw[s])): s for s in np.flatnonzero(h)}
    out = []
    for k in range(len(idx)):
        pos = int(idx[k]) * 32
        for _ in range(min(4096, len(codes) - k * 4096)):
            l = c = 0
            while (l, c) not in inv:
                c = (c << 1) | ((int(words[pos // 32]) >> (31 - pos % 32)) & 1)
                pos += 1
                l += 1
            out.append(inv[(l, c)])
    assert out == codes.tolist(), "the packed stream decodes back to the codes"


def _roundtrip(frame, params, user_peaks=None):
    st, s = O.compress_frame(frame, params, user_peaks=user_peaks)
    assert st == O.OK, st
    dec = decode_stream(s)
    st2, rec = O.decompress_frame(s, frame.shape)
    assert st2 == O.OK, st2
    return s, dec, rec


def pin_frame_roundtrip():
    p = O.make_params(atot_thr=300.0)
    f = tiny_frame(2, shape=(3, 21, 27))
    f[2, 5, 5] = np.array([0xFFC01234], np.uint32).view(np.float32)[0]  # a NaN with a payload
    f[2, 15, 20] = np.inf
    f[1, 10:12, 10:12] = 1.0e7
    s, dec, rec = _roundtrip(f, p)
    h = dec["header"]
    assert h["magic"] == 0x5A534252 and h["version"] == 1
    assert len(s) == h["total_bytes"] and len(s) % 16 == 0
    # ROI pixels exact, and they are exactly the windows of the stored peaks
    mask = O.roi_mask(f.shape, p, dec["peaks"])
    assert np.array_equal(rec[mask == 1].view(np.uint32), f[mask == 1].view(np.uint32))
    # every bin within eb (prequant outliers exact), non-ROI pixels carry their bin's value
    b = O.bin_frame(f, p.bin_h, p.bin_w)
    P, Hb, Wb = b.shape
    up = np.repeat(np.repeat(b, 2, axis=1), 2, axis=2)[:, :f.shape[1], :f.shape[2]]
    bg = mask == 0
    fin = np.isfinite(up)
    err = np.abs(rec.astype(np.float64) - up.astype(np.float64))
    assert np.all(err[bg & fin] <= p.abs_eb)
    nf = bg & ~fin
    assert np.array_equal(np.isnan(rec[nf]), np.isnan(up[nf]))
    assert np.array_equal(rec[nf & ~np.isnan(up)], up[nf & ~np.isnan(up)])
    nan_bits = dec["prequant"][:, 1][np.isnan(b.ravel()[dec["prequant"][:, 0]])]
    assert len(nan_bits) > 0 and np.all(nan_bits == 0x7FC00000), "NaN bins store one canonical NaN"
    # the decoded codes equal the oracle's own step outputs; delta comes back from codes + outliers
    q, pq = O.prequantize(b, p.abs_eb)
    d = O.lorenzo(q)
    assert np.array_equal(dec["codes"], O.quant_codes(d, p.quant_radius).ravel())
    assert dec["prequant"][:, 0].tolist() == np.flatnonzero(pq.ravel()).tolist()
    lo_idx = np.flatnonzero(dec["codes"] == 0)
    assert dec["lorenzo"][:, 0].tolist() == lo_idx.tolist()
    assert np.array_equal(dec["lorenzo"][:, 1].view(np.int32), d.ravel()[lo_idx])
    # the peaks stored are the peaks found
    st, peaks, n = O.find_peaks(f, p)
    assert np.array_equal(dec["peaks"], peaks)


def pin_identity_binning_bound():
    p = O.make_params(bin_h=1, bin_w=1, abs_eb=2.5, atot_thr=300.0)
    f = tiny_frame(4, shape=(2, 19, 23))
    s, dec, rec = _roundtrip(f, p)
    mask = O.roi_mask(f.shape, p, dec["peaks"])
    assert dec["header"]["n_peaks"] > 0
    err = np.abs(rec.astype(np.float64) - f.astype(np.float64))
    assert np.all(err[mask == 0] <= 2.5), "with 1x1 binning every background pixel is within eb"
    assert np.all(err[mask == 1] == 0)


def pin_user_peaks_and_corruption():
    p = O.make_params()
    f = tiny_frame(1)
    up = np.array([[1, 0, 0], [0, 11, 12], [0, 5, 5]], np.uint16)
    s, dec, rec = _roundtrip(f, p, user_peaks=up)
    assert np.array_equal(dec["peaks"], up), "user coordinates kept in the order given"
    st, _ = O.compress_frame(f, p, user_peaks=np.array([[2, 0, 0]], np.uint16))
    assert st == O.ERR_INVALID_ARG
    st, need = O.compress_frame(f, p, capacity=64)
    assert st == O.ERR_CAPACITY and need == len(O.compress_frame(f, p)[1])
    bad = s.copy()
    bad[0] ^= 1
    assert O.decompress_frame(bad, f.shape)[0] == O.ERR_CORRUPT_STREAM
    assert O.decompress_frame(s[:-16], f.shape)[0] == O.ERR_CORRUPT_STREAM


def pin_nonsquare_bins_roundtrip():
    for bh, bw in ((1, 3), (3, 2)):
        p = O.make_params(bin_h=bh, bin_w=bw, atot_thr=300.0, abs_eb=4.0)
        f = tiny_frame(5, shape=(2, 17, 22))
        s, dec, rec = _roundtrip(f, p)
        b = O.bin_frame(f, bh, bw)
        up = np.repeat(np.repeat(b, bh, axis=1), bw, axis=2)[:, :f.shape[1], :f.shape[2]]
        mask = O.roi_mask(f.shape, p, dec["peaks"])
        err = np.abs(rec.astype(np.float64) - up.astype(np.float64))
        assert np.all(err[mask == 0] <= 4.0), (bh, bw)
        assert np.array_equal(rec[mask == 1], f[mask == 1])


# ---------------------------------------------------------------- ROI coding (§4, fpzip-style)
def _zigzag(r: int) -> int:
    r = ((r + (1 << 31)) % (1 << 32)) - (1 << 31)  # as int32
    return (2 * r) if r >= 0 else (-2 * r - 1)


def _float_of_order(m: np.ndarray) -> np.ndarray:
    """Inverse of the order map, written from its definition: m >= 2^31 came
    from a sign bit of 0 (u = m - 2^31), m < 2^31 from a sign bit of 1 (u = NOT m)."""
    m = m.astype(np.uint64)
    u = np.where(m >= (1 << 31), m - (1 << 31), (~m) & 0xFFFFFFFF)
    return u.astype(np.uint32).view(np.float32)


def decode_roi_section(sec: np.ndarray, n: int, h: int, w: int, n_words: int):
    """Independent decoder of a coded ROI section: a {(length, codeword): class}
    map from the canonical rule, bits read one at a time, and the prediction
    undone as a 2-D prefix sum (cumulative sums down and across, modulo 2^32),
    which is what inverting the Lorenzo rule amounts to."""
    lengths = sec[:O.ROI_CLASSES].astype(int)
    order = sorted((l, c) for c, l in enumerate(lengths) if l > 0)
    table, code, prev = {}, 0, None
    for l, c in order:
        if prev is not None:
            code = (code + 1) << (l - prev)
        table[(l, code)] = c
        prev = l
    a16 = lambda x: (x + 15) & ~15
    offs = sec[48:48 + 4 * n].view("<u4")
    words = sec[48 + a16(4 * n):48 + a16(4 * n) + 4 * n_words].view("<u4")
    out = np.zeros((n, h, w), np.float32)
    bits_total = 0
    for k in range(n):
        pos = int(offs[k]) * 32
        start = pos

        def bit():
            nonlocal pos
            b = (int(words[pos // 32]) >> (31 - pos % 32)) & 1
            pos += 1
            return b
        z = np.zeros(h * w, np.int64)
        for i in range(h * w):
            l, cw = 0, 0
            while (l, cw) not in table:
                cw = (cw << 1) | bit()
                l += 1
                assert l <= 32
            c = table[(l, cw)]
            v = 0 if c == 0 else 1
            for _ in range(c - 1):
                v = (v << 1) | bit()
            z[i] = v
        bits_total += pos - start
        r = np.where(z & 1, -((z + 1) >> 1), z >> 1)  # unfold
        r = r.reshape(h, w)
        r[0, 0] += 1 << 31  # the first value was predicted by m(+0.0) = 2^31
        m = np.cumsum(np.cumsum(r, axis=0), axis=1) % (1 << 32)
        out[k] = _float_of_order(m)
    return lengths, out, bits_total


def pin_roi_order_and_classes():
    xs = np.array([-np.inf, -3e38, -1.0, -1e-40, -0.0, 0.0, 1e-40, 1.0, 2.0, 3e38, np.inf], np.float32)
    m = [O.roi_order_bits(float(x)) for x in xs]
    assert all(a < b for a, b in zip(m, m[1:])), "the integer order is the float order"
    assert O.roi_order_bits(0.0) == 1 << 31 and O.roi_order_bits(-0.0) == (1 << 31) - 1
    assert O.roi_order_bits(1.0) == 0x3F800000 + (1 << 31)
    for z, c in ((0, 0), (1, 1), (2, 2), (3, 2), (4, 3), (255, 8), (1 << 31, 32), (0xFFFFFFFF, 32)):
        assert O.roi_class(z) == c, (z, c)


def pin_roi_residual_closed_forms():
    # a constant window: only the first value carries anything
    for x in (0.0, 37.5, -2.25):
        z = O.roi_residuals(np.full((5, 7), x, np.float32))
        assert z[0, 0] == _zigzag(O.roi_order_bits(x) - (1 << 31))
        assert np.count_nonzero(z) == (z[0, 0] != 0)
    # float bits in a plane u = U0 + A i + B j: the 2-D predictor is exact inside,
    # the first row differs by B, the first column by A (A != B catches a swap)
    i, j = np.mgrid[0:6, 0:9]
    for sign in (0, 1):
        U0, A, B = 0x3F800000, 3, -2
        u = (U0 + A * i + B * j).astype(np.uint32) | np.uint32(sign << 31)
        z = O.roi_residuals(u.view(np.float32))
        s = -1 if sign else 1  # NOT u reverses the order of negative floats
        assert z[0, 0] == _zigzag(O.roi_order_bits(float(u.view(np.float32)[0, 0])) - (1 << 31))
        assert np.all(z[0, 1:] == _zigzag(s * B)), "first row: the left neighbour predicts"
        assert np.all(z[1:, 0] == _zigzag(s * A)), "first column: the value above predicts"
        assert np.all(z[1:, 1:] == 0), "inside: the Lorenzo rule is exact on a plane"


def pin_roi_roundtrip_and_independent_decoder():
    rng = np.random.default_rng(7)
    cases = [rng.normal(30, 8, (6, 17, 17)).astype(np.float32),       # background-like windows
             (rng.normal(30, 8, (3, 5, 3)) + np.arange(3)).astype(np.float32),
             rng.normal(0, 1e-3, (2, 9, 11)).astype(np.float32)]
    spec = rng.normal(100, 5, (2, 7, 7)).astype(np.float32)
    spec[0, 1, 1] = np.nan
    spec[0, 2, 2] = np.array([0xFFC01234], np.uint32).view(np.float32)[0]  # NaN with a payload
    spec[0, 3, 3], spec[0, 4, 4], spec[1, 0, 0], spec[1, 6, 6] = np.inf, -np.inf, -0.0, 1e-42
    cases.append(spec)
    cases.append(np.full((1, 1, 1), 5.0, np.float32))
    for win in cases:
        coding, nw, sec = O.roi_encode(win)
        n, h, w = win.shape
        st, dec = O.roi_decode(sec, coding, nw, n, h, w)
        assert st == O.OK and np.array_equal(dec.view(np.uint32), win.view(np.uint32)), "lossless, bit for bit"
        if coding == 2:
            assert np.array_equal(sec[:win.size * 4].view(np.float32).view(np.uint32), win.ravel().view(np.uint32))
            continue
        lengths, dec2, bits = decode_roi_section(sec, n, h, w, nw)
        assert np.array_equal(dec2.view(np.uint32), win.view(np.uint32)), "the independent decoder agrees"
        # the code is a complete prefix code, optimal for the class counts
        cls = np.array([O.roi_class(int(z)) for wi in win for z in O.roi_residuals(wi).ravel()])
        counts = np.bincount(cls, minlength=O.ROI_CLASSES)
        used = lengths[lengths > 0]
        if len(used) > 1:
            assert sum(2.0 ** -l for l in used) == 1.0
        extra = int(np.maximum(cls - 1, 0).sum())
        assert bits == heap_huffman_cost(counts) + extra, "Huffman-optimal classes plus the raw low bits"
        assert len(sec) == 48 + ((4 * n + 15) & ~15) + ((4 * nw + 15) & ~15)
    # incompressible windows (random bit patterns) fall back to the raw floats
    raw = rng.integers(0, 1 << 32, (4, 17, 17), dtype=np.uint64).astype(np.uint32).view(np.float32)
    coding, nw, sec = O.roi_encode(raw)
    assert coding == 2 and nw == 0 and np.array_equal(sec[:raw.size * 4], raw.view(np.uint8).ravel())
    assert O.roi_decode(sec, 2, 0, 4, 17, 17)[0] == O.OK


def pin_roi_corrupt_sections():
    rng = np.random.default_rng(8)
    win = rng.normal(30, 8, (3, 17, 17)).astype(np.float32)
    coding, nw, sec = O.roi_encode(win)
    assert coding == 1
    ok = lambda s, c=coding, w=nw: O.roi_decode(s, c, w, 3, 17, 17)[0]
    assert ok(sec) == O.OK
    assert ok(sec[:-16]) == O.ERR_CORRUPT_STREAM, "short section"
    assert ok(sec, w=nw + 4) == O.ERR_CORRUPT_STREAM, "word count off"
    bad = sec.copy()
    bad[0] = 40
    assert ok(bad) == O.ERR_CORRUPT_STREAM, "code length above 32"
    bad = sec.copy()
    bad[int(np.flatnonzero(sec[:33])[0])] += 1
    assert ok(bad) == O.ERR_CORRUPT_STREAM, "incomplete code"
    bad = sec.copy()
    bad[48:52] = np.array([1], "<u4").view(np.uint8)
    assert ok(bad) == O.ERR_CORRUPT_STREAM, "first window must start at word 0"
    bad = sec.copy()
    bad[52:56], bad[56:60] = bad[56:60].copy(), bad[52:56].copy()
    assert ok(bad) == O.ERR_CORRUPT_STREAM, "window offsets out of order"
    assert ok(sec, c=3) == O.ERR_CORRUPT_STREAM


def pin_roi_frame():
    """With the ROI coder the stream differs from the raw one only in where the
    windows live: the same header counts, peaks, lengths, index, outliers and
    bitstream, then a section that decodes to the raw windows."""
    f = tiny_frame(3, shape=(3, 30, 36))
    for i, (pn, r, c) in enumerate(((0, 8, 9), (1, 20, 25), (2, 2, 3))):
        f[pn, r - 1:r + 2, c - 1:c + 2] += 900.0 + 50 * i
    base = O.make_params(atot_thr=300.0)
    st0, s0 = O.compress_frame(f, base)
    p1 = O.make_params(atot_thr=300.0, roi_coder=1)
    s1, dec1, rec1 = _roundtrip(f, p1)
    h0, h1 = O.parse_header(s0), O.parse_header(s1)
    assert st0 == O.OK and h0["n_peaks"] >= 3 and h0["roi_coding"] == 0
    assert h1["roi_coding"] in (1, 2) and h1["roi_bytes"] > 0
    o0, o1 = O.section_offsets(h0), O.section_offsets(h1)
    assert o1["lengths"] == o1["roi"], "no windows in the ROI section"
    assert np.array_equal(s0[o0["lengths"]:o0["end"]], s1[o1["lengths"]:o1["roi_section"]])
    assert np.array_equal(s0[:o0["roi"]][:64], s1[:64]) and np.array_equal(s0[96:o0["roi"]], s1[96:o1["roi"]])
    assert len(s1) == o1["end"] == h1["total_bytes"]
    win = O.roi_extract(f, base, dec1["peaks"])
    coding, nw, sec = O.roi_encode(win)
    assert (coding, nw) == (h1["roi_coding"], h1["roi_words"]) and np.array_equal(s1[o1["roi_section"]:], sec)
    st, rec0 = O.decompress_frame(s0, f.shape)
    assert st == O.OK and np.array_equal(rec0.view(np.uint32), rec1.view(np.uint32)), "same frame back"
    bad = s1.copy()
    bad[80:84] = np.array([h1["roi_bytes"] - 16], "<u4").view(np.uint8)
    assert O.decompress_frame(bad, f.shape)[0] == O.ERR_CORRUPT_STREAM


def pin_non_hit_rejection():
    f = tiny_frame(3, shape=(3, 30, 36))
    for i, (pn, r, c) in enumerate(((0, 8, 9), (1, 20, 25), (2, 2, 3))):
        f[pn, r - 1:r + 2, c - 1:c + 2] += 900.0 + 50 * i
    p = O.make_params(atot_thr=300.0)
    st, peaks, n = O.find_peaks(f, p)
    assert st == O.OK and n >= 3
    st, ref = O.compress_frame(f, p)
    st_eq, s_eq = O.compress_frame(f, O.make_params(atot_thr=300.0, nhr_min_peaks=n))
    assert st_eq == O.OK and np.array_equal(s_eq, ref), "a hit with exactly nhr_min_peaks peaks is kept, unchanged"
    assert O.compress_frame(f, O.make_params(atot_thr=300.0, nhr_min_peaks=n + 1))[0] == O.REJECTED
    up = np.array([[0, 1, 1]], np.uint16)
    assert O.compress_frame(f, O.make_params(nhr_min_peaks=2), user_peaks=up)[0] == O.REJECTED
    assert O.compress_frame(f, O.make_params(nhr_min_peaks=1), user_peaks=up)[0] == O.OK
    # too many peaks is still CAPACITY, whatever the rejection threshold
    assert O.compress_frame(f, O.make_params(atot_thr=300.0, max_peaks=1, nhr_min_peaks=5))[0] == O.ERR_CAPACITY


# ---------------------------------------------------------------- chunks sharing a codebook (§5.3.4)
def _chunk_frames(n=6, seed=9, shape=(2, 20, 24)):
    fs = []
    for k in range(n):
        f = tiny_frame(seed + k, shape=shape)
        f[k % 2, 8, 9] += 900.0 + 40 * k  # a peak in every frame
        fs.append(f)
    return np.stack(fs)


def _codes_of(frame, p):
    b = O.bin_frame(frame, p.bin_h, p.bin_w)
    q, pq = O.prequantize(b, p.abs_eb)
    return O.quant_codes(O.lorenzo(q), p.quant_radius).ravel()


def pin_chunks_share_one_codebook():
    fs = _chunk_frames()
    p1 = O.make_params(atot_thr=300.0)
    # chunk_frames = 1: a call equals its frames compressed one by one
    st, streams, _ = O.compress_frames(fs, p1)
    assert (st == O.OK).all()
    for k in range(len(fs)):
        assert np.array_equal(streams[k], O.compress_frame(fs[k], p1)[1])
    p4 = O.make_params(atot_thr=300.0, chunk_frames=4)
    st, streams4, _ = O.compress_frames(fs, p4)
    assert (st == O.OK).all()
    nsym = 2 * p4.quant_radius
    for c0, c1 in ((0, 4), (4, 6)):  # chunks by frame index: [0, 4) and [4, 6)
        hs = [O.parse_header(streams4[k]) for k in range(c0, c1)]
        assert [h["back_ref"] for h in hs] == list(range(c1 - c0)), "the first frame of a chunk is its head"
        o = O.section_offsets(hs[0])
        lengths = streams4[c0][o["lengths"]:o["lengths"] + nsym].astype(int)
        # one codebook from the summed histogram: optimal for it (heap Huffman),
        # and equal to the oracle's lengths for that histogram
        hist = sum(np.bincount(_codes_of(fs[k], p4), minlength=nsym) for k in range(c0, c1))
        st_l, ref_len = O.huffman_lengths(hist.astype(np.uint64))
        assert np.array_equal(lengths, ref_len.astype(int))
        assert int((hist * lengths).sum()) == heap_huffman_cost(hist)
        for k in range(c0 + 1, c1):  # later frames keep no lengths: decoded with the head's
            ok = O.section_offsets(O.parse_header(streams4[k]))
            assert ok["chunk_index"] == ok["lengths"] and len(streams4[k]) == ok["end"]
            dec = decode_stream(streams4[k], lengths=lengths)
            assert np.array_equal(dec["codes"], _codes_of(fs[k], p4))
    # decoded frames equal the frames decoded from per-frame codebooks (only the code changes)
    st_d, rec4 = O.decompress_frames(streams4, fs.shape[1:])
    st_1, rec1 = O.decompress_frames(streams, fs.shape[1:])
    assert (st_d == O.OK).all() and (st_1 == O.OK).all()
    assert np.array_equal(rec4.view(np.uint32), rec1.view(np.uint32))
    # a later frame alone has no code lengths: its own decoder refuses it
    assert O.decompress_frame(streams4[1], fs.shape[1:])[0] == O.ERR_CORRUPT_STREAM
    assert O.decompress_frames([streams4[1]], fs.shape[1:])[0][0] == O.ERR_CORRUPT_STREAM
    # chunk membership follows the frame index: a change to frame 5 leaves chunk 0's streams alone
    fs2 = fs.copy()
    fs2[5] += 1.0
    st2, streams_b, _ = O.compress_frames(fs2, p4)
    assert all(np.array_equal(streams4[k], streams_b[k]) for k in range(4))


def pin_chunk_head_skips_frames_not_coded():
    """Frames rejected or in error do not feed the codebook; the head is the
    chunk's first coded frame."""
    fs = _chunk_frames(n=4)
    p = O.make_params(atot_thr=300.0, chunk_frames=4)
    up = np.zeros((4, p.max_peaks, 3), np.uint16)
    up[1, 0] = [0, 8, 9]
    up[2, 0] = [1, 8, 9]
    up[3, 0] = [0, 3, 3]
    n_user = np.array([0, 1, 1, 1], np.int64)
    pr = O.make_params(atot_thr=300.0, chunk_frames=4, nhr_min_peaks=1)
    st, streams, _ = O.compress_frames(fs, pr, user_peaks=up, n_user=n_user)
    assert st.tolist() == [O.REJECTED, O.OK, O.OK, O.OK]
    assert [O.parse_header(streams[k])["back_ref"] for k in (1, 2, 3)] == [0, 1, 2]
    nsym = 2 * pr.quant_radius
    hist = sum(np.bincount(_codes_of(fs[k], pr), minlength=nsym) for k in (1, 2, 3))
    o = O.section_offsets(O.parse_header(streams[1]))
    assert np.array_equal(streams[1][o["lengths"]:o["lengths"] + nsym], O.huffman_lengths(hist.astype(np.uint64))[1])
    st_d, rec = O.decompress_frames([streams[k] for k in (1, 2, 3)], fs.shape[1:])
    assert (st_d == O.OK).all()


ALL_PINS = [
    pin_candidates_brute_force, pin_candidate_special_cases, pin_evaluation_special_cases,
    pin_evaluation_brute_force, pin_find_peaks_frame, pin_roi, pin_binning, pin_prequantize,
    pin_lorenzo, pin_codes_histogram, pin_huffman_small, pin_huffman_optimal, pin_pack_decode,
    pin_frame_roundtrip, pin_identity_binning_bound, pin_user_peaks_and_corruption,
    pin_nonsquare_bins_roundtrip, pin_lorenzo_dims, pin_lorenzo_dims_roundtrip,
    pin_roi_order_and_classes, pin_roi_residual_closed_forms, pin_roi_roundtrip_and_independent_decoder,
    pin_roi_corrupt_sections, pin_roi_frame, pin_non_hit_rejection, pin_chunks_share_one_codebook,
    pin_chunk_head_skips_frames_not_coded,
]
