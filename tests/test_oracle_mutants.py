"""Plants plausible mistakes in copies of the CPU oracle and requires the pins
to catch every one of them.  Each mistake is a one-line edit of the oracle's C
source (a dropped term, a wrong sign, index or comparison, a transposed
operand); each mutant is compiled to a temporary library and the pins run
against it in a child process.  Mistakes are planted only in the oracle, on the
CPU."""
import json
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

MUTANTS = {
    # a1 local maximum
    "tie_rule_flipped": ("if (!(v > u)) return 0;", "if (!(v >= u)) return 0;"),
    "amax_strict": ("if (!(v >= amax_thr)) return 0;", "if (!(v > amax_thr)) return 0;"),
    "window_shrunk": ("for (long dr = -rank; dr <= rank; ++dr) {\n    for (long dc = -rank; dc <= rank; ++dc) {\n      const long rr = (long)r + dr, cc = (long)c + dc;\n      if (dr == 0 && dc == 0) continue;",
                      "for (long dr = -rank + 1; dr <= rank; ++dr) {\n    for (long dc = -rank; dc <= rank; ++dc) {\n      const long rr = (long)r + dr, cc = (long)c + dc;\n      if (dr == 0 && dc == 0) continue;"),
    # a2 evaluation
    "ring_inner_inclusive": ("if (d2 < r0 * r0 || d2 >= outer * outer) continue;\n      const long rr = (long)r + dr, cc = (long)c + dc;\n      if (!in_panel(rr, cc, rows, cols)) continue;\n      sum +=",
                             "if (d2 <= r0 * r0 || d2 >= outer * outer) continue;\n      const long rr = (long)r + dr, cc = (long)c + dc;\n      if (!in_panel(rr, cc, rows, cols)) continue;\n      sum +="),
    "sample_variance": ("var = ss / (float)n;", "var = n > 1 ? ss / (float)(n - 1) : 0.0f;"),
    "snr_without_sqrt": ("sigma * sqrtf((float)npix)", "sigma * (float)npix"),
    "atot_not_strict": ("if (!(atot > p->atot_thr)) return 0;", "if (!(atot >= p->atot_thr)) return 0;"),
    "npix_max_off_by_one": ("npix > p->npix_max", "npix >= p->npix_max"),
    "threshold_ignores_sigma": ("const float thr = p->pix_nsigma * sigma;", "const float thr = p->pix_nsigma;"),
    # a3 ROI
    "roi_off_centre": ("const long r0 = (long)peaks[3 * k + 1] - p->roi_h / 2;\n    const long c0 = (long)peaks[3 * k + 2] - p->roi_w / 2;\n    for (long i = 0; i < p->roi_h; ++i) {",
                       "const long r0 = (long)peaks[3 * k + 1] - p->roi_h / 2 + 1;\n    const long c0 = (long)peaks[3 * k + 2] - p->roi_w / 2;\n    for (long i = 0; i < p->roi_h; ++i) {"),
    "roi_fill_nonzero": ("? panel[(size_t)rr * g->cols + (size_t)cc] : 0.0f;", "? panel[(size_t)rr * g->cols + (size_t)cc] : 1.0f;"),
    # a4 binning
    "bin_full_count": ("s / (float)count;", "s / (float)(bin_h * bin_w);"),
    "bin_transposed": ("const float x = frame[pn * plane + (size_t)r * g->cols + c];", "const float x = frame[pn * plane + (size_t)(bi * bin_h + j % bin_h) * g->cols + (bj * bin_w + i % bin_w)];"),
    # a5 prequantisation
    "round_half_away": ("const float t = rintf(b * recip);", "const float t = roundf(b * recip);"),
    "bound_strict": ("if (fabs((double)b - (double)b_hat) > (double)abs_eb) outlier = 1;", "if (fabs((double)b - (double)b_hat) >= (double)abs_eb) outlier = 1;"),
    "no_bound_check": ("if (fabs((double)b - (double)b_hat) > (double)abs_eb) outlier = 1;", "(void)b_hat;"),
    "pq_limit_missing": ("int outlier = !isfinite(b) || !(fabsf(t) < ORC_PQ_LIMIT);", "int outlier = !isfinite(b);"),
    # a6 Lorenzo
    "lorenzo_diag_sign": ("- up - left + diag);", "- up - left - diag);"),
    "lorenzo_crosses_panels": ("const int64_t up = i > 0 ? qp[(size_t)(i - 1) * wb + j] : 0;",
                               "const int64_t up = (i > 0 || pn > 0) ? qp[(int64_t)(i - 1) * wb + j] : 0;"),
    "lorenzo1_resets_at_rows": ("const int64_t prev = k > 0 ? q[k - 1] : 0;", "const int64_t prev = k % wb > 0 ? q[k - 1] : 0;"),
    "lorenzo3_corner_sign": ("+ corner[1][1][1];\n        delta_out", "- corner[1][1][1];\n        delta_out"),
    "lorenzo3_no_stack": ("const int inside = (a == 0 || pn > 0) && (b == 0 || i > 0) && (c == 0 || j > 0);\n              corner[a][b][c] = inside ?",
                          "const int inside = (a == 0) && (b == 0 || i > 0) && (c == 0 || j > 0);\n              corner[a][b][c] = inside ?"),
    "dims_not_in_header": ("put_u32(out + 72, p->lorenzo_dims == 2 ? 0u : (uint32_t)p->lorenzo_dims);", "put_u32(out + 72, 0u);"),
    # a7 codes
    "code_sign_flipped": ("? (uint16_t)(d + radius)", "? (uint16_t)(radius - d)"),
    # a9 Huffman
    "huffman_internal_first": ("weight[next_leaf] <= weight[next_internal]", "weight[next_leaf] < weight[next_internal]"),
    "huffman_unsorted_ties": ("return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);", "return x->s > y->s ? -1 : (x->s < y->s ? 1 : 0);"),
    "canonical_no_shift": ("code = (code + 1) << (L - prev_len);", "code = (code + 1);"),
    # a10 packing
    "lsb_first": ("words_out[w] |= 1u << (31 - bit % 32);", "words_out[w] |= 1u << (bit % 32);"),
    "chunks_not_word_aligned": ("word_base += (uint32_t)((bit + 31) / 32);", "word_base += (uint32_t)(bit / 32);"),
    # a11 outliers
    "outlier_delta_dropped": ("put_u32(out + L.lorenzo + 8 * a + 4, (uint32_t)delta[i]);", "put_u32(out + L.lorenzo + 8 * a + 4, 0u);"),
    "nan_not_canonical": ("if (isnan(binned[i])) bits = ORC_CANONICAL_NAN;", ""),
    # a13 decompression
    "inverse_diag_sign": ("= delta[base + (size_t)i * wb + j] + up + left - diag;", "= delta[base + (size_t)i * wb + j] + up + left + diag;"),
    "inverse1_resets_at_rows": ("q[k] = delta[k] + (k > 0 ? q[k - 1] : 0);", "q[k] = delta[k] + (k % wb > 0 ? q[k - 1] : 0);"),
    "inverse3_corner_sign": ("+ corner[1][1][1];\n            q[(size_t)pn", "- corner[1][1][1];\n            q[(size_t)pn"),
    "restore_skips_roi": ("            frame_out[pn * plane + (size_t)(r0 + i) * g->cols + (size_t)(c0 + j)] =",
                          "            if (0) frame_out[pn * plane + (size_t)(r0 + i) * g->cols + (size_t)(c0 + j)] ="),
    # ROI coding (§4, fpzip-style) and non-hit rejection (§1, §4)
    "roi_order_ignores_sign": ("return (u & 0x80000000u) ? ~u : (u | 0x80000000u);", "return u | 0x80000000u;"),
    "roi_pred_no_diag": ("pred = up + left - diag;", "pred = up + left;"),
    "roi_first_pred_zero": ("        pred = 0x80000000u;\n", "        pred = 0u;\n"),
    "roi_zigzag_swapped": ("r >= 0 ? 2u * (uint32_t)r : 2u * (uint32_t)(-(int64_t)r) - 1u;",
                           "r >= 0 ? 2u * (uint32_t)r + 1u : 2u * (uint32_t)(-(int64_t)r) - 2u;"),
    "roi_class_short": ("  while (z) {\n    ++c;", "  while (z > 1) {\n    ++c;"),
    "roi_extra_lsb_first": ("for (int b = (int)c - 2; b >= 0; --b, ++bit)", "for (int b = 0; b <= (int)c - 2; ++b, ++bit)"),
    "roi_no_fallback": ("if (n_windows == 0 || roi_coded_bytes(n_windows, (uint32_t)words) >= raw) {",
                        "if (n_windows == 0) {"),
    "roi_section_size_not_in_header": ("put_u32(out + 80, (uint32_t)roi_bytes);", "put_u32(out + 80, 0u);"),
    "nhr_inclusive": ("if ((int64_t)n_peaks < (int64_t)p->nhr_min_peaks) {", "if ((int64_t)n_peaks <= (int64_t)p->nhr_min_peaks) {"),
    # chunks sharing one codebook (§5.3.4)
    "chunk_head_last": ("      if (head < 0) head = f;", "      head = f;"),
    "chunk_hist_not_summed": ("hsum[s2] += w[f].hist[s2];", "hsum[s2] = w[f].hist[s2];"),
    "chunk_lengths_always_kept": ("L.chunk_index = L.lengths + (lengths_here ? align16(n_symbols) : 0);",
                                  "L.chunk_index = L.lengths + align16(n_symbols);"),
    "upsample_wrong_axis": ("bhat[((size_t)pn * hb + r / p.bin_h) * wb + c / p.bin_w];", "bhat[((size_t)pn * hb + r / p.bin_w) * wb + c / p.bin_h];"),
}

_RUNNER = r"""
import json, sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins
failed = []
with oracle.use_library({lib!r}):
    for pin in oracle_pins.ALL_PINS:
        try:
            pin()
        except Exception as e:  # AssertionError or a downstream failure
            failed.append(pin.__name__)
print(json.dumps(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path), name)
    code = _RUNNER.format(root=ROOT, tests=HERE, lib=lib)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    if res.returncode != 0:
        return  # a crash is a caught mistake too
    failed = json.loads(res.stdout.strip().splitlines()[-1])
    assert failed, f"no pin caught the planted mistake {name!r}"
