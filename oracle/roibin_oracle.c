/*
 * ROIBIN-SZ oracle: a plain, slow, single-threaded CPU definition of the method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library, never
 * to stand in for it: only tests/, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Compile with -O2 -ffp-contract=off: every floating-point step below is meant
 * to round exactly once, in the order written.
 *
 * The steps follow the paper (arXiv 2206.11297) in its own order:
 *   peak finding (§4.2), ROI extraction (§4, §4.1), binning (§4.1, §6),
 *   absolute-error-bounded SZ-style coding of the binned background (§5.3.2,
 *   §5.3.3, §6), and the inverse for the round trip (§4.1).
 * Where the paper is silent the reading taken is stated at the step.
 */
#include "roibin_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int in_panel(long r, long c, long rows, long cols) {
  return r >= 0 && r < rows && c >= 0 && c < cols;
}

static uint64_t align16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

/* --------------------------------------------------------------------------
 * a1. Local-maximum candidate (§4.2): a pixel starts a peak when it is the
 * maximum of the (2 rank + 1)^2 window around it (7x7 for rank 3), clipped to
 * its panel, and it is not below amax_thr (300 ADU in the paper).  Reading for ties: the pixel must be >= every window pixel and
 * strictly > every window pixel that precedes it in row-major order, so a flat
 * plateau yields exactly one candidate, its first pixel.  Any NaN in the window
 * makes the comparison fail.
 * ------------------------------------------------------------------------ */
int orc_is_peak_candidate(const float* panel, uint32_t rows, uint32_t cols, uint32_t r,
                          uint32_t c, int32_t rank, float amax_thr) {
  const float v = panel[(size_t)r * cols + c];
  if (!(v >= amax_thr)) return 0;
  for (long dr = -rank; dr <= rank; ++dr) {
    for (long dc = -rank; dc <= rank; ++dc) {
      const long rr = (long)r + dr, cc = (long)c + dc;
      if (dr == 0 && dc == 0) continue;
      if (!in_panel(rr, cc, rows, cols)) continue;
      const float u = panel[(size_t)rr * cols + (size_t)cc];
      const int precedes = (dr < 0) || (dr == 0 && dc < 0);
      if (precedes) {
        if (!(v > u)) return 0;
      } else {
        if (!(v >= u)) return 0;
      }
    }
  }
  return 1;
}

/* --------------------------------------------------------------------------
 * a2. Candidate evaluation (§4.2).  The paper lists the tests: neighbouring
 * pixels above zero form the peak, total intensity over 600, SNR over 10, and
 * between 2 and 30 pixels.  It defines neither the background nor the noise.  Reading:
 *   - background ring: in-panel pixels with r0^2 <= di^2 + dj^2 < (r0+dr)^2;
 *     bkg = mean, sigma = population standard deviation (two passes),
 *     row-major order; an empty ring gives bkg = 0, sigma = 0;
 *   - peak pixels: in-panel pixels of the local-maximum window with
 *     I - bkg > pix_nsigma * sigma (pix_nsigma = 0 gives the paper's plain
 *     above-zero test after background subtraction);
 *   - npix = their count, atot = sum of (I - bkg) over them;
 *   - keep iff npix_min <= npix <= npix_max, atot > atot_thr and
 *     atot > son_min * sigma * sqrt(npix)  (SNR = atot / (sigma sqrt(npix))).
 * The accept/reject decision is taken in float32, the precision of the data
 * and of the kernel (the paper fixes none): every operation rounds once, in
 * the order written, and sqrtf is correctly rounded.
 * ------------------------------------------------------------------------ */
int orc_evaluate_peak(const float* panel, uint32_t rows, uint32_t cols, uint32_t r, uint32_t c,
                      const orc_params* p) {
  const long r0 = p->ring_r0, outer = (long)p->ring_r0 + p->ring_dr;
  const long reach = outer - 1;

  float sum = 0.0f;
  long n = 0;
  for (long dr = -reach; dr <= reach; ++dr) {
    for (long dc = -reach; dc <= reach; ++dc) {
      const long d2 = dr * dr + dc * dc;
      if (d2 < r0 * r0 || d2 >= outer * outer) continue;
      const long rr = (long)r + dr, cc = (long)c + dc;
      if (!in_panel(rr, cc, rows, cols)) continue;
      sum += panel[(size_t)rr * cols + (size_t)cc];
      ++n;
    }
  }
  float bkg = 0.0f, var = 0.0f;
  if (n > 0) {
    bkg = sum / (float)n;
    float ss = 0.0f;
    for (long dr = -reach; dr <= reach; ++dr) {
      for (long dc = -reach; dc <= reach; ++dc) {
        const long d2 = dr * dr + dc * dc;
        if (d2 < r0 * r0 || d2 >= outer * outer) continue;
        const long rr = (long)r + dr, cc = (long)c + dc;
        if (!in_panel(rr, cc, rows, cols)) continue;
        const float d = panel[(size_t)rr * cols + (size_t)cc] - bkg;
        ss += d * d;
      }
    }
    var = ss / (float)n;
  }
  const float sigma = sqrtf(var);
  const float thr = p->pix_nsigma * sigma;

  long npix = 0;
  float atot = 0.0f;
  for (long dr = -p->rank; dr <= p->rank; ++dr) {
    for (long dc = -p->rank; dc <= p->rank; ++dc) {
      const long rr = (long)r + dr, cc = (long)c + dc;
      if (!in_panel(rr, cc, rows, cols)) continue;
      const float d = panel[(size_t)rr * cols + (size_t)cc] - bkg;
      if (d > thr) {
        ++npix;
        atot += d;
      }
    }
  }
  if (npix < p->npix_min || npix > p->npix_max) return 0;
  if (!(atot > p->atot_thr)) return 0;
  if (!(atot > p->son_min * sigma * sqrtf((float)npix))) return 0;
  return 1;
}

/* a1 + a2 over a whole frame.  Peaks come out in (panel, row, col) order.
 * More than peaks_capacity accepted peaks is an error (no silent truncation);
 * *n_found then holds the full count. */
int orc_find_peaks(const float* frame, const orc_geometry* g, const orc_params* p,
                   uint16_t* peaks_out, uint32_t peaks_capacity, uint32_t* n_found) {
  uint32_t n = 0;
  const size_t plane = (size_t)g->rows * g->cols;
  for (uint32_t pn = 0; pn < g->n_panels; ++pn) {
    const float* panel = frame + pn * plane;
    for (uint32_t r = 0; r < g->rows; ++r) {
      for (uint32_t c = 0; c < g->cols; ++c) {
        if (!orc_is_peak_candidate(panel, g->rows, g->cols, r, c, p->rank, p->amax_thr)) continue;
        if (!orc_evaluate_peak(panel, g->rows, g->cols, r, c, p)) continue;
        if (n < peaks_capacity) {
          peaks_out[3 * n + 0] = (uint16_t)pn;
          peaks_out[3 * n + 1] = (uint16_t)r;
          peaks_out[3 * n + 2] = (uint16_t)c;
        }
        ++n;
      }
    }
  }
  *n_found = n;
  return n > peaks_capacity ? ORC_ERR_CAPACITY : ORC_OK;
}

/* --------------------------------------------------------------------------
 * a3. ROI extraction (§4, §4.1): one roi_h x roi_w window per peak (twice the
 * peak size plus one, 17x17), centred on the peak pixel: rows r - roi_h/2 ..
 * r - roi_h/2 + roi_h - 1, likewise for columns.  Positions past the panel edge
 * take a constant fill, 0.0f.  Windows never cross into another panel.
 * ------------------------------------------------------------------------ */
void orc_roi_extract(const float* frame, const orc_geometry* g, const orc_params* p,
                     const uint16_t* peaks, uint32_t n_peaks, float* roi_out) {
  const size_t plane = (size_t)g->rows * g->cols;
  const size_t win = (size_t)p->roi_h * (size_t)p->roi_w;
  for (uint32_t k = 0; k < n_peaks; ++k) {
    const float* panel = frame + peaks[3 * k] * plane;
    const long r0 = (long)peaks[3 * k + 1] - p->roi_h / 2;
    const long c0 = (long)peaks[3 * k + 2] - p->roi_w / 2;
    for (long i = 0; i < p->roi_h; ++i) {
      for (long j = 0; j < p->roi_w; ++j) {
        const long rr = r0 + i, cc = c0 + j;
        roi_out[k * win + (size_t)i * p->roi_w + (size_t)j] =
            in_panel(rr, cc, g->rows, g->cols) ? panel[(size_t)rr * g->cols + (size_t)cc] : 0.0f;
      }
    }
  }
}

/* The ROI mask: 1 on every in-panel pixel covered by some peak's window. */
void orc_roi_mask(const orc_geometry* g, const orc_params* p, const uint16_t* peaks,
                  uint32_t n_peaks, uint8_t* mask_out) {
  const size_t plane = (size_t)g->rows * g->cols;
  memset(mask_out, 0, plane * g->n_panels);
  for (uint32_t k = 0; k < n_peaks; ++k) {
    const long r0 = (long)peaks[3 * k + 1] - p->roi_h / 2;
    const long c0 = (long)peaks[3 * k + 2] - p->roi_w / 2;
    for (long i = 0; i < p->roi_h; ++i)
      for (long j = 0; j < p->roi_w; ++j)
        if (in_panel(r0 + i, c0 + j, g->rows, g->cols))
          mask_out[peaks[3 * k] * plane + (size_t)(r0 + i) * g->cols + (size_t)(c0 + j)] = 1;
  }
}

/* --------------------------------------------------------------------------
 * a4. Binning (§4.1, §6: the bin_h x bin_w window is replaced by the mean
 * of its values), applied to the whole frame including ROI pixels, per panel.
 * Reading for edges: a bin at the bottom/right edge of a panel whose size is
 * not a multiple of the factor averages only its in-panel pixels.  The sum
 * starts from the block's first pixel and adds the rest in row-major order in
 * float32, then one IEEE float32 division by the pixel count.
 * ------------------------------------------------------------------------ */
void orc_bin(const float* frame, const orc_geometry* g, int32_t bin_h, int32_t bin_w,
             float* binned_out) {
  const uint32_t hb = (g->rows + bin_h - 1) / bin_h, wb = (g->cols + bin_w - 1) / bin_w;
  const size_t plane = (size_t)g->rows * g->cols;
  for (uint32_t pn = 0; pn < g->n_panels; ++pn) {
    for (uint32_t bi = 0; bi < hb; ++bi) {
      for (uint32_t bj = 0; bj < wb; ++bj) {
        float s = 0.0f;
        int count = 0;
        for (int32_t i = 0; i < bin_h; ++i) {
          const uint32_t r = bi * bin_h + i;
          if (r >= g->rows) break;
          for (int32_t j = 0; j < bin_w; ++j) {
            const uint32_t c = bj * bin_w + j;
            if (c >= g->cols) break;
            const float x = frame[pn * plane + (size_t)r * g->cols + c];
            s = (count == 0) ? x : s + x;
            ++count;
          }
        }
        binned_out[((size_t)pn * hb + bi) * wb + bj] = s / (float)count;
      }
    }
  }
}

/* --------------------------------------------------------------------------
 * a5. Prequantisation for an absolute error bound eb (§5.3.3: |d - d~| within
 * eb, guaranteed on the binned data).  The SZ internals are not in the paper
 * (§5.3.2 names Lorenzo prediction and linear quantisation only).  Reading:
 * the dual-quantisation scheme of cuSZ (Tian et al., PACT 2020):
 *   q = rint(b * fl(1 / (2 eb)))  in float32, ties to even;
 *   b^ = fl(q * fl(2 eb));
 * a bin is a prequantisation outlier (kept losslessly, q taken as 0) when b is
 * not finite, |q| >= 2^28, or |b - b^| > eb (tested in fp64).  The bound is
 * therefore |b - b^| <= eb on every bin, exactly.  An outlier stores the bits
 * of b; a NaN bin stores the one quiet NaN 0x7FC00000, since NaN payloads are
 * not portable across processors.
 * ------------------------------------------------------------------------ */
void orc_prequantize(const float* binned, uint64_t m, float abs_eb, int32_t* q_out,
                     uint8_t* outlier_out) {
  const float two_eb = 2.0f * abs_eb;
  const float recip = 1.0f / two_eb;
  for (uint64_t i = 0; i < m; ++i) {
    const float b = binned[i];
    const float t = rintf(b * recip);
    int outlier = !isfinite(b) || !(fabsf(t) < ORC_PQ_LIMIT);
    if (!outlier) {
      const float b_hat = t * two_eb;
      if (fabs((double)b - (double)b_hat) > (double)abs_eb) outlier = 1;
    }
    q_out[i] = outlier ? 0 : (int32_t)t;
    outlier_out[i] = (uint8_t)outlier;
  }
}

/* a6. 2-D Lorenzo prediction on the integers (§5.3.2; §6 "dimension" 2 = a
 * panel): delta = q[i][j] - q[i-1][j] - q[i][j-1] + q[i-1][j-1] within each
 * binned panel, neighbours outside the panel taken as 0. */
void orc_lorenzo(const int32_t* q, uint32_t n_panels, uint32_t hb, uint32_t wb,
                 int32_t* delta_out) {
  for (uint32_t pn = 0; pn < n_panels; ++pn) {
    const int32_t* qp = q + (size_t)pn * hb * wb;
    int32_t* dp = delta_out + (size_t)pn * hb * wb;
    for (uint32_t i = 0; i < hb; ++i) {
      for (uint32_t j = 0; j < wb; ++j) {
        const int64_t up = i > 0 ? qp[(size_t)(i - 1) * wb + j] : 0;
        const int64_t left = j > 0 ? qp[(size_t)i * wb + j - 1] : 0;
        const int64_t diag = (i > 0 && j > 0) ? qp[(size_t)(i - 1) * wb + j - 1] : 0;
        dp[(size_t)i * wb + j] = (int32_t)((int64_t)qp[(size_t)i * wb + j] - up - left + diag);
      }
    }
  }
}

/* a6 in the dimension §6 names as a parameter of the method ("dimension": the
 * row of pixels, the entire panel, or the stack of panels).  Reading: the SZ
 * Lorenzo predictor of that order on the binned array [n_panels][hb][wb]
 *   dims 1: the whole frame as one row-major run, delta_k = q_k - q_(k-1);
 *   dims 2: each panel on its own (orc_lorenzo);
 *   dims 3: the panels as a volume, delta = q - (the seven-neighbour 3-D
 *           Lorenzo prediction from the previous panel, row and column);
 * neighbours outside the array taken as 0. */
void orc_lorenzo_nd(const int32_t* q, uint32_t n_panels, uint32_t hb, uint32_t wb, int32_t dims,
                    int32_t* delta_out) {
  const uint64_t m = (uint64_t)n_panels * hb * wb;
  if (dims == 1) {
    for (uint64_t k = 0; k < m; ++k) {
      const int64_t prev = k > 0 ? q[k - 1] : 0;
      delta_out[k] = (int32_t)((int64_t)q[k] - prev);
    }
    return;
  }
  if (dims == 2) {
    orc_lorenzo(q, n_panels, hb, wb, delta_out);
    return;
  }
  const size_t plane = (size_t)hb * wb;
  for (uint32_t pn = 0; pn < n_panels; ++pn) {
    for (uint32_t i = 0; i < hb; ++i) {
      for (uint32_t j = 0; j < wb; ++j) {
        /* the eight corners of the unit cube ending at (pn, i, j) */
        int64_t corner[2][2][2];
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
              const int inside = (a == 0 || pn > 0) && (b == 0 || i > 0) && (c == 0 || j > 0);
              corner[a][b][c] = inside ? q[(size_t)(pn - a) * plane + (size_t)(i - b) * wb + (j - c)] : 0;
            }
        const int64_t prediction = corner[1][0][0] + corner[0][1][0] + corner[0][0][1] - corner[1][1][0] -
                                   corner[1][0][1] - corner[0][1][1] + corner[1][1][1];
        delta_out[(size_t)pn * plane + (size_t)i * wb + j] = (int32_t)(corner[0][0][0] - prediction);
      }
    }
  }
}

/* a7. Linear-quantisation codes: code = delta + R when |delta| < R, else 0
 * (a Lorenzo outlier whose delta is stored on the side). */
void orc_quant_codes(const int32_t* delta, uint64_t m, int32_t radius, uint16_t* codes_out) {
  for (uint64_t i = 0; i < m; ++i) {
    const int32_t d = delta[i];
    codes_out[i] = (d > -radius && d < radius) ? (uint16_t)(d + radius) : (uint16_t)0;
  }
}

/* a8. Per-frame histogram of the codes (one codebook per event, chunk = 1,
 * §5.3.4). */
void orc_histogram(const uint16_t* codes, uint64_t m, uint32_t n_symbols, uint64_t* hist_out) {
  memset(hist_out, 0, sizeof(uint64_t) * n_symbols);
  for (uint64_t i = 0; i < m; ++i) hist_out[codes[i]] += 1;
}

/* --------------------------------------------------------------------------
 * a9. Huffman code lengths.  Not in the paper (SZ's entropy stage); the reading
 * fixes the ties so the result is unique:
 *   - leaves = symbols with a non-zero count, sorted by (count, symbol);
 *   - two-queue construction: each merge takes the two lightest nodes among
 *     the head of the leaf queue and the head of the internal-node queue
 *     (internal nodes in creation order); on equal weight the leaf is taken;
 *   - code length = leaf depth; a lone symbol gets length 1.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint64_t f;
  uint32_t s;
} orc_leaf;

static int leaf_cmp(const void* a, const void* b) {
  const orc_leaf* x = (const orc_leaf*)a;
  const orc_leaf* y = (const orc_leaf*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);
}

int orc_huffman_lengths(const uint64_t* hist, uint32_t n_symbols, uint8_t* len_out) {
  memset(len_out, 0, n_symbols);
  orc_leaf* leaves = (orc_leaf*)malloc(sizeof(orc_leaf) * (n_symbols + 1));
  uint32_t n = 0;
  for (uint32_t s = 0; s < n_symbols; ++s)
    if (hist[s] > 0) {
      leaves[n].f = hist[s];
      leaves[n].s = s;
      ++n;
    }
  if (n == 0) {
    free(leaves);
    return ORC_OK;
  }
  if (n == 1) {
    len_out[leaves[0].s] = 1;
    free(leaves);
    return ORC_OK;
  }
  qsort(leaves, n, sizeof(orc_leaf), leaf_cmp);

  /* nodes 0..n-1 are the sorted leaves, n..2n-2 the internal nodes */
  const uint32_t total = 2 * n - 1;
  uint64_t* weight = (uint64_t*)malloc(sizeof(uint64_t) * total);
  uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * total);
  uint32_t* depth = (uint32_t*)malloc(sizeof(uint32_t) * total);
  for (uint32_t i = 0; i < n; ++i) weight[i] = leaves[i].f;

  uint32_t next_leaf = 0, next_internal = n, created = n;
  for (uint32_t k = 0; k + 1 < n; ++k) {
    uint32_t pick[2];
    for (int t = 0; t < 2; ++t) {
      const int leaf_left = next_leaf < n;
      const int internal_left = next_internal < created;
      if (leaf_left && (!internal_left || weight[next_leaf] <= weight[next_internal]))
        pick[t] = next_leaf++;
      else
        pick[t] = next_internal++;
    }
    weight[created] = weight[pick[0]] + weight[pick[1]];
    parent[pick[0]] = created;
    parent[pick[1]] = created;
    ++created;
  }
  /* the root is the last node created; parents always have larger indices */
  depth[total - 1] = 0;
  for (int64_t i = (int64_t)total - 2; i >= 0; --i) depth[i] = depth[parent[i]] + 1;

  int status = ORC_OK;
  for (uint32_t i = 0; i < n; ++i) {
    if (depth[i] > 32) status = ORC_ERR_CODE_LENGTH;
    len_out[leaves[i].s] = (uint8_t)(depth[i] > 255 ? 255 : depth[i]);
  }
  free(weight);
  free(parent);
  free(depth);
  free(leaves);
  return status;
}

/* Canonical codes: symbols ordered by (length, symbol); the first gets the
 * all-zero code of its length; each next code is (previous + 1) shifted left by
 * the growth in length.  Absent symbols get code 0. */
void orc_canonical_codes(const uint8_t* len, uint32_t n_symbols, uint32_t* code_out) {
  memset(code_out, 0, sizeof(uint32_t) * n_symbols);
  uint64_t code = 0;
  int prev_len = 0, first = 1;
  for (int L = 1; L <= 32; ++L) {
    for (uint32_t s = 0; s < n_symbols; ++s) {
      if (len[s] != L) continue;
      if (first) {
        code = 0;
        first = 0;
      } else {
        code = (code + 1) << (L - prev_len);
      }
      code_out[s] = (uint32_t)code;
      prev_len = L;
    }
  }
}

/* --------------------------------------------------------------------------
 * a10. Bit-packing.  The code stream is cut into chunks of 4096 symbols; each
 * chunk starts on a 32-bit word boundary.  Inside a chunk, the codeword of each
 * symbol is appended most-significant bit first; stream bit b of a chunk is bit
 * (31 - b mod 32) of its word b / 32.  chunk_index_out[k] is the word offset of
 * chunk k.  Returns the total number of words.
 * ------------------------------------------------------------------------ */
uint32_t orc_pack_chunks(const uint16_t* codes, uint64_t m, const uint8_t* len,
                         const uint32_t* codewords, uint32_t* chunk_index_out,
                         uint32_t* words_out) {
  const uint64_t n_chunks = (m + ORC_CHUNK_SYMBOLS - 1) / ORC_CHUNK_SYMBOLS;
  uint32_t word_base = 0;
  for (uint64_t k = 0; k < n_chunks; ++k) {
    chunk_index_out[k] = word_base;
    const uint64_t lo = k * ORC_CHUNK_SYMBOLS;
    const uint64_t hi = (lo + ORC_CHUNK_SYMBOLS < m) ? lo + ORC_CHUNK_SYMBOLS : m;
    uint64_t bit = 0;
    for (uint64_t i = lo; i < hi; ++i) {
      const int L = len[codes[i]];
      const uint32_t cw = codewords[codes[i]];
      for (int b = L - 1; b >= 0; --b) {
        const uint32_t w = word_base + (uint32_t)(bit / 32);
        if (bit % 32 == 0) words_out[w] = 0;
        if ((cw >> b) & 1u) words_out[w] |= 1u << (31 - bit % 32);
        ++bit;
      }
    }
    word_base += (uint32_t)((bit + 31) / 32);
  }
  return word_base;
}

/* --------------------------------------------------------------------------
 * ROI coding (§4: the paper stores each region of interest losslessly with
 * fpzip, a predictive coder for floating-point data).  The coder here is our
 * own of that kind; it changes how the ROI windows are stored, never their
 * values (they come back bit for bit).  For each window, in row-major order:
 *   1. the float's bits u become an integer in the float's own order:
 *      m = u + 2^31 when the sign bit is 0, m = NOT u when it is 1;
 *   2. m is predicted modulo 2^32 by the 2-D Lorenzo rule inside the window,
 *      m[i-1][j] + m[i][j-1] - m[i-1][j-1], positions outside the window
 *      taken as 0, except the window's first value, predicted by 2^31 (+0.0);
 *   3. the residual r = m - prediction (mod 2^32, as int32) is folded to
 *      z = 2r for r >= 0 and -2r - 1 for r < 0;
 *   4. z is written as its class c (its bit length: 0 for z = 0, else 1..32),
 *      Huffman-coded over the 33 classes with one codebook per frame (the
 *      lengths and canonical codes of a9 and a10's bit order), followed by the
 *      c - 1 bits of z below its leading one, most significant first.
 * A window's bits start on a 32-bit word boundary.  Section layout:
 *   [0, 48)          u8 code length of each class (33), zero padded;
 *   [48, 48 + A)     u32 first word of each window, A = align16(4 n_windows);
 *   then             u32 words, padded to 16 bytes.
 * When that section would not be smaller than the raw windows, the raw float32
 * windows are stored instead (coding 2); the coded form is coding 1.
 * ------------------------------------------------------------------------ */
#define ORC_ROI_CLASSES 33u
#define ORC_ROI_HEAD 48u

uint32_t orc_roi_order_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

static float roi_float_of(uint32_t m) {
  const uint32_t u = (m & 0x80000000u) ? (m & 0x7FFFFFFFu) : ~m;
  float x;
  memcpy(&x, &u, 4);
  return x;
}

/* Steps 1-3 for one window: z_out[i * w + j]. */
void orc_roi_residuals(const float* win, int32_t h, int32_t w, uint32_t* z_out) {
  for (long i = 0; i < h; ++i) {
    for (long j = 0; j < w; ++j) {
      const uint32_t m = orc_roi_order_bits(win[i * w + j]);
      uint32_t pred;
      if (i == 0 && j == 0) {
        pred = 0x80000000u;
      } else {
        const uint32_t up = i > 0 ? orc_roi_order_bits(win[(i - 1) * w + j]) : 0u;
        const uint32_t left = j > 0 ? orc_roi_order_bits(win[i * w + j - 1]) : 0u;
        const uint32_t diag = (i > 0 && j > 0) ? orc_roi_order_bits(win[(i - 1) * w + j - 1]) : 0u;
        pred = up + left - diag;
      }
      const int32_t r = (int32_t)(m - pred);
      z_out[i * w + j] = r >= 0 ? 2u * (uint32_t)r : 2u * (uint32_t)(-(int64_t)r) - 1u;
    }
  }
}

uint32_t orc_roi_class(uint32_t z) {
  uint32_t c = 0;
  while (z) {
    ++c;
    z >>= 1;
  }
  return c;
}

static uint64_t roi_coded_bytes(uint32_t n_windows, uint32_t n_words) {
  return ORC_ROI_HEAD + align16((uint64_t)n_windows * 4) + align16((uint64_t)n_words * 4);
}

/* Writes the ROI section of n_windows windows (f32[n][h][w]) into out (at
 * least n * h * w * 4 + 64 bytes).  *coding is 1 (coded) or 2 (raw), *n_words
 * the coded section's words (0 for raw); returns the section's bytes. */
uint64_t orc_roi_encode(const float* windows, uint32_t n_windows, int32_t h, int32_t w, uint8_t* out,
                        uint32_t* coding, uint32_t* n_words) {
  const size_t win = (size_t)h * (size_t)w;
  const uint64_t raw = align16((uint64_t)n_windows * win * 4);
  uint32_t* z = (uint32_t*)malloc(sizeof(uint32_t) * (win * n_windows + 1));
  uint64_t hist[ORC_ROI_CLASSES];
  memset(hist, 0, sizeof(hist));
  for (uint32_t k = 0; k < n_windows; ++k) orc_roi_residuals(windows + k * win, h, w, z + k * win);
  for (size_t i = 0; i < win * n_windows; ++i) hist[orc_roi_class(z[i])] += 1;
  uint8_t len[ORC_ROI_CLASSES];
  uint32_t cw[ORC_ROI_CLASSES];
  orc_huffman_lengths(hist, ORC_ROI_CLASSES, len); /* 33 leaves: every length <= 32 */
  orc_canonical_codes(len, ORC_ROI_CLASSES, cw);
  /* sizes first: bits of each window, then the word count */
  uint64_t words = 0;
  for (uint32_t k = 0; k < n_windows; ++k) {
    uint64_t bits = 0;
    for (size_t i = 0; i < win; ++i) {
      const uint32_t c = orc_roi_class(z[k * win + i]);
      bits += len[c] + (c > 1 ? c - 1 : 0);
    }
    words += (bits + 31) / 32;
  }
  if (n_windows == 0 || roi_coded_bytes(n_windows, (uint32_t)words) >= raw) {
    memcpy(out, windows, (size_t)n_windows * win * 4);
    memset(out + (size_t)n_windows * win * 4, 0, raw - (size_t)n_windows * win * 4);
    *coding = 2;
    *n_words = 0;
    free(z);
    return raw;
  }
  const uint64_t total = roi_coded_bytes(n_windows, (uint32_t)words);
  memset(out, 0, total);
  memcpy(out, len, ORC_ROI_CLASSES);
  uint8_t* offs = out + ORC_ROI_HEAD;
  uint8_t* wbytes = offs + align16((uint64_t)n_windows * 4);
  uint64_t word0 = 0;
  for (uint32_t k = 0; k < n_windows; ++k) {
    const uint32_t o = (uint32_t)word0;
    memcpy(offs + 4 * k, &o, 4);
    uint64_t bit = 0;
    /* one bit at a time, most significant first: stream bit b of the window is
     * bit 31 - b % 32 of its word b / 32 */
    for (size_t i = 0; i < win; ++i) {
      const uint32_t zz = z[k * win + i], c = orc_roi_class(zz);
      for (int b = len[c] - 1; b >= 0; --b, ++bit)
        if ((cw[c] >> b) & 1u) {
          uint32_t v;
          memcpy(&v, wbytes + 4 * (word0 + bit / 32), 4);
          v |= 1u << (31 - bit % 32);
          memcpy(wbytes + 4 * (word0 + bit / 32), &v, 4);
        }
      for (int b = (int)c - 2; b >= 0; --b, ++bit)
        if ((zz >> b) & 1u) {
          uint32_t v;
          memcpy(&v, wbytes + 4 * (word0 + bit / 32), 4);
          v |= 1u << (31 - bit % 32);
          memcpy(wbytes + 4 * (word0 + bit / 32), &v, 4);
        }
    }
    word0 += (bit + 31) / 32;
  }
  *coding = 1;
  *n_words = (uint32_t)words;
  free(z);
  return total;
}

/* Inverse of orc_roi_encode.  A section whose size, code lengths, window
 * offsets or bits do not fit together gives ORC_ERR_CORRUPT_STREAM. */
int orc_roi_decode(const uint8_t* sec, uint64_t bytes, uint32_t coding, uint32_t n_words, uint32_t n_windows,
                   int32_t h, int32_t w, float* windows_out) {
  const size_t win = (size_t)h * (size_t)w;
  if (coding == 2) {
    if (n_words != 0 || bytes != align16((uint64_t)n_windows * win * 4)) return ORC_ERR_CORRUPT_STREAM;
    memcpy(windows_out, sec, (size_t)n_windows * win * 4);
    return ORC_OK;
  }
  if (coding != 1 || n_windows == 0 || bytes != roi_coded_bytes(n_windows, n_words)) return ORC_ERR_CORRUPT_STREAM;
  const uint8_t* len = sec;
  uint32_t count[34] = {0};
  uint64_t kraft = 0;
  uint32_t present = 0;
  for (uint32_t c = 0; c < ORC_ROI_CLASSES; ++c) {
    if (len[c] > 32) return ORC_ERR_CORRUPT_STREAM;
    if (len[c]) {
      count[len[c]]++;
      kraft += 1ull << (32 - len[c]);
      ++present;
    }
  }
  /* a complete code, or one class alone with length 1 */
  if (!(kraft == (1ull << 32) || (present == 1 && count[1] == 1))) return ORC_ERR_CORRUPT_STREAM;
  uint32_t first_code[34], first_index[34], sorted[ORC_ROI_CLASSES], n_sorted = 0;
  {
    uint64_t c = 0;
    int prev = 0;
    for (int L = 1; L <= 32; ++L) {
      first_index[L] = n_sorted;
      first_code[L] = 0;
      for (uint32_t s = 0; s < ORC_ROI_CLASSES; ++s)
        if (len[s] == L) sorted[n_sorted++] = s;
      if (count[L] == 0) continue;
      c = (prev == 0) ? 0 : (c + count[prev]) << (L - prev);
      first_code[L] = (uint32_t)c;
      prev = L;
    }
  }
  const uint8_t* offs = sec + ORC_ROI_HEAD;
  const uint8_t* wbytes = offs + align16((uint64_t)n_windows * 4);
  uint32_t* z = (uint32_t*)malloc(sizeof(uint32_t) * win);
  int status = ORC_OK;
  for (uint32_t k = 0; k < n_windows && status == ORC_OK; ++k) {
    uint32_t w0, w1;
    memcpy(&w0, offs + 4 * k, 4);
    if (k + 1 < n_windows) memcpy(&w1, offs + 4 * (k + 1), 4);
    else w1 = n_words;
    if ((k == 0 && w0 != 0) || w0 > w1 || w1 > n_words) {
      status = ORC_ERR_CORRUPT_STREAM;
      break;
    }
    const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
    uint64_t bit = 0;
#define ROI_NEXT_BIT(dst)                                                   \
  do {                                                                      \
    if (bit >= bit_end) {                                                   \
      status = ORC_ERR_CORRUPT_STREAM;                                      \
      break;                                                                \
    }                                                                       \
    uint32_t v_;                                                            \
    memcpy(&v_, wbytes + 4 * ((uint64_t)w0 + bit / 32), 4);                 \
    dst = (v_ >> (31 - bit % 32)) & 1u;                                     \
    ++bit;                                                                  \
  } while (0)
    for (size_t i = 0; i < win && status == ORC_OK; ++i) {
      uint64_t code = 0;
      int cls = -1;
      for (int L = 1; L <= 32 && status == ORC_OK; ++L) {
        uint32_t b;
        ROI_NEXT_BIT(b);
        if (status != ORC_OK) break;
        code = (code << 1) | b;
        if (count[L] && code >= first_code[L] && code - first_code[L] < count[L]) {
          cls = (int)sorted[first_index[L] + (code - first_code[L])];
          break;
        }
      }
      if (status != ORC_OK) break;
      if (cls < 0) {
        status = ORC_ERR_CORRUPT_STREAM;
        break;
      }
      uint32_t zz = cls == 0 ? 0u : 1u;
      for (int t = 0; t < cls - 1 && status == ORC_OK; ++t) {
        uint32_t b;
        ROI_NEXT_BIT(b);
        zz = (zz << 1) | b;
      }
      z[i] = zz;
    }
#undef ROI_NEXT_BIT
    if (status == ORC_OK && (bit + 31) / 32 != (uint64_t)(w1 - w0)) status = ORC_ERR_CORRUPT_STREAM;
    if (status != ORC_OK) break;
    /* the inverse of steps 3, 2 and 1, in the window's row-major order */
    uint32_t* m = (uint32_t*)malloc(sizeof(uint32_t) * win);
    for (long i = 0; i < h; ++i)
      for (long j = 0; j < w; ++j) {
        const uint32_t zz = z[i * w + j];
        const uint32_t r = (zz & 1u) ? ~(zz >> 1) : (zz >> 1);
        uint32_t pred;
        if (i == 0 && j == 0) {
          pred = 2147483648u; /* m(+0.0) */
        } else {
          const uint32_t above = i > 0 ? m[(i - 1) * w + j] : 0u;
          const uint32_t before = j > 0 ? m[i * w + j - 1] : 0u;
          const uint32_t corner = (i > 0 && j > 0) ? m[(i - 1) * w + j - 1] : 0u;
          pred = before + above - corner;
        }
        m[i * w + j] = r + pred;
        windows_out[k * win + (size_t)i * w + (size_t)j] = roi_float_of(m[i * w + j]);
      }
    free(m);
  }
  free(z);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Container, format version 1 (ours: the paper defines none).               */
/* ------------------------------------------------------------------------ */
static void put_u16(uint8_t* p, uint16_t v) { memcpy(p, &v, 2); }
static void put_u32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void put_u64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static uint16_t get_u16(const uint8_t* p) { uint16_t v; memcpy(&v, p, 2); return v; }
static uint32_t get_u32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t get_u64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

typedef struct {
  uint64_t peaks, roi, lengths, chunk_index, lorenzo, prequant, bitstream, total;
} orc_layout;

/* roi_in_place: the raw windows sit in the ROI section (ROI coding 0); with
 * the ROI coder they move to their own section after the bitstream, and the
 * ROI section is empty. */
static orc_layout layout_of(uint32_t n_peaks, const orc_params* p, uint32_t n_symbols,
                            uint32_t n_chunks, uint32_t n_lo, uint32_t n_pq, uint32_t words,
                            int roi_in_place, int lengths_here) {
  orc_layout L;
  L.peaks = ORC_HEADER_BYTES;
  L.roi = L.peaks + align16((uint64_t)n_peaks * 6);
  L.lengths = L.roi + (roi_in_place ? align16((uint64_t)n_peaks * p->roi_h * p->roi_w * 4) : 0);
  L.chunk_index = L.lengths + (lengths_here ? align16(n_symbols) : 0);
  L.lorenzo = L.chunk_index + align16((uint64_t)n_chunks * 4);
  L.prequant = L.lorenzo + align16((uint64_t)n_lo * 8);
  L.bitstream = L.prequant + align16((uint64_t)n_pq * 8);
  L.total = L.bitstream + align16((uint64_t)words * 4);
  return L;
}

static int params_valid(const orc_geometry* g, const orc_params* p) {
  if (g->n_panels < 1 || g->rows < 1 || g->cols < 1) return 0;
  if (g->n_panels > 65535 || g->rows > 65535 || g->cols > 65535) return 0;
  if (p->bin_h < 1 || p->bin_w < 1 || p->bin_h > 8 || p->bin_w > 8) return 0;
  if (p->roi_h < 1 || p->roi_w < 1 || p->roi_h > 63 || p->roi_w > 63) return 0;
  if (p->rank < 1 || p->rank > 7) return 0;
  if (p->ring_r0 < 1 || p->ring_dr < 1 || p->ring_r0 + p->ring_dr > 16) return 0;
  if (p->quant_radius < 2 || p->quant_radius > 512) return 0;
  if (p->max_peaks < 0 || p->max_peaks > 65535) return 0;
  if (p->lorenzo_dims < 1 || p->lorenzo_dims > 3) return 0;
  if (p->nhr_min_peaks < 0 || p->nhr_min_peaks > 8192) return 0;
  if (p->roi_coder < 0 || p->roi_coder > 1) return 0;
  if (p->chunk_frames < 1 || p->chunk_frames > 64) return 0;
  if (!(p->pix_nsigma >= 0.0f)) return 0;
  if (!(p->abs_eb > 0.0f) || !isfinite(2.0f * p->abs_eb) || !isfinite(1.0f / (2.0f * p->abs_eb)))
    return 0;
  const uint64_t hb = (g->rows + p->bin_h - 1) / p->bin_h, wb = (g->cols + p->bin_w - 1) / p->bin_w;
  if ((uint64_t)g->n_panels * hb * wb > ORC_MAX_SYMBOLS_PER_FRAME) return 0;
  return 1;
}

uint64_t orc_compress_bound(const orc_geometry* g, const orc_params* p) {
  if (!params_valid(g, p)) return 0;
  const uint64_t hb = (g->rows + p->bin_h - 1) / p->bin_h, wb = (g->cols + p->bin_w - 1) / p->bin_w;
  const uint64_t m = (uint64_t)g->n_panels * hb * wb;
  const uint64_t n_chunks = (m + ORC_CHUNK_SYMBOLS - 1) / ORC_CHUNK_SYMBOLS;
  /* every symbol at most 32 bits: at most m words, plus nothing else.  The
   * ROI coder never stores more than the raw windows (it falls back to them),
   * so the same bound holds for both ROI codings. */
  const orc_layout L = layout_of((uint32_t)p->max_peaks, p, 2u * (uint32_t)p->quant_radius,
                                 (uint32_t)n_chunks, (uint32_t)m, (uint32_t)m, (uint32_t)m, 1, 1);
  return L.total;
}

/* One frame's work up to its histogram (a1-a8).  A frame is "coded" when its
 * status is still ORC_OK here; only coded frames feed a chunk's codebook. */
typedef struct {
  int status;
  uint16_t* peaks;
  uint32_t n_peaks;
  float* binned;
  uint8_t* pq;
  int32_t* delta;
  uint16_t* codes;
  uint64_t* hist;
} orc_frame_work;

static void work_free(orc_frame_work* w) {
  free(w->peaks);
  free(w->binned);
  free(w->pq);
  free(w->delta);
  free(w->codes);
  free(w->hist);
  memset(w, 0, sizeof(*w));
}

/* a1-a8 for one frame.  user_peaks != NULL and n_user_peaks >= 0 replaces the
 * peak finder by a caller-supplied coordinate list (§4.2 allows the regions of
 * interest to be given as coordinates), kept in the order given.
 * Non-hit rejection (§1, §4: frames with too few peaks to index are dropped
 * before compression): with nhr_min_peaks > 0, a frame whose peak list has
 * fewer entries is not compressed and gets ORC_REJECTED.  Off (0) by default. */
static void frame_analyse(const float* frame, const orc_geometry* g, const orc_params* p, const uint16_t* user_peaks,
                          int64_t n_user_peaks, orc_frame_work* w) {
  memset(w, 0, sizeof(*w));
  const uint32_t hb = (g->rows + p->bin_h - 1) / p->bin_h, wb = (g->cols + p->bin_w - 1) / p->bin_w;
  const uint64_t m = (uint64_t)g->n_panels * hb * wb;
  const uint32_t n_symbols = 2u * (uint32_t)p->quant_radius;

  /* peaks */
  uint16_t* peaks = (uint16_t*)malloc(sizeof(uint16_t) * 3 * ((size_t)p->max_peaks + 1));
  w->peaks = peaks;
  uint32_t n_peaks = 0;
  if (user_peaks != NULL && n_user_peaks >= 0) {
    if (n_user_peaks > p->max_peaks) {
      w->status = ORC_ERR_CAPACITY;
      return;
    }
    for (int64_t k = 0; k < n_user_peaks; ++k) {
      if (user_peaks[3 * k] >= g->n_panels || user_peaks[3 * k + 1] >= g->rows ||
          user_peaks[3 * k + 2] >= g->cols) {
        w->status = ORC_ERR_INVALID_ARG;
        return;
      }
      memcpy(peaks + 3 * k, user_peaks + 3 * k, 6);
    }
    n_peaks = (uint32_t)n_user_peaks;
  } else {
    const int st = orc_find_peaks(frame, g, p, peaks, (uint32_t)p->max_peaks, &n_peaks);
    if (st != ORC_OK) {
      w->status = st;
      return;
    }
  }
  if ((int64_t)n_peaks < (int64_t)p->nhr_min_peaks) {
    w->status = ORC_REJECTED;
    return;
  }
  w->n_peaks = n_peaks;

  /* background path: bin -> prequantise -> Lorenzo -> codes -> histogram */
  float* binned = (float*)malloc(sizeof(float) * m);
  int32_t* q = (int32_t*)malloc(sizeof(int32_t) * m);
  uint8_t* pq = (uint8_t*)malloc(m);
  int32_t* delta = (int32_t*)malloc(sizeof(int32_t) * m);
  uint16_t* codes = (uint16_t*)malloc(sizeof(uint16_t) * m);
  uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * n_symbols);
  orc_bin(frame, g, p->bin_h, p->bin_w, binned);
  orc_prequantize(binned, m, p->abs_eb, q, pq);
  orc_lorenzo_nd(q, g->n_panels, hb, wb, p->lorenzo_dims, delta);
  orc_quant_codes(delta, m, p->quant_radius, codes);
  orc_histogram(codes, m, n_symbols, hist);
  free(q);
  w->binned = binned;
  w->pq = pq;
  w->delta = delta;
  w->codes = codes;
  w->hist = hist;
  w->status = ORC_OK;
}

/* a10-a12 for one coded frame with the codebook `len` (status cb_status from
 * a9).  back_ref = 0: the stream carries the code lengths; back_ref = b > 0:
 * the lengths live in the stream b frames earlier in the same call (the head
 * of its chunk), and this stream has none. */
static int frame_assemble(const float* frame, const orc_geometry* g, const orc_params* p, const orc_frame_work* w,
                          const uint8_t* len, int cb_status, uint32_t back_ref, uint8_t* out, uint64_t capacity,
                          uint64_t* out_bytes) {
  *out_bytes = 0;
  const uint32_t hb = (g->rows + p->bin_h - 1) / p->bin_h, wb = (g->cols + p->bin_w - 1) / p->bin_w;
  const uint64_t m = (uint64_t)g->n_panels * hb * wb;
  const uint32_t n_symbols = 2u * (uint32_t)p->quant_radius;
  const uint32_t n_chunks = (uint32_t)((m + ORC_CHUNK_SYMBOLS - 1) / ORC_CHUNK_SYMBOLS);
  const uint16_t* peaks = w->peaks;
  const uint32_t n_peaks = w->n_peaks;
  const float* binned = w->binned;
  const uint8_t* pq = w->pq;
  const int32_t* delta = w->delta;
  const uint16_t* codes = w->codes;
  uint32_t* cw = (uint32_t*)malloc(sizeof(uint32_t) * n_symbols);
  uint32_t* chunk_index = (uint32_t*)malloc(sizeof(uint32_t) * n_chunks);
  uint32_t* words = (uint32_t*)malloc(sizeof(uint32_t) * (m + 1));
  int status = cb_status;
  uint32_t n_words = 0;
  if (status == ORC_OK) {
    orc_canonical_codes(len, n_symbols, cw);
    n_words = orc_pack_chunks(codes, m, len, cw, chunk_index, words);
  }

  /* a11. outliers, in bin-index order */
  uint32_t n_lo = 0, n_pq = 0;
  for (uint64_t i = 0; i < m; ++i) {
    n_lo += codes[i] == 0;
    n_pq += pq[i] != 0;
  }
  const orc_layout L =
      layout_of(n_peaks, p, n_symbols, n_chunks, n_lo, n_pq, n_words, p->roi_coder == 0, back_ref == 0);
  /* the ROI windows, and with the coder their section after the bitstream */
  const size_t win = (size_t)p->roi_h * p->roi_w;
  float* roi = (float*)malloc(sizeof(float) * (win * n_peaks + 1));
  orc_roi_extract(frame, g, p, peaks, n_peaks, roi);
  uint8_t* roi_sec = NULL;
  uint64_t roi_bytes = 0;
  uint32_t roi_coding = 0, roi_words = 0;
  if (p->roi_coder == 1) {
    roi_sec = (uint8_t*)malloc(win * n_peaks * 4 + 64);
    roi_bytes = orc_roi_encode(roi, n_peaks, p->roi_h, p->roi_w, roi_sec, &roi_coding, &roi_words);
  }
  const uint64_t total = L.total + roi_bytes;
  if (status == ORC_OK) {
    *out_bytes = total;
    if (total > capacity) status = ORC_ERR_CAPACITY;
  }
  if (status == ORC_OK) {
    memset(out, 0, total);
    put_u32(out + 0, ORC_MAGIC);
    put_u32(out + 4, ORC_VERSION);
    put_u32(out + 8, g->n_panels);
    put_u32(out + 12, g->rows);
    put_u32(out + 16, g->cols);
    put_u16(out + 20, (uint16_t)p->roi_h);
    put_u16(out + 22, (uint16_t)p->roi_w);
    put_u16(out + 24, (uint16_t)p->bin_h);
    put_u16(out + 26, (uint16_t)p->bin_w);
    memcpy(out + 28, &p->abs_eb, 4);
    put_u32(out + 32, (uint32_t)p->quant_radius);
    put_u32(out + 36, n_peaks);
    put_u32(out + 40, n_lo);
    put_u32(out + 44, n_pq);
    put_u32(out + 48, (uint32_t)m);
    put_u32(out + 52, ORC_CHUNK_SYMBOLS);
    put_u32(out + 56, n_chunks);
    put_u32(out + 60, n_words);
    put_u64(out + 64, total);
    /* Lorenzo dimension: 0 stands for the default 2, so that 2-D streams keep
     * the 24 zero bytes that end the header */
    put_u32(out + 72, p->lorenzo_dims == 2 ? 0u : (uint32_t)p->lorenzo_dims);
    /* ROI coding (0: raw windows in the ROI section; 1: coded, 2: raw, in a
     * section after the bitstream), that section's bytes and coded words */
    put_u32(out + 76, roi_coding);
    put_u32(out + 80, (uint32_t)roi_bytes);
    put_u32(out + 84, roi_words);
    /* where the code lengths are: 0 here, b in the stream b frames earlier */
    put_u32(out + 88, back_ref);

    for (uint32_t k = 0; k < n_peaks; ++k)
      for (int t = 0; t < 3; ++t) put_u16(out + L.peaks + 6 * k + 2 * t, peaks[3 * k + t]);
    if (p->roi_coder == 0) memcpy(out + L.roi, roi, win * n_peaks * 4);
    else memcpy(out + L.total, roi_sec, roi_bytes);
    if (back_ref == 0) memcpy(out + L.lengths, len, n_symbols);
    for (uint32_t k = 0; k < n_chunks; ++k) put_u32(out + L.chunk_index + 4 * k, chunk_index[k]);
    uint32_t a = 0, b = 0;
    for (uint64_t i = 0; i < m; ++i) {
      if (codes[i] == 0) {
        put_u32(out + L.lorenzo + 8 * a, (uint32_t)i);
        put_u32(out + L.lorenzo + 8 * a + 4, (uint32_t)delta[i]);
        ++a;
      }
      if (pq[i]) {
        uint32_t bits;
        memcpy(&bits, &binned[i], 4);
        if (isnan(binned[i])) bits = ORC_CANONICAL_NAN;
        put_u32(out + L.prequant + 8 * b, (uint32_t)i);
        put_u32(out + L.prequant + 8 * b + 4, bits);
        ++b;
      }
    }
    for (uint32_t w2 = 0; w2 < n_words; ++w2) put_u32(out + L.bitstream + 4 * w2, words[w2]);
  }

  free(roi_sec);
  free(roi);
  free(words);
  free(chunk_index);
  free(cw);
  return status;
}

/* a9 + a12 over a call of n_frames frames (frames[f] at f * frame_px).  Chunks
 * (§5.3.4: a compressor call takes 1-64 events) are the frames f with the same
 * f / chunk_frames.  A chunk's coded frames share one Huffman codebook, built
 * from the sum of their histograms; the first coded frame of the chunk (its
 * head) stores the code lengths, and each later one records how many frames
 * back its head is.  chunk_frames = 1 gives each frame its own codebook.
 *   user_peaks   NULL, or u16[n_frames][max_peaks][3] with n_user_peaks[f]
 *                entries for frame f (n_user_peaks[f] < 0: the finder runs);
 *   outs         n_frames slots of `stride` bytes; out_bytes[f] the stream's
 *                size (on ORC_ERR_CAPACITY the size it needs), status[f] its
 *                outcome (ORC_OK, ORC_REJECTED or an error). */
int orc_compress_frames(const float* frames, uint32_t n_frames, const orc_geometry* g, const orc_params* p,
                        const uint16_t* user_peaks, const int64_t* n_user_peaks, uint8_t* outs, uint64_t stride,
                        uint64_t* out_bytes, int32_t* status) {
  for (uint32_t f = 0; f < n_frames; ++f) {
    out_bytes[f] = 0;
    status[f] = ORC_ERR_INVALID_ARG;
  }
  if (!params_valid(g, p)) return ORC_ERR_INVALID_ARG;
  const size_t frame_px = (size_t)g->n_panels * g->rows * g->cols;
  const uint32_t n_symbols = 2u * (uint32_t)p->quant_radius;
  const uint32_t C = (uint32_t)p->chunk_frames;
  orc_frame_work* w = (orc_frame_work*)calloc(n_frames + 1, sizeof(orc_frame_work));
  for (uint32_t f = 0; f < n_frames; ++f) {
    const uint16_t* up = user_peaks ? user_peaks + (size_t)f * (size_t)p->max_peaks * 3 : NULL;
    const int64_t nu = user_peaks ? n_user_peaks[f] : -1;
    frame_analyse(frames + f * frame_px, g, p, up, nu, &w[f]);
    status[f] = w[f].status;
  }
  uint64_t* hsum = (uint64_t*)malloc(sizeof(uint64_t) * n_symbols);
  uint8_t* len = (uint8_t*)malloc(n_symbols);
  for (uint32_t c0 = 0; c0 < n_frames; c0 += C) {
    const uint32_t c1 = c0 + C < n_frames ? c0 + C : n_frames;
    /* a9 once per chunk: the Huffman code of the chunk's summed histogram */
    memset(hsum, 0, sizeof(uint64_t) * n_symbols);
    int64_t head = -1;
    for (uint32_t f = c0; f < c1; ++f) {
      if (w[f].status != ORC_OK) continue;
      if (head < 0) head = f;
      for (uint32_t s2 = 0; s2 < n_symbols; ++s2) hsum[s2] += w[f].hist[s2];
    }
    if (head < 0) continue;
    const int cb = orc_huffman_lengths(hsum, n_symbols, len);
    for (uint32_t f = c0; f < c1; ++f) {
      if (w[f].status != ORC_OK) continue;
      status[f] = frame_assemble(frames + f * frame_px, g, p, &w[f], len, cb, f - (uint32_t)head,
                                 outs + f * stride, stride, &out_bytes[f]);
    }
  }
  for (uint32_t f = 0; f < n_frames; ++f) work_free(&w[f]);
  free(w);
  free(hsum);
  free(len);
  return ORC_OK;
}

/* a12. One frame on its own: a call of one frame (its own codebook). */
int orc_compress_frame(const float* frame, const orc_geometry* g, const orc_params* p,
                       const uint16_t* user_peaks, int64_t n_user_peaks, uint8_t* out,
                       uint64_t capacity, uint64_t* out_bytes) {
  *out_bytes = 0;
  if (!params_valid(g, p)) return ORC_ERR_INVALID_ARG;
  orc_frame_work w;
  frame_analyse(frame, g, p, user_peaks, user_peaks ? n_user_peaks : -1, &w);
  int status = w.status;
  if (status == ORC_OK) {
    const uint32_t n_symbols = 2u * (uint32_t)p->quant_radius;
    uint8_t* len = (uint8_t*)malloc(n_symbols);
    const int cb = orc_huffman_lengths(w.hist, n_symbols, len);
    status = frame_assemble(frame, g, p, &w, len, cb, 0, out, capacity, out_bytes);
    free(len);
  }
  work_free(&w);
  return status;
}

/* --------------------------------------------------------------------------
 * a13. Decompression (§4.1: restoration of the ROIs over the up-sampled
 * background).  decode -> delta -> 2-D prefix sum -> q -> b^ = fl(q * 2eb) ->
 * prequantisation outliers overwrite b^ -> every pixel of a bin takes b^ ->
 * every in-panel ROI position takes its stored value.
 * ------------------------------------------------------------------------ */
/* The fields of a stream's header, checked against the geometry and each
 * other, and the stream's layout. */
typedef struct {
  orc_params p;
  uint32_t n_peaks, n_lo, n_pq, n_chunks, n_words, roi_coding, roi_bytes, roi_words, back_ref;
  int dims;
  uint64_t m, total;
  orc_layout L;
} orc_header;

static int read_header(const uint8_t* in, uint64_t in_bytes, const orc_geometry* g, orc_header* h) {
  memset(h, 0, sizeof(*h));
  if (in_bytes < ORC_HEADER_BYTES) return ORC_ERR_CORRUPT_STREAM;
  if (get_u32(in) != ORC_MAGIC || get_u32(in + 4) != ORC_VERSION) return ORC_ERR_CORRUPT_STREAM;
  if (get_u32(in + 8) != g->n_panels || get_u32(in + 12) != g->rows || get_u32(in + 16) != g->cols)
    return ORC_ERR_INVALID_ARG;
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.roi_h = get_u16(in + 20);
  p.roi_w = get_u16(in + 22);
  p.bin_h = get_u16(in + 24);
  p.bin_w = get_u16(in + 26);
  memcpy(&p.abs_eb, in + 28, 4);
  p.quant_radius = (int32_t)get_u32(in + 32);
  const uint32_t n_peaks = get_u32(in + 36), n_lo = get_u32(in + 40), n_pq = get_u32(in + 44);
  const uint32_t m_hdr = get_u32(in + 48), chunk = get_u32(in + 52), n_chunks = get_u32(in + 56);
  const uint32_t n_words = get_u32(in + 60);
  const uint64_t total = get_u64(in + 64);
  const uint32_t dims_code = get_u32(in + 72);
  if (dims_code != 0 && dims_code != 1 && dims_code != 3) return ORC_ERR_CORRUPT_STREAM;
  const uint32_t roi_coding = get_u32(in + 76), roi_bytes = get_u32(in + 80), roi_words = get_u32(in + 84);
  if (roi_coding > 2 || (roi_coding == 0 && (roi_bytes | roi_words) != 0)) return ORC_ERR_CORRUPT_STREAM;
  const uint32_t back_ref = get_u32(in + 88);
  if (back_ref > 63) return ORC_ERR_CORRUPT_STREAM;  /* chunks hold at most 64 frames */
  const int dims = dims_code == 0 ? 2 : (int)dims_code;
  if (p.bin_h < 1 || p.bin_w < 1 || p.roi_h < 1 || p.roi_w < 1 || p.quant_radius < 2 ||
      p.quant_radius > 512 || chunk != ORC_CHUNK_SYMBOLS)
    return ORC_ERR_CORRUPT_STREAM;
  const uint32_t hb = (g->rows + p.bin_h - 1) / p.bin_h, wb = (g->cols + p.bin_w - 1) / p.bin_w;
  const uint64_t m = (uint64_t)g->n_panels * hb * wb;
  if (m != m_hdr || n_chunks != (m + chunk - 1) / chunk || n_lo > m || n_pq > m || n_words > m)
    return ORC_ERR_CORRUPT_STREAM;
  const uint32_t n_symbols = 2u * (uint32_t)p.quant_radius;
  const orc_layout L =
      layout_of(n_peaks, &p, n_symbols, n_chunks, n_lo, n_pq, n_words, roi_coding == 0, back_ref == 0);
  if (L.total + roi_bytes != total || total > in_bytes) return ORC_ERR_CORRUPT_STREAM;
  h->p = p;
  h->n_peaks = n_peaks;
  h->n_lo = n_lo;
  h->n_pq = n_pq;
  h->n_chunks = n_chunks;
  h->n_words = n_words;
  h->roi_coding = roi_coding;
  h->roi_bytes = roi_bytes;
  h->roi_words = roi_words;
  h->back_ref = back_ref;
  h->dims = dims;
  h->m = m;
  h->total = total;
  h->L = L;
  return ORC_OK;
}

/* Decodes one stream whose header is h, with the code lengths `len` (its own,
 * or its chunk head's). */
static int decode_stream(const uint8_t* in, const orc_header* h, const uint8_t* len, const orc_geometry* g,
                         float* frame_out) {
  const orc_params p = h->p;
  const uint32_t n_peaks = h->n_peaks, n_lo = h->n_lo, n_pq = h->n_pq, n_chunks = h->n_chunks;
  const uint32_t n_words = h->n_words, roi_coding = h->roi_coding, roi_bytes = h->roi_bytes;
  const uint32_t roi_words = h->roi_words, chunk = ORC_CHUNK_SYMBOLS;
  const int dims = h->dims;
  const uint64_t m = h->m;
  const orc_layout L = h->L;
  const uint32_t hb = (g->rows + p.bin_h - 1) / p.bin_h, wb = (g->cols + p.bin_w - 1) / p.bin_w;
  const uint32_t n_symbols = 2u * (uint32_t)p.quant_radius;
  /* the ROI windows: in place, or decoded from their section */
  const size_t win = (size_t)p.roi_h * p.roi_w;
  float* roi = (float*)malloc(sizeof(float) * (win * n_peaks + 1));
  if (roi_coding == 0) {
    memcpy(roi, in + L.roi, win * n_peaks * 4);
  } else if (orc_roi_decode(in + L.total, roi_bytes, roi_coding, roi_words, n_peaks, p.roi_h, p.roi_w, roi) !=
             ORC_OK) {
    free(roi);
    return ORC_ERR_CORRUPT_STREAM;
  }

  /* canonical decoding tables from the code lengths */
  uint32_t count[34] = {0};
  for (uint32_t s = 0; s < n_symbols; ++s) {
    if (len[s] > 32) return ORC_ERR_CORRUPT_STREAM;
    count[len[s]]++;
  }
  count[0] = 0;
  uint32_t* sorted = (uint32_t*)malloc(sizeof(uint32_t) * n_symbols);
  /* symbols ordered by (length, symbol); first_code[l] is the canonical code of
   * the first symbol of length l, found with the same rule that assigned them */
  uint32_t first_index[34], n_sorted = 0;
  uint64_t first_code[34];
  {
    uint64_t c = 0;
    int prev = 0;
    for (int l = 1; l <= 32; ++l) {
      first_index[l] = n_sorted;
      first_code[l] = 0;
      for (uint32_t s = 0; s < n_symbols; ++s)
        if (len[s] == l) sorted[n_sorted++] = s;
      if (count[l] == 0) continue;
      c = (prev == 0) ? 0 : (c + count[prev]) << (l - prev);
      first_code[l] = c;
      prev = l;
    }
  }

  int32_t* delta = (int32_t*)malloc(sizeof(int32_t) * m);
  int status = ORC_OK;
  const uint8_t* lo = in + L.lorenzo;
  uint32_t lo_next = 0;
  for (uint32_t k = 0; k < n_chunks && status == ORC_OK; ++k) {
    const uint32_t w0 = get_u32(in + L.chunk_index + 4 * k);
    const uint32_t w1 = (k + 1 < n_chunks) ? get_u32(in + L.chunk_index + 4 * (k + 1)) : n_words;
    if (w0 > w1 || w1 > n_words) {
      status = ORC_ERR_CORRUPT_STREAM;
      break;
    }
    const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
    uint64_t bit = 0;
    const uint64_t s0 = (uint64_t)k * chunk, s1 = (s0 + chunk < m) ? s0 + chunk : m;
    for (uint64_t i = s0; i < s1 && status == ORC_OK; ++i) {
      uint64_t code = 0;
      int sym = -1;
      for (int l = 1; l <= 32; ++l) {
        if (bit >= bit_end) break;
        const uint32_t word = get_u32(in + L.bitstream + 4 * ((uint64_t)w0 + bit / 32));
        code = (code << 1) | ((word >> (31 - bit % 32)) & 1u);
        ++bit;
        if (count[l] && code >= first_code[l] && code - first_code[l] < count[l]) {
          sym = (int)sorted[first_index[l] + (code - first_code[l])];
          break;
        }
      }
      if (sym < 0) {
        status = ORC_ERR_CORRUPT_STREAM;
        break;
      }
      if (sym == 0) {
        if (lo_next >= n_lo || get_u32(lo + 8 * lo_next) != i) {
          status = ORC_ERR_CORRUPT_STREAM;
          break;
        }
        delta[i] = (int32_t)get_u32(lo + 8 * lo_next + 4);
        ++lo_next;
      } else {
        delta[i] = sym - p.quant_radius;
      }
    }
  }
  if (status == ORC_OK && lo_next != n_lo) status = ORC_ERR_CORRUPT_STREAM;

  float* bhat = (float*)malloc(sizeof(float) * m);
  if (status == ORC_OK) {
    /* q = delta + the predictor's value from the q already rebuilt, in the
     * order of the array: the inverse of a6 in the stream's dimension */
    const float two_eb = 2.0f * p.abs_eb;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * m);
    if (dims == 1) {
      for (uint64_t k = 0; k < m; ++k) q[k] = delta[k] + (k > 0 ? q[k - 1] : 0);
    } else if (dims == 2) {
      for (uint32_t pn = 0; pn < g->n_panels; ++pn) {
        const size_t base = (size_t)pn * hb * wb;
        for (uint32_t i = 0; i < hb; ++i)
          for (uint32_t j = 0; j < wb; ++j) {
            const int64_t up = i > 0 ? q[base + (size_t)(i - 1) * wb + j] : 0;
            const int64_t left = j > 0 ? q[base + (size_t)i * wb + j - 1] : 0;
            const int64_t diag = (i > 0 && j > 0) ? q[base + (size_t)(i - 1) * wb + j - 1] : 0;
            q[base + (size_t)i * wb + j] = delta[base + (size_t)i * wb + j] + up + left - diag;
          }
      }
    } else {
      const size_t plane = (size_t)hb * wb;
      for (uint32_t pn = 0; pn < g->n_panels; ++pn)
        for (uint32_t i = 0; i < hb; ++i)
          for (uint32_t j = 0; j < wb; ++j) {
            int64_t corner[2][2][2];
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) {
                  const int inside = (a == 0 || pn > 0) && (b == 0 || i > 0) && (c == 0 || j > 0);
                  corner[a][b][c] = (inside && (a | b | c)) ? q[(size_t)(pn - a) * plane + (size_t)(i - b) * wb + (j - c)] : 0;
                }
            const int64_t prediction = corner[1][0][0] + corner[0][1][0] + corner[0][0][1] - corner[1][1][0] -
                                       corner[1][0][1] - corner[0][1][1] + corner[1][1][1];
            q[(size_t)pn * plane + (size_t)i * wb + j] = delta[(size_t)pn * plane + (size_t)i * wb + j] + prediction;
          }
    }
    for (uint64_t i = 0; i < m; ++i) bhat[i] = (float)(int32_t)q[i] * two_eb;
    free(q);
    const uint8_t* pq = in + L.prequant;
    uint64_t prev = 0;
    for (uint32_t k = 0; k < n_pq; ++k) {
      const uint32_t idx = get_u32(pq + 8 * k);
      if (idx >= m || (k > 0 && idx <= prev)) {
        status = ORC_ERR_CORRUPT_STREAM;
        break;
      }
      memcpy(&bhat[idx], pq + 8 * k + 4, 4);
      prev = idx;
    }
  }
  if (status == ORC_OK) {
    /* up-sample: every pixel takes its bin's value */
    const size_t plane = (size_t)g->rows * g->cols;
    for (uint32_t pn = 0; pn < g->n_panels; ++pn)
      for (uint32_t r = 0; r < g->rows; ++r)
        for (uint32_t c = 0; c < g->cols; ++c)
          frame_out[pn * plane + (size_t)r * g->cols + c] =
              bhat[((size_t)pn * hb + r / p.bin_h) * wb + c / p.bin_w];
    /* ROI restoration */
    const uint8_t* pk = in + L.peaks;
    for (uint32_t k = 0; k < n_peaks && status == ORC_OK; ++k) {
      const uint32_t pn = get_u16(pk + 6 * k), pr = get_u16(pk + 6 * k + 2), pc = get_u16(pk + 6 * k + 4);
      if (pn >= g->n_panels || pr >= g->rows || pc >= g->cols) {
        status = ORC_ERR_CORRUPT_STREAM;
        break;
      }
      const long r0 = (long)pr - p.roi_h / 2, c0 = (long)pc - p.roi_w / 2;
      for (long i = 0; i < p.roi_h; ++i)
        for (long j = 0; j < p.roi_w; ++j)
          if (in_panel(r0 + i, c0 + j, g->rows, g->cols))
            frame_out[pn * plane + (size_t)(r0 + i) * g->cols + (size_t)(c0 + j)] =
                roi[k * win + (size_t)i * p.roi_w + (size_t)j];
    }
  }
  free(roi);
  free(bhat);
  free(delta);
  free(sorted);
  return status;
}

int orc_decompress_frame(const uint8_t* in, uint64_t in_bytes, const orc_geometry* g,
                         float* frame_out) {
  orc_header h;
  const int st = read_header(in, in_bytes, g, &h);
  if (st != ORC_OK) return st;
  if (h.back_ref != 0) return ORC_ERR_CORRUPT_STREAM;  /* its code lengths are in another stream */
  return decode_stream(in, &h, in + h.L.lengths, g, frame_out);
}

/* A call of streams: frame f's stream at in + offsets[f].  A stream that keeps
 * no code lengths (back reference b > 0) takes them from the stream of frame
 * f - b of the same call, which must be in the call, keep its own lengths and
 * have the same alphabet; otherwise the frame is ORC_ERR_CORRUPT_STREAM. */
int orc_decompress_frames(const uint8_t* in, uint64_t in_bytes, const uint64_t* offsets, uint32_t n_frames,
                          const orc_geometry* g, float* frames_out, int32_t* status) {
  const size_t frame_px = (size_t)g->n_panels * g->rows * g->cols;
  for (uint32_t f = 0; f < n_frames; ++f) {
    orc_header h, hh;
    float* out = frames_out + f * frame_px;
    if (offsets[f] > in_bytes) {
      status[f] = ORC_ERR_CORRUPT_STREAM;
      continue;
    }
    int st = read_header(in + offsets[f], in_bytes - offsets[f], g, &h);
    const uint8_t* len = NULL;
    if (st == ORC_OK) {
      if (h.back_ref == 0) {
        len = in + offsets[f] + h.L.lengths;
      } else if (h.back_ref > f || offsets[f - h.back_ref] > in_bytes) {
        st = ORC_ERR_CORRUPT_STREAM;
      } else {
        const uint64_t o = offsets[f - h.back_ref];
        st = read_header(in + o, in_bytes - o, g, &hh);
        if (st == ORC_OK && (hh.back_ref != 0 || hh.p.quant_radius != h.p.quant_radius)) st = ORC_ERR_CORRUPT_STREAM;
        if (st == ORC_OK) len = in + o + hh.L.lengths;
        else st = ORC_ERR_CORRUPT_STREAM;
      }
    }
    if (st == ORC_OK) st = decode_stream(in + offsets[f], &h, len, g, out);
    status[f] = st;
  }
  return ORC_OK;
}
