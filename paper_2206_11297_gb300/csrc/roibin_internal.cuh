// roibin_internal.cuh - shared device code of the ROIBIN-SZ CUDA library.
//
// The arithmetic of every step lives here once, as __device__ functions, so
// that the per-stage kernels (plain_kernels.cu) and the fused cluster kernel
// (fused_kernel.cu) compute bit-identical results.  Float steps round exactly
// once each, in a fixed order (explicit _rn intrinsics; the library is also
// built with -fmad=false), so results do not depend on the launch shape.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "roibin.h"

namespace roibin {

// ---- stream format version 1 -------------------------------------------
constexpr uint32_t kMagic = 0x5A534252u;  // bytes "RBSZ"
constexpr uint32_t kVersion = 1u;
constexpr uint32_t kHeaderBytes = 96u;
constexpr uint32_t kChunk = 4096u;         // symbols per chunk of the bitstream
constexpr uint32_t kCanonicalNaN = 0x7FC00000u;
constexpr float kPqLimit = 268435456.0f;   // |q| < 2^28 keeps every delta in int32
constexpr uint32_t kMaxSymbols = 1024u;    // 2 * quant_radius <= 1024
constexpr uint32_t kMaxBinsPerFrame = 5702886u;
constexpr uint32_t kMaxPeaksLimit = 8192u;
constexpr uint32_t kThrCap = 16384u;       // pixels >= amax_thr listed per frame
                                           // before the dense candidate scan

// Everything a kernel needs to know about the geometry and the parameters.
struct DevParams {
  uint32_t P, H, W;   // panels, rows, cols
  uint32_t Hb, Wb;    // binned rows / cols per panel
  uint32_t M;         // bins per frame = P * Hb * Wb
  uint32_t n_chunks;  // ceil(M / kChunk)
  uint64_t frame_px;  // P * H * W
  int32_t bh, bw;
  float amax, atot_thr, son_min, pix_nsigma;
  int32_t rank, ring_r0, ring_dr, npix_min, npix_max;
  int32_t roi_h, roi_w;
  float eb, two_eb, recip;  // two_eb = fl(2 eb), recip = fl(1 / two_eb)
  float eb_lo, eb_hi;       // screen of the bound test (see prequantize)
  int32_t d_lo;             // residuals in [d_lo, d_lo + d_span] fit a code byte and the alphabet
  uint32_t d_span;
  int32_t R;                // quant radius
  uint32_t nsym;            // 2R
  uint32_t max_peaks;
  uint32_t thr_cap;
  int32_t dims;             // Lorenzo predictor order: 1 (frame run), 2 (panel), 3 (panel stack)
  int32_t nhr_min;          // non-hit rejection: frames with fewer peaks are not compressed (0: off)
  int32_t roi_coder;        // 0: raw ROI windows in place; 1: the lossless ROI coder (section at the end)
  uint32_t chunk;           // frames of a call per chunk sharing one codebook (1: a codebook per frame)
};

// ROI coding (the section after the bitstream): 33 classes of a folded residual
constexpr uint32_t kRoiClasses = 33u;
constexpr uint32_t kRoiHead = 48u;  // code lengths, zero padded
// bytes of the in-place ROI section of a frame with n peaks
__host__ __device__ inline uint64_t roi_in_place_bytes(const DevParams& p, uint32_t n) {
  return p.roi_coder ? 0u : (((uint64_t)n * p.roi_h * p.roi_w * 4 + 15u) & ~uint64_t(15u));
}

// Byte layout of one frame's stream, filled by the plan step.
struct FramePlan {
  uint32_t n_peaks, n_lo, n_pq, n_words;
  uint64_t off_peaks, off_roi, off_len, off_cidx, off_lo, off_pq, off_bits, total;
};

// Per-frame parameters read back from a stream header by the decompressor.
struct DecInfo {
  FramePlan pl;
  uint64_t base;      // byte offset of the stream in the input buffer
  float eb, two_eb;
  int32_t R, roi_h, roi_w;
  uint32_t nsym;
  uint32_t sparse;    // 1: a length-1 code, and few other symbols in every chunk
  uint32_t roi_coding, roi_words;  // header: ROI coding (0 in place, 1 coded, 2 raw at the end), its words
  uint32_t back_ref;               // frames back to the stream with the code lengths (0: this one)
  uint64_t off_roi_sec, roi_bytes; // the ROI section after the bitstream
};

// Per-frame scratch owned by the context (indexed by frame slot).
struct Scratch {
  uint32_t* thr_count;    // [n] pixels >= amax_thr seen (may exceed thr_cap)
  uint32_t* thr_idx;      // [n][thr_cap] pixel index within the frame
  uint32_t* peak_count;   // [n] accepted peaks (may exceed max_peaks)
  uint32_t* peak_key;     // [n][max_peaks] pixel index within the frame
  uint32_t* hist;         // [n][kMaxSymbols]
  uint8_t* cb_len;        // [n][kMaxSymbols]
  uint32_t* cb_code;      // [n][kMaxSymbols]
  uint16_t* codes;        // [n][n_chunks * kChunk] (plain path); bit 15 marks a
                          // prequantisation outlier, bits 0..9 hold the code
  int32_t* lo_delta;      // [n][M] Lorenzo-outlier deltas, written at their bin
  uint32_t* pq_bits;      // [n][M] prequantisation-outlier float bits, at their bin
  uint32_t* chunk_words;  // [n][n_chunks] words per chunk -> word offset of chunk
  uint32_t* chunk_lo;     // [n][n_chunks] Lorenzo outliers per chunk -> offset
  uint32_t* chunk_pq;     // [n][n_chunks] prequant outliers per chunk -> offset
  FramePlan* plan;        // [n]
  int32_t* status;        // [n]
  // decompression (aliases lo_delta / pq_bits: a context runs one call at a time)
  int32_t* dq;            // [n][M] delta, then q (multi-pass); the panel path keeps
                          // [n][P] first Lorenzo outlier of each panel at dq + f * M
  float* bhat;            // [n][M] (multi-pass); the panel path keeps [n][P] first
                          // prequantisation outlier of each panel at bhat + f * M
  uint32_t* dec_table;    // [n][kDecTableWords] canonical decoding tables
  uint32_t* dec_zero;     // [n] code-0 symbols decoded
  DecInfo* dec_info;      // [n]
  // persistent batched path (codes: esc side array; lo_delta, pq_bits shared)
  uint8_t* codes8;          // [n][n_chunks * kChunk] one code byte per bin
  uint32_t* pq_mask;        // [n][P][mask_words] prequantisation-outlier bits per panel
  uint32_t* hist_part;      // [n][P][kMaxSymbols] per-panel histograms
  uint32_t* peak_part;      // [n][P][max(max_peaks, 1)] per-panel sorted peaks
  uint32_t* peak_part_count;  // [n][P]
  uint32_t* pq_part_count;    // [n][P] prequantisation outliers per panel
  uint32_t* lane_bit;         // [n][n_chunks][32] bit offset of each lane's symbols in its chunk
  uint32_t* lane_lo;          // [n][n_chunks][32] Lorenzo outliers before the lane, in its chunk
  uint32_t* lane_pq;          // [n][n_chunks][32] prequantisation outliers before the lane
  uint32_t* frame_done;     // [6 n + 1] stage counters and flags, ticket counter
  // ROI coder (after either compression path)
  uint32_t* roi_hist;       // [n][kRoiClasses] classes of the frame's windows
  uint16_t* roi_cnt;        // [n][max_peaks][kRoiClasses] classes of each window
  uint32_t* roi_off;        // [n][max_peaks] first word of each window
  uint32_t* roi_book;       // [n][2 kRoiClasses] code length, then codeword, per class
  uint4* roi_plan;          // [n] coding, section words, section offset (lo, hi)
  uint32_t* chunk_ref;      // [n] frames back to the chunk's head (which keeps the code lengths); 0: a head
  // persistent batched path: candidate keys past a CTA's shared-memory list
  uint32_t* thr_spill;      // [thr_spill_ctas][kThrSpill], by CTA index
  uint32_t thr_spill_ctas;  // CTAs with a spill list (0: none)
  uint32_t* check;          // [2] checks build: first failed check id, failed checks
};

// Checks build (-DROIBIN_CHECKS): RB_CHECK(s, cond, id) is cond, and when cond
// is false it records check `id` (ROIBIN_CHECK_*) in s.check instead of
// trapping, so the caller skips the store it guards.  Other builds compile the
// condition out (true).
#ifdef ROIBIN_CHECKS
__device__ __forceinline__ bool rb_check(uint32_t* w, bool ok, uint32_t id) {
  if (!ok && w) {
    atomicCAS(w, 0u, id);
    atomicAdd(w + 1, 1u);
  }
  return ok;
}
#define RB_CHECK(s, cond, id) ::roibin::rb_check((s).check, (cond), (id))
#else
#define RB_CHECK(s, cond, id) true
#endif
constexpr uint32_t kSyncWordsPerFrame = 7;  // the persistent kernel's sync words per frame (+1: its ticket)
constexpr uint32_t kThrSpill = 3840;  // spilled candidate keys per CTA (4,096 with the shared list)

// count, first, index (34 words each), symbols; padded to 16 bytes
constexpr uint32_t kDecCanonWords = (34 + 34 + 34 + kMaxSymbols + 3) & ~3u;
// prefix table: entry for the next kDecLutBits bits = (length << 10) | symbol for
// codes of at most kDecLutBits bits, 0 for a longer code (u16 entries, two a word)
constexpr uint32_t kDecLutBits = 12;
constexpr uint32_t kDecLutWords = (1u << kDecLutBits) / 2;
constexpr uint32_t kDecTableWords = kDecCanonWords + kDecLutWords;

// ---- small helpers -------------------------------------------------------
__host__ __device__ inline uint64_t align16(uint64_t x) { return (x + 15u) & ~uint64_t(15u); }
__host__ __device__ inline uint32_t ceil_div(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

__device__ inline uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ inline uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }

// Inclusive warp scan of a u32.
__device__ inline uint32_t warp_incl_scan(uint32_t v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, d);
    if ((int)lane_id() >= d) v += n;
  }
  return v;
}

// Exclusive block scan of one u32 per thread (blockDim.x <= 1024, multiple of
// 32).  `tmp` holds >= 33 words of shared memory.  Returns the exclusive prefix;
// *total receives the block sum.  Contains __syncthreads.
__device__ inline uint32_t block_excl_scan(uint32_t v, uint32_t* tmp, uint32_t* total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < nwarps ? tmp[lane] : 0u;
    const uint32_t wi = warp_incl_scan(w);
    if (lane < nwarps) tmp[lane] = wi - w;
    if (lane == 31) tmp[32] = wi;
  }
  __syncthreads();
  const uint32_t r = tmp[warp] + incl - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

// ---- a4 + a5: one bin's value and its prequantisation ---------------------
// Bin mean: the block's first pixel, plus the others in row-major order, in
// float32, then one IEEE division by the number of in-panel pixels (§4.1, §6).
// Prequantisation (§5.3.3, dual quantisation): t = rint(b * recip); outlier
// when b is not finite, |t| >= 2^28 or |b - fl(t * 2eb)| > eb in fp64.
struct Quant {
  int32_t q;
  uint32_t outlier_bits;  // valid when outlier
  bool outlier;
};

// The fp64 test |b - b^| > eb is the definition.  It is evaluated as an fp32
// screen: d = fl(|b - b^|) has relative error <= 2^-24, so d < eb_lo proves
// "within" and d > eb_hi proves "outside" (eb_lo, eb_hi = eb (1 -+ 2^-20));
// only the rare d in [eb_lo, eb_hi] takes the exact fp64 test.  A non-finite b
// gives a non-finite t, so the |t| < 2^28 test also rejects NaN and Inf.
// The exact test, out of line so that its fp64 work is never hoisted out of
// the rare branch that needs it (fp64 throughput is low on this GPU).
static __device__ __noinline__ bool bound_exceeded_exact(float b, float bh, float eb) {
  return fabs(__dadd_rn((double)b, -(double)bh)) > (double)eb;
}

__device__ __forceinline__ Quant prequantize(float b, const DevParams& p) {
  Quant r;
  const float t = rintf(__fmul_rn(b, p.recip));
  bool out = !(fabsf(t) < kPqLimit);
  if (!out) {
    const float bh = __fmul_rn(t, p.two_eb);
    const float d = fabsf(__fsub_rn(b, bh));
    if (d > p.eb_hi) out = true;
    else if (d >= p.eb_lo) out = bound_exceeded_exact(b, bh, p.eb);
  }
  r.outlier = out;
  r.q = out ? 0 : (int32_t)t;
  r.outlier_bits = isnan(b) ? kCanonicalNaN : __float_as_uint(b);
  return r;
}

// The common case of prequantize: true when the screen alone proves the bin
// is not an outlier (then q is final); false sends the bin to prequantize.
__device__ __forceinline__ bool prequant_fast(float b, const DevParams& p, int32_t& q) {
  const float t = rintf(__fmul_rn(b, p.recip));
  const float d = __fsub_rn(b, __fmul_rn(t, p.two_eb));
  q = __float2int_rz(t);  // exact for the |t| < 2^28 the fast path accepts
  return (fabsf(t) < kPqLimit) & (fabsf(d) < p.eb_lo);
}

// 2x2 bin pair from two float4 (4 pixels of raw row 2i and of row 2i+1):
// sum in row-major order from the first pixel, one IEEE division.
__device__ __forceinline__ void bin_pair(const float4& a, const float4& b, bool two, float& b0, float& b1) {
  float s0 = __fadd_rn(a.x, a.y), s1 = __fadd_rn(a.z, a.w);
  if (two) {
    s0 = __fadd_rn(__fadd_rn(s0, b.x), b.y);
    s1 = __fadd_rn(__fadd_rn(s1, b.z), b.w);
  }
  // division by 2 or 4: the exact product with 0.5 or 0.25 is the correctly
  // rounded quotient, bit for bit, so this is the same IEEE division
  const float rc = two ? 0.25f : 0.5f;
  b0 = __fmul_rn(s0, rc);
  b1 = __fmul_rn(s1, rc);
}

// Histogram update by a whole warp (every lane calls; code 0xFFFF = no item).
// Lanes holding the frame's most common code (`common`, the zero residual)
// are counted with one ballot; the others are aggregated by value.
__device__ __forceinline__ void hist_add_warp(uint32_t* hist, uint32_t code, uint32_t common) {
  const uint32_t mc = __ballot_sync(0xffffffffu, code == common);
  if (mc && lane_id() == (uint32_t)(__ffs(mc) - 1)) atomicAdd(hist + common, (uint32_t)__popc(mc));
  const bool rest = code != common && code != 0xFFFFu;
  const uint32_t mr = __ballot_sync(0xffffffffu, rest);
  if (rest) {
    const uint32_t peers = __match_any_sync(mr, code);
    if ((peers & lanemask_lt()) == 0) atomicAdd(hist + code, (uint32_t)__popc(peers));
  }
}

// a7: code of a Lorenzo residual (code 0 = outlier).
__device__ __forceinline__ uint32_t quant_code(int32_t delta, int32_t R) {
  return (delta > -R && delta < R) ? (uint32_t)(delta + R) : 0u;
}

// ---- a1: local-maximum candidate (§4.2) ----------------------------------
// >= every pixel of the panel-clipped window, > every pixel before it in
// row-major order, and >= amax_thr.
__device__ inline bool is_candidate(const float* __restrict__ panel, int H, int W, int r, int c,
                                    int rank, float amax) {
  const float v = panel[(size_t)r * W + c];
  if (!(v >= amax)) return false;
  for (int dr = -rank; dr <= rank; ++dr) {
    const int rr = r + dr;
    if (rr < 0 || rr >= H) continue;
    for (int dc = -rank; dc <= rank; ++dc) {
      const int cc = c + dc;
      if (cc < 0 || cc >= W || (dr == 0 && dc == 0)) continue;
      const float u = __ldg(panel + (size_t)rr * W + cc);
      const bool precedes = dr < 0 || (dr == 0 && dc < 0);
      if (precedes ? !(v > u) : !(v >= u)) return false;
    }
  }
  return true;
}

// ---- a2: candidate evaluation (§4.2), float32 in a fixed order ------------
// `px(dr, dc)` returns the pixel at (r + dr, c + dc); it is only called for
// in-panel positions.  The sums run in row-major order and round once per
// operation, so the result does not depend on where the pixels come from.
// The decision is taken in float32 (the data's precision); the sums are
// chained in one lane so that the order is fixed.
template <class Px>
__device__ inline bool evaluate_peak_at(Px px, int H, int W, int r, int c, const DevParams& p) {
  const int r0 = p.ring_r0, outer = p.ring_r0 + p.ring_dr, reach = outer - 1;
  float sum = 0.0f;
  int n = 0;
  for (int dr = -reach; dr <= reach; ++dr) {
    for (int dc = -reach; dc <= reach; ++dc) {
      const int d2 = dr * dr + dc * dc;
      if (d2 < r0 * r0 || d2 >= outer * outer) continue;
      const int rr = r + dr, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      sum = __fadd_rn(sum, px(dr, dc));
      ++n;
    }
  }
  float bkg = 0.0f, var = 0.0f;
  if (n > 0) {
    bkg = __fdiv_rn(sum, (float)n);
    float ss = 0.0f;
    for (int dr = -reach; dr <= reach; ++dr) {
      for (int dc = -reach; dc <= reach; ++dc) {
        const int d2 = dr * dr + dc * dc;
        if (d2 < r0 * r0 || d2 >= outer * outer) continue;
        const int rr = r + dr, cc = c + dc;
        if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
        const float d = __fsub_rn(px(dr, dc), bkg);
        ss = __fadd_rn(ss, __fmul_rn(d, d));
      }
    }
    var = __fdiv_rn(ss, (float)n);
  }
  const float sigma = __fsqrt_rn(var);
  const float thr = __fmul_rn(p.pix_nsigma, sigma);
  int npix = 0;
  float atot = 0.0f;
  for (int dr = -p.rank; dr <= p.rank; ++dr) {
    for (int dc = -p.rank; dc <= p.rank; ++dc) {
      const int rr = r + dr, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      const float d = __fsub_rn(px(dr, dc), bkg);
      if (d > thr) {
        ++npix;
        atot = __fadd_rn(atot, d);
      }
    }
  }
  if (npix < p.npix_min || npix > p.npix_max) return false;
  if (!(atot > p.atot_thr)) return false;
  const float noise = __fmul_rn(__fmul_rn(p.son_min, sigma), __fsqrt_rn((float)npix));
  return atot > noise;
}

// a1 for one thread: (r, c) is >= amax_thr, >= every in-panel window pixel and
// > every window pixel before it in row-major order (the warp tests' rule).
template <class Px>
__device__ inline bool is_local_max_at(Px px, int H, int W, int r, int c, const DevParams& p) {
  const float v = px(0, 0);
  if (!(v >= p.amax)) return false;
  for (int dr = -p.rank; dr <= p.rank; ++dr) {
    for (int dc = -p.rank; dc <= p.rank; ++dc) {
      const int rr = r + dr, cc = c + dc;
      if ((dr == 0 && dc == 0) || rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      const float u = px(dr, dc);
      const bool before = dr < 0 || (dr == 0 && dc < 0);
      if (before ? !(v > u) : !(v >= u)) return false;
    }
  }
  return true;
}

// is_local_max_at + evaluate_peak_at for one compile-time window and ring
// (RANK, ring R0 .. R0 + DR): the same operations in the same order (so the
// same float32 results), with every loop unrolled, so that the compiler sees
// each neighbour's offset and issues the loads ahead of the ordered sums.
// In-panel tests stay per pixel (a candidate may sit at the panel's edge).
template <int RANK, int R0, int DR, class Px>
__device__ __forceinline__ bool peak_test_fixed(Px px, int H, int W, int r, int c, const DevParams& p) {
  constexpr int OUT = R0 + DR, RING = OUT - 1;
  const float v = px(0, 0);
  if (!(v >= p.amax)) return false;
  bool ok = true;
#pragma unroll
  for (int dr = -RANK; dr <= RANK; ++dr) {
#pragma unroll
    for (int dc = -RANK; dc <= RANK; ++dc) {
      if (dr == 0 && dc == 0) continue;
      const int rr = r + dr, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      const float u = px(dr, dc);
      ok &= (dr < 0 || (dr == 0 && dc < 0)) ? (v > u) : (v >= u);
    }
  }
  if (!ok) return false;
  float sum = 0.0f;
  int n = 0;
#pragma unroll
  for (int dr = -RING; dr <= RING; ++dr) {
#pragma unroll
    for (int dc = -RING; dc <= RING; ++dc) {
      if (dr * dr + dc * dc < R0 * R0 || dr * dr + dc * dc >= OUT * OUT) continue;
      const int rr = r + dr, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      sum = __fadd_rn(sum, px(dr, dc));
      ++n;
    }
  }
  float bkg = 0.0f, var = 0.0f;
  if (n > 0) {
    bkg = __fdiv_rn(sum, (float)n);
    float ss = 0.0f;
#pragma unroll
    for (int dr = -RING; dr <= RING; ++dr) {
#pragma unroll
      for (int dc = -RING; dc <= RING; ++dc) {
        if (dr * dr + dc * dc < R0 * R0 || dr * dr + dc * dc >= OUT * OUT) continue;
        const int rr = r + dr, cc = c + dc;
        if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
        const float d = __fsub_rn(px(dr, dc), bkg);
        ss = __fadd_rn(ss, __fmul_rn(d, d));
      }
    }
    var = __fdiv_rn(ss, (float)n);
  }
  const float sigma = __fsqrt_rn(var);
  const float thr = __fmul_rn(p.pix_nsigma, sigma);
  int npix = 0;
  float atot = 0.0f;
#pragma unroll
  for (int dr = -RANK; dr <= RANK; ++dr) {
#pragma unroll
    for (int dc = -RANK; dc <= RANK; ++dc) {
      const int rr = r + dr, cc = c + dc;
      if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
      const float d = __fsub_rn(px(dr, dc), bkg);
      if (d > thr) {
        ++npix;
        atot = __fadd_rn(atot, d);
      }
    }
  }
  if (npix < p.npix_min || npix > p.npix_max) return false;
  if (!(atot > p.atot_thr)) return false;
  const float noise = __fmul_rn(__fmul_rn(p.son_min, sigma), __fsqrt_rn((float)npix));
  return atot > noise;
}

// The same test for a candidate whose neighbourhood rows [rb0, rb1) of its
// panel sit in `band` (row pitch W).  It goes row by row: the row's pixels are
// read unconditionally from clamped in-band addresses (so the reads of a row
// are issued together), and out-of-panel or off-ring pixels are then masked
// out by selects, so no pixel is a branch.  The sums take exactly the
// in-panel pixels in row-major order, as evaluate_peak_at does, so the results
// are the same bit for bit.
template <int RANK, int R0, int DR>
__device__ __forceinline__ bool peak_test_band(const float* band, int rb0, int rb1, int H, int W, int r, int c,
                                               const DevParams& p) {
  constexpr int OUT = R0 + DR, RING = OUT - 1, REACH = RANK > RING ? RANK : RING, SIDE = 2 * REACH + 1;
  static_assert(SIDE <= 32, "one bit per column of the neighbourhood");
  int col[SIDE];        // clamped columns c - REACH .. c + REACH
  uint32_t col_in = 0;  // bit k: column c + k - REACH is in the panel
#pragma unroll
  for (int k = 0; k < SIDE; ++k) {
    const int cc = c + k - REACH;
    col_in |= (uint32_t)(cc >= 0 && cc < W) << k;
    col[k] = min(max(cc, 0), W - 1);
  }
  auto row_at = [&](int dr) { return band + (min(max(r + dr, rb0), rb1 - 1) - rb0) * W; };
  auto row_mask = [&](int dr) { return (r + dr >= 0 && r + dr < H) ? col_in : 0u; };
  const float v = band[(r - rb0) * W + c];
  if (!(v >= p.amax)) return false;
  bool ok = true;
#pragma unroll 1
  for (int dr = -RANK; dr <= RANK; ++dr) {
    const float* rp = row_at(dr);
    const uint32_t m = row_mask(dr);
    float x[2 * RANK + 1];
#pragma unroll
    for (int k = 0; k < 2 * RANK + 1; ++k) x[k] = rp[col[REACH - RANK + k]];
#pragma unroll
    for (int k = 0; k < 2 * RANK + 1; ++k) {
      const int dc = k - RANK;
      const bool in = ((m >> (REACH + dc)) & 1u) && (dr != 0 || dc != 0);
      const bool pass = (dr < 0 || (dr == 0 && dc < 0)) ? (v > x[k]) : (v >= x[k]);
      ok &= pass || !in;
    }
  }
  if (!ok) return false;
  float sum = 0.0f;
  int n = 0;
#pragma unroll 1
  for (int dr = -RING; dr <= RING; ++dr) {
    const float* rp = row_at(dr);
    const uint32_t m = row_mask(dr);
    float x[2 * RING + 1];
#pragma unroll
    for (int k = 0; k < 2 * RING + 1; ++k) x[k] = rp[col[REACH - RING + k]];
#pragma unroll
    for (int k = 0; k < 2 * RING + 1; ++k) {
      const int dc = k - RING, d2 = dr * dr + dc * dc;
      const bool in = ((m >> (REACH + dc)) & 1u) && d2 >= R0 * R0 && d2 < OUT * OUT;
      sum = in ? __fadd_rn(sum, x[k]) : sum;
      n += in;
    }
  }
  float bkg = 0.0f, var = 0.0f;
  if (n > 0) {
    bkg = __fdiv_rn(sum, (float)n);
    float ss = 0.0f;
#pragma unroll 1
    for (int dr = -RING; dr <= RING; ++dr) {
      const float* rp = row_at(dr);
      const uint32_t m = row_mask(dr);
      float x[2 * RING + 1];
#pragma unroll
      for (int k = 0; k < 2 * RING + 1; ++k) x[k] = rp[col[REACH - RING + k]];
#pragma unroll
      for (int k = 0; k < 2 * RING + 1; ++k) {
        const int dc = k - RING, d2 = dr * dr + dc * dc;
        const bool in = ((m >> (REACH + dc)) & 1u) && d2 >= R0 * R0 && d2 < OUT * OUT;
        const float d = __fsub_rn(x[k], bkg);
        ss = in ? __fadd_rn(ss, __fmul_rn(d, d)) : ss;
      }
    }
    var = __fdiv_rn(ss, (float)n);
  }
  const float sigma = __fsqrt_rn(var);
  const float thr = __fmul_rn(p.pix_nsigma, sigma);
  int npix = 0;
  float atot = 0.0f;
#pragma unroll 1
  for (int dr = -RANK; dr <= RANK; ++dr) {
    const float* rp = row_at(dr);
    const uint32_t m = row_mask(dr);
    float x[2 * RANK + 1];
#pragma unroll
    for (int k = 0; k < 2 * RANK + 1; ++k) x[k] = rp[col[REACH - RANK + k]];
#pragma unroll
    for (int k = 0; k < 2 * RANK + 1; ++k) {
      const float d = __fsub_rn(x[k], bkg);
      const bool take = ((m >> (REACH + k - RANK)) & 1u) && d > thr;
      npix += take;
      atot = take ? __fadd_rn(atot, d) : atot;
    }
  }
  if (npix < p.npix_min || npix > p.npix_max) return false;
  if (!(atot > p.atot_thr)) return false;
  const float noise = __fmul_rn(__fmul_rn(p.son_min, sigma), __fsqrt_rn((float)npix));
  return atot > noise;
}

// a1 + a2 for one thread: the unrolled form for the paper's window and ring
// (rank 3, ring 5 .. 7), else the general loops.  Same results either way.
template <class Px>
__device__ __forceinline__ bool peak_test_one(Px px, int H, int W, int r, int c, const DevParams& p) {
  if (p.rank == 3 && p.ring_r0 == 5 && p.ring_dr == 2) return peak_test_fixed<3, 5, 2>(px, H, W, r, c, p);
  return is_local_max_at(px, H, W, r, c, p) && evaluate_peak_at(px, H, W, r, c, p);
}

__device__ inline bool evaluate_peak(const float* __restrict__ panel, int H, int W, int r, int c,
                                     const DevParams& p) {
  return evaluate_peak_at([&](int dr, int dc) { return __ldg(panel + (size_t)(r + dr) * W + (c + dc)); },
                          H, W, r, c, p);
}

// One warp copies the roi_h x roi_w window centred on (r, c) of `panel` to
// dst (fill 0 past the panel edge).  Loads are batched ahead of the stores,
// 12 per lane, so a window of up to 384 pixels (19 x 19) costs one round trip.
__device__ inline void warp_copy_roi(const float* __restrict__ panel, int H, int W, int r, int c, int roi_h,
                                     int roi_w, float* dst) {
  const int r0 = r - roi_h / 2, c0 = c - roi_w / 2, win = roi_h * roi_w;
  const int lane = (int)lane_id();
  for (int base = 0; base < win; base += 12 * 32) {
    float vals[12];
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int e = base + u * 32 + lane;
      const int rr = r0 + e / roi_w, cc = c0 + e % roi_w;
      vals[u] = (e < win && rr >= 0 && rr < H && cc >= 0 && cc < W) ? __ldg(panel + (size_t)rr * W + cc) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int e = base + u * 32 + lane;
      if (e < win) dst[e] = vals[u];
    }
  }
}

// Reach of the neighbourhood a candidate needs: its window and its ring.
__host__ __device__ inline int peak_reach(const DevParams& p) {
  const int ring = p.ring_r0 + p.ring_dr - 1;
  return p.rank > ring ? p.rank : ring;
}

// Sum of buf[0 .. n) in index order, one rounding per add.  Every lane runs
// the same chain on broadcast shared-memory reads, eight loads ahead.
__device__ __forceinline__ float ordered_sum(const float* buf, int n) {
  float s = 0.0f;
  for (int k0 = 0; k0 < n; k0 += 8) {
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = k0 + u < n ? buf[k0 + u] : 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < n) s = __fadd_rn(s, t[u]);
  }
  return s;
}
// Sum of (buf[k] - m)^2 over k in [0, n), in index order.
__device__ __forceinline__ float ordered_sq_dev(const float* buf, int n, float m) {
  float s = 0.0f;
  for (int k0 = 0; k0 < n; k0 += 8) {
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = k0 + u < n ? buf[k0 + u] : 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u < n) {
        const float d = __fsub_rn(t[u], m);
        s = __fadd_rn(s, __fmul_rn(d, d));
      }
  }
  return s;
}

// A certain rejection for the evaluation below, without its ordered sums.
// The evaluation keeps a candidate only if at least npix_min window pixels have
// RN(x - bkg) > thr, where bkg = RN(S / nr) with S the ordered float32 sum of
// the ring, and thr = RN(pix_nsigma * RN(sqrt(RN(Q / nr)))) with Q the ordered
// sum of RN(RN(x - bkg)^2).  Here the warp bounds those values instead:
//   - a tree sum t of the ring and a tree sum of |x|: the ordered sum S_f lies
//     within (gamma_{nr-1} + gamma_12) * sum|x| of t (recursive summation
//     bounds; each lane adds at most 8 terms, then 5 shuffle levels), so
//     bkg lies in [RN(S_lo / nr), RN(S_hi / nr)] (RN is monotone);
//   - each squared deviation lies between the squares of the nearest and the
//     farthest rounded deviation over that interval; sums of those bounds
//     rounded down and up, widened by gamma_{nr-1}, enclose Q (a sum of
//     non-negative terms under RN is monotone in each term), so thr is at least
//     RN(pix_nsigma * RN(sqrt(RN(Q_lo / nr)))).
// A window pixel can pass only if RN(x - bkg_lo) exceeds that lowest threshold.
// If fewer than npix_min could, the evaluation would reject the candidate too.
// Non-finite values, an empty ring or an overflowing bound skip the screen.
__device__ __forceinline__ bool screen_rejects(const float (&x)[8], uint32_t ring, uint32_t win, const DevParams& p) {
  if (p.npix_min < 1) return false;
  float t = 0.0f, aabs = 0.0f;
  int nr = 0;
  bool finite = true;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const bool in_ring = (ring >> u) & 1u, in_win = (win >> u) & 1u;
    if (in_ring) {
      t = __fadd_rn(t, x[u]);
      aabs = __fadd_rn(aabs, fabsf(x[u]));
      ++nr;
    }
    if ((in_ring || in_win) && !isfinite(x[u])) finite = false;
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    t = __fadd_rn(t, __shfl_xor_sync(0xffffffffu, t, d));
    aabs = __fadd_rn(aabs, __shfl_xor_sync(0xffffffffu, aabs, d));
    nr += __shfl_xor_sync(0xffffffffu, nr, d);
  }
  if (!__all_sync(0xffffffffu, finite) || nr == 0) return false;
  // gamma_k <= 1.0001 k u for k <= 300 (u = 2^-24 < 5.97e-8): this covers
  // gamma_{nr-1} + gamma_12 with room, and the error of the tree sum of |x|
  const float g = __fmul_ru((float)(nr + 13), 6.0e-8f);
  const float err = __fmul_ru(aabs, __fmul_ru(g, 1.001f));
  const float s_lo = __fsub_rd(t, err), s_hi = __fadd_ru(t, err);
  if (!isfinite(s_lo) || !isfinite(s_hi)) return false;
  const float bl = __fdiv_rn(s_lo, (float)nr), bh = __fdiv_rn(s_hi, (float)nr);
  float ql = 0.0f, qh = 0.0f;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (!((ring >> u) & 1u)) continue;
    const float dl = __fsub_rn(x[u], bh), dh = __fsub_rn(x[u], bl);  // dl <= dh
    const float near = (dl <= 0.0f && dh >= 0.0f) ? 0.0f : fminf(fabsf(dl), fabsf(dh));
    const float far = fmaxf(fabsf(dl), fabsf(dh));
    ql = __fadd_rd(ql, __fmul_rn(near, near));
    qh = __fadd_ru(qh, __fmul_rn(far, far));
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    ql = __fadd_rd(ql, __shfl_xor_sync(0xffffffffu, ql, d));
    qh = __fadd_ru(qh, __shfl_xor_sync(0xffffffffu, qh, d));
  }
  if (!isfinite(qh)) return false;
  const float q_lo = __fmul_rd(ql, __fsub_rd(1.0f, g));
  const float thr_lo = __fmul_rn(p.pix_nsigma, __fsqrt_rn(__fdiv_rn(q_lo, (float)nr)));
  int possible = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const bool b = ((win >> u) & 1u) && __fsub_rn(x[u], bl) > thr_lo;
    possible += __popc(__ballot_sync(0xffffffffu, b));
  }
  return possible < p.npix_min;
}

// One warp tests and evaluates the pixel (r, c) of `panel` (a1 + a2) when its
// neighbourhood has at most 256 pixels (reach <= 7).  Lane l holds the pixels
// l, l + 32, ... of the (2 reach + 1)^2 square in row-major order, loaded in
// one round.  The local-maximum rule is checked on those registers.  The ring
// pixels, then the window pixels above threshold, are compacted in row-major
// order into `buf` (per-warp shared memory, (2 reach + 1)^2 floats) and summed
// there in that order, so the float32 results equal evaluate_peak_at's.
template <class Load, bool kScreen = false>
__device__ __noinline__ bool warp_peak_test_small(const float* __restrict__ panel, int H, int W, int r, int c,
                                                  const DevParams& p, float* buf, Load load) {
  const int reach = peak_reach(p), side = 2 * reach + 1, n = side * side;
  const int lane = (int)lane_id();
  const int in2 = p.ring_r0 * p.ring_r0, out2 = (p.ring_r0 + p.ring_dr) * (p.ring_r0 + p.ring_dr);
  float x[8];
  uint32_t ring = 0, win = 0, before = 0;
  // (row, column) of element e = u * 32 + lane of the square, stepped by 32
  // elements a round (two divisions in all)
  int qr = lane / side, qc = lane - qr * side;
  const int step_r = 32 / side, step_c = 32 - step_r * side;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int e = u * 32 + lane;
    const int dr = qr - reach, dc = qc - reach;
    qr += step_r;
    qc += step_c;
    if (qc >= side) {
      qc -= side;
      ++qr;
    }
    const int rr = r + dr, cc = c + dc;
    const bool in = e < n && rr >= 0 && rr < H && cc >= 0 && cc < W;
    x[u] = in ? load(panel + (size_t)rr * W + cc) : 0.0f;
    const int d2 = dr * dr + dc * dc;
    ring |= (uint32_t)(in && d2 >= in2 && d2 < out2) << u;
    win |= (uint32_t)(in && dr >= -p.rank && dr <= p.rank && dc >= -p.rank && dc <= p.rank) << u;
    before |= (uint32_t)(dr < 0 || (dr == 0 && dc < 0)) << u;
  }
  // the centre pixel e = reach * side + reach
  const int ec = reach * side + reach;
  float mine = 0.0f;
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (u == (ec >> 5)) mine = x[u];
  const float v = __shfl_sync(0xffffffffu, mine, ec & 31);
  bool ok = v >= p.amax;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (!((win >> u) & 1u) || u * 32 + lane == ec) continue;
    if ((before >> u) & 1u ? !(v > x[u]) : !(v >= x[u])) ok = false;
  }
  if (!__all_sync(0xffffffffu, ok)) return false;
  if constexpr (kScreen) {
    if (screen_rejects(x, ring, win, p)) return false;
  }
  // ring pixels in row-major order
  int nr = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const bool b = (ring >> u) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, b);
    if (b) buf[nr + __popc(m & lanemask_lt())] = x[u];
    nr += __popc(m);
  }
  __syncwarp();
  float bkg = 0.0f, var = 0.0f;
  if (nr > 0) {
    bkg = __fdiv_rn(ordered_sum(buf, nr), (float)nr);
    var = __fdiv_rn(ordered_sq_dev(buf, nr, bkg), (float)nr);
  }
  const float sigma = __fsqrt_rn(var);
  const float thr = __fmul_rn(p.pix_nsigma, sigma);
  __syncwarp();
  // window pixels above threshold, in row-major order
  int npix = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const float d = __fsub_rn(x[u], bkg);
    const bool b = ((win >> u) & 1u) && d > thr;
    const uint32_t m = __ballot_sync(0xffffffffu, b);
    if (b) buf[npix + __popc(m & lanemask_lt())] = d;
    npix += __popc(m);
  }
  __syncwarp();
  bool keep = npix >= p.npix_min && npix <= p.npix_max;
  if (keep) {
    const float atot = ordered_sum(buf, npix);
    const float noise = __fmul_rn(__fmul_rn(p.son_min, sigma), __fsqrt_rn((float)npix));
    keep = atot > p.atot_thr && atot > noise;
  }
  __syncwarp();
  return keep;
}

// One warp tests and evaluates the pixel (r, c) of `panel` (a1 + a2).  Small
// neighbourhoods (the usual case) run warp_peak_test_small; larger ones are
// staged in `nb` (per-warp shared memory, (2 reach + 1)^2 floats) with one
// round of independent loads, the local-maximum rule is tested
// in parallel, and lane 0 runs the evaluation in its fixed order.
// `load(addr)` reads global memory (plain or L2-only).  Every lane returns
// the same answer.
// kScreen: run screen_rejects before the ordered sums of the small path.
template <bool kScreen = false, class Load>
__device__ inline bool warp_peak_test(const float* __restrict__ panel, int H, int W, int r, int c,
                                      const DevParams& p, float* nb, Load load) {
  const int reach = peak_reach(p), side = 2 * reach + 1, n = side * side;
  if (n <= 256) return warp_peak_test_small<Load, kScreen>(panel, H, W, r, c, p, nb, load);
  const uint32_t lane = lane_id();
  // gather in batches: all loads of a batch are issued before any store, so
  // the batch costs one memory latency instead of one per element
  for (int base = 0; base < n; base += 8 * 32) {
    float vals[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * 32 + (int)lane;
      const int rr = r + e / side - reach, cc = c + e % side - reach;
      vals[u] = (e < n && rr >= 0 && rr < H && cc >= 0 && cc < W) ? load(panel + (size_t)rr * W + cc) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * 32 + (int)lane;
      if (e < n) nb[e] = vals[u];
    }
  }
  __syncwarp();
  const float v = nb[reach * side + reach];
  const int wside = 2 * p.rank + 1;
  bool ok = v >= p.amax;
  for (int e = (int)lane; e < wside * wside; e += 32) {
    const int dr = e / wside - p.rank, dc = e % wside - p.rank;
    const int rr = r + dr, cc = c + dc;
    if ((dr == 0 && dc == 0) || rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
    const float u = nb[(dr + reach) * side + (dc + reach)];
    const bool precedes = dr < 0 || (dr == 0 && dc < 0);
    if (precedes ? !(v > u) : !(v >= u)) ok = false;
  }
  ok = __all_sync(0xffffffffu, ok);
  bool keep = false;
  if (ok && lane == 0)
    keep = evaluate_peak_at([&](int dr, int dc) { return nb[(dr + reach) * side + (dc + reach)]; }, H, W, r,
                            c, p);
  keep = __shfl_sync(0xffffffffu, keep, 0);
  __syncwarp();
  return keep;
}

// ---- a9: deterministic Huffman codebook, built by one CTA ------------------
// Leaves are the symbols with a non-zero count sorted by (count, symbol); the
// two-queue merge takes the leaf on equal weights; code length = leaf depth
// (a lone symbol gets 1); canonical codes by (length, symbol) ascending.
struct HuffSmem {
  uint32_t f[kMaxSymbols];        // compacted counts (symbol order), then sorted
  uint16_t s[kMaxSymbols];        // compacted symbols, then sorted
  uint32_t sf[kMaxSymbols];
  uint16_t ss[kMaxSymbols];
  uint32_t w[2 * kMaxSymbols];    // node weights: leaves [0,n), internal [n,2n-1)
  uint16_t parent[2 * kMaxSymbols];
  uint32_t cnt_len[34];
  uint32_t first_code[34];
  uint32_t running[34];
  uint32_t warp_cnt[32][34];
  uint32_t scan_tmp[33];
  uint32_t n;
  int32_t status;
};

// hist: counts in shared or global memory (kMaxSymbols entries, nsym used).
// Writes len[nsym] and code[nsym] (shared or global).  Returns ROIBIN_OK or
// ROIBIN_ERR_CODE_LENGTH (same value in every thread).  All threads of the
// block must call it; blockDim.x must be a multiple of 32.
__device__ inline int build_codebook(const uint32_t* hist, uint32_t nsym, HuffSmem& h,
                                     uint8_t* len_out, uint32_t* code_out) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  // 1. compact the non-zero symbols, keeping symbol order
  uint32_t base = 0;
  for (uint32_t s0 = 0; s0 < nsym; s0 += nt) {
    const uint32_t s = s0 + tid;
    const uint32_t f = s < nsym ? hist[s] : 0u;
    uint32_t tot;
    const uint32_t pos = block_excl_scan(f > 0 ? 1u : 0u, h.scan_tmp, &tot);
    if (f > 0) {
      h.f[base + pos] = f;
      h.s[base + pos] = (uint16_t)s;
    }
    base += tot;
  }
  if (tid == 0) {
    h.n = base;
    h.status = ROIBIN_OK;
  }
  for (uint32_t L = tid; L < 34; L += nt) {
    h.cnt_len[L] = 0;
    h.running[L] = 0;
  }
  __syncthreads();
  const uint32_t n = h.n;
  // 2. rank sort by (count, symbol): symbols are already ascending
  for (uint32_t i = tid; i < n; i += nt) {
    const uint32_t fi = h.f[i];
    uint32_t rank = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t fj = h.f[j];
      rank += (fj < fi) || (fj == fi && j < i);
    }
    h.sf[rank] = fi;
    h.ss[rank] = h.s[i];
  }
  __syncthreads();
  for (uint32_t s = tid; s < nsym; s += nt) len_out[s] = 0;
  // 3. two-queue merge (sequential by nature; one thread)
  if (tid == 0 && n >= 2) {
    for (uint32_t i = 0; i < n; ++i) h.w[i] = h.sf[i];
    uint32_t nl = 0, ni = n, nc = n;
    for (uint32_t k = 0; k + 1 < n; ++k) {
      uint32_t a, b;
      if (nl < n && (ni >= nc || h.w[nl] <= h.w[ni])) a = nl++; else a = ni++;
      if (nl < n && (ni >= nc || h.w[nl] <= h.w[ni])) b = nl++; else b = ni++;
      h.w[nc] = h.w[a] + h.w[b];
      h.parent[a] = (uint16_t)nc;
      h.parent[b] = (uint16_t)nc;
      ++nc;
    }
  }
  __syncthreads();
  // 4. depths by walking to the root
  for (uint32_t i = tid; i < n; i += nt) {
    uint32_t d = 1;
    if (n >= 2) {
      const uint32_t root = 2 * n - 2;
      uint32_t x = i;
      d = 0;
      while (x != root && d <= 40) {
        x = h.parent[x];
        ++d;
      }
    }
    if (d > 32) h.status = ROIBIN_ERR_CODE_LENGTH;
    const uint32_t L = d > 33 ? 33 : d;
    len_out[h.ss[i]] = (uint8_t)L;
    atomicAdd(&h.cnt_len[L], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    uint64_t c = 0;
    uint32_t prev = 0;
    for (uint32_t L = 1; L <= 32; ++L) {
      h.first_code[L] = 0;
      if (h.cnt_len[L] == 0) continue;
      c = prev == 0 ? 0 : (c + h.cnt_len[prev]) << (L - prev);
      h.first_code[L] = (uint32_t)c;
      prev = L;
    }
  }
  __syncthreads();
  // 5. canonical codes: first_code[L] + rank among same-length symbols
  const uint32_t warp = tid >> 5, nwarps = nt >> 5;
  for (uint32_t s0 = 0; s0 < nsym; s0 += nt) {
    const uint32_t s = s0 + tid;
    const uint32_t L = s < nsym ? len_out[s] : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, L);
    const uint32_t lower = __popc(peers & lanemask_lt());
    for (uint32_t k = tid; k < 32 * 34; k += nt) (&h.warp_cnt[0][0])[k] = 0;
    __syncthreads();
    if (s < nsym && L > 0 && lower == 0) h.warp_cnt[warp][L] = __popc(peers);
    __syncthreads();
    if (s < nsym && L > 0 && L <= 32) {
      uint32_t before = h.running[L];
      for (uint32_t w = 0; w < warp; ++w) before += h.warp_cnt[w][L];
      code_out[s] = h.first_code[L] + before + lower;
    } else if (s < nsym) {
      code_out[s] = 0;
    }
    __syncthreads();
    if (tid < 34) {
      uint32_t add = 0;
      for (uint32_t w = 0; w < nwarps; ++w) add += h.warp_cnt[w][tid];
      h.running[tid] += add;
    }
    __syncthreads();
  }
  const int st = h.status;
  __syncthreads();
  return st;
}

// ---- a10: append a codeword into a zeroed word buffer in shared memory -------
// bit position `pos` counts from the chunk start; MSB of the codeword first.
__device__ __forceinline__ void put_bits(uint32_t* buf, uint32_t pos, uint32_t cw, uint32_t L) {
  const uint32_t w = pos >> 5, o = pos & 31u;
  if (o + L <= 32u) {
    atomicOr(buf + w, cw << (32u - o - L));
  } else {
    atomicOr(buf + w, cw >> (o + L - 32u));
    atomicOr(buf + w + 1, cw << (64u - o - L));
  }
}

// ---- launchers (one translation unit each) --------------------------------
struct PlainArgs {
  const float* frames;
  uint32_t n_frames;
  const uint16_t* user_peaks;   // nullable
  const uint32_t* user_npeaks;  // nullable
  uint8_t* out;
  uint64_t out_stride;
  uint64_t* frame_bytes;
  int32_t* frame_status;
  uint32_t bands_per_panel;
  uint32_t rows_per_step;
  uint32_t* peaks_key_out;    // fused path: each frame's final peak list, for roibin_last_peaks
  uint32_t* peaks_count_out;
  uint64_t* trace;            // fused path: kTracePoints globaltimer stamps per traced frame
  uint32_t trace_frames;
};
constexpr uint32_t kTracePoints = 16;

// Shape of the persistent batched kernel, chosen on the host (fused_kernel.cu).
struct FusedShape {
  uint32_t ctas_per_sm, n_ctas;  // resident CTAs per SM, grid size
  uint32_t k, U;                 // panels per streaming item; streaming items per frame
  uint32_t kG;                   // column groups per consumer lane (1, or 2 for panels above 868 columns)
  uint32_t RB;                   // binned rows per streaming step (2 or 3)
  uint32_t stages, stage_bytes;  // TMA ring: slots, bytes per slot (2 RB raw rows of k panels)
  uint32_t mask_words;           // prequantisation-outlier bitmask words per panel
  uint32_t side;                 // side of the peak-test neighbourhood
  uint32_t sort_n2;              // power of two >= max_peaks
  uint32_t peak_cap;             // max(max_peaks, 1)
  uint32_t n_chunks;
  uint32_t codes_stride;         // code bytes per frame slot (n_chunks * kChunk)
  uint32_t group_chunks, groups; // chunks per size/write work item; items per frame
  uint32_t lag1, lag2;           // frames between stages in the ticket order (per launch)
  uint32_t input_evict_first;    // L2 policy of the streamed rows (1 = evict first)
  uint32_t wait_limit;           // polls of a flag wait before it reports ROIBIN_ERR_TIMEOUT
  uint32_t band_rows;            // dense peaks: panel rows staged at once (band + halo)
  uint32_t smem_dense;           // shared memory of the dense-peaks variant (>= smem)
  uint32_t dense;                // multi-job launch: this job takes the dense-peaks code
  uint32_t off_ctl, off_bar, off_hist, off_pql, off_thr, off_ring, off_nb, off_acc, off_cand;  // streaming role
  uint32_t off_huff, off_total, off_cblen, off_cbcode, off_keys, off_cw, off_offs;  // codebook / plan roles
  uint32_t off_stage;                                                        // size / write roles
  uint32_t smem;
};
bool fused_plan(const DevParams& p, int device, int num_sms, FusedShape* out);
bool fused_shape_for(const DevParams& p, uint32_t ctas_per_sm, uint32_t rows_per_step, uint32_t stages,
                     FusedShape* out);
cudaError_t launch_fused(const DevParams& p, const Scratch& fs, const PlainArgs& a, const FusedShape& sh,
                         bool screen, cudaStream_t st);

// One persistent launch over several batches (fused_jobs.cu): each job is a
// batch of frames of one geometry with its own parameters, scratch, outputs
// and shape.  The launch's counter is cut into slices; each slice holds the
// next `chunk` tickets of every job, in job order, and each job's own tickets
// come in their order.  One slice (each job's tickets in one run, the next
// job filling the previous one's tail) was the fastest on a CSPAD + epix10k +
// 8 x 512 x 1024 batch: 7.35 ms, against 8.26 ms with 8 slices and 10.07 ms
// with 256 (running a job's HBM streaming beside another's latency-bound
// peak tests slowed the peak tests more than it gained).
constexpr uint32_t kMaxFusedJobs = 16;
constexpr uint32_t kJobSlices = 1;  // slices of a launch (fewer if every job has fewer tickets)
struct FusedJob {
  DevParams p;
  Scratch s;              // frame_done: this job's sync words in the launch's buffer
  PlainArgs a;
  FusedShape sh;
  uint32_t tickets;       // the job's own tickets (those of a k_fused launch of it)
  uint32_t chunk;         // of them per slice
  uint32_t cbegin, cend;  // the job's place [cbegin, cend) in a slice
  uint32_t dense;         // the dense-peaks code
};
struct FusedJobs {
  uint32_t* ticket;       // the launch's ticket counter (zero before the launch)
  uint32_t total;         // tickets of the launch: slices x slice
  uint32_t slice;         // tickets per slice (the jobs' chunks)
  uint32_t n_jobs;
  FusedJob job[kMaxFusedJobs];
};
// Gives every job of *m (p, s, a and dense set) a shape for one joint launch:
// the CTAs per SM and ring slots are common, the first pair every job fits
// (two binned rows per step; tuned[i] gives job i's wait limit); sets the
// jobs' lags and ticket slices, m->total, the launch's shared memory and
// grid.  False if no common shape exists or the tickets overflow.
bool fused_jobs_plan(FusedJobs* m, const FusedShape* tuned, int num_sms, uint32_t* smem, uint32_t* grid);
cudaError_t launch_fused_jobs(const FusedJobs& m, uint32_t smem, uint32_t grid, cudaStream_t st);

// Each launcher enqueues one kernel and returns cudaGetLastError().
// `timer` may be null; when set, it brackets the launch with events.
struct KernelTimer {
  void (*begin)(void* self, int kernel_id, cudaStream_t s);
  void (*end)(void* self, int kernel_id, cudaStream_t s);
  void* self;
};

enum KernelId {
  K_RESET = 0,
  K_STREAM,
  K_PEAKS,
  K_PEAKS_FINAL,
  K_HUFFMAN,
  K_CHUNKS,
  K_PLAN,
  K_ENCODE,
  K_ROI,
  K_FUSED,
  K_DEC_PARSE,
  K_DEC_DECODE,
  K_DEC_LORENZO,
  K_DEC_ROWS,
  K_DEC_COLS,
  K_DEC_PQ,
  K_DEC_UPSAMPLE,
  K_DEC_ROI,
  K_DEC_PANEL,
  K_ROI_MASK,
  K_PACK,
  K_DEC_CARRY,
  K_ROI_CODE,
  K_DEC_ROI_CODED,
  K_COUNT
};
const char* kernel_name(int id);

cudaError_t launch_reset(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st);
cudaError_t launch_stream(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_peaks(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_peaks_final(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_huffman(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st);
cudaError_t launch_chunks(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st);
cudaError_t launch_plan(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_encode(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_roi(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
// ROI coder: classes and counts per window, codebook and layout per frame,
// then the bits (three kernels); frames whose status is not OK are skipped
cudaError_t launch_roi_code(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st);
cudaError_t launch_last_peaks(const DevParams& p, const Scratch& s, uint16_t* peaks, uint32_t* npeaks,
                              uint32_t n, cudaStream_t st);

struct DecArgs {
  const uint8_t* in;
  uint64_t in_bytes;
  const uint64_t* offsets;
  uint32_t n_frames;
  float* out;
  int32_t* frame_status;
};
cudaError_t launch_dec_parse(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_decode(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_lorenzo(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_rows(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_cols(const DevParams& p, const Scratch& s, const DecArgs& a, bool dequant, cudaStream_t st);
cudaError_t launch_dec_carry(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_pq(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_upsample(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_roi(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
// restores the ROI windows of frames with a coded (or moved raw) ROI section
cudaError_t launch_dec_roi_coded(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
// copies the per-frame statuses to the caller (ends every decompression)
cudaError_t launch_dec_finish(const Scratch& s, const DecArgs& a, cudaStream_t st);
// the panel path: decode through the prefix table into symbols, then one block
// per (frame, panel) rebuilds the panel strip by strip
uint32_t dec_panel_rows(const DevParams& p);  // binned rows per strip; 0: panel path unavailable
// the decoders of the panel path: k_dec_decode_sparse, then k_dec_decode_dense
cudaError_t launch_dec_decoders(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_dec_panel(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st);
cudaError_t launch_roi_mask(const DevParams& p, const uint16_t* peaks, const uint32_t* npeaks,
                            uint32_t n, uint8_t* mask, cudaStream_t st);
cudaError_t launch_pack(const uint8_t* src, uint64_t stride, const uint64_t* sizes, const uint64_t* offsets,
                        uint32_t n, uint8_t* dst, cudaStream_t st);

// ---------------------------------------------------------------------------
// mbarrier + TMA bulk-copy helpers (the fused streaming ring, the decompressor's
// symbol strips)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// A waiting thread is suspended (up to kSuspendNs per try) until the phase
// completes instead of spinning on the barrier.
constexpr uint32_t kSuspendNs = 1000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kSpinLimit = 1u << 21;  // bounded mbarrier wait (about 2 s at most)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared, completion counted on `bar`, L2 evict-first.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// L2 policy for data read once.
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

}  // namespace roibin
