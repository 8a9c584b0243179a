// roi_coder.cu - lossless coding of the ROI windows and its inverse.
//
// The paper keeps every region of interest losslessly with fpzip, a predictive
// coder for floating-point data (§4).  This coder is our own of that kind, and
// the stream format in include/roibin.h defines it.  For each window, row-major:
//   - the float's bits u become m, an integer in the float's order
//     (u + 2^31 for a sign bit of 0, NOT u for a sign bit of 1);
//   - m is predicted modulo 2^32 by the 2-D Lorenzo rule inside the window
//     (neighbours outside it 0; the first value by 2^31, which is m(+0.0));
//   - the residual r, as int32, is folded to z = 2r or -2r - 1;
//   - z is sent as its bit length c (a class 0..32), Huffman-coded with one
//     codebook per frame, then the c - 1 bits of z below its leading one.
// Each window's bits start on a word.  When the coded section would not be
// smaller than the raw windows, the raw windows are stored instead.
//
// The coded section follows the bitstream, so it is written after either
// compression path by the same three kernels (the bytes therefore cannot
// depend on the path):
//   k_roi_classes  warp per window: class counts per window and per frame;
//   k_roi_plan     block per frame: codebook, words per window (from the
//                  counts), their offsets, the choice coded/raw, the section
//                  head, the frame's header fields and size;
//   k_roi_write    warp per window: the bits (or the raw floats).
// k_dec_roi_coded is the inverse: a thread per window decodes its values and
// writes the in-panel pixels over the decompressed background.
#include <cuda_runtime.h>

#include <algorithm>

#include "roibin_internal.cuh"

namespace roibin {

constexpr uint32_t kRoiWarps = 8;   // windows per block and pass (coding kernels)
constexpr uint32_t kRoiBlocks = 8;  // blocks per frame (coding kernels)

__device__ __forceinline__ uint32_t roi_order(float x) {
  const uint32_t u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float roi_unorder(uint32_t m) {
  return __uint_as_float((m & 0x80000000u) ? (m & 0x7FFFFFFFu) : ~m);
}
__device__ __forceinline__ uint32_t roi_fold(int32_t r) { return ((uint32_t)r << 1) ^ (uint32_t)(r >> 31); }
__device__ __forceinline__ uint32_t roi_unfold(uint32_t z) { return (z >> 1) ^ (0u - (z & 1u)); }
__device__ __forceinline__ uint32_t roi_class(uint32_t z) { return 32u - (uint32_t)__clz(z); }

// The frames whose windows are coded: every frame whose main path succeeded,
// and every frame that only ran out of output room (its size must still count
// the section).  Frames with too many peaks, rejected frames and errors are not.
__device__ __forceinline__ bool roi_frame_live(const PlainArgs& a, uint32_t f) {
  const int32_t st = a.frame_status[f];
  return st == ROIBIN_OK || (st == ROIBIN_ERR_CAPACITY && a.frame_bytes[f] > 0);
}

// A warp stages window k of frame f (its order bits; 0.0f past the panel edge).
__device__ __forceinline__ void roi_stage(const DevParams& p, const PlainArgs& a, const Scratch& s, uint32_t f,
                                          uint32_t k, uint32_t* mm) {
  const uint32_t px = s.peak_key[(size_t)f * p.max_peaks + k], plane = p.H * p.W;
  const uint32_t pn = px / plane, rem = px - pn * plane;
  const int r0 = (int)(rem / p.W) - p.roi_h / 2, c0 = (int)(rem % p.W) - p.roi_w / 2;
  const float* panel = a.frames + (size_t)f * p.frame_px + (size_t)pn * plane;
  const int win = p.roi_h * p.roi_w, lane = (int)lane_id();
  for (int base = 0; base < win; base += 12 * 32) {  // 12 loads in flight per lane, then the stores
    float vals[12];
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int e = base + u * 32 + lane;
      const int rr = r0 + e / p.roi_w, cc = c0 + e % p.roi_w;
      const bool in = e < win && rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W;
      vals[u] = in ? __ldg(panel + (size_t)rr * p.W + cc) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 12; ++u) {
      const int e = base + u * 32 + lane;
      if (e < win) mm[e] = roi_order(vals[u]);
    }
  }
  __syncwarp();
}

// Folded residual of element e of a staged window of width w.
__device__ __forceinline__ uint32_t roi_residual(const uint32_t* mm, int e, int w) {
  const int i = e / w, j = e - i * w;
  uint32_t pred = 0x80000000u;
  if (e > 0) pred = (i > 0 ? mm[e - w] : 0u) + (j > 0 ? mm[e - 1] : 0u) - (i > 0 && j > 0 ? mm[e - w - 1] : 0u);
  return roi_fold((int32_t)(mm[e] - pred));
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRoiWarps * 32) k_roi_classes(DevParams p, Scratch s, PlainArgs a) {
  extern __shared__ uint32_t roi_sm[];  // [kRoiWarps][win] staged windows
  __shared__ uint32_t bh[kRoiClasses];
  __shared__ uint32_t wc[kRoiWarps][kRoiClasses];
  const uint32_t f = blockIdx.y, warp = threadIdx.x >> 5, lane = lane_id();
  if (!roi_frame_live(a, f)) return;
  const uint32_t n = s.peak_count[f], win = (uint32_t)(p.roi_h * p.roi_w);
  const uint32_t mp = max(p.max_peaks, 1u);
  uint32_t* mm = roi_sm + warp * win;
  for (uint32_t c = threadIdx.x; c < kRoiClasses; c += blockDim.x) bh[c] = 0;
  __syncthreads();
  for (uint32_t k = blockIdx.x * kRoiWarps + warp; k < n; k += gridDim.x * kRoiWarps) {
    for (uint32_t c = lane; c < kRoiClasses; c += 32) wc[warp][c] = 0;
    roi_stage(p, a, s, f, k, mm);
    for (uint32_t e0 = 0; e0 < win; e0 += 32) {  // lanes with the same class add once
      const uint32_t e = e0 + lane;
      const uint32_t c = e < win ? roi_class(roi_residual(mm, (int)e, p.roi_w)) : kRoiClasses;
      const uint32_t peers = __match_any_sync(0xffffffffu, c);
      if (c < kRoiClasses && (peers & lanemask_lt()) == 0) atomicAdd(&wc[warp][c], (uint32_t)__popc(peers));
    }
    __syncwarp();
    uint16_t* cnt = s.roi_cnt + ((size_t)f * mp + k) * kRoiClasses;
    for (uint32_t c = lane; c < kRoiClasses; c += 32) {
      const uint32_t v = wc[warp][c];
      cnt[c] = (uint16_t)v;
      if (v) atomicAdd(&bh[c], v);
    }
    __syncwarp();
  }
  __syncthreads();
  for (uint32_t c = threadIdx.x; c < kRoiClasses; c += blockDim.x)
    if (bh[c]) atomicAdd(s.roi_hist + (size_t)f * kRoiClasses + c, bh[c]);
}

// ---------------------------------------------------------------------------
constexpr int kRoiPlanThreads = 256;
__global__ void __launch_bounds__(kRoiPlanThreads) k_roi_plan(DevParams p, Scratch s, PlainArgs a) {
  extern __shared__ __align__(16) unsigned char plan_sm[];
  HuffSmem& hs = *reinterpret_cast<HuffSmem*>(plan_sm);
  __shared__ uint8_t len[kRoiClasses];
  __shared__ uint32_t cw[kRoiClasses];
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry;
  const uint32_t f = blockIdx.x, tid = threadIdx.x;
  const bool live = roi_frame_live(a, f);
  if (!live) {
    if (tid == 0) s.roi_plan[f] = make_uint4(0u, 0u, 0u, 0u);  // nothing to write
    return;
  }
  const uint32_t n = s.peak_count[f], win = (uint32_t)(p.roi_h * p.roi_w);
  const uint32_t mp = max(p.max_peaks, 1u);
  const uint64_t base = a.frame_bytes[f];  // the stream so far (16-byte multiple)
  const uint64_t raw = align16((uint64_t)n * win * 4);
  uint32_t coding = 2, words = 0;
  uint64_t bytes = raw;
  if (n > 0) {
    build_codebook(s.roi_hist + (size_t)f * kRoiClasses, kRoiClasses, hs, len, cw);  // 33 classes: lengths <= 32
    if (tid == 0) carry = 0;
    __syncthreads();
    // words of each window from its class counts, then their offsets
    uint32_t* off = s.roi_off + (size_t)f * mp;
    const uint16_t* cnt = s.roi_cnt + (size_t)f * mp * kRoiClasses;
    for (uint32_t k0 = 0; k0 < n; k0 += kRoiPlanThreads) {
      const uint32_t k = k0 + tid;
      uint32_t w = 0;
      if (k < n) {
        uint32_t bits = 0;
        for (uint32_t c = 0; c < kRoiClasses; ++c)
          bits += (uint32_t)cnt[(size_t)k * kRoiClasses + c] * (len[c] + (c > 1 ? c - 1 : 0u));
        w = (bits + 31) / 32;
      }
      uint32_t tot;
      const uint32_t ex = block_excl_scan(w, tmp, &tot);
      if (k < n) off[k] = carry + ex;
      __syncthreads();
      if (tid == 0) carry += tot;
      __syncthreads();
    }
    words = carry;
    const uint64_t coded = kRoiHead + align16((uint64_t)n * 4) + align16((uint64_t)words * 4);
    if (coded < raw) {
      coding = 1;
      bytes = coded;
    }
  }
  const uint64_t total = base + bytes;
  const bool fits = a.frame_status[f] == ROIBIN_OK && total <= a.out_stride;
  __syncthreads();
  if (tid == 0) {
    a.frame_bytes[f] = total;
    if (!fits) a.frame_status[f] = ROIBIN_ERR_CAPACITY;
    s.roi_plan[f] = fits ? make_uint4(coding, coding == 1 ? words : 0u, (uint32_t)base, (uint32_t)(base >> 32))
                         : make_uint4(0u, 0u, 0u, 0u);
  }
  if (!fits) return;
  if (!RB_CHECK(s, base + bytes <= a.out_stride, ROIBIN_CHECK_ROI)) return;
  uint8_t* out = a.out + (size_t)f * a.out_stride;
  if (tid == 0) {
    uint32_t* h = reinterpret_cast<uint32_t*>(out);
    h[16] = (uint32_t)(total & 0xFFFFFFFFu);
    h[17] = (uint32_t)(total >> 32);
    h[19] = coding;
    h[20] = (uint32_t)bytes;
    h[21] = coding == 1 ? words : 0u;
  }
  uint8_t* sec = out + base;
  if (coding == 1) {
    for (uint32_t b = tid; b < kRoiHead; b += kRoiPlanThreads) sec[b] = b < kRoiClasses ? len[b] : 0u;
    uint32_t* off = reinterpret_cast<uint32_t*>(sec + kRoiHead);
    const uint32_t* so = s.roi_off + (size_t)f * mp;
    for (uint32_t k = tid; k < (uint32_t)(align16((uint64_t)n * 4) / 4); k += kRoiPlanThreads) off[k] = k < n ? so[k] : 0u;
    const uint64_t w_end = kRoiHead + align16((uint64_t)n * 4) + (uint64_t)words * 4;
    for (uint64_t b = w_end + tid; b < bytes; b += kRoiPlanThreads) sec[b] = 0;
    for (uint32_t c = tid; c < kRoiClasses; c += kRoiPlanThreads) {
      s.roi_book[(size_t)f * 2 * kRoiClasses + c] = len[c];
      s.roi_book[(size_t)f * 2 * kRoiClasses + kRoiClasses + c] = cw[c];
    }
  } else {
    for (uint64_t b = (uint64_t)n * win * 4 + tid; b < bytes; b += kRoiPlanThreads) sec[b] = 0;
  }
}

// ---------------------------------------------------------------------------
// Words a window's bits can take at most: 63 bits per value, plus a word of slack.
__host__ __device__ inline uint32_t roi_max_words(uint32_t win) { return (win * 63u + 31u) / 32u + 1u; }

__global__ void __launch_bounds__(kRoiWarps * 32) k_roi_write(DevParams p, Scratch s, PlainArgs a) {
  // [warps][win] staged windows, then [warps][roi_max_words(win)] their words; the
  // block has as many warps (up to kRoiWarps) as leave room for both
  extern __shared__ uint32_t roi_sm[];
  __shared__ uint32_t len[kRoiClasses], cw[kRoiClasses];
  const uint32_t f = blockIdx.y, warp = threadIdx.x >> 5, lane = lane_id();
  const uint4 plan = s.roi_plan[f];
  if (plan.x == 0) return;
  const uint32_t n = s.peak_count[f], win = (uint32_t)(p.roi_h * p.roi_w);
  const uint32_t mp = max(p.max_peaks, 1u);
  uint8_t* sec = a.out + (size_t)f * a.out_stride + ((uint64_t)plan.z | ((uint64_t)plan.w << 32));
  const uint32_t plane = p.H * p.W;
  if (plan.x == 2) {  // raw windows
    for (uint32_t k = blockIdx.x * (blockDim.x >> 5) + warp; k < n; k += gridDim.x * (blockDim.x >> 5)) {
      const uint32_t px = s.peak_key[(size_t)f * p.max_peaks + k], pn = px / plane, rem = px - pn * plane;
      if (RB_CHECK(s, ((uint64_t)plan.z | ((uint64_t)plan.w << 32)) + (uint64_t)(k + 1) * win * 4 <= a.out_stride,
                   ROIBIN_CHECK_ROI))
        warp_copy_roi(a.frames + (size_t)f * p.frame_px + (size_t)pn * plane, p.H, p.W, (int)(rem / p.W),
                      (int)(rem % p.W), p.roi_h, p.roi_w, reinterpret_cast<float*>(sec) + (size_t)k * win);
    }
    return;
  }
  for (uint32_t c = threadIdx.x; c < kRoiClasses; c += blockDim.x) {
    len[c] = s.roi_book[(size_t)f * 2 * kRoiClasses + c];
    cw[c] = s.roi_book[(size_t)f * 2 * kRoiClasses + kRoiClasses + c];
  }
  __syncthreads();
  uint32_t* words = reinterpret_cast<uint32_t*>(sec + kRoiHead + align16((uint64_t)n * 4));
  const uint32_t* off = s.roi_off + (size_t)f * mp;
  const uint32_t nwarps = blockDim.x >> 5;
  uint32_t* mm = roi_sm + warp * win;
  uint32_t* wb = roi_sm + nwarps * win + warp * roi_max_words(win);  // the window's words, then copied out
  for (uint32_t k = blockIdx.x * nwarps + warp; k < n; k += gridDim.x * nwarps) {
    const uint32_t w0 = off[k], w1 = k + 1 < n ? off[k + 1] : plan.y;
    // a window's words fit its staging area and the frame's word count (warp-uniform)
    if (!RB_CHECK(s, w0 <= w1 && w1 <= plan.y && w1 - w0 <= roi_max_words(win), ROIBIN_CHECK_ROI_WORDS)) continue;
    roi_stage(p, a, s, f, k, mm);
    for (uint32_t w = lane; w < w1 - w0; w += 32) wb[w] = 0;  // every bit lands below w1 - w0
    __syncwarp();
    uint32_t pos = 0;  // bits of the window before this round
    for (uint32_t e0 = 0; e0 < win; e0 += 32) {
      const uint32_t e = e0 + lane;
      uint64_t v = 0;
      uint32_t L = 0;
      if (e < win) {
        const uint32_t z = roi_residual(mm, (int)e, p.roi_w), c = roi_class(z);
        L = len[c];
        v = cw[c];
        if (c > 1) {  // the codeword, then the c - 1 bits below the leading one
          v = (v << (c - 1)) | (z & ((1u << (c - 1)) - 1u));
          L += c - 1;
        }
      }
      const uint32_t incl = warp_incl_scan(L);
      const uint32_t at = pos + incl - L;
      if (L) {
        // place the L (<= 63) bits at window bit `at`, MSB first, across at most three words
        const uint32_t o = at & 31u, sh = 96u - o - L;  // 2 <= sh <= 95
        const uint64_t hi = sh >= 64 ? v << (sh - 64) : v >> (64 - sh);
        const uint64_t lo = sh >= 64 ? 0ull : v << sh;
        uint32_t* wp = wb + (at >> 5);
        const uint32_t a0 = (uint32_t)hi, a1 = (uint32_t)(lo >> 32), a2 = (uint32_t)lo;
        if (a0) atomicOr(wp, a0);
        if (a1) atomicOr(wp + 1, a1);
        if (a2) atomicOr(wp + 2, a2);
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    for (uint32_t w = lane; w < w1 - w0; w += 32) words[w0 + w] = wb[w];
    __syncwarp();
  }
}

cudaError_t launch_roi_code(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  const uint32_t win = (uint32_t)(p.roi_h * p.roi_w);
  const size_t smem = kRoiWarps * (size_t)win * 4;  // 8 windows of up to 63 x 63 floats: 127 KB at most
  // the writer also stages each window's words (at most 63 bits per value):
  // as many warps as fit (a 63 x 63 window leaves room for 4)
  const size_t per_warp = ((size_t)win + roi_max_words(win)) * 4;
  const uint32_t wwarps = (uint32_t)std::min<size_t>(kRoiWarps, (220u * 1024u) / per_warp);
  const size_t smem_w = wwarps * per_warp;
  // the shared memory each kernel needs, set per call (sizes follow the window)
  cudaError_t e = cudaFuncSetAttribute(k_roi_classes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_roi_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_roi_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HuffSmem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.roi_hist, 0, sizeof(uint32_t) * kRoiClasses * a.n_frames, st);
  if (e != cudaSuccess) return e;
  const dim3 grid(kRoiBlocks, a.n_frames);
  k_roi_classes<<<grid, kRoiWarps * 32, smem, st>>>(p, s, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_roi_plan<<<a.n_frames, kRoiPlanThreads, sizeof(HuffSmem), st>>>(p, s, a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_roi_write<<<grid, wwarps * 32, smem_w, st>>>(p, s, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Decompression: frames whose ROI section follows the bitstream (coding 1 or
// 2).  One thread per window; every check of the section is the oracle's: the
// section's size, the code lengths (at most 32, a complete code or one class
// of length 1), the window offsets (the first 0, ascending, within the
// words), no code or bit past the window's words, and exactly its words used.
constexpr int kDecRoiThreads = 128;
__global__ void __launch_bounds__(kDecRoiThreads) k_dec_roi_coded(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t count[33], first[33], index0[33], sorted[kRoiClasses];
  __shared__ int ok;
  const uint32_t f = blockIdx.y, tid = threadIdx.x;
  if (tid == 0) ok = s.status[f] == ROIBIN_OK && s.dec_info[f].roi_coding != 0;
  __syncthreads();
  if (!ok) return;
  const DecInfo& di = s.dec_info[f];
  const uint32_t n = di.pl.n_peaks, coding = di.roi_coding, W = di.roi_words;
  const uint32_t rh = (uint32_t)di.roi_h, rw = (uint32_t)di.roi_w, win = rh * rw;
  const uint8_t* base = a.in + di.base;
  const uint8_t* sec = base + di.off_roi_sec;
  const uint16_t* pk = reinterpret_cast<const uint16_t*>(base + di.pl.off_peaks);
  if (tid == 0) {
    const uint64_t want = coding == 2 ? align16((uint64_t)n * win * 4)
                                      : kRoiHead + align16((uint64_t)n * 4) + align16((uint64_t)W * 4);
    if (di.roi_bytes != want || (coding == 2 && W != 0) || (coding == 1 && n == 0)) ok = 0;
    if (ok && coding == 1) {
      for (uint32_t L = 0; L <= 32; ++L) count[L] = 0;
      uint64_t kraft = 0;
      uint32_t present = 0;
      for (uint32_t c = 0; c < kRoiClasses; ++c) {
        const uint32_t L = sec[c];
        if (L > 32) ok = 0;
        else if (L) {
          ++count[L];
          kraft += 1ull << (32 - L);
          ++present;
        }
      }
      if (ok && !(kraft == (1ull << 32) || (present == 1 && count[1] == 1))) ok = 0;
      if (ok) {  // canonical order: by (length, class)
        uint64_t c = 0;
        uint32_t prev = 0, idx = 0;
        for (uint32_t L = 1; L <= 32; ++L) {
          index0[L] = idx;
          first[L] = 0;
          for (uint32_t k = 0; k < kRoiClasses; ++k)
            if (sec[k] == L) sorted[idx++] = k;
          if (count[L] == 0) continue;
          c = prev == 0 ? 0 : (c + count[prev]) << (L - prev);
          first[L] = (uint32_t)c;
          prev = L;
        }
      }
    }
    if (!ok) s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
  }
  __syncthreads();
  if (!ok) return;
  const uint32_t* off = reinterpret_cast<const uint32_t*>(sec + kRoiHead);
  const uint32_t* words = reinterpret_cast<const uint32_t*>(sec + kRoiHead + align16((uint64_t)n * 4));
  bool bad = false;
  for (uint32_t k = blockIdx.x * blockDim.x + tid; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t kp = pk[3 * k], r = pk[3 * k + 1], c = pk[3 * k + 2];
    if (kp >= p.P || r >= p.H || c >= p.W) {
      bad = true;
      continue;
    }
    float* panel = a.out + (size_t)f * p.frame_px + (size_t)kp * p.H * p.W;
    const int r0 = (int)r - (int)rh / 2, c0 = (int)c - (int)rw / 2;
    if (coding == 2) {
      const float* rv = reinterpret_cast<const float*>(sec) + (size_t)k * win;
      for (uint32_t e = 0; e < win; ++e) {
        const int rr = r0 + (int)(e / rw), cc = c0 + (int)(e % rw);
        if (rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W) panel[(size_t)rr * p.W + cc] = rv[e];
      }
      continue;
    }
    const uint32_t w0 = off[k], w1 = k + 1 < n ? off[k + 1] : W;
    if ((k == 0 && w0 != 0) || w0 > w1 || w1 > W) {
      bad = true;
      continue;
    }
    const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
    uint64_t buf = 0, bit = 0;  // buf: the next bits, MSB first; words past w1 read as 0
    uint32_t nbuf = 0, wi = w0;
    auto refill = [&]() {
      while (nbuf <= 32) {
        buf |= (uint64_t)(wi < w1 ? words[wi] : 0u) << (32 - nbuf);
        ++wi;
        nbuf += 32;
      }
    };
    uint32_t above[63];  // m of the row above (the window is at most 63 wide)
    uint32_t left = 0, diag = 0;
    bool wbad = false;
    for (uint32_t i = 0; i < rh && !wbad; ++i) {
      for (uint32_t j = 0; j < rw; ++j) {
        refill();
        // the class: the shortest codeword that matches the next bits
        uint32_t cls = 0xFFFFFFFFu, L = 1;
        for (; L <= 32; ++L) {
          const uint32_t code = (uint32_t)(buf >> (64 - L));
          if (count[L] && code - first[L] < count[L]) {
            cls = sorted[index0[L] + code - first[L]];
            break;
          }
        }
        if (cls == 0xFFFFFFFFu) {
          wbad = true;
          break;
        }
        buf <<= L;
        nbuf -= L;
        bit += L;
        refill();
        uint32_t z = cls == 0 ? 0u : 1u;
        if (cls > 1) {
          z = (1u << (cls - 1)) | (uint32_t)(buf >> (64 - (cls - 1)));
          buf <<= cls - 1;
          nbuf -= cls - 1;
          bit += cls - 1;
        }
        if (bit > bit_end) {
          wbad = true;
          break;
        }
        const uint32_t up = i > 0 ? above[j] : 0u;
        const uint32_t pred = (i == 0 && j == 0) ? 0x80000000u : up + (j > 0 ? left : 0u) - (i > 0 && j > 0 ? diag : 0u);
        const uint32_t m = roi_unfold(z) + pred;
        diag = up;
        left = m;
        above[j] = m;
        const int rr = r0 + (int)i, cc = c0 + (int)j;
        if (rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W) panel[(size_t)rr * p.W + cc] = roi_unorder(m);
      }
    }
    if (wbad || (bit + 31) / 32 != (uint64_t)(w1 - w0)) bad = true;
  }
  if (bad) s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
}

cudaError_t launch_dec_roi_coded(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  (void)p;
  const dim3 grid(16, a.n_frames);
  k_dec_roi_coded<<<grid, kDecRoiThreads, 0, st>>>(p, s, a);
  return cudaGetLastError();
}

}  // namespace roibin
