// plain_kernels.cu - the per-stage compression path: one kernel per step of
// the method, intermediates in device memory.  Every kernel takes frames from
// blockIdx.y (one grid row per frame of the batch).
//
//   reset -> stream (a4-a8 + amax scan) -> peaks (a1-a2) -> peaks_final
//   -> huffman (a9) -> chunks (a10/a11 sizes) -> plan (offsets, header)
//   -> encode (a10 + a11) -> roi (a3)
#include <cuda_runtime.h>

#include "roibin_internal.cuh"

namespace roibin {

const char* kernel_name(int id) {
  static const char* names[K_COUNT] = {
      "reset", "stream", "peaks", "peaks_final", "huffman", "chunks", "plan", "encode", "roi",
      "fused", "dec_parse", "dec_decode", "dec_lorenzo", "dec_rows", "dec_cols", "dec_pq",
      "dec_upsample", "dec_roi", "dec_panel", "roi_mask", "pack", "dec_carry", "roi_code", "dec_roi_coded"};
  return (id >= 0 && id < K_COUNT) ? names[id] : "?";
}

// ---------------------------------------------------------------------------
// reset: per-frame counters and histograms start at zero.
__global__ void k_reset(DevParams p, Scratch s, uint32_t n) {
  const uint32_t stride = gridDim.x * blockDim.x;
  const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (uint32_t i = t0; i < n * kMaxSymbols; i += stride) s.hist[i] = 0;
  for (uint32_t i = t0; i < n; i += stride) {
    s.thr_count[i] = 0;
    s.peak_count[i] = 0;
    s.status[i] = ROIBIN_OK;
  }
}

// ---------------------------------------------------------------------------
// stream: bins, prequantises, predicts and codes one band of binned rows of
// one panel; also lists the pixels >= amax_thr for the peak finder.
//
// Block (bands_per_panel * P, n_frames), 256 threads.  The band is processed
// in steps of rows_per_step binned rows: phase A reads the raw rows and writes
// q of the step into shared memory (row 0 holds the row above the step), phase
// B forms the 2-D Lorenzo residuals, codes, the histogram and the outliers.
// Bands that start below the top of a panel first recompute q of the row above
// them (the halo row; its outliers and pixels belong to the band above).
constexpr int kStreamThreads = 256;

struct StreamSmem {
  uint32_t hist[kMaxSymbols];
};

// phase A for one binned row segment, vector path: bin 2x2, W % 4 == 0.
// Item = 4 consecutive pixels of the two raw rows = 2 bins.
template <bool kOwn>
__device__ __forceinline__ void phase_a_v4(const float* __restrict__ panel, const DevParams& p,
                                           uint32_t i0, uint32_t rows, int32_t* qrow0,
                                           uint8_t* pqf, Scratch& s, uint32_t f, uint32_t pn) {
  const uint32_t NP = p.W >> 2;  // items per binned row
  const uint32_t items = rows * NP;
  constexpr int U = 4;
  for (uint32_t base = threadIdx.x; base < items; base += kStreamThreads * U) {
    float4 a[U], b[U];
    bool two[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t it = base + u * kStreamThreads;
      two[u] = false;
      a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      b[u] = a[u];
      if (it < items) {
        const uint32_t il = it / NP, pr = it - il * NP;
        const uint32_t ra = 2 * (i0 + il);
        a[u] = __ldg(reinterpret_cast<const float4*>(panel + (size_t)ra * p.W) + pr);
        two[u] = ra + 1 < p.H;
        if (two[u]) b[u] = __ldg(reinterpret_cast<const float4*>(panel + (size_t)(ra + 1) * p.W) + pr);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint32_t it = base + u * kStreamThreads;
      if (it >= items) continue;
      const uint32_t il = it / NP, pr = it - il * NP;
      const uint32_t i = i0 + il, j0 = 2 * pr;
      float v0, v1;
      bin_pair(a[u], b[u], two[u], v0, v1);
      const Quant q0 = prequantize(v0, p);
      const Quant q1 = prequantize(v1, p);
      *reinterpret_cast<int2*>(qrow0 + (size_t)il * p.Wb + j0) = make_int2(q0.q, q1.q);
      if (kOwn) {
        pqf[(size_t)il * p.Wb + j0] = q0.outlier;
        pqf[(size_t)il * p.Wb + j0 + 1] = q1.outlier;
        const uint32_t bin0 = (pn * p.Hb + i) * p.Wb + j0;
        if (q0.outlier) s.pq_bits[(size_t)f * p.M + bin0] = q0.outlier_bits;
        if (q1.outlier) s.pq_bits[(size_t)f * p.M + bin0 + 1] = q1.outlier_bits;
        // pixels >= amax_thr for the peak finder (rare: screen with the max)
        const float m = fmaxf(fmaxf(fmaxf(a[u].x, a[u].y), fmaxf(a[u].z, a[u].w)),
                              fmaxf(fmaxf(b[u].x, b[u].y), fmaxf(b[u].z, b[u].w)));
        if (m >= p.amax) {
          const float px[8] = {a[u].x, a[u].y, a[u].z, a[u].w, b[u].x, b[u].y, b[u].z, b[u].w};
          const int npx = two[u] ? 8 : 4;
          for (int k = 0; k < npx; ++k) {
            if (px[k] >= p.amax) {
              const uint32_t r = 2 * i + (k >> 2), col = 4 * pr + (k & 3);
              const uint32_t slot = atomicAdd(s.thr_count + f, 1u);
              if (slot < p.thr_cap)
                s.thr_idx[(size_t)f * p.thr_cap + slot] = (pn * p.H + r) * p.W + col;
            }
          }
        }
      }
    }
  }
}

// phase A, generic path: any bin size and alignment; item = one bin.
template <bool kOwn>
__device__ __forceinline__ void phase_a_generic(const float* __restrict__ panel, const DevParams& p,
                                                uint32_t i0, uint32_t rows, int32_t* qrow0,
                                                uint8_t* pqf, Scratch& s, uint32_t f, uint32_t pn) {
  const uint32_t items = rows * p.Wb;
  for (uint32_t it = threadIdx.x; it < items; it += kStreamThreads) {
    const uint32_t il = it / p.Wb, j = it - il * p.Wb;
    const uint32_t i = i0 + il;
    float sum = 0.0f;
    int cnt = 0;
    for (int di = 0; di < p.bh; ++di) {
      const uint32_t r = i * p.bh + di;
      if (r >= p.H) break;
      for (int dj = 0; dj < p.bw; ++dj) {
        const uint32_t c = j * p.bw + dj;
        if (c >= p.W) break;
        const float x = __ldg(panel + (size_t)r * p.W + c);
        sum = cnt == 0 ? x : __fadd_rn(sum, x);
        ++cnt;
        if (kOwn && x >= p.amax) {
          const uint32_t slot = atomicAdd(s.thr_count + f, 1u);
          if (slot < p.thr_cap) s.thr_idx[(size_t)f * p.thr_cap + slot] = (pn * p.H + r) * p.W + c;
        }
      }
    }
    const Quant q = prequantize(__fdiv_rn(sum, (float)cnt), p);
    qrow0[(size_t)il * p.Wb + j] = q.q;
    if (kOwn) {
      pqf[(size_t)il * p.Wb + j] = q.outlier;
      if (q.outlier) s.pq_bits[(size_t)f * p.M + (pn * p.Hb + i) * p.Wb + j] = q.outlier_bits;
    }
  }
}

__global__ void __launch_bounds__(kStreamThreads) k_stream(DevParams p, Scratch s, PlainArgs a,
                                                           int vec4) {
  extern __shared__ __align__(16) unsigned char dsm[];
  StreamSmem& sm = *reinterpret_cast<StreamSmem*>(dsm);
  const uint32_t RB = a.rows_per_step;
  int32_t* qbuf = reinterpret_cast<int32_t*>(dsm + sizeof(StreamSmem));  // [(RB+1) * Wb]
  uint8_t* pqf = reinterpret_cast<uint8_t*>(qbuf + (size_t)(RB + 1) * p.Wb);  // [RB * Wb]
  // 3-D predictor: the same rows of the previous panel, [(RB+1) * Wb] after pqf
  int32_t* qprev = reinterpret_cast<int32_t*>(pqf + align16((uint64_t)RB * p.Wb));

  const uint32_t f = blockIdx.y;
  const uint32_t pn = blockIdx.x / a.bands_per_panel, band = blockIdx.x % a.bands_per_panel;
  const uint32_t rows_per_band = ceil_div(p.Hb, a.bands_per_panel);
  const uint32_t ib = band * rows_per_band;
  const uint32_t ie = min(p.Hb, ib + rows_per_band);
  if (ib >= ie) return;
  const float* panel = a.frames + (size_t)f * p.frame_px + (size_t)pn * p.H * p.W;
  const float* prev_panel = panel - (size_t)p.H * p.W;  // read only when pn > 0
  const bool stack = p.dims == 3 && pn > 0;            // the 3-D predictor's previous panel

  for (uint32_t k = threadIdx.x; k < p.nsym; k += kStreamThreads) sm.hist[k] = 0;
  // the row above the band; for the 1-D predictor at the top of a panel, the
  // previous panel's last row (its last bin precedes this panel's first)
  if (ib == 0 && !(p.dims == 1 && pn > 0)) {
    for (uint32_t j = threadIdx.x; j < p.Wb; j += kStreamThreads) qbuf[j] = 0;
  } else {
    const float* src = ib == 0 ? prev_panel : panel;
    const uint32_t row = ib == 0 ? p.Hb - 1 : ib - 1;
    if (vec4) phase_a_v4<false>(src, p, row, 1, qbuf, pqf, s, f, pn);
    else phase_a_generic<false>(src, p, row, 1, qbuf, pqf, s, f, pn);
  }
  if (stack) {
    if (ib == 0) {
      for (uint32_t j = threadIdx.x; j < p.Wb; j += kStreamThreads) qprev[j] = 0;
    } else if (vec4) {
      phase_a_v4<false>(prev_panel, p, ib - 1, 1, qprev, pqf, s, f, pn);
    } else {
      phase_a_generic<false>(prev_panel, p, ib - 1, 1, qprev, pqf, s, f, pn);
    }
  }
  __syncthreads();

  uint16_t* codes = s.codes + (size_t)f * ((size_t)p.n_chunks * kChunk);
  for (uint32_t i0 = ib; i0 < ie; i0 += RB) {
    const uint32_t rows = min(RB, ie - i0);
    if (vec4) phase_a_v4<true>(panel, p, i0, rows, qbuf + p.Wb, pqf, s, f, pn);
    else phase_a_generic<true>(panel, p, i0, rows, qbuf + p.Wb, pqf, s, f, pn);
    if (stack) {
      if (vec4) phase_a_v4<false>(prev_panel, p, i0, rows, qprev + p.Wb, pqf, s, f, pn);
      else phase_a_generic<false>(prev_panel, p, i0, rows, qprev + p.Wb, pqf, s, f, pn);
    }
    __syncthreads();
    // phase B: residuals, codes, histogram, outliers
    const uint32_t items = rows * p.Wb;
    const uint32_t iters = ceil_div(items, kStreamThreads);
    for (uint32_t t = 0; t < iters; ++t) {
      const uint32_t it = t * kStreamThreads + threadIdx.x;
      uint32_t code = 0xFFFFu;  // sentinel: no item
      if (it < items) {
        const uint32_t il = it / p.Wb, j = it - il * p.Wb;
        const int32_t* cur = qbuf + (size_t)(il + 1) * p.Wb;
        const int32_t* up = qbuf + (size_t)il * p.Wb;
        const int32_t qc = cur[j], qu = up[j];
        const int32_t ql = j > 0 ? cur[j - 1] : 0, qd = j > 0 ? up[j - 1] : 0;
        // integer differences wrap like the oracle's int64 result cast to int32
        int32_t delta;
        if (p.dims == 1) {
          delta = (int32_t)((uint32_t)qc - (uint32_t)(j > 0 ? ql : up[p.Wb - 1]));
        } else {
          uint32_t d = (uint32_t)qc - (uint32_t)qu - (uint32_t)ql + (uint32_t)qd;
          if (stack) {  // minus the previous panel's 2-D difference at the same place
            const int32_t* pc = qprev + (size_t)(il + 1) * p.Wb;
            const int32_t* pu = qprev + (size_t)il * p.Wb;
            d -= (uint32_t)pc[j] - (uint32_t)pu[j] - (uint32_t)(j > 0 ? pc[j - 1] : 0) +
                 (uint32_t)(j > 0 ? pu[j - 1] : 0);
          }
          delta = (int32_t)d;
        }
        code = quant_code(delta, p.R);
        const uint32_t bin = (pn * p.Hb + i0 + il) * p.Wb + j;
        const uint32_t flag = pqf[(size_t)il * p.Wb + j] ? 0x8000u : 0u;
        codes[bin] = (uint16_t)(code | flag);
        if (code == 0) s.lo_delta[(size_t)f * p.M + bin] = delta;
      }
      hist_add_warp(sm.hist, code, (uint32_t)p.R);
    }
    __syncthreads();
    // the last row of this step is the row above the next one
    for (uint32_t j = threadIdx.x; j < p.Wb; j += kStreamThreads) {
      qbuf[j] = qbuf[(size_t)rows * p.Wb + j];
      if (stack) qprev[j] = qprev[(size_t)rows * p.Wb + j];
    }
    __syncthreads();
  }
  for (uint32_t k = threadIdx.x; k < p.nsym; k += kStreamThreads)
    if (sm.hist[k]) atomicAdd(s.hist + (size_t)f * kMaxSymbols + k, sm.hist[k]);
}

// ---------------------------------------------------------------------------
// peaks: local-maximum test and evaluation of every listed pixel (or, when
// the list overflowed, of every pixel >= amax_thr of the frame), one warp per
// pixel.  Accepted peaks are appended in any order; peaks_final sorts them.
constexpr int kPeakBlocks = 16;
constexpr int kPeakWarps = 8;

__global__ void __launch_bounds__(kPeakWarps * 32) k_peaks(DevParams p, Scratch s, PlainArgs a) {
  extern __shared__ float nb_all[];
  __shared__ uint32_t q_all[kPeakWarps * 32];  // 32 candidate slots per warp (dense frames)
  const int side = 2 * peak_reach(p) + 1;
  float* nb = nb_all + (threadIdx.x >> 5) * side * side;
  const uint32_t f = blockIdx.y;
  const float* frame = a.frames + (size_t)f * p.frame_px;
  const uint32_t count = s.thr_count[f];
  const uint32_t warp = blockIdx.x * kPeakWarps + (threadIdx.x >> 5);
  const uint32_t nwarps = gridDim.x * kPeakWarps;
  const uint32_t plane = p.H * p.W;
  auto test = [&](uint32_t px) {
    const uint32_t pn = px / plane, rem = px - pn * plane;
    const uint32_t r = rem / p.W, c = rem - r * p.W;
    const float* panel = frame + (size_t)pn * plane;
    if (warp_peak_test<true>(panel, p.H, p.W, r, c, p, nb, [](const float* q) { return __ldg(q); })) {
      if (lane_id() == 0) {
        const uint32_t slot = atomicAdd(s.peak_count + f, 1u);
        if (slot < p.max_peaks) s.peak_key[(size_t)f * p.max_peaks + slot] = px;
      }
    }
  };
  if (count <= p.thr_cap) {
    for (uint32_t e = warp; e < count; e += nwarps) test(s.thr_idx[(size_t)f * p.thr_cap + e]);
    return;
  }
  // dense: the warp reads 512 pixels per round with four independent float4
  // loads per lane (frames start 16-byte aligned; a frame of fewer than a
  // multiple of 4 pixels takes the scalar loop), then tests those >= amax_thr
  if (p.frame_px % 4 == 0 && (reinterpret_cast<uintptr_t>(frame) & 15u) == 0) {
    // many candidates: one lane per candidate.  Pixels >= amax_thr are gathered
    // 32 at a time and each lane runs the local-maximum rule and the evaluation
    // on its own, in the sequential order the warp tests reproduce
    // (is_local_max_at, evaluate_peak_at), so a warp instruction serves 32
    const uint32_t lane = lane_id();
    uint32_t* slots = q_all + (threadIdx.x >> 5) * 32;
    uint32_t mine = 0, nq = 0;  // nq: candidates held by lanes 0 .. nq - 1 (the same in every lane)
    auto flush = [&]() {
      if (lane < nq) {
        const uint32_t pn = mine / plane, rem = mine - pn * plane;
        const int r = (int)(rem / p.W), c = (int)(rem - (uint32_t)r * p.W);
        const float* pan = frame + (size_t)pn * plane;
        auto px = [&](int dr, int dc) { return __ldg(pan + (size_t)(r + dr) * p.W + (c + dc)); };
        if (is_local_max_at(px, (int)p.H, (int)p.W, r, c, p) && evaluate_peak_at(px, (int)p.H, (int)p.W, r, c, p)) {
          const uint32_t slot = atomicAdd(s.peak_count + f, 1u);
          if (slot < p.max_peaks) s.peak_key[(size_t)f * p.max_peaks + slot] = mine;
        }
      }
      __syncwarp();
      nq = 0;
    };
    const uint64_t n4 = p.frame_px / 4;
    const float4* f4 = reinterpret_cast<const float4*>(frame);
    for (uint64_t b4 = (uint64_t)warp * 128; b4 < n4; b4 += (uint64_t)nwarps * 128) {
      float4 q[4];
      uint32_t valid = 0;  // bit u: the lane's u-th float4 lies inside the frame
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint64_t i4 = b4 + u * 32 + lane_id();
        valid |= (uint32_t)(i4 < n4) << u;
        q[u] = i4 < n4 ? __ldg(f4 + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      uint32_t hot = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if ((valid >> u) & 1u)
          hot |= (uint32_t)(q[u].x >= p.amax) << (4 * u) | (uint32_t)(q[u].y >= p.amax) << (4 * u + 1) |
                 (uint32_t)(q[u].z >= p.amax) << (4 * u + 2) | (uint32_t)(q[u].w >= p.amax) << (4 * u + 3);
      for (uint32_t j = 0; j < 16; ++j) {
        uint32_t m = __ballot_sync(0xffffffffu, (hot >> j) & 1u);
        const uint32_t px0 = (uint32_t)(4 * (b4 + (j >> 2) * 32)) + (j & 3u);  // pixel of lane 0
        while (m) {
          // the first `take` hot lanes hand their pixels to lanes nq .. nq + take - 1
          const uint32_t take = min((uint32_t)__popc(m), 32u - nq);
          const uint32_t k = __popc(m & lanemask_lt());
          const bool go = ((m >> lane) & 1u) && k < take;
          if (go) slots[nq + k] = px0 + 4 * lane;
          m &= ~__ballot_sync(0xffffffffu, go);
          __syncwarp();
          if (lane >= nq && lane < nq + take) mine = slots[lane];
          __syncwarp();
          nq += take;
          if (nq == 32) flush();
        }
      }
    }
    if (nq) flush();
    return;
  }
  for (uint64_t base = (uint64_t)warp * 32; base < p.frame_px; base += (uint64_t)nwarps * 32) {
    const uint64_t px = base + lane_id();
    const bool hot = px < p.frame_px && __ldg(frame + px) >= p.amax;
    uint32_t m = __ballot_sync(0xffffffffu, hot);
    while (m) {
      const uint32_t l = __ffs(m) - 1;
      m &= m - 1;
      test((uint32_t)(base + l));
    }
  }
}

// peaks_final: one block per frame.  Found peaks: sort ascending (pixel index
// = (panel, row, col) order), CAPACITY past max_peaks.  User peaks: validate
// and keep the given order.
__global__ void __launch_bounds__(1024) k_peaks_final(DevParams p, Scratch s, PlainArgs a) {
  extern __shared__ uint32_t keys[];  // [pow2 >= max_peaks]
  __shared__ int bad;
  const uint32_t f = blockIdx.x;
  uint32_t* out = s.peak_key + (size_t)f * p.max_peaks;
  if (a.user_peaks) {
    const uint32_t n = a.user_npeaks[f];
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    if (n > p.max_peaks) {
      if (threadIdx.x == 0) {
        s.status[f] = ROIBIN_ERR_CAPACITY;
        s.peak_count[f] = n;
      }
      return;
    }
    const uint16_t* up = a.user_peaks + (size_t)f * p.max_peaks * 3;
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t pn = up[3 * k], r = up[3 * k + 1], c = up[3 * k + 2];
      if (pn >= p.P || r >= p.H || c >= p.W) bad = 1;
      else out[k] = (pn * p.H + r) * p.W + c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s.peak_count[f] = n;
      if (bad) s.status[f] = ROIBIN_ERR_INVALID_ARG;
      else if (n < (uint32_t)p.nhr_min) s.status[f] = ROIBIN_REJECTED;  // non-hit rejection
    }
    return;
  }
  const uint32_t count = s.peak_count[f];
  if (count > p.max_peaks) {
    if (threadIdx.x == 0) s.status[f] = ROIBIN_ERR_CAPACITY;
    return;
  }
  uint32_t n2 = 1;
  while (n2 < count) n2 <<= 1;
  for (uint32_t k = threadIdx.x; k < n2; k += blockDim.x) keys[k] = k < count ? out[k] : 0xFFFFFFFFu;
  __syncthreads();
  // bitonic sort, ascending
  for (uint32_t size = 2; size <= n2; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t k = threadIdx.x; k < n2; k += blockDim.x) {
        const uint32_t partner = k ^ stride;
        if (partner > k) {
          const bool up = (k & size) == 0;
          const uint32_t x = keys[k], y = keys[partner];
          if ((x > y) == up) {
            keys[k] = y;
            keys[partner] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t k = threadIdx.x; k < count; k += blockDim.x) out[k] = keys[k];
  // non-hit rejection (§1, §4): too few peaks, the frame is not compressed
  if (threadIdx.x == 0 && count < (uint32_t)p.nhr_min) s.status[f] = ROIBIN_REJECTED;
}

// ---------------------------------------------------------------------------
// huffman: one block per chunk of frames builds its canonical codebook (§5.3.4:
// chunk_frames frames of the call share one).  A chunk of one frame (the
// default) builds the frame's own codebook.  A larger chunk builds the code of
// the summed histogram of its coded frames (status OK) and gives it to each of
// them; chunk_ref[f] = f - the chunk's first coded frame, which alone keeps
// the code lengths in its stream.
__global__ void __launch_bounds__(1024) k_huffman(DevParams p, Scratch s, uint32_t n_frames) {
  extern __shared__ __align__(16) unsigned char dsm[];
  HuffSmem& h = *reinterpret_cast<HuffSmem*>(dsm);
  uint32_t* hsum = reinterpret_cast<uint32_t*>(dsm + align16(sizeof(HuffSmem)));  // [kMaxSymbols]
  __shared__ int head;
  const uint32_t c0 = blockIdx.x * p.chunk, c1 = min(n_frames, c0 + p.chunk);
  if (p.chunk == 1) {
    const uint32_t f = c0;
    const int st = build_codebook(s.hist + (size_t)f * kMaxSymbols, p.nsym, h,
                                  s.cb_len + (size_t)f * kMaxSymbols, s.cb_code + (size_t)f * kMaxSymbols);
    if (threadIdx.x == 0) {
      if (st != ROIBIN_OK && s.status[f] == ROIBIN_OK) s.status[f] = st;
      s.chunk_ref[f] = 0;
    }
    return;
  }
  if (threadIdx.x == 0) {
    head = -1;
    for (uint32_t f = c0; f < c1 && head < 0; ++f)
      if (s.status[f] == ROIBIN_OK) head = (int)f;
  }
  __syncthreads();
  if (head < 0) return;  // no coded frame in the chunk
  for (uint32_t k = threadIdx.x; k < p.nsym; k += blockDim.x) {
    uint32_t t = 0;
    for (uint32_t f = c0; f < c1; ++f)
      if (s.status[f] == ROIBIN_OK) t += s.hist[(size_t)f * kMaxSymbols + k];
    hsum[k] = t;
  }
  __syncthreads();
  const int st = build_codebook(hsum, p.nsym, h, s.cb_len + (size_t)head * kMaxSymbols,
                                s.cb_code + (size_t)head * kMaxSymbols);
  __syncthreads();
  for (uint32_t f = (uint32_t)head + 1; f < c1; ++f) {
    if (s.status[f] != ROIBIN_OK) continue;
    for (uint32_t k = threadIdx.x; k < p.nsym; k += blockDim.x) {
      s.cb_len[(size_t)f * kMaxSymbols + k] = s.cb_len[(size_t)head * kMaxSymbols + k];
      s.cb_code[(size_t)f * kMaxSymbols + k] = s.cb_code[(size_t)head * kMaxSymbols + k];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (uint32_t f = (uint32_t)head; f < c1; ++f) {
      if (s.status[f] != ROIBIN_OK) continue;
      s.chunk_ref[f] = f - (uint32_t)head;
      if (st != ROIBIN_OK) s.status[f] = st;
    }
}

// ---------------------------------------------------------------------------
// chunks: bits, Lorenzo outliers and prequantisation outliers per chunk.
constexpr int kChunkThreads = 128;  // 32 symbols per thread
__global__ void __launch_bounds__(kChunkThreads) k_chunks(DevParams p, Scratch s) {
  __shared__ uint8_t len[kMaxSymbols];
  __shared__ uint32_t red[3][kChunkThreads / 32];
  const uint32_t k = blockIdx.x, f = blockIdx.y;
  for (uint32_t i = threadIdx.x; i < p.nsym; i += kChunkThreads) len[i] = s.cb_len[(size_t)f * kMaxSymbols + i];
  __syncthreads();
  const uint16_t* codes = s.codes + (size_t)f * ((size_t)p.n_chunks * kChunk) + (size_t)k * kChunk;
  const uint32_t first = k * kChunk + threadIdx.x * 32;
  uint32_t bits = 0, lo = 0, pq = 0;
  const uint4* v = reinterpret_cast<const uint4*>(codes + threadIdx.x * 32);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 w = v[q];
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const uint32_t idx = first + q * 8 + h;
      const uint32_t c16 = (ww[h >> 1] >> ((h & 1) * 16)) & 0xFFFFu;
      if (idx < p.M) {
        const uint32_t code = c16 & 0x3FFu;
        bits += len[code];
        lo += code == 0;
        pq += c16 >> 15;
      }
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    bits += __shfl_xor_sync(0xffffffffu, bits, d);
    lo += __shfl_xor_sync(0xffffffffu, lo, d);
    pq += __shfl_xor_sync(0xffffffffu, pq, d);
  }
  if (lane_id() == 0) {
    red[0][threadIdx.x >> 5] = bits;
    red[1][threadIdx.x >> 5] = lo;
    red[2][threadIdx.x >> 5] = pq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tb = 0, tl = 0, tp = 0;
    for (int w = 0; w < kChunkThreads / 32; ++w) {
      tb += red[0][w];
      tl += red[1][w];
      tp += red[2][w];
    }
    const size_t o = (size_t)f * p.n_chunks + k;
    s.chunk_words[o] = (tb + 31) / 32;
    s.chunk_lo[o] = tl;
    s.chunk_pq[o] = tp;
  }
}

// ---------------------------------------------------------------------------
// plan: one block per frame.  Turns the per-chunk counts into offsets, lays
// out the frame, checks the output stride, and writes the header, the peaks,
// the code lengths, the chunk index and every padding byte.
__device__ inline void zero_bytes(uint8_t* base, uint64_t from, uint64_t to) {
  for (uint64_t b = from + threadIdx.x; b < to; b += blockDim.x) base[b] = 0;
}

__global__ void __launch_bounds__(1024) k_plan(DevParams p, Scratch s, PlainArgs a) {
  __shared__ uint32_t tmp[33];
  __shared__ uint32_t carry[3];
  const uint32_t f = blockIdx.x;
  int st = s.status[f];
  if (st != ROIBIN_OK) {
    if (threadIdx.x == 0) {
      a.frame_bytes[f] = 0;
      a.frame_status[f] = st;
      FramePlan pl = {};
      s.plan[f] = pl;
    }
    return;
  }
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  uint32_t* cw = s.chunk_words + (size_t)f * p.n_chunks;
  uint32_t* cl = s.chunk_lo + (size_t)f * p.n_chunks;
  uint32_t* cp = s.chunk_pq + (size_t)f * p.n_chunks;
  for (uint32_t k0 = 0; k0 < p.n_chunks; k0 += blockDim.x) {
    const uint32_t k = k0 + threadIdx.x;
    const uint32_t w = k < p.n_chunks ? cw[k] : 0u;
    const uint32_t l = k < p.n_chunks ? cl[k] : 0u;
    const uint32_t q = k < p.n_chunks ? cp[k] : 0u;
    uint32_t tw, tl, tq;
    const uint32_t ew = block_excl_scan(w, tmp, &tw);
    const uint32_t el = block_excl_scan(l, tmp, &tl);
    const uint32_t eq = block_excl_scan(q, tmp, &tq);
    if (k < p.n_chunks) {
      cw[k] = carry[0] + ew;
      cl[k] = carry[1] + el;
      cp[k] = carry[2] + eq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += tw;
      carry[1] += tl;
      carry[2] += tq;
    }
    __syncthreads();
  }
  FramePlan pl;
  pl.n_peaks = s.peak_count[f];
  pl.n_words = carry[0];
  pl.n_lo = carry[1];
  pl.n_pq = carry[2];
  pl.off_peaks = kHeaderBytes;
  pl.off_roi = pl.off_peaks + align16((uint64_t)pl.n_peaks * 6);
  const uint32_t ref = p.chunk > 1 ? s.chunk_ref[f] : 0u;  // the code lengths live in the chunk's head
  pl.off_len = pl.off_roi + roi_in_place_bytes(p, pl.n_peaks);
  pl.off_cidx = pl.off_len + (ref == 0 ? align16(p.nsym) : 0);
  pl.off_lo = pl.off_cidx + align16((uint64_t)p.n_chunks * 4);
  pl.off_pq = pl.off_lo + align16((uint64_t)pl.n_lo * 8);
  pl.off_bits = pl.off_pq + align16((uint64_t)pl.n_pq * 8);
  pl.total = pl.off_bits + align16((uint64_t)pl.n_words * 4);
  if (pl.total > a.out_stride) st = ROIBIN_ERR_CAPACITY;
  if (threadIdx.x == 0) {
    s.plan[f] = pl;
    s.status[f] = st;
    a.frame_bytes[f] = pl.total;
    a.frame_status[f] = st;
  }
  if (st != ROIBIN_OK) return;
  if (!RB_CHECK(s, pl.total <= a.out_stride, ROIBIN_CHECK_PLAN_TOTAL)) return;

  uint8_t* out = a.out + (size_t)f * a.out_stride;
  if (threadIdx.x == 0) {
    uint32_t* h = reinterpret_cast<uint32_t*>(out);
    h[0] = kMagic;
    h[1] = kVersion;
    h[2] = p.P;
    h[3] = p.H;
    h[4] = p.W;
    h[5] = (uint32_t)p.roi_h | ((uint32_t)p.roi_w << 16);
    h[6] = (uint32_t)p.bh | ((uint32_t)p.bw << 16);
    h[7] = __float_as_uint(p.eb);
    h[8] = (uint32_t)p.R;
    h[9] = pl.n_peaks;
    h[10] = pl.n_lo;
    h[11] = pl.n_pq;
    h[12] = p.M;
    h[13] = kChunk;
    h[14] = p.n_chunks;
    h[15] = pl.n_words;
    h[16] = (uint32_t)(pl.total & 0xFFFFFFFFu);
    h[17] = (uint32_t)(pl.total >> 32);
    h[18] = p.dims == 2 ? 0u : (uint32_t)p.dims;  // Lorenzo dimension, 0 for the default 2
    for (int i = 19; i < 24; ++i) h[i] = 0;
    h[22] = ref;  // frames back to the stream with the code lengths (0: this one)
  }
  // peaks (u16 triples) + padding
  const uint32_t* keys = s.peak_key + (size_t)f * p.max_peaks;
  uint16_t* pk = reinterpret_cast<uint16_t*>(out + pl.off_peaks);
  for (uint32_t k = threadIdx.x; k < pl.n_peaks; k += blockDim.x) {
    const uint32_t px = keys[k];
    const uint32_t pn = px / (p.H * p.W), rem = px - pn * p.H * p.W;
    pk[3 * k] = (uint16_t)pn;
    pk[3 * k + 1] = (uint16_t)(rem / p.W);
    pk[3 * k + 2] = (uint16_t)(rem % p.W);
  }
  zero_bytes(out, pl.off_peaks + (uint64_t)pl.n_peaks * 6, pl.off_roi);
  zero_bytes(out, pl.off_roi + (p.roi_coder ? 0 : (uint64_t)pl.n_peaks * p.roi_h * p.roi_w * 4), pl.off_len);
  // code lengths + padding (a chunk's head only)
  if (ref == 0) {
    for (uint32_t k = threadIdx.x; k < p.nsym; k += blockDim.x)
      out[pl.off_len + k] = s.cb_len[(size_t)f * kMaxSymbols + k];
    zero_bytes(out, pl.off_len + p.nsym, pl.off_cidx);
  }
  // chunk index + padding
  uint32_t* ci = reinterpret_cast<uint32_t*>(out + pl.off_cidx);
  for (uint32_t k = threadIdx.x; k < p.n_chunks; k += blockDim.x) ci[k] = cw[k];
  zero_bytes(out, pl.off_cidx + (uint64_t)p.n_chunks * 4, pl.off_lo);
  zero_bytes(out, pl.off_lo + (uint64_t)pl.n_lo * 8, pl.off_pq);
  zero_bytes(out, pl.off_pq + (uint64_t)pl.n_pq * 8, pl.off_bits);
  zero_bytes(out, pl.off_bits + (uint64_t)pl.n_words * 4, pl.total);
}

// ---------------------------------------------------------------------------
// encode: one block per chunk writes its words of the bitstream and its
// Lorenzo and prequantisation outliers, in bin order.
__global__ void __launch_bounds__(kChunkThreads) k_encode(DevParams p, Scratch s, PlainArgs a) {
  __shared__ uint8_t len[kMaxSymbols];
  __shared__ uint32_t cwd[kMaxSymbols];
  __shared__ uint32_t buf[kChunk];  // worst case: 4096 codes of 32 bits
  __shared__ uint32_t tmp[33];
  const uint32_t k = blockIdx.x, f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  for (uint32_t i = threadIdx.x; i < p.nsym; i += kChunkThreads) {
    len[i] = s.cb_len[(size_t)f * kMaxSymbols + i];
    cwd[i] = s.cb_code[(size_t)f * kMaxSymbols + i];
  }
  __syncthreads();
  const uint16_t* codes = s.codes + (size_t)f * ((size_t)p.n_chunks * kChunk) + (size_t)k * kChunk;
  const uint32_t first = k * kChunk + threadIdx.x * 32;
  uint16_t c[32];
  const uint4* v = reinterpret_cast<const uint4*>(codes + threadIdx.x * 32);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 w = v[q];
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 8; ++h) c[q * 8 + h] = (uint16_t)((ww[h >> 1] >> ((h & 1) * 16)) & 0xFFFFu);
  }
  uint32_t bits = 0, nlo = 0, npq = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    if (first + i < p.M) {
      bits += len[c[i] & 0x3FFu];
      nlo += (c[i] & 0x3FFu) == 0;
      npq += c[i] >> 15;
    }
  }
  uint32_t tot_bits, tot_lo, tot_pq;
  uint32_t pos = block_excl_scan(bits, tmp, &tot_bits);
  uint32_t lo_rank = block_excl_scan(nlo, tmp, &tot_lo);
  uint32_t pq_rank = block_excl_scan(npq, tmp, &tot_pq);
  const uint32_t n_words = (tot_bits + 31) / 32;
  for (uint32_t w = threadIdx.x; w < n_words; w += kChunkThreads) buf[w] = 0;
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    if (first + i < p.M) {
      const uint32_t code = c[i] & 0x3FFu;
      const uint32_t L = len[code];
      put_bits(buf, pos, cwd[code], L);
      pos += L;
    }
  }
  __syncthreads();
  const FramePlan& pl = s.plan[f];
  uint8_t* out = a.out + (size_t)f * a.out_stride;
  const size_t o = (size_t)f * p.n_chunks + k;
  uint32_t* dst = reinterpret_cast<uint32_t*>(out + pl.off_bits) + s.chunk_words[o];
  if (RB_CHECK(s, s.chunk_words[o] + n_words <= pl.n_words, ROIBIN_CHECK_BITSTREAM))
    for (uint32_t w = threadIdx.x; w < n_words; w += kChunkThreads) dst[w] = buf[w];
  if ((tot_lo | tot_pq) && RB_CHECK(s, s.chunk_lo[o] + lo_rank + nlo <= pl.n_lo &&
                                            s.chunk_pq[o] + pq_rank + npq <= pl.n_pq, ROIBIN_CHECK_OUTLIERS)) {
    uint2* lo_out = reinterpret_cast<uint2*>(out + pl.off_lo) + s.chunk_lo[o] + lo_rank;
    uint2* pq_out = reinterpret_cast<uint2*>(out + pl.off_pq) + s.chunk_pq[o] + pq_rank;
    for (int i = 0; i < 32; ++i) {
      const uint32_t idx = first + i;
      if (idx >= p.M) break;
      if ((c[i] & 0x3FFu) == 0) {
        *lo_out++ = make_uint2(idx, (uint32_t)s.lo_delta[(size_t)f * p.M + idx]);
      }
      if (c[i] >> 15) *pq_out++ = make_uint2(idx, s.pq_bits[(size_t)f * p.M + idx]);
    }
  }
}

// ---------------------------------------------------------------------------
// roi: one warp per peak copies its window (fill 0 past the panel edge).
__global__ void __launch_bounds__(256) k_roi(DevParams p, Scratch s, PlainArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const FramePlan& pl = s.plan[f];
  const uint32_t k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= pl.n_peaks) return;
  const uint32_t px = s.peak_key[(size_t)f * p.max_peaks + k];
  const uint32_t pn = px / (p.H * p.W), rem = px - pn * p.H * p.W;
  const int r = (int)(rem / p.W), c = (int)(rem % p.W);
  const float* panel = a.frames + (size_t)f * p.frame_px + (size_t)pn * p.H * p.W;
  float* dst = reinterpret_cast<float*>(a.out + (size_t)f * a.out_stride + pl.off_roi) +
               (size_t)k * p.roi_h * p.roi_w;
  if (RB_CHECK(s, pl.off_roi + (uint64_t)(k + 1) * p.roi_h * p.roi_w * 4 <= pl.total, ROIBIN_CHECK_ROI))
    warp_copy_roi(panel, p.H, p.W, r, c, p.roi_h, p.roi_w, dst);
}

// last_peaks: peak lists of the last call as (panel, row, col) triples.
__global__ void k_last_peaks(DevParams p, Scratch s, uint16_t* peaks, uint32_t* npeaks) {
  const uint32_t f = blockIdx.x;
  const uint32_t count = s.peak_count[f];
  if (threadIdx.x == 0) npeaks[f] = count;
  const uint32_t n = min(count, p.max_peaks);
  for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
    const uint32_t px = s.peak_key[(size_t)f * p.max_peaks + k];
    const uint32_t pn = px / (p.H * p.W), rem = px - pn * p.H * p.W;
    uint16_t* o = peaks + ((size_t)f * p.max_peaks + k) * 3;
    o[0] = (uint16_t)pn;
    o[1] = (uint16_t)(rem / p.W);
    o[2] = (uint16_t)(rem % p.W);
  }
}

// ---------------------------------------------------------------------------
// launchers
static size_t stream_smem_bytes(const DevParams& p, uint32_t rows_per_step) {
  const size_t q_rows = (size_t)(rows_per_step + 1) * p.Wb * 4;
  return sizeof(StreamSmem) + q_rows + align16((uint64_t)rows_per_step * p.Wb) + (p.dims == 3 ? q_rows : 0);
}

cudaError_t launch_reset(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st) {
  const uint32_t blocks = min(1024u, ceil_div(n * kMaxSymbols, 256));
  k_reset<<<blocks, 256, 0, st>>>(p, s, n);
  return cudaGetLastError();
}

cudaError_t launch_stream(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  const bool vec4 = p.bh == 2 && p.bw == 2 && (p.W % 4) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.frames) % 16) == 0;
  const size_t smem = stream_smem_bytes(p, a.rows_per_step);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_stream, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(a.bands_per_panel * p.P, a.n_frames);
  k_stream<<<grid, kStreamThreads, smem, st>>>(p, s, a, vec4 ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_peaks(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  if (a.user_peaks) return cudaSuccess;
  const int side = 2 * peak_reach(p) + 1;
  const size_t smem = (size_t)kPeakWarps * side * side * sizeof(float);
  dim3 grid(kPeakBlocks, a.n_frames);
  k_peaks<<<grid, kPeakWarps * 32, smem, st>>>(p, s, a);
  return cudaGetLastError();
}

cudaError_t launch_peaks_final(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  uint32_t n2 = 1;
  while (n2 < p.max_peaks) n2 <<= 1;
  const size_t smem = (size_t)n2 * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_peaks_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_peaks_final<<<a.n_frames, 1024, smem, st>>>(p, s, a);
  return cudaGetLastError();
}

cudaError_t launch_huffman(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_huffman, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(align16(sizeof(HuffSmem)) + kMaxSymbols * 4));
    attr_set = true;
  }
  k_huffman<<<ceil_div(n, p.chunk), 1024, align16(sizeof(HuffSmem)) + kMaxSymbols * 4, st>>>(p, s, n);
  return cudaGetLastError();
}

cudaError_t launch_chunks(const DevParams& p, const Scratch& s, uint32_t n, cudaStream_t st) {
  dim3 grid(p.n_chunks, n);
  k_chunks<<<grid, kChunkThreads, 0, st>>>(p, s);
  return cudaGetLastError();
}

cudaError_t launch_plan(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  k_plan<<<a.n_frames, 1024, 0, st>>>(p, s, a);
  return cudaGetLastError();
}

cudaError_t launch_encode(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  dim3 grid(p.n_chunks, a.n_frames);
  k_encode<<<grid, kChunkThreads, 0, st>>>(p, s, a);
  return cudaGetLastError();
}

cudaError_t launch_roi(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st) {
  if (p.max_peaks == 0) return cudaSuccess;
  dim3 grid(ceil_div(p.max_peaks, 8), a.n_frames);
  k_roi<<<grid, 256, 0, st>>>(p, s, a);
  return cudaGetLastError();
}

cudaError_t launch_last_peaks(const DevParams& p, const Scratch& s, uint16_t* peaks, uint32_t* npeaks,
                              uint32_t n, cudaStream_t st) {
  k_last_peaks<<<n, 256, 0, st>>>(p, s, peaks, npeaks);
  return cudaGetLastError();
}

}  // namespace roibin
