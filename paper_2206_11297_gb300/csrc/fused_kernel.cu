// fused_kernel.cu - the persistent cluster kernel: the whole method for a
// batch of frames in one launch.
//
// A cluster of C CTAs owns one frame at a time (frames c, c + n_clusters, ...).
// The frame's binned rows are split into C contiguous ranges, one per CTA.
//
// Phase 1 (per CTA, HBM-bound): raw rows stream into a ring of shared-memory
// stages by TMA bulk copies (cp.async.bulk + mbarrier); each stage is binned,
// prequantised, Lorenzo-predicted and coded.  The codes stay on chip: one
// byte per bin in the CTA's shared memory (byte = residual + 128 for
// |residual| <= 126, 0 = Lorenzo outlier, 255 = escape to a side array), so a
// CSPAD frame's 577,344 codes fit in the cluster's distributed shared memory.
// Pixels >= amax_thr are listed for the peak finder.
//
// Phase 2 (per cluster): candidate evaluation (a1, a2), the cluster-wide
// histogram read through distributed shared memory and the Huffman codebook
// (a9, built redundantly by every CTA), then per-chunk sizes, a cluster-wide
// scan, the frame layout, and the chunk-parallel bit-packing (a10) with the
// outliers (a11) and the ROI windows (a3) written straight to the output.
//
// Frames never exchange data, so the clusters never wait on one another;
// within a cluster, cluster barriers order the phases.  Every wait on an
// mbarrier is bounded: on timeout the frame is marked ROIBIN_ERR_TIMEOUT.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "roibin_internal.cuh"

namespace cg = cooperative_groups;

namespace roibin {

constexpr int kFT = 512;       // threads per CTA
constexpr int kFW = kFT / 32;  // warps per CTA
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier wait

struct FusedMisc {
  FramePlan pl;
  int32_t status;
  int32_t timeout;
  uint32_t n_peaks;
  uint32_t bad;
  uint32_t tmp[33];
  uint32_t carry[3];
};

// ---- small PTX helpers ------------------------------------------------------
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// ---- geometry helpers (bin 2x2) ---------------------------------------------
// First raw row (global numbering p * H + r) of global binned row g.
__device__ __forceinline__ uint32_t raw_begin(const DevParams& p, uint32_t g) {
  const uint32_t pn = g / p.Hb, i = g - pn * p.Hb;
  return pn * p.H + 2 * i;
}
__device__ __forceinline__ uint32_t raw_end(const DevParams& p, uint32_t g) {
  const uint32_t pn = g / p.Hb, i = g - pn * p.Hb;
  return pn * p.H + min(2 * i + 2, p.H);
}

// Symbol of a stored byte.
__device__ __forceinline__ uint32_t byte_code(uint32_t b, uint32_t bin, const DevParams& p,
                                              const uint16_t* esc) {
  if (b == 0) return 0;
  if (b == 255) return __ldcg(esc + bin);
  return b - 128 + (uint32_t)p.R;
}

struct Layout {
  uint64_t* bars;
  uint32_t* hist;       // [kMaxSymbols] this CTA's histogram
  uint8_t* cb_len;      // [kMaxSymbols]
  uint32_t* cb_code;    // [kMaxSymbols]
  uint32_t* own;        // [3][chunks_per_cta] per-chunk words / lo / pq of own chunks
  FusedMisc* misc;
  uint32_t* pq;         // [cap_bins / 32 + 1] prequantisation-outlier bits of own bins
  int32_t* qbuf;        // [(RB + 1) * Wb]
  uint8_t* codes;       // [cap_bins (+16)]
  unsigned char* un;    // union: ring | peak-test buffers | Huffman scratch | keys + chunk scans
};

__device__ __forceinline__ Layout layout_of(unsigned char* sm, const FusedShape& sh) {
  Layout L;
  L.bars = reinterpret_cast<uint64_t*>(sm + sh.off_bar);
  L.hist = reinterpret_cast<uint32_t*>(sm + sh.off_hist);
  L.cb_len = sm + sh.off_cb_len;
  L.cb_code = reinterpret_cast<uint32_t*>(sm + sh.off_cb_code);
  L.own = reinterpret_cast<uint32_t*>(sm + sh.off_own);
  L.misc = reinterpret_cast<FusedMisc*>(sm + sh.off_misc);
  L.pq = reinterpret_cast<uint32_t*>(sm + sh.off_pq);
  L.qbuf = reinterpret_cast<int32_t*>(sm + sh.off_qbuf);
  L.codes = sm + sh.off_codes;
  L.un = sm + sh.off_union;
  return L;
}

// q of one global binned row straight from global memory (the halo row above a
// CTA's range when that range starts inside a panel).
__device__ void halo_row(const float* frame, const DevParams& p, uint32_t g, int32_t* qrow) {
  const uint32_t pn = g / p.Hb, i = g - pn * p.Hb;
  const float* panel = frame + (size_t)pn * p.H * p.W;
  const uint32_t NP = p.W >> 2;
  for (uint32_t pr = threadIdx.x; pr < NP; pr += kFT) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(panel + (size_t)(2 * i) * p.W) + pr);
    const bool two = 2 * i + 1 < p.H;
    const float4 b = two ? __ldg(reinterpret_cast<const float4*>(panel + (size_t)(2 * i + 1) * p.W) + pr)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    float v0, v1;
    bin_pair(a, b, two, v0, v1);
    qrow[2 * pr] = prequantize(v0, p).q;
    qrow[2 * pr + 1] = prequantize(v1, p).q;
  }
}

// Writes the header, the peaks, the code lengths, the chunk index and every
// padding byte of a frame (block-cooperative).  keys: pixel index per peak.
__device__ void write_frame_head(uint8_t* out, const DevParams& p, const FramePlan& pl, const uint32_t* keys,
                                 const uint8_t* cb_len, const uint32_t* chunk_word_off) {
  if (threadIdx.x == 0) {
    uint32_t h[24];
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
    for (int i = 18; i < 24; ++i) h[i] = 0;
    uint4* o4 = reinterpret_cast<uint4*>(out);
    for (int i = 0; i < 6; ++i) o4[i] = make_uint4(h[4 * i], h[4 * i + 1], h[4 * i + 2], h[4 * i + 3]);
  }
  const uint32_t plane = p.H * p.W;
  uint16_t* pk = reinterpret_cast<uint16_t*>(out + pl.off_peaks);
  for (uint32_t k = threadIdx.x; k < pl.n_peaks; k += blockDim.x) {
    const uint32_t px = keys[k];
    const uint32_t pn = px / plane, rem = px - pn * plane;
    pk[3 * k] = (uint16_t)pn;
    pk[3 * k + 1] = (uint16_t)(rem / p.W);
    pk[3 * k + 2] = (uint16_t)(rem % p.W);
  }
  auto zero = [&](uint64_t from, uint64_t to) {
    for (uint64_t b = from + threadIdx.x; b < to; b += blockDim.x) out[b] = 0;
  };
  zero(pl.off_peaks + (uint64_t)pl.n_peaks * 6, pl.off_roi);
  zero(pl.off_roi + (uint64_t)pl.n_peaks * p.roi_h * p.roi_w * 4, pl.off_len);
  for (uint32_t k = threadIdx.x; k < p.nsym; k += blockDim.x) out[pl.off_len + k] = cb_len[k];
  zero(pl.off_len + p.nsym, pl.off_cidx);
  uint32_t* ci = reinterpret_cast<uint32_t*>(out + pl.off_cidx);
  for (uint32_t k = threadIdx.x; k < p.n_chunks; k += blockDim.x) ci[k] = chunk_word_off[k];
  zero(pl.off_cidx + (uint64_t)p.n_chunks * 4, pl.off_lo);
  zero(pl.off_lo + (uint64_t)pl.n_lo * 8, pl.off_pq);
  zero(pl.off_pq + (uint64_t)pl.n_pq * 8, pl.off_bits);
  zero(pl.off_bits + (uint64_t)pl.n_words * 4, pl.total);
}

__device__ __forceinline__ uint32_t chunk_begin_of(uint32_t rank, const FusedShape& sh, const DevParams& p) {
  const uint64_t b = (uint64_t)rank * sh.cap_bins;
  const uint64_t k = (b + kChunk - 1) / kChunk;
  return k < p.n_chunks ? (uint32_t)k : p.n_chunks;
}

__global__ void __launch_bounds__(kFT, 1) k_fused(DevParams p, Scratch fs, PlainArgs a, FusedShape sh) {
  extern __shared__ __align__(128) unsigned char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const uint32_t rank = cl.block_rank();
  const uint32_t C = sh.C;
  const uint32_t cid = blockIdx.x / C;
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  Layout L = layout_of(sm, sh);
  FusedMisc& ms = *L.misc;

  const uint32_t g_total = p.P * p.Hb;
  const uint32_t g0 = min(g_total, rank * sh.rows_per_cta);
  const uint32_t g1 = min(g_total, g0 + sh.rows_per_cta);
  const uint32_t bin0 = g0 * p.Wb;  // first bin owned by this CTA
  const uint32_t n_steps = g1 > g0 ? ceil_div(g1 - g0, sh.RB) : 0;
  const uint32_t k_lo = chunk_begin_of(rank, sh, p), k_hi = chunk_begin_of(rank + 1, sh, p);
  const uint32_t NP = p.W >> 2;
  const int side = 2 * peak_reach(p) + 1;

  // slot-local global scratch
  uint32_t* thr_count = fs.thr_count + cid;
  uint32_t* thr_idx = fs.thr_idx + (size_t)cid * p.thr_cap;
  uint32_t* peak_count = fs.peak_count + cid;
  uint32_t* peak_key = fs.peak_key + (size_t)cid * (p.max_peaks ? p.max_peaks : 1);
  int32_t* lo_delta = fs.lo_delta + (size_t)cid * p.M;
  uint32_t* pq_bits = fs.pq_bits + (size_t)cid * p.M;
  uint16_t* esc = fs.codes + (size_t)cid * p.M;

  if (tid == 0) {
    for (uint32_t b = 0; b < sh.stages; ++b) mbar_init(L.bars + b, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t ring_iter = 0;  // stages consumed so far (uniform in the CTA)

  for (uint32_t f = cid; f < a.n_frames; f += sh.n_clusters) {
    const float* frame = a.frames + (size_t)f * p.frame_px;
    uint8_t* out = a.out + (size_t)f * a.out_stride;
    // ================= phase 1: stream, bin, quantise, predict, code =================
    for (uint32_t k = tid; k < p.nsym; k += kFT) L.hist[k] = 0;
    for (uint32_t k = tid; k < sh.cap_bins / 32 + 1; k += kFT) L.pq[k] = 0;
    if (tid == 0) ms.timeout = 0;
    auto issue = [&](uint32_t st) {  // thread 0 only
      const uint32_t gA = g0 + st * sh.RB, gB = min(g1, gA + sh.RB);
      const uint32_t r0 = raw_begin(p, gA), r1 = raw_end(p, gB - 1);
      const uint32_t slot = (ring_iter + st) % sh.stages;
      const uint32_t bytes = (r1 - r0) * p.W * 4;
      fence_proxy_async();
      mbar_expect_tx(L.bars + slot, bytes);
      tma_load_1d(L.un + (size_t)slot * sh.stage_bytes, frame + (size_t)r0 * p.W, bytes, L.bars + slot);
    };
    if (tid == 0)
      for (uint32_t st = 0; st < min(sh.stages, n_steps); ++st) issue(st);
    // the row above the range
    if (g0 > 0 && g0 % p.Hb != 0 && g0 < g1) halo_row(frame, p, g0 - 1, L.qbuf);
    else
      for (uint32_t j = tid; j < p.Wb; j += kFT) L.qbuf[j] = 0;
    __syncthreads();

    for (uint32_t st = 0; st < n_steps; ++st) {
      const uint32_t slot = (ring_iter + st) % sh.stages;
      const uint32_t parity = ((ring_iter + st) / sh.stages) & 1u;
      const uint32_t gA = g0 + st * sh.RB, rows = min(sh.RB, g1 - gA);
      const uint32_t rA = raw_begin(p, gA);
      if (!mbar_wait(L.bars + slot, parity)) ms.timeout = 1;
      const float4* ring = reinterpret_cast<const float4*>(L.un + (size_t)slot * sh.stage_bytes);
      // phase A: q of every bin of the stage
      const uint32_t items = rows * NP;
      for (uint32_t it = tid; it < items; it += kFT) {
        const uint32_t il = it / NP, pr = it - il * NP;
        const uint32_t g = gA + il;
        const uint32_t pn = g / p.Hb, i = g - pn * p.Hb;
        const uint32_t ra = pn * p.H + 2 * i - rA;
        const bool two = 2 * i + 1 < p.H;
        const float4 va = ring[(size_t)ra * NP + pr];
        const float4 vb = two ? ring[(size_t)(ra + 1) * NP + pr] : make_float4(0.f, 0.f, 0.f, 0.f);
        float v0, v1;
        bin_pair(va, vb, two, v0, v1);
        const Quant q0 = prequantize(v0, p), q1 = prequantize(v1, p);
        *reinterpret_cast<int2*>(L.qbuf + (size_t)(il + 1) * p.Wb + 2 * pr) = make_int2(q0.q, q1.q);
        const uint32_t lb = (g - g0) * p.Wb + 2 * pr;  // local bin of the pair
        if (q0.outlier | q1.outlier) {
          atomicOr(L.pq + (lb >> 5), ((uint32_t)q0.outlier | ((uint32_t)q1.outlier << 1)) << (lb & 31));
          if (q0.outlier) pq_bits[bin0 + lb] = q0.outlier_bits;
          if (q1.outlier) pq_bits[bin0 + lb + 1] = q1.outlier_bits;
        }
        const float m = fmaxf(fmaxf(fmaxf(va.x, va.y), fmaxf(va.z, va.w)),
                              fmaxf(fmaxf(vb.x, vb.y), fmaxf(vb.z, vb.w)));
        if (m >= p.amax) {
          const float px[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
          const int npx = two ? 8 : 4;
          for (int k = 0; k < npx; ++k) {
            if (px[k] >= p.amax) {
              const uint32_t r = 2 * i + (k >> 2), col = 4 * pr + (k & 3);
              const uint32_t s = atomicAdd(thr_count, 1u);
              if (s < p.thr_cap) thr_idx[s] = (pn * p.H + r) * p.W + col;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0 && st + sh.stages < n_steps) issue(st + sh.stages);  // the slot is free again
      // phase B: residuals, codes, histogram, outliers
      const uint32_t iters = ceil_div(items, kFT);
      for (uint32_t t = 0; t < iters; ++t) {
        const uint32_t it = t * kFT + tid;
        uint32_t c0 = 0xFFFFu, c1 = 0xFFFFu;
        if (it < items) {
          const uint32_t il = it / NP, pr = it - il * NP;
          const uint32_t g = gA + il;
          const uint32_t i = g % p.Hb;
          const uint32_t j0 = 2 * pr;
          const int32_t* cur = L.qbuf + (size_t)(il + 1) * p.Wb;
          const int32_t* up = L.qbuf + (size_t)il * p.Wb;
          const int2 qc = *reinterpret_cast<const int2*>(cur + j0);
          int2 qu = make_int2(0, 0);
          if (i > 0) qu = *reinterpret_cast<const int2*>(up + j0);
          const int32_t ql = j0 > 0 ? cur[j0 - 1] : 0;
          const int32_t qd = (j0 > 0 && i > 0) ? up[j0 - 1] : 0;
          const int32_t d0 = qc.x - qu.x - ql + qd;
          const int32_t d1 = qc.y - qu.y - qc.x + qu.x;
          c0 = quant_code(d0, p.R);
          c1 = quant_code(d1, p.R);
          const uint32_t lb = (g - g0) * p.Wb + j0;
          auto to_byte = [&](int32_t d, uint32_t c, uint32_t bin) -> uint32_t {
            if (c == 0) {
              lo_delta[bin] = d;
              return 0u;
            }
            if (d >= -127 && d <= 126) return (uint32_t)(d + 128);
            esc[bin] = (uint16_t)c;
            return 255u;
          };
          const uint32_t b0 = to_byte(d0, c0, bin0 + lb), b1 = to_byte(d1, c1, bin0 + lb + 1);
          *reinterpret_cast<uint16_t*>(L.codes + lb) = (uint16_t)(b0 | (b1 << 8));
        }
        hist_add_warp(L.hist, c0, (uint32_t)p.R);
        hist_add_warp(L.hist, c1, (uint32_t)p.R);
      }
      __syncthreads();
      for (uint32_t j = tid; j < p.Wb; j += kFT) L.qbuf[j] = L.qbuf[(size_t)rows * p.Wb + j];
      __syncthreads();
    }
    ring_iter += n_steps;

    // ================= phase 2 =================
    cl.sync();  // A: codes, histograms and the amax list of the frame are complete
    const bool user = a.user_peaks != nullptr;
    if (!user) {  // a1 + a2: candidates, one warp per listed pixel
      float* nb = reinterpret_cast<float*>(L.un) + warp * side * side;
      const uint32_t cnt = __ldcg(thr_count);
      const uint32_t plane = p.H * p.W;
      auto test = [&](uint32_t px) {
        const uint32_t pn = px / plane, rem = px - pn * plane;
        const uint32_t r = rem / p.W, c = rem - r * p.W;
        const float* panel = frame + (size_t)pn * plane;
        if (warp_peak_test(panel, p.H, p.W, r, c, p, nb, [](const float* q) { return __ldg(q); }) &&
            lane == 0) {
          const uint32_t s = atomicAdd(peak_count, 1u);
          if (s < p.max_peaks) peak_key[s] = px;
        }
      };
      const uint32_t gw = rank * kFW + warp, nw = C * kFW;
      if (cnt <= p.thr_cap) {
        for (uint32_t e = gw; e < cnt; e += nw) test(__ldcg(thr_idx + e));
      } else {
        for (uint64_t base = (uint64_t)gw * 32; base < p.frame_px; base += (uint64_t)nw * 32) {
          const uint64_t px = base + lane;
          const bool hot = px < p.frame_px && __ldg(frame + px) >= p.amax;
          uint32_t m = __ballot_sync(0xffffffffu, hot);
          while (m) {
            const uint32_t l = __ffs(m) - 1;
            m &= m - 1;
            test((uint32_t)(base + l));
          }
        }
      }
    }
    __syncthreads();
    // a8 + a9: cluster histogram and codebook (every CTA builds the same one)
    HuffSmem& hs = *reinterpret_cast<HuffSmem*>(L.un);
    uint32_t* total = reinterpret_cast<uint32_t*>(L.un + sizeof(HuffSmem));
    for (uint32_t s = tid; s < p.nsym; s += kFT) {
      uint32_t v = 0;
      for (uint32_t r = 0; r < C; ++r) v += cl.map_shared_rank(L.hist, r)[s];
      total[s] = v;
    }
    __syncthreads();
    const int cb_status = build_codebook(total, p.nsym, hs, L.cb_len, L.cb_code);
    cl.sync();  // B: the peak list is complete
    // the frame's peaks: keys in the union (sorted when found, as given when supplied)
    uint32_t* keys = reinterpret_cast<uint32_t*>(L.un);
    if (tid == 0) {
      ms.status = cb_status;
      ms.bad = 0;
    }
    __syncthreads();
    uint32_t n_pk;
    if (user) {
      n_pk = a.user_npeaks[f];
      if (n_pk > p.max_peaks) {
        if (tid == 0 && ms.status == ROIBIN_OK) ms.status = ROIBIN_ERR_CAPACITY;
      } else {
        const uint16_t* up = a.user_peaks + (size_t)f * p.max_peaks * 3;
        for (uint32_t k = tid; k < n_pk; k += kFT) {
          const uint32_t pn = up[3 * k], r = up[3 * k + 1], c = up[3 * k + 2];
          if (pn >= p.P || r >= p.H || c >= p.W) ms.bad = 1;
          else keys[k] = (pn * p.H + r) * p.W + c;
        }
        __syncthreads();
        if (tid == 0 && ms.bad && ms.status == ROIBIN_OK) ms.status = ROIBIN_ERR_INVALID_ARG;
      }
    } else {
      n_pk = __ldcg(peak_count);
      if (n_pk > p.max_peaks) {
        if (tid == 0 && ms.status == ROIBIN_OK) ms.status = ROIBIN_ERR_CAPACITY;
      } else {
        uint32_t n2 = 1;
        while (n2 < n_pk) n2 <<= 1;
        for (uint32_t k = tid; k < n2; k += kFT) keys[k] = k < n_pk ? __ldcg(peak_key + k) : 0xFFFFFFFFu;
        __syncthreads();
        for (uint32_t size = 2; size <= n2; size <<= 1) {
          for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t k = tid; k < n2; k += kFT) {
              const uint32_t partner = k ^ stride;
              if (partner > k) {
                const bool upw = (k & size) == 0;
                const uint32_t x = keys[k], y = keys[partner];
                if ((x > y) == upw) {
                  keys[k] = y;
                  keys[partner] = x;
                }
              }
            }
            __syncthreads();
          }
        }
      }
    }
    __syncthreads();
    const int32_t status0 = ms.status;
    if (rank == 0) {  // the frame's peak list, for roibin_last_peaks
      if (tid == 0) a.peaks_count_out[f] = n_pk;
      if (n_pk <= p.max_peaks)
        for (uint32_t k = tid; k < n_pk; k += kFT) a.peaks_key_out[(size_t)f * p.max_peaks + k] = keys[k];
    }
    // a10/a11 sizes of the chunks this CTA owns (one warp per chunk, 128 symbols per lane)
    auto owner_of = [&](uint32_t bin) { return bin / sh.cap_bins; };
    auto load4 = [&](uint32_t bin, uint32_t& w, uint32_t& pqn) {  // bin % 4 == 0
      const uint32_t o = owner_of(bin), local = bin - o * sh.cap_bins;
      const uint8_t* cptr = o == rank ? L.codes : cl.map_shared_rank(L.codes, o);
      const uint32_t* pptr = o == rank ? L.pq : cl.map_shared_rank(L.pq, o);
      w = *reinterpret_cast<const uint32_t*>(cptr + local);
      pqn = (pptr[local >> 5] >> (local & 31)) & 0xFu;
    };
    if (status0 == ROIBIN_OK) {
      for (uint32_t k = k_lo + warp; k < k_hi; k += kFW) {
        const uint32_t s0 = min(p.M, k * kChunk + lane * 128), s1 = min(p.M, min((k + 1) * kChunk, s0 + 128));
        uint32_t bits = 0, nlo = 0, npq = 0;
        for (uint32_t i = s0; i < s1; i += 4) {
          uint32_t w, pqn;
          load4(i, w, pqn);
          for (uint32_t t = 0; t < 4 && i + t < s1; ++t) {
            const uint32_t code = byte_code((w >> (8 * t)) & 0xFFu, i + t, p, esc);
            bits += L.cb_len[code];
            nlo += code == 0;
            npq += (pqn >> t) & 1u;
          }
        }
        for (int d = 16; d > 0; d >>= 1) {
          bits += __shfl_xor_sync(0xffffffffu, bits, d);
          nlo += __shfl_xor_sync(0xffffffffu, nlo, d);
          npq += __shfl_xor_sync(0xffffffffu, npq, d);
        }
        if (lane == 0) {
          L.own[k - k_lo] = (bits + 31) / 32;
          L.own[sh.chunks_per_cta + k - k_lo] = nlo;
          L.own[2 * sh.chunks_per_cta + k - k_lo] = npq;
        }
      }
    }
    cl.sync();  // C: chunk sizes visible; every CTA has read the peak counters
    if (rank == 0 && tid == 0) {
      *thr_count = 0;
      *peak_count = 0;
    }
    if (status0 == ROIBIN_OK) {
      // every chunk's offsets, from the owners' shared memory
      uint32_t* keys_end = keys + (n_pk > 0 ? n_pk : 1);
      uint32_t* cw = reinterpret_cast<uint32_t*>(
          (reinterpret_cast<uintptr_t>(keys_end) + 15) & ~uintptr_t(15));
      uint32_t* clo = cw + p.n_chunks;
      uint32_t* cpq = clo + p.n_chunks;
      for (uint32_t k = tid; k < p.n_chunks; k += kFT) {
        const uint32_t o = owner_of(min(p.M - 1, k * kChunk));
        const uint32_t* ow = o == rank ? L.own : cl.map_shared_rank(L.own, o);
        const uint32_t kk = k - chunk_begin_of(o, sh, p);
        cw[k] = ow[kk];
        clo[k] = ow[sh.chunks_per_cta + kk];
        cpq[k] = ow[2 * sh.chunks_per_cta + kk];
      }
      if (tid < 3) ms.carry[tid] = 0;
      __syncthreads();
      for (uint32_t k0 = 0; k0 < p.n_chunks; k0 += kFT) {
        const uint32_t k = k0 + tid;
        const uint32_t w = k < p.n_chunks ? cw[k] : 0u, l = k < p.n_chunks ? clo[k] : 0u,
                       q = k < p.n_chunks ? cpq[k] : 0u;
        uint32_t tw, tl, tq;
        const uint32_t ew = block_excl_scan(w, ms.tmp, &tw);
        const uint32_t el = block_excl_scan(l, ms.tmp, &tl);
        const uint32_t eq = block_excl_scan(q, ms.tmp, &tq);
        if (k < p.n_chunks) {
          cw[k] = ms.carry[0] + ew;
          clo[k] = ms.carry[1] + el;
          cpq[k] = ms.carry[2] + eq;
        }
        __syncthreads();
        if (tid == 0) {
          ms.carry[0] += tw;
          ms.carry[1] += tl;
          ms.carry[2] += tq;
        }
        __syncthreads();
      }
      FramePlan pl;
      pl.n_peaks = n_pk;
      pl.n_words = ms.carry[0];
      pl.n_lo = ms.carry[1];
      pl.n_pq = ms.carry[2];
      pl.off_peaks = kHeaderBytes;
      pl.off_roi = pl.off_peaks + align16((uint64_t)pl.n_peaks * 6);
      pl.off_len = pl.off_roi + align16((uint64_t)pl.n_peaks * p.roi_h * p.roi_w * 4);
      pl.off_cidx = pl.off_len + align16(p.nsym);
      pl.off_lo = pl.off_cidx + align16((uint64_t)p.n_chunks * 4);
      pl.off_pq = pl.off_lo + align16((uint64_t)pl.n_lo * 8);
      pl.off_bits = pl.off_pq + align16((uint64_t)pl.n_pq * 8);
      pl.total = pl.off_bits + align16((uint64_t)pl.n_words * 4);
      const bool fits = pl.total <= a.out_stride;
      if (rank == 0 && tid == 0) {
        int32_t timeout = 0;
        for (uint32_t r = 0; r < C; ++r) timeout |= cl.map_shared_rank(&ms.timeout, r)[0];
        a.frame_bytes[f] = pl.total;
        a.frame_status[f] = fits ? (timeout ? ROIBIN_ERR_TIMEOUT : ROIBIN_OK) : ROIBIN_ERR_CAPACITY;
      }
      if (fits) {
        if (rank == 0) write_frame_head(out, p, pl, keys, L.cb_len, cw);
        // a10 + a11: bit-packing and outliers of the own chunks
        uint32_t* words = reinterpret_cast<uint32_t*>(out + pl.off_bits);
        uint2* lo_out = reinterpret_cast<uint2*>(out + pl.off_lo);
        uint2* pq_out = reinterpret_cast<uint2*>(out + pl.off_pq);
        for (uint32_t k = k_lo + warp; k < k_hi; k += kFW) {
          const uint32_t w0 = cw[k], nw = (k + 1 < p.n_chunks ? cw[k + 1] : pl.n_words) - w0;
          for (uint32_t w = lane; w < nw; w += 32) words[w0 + w] = 0;
          __threadfence_block();
          __syncwarp();
          const uint32_t s0 = min(p.M, k * kChunk + lane * 128), s1 = min(p.M, min((k + 1) * kChunk, s0 + 128));
          uint32_t bits = 0, nlo = 0, npq = 0;
          for (uint32_t i = s0; i < s1; i += 4) {
            uint32_t w, pqn;
            load4(i, w, pqn);
            for (uint32_t t = 0; t < 4 && i + t < s1; ++t) {
              const uint32_t code = byte_code((w >> (8 * t)) & 0xFFu, i + t, p, esc);
              bits += L.cb_len[code];
              nlo += code == 0;
              npq += (pqn >> t) & 1u;
            }
          }
          const uint32_t bit_incl = warp_incl_scan(bits), lo_incl = warp_incl_scan(nlo),
                         pq_incl = warp_incl_scan(npq);
          const uint32_t start = bit_incl - bits;
          uint32_t wi = w0 + start / 32;
          const uint32_t o = start & 31u;
          uint64_t acc = 0;
          uint32_t nacc = o;
          bool first = o != 0;  // the first word is shared with the previous lane
          uint32_t lo_pos = clo[k] + lo_incl - nlo, pq_pos = cpq[k] + pq_incl - npq;
          for (uint32_t i = s0; i < s1; i += 4) {
            uint32_t w, pqn;
            load4(i, w, pqn);
            for (uint32_t t = 0; t < 4 && i + t < s1; ++t) {
              const uint32_t bin = i + t;
              const uint32_t code = byte_code((w >> (8 * t)) & 0xFFu, bin, p, esc);
              const uint32_t Lc = L.cb_len[code];
              acc |= (uint64_t)L.cb_code[code] << (64 - nacc - Lc);
              nacc += Lc;
              if (nacc >= 32) {
                const uint32_t word = (uint32_t)(acc >> 32);
                if (first) atomicOr(words + wi, word);
                else words[wi] = word;
                first = false;
                ++wi;
                acc <<= 32;
                nacc -= 32;
              }
              if (code == 0) lo_out[lo_pos++] = make_uint2(bin, (uint32_t)__ldcg(lo_delta + bin));
              if ((pqn >> t) & 1u) pq_out[pq_pos++] = make_uint2(bin, __ldcg(pq_bits + bin));
            }
          }
          if (nacc > 0) atomicOr(words + wi, (uint32_t)(acc >> 32));  // shared with the next lane
        }
        // a3: ROI windows of peaks k = rank, rank + C, ... (one warp per peak)
        float* roi = reinterpret_cast<float*>(out + pl.off_roi);
        const uint32_t win = (uint32_t)(p.roi_h * p.roi_w), plane = p.H * p.W;
        for (uint32_t k = rank + C * warp; k < n_pk; k += C * kFW) {
          const uint32_t px = keys[k];
          const uint32_t pn = px / plane, rem = px - pn * plane;
          const int r = (int)(rem / p.W), c = (int)(rem % p.W);
          const float* panel = frame + (size_t)pn * plane;
          const int r0 = r - p.roi_h / 2, c0 = c - p.roi_w / 2;
          for (uint32_t e = lane; e < win; e += 32) {
            const int rr = r0 + (int)(e / p.roi_w), cc = c0 + (int)(e % p.roi_w);
            const bool in = rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W;
            roi[(size_t)k * win + e] = in ? __ldg(panel + (size_t)rr * p.W + cc) : 0.0f;
          }
        }
      }
    } else if (rank == 0 && tid == 0) {
      a.frame_bytes[f] = 0;
      a.frame_status[f] = status0;
    }
    cl.sync();  // D: nobody reads this frame's codes any more
  }
}

// ---------------------------------------------------------------------------
// host side: shape, support check, launch
static bool make_shape(const DevParams& p, uint32_t C, uint32_t stages, FusedShape* out) {
  FusedShape sh{};
  sh.C = C;
  const uint32_t g_total = p.P * p.Hb;
  uint32_t rows = ceil_div(g_total, C);
  rows += rows & 1u;  // even: keeps cap_bins a multiple of 4
  sh.rows_per_cta = rows;
  sh.cap_bins = rows * p.Wb;
  sh.RB = max(1u, min(16u, (uint32_t)(4 * kFT) / p.W));
  sh.stages = stages;
  sh.stage_bytes = 2 * sh.RB * p.W * 4;
  sh.chunks_per_cta = ceil_div(sh.cap_bins, kChunk) + 1;
  const int side = 2 * peak_reach(p) + 1;
  uint32_t n2 = 1;
  while (n2 < max(p.max_peaks, 1u)) n2 <<= 1;
  const uint64_t ring = (uint64_t)stages * sh.stage_bytes;
  const uint64_t nbuf = (uint64_t)kFW * side * side * 4;
  const uint64_t huff = sizeof(HuffSmem) + kMaxSymbols * 4;
  const uint64_t scans = (uint64_t)n2 * 4 + 16 + 3ull * p.n_chunks * 4;
  uint64_t un = ring;
  if (nbuf > un) un = nbuf;
  if (huff > un) un = huff;
  if (scans > un) un = scans;
  uint64_t off = 0;
  auto take = [&](uint64_t bytes, uint64_t align) {
    off = (off + align - 1) / align * align;
    const uint64_t o = off;
    off += bytes;
    return (uint32_t)o;
  };
  sh.off_bar = take(8 * stages, 16);
  sh.off_hist = take(kMaxSymbols * 4, 16);
  sh.off_cb_len = take(kMaxSymbols, 16);
  sh.off_cb_code = take(kMaxSymbols * 4, 16);
  sh.off_own = take(3ull * sh.chunks_per_cta * 4, 16);
  sh.off_misc = take(sizeof(FusedMisc), 16);
  sh.off_pq = take((sh.cap_bins / 32 + 1) * 4, 16);
  sh.off_qbuf = take((uint64_t)(sh.RB + 1) * p.Wb * 4, 16);
  sh.off_codes = take(sh.cap_bins + 16, 16);
  sh.off_union = take(un, 128);
  sh.union_bytes = (uint32_t)un;
  sh.smem = (uint32_t)off;
  *out = sh;
  return off <= 227 * 1024;
}

bool fused_plan(const DevParams& p, int device, int num_sms, FusedShape* out) {
  if (p.bh != 2 || p.bw != 2 || (p.W % 4) != 0 || p.n_chunks > 4096) return false;
  cudaFuncSetAttribute(k_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  const uint32_t cands[][2] = {{16, 4}, {16, 3}, {16, 2}, {8, 4}, {8, 3}, {8, 2}};
  for (const auto& cs : cands) {
    FusedShape sh;
    if (!make_shape(p, cs[0], cs[1], &sh)) continue;
    if (cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sh.C * 64, 1, 1);
    cfg.blockDim = dim3(kFT, 1, 1);
    cfg.dynamicSmemBytes = sh.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sh.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n_clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&n_clusters, (void*)k_fused, &cfg) != cudaSuccess || n_clusters < 1) {
      cudaGetLastError();
      continue;
    }
    sh.n_clusters = (uint32_t)n_clusters;
    (void)device;
    (void)num_sms;
    *out = sh;
    return true;
  }
  return false;
}

cudaError_t launch_fused(const DevParams& p, const Scratch& fs, const PlainArgs& a, const FusedShape& sh,
                         cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  const uint32_t n_clusters = min(sh.n_clusters, a.n_frames);
  FusedShape s2 = sh;
  s2.n_clusters = n_clusters;
  cfg.gridDim = dim3(sh.C * n_clusters, 1, 1);
  cfg.blockDim = dim3(kFT, 1, 1);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = sh.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused, p, fs, a, s2);
}

}  // namespace roibin
