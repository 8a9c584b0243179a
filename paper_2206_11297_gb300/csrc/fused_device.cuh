// fused_device.cuh - the device code of the persistent batched kernel: its
// work items (streaming, codebook, chunk sizes, writing), their shared-memory
// views, the flags between them and the body of one ticket.  Two kernels run
// it: k_fused (fused_kernel.cu), over the frames of one geometry, and
// k_fused_jobs (fused_jobs.cu), over several such batches in one launch.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "roibin_internal.cuh"

namespace roibin {
// local to each kernel's translation unit (each compiles its own copy)
namespace {

constexpr int kPT = 256;       // threads per CTA
constexpr int kPW = kPT / 32;  // warps per CTA
constexpr uint32_t kMaxK = 8;   // panels per streaming item
constexpr uint32_t kConsumerWarps = 7;  // warps that code rows (31 columns each)
constexpr uint32_t kGroupCols = kConsumerWarps * 31;  // float4 columns of one column group
constexpr uint32_t kMaxG = 2;           // column groups per consumer lane
constexpr uint32_t kProducerWarp = 7;   // the warp whose lane 0 issues the row copies
constexpr uint32_t kThrLocalCap = 256;
constexpr uint32_t kBlockKey = 1u << 31;  // a listed 2x4 block (else a listed candidate pixel)
constexpr uint32_t kPqList = 128;  // prequantisation outliers an item lists before rescanning
constexpr uint32_t kLagSize = 65535, kLagWrite = 64;  // see launch_fused
constexpr uint32_t kPanelTimedOut = 0xFFFFFFFFu;  // peak count of an item whose rows never arrived

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// 16-byte streaming load: no L1 allocation, first in line for L2 eviction.
__device__ __forceinline__ float4 ld_stream(const float* ptr, uint64_t policy) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(ptr), "l"(policy));
  return v;
}
__device__ __forceinline__ uint64_t evict_normal_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 16-bit store that asks L2 to keep the line (code bytes wait there until packed)
__device__ __forceinline__ void st_keep_u16(void* ptr, uint16_t v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.u16 [%0], %1, %2;" ::"l"(ptr), "h"(v), "l"(policy) : "memory");
}
// The same, predicated on `pred` inside the instruction (no branch).
__device__ __forceinline__ void st_keep_u16_if(void* ptr, uint16_t v, uint64_t policy, bool pred) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %3, 0;\n @q st.global.L2::cache_hint.u16 [%0], %1, %2;\n}\n" ::"l"(ptr),
      "h"(v), "l"(policy), "r"((uint32_t)pred)
      : "memory");
}
// Requests the 128-byte line holding ptr into L2 (no register written, no wait).
__device__ __forceinline__ void prefetch_l2(const void* ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}
// Drops a 128-byte line from L2 without writing it back (its contents are dead).
__device__ __forceinline__ void discard_line(const void* ptr) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(ptr) : "memory");
}

// Symbol of a stored code byte.
__device__ __forceinline__ uint32_t byte_code(uint32_t b, const uint16_t* esc_bin, int32_t R) {
  if (b == 0) return 0;
  if (b == 255) return __ldcg(esc_bin);
  return b - 128 + (uint32_t)R;
}

// Writes the header, the peaks, the code lengths, the chunk index and every
// padding byte of a frame (block-cooperative).  keys (pixel index per peak)
// and cb_len are global arrays written by other CTAs: read through L2.
__device__ void write_frame_head(uint8_t* out, const DevParams& p, const FramePlan& pl, const uint32_t* keys,
                                 const uint8_t* cb_len, const uint32_t* chunk_word_off, uint32_t ref) {
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
    h[18] = p.dims == 2 ? 0u : (uint32_t)p.dims;  // Lorenzo dimension, 0 for the default 2
    h[22] = ref;  // frames back to the stream with the code lengths (0: this one)
    uint4* o4 = reinterpret_cast<uint4*>(out);
    for (int i = 0; i < 6; ++i) o4[i] = make_uint4(h[4 * i], h[4 * i + 1], h[4 * i + 2], h[4 * i + 3]);
  }
  const uint32_t plane = p.H * p.W;
  uint16_t* pk = reinterpret_cast<uint16_t*>(out + pl.off_peaks);
  for (uint32_t k = threadIdx.x; k < pl.n_peaks; k += blockDim.x) {
    const uint32_t px = __ldcg(keys + k);
    const uint32_t pn = px / plane, rem = px - pn * plane;
    pk[3 * k] = (uint16_t)pn;
    pk[3 * k + 1] = (uint16_t)(rem / p.W);
    pk[3 * k + 2] = (uint16_t)(rem % p.W);
  }
  auto zero = [&](uint64_t from, uint64_t to) {
    for (uint64_t b = from + threadIdx.x; b < to; b += blockDim.x) out[b] = 0;
  };
  zero(pl.off_peaks + (uint64_t)pl.n_peaks * 6, pl.off_roi);
  zero(pl.off_roi + (p.roi_coder ? 0 : (uint64_t)pl.n_peaks * p.roi_h * p.roi_w * 4), pl.off_len);
  if (ref == 0) {  // the code lengths: a chunk's head only
    for (uint32_t k = threadIdx.x; k < p.nsym; k += blockDim.x) out[pl.off_len + k] = __ldcg(cb_len + k);
    zero(pl.off_len + p.nsym, pl.off_cidx);
  }
  uint32_t* ci = reinterpret_cast<uint32_t*>(out + pl.off_cidx);
  for (uint32_t k = threadIdx.x; k < p.n_chunks; k += blockDim.x) ci[k] = chunk_word_off[k];
  zero(pl.off_cidx + (uint64_t)p.n_chunks * 4, pl.off_lo);
  zero(pl.off_lo + (uint64_t)pl.n_lo * 8, pl.off_pq);
  zero(pl.off_pq + (uint64_t)pl.n_pq * 8, pl.off_bits);
  zero(pl.off_bits + (uint64_t)pl.n_words * 4, pl.total);
}

// Shared-memory views (byte offsets from FusedShape).  The streaming role and
// the finalising role of a CTA never overlap in time, so their buffers share
// one allocation; the control words sit in front of both.
struct StreamView {
  uint32_t* hist;  // [nsym]
  uint32_t* pql;   // [kPqList] prequantisation outliers of the item (item-local bin index)
  uint32_t* thr;   // [kThrLocalCap] listed candidates (item-local pixel) or 2x4 blocks (kBlockKey set)
  float* thrv;     // [kThrLocalCap] value of each listed candidate
  float* nb;       // [kPW][side^2] peak-test neighbourhoods (aliases the ring)
  uint32_t* acc;   // [sort_n2] accepted peaks of the item (aliases the ring)
  uint32_t* cand;  // [kThrLocalCap] listed candidates left after pruning (aliases the ring)
  uint32_t* ctl;
  unsigned char* ring;  // [stages][stage_bytes] raw rows in flight
  uint64_t* bars;       // [2 stages] per ring slot: rows landed, slot released
};
struct FinView {
  HuffSmem* hs;
  uint32_t* total;  // [kMaxSymbols]
  uint8_t* cb_len;  // [kMaxSymbols]
  uint32_t* cb_code;
  uint32_t* keys;  // [peak_cap]
  uint32_t* cw;    // [n_chunks] chunk words -> word offsets; then lo, pq
  uint32_t* clo;
  uint32_t* cpq;
  uint32_t* offs;  // [U] offset of each item's peaks in the frame list
  uint32_t* ctl;
};
enum {
  CTL_THR = 0,
  CTL_ACC,
  CTL_ITEM,
  CTL_LAST,
  CTL_BAD,
  CTL_STATUS,
  CTL_CARRY0,
  CTL_CARRY1,
  CTL_CARRY2,
  CTL_WAIT,
  CTL_TIMEOUT,
  CTL_NZ,                       // codes other than the zero residual's in the item
  CTL_PQN,                      // prequantisation outliers in the item
  CTL_NCAND,                    // listed candidates left after pruning
  CTL_BAND,                     // band copies so far (the band barrier's phase)
  CTL_PQ,                       // [kMaxK] prequantisation outliers per panel of the item
  CTL_TMP = CTL_PQ + kMaxK,
  CTL_WORDS = CTL_TMP + 33
};

__device__ __forceinline__ StreamView stream_view(unsigned char* sm, const FusedShape& sh) {
  StreamView v;
  v.hist = reinterpret_cast<uint32_t*>(sm + sh.off_hist);
  v.pql = reinterpret_cast<uint32_t*>(sm + sh.off_pql);
  v.thr = reinterpret_cast<uint32_t*>(sm + sh.off_thr);
  v.thrv = reinterpret_cast<float*>(sm + sh.off_thr + kThrLocalCap * 4);
  v.nb = reinterpret_cast<float*>(sm + sh.off_nb);
  v.acc = reinterpret_cast<uint32_t*>(sm + sh.off_acc);
  v.cand = reinterpret_cast<uint32_t*>(sm + sh.off_cand);
  v.ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  v.ring = sm + sh.off_ring;
  v.bars = reinterpret_cast<uint64_t*>(sm + sh.off_bar);
  return v;
}
__device__ __forceinline__ FinView fin_view(unsigned char* sm, const FusedShape& sh) {
  FinView v;
  v.hs = reinterpret_cast<HuffSmem*>(sm + sh.off_huff);
  v.total = reinterpret_cast<uint32_t*>(sm + sh.off_total);
  v.cb_len = sm + sh.off_cblen;
  v.cb_code = reinterpret_cast<uint32_t*>(sm + sh.off_cbcode);
  v.keys = reinterpret_cast<uint32_t*>(sm + sh.off_keys);
  v.cw = reinterpret_cast<uint32_t*>(sm + sh.off_cw);
  v.clo = v.cw + sh.n_chunks;
  v.cpq = v.clo + sh.n_chunks;
  v.offs = reinterpret_cast<uint32_t*>(sm + sh.off_offs);
  v.ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  return v;
}

// ---------------------------------------------------------------------------
// a1 + a2 for an item with more candidates than its list holds (hot pixels),
// one lane per candidate, every pixel read from shared memory.  The item's
// panels are taken in bands of rows: a band of B rows plus `reach` rows above
// and below (the whole neighbourhood of every candidate in it) is staged in
// the ring's memory by one bulk copy.  The band's pixels >=
// amax_thr are ranked in a block-wide scan (each thread counts its own run of
// the band, then the runs' counts are scanned), and rank q goes to thread
// q mod 256 in rounds, so every thread holds a candidate whatever their number.
// Each thread runs the local-maximum rule and the evaluation in the sequential
// order of is_local_max_at / evaluate_peak_at.  Accepted pixels (item-local
// index) are collected in the item's slot of s.peak_part; the caller sorts them.
__device__ __noinline__ void dense_band_peaks(const DevParams& p, const Scratch& s, const FusedShape& sh,
                                              const StreamView& v, const float* item_px, uint32_t kp, size_t fu) {
  const uint32_t tid = threadIdx.x, W = p.W, H = p.H, plane = H * W;
  const uint32_t reach = (uint32_t)peak_reach(p), B = sh.band_rows - 2 * reach;
  float* band = reinterpret_cast<float*>(v.ring);
  uint32_t* run_start = v.thr;  // [kPT] first rank of each thread's run
  uint32_t* acc = s.peak_part + fu * sh.peak_cap;
  uint64_t* band_bar = v.bars + 2 * sh.stages;
  const uint64_t pol = evict_normal_policy();  // a band's halo rows are read again by the next band
  uint32_t bands_done = v.ctl[CTL_BAND];
  for (uint32_t j = 0; j < kp; ++j) {
    const float* pan = item_px + (size_t)j * plane;
    for (uint32_t r0 = 0; r0 < H; r0 += B) {
      const uint32_t r1 = min(H, r0 + B);
      const uint32_t rb0 = r0 >= reach ? r0 - reach : 0u, rb1 = min(H, r1 + reach);
      __syncthreads();  // the previous band is no longer read
      // one bulk copy of the band's rows (contiguous in the panel, 16-byte
      // aligned: W % 4 == 0), its arrival counted on the band barrier
      if (tid == 0) {
        fence_proxy_async();  // the band's memory was last read through the generic proxy
        const uint32_t bytes = (rb1 - rb0) * W * 4;
        mbar_expect_tx(band_bar, bytes);
        tma_load_1d(band, pan + (size_t)rb0 * W, bytes, band_bar, pol);
      }
      const bool landed = mbar_wait(band_bar, (bands_done++) & 1u);
      if (!__syncthreads_and(landed)) {  // the copy never arrived: the item is marked, see process_item
        if (tid == 0) {
          v.ctl[CTL_TIMEOUT] = 1;
          v.ctl[CTL_BAND] = bands_done;
        }
        __syncthreads();
        return;
      }
      // pass 1: each thread counts the candidates of its run of the band's own rows
      const float* core = band + (size_t)(r0 - rb0) * W;
      const uint32_t n_core = (r1 - r0) * W, run = ceil_div(n_core, kPT);
      const uint32_t x0 = min(n_core, tid * run), x1 = min(n_core, x0 + run);
      uint32_t cnt = 0;
      for (uint32_t x = x0; x < x1; ++x) cnt += core[x] >= p.amax;
      uint32_t total;
      const uint32_t first = block_excl_scan(cnt, v.ctl + CTL_TMP, &total);
      run_start[tid] = first;
      __syncthreads();
      // pass 2: rank q -> the run holding it (the last run starting at or before
      // q), then the (q - start)-th candidate of that run
      for (uint32_t q0 = 0; q0 < total; q0 += kPT) {
        const uint32_t q = q0 + tid;
        if (q >= total) continue;
        uint32_t lo = 0, hi = kPT - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (run_start[mid] <= q) lo = mid;
          else hi = mid - 1;
        }
        uint32_t skip = q - run_start[lo], x = min(n_core, lo * run);
        for (;; ++x)
          if (core[x] >= p.amax && skip-- == 0) break;
        const int r = (int)(r0 + x / W), c = (int)(x % W);
        const float* at = band + (size_t)(r - (int)rb0) * W + c;
        auto px = [&](int dr, int dc) { return at[dr * (int)W + dc]; };
        if (peak_test_one(px, (int)H, (int)W, r, c, p)) {
          const uint32_t slot = atomicAdd(v.ctl + CTL_ACC, 1u);
          if (slot < sh.peak_cap) acc[slot] = j * plane + (uint32_t)r * W + (uint32_t)c;
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) v.ctl[CTL_BAND] = bands_done;
  // the item's accepted pixels into the shared list the caller sorts
  const uint32_t n_acc = v.ctl[CTL_ACC];
  if (n_acc <= p.max_peaks)
    for (uint32_t k = tid; k < n_acc; k += kPT) v.acc[k] = __ldcg(acc + k);
}

// ---------------------------------------------------------------------------
// One streaming item: panels pn0 .. pn0 + kp - 1 of frame f, side by side.
//
// A consumer lane owns float4 columns of the item (two bins per binned row),
// one per column group, and walks down the rows.  The q values of the row
// above stay in its registers; the bin to the left comes from the previous
// lane by shuffle, and lane 0 reads the previous warp's last column from
// shared memory.  A step covers RB binned rows: phase A bins and
// prequantises them into registers, one barrier (it also frees the ring
// slot), then phase B forms the Lorenzo residuals, code bytes and histogram.
// kRt: the dense-peaks choice is read from sh.dense at run time instead of
// kDense (one copy of the code for both, as the multi-job kernel wants).
template <int RB, bool kDense, int kG, bool kRt = false>
__device__ void process_item(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                             unsigned char* sm, uint32_t f, uint32_t u, uint32_t& ring_iter) {
  const StreamView v = stream_view(sm, sh);
  const bool dense = kRt ? sh.dense != 0 : kDense;
  // input rows: evict-first (or normal) in L2; code bytes: evict-last until packed
  const uint64_t pol = sh.input_evict_first ? evict_first_policy() : evict_normal_policy();
  const uint64_t keep_pol = evict_last_policy();
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  const uint32_t NP = p.W >> 2, Mp = p.Hb * p.Wb, plane = p.H * p.W;
  const uint32_t pn0 = u * sh.k, kp = min(sh.k, p.P - pn0);
  // lane l >= 1 of warp w owns float4 column 217 g + 31 w + l - 1 of the item
  // in each column group g; lane 0 recomputes the column before (the previous
  // warp's last) for its left neighbour, so warps never wait for one another
  const uint32_t C = kp * NP;
  const float* item_px = a.frames + (size_t)f * p.frame_px + (size_t)pn0 * plane;
  const uint32_t slot_floats = 2 * RB * p.W;  // one panel's rows in a ring slot
  const size_t fu = (size_t)f * p.P + u;
  uint64_t* full_bar = v.bars;                 // [stages] rows landed (TMA transaction count)
  uint64_t* empty_bar = v.bars + sh.stages;    // [stages] every consumer warp is done with the slot

  uint64_t* trace = (a.trace && f < a.trace_frames && tid == 0)
                       ? a.trace + (size_t)a.trace_frames * kTracePoints + fu * 4
                       : nullptr;
  if (trace) trace[0] = global_ns();
  for (uint32_t k = tid; k < p.nsym; k += kPT) v.hist[k] = 0;
  if (tid == 0) {
    v.ctl[CTL_THR] = 0;
    v.ctl[CTL_NZ] = 0;
    v.ctl[CTL_PQN] = 0;
  }
  if (tid < kMaxK) v.ctl[CTL_PQ + tid] = 0;
  if (a.user_peaks && tid == 0) s.peak_part_count[fu] = 0;
  __syncthreads();  // hist, masks and counters are zero

  const uint32_t n_steps = ceil_div(p.Hb, (uint32_t)RB);
  const bool find = a.user_peaks == nullptr;
  // candidates past the shared list go to the CTA's list in global memory
  // (the dense-peaks variant tests such items band by band instead)
  const bool spills = !dense && blockIdx.x < s.thr_spill_ctas;
  auto spill_at = [&](uint32_t e) -> uint32_t& { return s.thr_spill[(size_t)blockIdx.x * kThrSpill + e]; };
  bool timed_out = false;
  uint32_t slot = ring_iter % sh.stages, phase = (ring_iter / sh.stages) & 1u;
  auto advance = [&]() {
    if (++slot == sh.stages) {
      slot = 0;
      phase ^= 1u;
    }
  };
  if (warp == kProducerWarp) {
    // producer: step st = raw rows [2 st RB, min(H, 2 (st + 1) RB)) of each
    // panel, one bulk copy per panel, once every consumer has left the slot
    if (lane == 0) {
      for (uint32_t st = 0; st < n_steps; ++st) {
        if (!mbar_wait(empty_bar + slot, phase ^ 1u)) timed_out = true;
        const uint32_t r0 = 2 * st * RB, r1 = min(p.H, 2 * (st + 1) * RB);
        const uint32_t bytes = (r1 - r0) * p.W * 4;
        float* dst = reinterpret_cast<float*>(v.ring + (size_t)slot * sh.stage_bytes);
        fence_proxy_async();
        mbar_expect_tx(full_bar + slot, bytes * kp);
        for (uint32_t j = 0; j < kp; ++j)
          tma_load_1d(dst + (size_t)j * slot_floats, item_px + (size_t)j * plane + (size_t)r0 * p.W, bytes,
                      full_bar + slot, pol);
        advance();
      }
    }
  } else if (31 * warp >= C) {
    // a consumer warp without columns in this item still releases every slot
    for (uint32_t st = 0; st < n_steps; ++st) {
      if (!mbar_wait(full_bar + slot, phase)) timed_out = true;
      if (lane == 0) mbar_arrive(empty_bar + slot);
      advance();
    }
  } else {
    // kG column groups: a panel of up to 868 kG pixels per row fits one item
    struct Col {
      bool owned, first;
      uint32_t pi, pc;
      uint8_t* codes;      // the column's code bytes in binned row 0
      uint16_t* esc;       // the lane's panel: escape codes, Lorenzo-outlier deltas and
      int32_t* lo_delta;   // prequantisation-outlier bits, at their bin
      uint32_t* pq_bits;
    };
    Col cols[kG];
    int2 qu[kG];   // q of the lane's two bins in the row above, per group
    int32_t qd[kG];  // q of the bin left of them in the row above
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      Col& c = cols[g];
      const int gc = (int)kGroupCols * g + 31 * (int)warp + (int)lane - 1;
      const bool ok = gc >= 0 && (uint32_t)gc < C;
      c.owned = ok && lane >= 1 && warp < kConsumerWarps;
      const uint32_t gcol = ok ? (uint32_t)gc : 0u;
      c.pi = gcol / NP;
      c.pc = gcol - c.pi * NP;
      c.first = c.pc == 0;  // the bin to the left lies outside the panel
      const size_t fbin = (size_t)f * p.M + (size_t)(pn0 + c.pi) * Mp;  // first bin of the lane's panel
      c.codes = s.codes8 + (size_t)f * sh.codes_stride + (size_t)(pn0 + c.pi) * Mp + 2 * c.pc;
      c.esc = s.codes + fbin;
      c.lo_delta = s.lo_delta + fbin;
      c.pq_bits = s.pq_bits + fbin;
      qu[g] = make_int2(0, 0);
      qd[g] = 0;
    }

    // One step: RB binned rows.  FULL steps have RB rows of two raw rows each
    // (every step but possibly the panel's last), so they need no row checks.
    // Rare cases (prequantisation screen undecided, a block >= amax_thr, a
    // non-zero residual) are flagged per row and handled after the rows by
    // the whole warp, so the common path has no divergent branch.  Every
    // group reads its rows (phase A) before the warp leaves the ring slot.
    auto step = [&](uint32_t st, auto full_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      const uint32_t i0 = st * RB;
      int2 qa[kG][RB];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const uint32_t pi = cols[g].pi, pc = cols[g].pc;
        const bool owned = cols[g].owned;
        uint32_t* pq_bits = cols[g].pq_bits;
        const float4* rows =
            reinterpret_cast<const float4*>(v.ring + (size_t)slot * sh.stage_bytes) + pi * (slot_floats / 4) + pc;
        // phase A: q of the lane's bins in the step's rows
        uint32_t redo = 0, hot = 0;  // bit ii: row ii needs the full test / holds a block >= amax_thr
#pragma unroll
        for (int ii = 0; ii < RB; ++ii) {
          const uint32_t i = i0 + ii;
          qa[g][ii] = make_int2(0, 0);
          if (!FULL && i >= p.Hb) continue;
          const bool two = FULL || 2 * i + 1 < p.H;
          const float4 va = rows[(2 * ii) * NP];
          const float4 vb = two ? rows[(2 * ii + 1) * NP] : make_float4(0.f, 0.f, 0.f, 0.f);
          float v0, v1;
          bin_pair(va, vb, two, v0, v1);
          int32_t q0, q1;
          const bool ok = prequant_fast(v0, p, q0) & prequant_fast(v1, p, q1);
          redo |= (uint32_t)!ok << ii;
          qa[g][ii] = make_int2(q0, q1);
          if (find) {
            const float m =
                fmaxf(fmaxf(fmaxf(va.x, va.y), fmaxf(va.z, va.w)), fmaxf(fmaxf(vb.x, vb.y), fmaxf(vb.z, vb.w)));
            hot |= (uint32_t)(m >= p.amax) << ii;
          }
        }
        if (__any_sync(0xffffffffu, redo != 0)) {  // the screen could not decide: the full test
#pragma unroll
          for (int ii = 0; ii < RB; ++ii) {
            if (!((redo >> ii) & 1u)) continue;
            const uint32_t i = i0 + ii;
            const bool two = 2 * i + 1 < p.H;
            const float4 va = rows[(2 * ii) * NP];
            const float4 vb = two ? rows[(2 * ii + 1) * NP] : make_float4(0.f, 0.f, 0.f, 0.f);
            float v0, v1;
            bin_pair(va, vb, two, v0, v1);
            const Quant Q0 = prequantize(v0, p), Q1 = prequantize(v1, p);
            qa[g][ii] = make_int2(Q0.q, Q1.q);
            if (owned && (Q0.outlier | Q1.outlier)) {
              const uint32_t lb = i * p.Wb + 2 * pc;
              atomicAdd(v.ctl + CTL_PQ + pi, (uint32_t)Q0.outlier + (uint32_t)Q1.outlier);
              const uint32_t at = atomicAdd(v.ctl + CTL_PQN, (uint32_t)Q0.outlier + (uint32_t)Q1.outlier);
              uint32_t e = at;
              if (Q0.outlier) {
                pq_bits[lb] = Q0.outlier_bits;
                if (e < kPqList) v.pql[e] = pi * Mp + lb;
                ++e;
              }
              if (Q1.outlier) {
                pq_bits[lb + 1] = Q1.outlier_bits;
                if (e < kPqList) v.pql[e] = pi * Mp + lb + 1;
              }
            }
          }
        }
        if (!owned) hot = 0;
        if (__any_sync(0xffffffffu, hot != 0)) {
          // a 2x4 block holding a pixel >= amax_thr.  With rank >= 3 the block
          // lies inside the window of each of its pixels, so only its first
          // maximum can be a candidate: that pixel and its value are listed.
          // With a smaller rank the block itself is listed.
#pragma unroll
          for (int ii = 0; ii < RB; ++ii) {
            if (!((hot >> ii) & 1u)) continue;
            const uint32_t i = i0 + ii;
            uint32_t key = kBlockKey | (pi * plane + 2 * i * p.W + 4 * pc);
            float best = 0.0f;
            if (p.rank >= 3) {
              const bool two = 2 * i + 1 < p.H;
              const float4 va = rows[(2 * ii) * NP];
              const float4 vb = rows[(2 * ii + 1) * NP];  // inside the slot; used only when two
              const float px[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
              uint32_t at = 0;
              best = px[0];
#pragma unroll
              for (int e = 1; e < 8; ++e)
                if ((e < 4 || two) && (px[e] > best || best != best)) {
                  best = px[e];
                  at = e;
                }
              key = pi * plane + (2 * i + (at >> 2)) * p.W + 4 * pc + (at & 3u);
            }
            const uint32_t slot_t = atomicAdd(v.ctl + CTL_THR, 1u);
            if (slot_t < kThrLocalCap) {
              v.thr[slot_t] = key;
              v.thrv[slot_t] = best;
            } else if (spills && slot_t - kThrLocalCap < kThrSpill) {
              spill_at(slot_t - kThrLocalCap) = key;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty_bar + slot);  // this warp is done with the slot
      advance();
      // phase B: residuals and code bytes.  A pair of zero residuals (the
      // common case) stores 0x8080 and is not counted: the zero residual's
      // histogram count is derived from the bin count at the flush.
      // Residuals in [-128, 127] store residual + 128 here; the rare pass
      // below fixes the bytes of outliers and escapes and counts every
      // non-zero residual.
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const uint32_t pc = cols[g].pc;
        const bool owned = cols[g].owned, first_col = cols[g].first;
        uint8_t* codes = cols[g].codes;
        uint16_t* esc = cols[g].esc;
        int32_t* lo_delta = cols[g].lo_delta;
        uint32_t nz = 0;
        const int2 qu_step = qu[g];  // the chain's start, replayed by the rare pass
        const int32_t qd_step = qd[g];
        auto left_of = [&](int ii) {  // q of the bin left of the lane's bins in row i0 + ii
          const int32_t from_lane = __shfl_up_sync(0xffffffffu, qa[g][ii].y, 1);
          return first_col ? 0 : from_lane;
        };
#pragma unroll
        for (int ii = 0; ii < RB; ++ii) {
          const uint32_t i = i0 + ii;
          if (!FULL && i >= p.Hb) break;
          const int32_t left = left_of(ii);
          const int32_t d0 = qa[g][ii].x - qu[g].x - left + qd[g];
          const int32_t d1 = qa[g][ii].y - qu[g].y - qa[g][ii].x + qu[g].x;
          qu[g] = qa[g][ii];
          qd[g] = left;
          nz |= (uint32_t)((d0 | d1) != 0) << ii;
          const uint32_t pair = (uint32_t)((d0 + 128) & 0xFF) | ((uint32_t)((d1 + 128) & 0xFF) << 8);
          st_keep_u16_if(codes + (size_t)i * p.Wb, (uint16_t)pair, keep_pol,
                         owned && RB_CHECK(s, i < p.Hb && 2 * pc + 1 < p.Wb, ROIBIN_CHECK_CODES));  // 2 pc is even
        }
        if (!owned) nz = 0;
        if (__any_sync(0xffffffffu, nz != 0)) {
          int2 qu_r = qu_step;
          int32_t qd_r = qd_step;
#pragma unroll
          for (int ii = 0; ii < RB; ++ii) {
            const uint32_t i = i0 + ii;
            if (!FULL && i >= p.Hb) break;
            const int32_t left = left_of(ii);
            const int32_t d0 = qa[g][ii].x - qu_r.x - left + qd_r;
            const int32_t d1 = qa[g][ii].y - qu_r.y - qa[g][ii].x + qu_r.x;
            qu_r = qa[g][ii];
            qd_r = left;
            const bool row_nz = (nz >> ii) & 1u;
            if (!__any_sync(0xffffffffu, row_nz)) continue;
            uint32_t c0 = 0xFFFFu, c1 = 0xFFFFu;
            if (row_nz) {
              const uint32_t lb = i * p.Wb + 2 * pc;
              c0 = quant_code(d0, p.R);
              c1 = quant_code(d1, p.R);
              // byte = residual + 128 for residuals in [-127, 126]; 0 = Lorenzo
              // outlier (delta on the side); 255 = escape (code on the side)
              auto to_byte = [&](int32_t d, uint32_t c, uint32_t bin) -> uint32_t {
                if (c == 0) {
                  lo_delta[bin] = d;
                  return 0u;
                }
                if (d >= -127 && d <= 126) return (uint32_t)(d + 128);
                esc[bin] = (uint16_t)c;
                return 255u;
              };
              const uint32_t b0 = to_byte(d0, c0, lb), b1 = to_byte(d1, c1, lb + 1);
              if (b0 != (uint32_t)((d0 + 128) & 0xFF) || b1 != (uint32_t)((d1 + 128) & 0xFF))
                st_keep_u16_if(codes + (size_t)i * p.Wb, (uint16_t)(b0 | (b1 << 8)), keep_pol, true);
            }
            hist_add_warp(v.hist, c0 != (uint32_t)p.R ? c0 : 0xFFFFu, 0xFFFFFFFFu);
            hist_add_warp(v.hist, c1 != (uint32_t)p.R ? c1 : 0xFFFFu, 0xFFFFFFFFu);
          }
        }
      }
    };
    for (uint32_t st = 0; st < n_steps; ++st) {
      if (!mbar_wait(full_bar + slot, phase)) timed_out = true;
      const uint32_t i_end = (st + 1) * RB;
      if (i_end <= p.Hb && 2 * i_end <= p.H) step(st, std::integral_constant<bool, true>{});
      else step(st, std::integral_constant<bool, false>{});
    }
  }
  if (timed_out) v.ctl[CTL_TIMEOUT] = 1;
  ring_iter += n_steps;
  __syncthreads();
  // The peak tests below read the neighbourhood of every listed candidate
  // again, rows the ring streamed (evict-first) as long as an item ago: those
  // lines are requested into L2 now, so their latency passes during the
  // flushes and the pruning pass instead of in the tests.
  if (find && v.ctl[CTL_THR] <= kThrLocalCap) {
    const uint32_t cnt = v.ctl[CTL_THR];
    const int reach = peak_reach(p);
    const uint32_t span = 2u * (uint32_t)reach + 2u;  // raw rows around a listed pixel or 2x4 block
    for (uint32_t e = tid; e < cnt * span; e += kPT) {
      const uint32_t k = e / span, d = e - k * span;
      const uint32_t key = v.thr[k] & ~kBlockKey, pj = key / plane, rem = key - pj * plane;
      const uint32_t r0 = rem / p.W;
      const int r = (int)r0 - reach + (int)d, c = (int)(rem - r0 * p.W);
      if (r < 0 || r >= (int)p.H) continue;
      const int c0 = max(c - reach, 0), c1 = min(c + 3 + reach, (int)p.W - 1);
      const float* row = item_px + (size_t)pj * plane + (size_t)r * p.W;
      prefetch_l2(row + c0);
      if ((reinterpret_cast<uintptr_t>(row + c0) >> 7) != (reinterpret_cast<uintptr_t>(row + c1) >> 7))
        prefetch_l2(row + c1);
    }
  }
  // the zero residual's count: every bin of the item not counted elsewhere
  {
    uint32_t part = 0;
    for (uint32_t k = tid; k < p.nsym; k += kPT) part += k != (uint32_t)p.R ? v.hist[k] : 0u;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (lane == 0 && part) atomicAdd(v.ctl + CTL_NZ, part);
    __syncthreads();
    if (tid == 0) v.hist[p.R] = kp * Mp - v.ctl[CTL_NZ];
    __syncthreads();
  }
  if (trace) trace[1] = global_ns();
  // flush the item's histogram and its panels' outlier bits (disjoint slots)
  for (uint32_t k = tid; k < p.nsym; k += kPT) s.hist_part[fu * kMaxSymbols + k] = v.hist[k];
  const uint32_t n_pq_item = v.ctl[CTL_PQN];
  for (uint32_t j = 0; j < kp; ++j) {
    const uint32_t n_pq = v.ctl[CTL_PQ + j];
    const size_t fp = (size_t)f * p.P + pn0 + j;
    if (n_pq)  // the panel's bitmask, set below
      for (uint32_t k = tid; k < sh.mask_words; k += kPT) s.pq_mask[fp * sh.mask_words + k] = 0;
    if (tid == 0) s.pq_part_count[fp] = n_pq;
  }
  if (n_pq_item) {
    __syncthreads();  // the masks are zero
    uint32_t* gmask = s.pq_mask + ((size_t)f * p.P + pn0) * sh.mask_words;
    if (n_pq_item <= kPqList) {
      for (uint32_t e = tid; e < n_pq_item; e += kPT) {
        const uint32_t b = v.pql[e], pj = b / Mp, lb = b - pj * Mp;
        atomicOr(gmask + pj * sh.mask_words + (lb >> 5), 1u << (lb & 31));
      }
    } else {
      // more outliers than the list holds: find them again from the input
      for (uint32_t b = tid; b < kp * Mp; b += kPT) {
        const uint32_t pj = b / Mp, lb = b - pj * Mp, i = lb / p.Wb, jb = lb - i * p.Wb;
        const float* px = item_px + (size_t)pj * plane + (size_t)(2 * i) * p.W + 2 * jb;
        const bool two = 2 * i + 1 < p.H;
        const float4 va = make_float4(__ldg(px), __ldg(px + 1), 0.f, 0.f);
        const float4 vb = two ? make_float4(__ldg(px + p.W), __ldg(px + p.W + 1), 0.f, 0.f)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        float v0, v1;
        bin_pair(va, vb, two, v0, v1);
        if (prequantize(v0, p).outlier) atomicOr(gmask + pj * sh.mask_words + (lb >> 5), 1u << (lb & 31));
      }
    }
  }

  // a1 + a2 on the listed blocks (on every pixel >= amax_thr if the list overflowed)
  if (find) {
    if (tid == 0) v.ctl[CTL_ACC] = 0;
    __syncthreads();
    const uint32_t cnt = v.ctl[CTL_THR];
    float* nb = v.nb + warp * sh.side * sh.side;
    auto test = [&](uint32_t lp) {  // lp: pixel index within the item
      const uint32_t pj = lp / plane, rem = lp - pj * plane;
      const uint32_t r = rem / p.W, c = rem - r * p.W;
      auto ld = [](const float* q) { return __ldg(q); };
      const float* pan = item_px + (size_t)pj * plane;
      const bool hit = kRt ? (dense ? warp_peak_test<true>(pan, p.H, p.W, r, c, p, nb, ld)
                                    : warp_peak_test<false>(pan, p.H, p.W, r, c, p, nb, ld))
                           : warp_peak_test<kDense>(pan, p.H, p.W, r, c, p, nb, ld);
      if (hit && lane == 0) {
        const uint32_t slot = atomicAdd(v.ctl + CTL_ACC, 1u);
        if (slot < sh.sort_n2) v.acc[slot] = lp;
      }
    };
    // a listed pixel is tested; a listed 2x4 block is screened first (a pixel
    // beaten inside its own block, which lies inside its window, by the
    // local-maximum rule can never be a candidate)
    auto test_listed = [&](uint32_t listed) {
      if (!(listed & kBlockKey)) {
        test(listed);
        return;
      }
      const uint32_t key = listed & ~kBlockKey, pj = key / plane, rem = key - pj * plane;
      const uint32_t r0 = rem / p.W;
      const uint32_t npx = r0 + 1 < p.H ? 8u : 4u;
      const uint32_t me = lane & 7u;
      const float x = me < npx ? __ldg(item_px + key + (me >> 2) * p.W + (me & 3u)) : 0.0f;
      bool keep = lane < npx && x >= p.amax;
#pragma unroll
      for (uint32_t q = 0; q < 8; ++q) {
        const float y = __shfl_sync(0xffffffffu, x, q);
        const int dc = (int)(q & 3u) - (int)(me & 3u);
        if (q == me || q >= npx || dc > p.rank || -dc > p.rank) continue;
        if (q < me ? !(x > y) : !(x >= y)) keep = false;
      }
      uint32_t m = __ballot_sync(0xffffffffu, keep);
      while (m) {
        const uint32_t l = __ffs(m) - 1;
        m &= m - 1;
        test(key + (l >> 2) * p.W + (l & 3u));
      }
    };
    if (cnt <= kThrLocalCap + (spills ? kThrSpill : 0u)) {
      // a listed candidate beaten by another candidate of the shared list
      // inside its window (larger, or equal and earlier in row-major order)
      // fails the local-maximum rule; the others are tested in full
      const uint32_t cnt_local = min(cnt, kThrLocalCap);
      if (tid == 0) v.ctl[CTL_NCAND] = 0;
      // each listed pixel's (panel, row, col), decoded once, in the per-warp
      // neighbourhood buffers (unused until the tests): the pairwise pass below
      // then compares without dividing
      uint32_t* pos = reinterpret_cast<uint32_t*>(v.nb);
      const bool decoded = (uint64_t)kPW * sh.side * sh.side >= 2ull * cnt_local;
      if (decoded)
        for (uint32_t e = tid; e < cnt_local; e += kPT) {
          const uint32_t key = v.thr[e], pj = key / plane, rem = key - pj * plane, r = rem / p.W;
          pos[2 * e] = (key & kBlockKey) ? 0xFFFFFFFFu : pj;
          pos[2 * e + 1] = (r << 16) | (rem - r * p.W);
        }
      __syncthreads();
      // a warp per listed pixel, its lanes over the others (a thread per pixel
      // walking the whole list ran 3.7 us an item, a chain of shared loads)
      for (uint32_t e = warp; e < cnt_local; e += kPW) {
        const uint32_t key = v.thr[e];
        bool keep = true;
        if (!(key & kBlockKey)) {
          const float x = v.thrv[e];
          keep = x >= p.amax;
          uint32_t pj, r, c;
          if (decoded) {
            pj = pos[2 * e];
            r = pos[2 * e + 1] >> 16;
            c = pos[2 * e + 1] & 0xFFFFu;
          } else {
            pj = key / plane;
            const uint32_t rem = key - pj * plane;
            r = rem / p.W;
            c = rem - r * p.W;
          }
          bool beaten = false;
          for (uint32_t o = lane; keep && o < cnt_local; o += 32) {
            if (o == e) continue;
            uint32_t pj2, r2, c2;
            if (decoded) {
              pj2 = pos[2 * o];  // a listed block: no panel matches
              r2 = pos[2 * o + 1] >> 16;
              c2 = pos[2 * o + 1] & 0xFFFFu;
            } else {
              const uint32_t k2 = v.thr[o];
              if (k2 & kBlockKey) continue;  // a listed block
              pj2 = k2 / plane;
              const uint32_t rem2 = k2 - pj2 * plane;
              r2 = rem2 / p.W;
              c2 = rem2 - r2 * p.W;
            }
            if (pj2 != pj) continue;  // another panel, or a listed block
            const int dr = (int)r2 - (int)r, dc = (int)c2 - (int)c;
            if (dr > p.rank || -dr > p.rank || dc > p.rank || -dc > p.rank) continue;
            const float y = v.thrv[o];
            if (y > x || (y == x && v.thr[o] < key)) beaten = true;
          }
          keep = keep && !__any_sync(0xffffffffu, beaten);
        }
        if (keep && lane == 0) v.cand[atomicAdd(v.ctl + CTL_NCAND, 1u)] = key;
      }
      __syncthreads();
      const uint32_t n_cand = v.ctl[CTL_NCAND];
      for (uint32_t e = warp; e < n_cand; e += kPW) test_listed(v.cand[e]);
      // the spilled candidates (written before the barriers above)
      for (uint32_t e = warp; e < cnt - cnt_local; e += kPW) test_listed(spill_at(e));
    } else {
      // every pixel >= amax_thr of the item, one warp test each
      auto scan_all = [&]() {
        const uint32_t n_px = kp * plane;
        for (uint32_t base = warp * 32; base < n_px; base += kPW * 32) {
          const uint32_t lp = base + lane;
          const bool hot = lp < n_px && __ldg(item_px + lp) >= p.amax;
          uint32_t m = __ballot_sync(0xffffffffu, hot);
          while (m) {
            const uint32_t l = __ffs(m) - 1;
            m &= m - 1;
            test(base + l);
          }
        }

      };
      if constexpr (kDense || kRt) {
        if (dense) {
          if (sh.band_rows >= 2u * (uint32_t)peak_reach(p) + 2u) {
            dense_band_peaks(p, s, sh, v, item_px, kp, fu);
          } else {
          // many candidates (hot pixels): one lane per candidate.  The warp gathers
          // the pixels >= amax_thr of its slices, 32 at a time, and each lane runs
          // the local-maximum rule and the evaluation on its own candidate in the
          // sequential order the warp tests reproduce (is_local_max_at,
          // evaluate_peak_at), so a warp instruction serves 32 candidates
          const uint32_t n_px = kp * plane;
          uint32_t mine = 0, nq = 0;  // nq: candidates held by lanes 0 .. nq - 1 (the same in every lane)
          auto flush = [&]() {
            if (lane < nq) {
              const uint32_t pj = mine / plane, rem = mine - pj * plane;
              const int r = (int)(rem / p.W), c = (int)(rem - (uint32_t)r * p.W);
              const float* pan = item_px + (size_t)pj * plane;
              auto px = [&](int dr, int dc) { return __ldg(pan + (size_t)(r + dr) * p.W + (c + dc)); };
              if (is_local_max_at(px, (int)p.H, (int)p.W, r, c, p) && evaluate_peak_at(px, (int)p.H, (int)p.W, r, c, p)) {
                const uint32_t slot = atomicAdd(v.ctl + CTL_ACC, 1u);
                if (slot < sh.sort_n2) v.acc[slot] = mine;
              }
            }
            __syncwarp();
            nq = 0;
          };
          for (uint32_t base = warp * 32; base < n_px; base += kPW * 32) {
            const uint32_t lp = base + lane;
            const bool hot = lp < n_px && __ldg(item_px + lp) >= p.amax;
            uint32_t m = __ballot_sync(0xffffffffu, hot);
            while (m) {
              // the first `take` hot lanes hand their pixels to lanes nq .. nq + take - 1
              // (this fallback serves panels too wide for a band of rows in shared memory)
              // through the warp's 32 slots of the candidate list (unused on this path)
              static_assert(kThrLocalCap >= kPW * 32, "32 candidate slots per warp");
              uint32_t* q = v.cand + warp * 32;
              const uint32_t take = min((uint32_t)__popc(m), 32u - nq);
              const uint32_t k = __popc(m & lanemask_lt());
              const bool go = ((m >> lane) & 1u) && k < take;
              if (go) q[nq + k] = base + lane;
              m &= ~__ballot_sync(0xffffffffu, go);
              __syncwarp();
              if (lane >= nq && lane < nq + take) mine = q[lane];
              __syncwarp();
              nq += take;
              if (nq == 32) flush();
            }
          }
          if (nq) flush();
          }
        } else {
          scan_all();
        }
      } else {
        scan_all();
      }
    }
    __syncthreads();
    const uint32_t n_acc = v.ctl[CTL_ACC];
    if (n_acc <= p.max_peaks) {  // sort the item's peaks: (panel, row, col) order
      uint32_t n2 = 1;
      while (n2 < n_acc) n2 <<= 1;
      for (uint32_t k = n_acc + tid; k < n2; k += kPT) v.acc[k] = 0xFFFFFFFFu;
      __syncthreads();
      for (uint32_t size = 2; size <= n2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t k = tid; k < n2; k += kPT) {
            const uint32_t partner = k ^ stride;
            if (partner > k) {
              const bool upw = (k & size) == 0;
              const uint32_t x = v.acc[k], y = v.acc[partner];
              if ((x > y) == upw) {
                v.acc[k] = y;
                v.acc[partner] = x;
              }
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t k = tid; k < n_acc; k += kPT) s.peak_part[fu * sh.peak_cap + k] = pn0 * plane + v.acc[k];
    }
    if (tid == 0) s.peak_part_count[fu] = n_acc;
  }
  __syncthreads();
  if (tid == 0 && v.ctl[CTL_TIMEOUT]) {  // a copy never arrived: the frame is marked, see frame_codebook
    s.peak_part_count[fu] = kPanelTimedOut;
    v.ctl[CTL_TIMEOUT] = 0;
  }
  if (trace) trace[2] = global_ns();
}

// ---------------------------------------------------------------------------
// After its panels, a frame moves through three more stages:
//   (1) the CTA that completes the frame's last panel gathers the peak list
//       and builds the codebook;
//   (2) chunk-size items count the bits and outliers of groups of chunks;
//       the last one scans, lays the frame out and writes its head;
//   (3) chunk-write items pack the bits, write the outliers and the ROI
//       windows, and drop their code bytes from L2.
// One atomic ticket counter orders all work: round r holds the panels of
// frame r, the size items of frame r - lag1 and the write items of frame
// r - lag1 - lag2.  Stages hand over through release/acquire flags.  A CTA only
// ever waits for work handed out to an earlier ticket, which is running or
// done, so every wait ends; waits are bounded anyway (ROIBIN_ERR_TIMEOUT).
constexpr uint32_t kWaitLimit = 1u << 22;

// Per-frame words, zeroed before each launch:
//   panel_done, size_done   streaming / size items finished;
//   ready_cb, ready_plan    the codebook / the plan is published;
//   timed_out               set by any item whose flag wait gave up (sticky: no
//                           later write of the frame's status can clear it);
//   fin_count               the plan and the write items finished; the one that
//                           finishes last settles the frame's status;
//   chunk_done              (per chunk of frames) frames whose peaks are known.
struct SyncWords {
  uint32_t *panel_done, *size_done, *ready_cb, *ready_plan, *timed_out, *fin_count, *chunk_done, *ticket;
};
__device__ __forceinline__ SyncWords sync_words(const Scratch& s, uint32_t n) {
  SyncWords w;
  w.panel_done = s.frame_done;
  w.size_done = s.frame_done + n;
  w.ready_cb = s.frame_done + 2 * n;
  w.ready_plan = s.frame_done + 3 * n;
  w.timed_out = s.frame_done + 4 * n;
  w.fin_count = s.frame_done + 5 * n;
  w.chunk_done = s.frame_done + 6 * n;
  w.ticket = s.frame_done + kSyncWordsPerFrame * n;
  return w;
}

// Called by thread 0 of the plan and of every write item of frame g once its
// work is visible (after a __threadfence): the last of them to finish sees
// every give-up of the frame's items, and a frame any of them gave up on is
// reported ROIBIN_ERR_TIMEOUT with no bytes, whatever the plan wrote before.
__device__ __forceinline__ void finish_frame_item(const PlainArgs& a, const FusedShape& sh, const SyncWords& sw,
                                                  uint32_t g) {
  if (atomicAdd(sw.fin_count + g, 1u) != sh.groups) return;
  __threadfence();
  if (__ldcg(sw.timed_out + g)) {
    a.frame_status[g] = ROIBIN_ERR_TIMEOUT;
    a.frame_bytes[g] = 0;
  }
}

__device__ __forceinline__ void flag_release(uint32_t* f) {
  __threadfence();
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(1u) : "memory");
}
__device__ __forceinline__ uint32_t flag_acquire(const uint32_t* f) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  return v;
}
// Thread 0 waits (bounded: `limit` polls) for a flag; every thread gets the
// outcome.  limit = 0 polls nothing, so the wait gives up at once.
__device__ bool wait_flag(const uint32_t* f, uint32_t* slot, uint32_t limit) {
  if (threadIdx.x == 0) {
    uint32_t ok = 0;
    for (uint32_t i = 0; i < limit; ++i) {
      if (flag_acquire(f)) {
        ok = 1;
        break;
      }
      __nanosleep(128);
    }
    *slot = ok;
  }
  __syncthreads();
  const bool ok = *slot != 0;
  __syncthreads();
  return ok;
}

// (1b) chunks of frames sharing one codebook (§5.3.4; chunk_frames > 1).  Each
// frame's CTA publishes the frame's histogram (in FinView::total) and its
// status after the peaks; the CTA that completes the chunk's last frame sums
// the histograms of the chunk's coded frames (status OK), builds the code,
// gives it to each of them with its distance to the chunk's head (the first
// coded frame, whose stream alone keeps the code lengths), and releases every
// frame of the chunk to its size items.
__device__ void chunk_codebook(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                               unsigned char* sm, uint32_t f, const SyncWords& sw) {
  const FinView v = fin_view(sm, sh);
  const uint32_t tid = threadIdx.x;
  for (uint32_t k = tid; k < p.nsym; k += kPT) s.hist[(size_t)f * kMaxSymbols + k] = v.total[k];
  if (tid == 0) s.status[f] = (int32_t)v.ctl[CTL_STATUS];
  __threadfence();
  __syncthreads();
  const uint32_t j = f / p.chunk, c0 = j * p.chunk, c1 = min(a.n_frames, c0 + p.chunk);
  if (tid == 0) v.ctl[CTL_LAST] = atomicAdd(sw.chunk_done + j, 1u) == c1 - c0 - 1 ? 1u : 0u;
  __syncthreads();
  if (!v.ctl[CTL_LAST]) return;  // another frame's CTA completes the chunk
  __threadfence();
  if (tid == 0) {
    int head = -1;
    for (uint32_t g = c0; g < c1 && head < 0; ++g)
      if (__ldcg(s.status + g) == ROIBIN_OK) head = (int)g;
    v.ctl[CTL_CARRY1] = head < 0 ? 0xFFFFFFFFu : (uint32_t)head;
  }
  __syncthreads();
  const uint32_t head = v.ctl[CTL_CARRY1];
  if (head != 0xFFFFFFFFu) {
    for (uint32_t k = tid; k < p.nsym; k += kPT) {
      uint32_t t = 0;
      for (uint32_t g = head; g < c1; ++g)
        if (__ldcg(s.status + g) == ROIBIN_OK) t += __ldcg(s.hist + (size_t)g * kMaxSymbols + k);
      v.total[k] = t;
    }
    __syncthreads();
    const int cb = build_codebook(v.total, p.nsym, *v.hs, v.cb_len, v.cb_code);
    for (uint32_t g = head; g < c1; ++g) {
      if (__ldcg(s.status + g) != ROIBIN_OK) continue;
      for (uint32_t k = tid; k < p.nsym; k += kPT) {
        s.cb_len[(size_t)g * kMaxSymbols + k] = v.cb_len[k];
        s.cb_code[(size_t)g * kMaxSymbols + k] = v.cb_code[k];
      }
    }
    __syncthreads();
    if (tid == 0)
      for (uint32_t g = head; g < c1; ++g) {
        if (__ldcg(s.status + g) != ROIBIN_OK) continue;
        s.chunk_ref[g] = g - head;
        if (cb != ROIBIN_OK) s.status[g] = cb;
      }
  }
  __syncthreads();
  if (tid == 0)
    for (uint32_t g = c0; g < c1; ++g) flag_release(sw.ready_cb + g);
}

// The 3-D predictor (a6 over the panel stack, §6) from the streamed 2-D
// residuals: the 3-D residual of a bin is, exactly in integers, its 2-D
// residual minus the 2-D residual of the same bin in the panel before (the
// panel's own residual for the first panel).  One CTA rewrites the frame's
// code bytes, escape codes and Lorenzo-outlier deltas in place.  A bin's new
// value depends only on the same bin of the panel below, so the panel's bins
// are taken in slices, and a slice goes from the last panel down: the slice of
// the panel below is read into shared memory (16-byte loads of whole lines),
// the panel's new bytes are written from there, and that slice becomes the
// next step's own.  The frame's histogram of the new codes goes to `total`.
// `stage` is the Huffman scratch (unused until the codebook is built).
__device__ __noinline__ void stack_residuals(const DevParams& p, const Scratch& s, const FusedShape& sh, uint32_t* total,
                                             unsigned char* stage, uint32_t f) {
  const uint32_t tid = threadIdx.x, lane = lane_id();
  for (uint32_t k = tid; k < p.nsym; k += kPT) total[k] = 0;
  uint8_t* codes = s.codes8 + (size_t)f * sh.codes_stride;  // 16-byte aligned (whole chunks per frame)
  uint16_t* esc = s.codes + (size_t)f * p.M;
  int32_t* lo = s.lo_delta + (size_t)f * p.M;
  const uint32_t Mp = p.Hb * p.Wb;  // even: the fused path has an even binned width
  const int32_t R = p.R;
  // two slice buffers in the stage, each a slice plus the 15 bytes before its first line
  constexpr uint32_t kStage = sizeof(HuffSmem) > 4096 ? (uint32_t)sizeof(HuffSmem) : 4096u;
  constexpr uint32_t kSlice = (kStage / 2 - 16) & ~15u;
  uint8_t* buf[2] = {stage, stage + kSlice + 16};
  uint32_t zeros = 0;  // codes of the zero residual this thread saw (the common code)
  auto residual = [&](uint32_t b, uint32_t bin) -> int32_t {  // the stored 2-D residual from its byte
    if (b == 0) return lo[bin];
    if (b == 255) return (int32_t)esc[bin] - R;
    return (int32_t)b - 128;
  };
  auto count = [&](uint32_t c) {
    if (c == (uint32_t)R) ++zeros;
    else atomicAdd(total + c, 1u);
  };
  // bytes [from, from + len) of the frame's codes into b (byte i at b[(from & 15) + i])
  auto load = [&](uint8_t* b, uint32_t from, uint32_t len) {
    const uint32_t a = from & ~15u, words = (from - a + len + 15) / 16;
    const uint4* src = reinterpret_cast<const uint4*>(codes + a);
    for (uint32_t w = tid; w < words; w += kPT) reinterpret_cast<uint4*>(b)[w] = __ldcg(src + w);
  };
  __syncthreads();
  for (uint32_t x0 = 0; x0 < Mp; x0 += kSlice) {
    const uint32_t len = min(kSlice, Mp - x0);  // even (Mp and kSlice are)
    uint32_t cur = 0;
    load(buf[cur], (p.P - 1) * Mp + x0, len);
    for (uint32_t pn = p.P - 1; pn >= 1; --pn) {
      const uint32_t at = pn * Mp + x0, below_at = at - Mp;
      load(buf[cur ^ 1u], below_at, len);
      __syncthreads();  // both slices are in shared memory
      const uint8_t* cb8 = buf[cur] + (at & 15u);
      const uint8_t* bb8 = buf[cur ^ 1u] + (below_at & 15u);
      for (uint32_t i = 2 * tid; i < len; i += 2 * kPT) {  // two bins a thread: 2-byte aligned in the frame
        // the common case: both bins hold the zero residual in both panels, so
        // the new residuals are zero too and the stored bytes stay as they are
        if (*reinterpret_cast<const uint16_t*>(cb8 + i) == 0x8080u &&
            *reinterpret_cast<const uint16_t*>(bb8 + i) == 0x8080u) {
          zeros += 2;
          continue;
        }
        uint32_t pair = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t bin = at + i + j;
          const uint32_t cb = cb8[i + j], bb = bb8[i + j];
          int32_t d3;
          if (cb != 0 && cb != 255 && bb != 0 && bb != 255) d3 = (int32_t)cb - (int32_t)bb;  // both ordinary
          else d3 = (int32_t)((uint32_t)residual(cb, bin) - (uint32_t)residual(bb, bin - Mp));  // as the oracle's int64 -> int32
          const uint32_t c = quant_code(d3, R);
          uint32_t y;
          if (c == 0) {
            lo[bin] = d3;
            y = 0;
          } else if (d3 >= -127 && d3 <= 126) {
            y = (uint32_t)(d3 + 128);
          } else {
            esc[bin] = (uint16_t)c;
            y = 255;
          }
          pair |= y << (8 * j);
          count(c);
        }
        *reinterpret_cast<uint16_t*>(codes + at + i) = (uint16_t)pair;
      }
      __syncthreads();  // the slice is done before its buffer takes the next panel's
      cur ^= 1u;
    }
    __syncthreads();  // a single panel: its slice has just been read
    // the first panel keeps its 2-D residuals: only counted
    const uint8_t* cb8 = buf[cur] + (x0 & 15u);
    for (uint32_t i = tid; i < len; i += kPT) count(quant_code(residual(cb8[i], x0 + i), R));
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  if (lane == 0 && zeros) atomicAdd(total + R, zeros);
  __syncthreads();
}

// (1) peak list + codebook of frame f, by the CTA that completed its last streaming item.
__device__ void frame_codebook(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                               unsigned char* sm, uint32_t f, const SyncWords& sw) {
  const FinView v = fin_view(sm, sh);
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  uint64_t* trace = (a.trace && f < a.trace_frames && tid == 0) ? a.trace + (size_t)f * kTracePoints : nullptr;
  if (trace) trace[0] = global_ns();
  // a8: the frame's histogram; prequantisation outliers in the frame
  if (p.dims == 3) {
    stack_residuals(p, s, sh, v.total, sm + sh.off_huff, f);
  } else {
    for (uint32_t k = tid; k < p.nsym; k += kPT) {
      uint32_t t = 0;
      for (uint32_t u = 0; u < sh.U; ++u) t += __ldcg(s.hist_part + ((size_t)f * p.P + u) * kMaxSymbols + k);
      v.total[k] = t;
    }
  }
  if (tid == 0) {
    uint32_t t = 0;
    for (uint32_t pn = 0; pn < p.P; ++pn) t += __ldcg(s.pq_part_count + (size_t)f * p.P + pn);
    s.plan[f].n_pq = t;  // provisional: read by the size items to skip the outlier bits
    v.ctl[CTL_STATUS] = ROIBIN_OK;
    v.ctl[CTL_BAD] = 0;
    v.ctl[CTL_CARRY0] = 0;
  }
  __syncthreads();
  // the peak list: per-item sorted lists concatenated in item (= panel) order, or the user's
  uint32_t* keys = a.peaks_key_out + (size_t)f * p.max_peaks;
  if (a.user_peaks) {
    const uint32_t n = a.user_npeaks[f];
    if (tid == 0) {
      v.ctl[CTL_CARRY0] = n;
      for (uint32_t u = 0; u < sh.U; ++u)
        if (__ldcg(s.peak_part_count + (size_t)f * p.P + u) == kPanelTimedOut)
          v.ctl[CTL_BAD] = 2;
    }
    if (n > p.max_peaks) {
      if (tid == 0) v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_ERR_CAPACITY;
    } else {
      const uint16_t* up = a.user_peaks + (size_t)f * p.max_peaks * 3;
      for (uint32_t k = tid; k < n; k += kPT) {
        const uint32_t pn = up[3 * k], r = up[3 * k + 1], c = up[3 * k + 2];
        if (pn >= p.P || r >= p.H || c >= p.W) v.ctl[CTL_BAD] = 1;
        else keys[k] = (pn * p.H + r) * p.W + c;
      }
    }
  } else {
    if (tid == 0) {
      uint32_t n = 0;
      bool over = false;
      bool timeout = false;
      for (uint32_t u = 0; u < sh.U; ++u) {
        const uint32_t c = __ldcg(s.peak_part_count + (size_t)f * p.P + u);
        if (c == kPanelTimedOut) timeout = true;
        else if (c > p.max_peaks) over = true;
        v.offs[u] = n;
        if (c != kPanelTimedOut) n += c;
      }
      if (over || n > p.max_peaks) v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_ERR_CAPACITY;
      if (timeout) v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_ERR_TIMEOUT;
      v.ctl[CTL_CARRY0] = timeout ? 0 : n;
    }
    __syncthreads();
    if (v.ctl[CTL_STATUS] == ROIBIN_OK) {
      for (uint32_t u = warp; u < sh.U; u += kPW) {
        const uint32_t c = __ldcg(s.peak_part_count + (size_t)f * p.P + u), off = v.offs[u];
        for (uint32_t k = lane; k < c; k += 32)
          keys[off + k] = __ldcg(s.peak_part + ((size_t)f * p.P + u) * sh.peak_cap + k);
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (v.ctl[CTL_BAD] == 2) v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_ERR_TIMEOUT;
    else if (v.ctl[CTL_BAD] && v.ctl[CTL_STATUS] == ROIBIN_OK) v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_ERR_INVALID_ARG;
    // non-hit rejection (§1, §4): too few peaks, the frame is not compressed
    if (v.ctl[CTL_STATUS] == ROIBIN_OK && v.ctl[CTL_CARRY0] < (uint32_t)p.nhr_min)
      v.ctl[CTL_STATUS] = (uint32_t)ROIBIN_REJECTED;
    a.peaks_count_out[f] = v.ctl[CTL_CARRY0];
  }
  if (trace) trace[1] = global_ns();
  if (p.chunk > 1) {
    chunk_codebook(p, s, a, sh, sm, f, sw);
    return;
  }
  // a9: the codebook, published in the frame's global tables
  const int cb = build_codebook(v.total, p.nsym, *v.hs, v.cb_len, v.cb_code);
  for (uint32_t k = tid; k < p.nsym; k += kPT) {
    s.cb_len[(size_t)f * kMaxSymbols + k] = v.cb_len[k];
    s.cb_code[(size_t)f * kMaxSymbols + k] = v.cb_code[k];
  }
  if (tid == 0) {
    int32_t st = (int32_t)v.ctl[CTL_STATUS];
    if (st == ROIBIN_OK && cb != ROIBIN_OK) st = cb;
    s.status[f] = st;
  }
  __syncthreads();
  if (trace) trace[2] = global_ns();
  if (tid == 0) flag_release(sw.ready_cb + f);
}

// Per-byte tables of a frame's codebook (byte = stored code byte):
//   btab[b] = codeword << 32 | length  (0 for the escape byte 255)
//   ctab[b] = length | (b == 0) << 21 | (b == 255) << 42, so that summing
//             ctab over a lane's bytes counts bits, Lorenzo outliers and
//             escapes in one 64-bit add per symbol.
constexpr uint32_t kField = 21;
__device__ void load_byte_tables(const DevParams& p, const Scratch& s, uint32_t f, uint64_t* btab, uint64_t* ctab) {
  for (uint32_t b = threadIdx.x; b < 256; b += kPT) {
    uint64_t e = 0;
    if (b != 255) {
      const int32_t code = b == 0 ? 0 : (int32_t)b - 128 + p.R;
      if (code >= 0 && code < (int32_t)p.nsym) {
        const uint32_t L = __ldcg(s.cb_len + (size_t)f * kMaxSymbols + code);
        const uint32_t cw = __ldcg(s.cb_code + (size_t)f * kMaxSymbols + code);
        e = ((uint64_t)cw << 32) | L;
      }
    }
    btab[b] = e;
    ctab[b] = (e & 0xFFu) | ((uint64_t)(b == 0) << kField) | ((uint64_t)(b == 255) << (2 * kField));
  }
}

// (length, codeword) of the symbol stored as byte b at bin `bin` of frame f.
__device__ __forceinline__ uint64_t symbol_entry(const DevParams& p, const Scratch& s, uint32_t f, const uint64_t* btab,
                                                 uint32_t b, uint32_t bin) {
  uint64_t e = btab[b];
  if (b == 255) {  // escape: the code sits in the side array
    const uint32_t code = __ldcg(s.codes + (size_t)f * p.M + bin);
    e = ((uint64_t)__ldcg(s.cb_code + (size_t)f * kMaxSymbols + code) << 32) |
        __ldcg(s.cb_len + (size_t)f * kMaxSymbols + code);
  }
  return e;
}

__device__ __forceinline__ uint32_t pq_bit_of(const DevParams& p, const Scratch& s, const FusedShape& sh, uint32_t f,
                                              uint32_t bin) {
  const uint32_t Mp = p.Hb * p.Wb;
  const uint32_t pn = bin / Mp, lb = bin - pn * Mp;
  // a panel without prequantisation outliers never wrote its mask words
  if (__ldcg(s.pq_part_count + (size_t)f * p.P + pn) == 0) return 0u;
  return (__ldcg(s.pq_mask + ((size_t)f * p.P + pn) * sh.mask_words + (lb >> 5)) >> (lb & 31)) & 1u;
}

// A warp stages one chunk's 4096 code bytes in its shared buffer with
// coalesced 16-byte loads; word w of the chunk sits at w + w / 32, so lane l
// reading its words 32 l .. 32 l + 31 hits 32 different banks.
constexpr uint32_t kStageWords = kChunk / 4 + kChunk / 128;  // 1056
__device__ __forceinline__ void stage_chunk(const uint8_t* codes_frame, uint32_t k, uint32_t* wbuf) {
  const uint4* src = reinterpret_cast<const uint4*>(codes_frame + (size_t)k * kChunk);
  const uint32_t lane = lane_id();
  uint4 u[8];
#pragma unroll
  for (int it = 0; it < 8; ++it) u[it] = __ldcg(src + it * 32 + lane);
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const uint32_t w = 4 * (it * 32 + lane);
    uint32_t* d = wbuf + w + (w >> 5);
    d[0] = u[it].x;
    d[1] = u[it].y;
    d[2] = u[it].z;
    d[3] = u[it].w;
  }
  __syncwarp();
}

// Bits, Lorenzo outliers and prequantisation outliers of the lane's 128
// symbols [s0, s1) of a staged chunk: one table add per symbol; escapes (rare)
// are resolved afterwards.
__device__ __forceinline__ void lane_counts(const DevParams& p, const Scratch& s, const FusedShape& sh, uint32_t f,
                                            const uint64_t* btab, const uint64_t* ctab, const uint32_t* wbuf,
                                            uint32_t s0, uint32_t s1, bool any_pq, uint32_t& bits, uint32_t& nlo,
                                            uint32_t& npq) {
  const uint32_t* lw = wbuf + 33 * lane_id();
  const uint32_t n = s1 > s0 ? s1 - s0 : 0;  // symbols of this lane (<= 128)
  const uint32_t full = n >> 2;
  uint64_t acc = 0;
  const uint64_t c4 = 4 * ctab[0x80];  // four zero residuals
#pragma unroll 4
  for (uint32_t w = 0; w < full; ++w) {
    const uint32_t word = lw[w];
    if (word == 0x80808080u)
      acc += c4;
    else
      acc += ctab[word & 0xFFu] + ctab[(word >> 8) & 0xFFu] + ctab[(word >> 16) & 0xFFu] + ctab[word >> 24];
  }
  if (n & 3u) {
    const uint32_t word = lw[full];
    for (uint32_t t = 0; t < (n & 3u); ++t) acc += ctab[(word >> (8 * t)) & 0xFFu];
  }
  const uint64_t mask = (1ull << kField) - 1;
  bits = (uint32_t)(acc & mask);
  nlo = (uint32_t)((acc >> kField) & mask);
  const uint32_t nesc = (uint32_t)(acc >> (2 * kField));
  if (nesc) {
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t b = (lw[i >> 2] >> (8 * (i & 3))) & 0xFFu;
      if (b == 255) bits += (uint32_t)symbol_entry(p, s, f, btab, b, s0 + i);
    }
  }
  npq = 0;
  if (any_pq)
    for (uint32_t i = s0; i < s1; ++i) npq += pq_bit_of(p, s, sh, f, i);
}

// (2) chunk sizes of one group of chunks of frame g.
__device__ void size_item(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                          unsigned char* sm, uint32_t g, uint32_t grp, const SyncWords& sw) {
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  uint32_t* ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  uint64_t* btab = reinterpret_cast<uint64_t*>(sm + sh.off_huff);
  uint64_t* ctab = btab + 256;
  unsigned long long* acct = (a.trace && g < a.trace_frames && tid == 0)
                                 ? reinterpret_cast<unsigned long long*>(a.trace + (size_t)g * kTracePoints)
                                 : nullptr;
  const uint64_t t_in = acct ? global_ns() : 0;
  const bool ready = wait_flag(sw.ready_cb + g, ctl + CTL_WAIT, sh.wait_limit);
  if (acct) atomicAdd(acct + 7, (unsigned long long)(global_ns() - t_in));
  if (!ready && tid == 0) atomicOr(sw.timed_out + g, 1u);
  const bool ok = ready && __ldcg(s.status + g) == ROIBIN_OK;
  if (ok) {
    load_byte_tables(p, s, g, btab, ctab);
    __syncthreads();
    const bool any_pq = __ldcg(&s.plan[g].n_pq) != 0;
    const uint8_t* codes = s.codes8 + (size_t)g * sh.codes_stride;
    const uint32_t k_end = min(p.n_chunks, (grp + 1) * sh.group_chunks);
    uint32_t* wbuf = reinterpret_cast<uint32_t*>(sm + sh.off_stage) + warp * kStageWords;
    const uint64_t t_loop = acct ? global_ns() : 0;
    for (uint32_t k = grp * sh.group_chunks + warp; k < k_end; k += kPW) {
      const uint32_t s0 = k * kChunk + lane * 128, s1 = min(p.M, s0 + 128);
      stage_chunk(codes, k, wbuf);
      uint32_t bits, nlo, npq;
      lane_counts(p, s, sh, g, btab, ctab, wbuf, s0, s1, any_pq, bits, nlo, npq);
      __syncwarp();
      const uint32_t bit_incl = warp_incl_scan(bits), lo_incl = warp_incl_scan(nlo), pq_incl = warp_incl_scan(npq);
      // where each lane's bits and outliers start inside the chunk, for the write items
      const size_t o = (size_t)g * p.n_chunks + k;
      s.lane_bit[o * 32 + lane] = bit_incl - bits;
      s.lane_lo[o * 32 + lane] = lo_incl - nlo;
      s.lane_pq[o * 32 + lane] = pq_incl - npq;
      if (lane == 31) {
        s.chunk_words[o] = (bit_incl + 31) / 32;
        s.chunk_lo[o] = lo_incl;
        s.chunk_pq[o] = pq_incl;
      }
    }
    __syncthreads();
    if (acct) atomicAdd(acct + 9, (unsigned long long)(global_ns() - t_loop));
  }
  if (acct) atomicAdd(acct + 5, (unsigned long long)(global_ns() - t_in));
  __threadfence();
  __syncthreads();
  if (tid == 0) ctl[CTL_LAST] = atomicAdd(sw.size_done + g, 1u) == sh.groups - 1 ? 1u : 0u;
  __syncthreads();
  if (!ctl[CTL_LAST]) return;
  __threadfence();
  // the frame's plan: scan the chunks, lay the frame out, write its head
  uint64_t* trace = (a.trace && g < a.trace_frames && tid == 0) ? a.trace + (size_t)g * kTracePoints : nullptr;
  if (trace) trace[3] = global_ns();
  // a size item of the frame that gave up waiting for the codebook left the
  // chunk counts unfinished: the frame stops here (its give-up was published
  // before its size_done increment, which this CTA has seen)
  int32_t st = __ldcg(sw.timed_out + g) ? ROIBIN_ERR_TIMEOUT : __ldcg(s.status + g);
  const uint32_t ref = p.chunk > 1 ? __ldcg(s.chunk_ref + g) : 0u;  // frames back to the chunk's head
  uint32_t* cw = reinterpret_cast<uint32_t*>(sm + sh.off_cw);
  uint32_t* clo = cw + p.n_chunks;
  uint32_t* cpq = clo + p.n_chunks;
  FramePlan pl{};
  if (st == ROIBIN_OK) {
    if (tid < 3) ctl[CTL_CARRY0 + tid] = 0;
    for (uint32_t k = tid; k < p.n_chunks; k += kPT) {
      const size_t o = (size_t)g * p.n_chunks + k;
      cw[k] = __ldcg(s.chunk_words + o);
      clo[k] = __ldcg(s.chunk_lo + o);
      cpq[k] = __ldcg(s.chunk_pq + o);
    }
    __syncthreads();
    for (uint32_t k0 = 0; k0 < p.n_chunks; k0 += kPT) {
      const uint32_t k = k0 + tid;
      const uint32_t w = k < p.n_chunks ? cw[k] : 0u, l = k < p.n_chunks ? clo[k] : 0u,
                     q = k < p.n_chunks ? cpq[k] : 0u;
      uint32_t tw, tl, tq;
      const uint32_t ew = block_excl_scan(w, ctl + CTL_TMP, &tw);
      const uint32_t el = block_excl_scan(l, ctl + CTL_TMP, &tl);
      const uint32_t eq = block_excl_scan(q, ctl + CTL_TMP, &tq);
      if (k < p.n_chunks) {
        cw[k] = ctl[CTL_CARRY0] + ew;
        clo[k] = ctl[CTL_CARRY1] + el;
        cpq[k] = ctl[CTL_CARRY2] + eq;
      }
      __syncthreads();
      if (tid == 0) {
        ctl[CTL_CARRY0] += tw;
        ctl[CTL_CARRY1] += tl;
        ctl[CTL_CARRY2] += tq;
      }
      __syncthreads();
    }
    pl.n_peaks = __ldcg(a.peaks_count_out + g);
    pl.n_words = ctl[CTL_CARRY0];
    pl.n_lo = ctl[CTL_CARRY1];
    pl.n_pq = ctl[CTL_CARRY2];
    pl.off_peaks = kHeaderBytes;
    pl.off_roi = pl.off_peaks + align16((uint64_t)pl.n_peaks * 6);
    pl.off_len = pl.off_roi + roi_in_place_bytes(p, pl.n_peaks);
    pl.off_cidx = pl.off_len + (ref == 0 ? align16(p.nsym) : 0);  // a chunk's head keeps the lengths
    pl.off_lo = pl.off_cidx + align16((uint64_t)p.n_chunks * 4);
    pl.off_pq = pl.off_lo + align16((uint64_t)pl.n_lo * 8);
    pl.off_bits = pl.off_pq + align16((uint64_t)pl.n_pq * 8);
    pl.total = pl.off_bits + align16((uint64_t)pl.n_words * 4);
    if (pl.total > a.out_stride) st = ROIBIN_ERR_CAPACITY;
  }
  if (tid == 0) {
    a.frame_bytes[g] = (st == ROIBIN_OK || st == ROIBIN_ERR_CAPACITY) ? pl.total : 0;
    a.frame_status[g] = st;
    s.status[g] = st;
  }
  if (st == ROIBIN_OK) {
    for (uint32_t k = tid; k < p.n_chunks; k += kPT) {  // offsets for the write items
      const size_t o = (size_t)g * p.n_chunks + k;
      s.chunk_words[o] = cw[k];
      s.chunk_lo[o] = clo[k];
      s.chunk_pq[o] = cpq[k];
    }
    if (tid == 0) s.plan[g] = pl;
    if (RB_CHECK(s, pl.total <= a.out_stride, ROIBIN_CHECK_PLAN_TOTAL))
      write_frame_head(a.out + (size_t)g * a.out_stride, p, pl, a.peaks_key_out + (size_t)g * p.max_peaks,
                       s.cb_len + (size_t)g * kMaxSymbols, cw, ref);
  }
  __syncthreads();
  if (trace) trace[4] = global_ns();
  if (tid == 0) {
    flag_release(sw.ready_plan + g);
    finish_frame_item(a, sh, sw, g);
  }
}

// (3) bits, outliers and ROI windows of one group of chunks of frame g.
__device__ void write_item_work(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                                unsigned char* sm, uint32_t g, uint32_t grp, unsigned long long* acct,
                                uint64_t t_in);

__device__ void write_item(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                           unsigned char* sm, uint32_t g, uint32_t grp, const SyncWords& sw) {
  const uint32_t tid = threadIdx.x;
  uint32_t* ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  unsigned long long* acct = (a.trace && g < a.trace_frames && tid == 0)
                                 ? reinterpret_cast<unsigned long long*>(a.trace + (size_t)g * kTracePoints)
                                 : nullptr;
  const uint64_t t_in = acct ? global_ns() : 0;
  const bool ready = wait_flag(sw.ready_plan + g, ctl + CTL_WAIT, sh.wait_limit);
  if (acct) atomicAdd(acct + 8, (unsigned long long)(global_ns() - t_in));
  if (!ready && tid == 0) atomicOr(sw.timed_out + g, 1u);
  // a plan that gave up (timed_out, published before ready_plan) wrote no
  // layout for this launch: nothing of the frame is written then
  if (ready && __ldcg(sw.timed_out + g) == 0 && __ldcg(s.status + g) == ROIBIN_OK)
    write_item_work(p, s, a, sh, sm, g, grp, acct, t_in);
  __threadfence();
  __syncthreads();
  if (tid == 0) finish_frame_item(a, sh, sw, g);
}

__device__ void write_item_work(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                                unsigned char* sm, uint32_t g, uint32_t grp, unsigned long long* acct,
                                uint64_t t_in) {
  const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  uint64_t* btab = reinterpret_cast<uint64_t*>(sm + sh.off_huff);
  uint64_t* ctab = btab + 256;
  load_byte_tables(p, s, g, btab, ctab);
  FramePlan pl;
  pl.n_peaks = __ldcg(&s.plan[g].n_peaks);
  pl.n_pq = __ldcg(&s.plan[g].n_pq);
  pl.n_words = __ldcg(&s.plan[g].n_words);
  pl.off_roi = __ldcg(reinterpret_cast<const unsigned long long*>(&s.plan[g].off_roi));
  pl.off_lo = __ldcg(reinterpret_cast<const unsigned long long*>(&s.plan[g].off_lo));
  pl.off_pq = __ldcg(reinterpret_cast<const unsigned long long*>(&s.plan[g].off_pq));
  pl.off_bits = __ldcg(reinterpret_cast<const unsigned long long*>(&s.plan[g].off_bits));
#ifdef ROIBIN_CHECKS
  pl.n_lo = __ldcg(&s.plan[g].n_lo);  // the bounds of the checks below
  pl.total = __ldcg(reinterpret_cast<const unsigned long long*>(&s.plan[g].total));
#endif
  __syncthreads();
  uint8_t* out = a.out + (size_t)g * a.out_stride;
  uint32_t* words = reinterpret_cast<uint32_t*>(out + pl.off_bits);
  uint2* lo_out = reinterpret_cast<uint2*>(out + pl.off_lo);
  uint2* pq_out = reinterpret_cast<uint2*>(out + pl.off_pq);
  const bool any_pq = pl.n_pq != 0;
  const uint8_t* codes = s.codes8 + (size_t)g * sh.codes_stride;
  const int32_t* lo_delta = s.lo_delta + (size_t)g * p.M;
  const uint32_t* pq_bits = s.pq_bits + (size_t)g * p.M;
  const uint32_t k_begin = grp * sh.group_chunks, k_end = min(p.n_chunks, (grp + 1) * sh.group_chunks);
  uint32_t* wbuf = reinterpret_cast<uint32_t*>(sm + sh.off_stage) + warp * kStageWords;
  // eight zero-residual symbols at once (their codeword repeated), when they fit 32 bits
  const uint64_t zero_entry = btab[0x80];
  const uint32_t len1 = (uint32_t)zero_entry, cw1 = (uint32_t)(zero_entry >> 32);
  const bool run8 = len1 >= 1 && len1 <= 4;
  const uint32_t len8 = 8 * len1;
  uint32_t cw8 = 0;
  if (run8)
    for (int t = 0; t < 8; ++t) cw8 = (cw8 << len1) | cw1;
  // and 32 of them at once when their codeword is one bit (a 32-bit word of it)
  const bool run32 = len1 == 1;
  const uint32_t cw32 = cw1 ? 0xFFFFFFFFu : 0u;
  const uint64_t t_loop = acct ? global_ns() : 0;
  for (uint32_t k = k_begin + warp; k < k_end; k += kPW) {
    const size_t o = (size_t)g * p.n_chunks + k;
    const uint32_t w0 = __ldcg(s.chunk_words + o);
    // In a full chunk every lane codes 128 symbols (>= 128 bits), so a word is
    // shared by at most two neighbouring lanes: lane l keeps its first, partial
    // word and ORs in lane l-1's last, partial word received by shuffle; every
    // word is then written once.  The frame's last chunk may be partial: its
    // words are zeroed and the shared ones merged with atomics.
    const bool full = (k + 1) * kChunk <= p.M;
    if (!full) {
      const uint32_t w1 = pl.n_words;
      for (uint32_t w = w0 + lane; w < w1; w += 32)
        if (RB_CHECK(s, (uint64_t)pl.off_bits + 4ull * (w + 1) <= pl.total, ROIBIN_CHECK_BITSTREAM)) words[w] = 0;
      __threadfence_block();
      __syncwarp();
    }
    const uint32_t s0 = k * kChunk + lane * 128, s1 = min(p.M, s0 + 128);
    stage_chunk(codes, k, wbuf);
    const uint32_t start = __ldcg(s.lane_bit + o * 32 + lane);
    const uint32_t first_idx = w0 + start / 32;
    uint32_t wi = first_idx;
    uint64_t accb = 0;
    uint32_t nacc = start & 31u;
    bool first = nacc != 0;  // the first word is shared with the previous lane
    uint32_t head = 0;       // full chunks: the shared first word, held back
    uint32_t lo_pos = __ldcg(s.chunk_lo + o) + __ldcg(s.lane_lo + o * 32 + lane);
    uint32_t pq_pos = __ldcg(s.chunk_pq + o) + __ldcg(s.lane_pq + o * 32 + lane);
    // append `len` (<= 32) bits, emitting each completed 32-bit word
    auto append = [&](uint32_t cw, uint32_t len) {
      accb |= (uint64_t)cw << (64 - nacc - len);
      nacc += len;
      if (nacc >= 32) {
        const uint32_t word = (uint32_t)(accb >> 32);
        if (first) {
          if (full) head = word;
          else if (RB_CHECK(s, wi < pl.n_words, ROIBIN_CHECK_BITSTREAM)) atomicOr(words + wi, word);
        } else if (RB_CHECK(s, wi < pl.n_words, ROIBIN_CHECK_BITSTREAM)) {
          words[wi] = word;
        }
        first = false;
        ++wi;
        accb <<= 32;
        nacc -= 32;
      }
    };
    const uint32_t* lw = wbuf + 33 * lane;
    const uint32_t n = s1 > s0 ? s1 - s0 : 0;
    for (uint32_t w = 0; w < (n + 3) / 4; ++w) {
      const uint32_t word = lw[w];
      const uint32_t cnt = min(4u, n - 4 * w);
      // fastest path: 32 zero residuals (bytes 0x80) in a row, one append of a full word
      if (run32 && 4 * w + 32 <= n) {
        uint32_t all = word, any = word;
#pragma unroll
        for (uint32_t t = 1; t < 8; ++t) {
          all &= lw[w + t];
          any |= lw[w + t];
        }
        if (all == 0x80808080u && any == 0x80808080u) {
          append(cw32, 32);
          w += 7;
          continue;
        }
      }
      // next: eight zero residuals in a row, one append
      if (run8 && 4 * w + 8 <= n && (word & lw[w + 1]) == 0x80808080u && (word | lw[w + 1]) == 0x80808080u) {
        append(cw8, len8);
        ++w;
        continue;
      }
      // fast path: four ordinary bytes (no 0 = outlier, no 255 = escape) whose
      // codewords fit 32 bits together are appended at once
      const bool has0 = ((word - 0x01010101u) & ~word & 0x80808080u) != 0;
      const bool has255 = ((~word - 0x01010101u) & word & 0x80808080u) != 0;
      if (cnt == 4 && !has0 && !has255) {
        const uint64_t e0 = btab[word & 0xFFu], e1 = btab[(word >> 8) & 0xFFu], e2 = btab[(word >> 16) & 0xFFu],
                       e3 = btab[word >> 24];
        const uint32_t L0 = (uint32_t)e0, L1 = (uint32_t)e1, L2 = (uint32_t)e2, L3 = (uint32_t)e3;
        if (L0 + L1 + L2 + L3 <= 32) {
          uint32_t combo = (uint32_t)(e0 >> 32);
          combo = (combo << L1) | (uint32_t)(e1 >> 32);
          combo = (combo << L2) | (uint32_t)(e2 >> 32);
          combo = (combo << L3) | (uint32_t)(e3 >> 32);
          append(combo, L0 + L1 + L2 + L3);
          continue;
        }
      }
      for (uint32_t t = 0; t < cnt; ++t) {
        const uint32_t bin = s0 + 4 * w + t;
        const uint32_t b = (word >> (8 * t)) & 0xFFu;
        const uint64_t e = symbol_entry(p, s, g, btab, b, bin);
        append((uint32_t)(e >> 32), (uint32_t)e);
        if (b == 0 && RB_CHECK(s, lo_pos < pl.n_lo, ROIBIN_CHECK_OUTLIERS))
          lo_out[lo_pos++] = make_uint2(bin, (uint32_t)__ldcg(lo_delta + bin));
      }
    }
    if (full) {
      const uint32_t tail = nacc > 0 ? (uint32_t)(accb >> 32) : 0u;  // shared with the next lane
      const uint32_t prev_tail = __shfl_up_sync(0xffffffffu, tail, 1);
      if ((start & 31u) != 0 && RB_CHECK(s, first_idx < pl.n_words, ROIBIN_CHECK_BITSTREAM))
        words[first_idx] = head | prev_tail;
      if (lane == 31 && nacc > 0 && RB_CHECK(s, wi < pl.n_words, ROIBIN_CHECK_BITSTREAM))
        words[wi] = tail;  // the chunk's last word, zero padded
    } else if (nacc > 0 && RB_CHECK(s, wi < pl.n_words, ROIBIN_CHECK_BITSTREAM)) {
      atomicOr(words + wi, (uint32_t)(accb >> 32));  // shared with the next lane
    }
    __syncwarp();
    if (any_pq)
      for (uint32_t i = s0; i < s1; ++i)
        if (pq_bit_of(p, s, sh, g, i) && RB_CHECK(s, pq_pos < pl.n_pq, ROIBIN_CHECK_OUTLIERS))
          pq_out[pq_pos++] = make_uint2(i, __ldcg(pq_bits + i));
  }
  __syncthreads();
  const uint64_t t_roi = acct ? global_ns() : 0;
  if (acct) atomicAdd(acct + 10, (unsigned long long)(t_roi - t_loop));
  // a3: ROI windows of peaks k = grp, grp + groups, ... (one warp per peak)
  float* roi = reinterpret_cast<float*>(out + pl.off_roi);
  const uint32_t win = (uint32_t)(p.roi_h * p.roi_w), plane = p.H * p.W;
  const float* frame = a.frames + (size_t)g * p.frame_px;
  const uint32_t* keys = a.peaks_key_out + (size_t)g * p.max_peaks;
  const uint32_t n_in_place = p.roi_coder ? 0u : pl.n_peaks;  // else the ROI coder writes them
  for (uint32_t k = grp + sh.groups * warp; k < n_in_place; k += sh.groups * kPW) {
    const uint32_t px = __ldcg(keys + k);
    const uint32_t pn = px / plane, rem = px - pn * plane;
    const int r = (int)(rem / p.W), c = (int)(rem % p.W);
    if (RB_CHECK(s, pl.off_roi + (uint64_t)(k + 1) * win * 4 <= a.out_stride, ROIBIN_CHECK_ROI))
      warp_copy_roi(frame + (size_t)pn * plane, p.H, p.W, r, c, p.roi_h, p.roi_w, roi + (size_t)k * win);
  }
  // this group's code bytes are dead: drop them from L2 without a write-back
  __syncthreads();
  if (acct) atomicAdd(acct + 11, (unsigned long long)(global_ns() - t_roi));
  const uint32_t b0 = k_begin * kChunk, b1 = min(p.M, k_end * kChunk);
  for (uint32_t l = b0 / 128 + tid; l < ceil_div(b1, 128); l += kPT) discard_line(codes + (size_t)l * 128);
  if (acct) atomicAdd(acct + 6, (unsigned long long)(global_ns() - t_in));
}

// ---------------------------------------------------------------------------
// One ticket t of a launch over the n frames of one geometry (the order is
// above: round r = t / (U + 2 groups) holds the panels of frame r, the size
// items of frame r - lag1 and the write items of frame r - lag1 - lag2).
// Every thread of the CTA calls it; tickets past the work do nothing and
// return false.  k_fused keeps this body inline in its own loop (the same
// code, which compiled with fewer register spills there).
template <bool kDense, int kG, bool kRt = false>
__device__ __forceinline__ bool fused_ticket(const DevParams& p, const Scratch& s, const PlainArgs& a,
                                             const FusedShape& sh, const SyncWords& sw, unsigned char* sm,
                                             uint32_t t, uint32_t& ring_iter) {
  uint32_t* ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  const uint32_t n = a.n_frames, lag1 = sh.lag1, lag2 = lag1 + sh.lag2, round = sh.U + 2 * sh.groups;
  const uint32_t r = t / round, j = t - r * round;
  if (j < sh.U) {
    if (r >= n) return false;
    if constexpr (kRt || kG > 1) {  // RB = 2 only (the multi-job plan keeps to it)
      process_item<2, kDense, kG, kRt>(p, s, a, sh, sm, r, j, ring_iter);
    } else {
      if (sh.RB == 2) process_item<2, kDense, kG>(p, s, a, sh, sm, r, j, ring_iter);
      else process_item<3, kDense, 1>(p, s, a, sh, sm, r, j, ring_iter);
    }
    // publish the item; the CTA that completes the frame builds its codebook
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ctl[CTL_LAST] = atomicAdd(sw.panel_done + r, 1u) == sh.U - 1 ? 1u : 0u;
    __syncthreads();
    if (ctl[CTL_LAST]) {
      __threadfence();
      frame_codebook(p, s, a, sh, sm, r, sw);
    }
  } else if (j < sh.U + sh.groups) {
    if (r < lag1 || r - lag1 >= n) return false;
    size_item(p, s, a, sh, sm, r - lag1, j - sh.U, sw);
  } else {
    if (r < lag2 || r - lag2 >= n) return false;
    write_item(p, s, a, sh, sm, r - lag2, j - sh.U - sh.groups, sw);
  }
  return true;
}

// Tickets of one launch over n frames of this shape.
__host__ __device__ inline uint64_t fused_tickets(const FusedShape& sh, uint32_t n) {
  return (uint64_t)(n + sh.lag1 + sh.lag2) * (sh.U + 2 * sh.groups);
}

// The CTA's ring barriers (full: the producer's expect_tx; empty: one arrival
// per consumer warp) and its give-up flag, before its first item.
__device__ __forceinline__ void fused_cta_init(unsigned char* sm, const FusedShape& sh) {
  if (threadIdx.x == 0) {
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + sh.off_bar);
    for (uint32_t b = 0; b < sh.stages; ++b) {
      mbar_init(bars + b, 1);
      mbar_init(bars + sh.stages + b, kConsumerWarps);
    }
    mbar_init(bars + 2 * sh.stages, 1);  // the dense-peaks band copies
    fence_mbar_init();
    reinterpret_cast<uint32_t*>(sm + sh.off_ctl)[CTL_TIMEOUT] = 0;
    reinterpret_cast<uint32_t*>(sm + sh.off_ctl)[CTL_BAND] = 0;
  }
  __syncthreads();
}

// The next ticket of the launch's counter, the same in every thread of the CTA.
__device__ __forceinline__ uint32_t fused_next_ticket(unsigned char* sm, const FusedShape& sh, uint32_t* counter) {
  uint32_t* ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  if (threadIdx.x == 0) ctl[CTL_ITEM] = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t t = ctl[CTL_ITEM];
  __syncthreads();
  return t;
}

}  // namespace
}  // namespace roibin
