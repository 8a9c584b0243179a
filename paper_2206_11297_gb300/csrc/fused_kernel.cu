// fused_kernel.cu - the persistent batched kernel: the whole method for a
// batch of frames in one launch.
//
// Work items are handed out in order by an atomic ticket counter to a grid of
// resident CTAs (several per SM).  A streaming item is a group of k panels of
// one frame side by side (k NP <= 217 kG float4 columns, NP = cols / 4, kG
// column groups of 217: 1, or 2 for panels wider than 868 columns).  For it
// a CTA:
//   - streams the raw rows through a ring of 1-D TMA bulk copies (L2
//     evict-first) while the previous rows are coded;
//   - walks down the rows with one thread per float4 column (two bins per
//     binned row): bins, prequantises, predicts with the 2-D Lorenzo rule from
//     registers (row above) and shuffles (bin to the left) and writes one byte
//     per bin (byte = residual + 128 for residuals in [-127, 126], 0 = Lorenzo
//     outlier, 255 = escape whose code sits in a side array);
//   - keeps the item's histogram, prequantisation-outlier bits and the 2x4
//     blocks holding a pixel >= amax_thr in shared memory and flushes them to
//     per-item and per-panel slots with plain stores;
//   - screens the listed blocks, tests and evaluates the surviving candidates
//     and stores its sorted peak list.
// The rest of a frame's work (codebook, chunk sizes, layout, bit-packing)
// runs as later work items of the same kernel (see the stages below), so the
// latency-bound coding of earlier frames overlaps the HBM-bound streaming of
// later ones.  After use, a frame's code bytes are dropped from L2 without a
// write-back.
#include "fused_device.cuh"

namespace roibin {

// ---------------------------------------------------------------------------
// kDense: the variant for frames with many peak candidates (hot pixels).  Its
// warp tests of listed candidates first try the exact rejection screen
// (screen_rejects), and an item whose candidates overflow the list evaluates
// them one per lane.  Both variants write the same bytes.
// kG: column groups per consumer lane (FusedShape::kG; 2 only with RB = 2).
template <bool kDense, int kG>
__global__ void __launch_bounds__(kPT, 4) k_fused(DevParams p, Scratch s, PlainArgs a, FusedShape sh) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint32_t* ctl = reinterpret_cast<uint32_t*>(sm + sh.off_ctl);
  const SyncWords sw = sync_words(s, a.n_frames);
  const uint32_t n = a.n_frames, lag1 = sh.lag1, lag2 = lag1 + sh.lag2, round = sh.U + 2 * sh.groups;
  const uint64_t total = fused_tickets(sh, n);
  fused_cta_init(sm, sh);
  uint32_t ring_iter = 0;  // ring stages consumed so far (the same in every thread)
  for (;;) {
    if (threadIdx.x == 0) ctl[CTL_ITEM] = atomicAdd(sw.ticket, 1u);
    __syncthreads();
    const uint32_t t = ctl[CTL_ITEM];
    __syncthreads();
    if (t >= total) break;
    // the body of fused_ticket
    const uint32_t r = t / round, j = t - r * round;
    if (j < sh.U) {
      if (r >= n) continue;
      if (kG > 1 || sh.RB == 2) process_item<2, kDense, kG>(p, s, a, sh, sm, r, j, ring_iter);
      else process_item<3, kDense, 1>(p, s, a, sh, sm, r, j, ring_iter);
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
      if (r < lag1 || r - lag1 >= n) continue;
      size_item(p, s, a, sh, sm, r - lag1, j - sh.U, sw);
    } else {
      if (r < lag2 || r - lag2 >= n) continue;
      write_item(p, s, a, sh, sm, r - lag2, j - sh.U - sh.groups, sw);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// Shared memory a CTA of this shape needs (0 if the shape is impossible).
static bool make_shape(const DevParams& p, uint32_t ctas_per_sm, uint32_t rb, uint32_t stages, FusedShape* out) {
  FusedShape sh{};
  const uint32_t NP = p.W / 4;
  if (NP < 1 || NP > kMaxG * kGroupCols || rb < 2 || rb > 3) return false;
  sh.kG = ceil_div(NP, kGroupCols);
  if (sh.kG > 1 && rb != 2) return false;  // wide panels: two binned rows per step
  sh.k = min(kMaxK, sh.kG * kGroupCols / NP);
  if ((uint64_t)sh.k * p.H * p.W >= kBlockKey) return false;  // item-local keys stay below the flag
  sh.U = ceil_div(p.P, sh.k);
  sh.RB = rb;
  sh.stages = stages;
  // the streamed rows are read once: first out of L2, so that the code bytes
  // (evict-last) stay there longer (1,000 CSPAD-like frames: +1%)
  sh.input_evict_first = 1;
  sh.wait_limit = kWaitLimit;
  sh.stage_bytes = sh.k * 2 * rb * p.W * 4;
  sh.ctas_per_sm = ctas_per_sm;
  sh.mask_words = ceil_div(p.Hb * p.Wb, 32) + 1;
  sh.side = 2 * (uint32_t)peak_reach(p) + 1;
  uint32_t n2 = 1;
  while (n2 < max(p.max_peaks, 1u)) n2 <<= 1;
  sh.sort_n2 = n2;
  sh.peak_cap = max(p.max_peaks, 1u);
  sh.n_chunks = p.n_chunks;
  sh.codes_stride = p.n_chunks * kChunk;
  sh.group_chunks = 2 * kPW;
  sh.groups = ceil_div(p.n_chunks, sh.group_chunks);
  uint64_t off = 0;
  auto take = [&](uint64_t bytes) {
    off = (off + 15) / 16 * 16;
    const uint64_t o = off;
    off += bytes;
    return (uint32_t)o;
  };
  sh.off_ctl = take((uint64_t)CTL_WORDS * 4);  // every role uses the control words
  sh.off_bar = take(16ull * stages + 8);  // ring full / empty barriers, then the band barrier
  const uint64_t base = off;
  // streaming role; the peak tests reuse the ring once the rows are consumed
  sh.off_hist = take(kMaxSymbols * 4);
  sh.off_pql = take(kPqList * 4);
  sh.off_thr = take(kThrLocalCap * 8);  // keys, then values
  off = (off + 127) / 128 * 128;
  sh.off_ring = take((uint64_t)stages * sh.stage_bytes);
  const uint64_t ring_end = off;
  off = sh.off_ring;
  sh.off_nb = take((uint64_t)kPW * sh.side * sh.side * 4);
  sh.off_acc = take((uint64_t)n2 * 4);
  sh.off_cand = take(kThrLocalCap * 4);
  const uint64_t stream_end = off > ring_end ? off : ring_end;
  // codebook role / size, write and plan roles (overlap the streaming role)
  off = base;
  sh.off_huff = take(sizeof(HuffSmem) > 4096 ? sizeof(HuffSmem) : 4096);  // Huffman scratch | byte tables
  const uint64_t after_huff = off;
  off = sh.off_huff + 4096;  // chunk staging of the size and write items (after the byte tables)
  sh.off_stage = take((uint64_t)kPW * kStageWords * 4);
  const uint64_t stage_end = off;
  off = after_huff;
  sh.off_total = take(kMaxSymbols * 4);
  sh.off_cblen = take(kMaxSymbols);
  sh.off_cbcode = take(kMaxSymbols * 4);
  sh.off_keys = take(16);
  sh.off_cw = take(3ull * p.n_chunks * 4);
  sh.off_offs = take((uint64_t)sh.U * 4);
  const uint64_t fin_end = off > stage_end ? off : stage_end;
  sh.smem = (uint32_t)(stream_end > fin_end ? stream_end : fin_end);
  // The dense-peaks variant takes all the shared memory its CTAs per SM leave
  // it: from the ring on, that memory holds a band of rows of one panel once
  // the item's rows are coded.  A band's candidates are tested in parallel, one
  // per thread, so a taller band keeps more threads busy.
  const uint32_t share = 233472u / ctas_per_sm - 1024u;
  sh.smem_dense = sh.smem > share ? sh.smem : (share < 227u * 1024u ? share : 227u * 1024u);
  sh.band_rows = (sh.smem_dense - sh.off_ring) / (p.W * 4);
  *out = sh;
  return sh.smem <= 227 * 1024;
}

// The kernel instantiation for a shape: dense-peaks variant or not, column groups.
static const void* fused_kernel(bool dense, uint32_t kG) {
  if (kG > 1) return dense ? (const void*)k_fused<true, kMaxG> : (const void*)k_fused<false, kMaxG>;
  return dense ? (const void*)k_fused<true, 1> : (const void*)k_fused<false, 1>;
}

bool fused_shape_for(const DevParams& p, uint32_t ctas_per_sm, uint32_t rows_per_step, uint32_t stages,
                     FusedShape* out) {
  // the 2-D predictor, or the 3-D one (the 2-D residuals stacked by the codebook stage)
  if (p.dims < 2 || p.bh != 2 || p.bw != 2 || (p.W % 4) != 0 || p.W / 4 > kMaxG * kGroupCols) return false;
  if (ctas_per_sm < 1 || ctas_per_sm > 8 || stages < 1 || stages > 8) return false;
  if (rows_per_step != 0 && (rows_per_step < 2 || rows_per_step > 3)) return false;
  FusedShape sh;
  bool ok = false;
  if (rows_per_step) {
    ok = make_shape(p, ctas_per_sm, rows_per_step, stages, &sh);
  } else {
    // the most rows per step whose shared memory lets ctas_per_sm CTAs share an SM
    const uint32_t budget = 233472u / ctas_per_sm - 1024u;
    for (uint32_t rb = 3; rb >= 2 && !ok; --rb) ok = make_shape(p, ctas_per_sm, rb, stages, &sh) && sh.smem <= budget;
  }
  if (!ok) return false;
  const void* kern = fused_kernel(false, sh.kG);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPT, sh.smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return false;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sh.ctas_per_sm = min((uint32_t)per_sm, ctas_per_sm);
  sh.n_ctas = sh.ctas_per_sm * (uint32_t)sms;
  *out = sh;
  return true;
}

bool fused_plan(const DevParams& p, int device, int num_sms, FusedShape* out) {
  (void)device;
  (void)num_sms;
  // measured on CSPAD-like frames: 2 binned rows per step through a 3-slot
  // ring, 4 CTAs per SM, is the fastest shape that fits
  return fused_shape_for(p, 4, 2, 3, out) || fused_shape_for(p, 4, 2, 2, out) || fused_shape_for(p, 3, 2, 3, out) ||
         fused_shape_for(p, 2, 2, 2, out) || fused_shape_for(p, 1, 2, 1, out);
}

cudaError_t launch_fused(const DevParams& p, const Scratch& s, const PlainArgs& a, const FusedShape& sh,
                         bool screen, cudaStream_t st) {
  // stage counters, ready flags and the ticket counter start at zero
  cudaError_t e = cudaMemsetAsync(s.frame_done, 0, sizeof(uint32_t) * (kSyncWordsPerFrame * (uint64_t)a.n_frames + 1), st);
  if (e != cudaSuccess) return e;
  const uint32_t smem = screen ? sh.smem_dense : sh.smem;
  e = cudaFuncSetAttribute(fused_kernel(screen, sh.kG), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  FusedShape s2 = sh;
  // frames between the stages in the ticket order.  Streaming -> chunk sizes:
  // the whole batch, so every frame streams before any is sized.  Streaming
  // is bound by the bytes each CTA keeps in flight, and a CTA on a coding
  // item has none; interleaving the stages (a lag of 256 frames) ran 6% slower
  // at 1,000 frames.  Chunk sizes -> writing: 64 frames, so that a frame's
  // plan is ready when its write items come up.
  s2.lag1 = a.n_frames < kLagSize ? a.n_frames : kLagSize;
  s2.lag2 = a.n_frames < kLagWrite ? a.n_frames : kLagWrite;
  const uint64_t tickets = fused_tickets(s2, a.n_frames);
  const uint32_t grid = (uint32_t)(tickets < sh.n_ctas ? tickets : sh.n_ctas);
  if (sh.kG > 1) {
    if (screen) k_fused<true, kMaxG><<<grid, kPT, smem, st>>>(p, s, a, s2);
    else k_fused<false, kMaxG><<<grid, kPT, smem, st>>>(p, s, a, s2);
  } else {
    if (screen) k_fused<true, 1><<<grid, kPT, smem, st>>>(p, s, a, s2);
    else k_fused<false, 1><<<grid, kPT, smem, st>>>(p, s, a, s2);
  }
  return cudaGetLastError();
}

}  // namespace roibin
