// roibin_api.cu - host side of the C ABI declared in include/roibin.h:
// argument validation, the context (preallocated scratch, §4.1's
// zero-allocation principle), launch sequencing and the host-memory path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <memory>
#include <new>
#include <vector>

#include "roibin.h"
#include "roibin_internal.cuh"

using namespace roibin;

struct TimedLaunch {
  int id;
  cudaEvent_t start, stop;
};

struct roibin_graph {
  int device = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t launches = 0;
  uint32_t* sync = nullptr;  // ROIBIN_GRAPH_FUSED: the joint launch's ticket counter and sync words
};

struct roibin_ctx {
  int device = 0;
  int num_sms = 0;
  roibin_geometry g{};
  roibin_params prm{};
  DevParams dp{};
  Scratch s{};
  void* scratch = nullptr;
  uint64_t scratch_bytes = 0;
  std::vector<uint64_t> guards;  // checks build: byte offsets of the scratch guard bands
  uint64_t budget = 0;
  uint32_t max_frames = 0;
  int path_req = ROIBIN_PATH_AUTO;
  int auto_path = 0;  // the path AUTO takes once the autotuner has timed both (0: not yet)
  int dec_path_req = ROIBIN_DEC_AUTO;
  uint32_t plain_rows = 0, plain_bands = 0;  // plain-path shape; 0: chosen per call
  bool fused_ok = false;
  bool fused_dense_peaks = false;  // the fused kernel's variant for many peak candidates
  FusedShape fshape{};
  uint32_t wait_limit = 0;  // 0: the fused kernel's default poll limit; else this many polls
  bool wait_limit_set = false;
  uint64_t* trace = nullptr;
  uint32_t trace_frames = 0;
  uint32_t last_launches = 0;
  // timing
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> free_events;
  // host path
  void* host_stage = nullptr;
  uint64_t host_stage_bytes = 0;
  float* h_frames_dev = nullptr;
  uint8_t* h_out_dev = nullptr;
  uint8_t* h_packed_dev = nullptr;
  uint64_t* h_bytes_dev = nullptr;
  uint64_t* h_offsets_dev = nullptr;
  int32_t* h_status_dev = nullptr;
  uint64_t h_stride = 0;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> slice_events;
};

namespace {

int validate_impl(const roibin_geometry* g, const roibin_params* p) {
  if (!g || !p) return ROIBIN_ERR_INVALID_ARG;
  if (g->n_panels < 1 || g->rows < 1 || g->cols < 1) return ROIBIN_ERR_INVALID_ARG;
  if (g->n_panels > 65535 || g->rows > 65535 || g->cols > 65535) return ROIBIN_ERR_INVALID_ARG;
  if (p->bin_h < 1 || p->bin_w < 1 || p->bin_h > 8 || p->bin_w > 8) return ROIBIN_ERR_INVALID_ARG;
  if (p->roi_h < 1 || p->roi_w < 1 || p->roi_h > 63 || p->roi_w > 63) return ROIBIN_ERR_INVALID_ARG;
  if (p->rank < 1 || p->rank > 7) return ROIBIN_ERR_INVALID_ARG;
  if (p->ring_r0 < 1 || p->ring_dr < 1 || p->ring_r0 + p->ring_dr > 16) return ROIBIN_ERR_INVALID_ARG;
  if (p->npix_min < 0 || p->npix_max < p->npix_min) return ROIBIN_ERR_INVALID_ARG;
  if (p->quant_radius < 2 || p->quant_radius > 512) return ROIBIN_ERR_INVALID_ARG;
  if (p->max_peaks < 0 || p->max_peaks > (int32_t)kMaxPeaksLimit) return ROIBIN_ERR_INVALID_ARG;
  if (p->lorenzo_dims < 1 || p->lorenzo_dims > 3) return ROIBIN_ERR_INVALID_ARG;
  if (p->nhr_min_peaks < 0 || p->nhr_min_peaks > (int32_t)kMaxPeaksLimit) return ROIBIN_ERR_INVALID_ARG;
  if (p->roi_coder < 0 || p->roi_coder > 1) return ROIBIN_ERR_INVALID_ARG;
  if (p->chunk_frames < 1 || p->chunk_frames > 64) return ROIBIN_ERR_INVALID_ARG;
  if (!(p->pix_nsigma >= 0.0f) || std::isnan(p->amax_thr) || std::isnan(p->atot_thr) ||
      std::isnan(p->son_min))
    return ROIBIN_ERR_INVALID_ARG;
  const float two_eb = 2.0f * p->abs_eb;
  if (!(p->abs_eb > 0.0f) || !std::isfinite(two_eb) || !std::isfinite(1.0f / two_eb))
    return ROIBIN_ERR_INVALID_ARG;
  const uint64_t hb = (g->rows + p->bin_h - 1) / p->bin_h, wb = (g->cols + p->bin_w - 1) / p->bin_w;
  if (wb > 8192) return ROIBIN_ERR_INVALID_ARG;
  if ((uint64_t)g->n_panels * hb * wb > kMaxBinsPerFrame) return ROIBIN_ERR_INVALID_ARG;
  return ROIBIN_OK;
}

DevParams make_dev_params(const roibin_geometry& g, const roibin_params& p) {
  DevParams d{};
  d.P = g.n_panels;
  d.H = g.rows;
  d.W = g.cols;
  d.bh = p.bin_h;
  d.bw = p.bin_w;
  d.Hb = (g.rows + p.bin_h - 1) / p.bin_h;
  d.Wb = (g.cols + p.bin_w - 1) / p.bin_w;
  d.M = d.P * d.Hb * d.Wb;
  d.n_chunks = ceil_div(d.M, kChunk);
  d.frame_px = (uint64_t)d.P * d.H * d.W;
  d.amax = p.amax_thr;
  d.atot_thr = p.atot_thr;
  d.son_min = p.son_min;
  d.pix_nsigma = p.pix_nsigma;
  d.rank = p.rank;
  d.ring_r0 = p.ring_r0;
  d.ring_dr = p.ring_dr;
  d.npix_min = p.npix_min;
  d.npix_max = p.npix_max;
  d.roi_h = p.roi_h;
  d.roi_w = p.roi_w;
  d.eb = p.abs_eb;
  // host float arithmetic, one IEEE rounding each
  volatile float two = 2.0f * p.abs_eb;
  d.two_eb = two;
  volatile float rec = 1.0f / d.two_eb;
  d.recip = rec;
  if (p.abs_eb >= 1e-30f) {
    d.eb_lo = (float)((double)p.abs_eb * (1.0 - 1.0 / 1048576.0));
    d.eb_hi = (float)((double)p.abs_eb * (1.0 + 1.0 / 1048576.0));
  } else {  // tiny bounds: always take the exact test
    d.eb_lo = 0.0f;
    d.eb_hi = INFINITY;
  }
  d.R = p.quant_radius;
  d.d_lo = std::max(-127, -(p.quant_radius - 1));
  d.d_span = (uint32_t)(std::min(126, p.quant_radius - 1) - d.d_lo);
  d.nsym = 2u * (uint32_t)p.quant_radius;
  d.max_peaks = (uint32_t)p.max_peaks;
  d.thr_cap = kThrCap;
  d.dims = p.lorenzo_dims;
  d.nhr_min = p.nhr_min_peaks;
  d.roi_coder = p.roi_coder;
  d.chunk = (uint32_t)p.chunk_frames;
  return d;
}

uint64_t bound_impl(const DevParams& d) {
  const uint64_t m = d.M;
  uint64_t o = kHeaderBytes;
  o += align16((uint64_t)d.max_peaks * 6);
  o += align16((uint64_t)d.max_peaks * d.roi_h * d.roi_w * 4);
  o += align16(d.nsym);
  o += align16((uint64_t)d.n_chunks * 4);
  o += align16(m * 8);  // Lorenzo outliers
  o += align16(m * 8);  // prequantisation outliers
  o += align16(m * 4);  // at most 32 bits per symbol
  return o;
}

// Checks build: a guard band of this many bytes (0xA5) before every section.
constexpr uint64_t kGuardBytes = 256;
constexpr uint8_t kGuardByte = 0xA5;

struct Carver {
  uint8_t* base;
  std::vector<uint64_t>* guards = nullptr;  // checks build: where the guard bands go
  uint64_t off = 0;
  template <class T>
  T* take(uint64_t count) {
    off = (off + 255) & ~uint64_t(255);
#ifdef ROIBIN_CHECKS
    if (guards) guards->push_back(off);
    off += kGuardBytes;
#endif
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Bands per panel of the plain path: each band takes at least two binned rows.
uint32_t max_plain_bands(const DevParams& d) { return std::max<uint32_t>(1, ceil_div(d.Hb, 2)); }
// Rows per step of the plain path that fit its shared memory.
bool plain_rows_ok(const DevParams& d, uint32_t rows) {
  const uint64_t q_rows = (uint64_t)(rows + 1) * d.Wb * 4 * (d.dims == 3 ? 2 : 1);  // 3-D: the previous panel too
  return rows >= 1 && rows <= 16 && q_rows + (uint64_t)rows * d.Wb + 16 + 4096 <= 200 * 1024;
}

// Lays out the per-frame scratch for n frames, and candidate spill lists for
// spill_ctas CTAs of the persistent kernel; with base == nullptr only sizes it.
uint64_t carve_scratch(const DevParams& d, uint32_t n, uint8_t* base, Scratch* s, uint32_t spill_ctas,
                       std::vector<uint64_t>* guards = nullptr) {
  Carver c{base, guards};
  Scratch t{};
  t.check = c.take<uint32_t>(2);
  t.thr_count = c.take<uint32_t>(n);
  t.thr_idx = c.take<uint32_t>((uint64_t)n * d.thr_cap);
  t.peak_count = c.take<uint32_t>(n);
  t.peak_key = c.take<uint32_t>((uint64_t)n * std::max<uint32_t>(d.max_peaks, 1));
  t.hist = c.take<uint32_t>((uint64_t)n * kMaxSymbols);
  t.cb_len = c.take<uint8_t>((uint64_t)n * kMaxSymbols);
  t.cb_code = c.take<uint32_t>((uint64_t)n * kMaxSymbols);
  t.codes = c.take<uint16_t>((uint64_t)n * d.n_chunks * kChunk);
  t.lo_delta = c.take<int32_t>((uint64_t)n * d.M);
  t.pq_bits = c.take<uint32_t>((uint64_t)n * d.M);
  t.chunk_words = c.take<uint32_t>((uint64_t)n * d.n_chunks);
  t.chunk_lo = c.take<uint32_t>((uint64_t)n * d.n_chunks);
  t.chunk_pq = c.take<uint32_t>((uint64_t)n * d.n_chunks);
  t.plan = c.take<FramePlan>(n);
  t.status = c.take<int32_t>(n);
  t.dec_table = c.take<uint32_t>((uint64_t)n * kDecTableWords);
  t.dec_zero = c.take<uint32_t>(n);
  t.dec_info = c.take<DecInfo>(n);
  t.dq = t.lo_delta;
  t.bhat = reinterpret_cast<float*>(t.pq_bits);
  const uint64_t mask_words = ceil_div(d.Hb * d.Wb, 32) + 1;
  t.codes8 = c.take<uint8_t>((uint64_t)n * d.n_chunks * kChunk);
  t.pq_mask = c.take<uint32_t>((uint64_t)n * d.P * mask_words);
  t.hist_part = c.take<uint32_t>((uint64_t)n * d.P * kMaxSymbols);
  t.peak_part = c.take<uint32_t>((uint64_t)n * d.P * std::max<uint32_t>(d.max_peaks, 1));
  t.peak_part_count = c.take<uint32_t>((uint64_t)n * d.P);
  t.pq_part_count = c.take<uint32_t>((uint64_t)n * d.P);
  t.lane_bit = c.take<uint32_t>((uint64_t)n * d.n_chunks * 32);
  t.lane_lo = c.take<uint32_t>((uint64_t)n * d.n_chunks * 32);
  t.lane_pq = c.take<uint32_t>((uint64_t)n * d.n_chunks * 32);
  t.frame_done = c.take<uint32_t>(kSyncWordsPerFrame * (uint64_t)n + 1);  // the fused kernel's sync words
  t.chunk_ref = c.take<uint32_t>(n);
  t.thr_spill_ctas = spill_ctas;
  if (spill_ctas) t.thr_spill = c.take<uint32_t>((uint64_t)spill_ctas * kThrSpill);
  if (d.roi_coder) {
    const uint64_t mp = std::max<uint32_t>(d.max_peaks, 1);
    t.roi_hist = c.take<uint32_t>((uint64_t)n * kRoiClasses);
    t.roi_cnt = c.take<uint16_t>((uint64_t)n * mp * kRoiClasses);
    t.roi_off = c.take<uint32_t>((uint64_t)n * mp);
    t.roi_book = c.take<uint32_t>((uint64_t)n * 2 * kRoiClasses);
    t.roi_plan = c.take<uint4>(n);
  }
#ifdef ROIBIN_CHECKS
  if (guards) guards->push_back((c.off + 255) & ~uint64_t(255));  // after the last section
  c.off = ((c.off + 255) & ~uint64_t(255)) + kGuardBytes;
#endif
  if (s) *s = t;
  return c.off + 256;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ROIBIN_OK : ROIBIN_ERR_CUDA; }

cudaEvent_t get_event(roibin_ctx* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs one launcher, bracketed by timing events when enabled.
template <class F>
cudaError_t timed(roibin_ctx* ctx, int id, cudaStream_t st, F&& launch) {
  ctx->last_launches++;
  if (!ctx->timing) return launch();
  TimedLaunch t{id, get_event(ctx), get_event(ctx)};
  cudaEventRecord(t.start, st);
  const cudaError_t e = launch();
  cudaEventRecord(t.stop, st);
  ctx->pending.push_back(t);
  return e;
}

void choose_shape(const roibin_ctx* ctx, uint32_t n_frames, PlainArgs* a) {
  const DevParams& d = ctx->dp;
  a->rows_per_step = std::max<uint32_t>(1, std::min<uint32_t>(16, 2048 / std::max<uint32_t>(d.Wb, 1)));
  const uint32_t target = 4u * (uint32_t)std::max(ctx->num_sms, 1);
  const uint32_t base = d.P * n_frames;
  uint32_t bands = 1;
  if (base < target) bands = ceil_div(target, base);
  bands = std::min<uint32_t>(bands, max_plain_bands(d));
  a->bands_per_panel = bands;
  // a shape set by roibin_ctx_set_plain_shape (or the autotuner) wins
  if (ctx->plain_rows) a->rows_per_step = ctx->plain_rows;
  if (ctx->plain_bands) a->bands_per_panel = ctx->plain_bands;
}

// The ROI coder after either path (three kernels; none without the coder).
int roi_code(roibin_ctx* ctx, const PlainArgs& a, cudaStream_t st) {
  if (!ctx->dp.roi_coder) return ROIBIN_OK;
  const cudaError_t e = timed(ctx, K_ROI_CODE, st, [&] { return launch_roi_code(ctx->dp, ctx->s, a, st); });
  ctx->last_launches += 2;  // the coder is three kernels
  return cuda_status(e);
}

int compress_plain(roibin_ctx* ctx, const PlainArgs& a, cudaStream_t st) {
  const DevParams& p = ctx->dp;
  const Scratch& s = ctx->s;
  cudaError_t e;
  if ((e = timed(ctx, K_RESET, st, [&] { return launch_reset(p, s, a.n_frames, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_STREAM, st, [&] { return launch_stream(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if (!a.user_peaks)
    if ((e = timed(ctx, K_PEAKS, st, [&] { return launch_peaks(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_PEAKS_FINAL, st, [&] { return launch_peaks_final(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_HUFFMAN, st, [&] { return launch_huffman(p, s, a.n_frames, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_CHUNKS, st, [&] { return launch_chunks(p, s, a.n_frames, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_PLAN, st, [&] { return launch_plan(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_ENCODE, st, [&] { return launch_encode(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if (p.max_peaks > 0 && !p.roi_coder)
    if ((e = timed(ctx, K_ROI, st, [&] { return launch_roi(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  return roi_code(ctx, a, st);
}

int resolved_dec_path(const roibin_ctx* ctx) {
  if (ctx->dec_path_req == ROIBIN_DEC_MULTIPASS) return ROIBIN_DEC_MULTIPASS;
  return dec_panel_rows(ctx->dp) && ctx->dp.dims == 2 ? ROIBIN_DEC_PANEL : ROIBIN_DEC_MULTIPASS;
}

int resolved_path(const roibin_ctx* ctx) {
  if (ctx->path_req == ROIBIN_PATH_PLAIN) return ROIBIN_PATH_PLAIN;
  if (ctx->path_req == ROIBIN_PATH_FUSED) return ROIBIN_PATH_FUSED;
  if (!ctx->fused_ok) return ROIBIN_PATH_PLAIN;
  return ctx->auto_path ? ctx->auto_path : ROIBIN_PATH_FUSED;
}

// The checks roibin_compress makes on its arguments.
bool compress_args_ok(const roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, const uint16_t* d_peaks,
                      const uint32_t* d_npeaks, const uint8_t* d_out, uint64_t out_stride,
                      const uint64_t* d_frame_bytes, const int32_t* d_frame_status) {
  if (!ctx || !d_frames || !d_out || !d_frame_bytes || !d_frame_status) return false;
  if (n_frames < 1 || n_frames > ctx->max_frames) return false;
  if ((d_peaks == nullptr) != (d_npeaks == nullptr)) return false;
  if (out_stride < 16 || out_stride % 16 != 0) return false;
  if (reinterpret_cast<uintptr_t>(d_frames) % 16 != 0 || reinterpret_cast<uintptr_t>(d_out) % 16 != 0) return false;
  return true;
}
// The arguments every kernel of a compress call gets.
PlainArgs plain_args(const roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, const uint16_t* d_peaks,
                     const uint32_t* d_npeaks, uint8_t* d_out, uint64_t out_stride, uint64_t* d_frame_bytes,
                     int32_t* d_frame_status) {
  PlainArgs a{};
  a.frames = d_frames;
  a.n_frames = n_frames;
  a.user_peaks = d_peaks;
  a.user_npeaks = d_npeaks;
  a.out = d_out;
  a.out_stride = out_stride;
  a.frame_bytes = d_frame_bytes;
  a.frame_status = d_frame_status;
  choose_shape(ctx, n_frames, &a);
  a.peaks_key_out = ctx->s.peak_key;
  a.peaks_count_out = ctx->s.peak_count;
  a.trace = ctx->trace;
  a.trace_frames = ctx->trace_frames;
  return a;
}

// The call takes the persistent kernel.
bool takes_fused(const roibin_ctx* ctx, uint32_t n_frames) {
  return resolved_path(ctx) == ROIBIN_PATH_FUSED && (uint64_t)n_frames * ctx->dp.P < (1ull << 31);
}

int compress_device(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, const uint16_t* d_peaks,
                    const uint32_t* d_npeaks, uint8_t* d_out, uint64_t out_stride, uint64_t* d_frame_bytes,
                    int32_t* d_frame_status, cudaStream_t st) {
  const PlainArgs a =
      plain_args(ctx, d_frames, n_frames, d_peaks, d_npeaks, d_out, out_stride, d_frame_bytes, d_frame_status);
  if (takes_fused(ctx, n_frames)) {
    FusedShape sh = ctx->fshape;
    if (ctx->wait_limit_set) sh.wait_limit = ctx->wait_limit;
    cudaError_t e = timed(ctx, K_FUSED, st,
                          [&] { return launch_fused(ctx->dp, ctx->s, a, sh, ctx->fused_dense_peaks, st); });
    if (e != cudaSuccess) return cuda_status(e);
    return roi_code(ctx, a, st);
  }
  return compress_plain(ctx, a, st);
}

// The fixed scratch area of roibin_compress_frame_static, one per device (a
// module global exists once in every device context that loads the library).
__device__ __align__(256) unsigned char g_static_scratch[ROIBIN_STATIC_SCRATCH_BYTES];

// The area's address belongs to the CUDA context that loaded the library's
// device code: a reset device (cudaDeviceReset) or a caller's own driver
// context loads it anew, at another address.  So the address is looked up once
// per context, keyed by the context's unique id (cuCtxGetId, which is never
// reused), with that context current.
constexpr int kStaticMaxContexts = 64;
struct StaticEntry {
  unsigned long long ctx_id;
  void* base;
};
std::mutex g_static_mutex;
StaticEntry g_static_cache[kStaticMaxContexts] = {};
int g_static_used = 0;

using CtxGetCurrentFn = int (*)(void**);
using CtxGetIdFn = int (*)(void*, unsigned long long*);

// Unique id of the current context; false when the driver cannot say.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    cudaGetLastError();
    looked = true;
  }
  void* ctx = nullptr;
  return get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

// Address of the area in the current context: looked up (cudaGetSymbolAddress)
// the first time a context calls, then taken from the cache.
cudaError_t static_scratch_base(void** out) {
  std::lock_guard<std::mutex> lock(g_static_mutex);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  if (have_id)
    for (int i = 0; i < g_static_used; ++i)
      if (g_static_cache[i].ctx_id == id) {
        *out = g_static_cache[i].base;
        return cudaSuccess;
      }
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) return e;
  // once the key is known it is cached; otherwise (or with the cache full)
  // the lookup simply runs on every call
  if (have_id && g_static_used < kStaticMaxContexts) g_static_cache[g_static_used++] = {id, ptr};
  *out = ptr;
  return cudaSuccess;
}

// Times `calls` compress calls (after one warm-up) with CUDA events; < 0 on error.
float time_compress(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, uint8_t* d_out, uint64_t out_stride,
                    uint64_t* d_frame_bytes, int32_t* d_frame_status, cudaStream_t st, cudaEvent_t e0,
                    cudaEvent_t e1, int* status) {
  *status = compress_device(ctx, d_frames, n_frames, nullptr, nullptr, d_out, out_stride, d_frame_bytes,
                            d_frame_status, st);  // warm-up
  if (*status != ROIBIN_OK) return -1.0f;
  cudaEventRecord(e0, st);
  for (int rep = 0; rep < 2 && *status == ROIBIN_OK; ++rep)
    *status = compress_device(ctx, d_frames, n_frames, nullptr, nullptr, d_out, out_stride, d_frame_bytes,
                              d_frame_status, st);
  cudaEventRecord(e1, st);
  if (cudaEventSynchronize(e1) != cudaSuccess) *status = ROIBIN_ERR_CUDA;
  float ms = 0.0f;
  if (*status != ROIBIN_OK || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
  return ms;
}

// The plain path's autotuner: rows per step 1..16 (powers of two that fit)
// times bands per panel 1..16 (powers of two up to the panel's limit).
int autotune_plain(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, uint8_t* d_out, uint64_t out_stride,
                   uint64_t* d_frame_bytes, int32_t* d_frame_status, cudaStream_t st, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return ROIBIN_ERR_CUDA;
  }
  const int path_was = ctx->path_req;
  const uint32_t keep_rows = ctx->plain_rows, keep_bands = ctx->plain_bands;
  ctx->path_req = ROIBIN_PATH_PLAIN;
  uint32_t best_rows = keep_rows, best_bands = keep_bands;
  float best_t = -1.0f;
  int status = ROIBIN_OK;
  for (uint32_t rows = 1; rows <= 16 && status == ROIBIN_OK; rows *= 2) {
    if (!plain_rows_ok(ctx->dp, rows) || rows > ctx->dp.Hb) continue;
    for (uint32_t bands = 1; bands <= 16 && bands <= max_plain_bands(ctx->dp) && status == ROIBIN_OK; bands *= 2) {
      ctx->plain_rows = rows;
      ctx->plain_bands = bands;
      const float ms = time_compress(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status,
                                     st, e0, e1, &status);
      if (ms >= 0 && (best_t < 0 || ms < best_t)) {
        best_t = ms;
        best_rows = rows;
        best_bands = bands;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->path_req = path_was;
  const bool ok = status == ROIBIN_OK && best_t >= 0;
  ctx->plain_rows = ok ? best_rows : keep_rows;
  ctx->plain_bands = ok ? best_bands : keep_bands;
  if (best_ms && ok) *best_ms = best_t / 2.0f;
  return status;
}

// The fused path's autotuner: every fused shape that fits (CTAs per SM 2..4,
// rows per step 2..3, ring slots 2..4).
int autotune_fused(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, uint8_t* d_out,
                   uint64_t out_stride, uint64_t* d_frame_bytes, int32_t* d_frame_status, void* stream,
                   float* best_ms) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return ROIBIN_ERR_CUDA;
  }
  const int path_was = ctx->path_req;
  const FusedShape keep = ctx->fshape;
  ctx->path_req = ROIBIN_PATH_FUSED;
  FusedShape best = keep;
  float best_t = -1.0f;
  int status = ROIBIN_OK;
  for (uint32_t cps = 4; cps >= 2 && status == ROIBIN_OK; --cps) {
    for (uint32_t rb = 2; rb <= 3 && status == ROIBIN_OK; ++rb) {
      for (uint32_t stages = 2; stages <= 4 && status == ROIBIN_OK; ++stages) {
        FusedShape sh;
        if (!fused_shape_for(ctx->dp, cps, rb, stages, &sh) || sh.ctas_per_sm != cps) continue;
        ctx->fshape = sh;
        status = compress_device(ctx, d_frames, n_frames, nullptr, nullptr, d_out, out_stride, d_frame_bytes,
                                 d_frame_status, st);  // warm-up
        if (status != ROIBIN_OK) break;
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 2 && status == ROIBIN_OK; ++rep)
          status = compress_device(ctx, d_frames, n_frames, nullptr, nullptr, d_out, out_stride, d_frame_bytes,
                                   d_frame_status, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) status = ROIBIN_ERR_CUDA;
        float ms = 0.0f;
        if (status == ROIBIN_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best_t < 0 || ms < best_t)) {
          best_t = ms;
          best = sh;
        }
      }
    }
  }
  // the dense-peaks variant, on the best shape
  const bool dense_was = ctx->fused_dense_peaks;
  bool best_dense = dense_was;
  if (status == ROIBIN_OK && best_t >= 0) {
    ctx->fshape = best;
    for (int scr = 0; scr < 2 && status == ROIBIN_OK; ++scr) {
      ctx->fused_dense_peaks = scr != 0;
      const float ms = time_compress(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status,
                                     st, e0, e1, &status);
      if (ms >= 0 && (scr == 0 || ms < best_t)) {
        best_t = ms;
        best_dense = scr != 0;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->path_req = path_was;
  ctx->fshape = status == ROIBIN_OK && best_t >= 0 ? best : keep;
  ctx->fused_dense_peaks = status == ROIBIN_OK && best_t >= 0 ? best_dense : dense_was;
  if (best_ms && best_t >= 0) *best_ms = best_t / 2.0f;
  return status;
}


}  // namespace

// ===========================================================================
extern "C" {

int roibin_default_params(roibin_params* p) {
  if (!p) return ROIBIN_ERR_INVALID_ARG;
  p->amax_thr = 300.0f;
  p->atot_thr = 600.0f;
  p->son_min = 10.0f;
  p->pix_nsigma = 3.0f;
  p->rank = 3;
  p->ring_r0 = 5;
  p->ring_dr = 2;
  p->npix_min = 2;
  p->npix_max = 30;
  p->roi_h = 17;
  p->roi_w = 17;
  p->bin_h = 2;
  p->bin_w = 2;
  p->abs_eb = 10.0f;
  p->quant_radius = 512;
  p->max_peaks = 2048;
  p->lorenzo_dims = 2;
  p->nhr_min_peaks = 0;
  p->roi_coder = 0;
  p->chunk_frames = 1;
  return ROIBIN_OK;
}

int roibin_validate(const roibin_geometry* g, const roibin_params* p) { return validate_impl(g, p); }

uint64_t roibin_compress_bound(const roibin_geometry* g, const roibin_params* p) {
  if (validate_impl(g, p) != ROIBIN_OK) return 0;
  return bound_impl(make_dev_params(*g, *p));
}

int roibin_ctx_create(roibin_ctx** out, const roibin_geometry* g, const roibin_params* p,
                      uint32_t max_frames_per_call, uint64_t hbm_budget_bytes, int device) {
  if (!out) return ROIBIN_ERR_INVALID_ARG;
  *out = nullptr;
  int st = validate_impl(g, p);
  if (st != ROIBIN_OK) return st;
  if (max_frames_per_call < 1 || max_frames_per_call > 65535) return ROIBIN_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return ROIBIN_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  roibin_ctx* ctx = new (std::nothrow) roibin_ctx();
  if (!ctx) return ROIBIN_ERR_OUT_OF_BUDGET;
  ctx->device = device;
  ctx->g = *g;
  ctx->prm = *p;
  ctx->dp = make_dev_params(*g, *p);
  ctx->max_frames = max_frames_per_call;
  ctx->budget = hbm_budget_bytes;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  ctx->fused_ok = fused_plan(ctx->dp, device, ctx->num_sms, &ctx->fshape);
  // a spill list for every CTA the persistent kernel may run (at most 8 per SM)
  const uint32_t spill_ctas = ctx->fused_ok ? 8u * (uint32_t)ctx->num_sms : 0u;
  const uint64_t need = carve_scratch(ctx->dp, max_frames_per_call, nullptr, nullptr, spill_ctas);
  if (hbm_budget_bytes && need > hbm_budget_bytes) {
    delete ctx;
    return ROIBIN_ERR_OUT_OF_BUDGET;
  }
  if (cudaMalloc(&ctx->scratch, need) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return ROIBIN_ERR_OUT_OF_BUDGET;
  }
  ctx->scratch_bytes = need;
  carve_scratch(ctx->dp, max_frames_per_call, static_cast<uint8_t*>(ctx->scratch), &ctx->s, spill_ctas,
                &ctx->guards);
  // the check words start at zero; the guard bands (checks build) hold their pattern
  bool set = cudaMemset(ctx->s.check, 0, 8) == cudaSuccess;
  for (uint64_t g : ctx->guards)
    set = set && cudaMemset(static_cast<uint8_t*>(ctx->scratch) + g, kGuardByte, kGuardBytes) == cudaSuccess;
  if (!set || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctx->scratch);
    delete ctx;
    return ROIBIN_ERR_CUDA;
  }
  *out = ctx;
  return ROIBIN_OK;
}

int roibin_ctx_debug_status(roibin_ctx* ctx, uint32_t* checks_build, uint32_t* first_check, uint32_t* failed,
                            uint64_t* bad_guard) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (checks_build) *checks_build = 0;
  if (first_check) *first_check = 0;
  if (failed) *failed = 0;
  if (bad_guard) *bad_guard = UINT64_MAX;
#ifndef ROIBIN_CHECKS
  return ROIBIN_OK;
#else
  if (checks_build) *checks_build = 1;
  if (cudaSetDevice(ctx->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return ROIBIN_ERR_CUDA;
  uint32_t w[2] = {0, 0};
  if (cudaMemcpy(w, ctx->s.check, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return ROIBIN_ERR_CUDA;
  uint64_t bad = UINT64_MAX;
  uint8_t band[kGuardBytes];
  for (uint64_t g : ctx->guards) {
    if (cudaMemcpy(band, static_cast<uint8_t*>(ctx->scratch) + g, kGuardBytes, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return ROIBIN_ERR_CUDA;
    for (uint64_t b = 0; b < kGuardBytes && bad == UINT64_MAX; ++b)
      if (band[b] != kGuardByte) bad = g;
    if (bad != UINT64_MAX) break;
  }
  if (first_check) *first_check = w[0];
  if (failed) *failed = w[1];
  if (bad_guard) *bad_guard = bad;
  return (w[0] || w[1] || bad != UINT64_MAX) ? ROIBIN_ERR_CHECK : ROIBIN_OK;
#endif
}

int roibin_ctx_debug_poke_guard(roibin_ctx* ctx, uint32_t index) {
#ifndef ROIBIN_CHECKS
  (void)ctx;
  (void)index;
  return ROIBIN_ERR_INVALID_ARG;
#else
  if (!ctx || index >= ctx->guards.size()) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  const uint32_t word = 0x12345678u;
  return cuda_status(cudaMemcpy(static_cast<uint8_t*>(ctx->scratch) + ctx->guards[index] + 64, &word, 4,
                                cudaMemcpyHostToDevice));
#endif
}

int roibin_ctx_destroy(roibin_ctx* ctx) {
  if (!ctx) return ROIBIN_OK;
  // checks build: the guard bands and device checks, before the scratch goes
  const int checked = roibin_ctx_debug_status(ctx, nullptr, nullptr, nullptr, nullptr);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  for (auto e : ctx->slice_events) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->host_stage) cudaFree(ctx->host_stage);
  if (ctx->scratch) cudaFree(ctx->scratch);
  delete ctx;
  return checked == ROIBIN_ERR_CHECK ? ROIBIN_ERR_CHECK : ROIBIN_OK;
}

uint64_t roibin_ctx_scratch_bytes(const roibin_ctx* ctx) {
  return ctx ? ctx->scratch_bytes + ctx->host_stage_bytes : 0;
}

int roibin_ctx_set_path(roibin_ctx* ctx, int path) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (path != ROIBIN_PATH_AUTO && path != ROIBIN_PATH_PLAIN && path != ROIBIN_PATH_FUSED)
    return ROIBIN_ERR_INVALID_ARG;
  if (path == ROIBIN_PATH_FUSED && !ctx->fused_ok) return ROIBIN_ERR_INVALID_ARG;
  ctx->path_req = path;
  return ROIBIN_OK;
}

int roibin_ctx_set_fused_shape(roibin_ctx* ctx, uint32_t ctas_per_sm, uint32_t rows_per_step, uint32_t stages) {
  if (!ctx || !ctx->fused_ok) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  FusedShape sh;
  if (!fused_shape_for(ctx->dp, ctas_per_sm, rows_per_step, stages, &sh)) return ROIBIN_ERR_INVALID_ARG;
  ctx->fshape = sh;
  return ROIBIN_OK;
}

int roibin_ctx_fused_shape(const roibin_ctx* ctx, uint32_t* ctas_per_sm, uint32_t* rows_per_step,
                           uint32_t* stages, uint32_t* grid_ctas, uint32_t* smem_bytes) {
  if (!ctx || !ctx->fused_ok) return ROIBIN_ERR_INVALID_ARG;
  if (ctas_per_sm) *ctas_per_sm = ctx->fshape.ctas_per_sm;
  if (rows_per_step) *rows_per_step = ctx->fshape.RB;
  if (stages) *stages = ctx->fshape.stages;
  if (grid_ctas) *grid_ctas = ctx->fshape.n_ctas;
  if (smem_bytes) *smem_bytes = ctx->fshape.smem;
  return ROIBIN_OK;
}

int roibin_ctx_set_fused_dense_peaks(roibin_ctx* ctx, int on) {
  if (!ctx || !ctx->fused_ok) return ROIBIN_ERR_INVALID_ARG;
  ctx->fused_dense_peaks = on != 0;
  return ROIBIN_OK;
}

int roibin_ctx_fused_dense_peaks(const roibin_ctx* ctx) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  return ctx->fused_dense_peaks ? 1 : 0;
}

int roibin_ctx_set_plain_shape(roibin_ctx* ctx, uint32_t rows_per_step, uint32_t bands_per_panel) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (rows_per_step && !plain_rows_ok(ctx->dp, rows_per_step)) return ROIBIN_ERR_INVALID_ARG;
  if (bands_per_panel > max_plain_bands(ctx->dp)) return ROIBIN_ERR_INVALID_ARG;
  ctx->plain_rows = rows_per_step;
  ctx->plain_bands = bands_per_panel;
  return ROIBIN_OK;
}

int roibin_ctx_plain_shape(const roibin_ctx* ctx, uint32_t* rows_per_step, uint32_t* bands_per_panel) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (rows_per_step) *rows_per_step = ctx->plain_rows;
  if (bands_per_panel) *bands_per_panel = ctx->plain_bands;
  return ROIBIN_OK;
}


int roibin_ctx_autotune(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, uint8_t* d_out,
                        uint64_t out_stride, uint64_t* d_frame_bytes, int32_t* d_frame_status, void* stream,
                        float* best_ms) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (!d_frames || !d_out || !d_frame_bytes || !d_frame_status) return ROIBIN_ERR_INVALID_ARG;
  if (n_frames < 1 || n_frames > ctx->max_frames) return ROIBIN_ERR_INVALID_ARG;
  if (out_stride < 16 || out_stride % 16 != 0) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!ctx->fused_ok || ctx->path_req == ROIBIN_PATH_PLAIN)
    return autotune_plain(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status, st, best_ms);
  if (ctx->path_req == ROIBIN_PATH_FUSED)
    return autotune_fused(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status, stream,
                          best_ms);
  // AUTO with both paths: tune each, and let AUTO take the faster one
  float t_fused = -1.0f, t_plain = -1.0f;
  int status = autotune_fused(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status, stream,
                              &t_fused);
  if (status != ROIBIN_OK) return status;
  status = autotune_plain(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status, st, &t_plain);
  if (status != ROIBIN_OK) return status;
  // The fused search ran first, while the clocks may still have been ramping
  // up: time the two tuned paths again in alternation and keep each one's best.
  if (t_plain >= 0.0f && t_fused >= 0.0f) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      return ROIBIN_ERR_CUDA;
    }
    for (int round = 0; round < 3 && status == ROIBIN_OK; ++round) {
      for (int path : {ROIBIN_PATH_FUSED, ROIBIN_PATH_PLAIN}) {
        ctx->path_req = path;
        const float ms = time_compress(ctx, d_frames, n_frames, d_out, out_stride, d_frame_bytes, d_frame_status,
                                       st, e0, e1, &status) / 2.0f;
        float& best = path == ROIBIN_PATH_FUSED ? t_fused : t_plain;
        if (status == ROIBIN_OK && ms < best) best = ms;
        if (status != ROIBIN_OK) break;
      }
    }
    ctx->path_req = ROIBIN_PATH_AUTO;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != ROIBIN_OK) return status;
  }
  ctx->auto_path = (t_plain >= 0.0f && t_fused >= 0.0f && t_plain < t_fused) ? ROIBIN_PATH_PLAIN : ROIBIN_PATH_FUSED;
  if (best_ms) *best_ms = ctx->auto_path == ROIBIN_PATH_PLAIN ? t_plain : t_fused;
  return ROIBIN_OK;
}

int roibin_ctx_set_wait_limit(roibin_ctx* ctx, int64_t polls) {
  if (!ctx || polls > (int64_t)UINT32_MAX) return ROIBIN_ERR_INVALID_ARG;
  ctx->wait_limit_set = polls >= 0;
  ctx->wait_limit = polls >= 0 ? (uint32_t)polls : 0u;
  return ROIBIN_OK;
}

int roibin_ctx_set_trace(roibin_ctx* ctx, uint64_t* d_trace, uint32_t n_frames) {
  if (!ctx || (n_frames > 0 && !d_trace)) return ROIBIN_ERR_INVALID_ARG;
  ctx->trace = n_frames ? d_trace : nullptr;
  ctx->trace_frames = n_frames;
  return ROIBIN_OK;
}

int roibin_ctx_resolved_path(const roibin_ctx* ctx) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  return resolved_path(ctx);
}

int roibin_compress(roibin_ctx* ctx, const float* d_frames, uint32_t n_frames, const uint16_t* d_peaks,
                    const uint32_t* d_npeaks, uint8_t* d_out, uint64_t out_stride, uint64_t* d_frame_bytes,
                    int32_t* d_frame_status, void* stream) {
  if (!compress_args_ok(ctx, d_frames, n_frames, d_peaks, d_npeaks, d_out, out_stride, d_frame_bytes,
                        d_frame_status))
    return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  ctx->last_launches = 0;
  return compress_device(ctx, d_frames, n_frames, d_peaks, d_npeaks, d_out, out_stride, d_frame_bytes,
                         d_frame_status, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
namespace {
// The end of every decompression: the ROI windows of frames whose ROI section
// comes after the bitstream (any stream may carry one), then the statuses.
int dec_finish(roibin_ctx* ctx, const DecArgs& a, cudaStream_t st) {
  cudaError_t e;
  if ((e = timed(ctx, K_DEC_ROI_CODED, st, [&] { return launch_dec_roi_coded(ctx->dp, ctx->s, a, st); })) !=
      cudaSuccess)
    return cuda_status(e);
  ctx->last_launches++;  // the status copy
  return cuda_status(launch_dec_finish(ctx->s, a, st));
}
}  // namespace
extern "C" {

int roibin_decompress(roibin_ctx* ctx, const uint8_t* d_in, uint64_t in_bytes, const uint64_t* d_frame_offsets,
                      uint32_t n_frames, float* d_frames_out, int32_t* d_frame_status, void* stream) {
  if (!ctx || !d_in || !d_frame_offsets || !d_frames_out || !d_frame_status) return ROIBIN_ERR_INVALID_ARG;
  if (n_frames < 1 || n_frames > ctx->max_frames) return ROIBIN_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_in) % 16 != 0) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DecArgs a{d_in, in_bytes, d_frame_offsets, n_frames, d_frames_out, d_frame_status};
  const DevParams& p = ctx->dp;
  const Scratch& s = ctx->s;
  ctx->last_launches = 0;
  cudaError_t e;
  if ((e = timed(ctx, K_DEC_PARSE, st, [&] { return launch_dec_parse(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if (resolved_dec_path(ctx) == ROIBIN_DEC_PANEL) {
    if ((e = timed(ctx, K_DEC_DECODE, st, [&] { return launch_dec_decoders(p, s, a, st); })) != cudaSuccess)
      return cuda_status(e);
    ctx->last_launches++;  // the decode step is two kernels: sparse frames, then dense ones
    if ((e = timed(ctx, K_DEC_PANEL, st, [&] { return launch_dec_panel(p, s, a, st); })) != cudaSuccess)
      return cuda_status(e);
    return dec_finish(ctx, a, st);
  }
  if ((e = timed(ctx, K_DEC_DECODE, st, [&] { return launch_dec_decode(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_DEC_LORENZO, st, [&] { return launch_dec_lorenzo(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_DEC_ROWS, st, [&] { return launch_dec_rows(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  // the inverse predictor after the row sums: down the columns (2-D), then
  // across the panels (3-D); or the carry from row to row (1-D)
  if (p.dims >= 2)
    if ((e = timed(ctx, K_DEC_COLS, st, [&] { return launch_dec_cols(p, s, a, p.dims == 2, st); })) != cudaSuccess)
      return cuda_status(e);
  if (p.dims != 2)
    if ((e = timed(ctx, K_DEC_CARRY, st, [&] { return launch_dec_carry(p, s, a, st); })) != cudaSuccess)
      return cuda_status(e);
  if ((e = timed(ctx, K_DEC_PQ, st, [&] { return launch_dec_pq(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_DEC_UPSAMPLE, st, [&] { return launch_dec_upsample(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  if ((e = timed(ctx, K_DEC_ROI, st, [&] { return launch_dec_roi(p, s, a, st); })) != cudaSuccess) return cuda_status(e);
  return dec_finish(ctx, a, st);
}

int roibin_ctx_set_decompress_path(roibin_ctx* ctx, int path) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (path != ROIBIN_DEC_AUTO && path != ROIBIN_DEC_PANEL && path != ROIBIN_DEC_MULTIPASS)
    return ROIBIN_ERR_INVALID_ARG;
  if (path == ROIBIN_DEC_PANEL && (dec_panel_rows(ctx->dp) == 0 || ctx->dp.dims != 2)) return ROIBIN_ERR_INVALID_ARG;
  ctx->dec_path_req = path;
  return ROIBIN_OK;
}

int roibin_ctx_resolved_decompress_path(const roibin_ctx* ctx) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  return resolved_dec_path(ctx);
}

int roibin_graph_create(roibin_graph** out, const roibin_job* jobs, uint32_t n_jobs, int flags) {
  if (!out) return ROIBIN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!jobs || n_jobs == 0) return ROIBIN_ERR_INVALID_ARG;
  if (flags != ROIBIN_GRAPH_SERIAL && flags != ROIBIN_GRAPH_CONCURRENT && flags != ROIBIN_GRAPH_FUSED)
    return ROIBIN_ERR_INVALID_ARG;
  const bool concurrent = flags == ROIBIN_GRAPH_CONCURRENT, fused = flags == ROIBIN_GRAPH_FUSED;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const roibin_job& b = jobs[j];
    if (!compress_args_ok(b.ctx, b.d_frames, b.n_frames, b.d_peaks, b.d_npeaks, b.d_out, b.out_stride,
                          b.d_frame_bytes, b.d_frame_status))
      return ROIBIN_ERR_INVALID_ARG;
    if (b.ctx->device != jobs[0].ctx->device) return ROIBIN_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < j; ++i)
      if (jobs[i].ctx == b.ctx) return ROIBIN_ERR_INVALID_ARG;
  }
  const int device = jobs[0].ctx->device;
  if (cudaSetDevice(device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  // ROIBIN_GRAPH_FUSED: the jobs that take the persistent kernel share one
  // launch (their sync words and the ticket counter in one buffer the graph
  // owns and zeroes); the others follow it, one after another
  std::vector<uint32_t> joint, alone;
  std::unique_ptr<FusedJobs> fj;
  uint32_t* sync = nullptr;
  uint64_t sync_words = 1;
  uint32_t fj_smem = 0, fj_grid = 0;
  for (uint32_t j = 0; j < n_jobs; ++j)
    ((fused && takes_fused(jobs[j].ctx, jobs[j].n_frames) && joint.size() < kMaxFusedJobs) ? joint : alone)
        .push_back(j);
  if (!joint.empty()) {
    fj.reset(new (std::nothrow) FusedJobs{});
    if (!fj) return ROIBIN_ERR_OUT_OF_BUDGET;
    for (uint32_t j : joint) sync_words += kSyncWordsPerFrame * (uint64_t)jobs[j].n_frames + 1;
    if (cudaMalloc(&sync, sync_words * 4) != cudaSuccess) {
      cudaGetLastError();
      return ROIBIN_ERR_OUT_OF_BUDGET;
    }
    std::vector<FusedShape> tuned(joint.size());
    uint64_t off = 1;  // word 0: the ticket counter
    for (uint32_t i = 0; i < joint.size(); ++i) {
      const roibin_job& b = jobs[joint[i]];
      FusedJob& J = fj->job[i];
      J.p = b.ctx->dp;
      J.s = b.ctx->s;
      J.s.frame_done = sync + off;
      off += kSyncWordsPerFrame * (uint64_t)b.n_frames + 1;
      J.a = plain_args(b.ctx, b.d_frames, b.n_frames, b.d_peaks, b.d_npeaks, b.d_out, b.out_stride,
                       b.d_frame_bytes, b.d_frame_status);
      J.dense = b.ctx->fused_dense_peaks ? 1u : 0u;
      tuned[i] = b.ctx->fshape;
      if (b.ctx->wait_limit_set) tuned[i].wait_limit = b.ctx->wait_limit;
    }
    fj->ticket = sync;
    fj->n_jobs = (uint32_t)joint.size();
    if (!fused_jobs_plan(fj.get(), tuned.data(), jobs[0].ctx->num_sms, &fj_smem, &fj_grid)) {
      cudaFree(sync);
      return ROIBIN_ERR_INVALID_ARG;
    }
  }
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> side(n_jobs, nullptr);
  std::vector<cudaEvent_t> ev(n_jobs + 1, nullptr);
  bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
  for (uint32_t j = 0; ok && j < n_jobs; ++j) ok = cudaStreamCreateWithFlags(&side[j], cudaStreamNonBlocking) == cudaSuccess;
  for (uint32_t j = 0; ok && j <= n_jobs; ++j) ok = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming) == cudaSuccess;
  int status = ok ? ROIBIN_OK : ROIBIN_ERR_CUDA;
  uint32_t launches = 0;
  cudaGraph_t graph = nullptr;
  // relaxed mode: the fused launcher sets a kernel attribute while capturing
  if (status == ROIBIN_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    status = ROIBIN_ERR_CUDA;
  if (status == ROIBIN_OK && fused) {
    if (!joint.empty()) {
      if (cudaMemsetAsync(sync, 0, sync_words * 4, cs) != cudaSuccess ||
          launch_fused_jobs(*fj, fj_smem, fj_grid, cs) != cudaSuccess)
        status = ROIBIN_ERR_CUDA;
      launches += 1;
      for (uint32_t i = 0; status == ROIBIN_OK && i < joint.size(); ++i) {  // the ROI coder after the joint launch
        roibin_ctx* ctx = jobs[joint[i]].ctx;
        const bool timing = ctx->timing;
        ctx->timing = false;
        ctx->last_launches = 0;
        status = roi_code(ctx, fj->job[i].a, cs);
        ctx->timing = timing;
        launches += ctx->last_launches;
      }
    }
    for (uint32_t j : alone) {
      if (status != ROIBIN_OK) break;
      const roibin_job& b = jobs[j];
      const bool timing = b.ctx->timing;
      b.ctx->timing = false;
      b.ctx->last_launches = 0;
      status = compress_device(b.ctx, b.d_frames, b.n_frames, b.d_peaks, b.d_npeaks, b.d_out, b.out_stride,
                               b.d_frame_bytes, b.d_frame_status, cs);
      b.ctx->timing = timing;
      launches += b.ctx->last_launches;
    }
    // capture always ends, so that the stream leaves capture mode
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && status == ROIBIN_OK) status = ROIBIN_ERR_CUDA;
  } else if (status == ROIBIN_OK) {
    if (cudaEventRecord(ev[n_jobs], cs) != cudaSuccess) status = ROIBIN_ERR_CUDA;  // the fork
    for (uint32_t j = 0; status == ROIBIN_OK && j < n_jobs; ++j) {
      const roibin_job& b = jobs[j];
      // concurrent: a branch that forks from the start; serial: the capture stream itself
      cudaStream_t js = concurrent ? side[j] : cs;
      if (concurrent && cudaStreamWaitEvent(js, ev[n_jobs], 0) != cudaSuccess) {
        status = ROIBIN_ERR_CUDA;
        break;
      }
      const bool timing = b.ctx->timing;  // no timing events inside a graph
      b.ctx->timing = false;
      b.ctx->last_launches = 0;
      status = compress_device(b.ctx, b.d_frames, b.n_frames, b.d_peaks, b.d_npeaks, b.d_out, b.out_stride,
                               b.d_frame_bytes, b.d_frame_status, js);
      b.ctx->timing = timing;
      launches += b.ctx->last_launches;
      if (concurrent && status == ROIBIN_OK &&
          (cudaEventRecord(ev[j], js) != cudaSuccess || cudaStreamWaitEvent(cs, ev[j], 0) != cudaSuccess))  // the join
        status = ROIBIN_ERR_CUDA;
    }
    // capture always ends, so that the streams leave capture mode
    if (cudaStreamEndCapture(cs, &graph) != cudaSuccess && status == ROIBIN_OK) status = ROIBIN_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  if (status == ROIBIN_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) status = ROIBIN_ERR_CUDA;
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  for (auto st : side)
    if (st) cudaStreamDestroy(st);
  if (cs) cudaStreamDestroy(cs);
  roibin_graph* g = status == ROIBIN_OK ? new (std::nothrow) roibin_graph : nullptr;
  if (status == ROIBIN_OK && !g) status = ROIBIN_ERR_OUT_OF_BUDGET;
  if (status != ROIBIN_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (sync) cudaFree(sync);
    cudaGetLastError();
    return status;
  }
  g->device = device;
  g->graph = graph;
  g->exec = exec;
  g->launches = launches;
  g->sync = sync;
  *out = g;
  return ROIBIN_OK;
}

int roibin_graph_launch(roibin_graph* g, void* stream) {
  if (!g || !g->exec) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(g->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  return cuda_status(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
}

int roibin_graph_launch_count(const roibin_graph* g) { return g ? (int)g->launches : ROIBIN_ERR_INVALID_ARG; }

int roibin_graph_destroy(roibin_graph* g) {
  if (!g) return ROIBIN_OK;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->sync) cudaFree(g->sync);
  delete g;
  return ROIBIN_OK;
}

int roibin_ctx_reserve_host_path(roibin_ctx* ctx) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  if (ctx->host_stage) return ROIBIN_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  const uint64_t n = ctx->max_frames;
  const uint64_t stride = bound_impl(ctx->dp);
  Carver c{nullptr};
  c.take<float>(n * ctx->dp.frame_px);
  c.take<uint8_t>(n * stride);
  c.take<uint8_t>(n * stride);
  c.take<uint64_t>(n + 1);
  c.take<uint64_t>(n + 1);
  c.take<int32_t>(n);
  const uint64_t need = c.off + 256;
  if (ctx->budget && ctx->scratch_bytes + need > ctx->budget) return ROIBIN_ERR_OUT_OF_BUDGET;
  void* base = nullptr;
  if (cudaMalloc(&base, need) != cudaSuccess) {
    cudaGetLastError();
    return ROIBIN_ERR_OUT_OF_BUDGET;
  }
  Carver d{static_cast<uint8_t*>(base)};
  ctx->h_frames_dev = d.take<float>(n * ctx->dp.frame_px);
  ctx->h_out_dev = d.take<uint8_t>(n * stride);
  ctx->h_packed_dev = d.take<uint8_t>(n * stride);
  ctx->h_bytes_dev = d.take<uint64_t>(n + 1);
  ctx->h_offsets_dev = d.take<uint64_t>(n + 1);
  ctx->h_status_dev = d.take<int32_t>(n);
  ctx->h_stride = stride;
  ctx->host_stage = base;
  ctx->host_stage_bytes = need;
  if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) return ROIBIN_ERR_CUDA;
  return ROIBIN_OK;
}

}  // extern "C"

namespace roibin {
// exclusive scan of frame sizes -> packed offsets; offsets[n] = total
__global__ void k_pack_offsets(const uint64_t* sizes, uint64_t* offsets, uint32_t n) {
  __shared__ uint64_t carry;
  __shared__ uint64_t tmp[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t b = 0; b < n; b += blockDim.x) {
    const uint32_t i = b + threadIdx.x;
    const uint64_t v = i < n ? sizes[i] : 0;
    tmp[threadIdx.x] = v;
    __syncthreads();
    for (uint32_t d = 1; d < blockDim.x; d <<= 1) {
      const uint64_t add = threadIdx.x >= d ? tmp[threadIdx.x - d] : 0;
      __syncthreads();
      tmp[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) offsets[i] = carry + tmp[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += tmp[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n] = carry;
}
}  // namespace roibin

extern "C" {

int roibin_compress_host(roibin_ctx* ctx, const float* h_frames, uint32_t n_frames, uint8_t* h_out,
                         uint64_t h_out_capacity, uint64_t* h_frame_bytes, int32_t* h_frame_status,
                         void* stream) {
  if (!ctx || !h_frames || !h_out || !h_frame_bytes || !h_frame_status) return ROIBIN_ERR_INVALID_ARG;
  if (!ctx->host_stage) return ROIBIN_ERR_INVALID_ARG;
  if (n_frames < 1 || n_frames > ctx->max_frames) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t frame_bytes = ctx->dp.frame_px * 4;
  // slices: copy slice i+1 while slice i compresses
  const uint32_t n_slices = std::min<uint32_t>(8, n_frames);
  const uint32_t per = ceil_div(n_frames, n_slices);
  while (ctx->slice_events.size() < n_slices + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return ROIBIN_ERR_CUDA;
    ctx->slice_events.push_back(e);
  }
  // the copy stream must not overwrite staging still read by a previous call
  cudaEvent_t fence = ctx->slice_events[n_slices];
  cudaEventRecord(fence, st);
  cudaStreamWaitEvent(ctx->copy_stream, fence, 0);
  for (uint32_t k = 0; k < n_slices; ++k) {
    const uint32_t f0 = k * per, f1 = std::min(n_frames, f0 + per);
    if (f0 >= f1) break;
    if (cudaMemcpyAsync(ctx->h_frames_dev + (size_t)f0 * ctx->dp.frame_px, h_frames + (size_t)f0 * ctx->dp.frame_px,
                        (size_t)(f1 - f0) * frame_bytes, cudaMemcpyHostToDevice, ctx->copy_stream) != cudaSuccess)
      return ROIBIN_ERR_CUDA;
    cudaEventRecord(ctx->slice_events[k], ctx->copy_stream);
  }
  ctx->last_launches = 0;
  for (uint32_t k = 0; k < n_slices; ++k) {
    const uint32_t f0 = k * per, f1 = std::min(n_frames, f0 + per);
    if (f0 >= f1) break;
    cudaStreamWaitEvent(st, ctx->slice_events[k], 0);
    const int rc = compress_device(ctx, ctx->h_frames_dev + (size_t)f0 * ctx->dp.frame_px, f1 - f0, nullptr,
                                   nullptr, ctx->h_out_dev + (size_t)f0 * ctx->h_stride, ctx->h_stride,
                                   ctx->h_bytes_dev + f0, ctx->h_status_dev + f0, st);
    if (rc != ROIBIN_OK) return rc;
  }
  k_pack_offsets<<<1, 1024, 0, st>>>(ctx->h_bytes_dev, ctx->h_offsets_dev, n_frames);
  if (cudaGetLastError() != cudaSuccess) return ROIBIN_ERR_CUDA;
  if (launch_pack(ctx->h_out_dev, ctx->h_stride, ctx->h_bytes_dev, ctx->h_offsets_dev, n_frames,
                  ctx->h_packed_dev, st) != cudaSuccess)
    return ROIBIN_ERR_CUDA;
  ctx->last_launches += 2;
  uint64_t total = 0;
  if (cudaMemcpyAsync(&total, ctx->h_offsets_dev + n_frames, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(h_frame_bytes, ctx->h_bytes_dev, (size_t)n_frames * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(h_frame_status, ctx->h_status_dev, (size_t)n_frames * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ROIBIN_ERR_CUDA;
  if (total > h_out_capacity) return ROIBIN_ERR_CAPACITY;
  if (cudaMemcpyAsync(h_out, ctx->h_packed_dev, total, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ROIBIN_ERR_CUDA;
  return ROIBIN_OK;
}

int roibin_roi_mask(roibin_ctx* ctx, const uint16_t* d_peaks, const uint32_t* d_npeaks, uint32_t n_frames,
                    uint8_t* d_mask, void* stream) {
  if (!ctx || !d_peaks || !d_npeaks || !d_mask || n_frames < 1) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  return cuda_status(launch_roi_mask(ctx->dp, d_peaks, d_npeaks, n_frames, d_mask,
                                     static_cast<cudaStream_t>(stream)));
}

int roibin_last_peaks(roibin_ctx* ctx, uint16_t* d_peaks, uint32_t* d_npeaks, uint32_t n_frames, void* stream) {
  if (!ctx || !d_peaks || !d_npeaks || n_frames < 1 || n_frames > ctx->max_frames) return ROIBIN_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  return cuda_status(launch_last_peaks(ctx->dp, ctx->s, d_peaks, d_npeaks, n_frames,
                                       static_cast<cudaStream_t>(stream)));
}

int roibin_ctx_enable_timing(roibin_ctx* ctx, int enable) {
  if (!ctx) return ROIBIN_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return ROIBIN_OK;
}

int roibin_ctx_kernel_times(roibin_ctx* ctx, const char** names, double* total_ms, uint32_t* launches,
                            int max_kernels, int* n_kernels) {
  if (!ctx || !n_kernels) return ROIBIN_ERR_INVALID_ARG;
  double sum[K_COUNT] = {0};
  uint32_t cnt[K_COUNT] = {0};
  int rc = ROIBIN_OK;
  for (auto& t : ctx->pending) {
    if (cudaEventSynchronize(t.stop) != cudaSuccess) rc = ROIBIN_ERR_CUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
      sum[t.id] += ms;
      cnt[t.id]++;
    }
    ctx->free_events.push_back(t.start);
    ctx->free_events.push_back(t.stop);
  }
  ctx->pending.clear();
  int k = 0;
  for (int id = 0; id < K_COUNT; ++id) {
    if (!cnt[id]) continue;
    if (k < max_kernels) {
      if (names) names[k] = kernel_name(id);
      if (total_ms) total_ms[k] = sum[id];
      if (launches) launches[k] = cnt[id];
    }
    ++k;
  }
  *n_kernels = k;
  return rc;
}

uint32_t roibin_ctx_last_launch_count(const roibin_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

int roibin_compress_frame_static(const roibin_geometry* g, const roibin_params* p, const float* d_frame,
                                 const uint16_t* d_peaks, const uint32_t* d_npeaks, uint8_t* d_out,
                                 uint64_t out_capacity, uint64_t* d_frame_bytes, int32_t* d_frame_status,
                                 void* stream) {
  const int v = validate_impl(g, p);
  if (v != ROIBIN_OK) return v;
  if (!d_frame || !d_out || !d_frame_bytes || !d_frame_status) return ROIBIN_ERR_INVALID_ARG;
  if ((d_peaks == nullptr) != (d_npeaks == nullptr)) return ROIBIN_ERR_INVALID_ARG;
  if (out_capacity < 16 || out_capacity % 16 != 0) return ROIBIN_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_frame) % 16 != 0 || reinterpret_cast<uintptr_t>(d_out) % 16 != 0)
    return ROIBIN_ERR_INVALID_ARG;
  const DevParams dp = make_dev_params(*g, *p);
  if (carve_scratch(dp, 1, nullptr, nullptr, 0) > ROIBIN_STATIC_SCRATCH_BYTES) return ROIBIN_ERR_OUT_OF_BUDGET;
  int device = 0, sms = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  void* base = nullptr;
  if (static_scratch_base(&base) != cudaSuccess) return ROIBIN_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return ROIBIN_ERR_CUDA;
  Scratch s{};
  carve_scratch(dp, 1, static_cast<uint8_t*>(base), &s, 0);
  PlainArgs a{};
  a.frames = d_frame;
  a.n_frames = 1;
  a.user_peaks = d_peaks;
  a.user_npeaks = d_npeaks;
  a.out = d_out;
  a.out_stride = out_capacity;
  a.frame_bytes = d_frame_bytes;
  a.frame_status = d_frame_status;
  // one frame: split each panel into bands so that the grid covers the GPU
  a.rows_per_step = std::max<uint32_t>(1, std::min<uint32_t>(16, 2048 / std::max<uint32_t>(dp.Wb, 1)));
  const uint32_t target = 4u * (uint32_t)std::max(sms, 1);
  a.bands_per_panel = std::min<uint32_t>(dp.P < target ? ceil_div(target, dp.P) : 1u,
                                         std::max<uint32_t>(1, ceil_div(dp.Hb, 2)));
  a.peaks_key_out = s.peak_key;
  a.peaks_count_out = s.peak_count;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = launch_reset(dp, s, 1, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_stream(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if (!a.user_peaks && (e = launch_peaks(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_peaks_final(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_huffman(dp, s, 1, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_chunks(dp, s, 1, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_plan(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if ((e = launch_encode(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if (dp.max_peaks > 0 && !dp.roi_coder && (e = launch_roi(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  if (dp.roi_coder && (e = launch_roi_code(dp, s, a, st)) != cudaSuccess) return cuda_status(e);
  return ROIBIN_OK;
}

const char* roibin_status_string(int status) {
  switch (status) {
    case ROIBIN_OK: return "ok";
    case ROIBIN_ERR_INVALID_ARG: return "invalid argument";
    case ROIBIN_ERR_CAPACITY: return "capacity exceeded (peaks or output stride)";
    case ROIBIN_ERR_CORRUPT_STREAM: return "corrupt compressed stream";
    case ROIBIN_ERR_OUT_OF_BUDGET: return "device memory budget exceeded";
    case ROIBIN_ERR_CUDA: return "CUDA runtime error";
    case ROIBIN_ERR_TIMEOUT: return "bounded device wait timed out";
    case ROIBIN_ERR_CODE_LENGTH: return "Huffman code longer than 32 bits";
    case ROIBIN_ERR_CHECK: return "checks build: a device bounds check failed or a guard band was overwritten";
    default: return "unknown status";
  }
}

}  // extern "C"
