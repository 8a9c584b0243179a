// decompress_kernels.cu - the round trip (§4.1: ROIs restored exactly over the
// up-sampled background) and the ROI mask.
//
//   parse (header, layout, decoding tables) -> decode (chunk-parallel
//   canonical Huffman) -> lorenzo outliers -> row prefix sums -> column prefix
//   sums + dequantisation -> prequantisation outliers -> up-sampling -> ROI
//   restoration -> status
//
// Every index taken from the stream is bounds-checked; a failed check marks
// the frame ROIBIN_ERR_CORRUPT_STREAM and skips the access.
#include <cuda_runtime.h>

#include "roibin_internal.cuh"

namespace roibin {

constexpr int32_t kSentinel = INT32_MIN;  // delta of a code-0 bin until its outlier arrives

__device__ __forceinline__ void mark_corrupt(Scratch& s, uint32_t f) {
  s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
}

// parse: one block per frame.
__global__ void __launch_bounds__(256) k_dec_parse(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t hdr[24];
  __shared__ int ok;
  __shared__ uint32_t cnt[34];
  __shared__ uint32_t nsym_s;
  const uint32_t f = blockIdx.x;
  if (threadIdx.x == 0) {
    s.dec_zero[f] = 0;
    ok = 1;
    const uint64_t base = a.offsets[f];
    if ((base & 15u) != 0 || base + kHeaderBytes > a.in_bytes) ok = 0;
    if (ok) {
      const uint32_t* h = reinterpret_cast<const uint32_t*>(a.in + base);
      for (int i = 0; i < 24; ++i) hdr[i] = h[i];
    }
  }
  __syncthreads();
  DecInfo di = {};
  if (ok) {
    di.base = a.offsets[f];
    const uint32_t roi_h = hdr[5] & 0xFFFFu, roi_w = hdr[5] >> 16;
    const uint32_t bh = hdr[6] & 0xFFFFu, bw = hdr[6] >> 16;
    di.eb = __uint_as_float(hdr[7]);
    di.two_eb = __fmul_rn(2.0f, di.eb);
    di.R = (int32_t)hdr[8];
    di.roi_h = (int32_t)roi_h;
    di.roi_w = (int32_t)roi_w;
    di.nsym = 2u * hdr[8];
    FramePlan& pl = di.pl;
    pl.n_peaks = hdr[9];
    pl.n_lo = hdr[10];
    pl.n_pq = hdr[11];
    pl.n_words = hdr[15];
    const uint64_t total = (uint64_t)hdr[16] | ((uint64_t)hdr[17] << 32);
    if (hdr[0] != kMagic || hdr[1] != kVersion || hdr[2] != p.P || hdr[3] != p.H || hdr[4] != p.W ||
        bh != (uint32_t)p.bh || bw != (uint32_t)p.bw || roi_h < 1 || roi_h > 63 || roi_w < 1 ||
        roi_w > 63 || hdr[8] < 2 || hdr[8] > 512 || hdr[12] != p.M || hdr[13] != kChunk ||
        hdr[14] != p.n_chunks || pl.n_lo > p.M || pl.n_pq > p.M || pl.n_words > p.M ||
        pl.n_peaks > 65535u || !(di.eb > 0.0f) || !isfinite(di.two_eb))
      ok = 0;
    pl.off_peaks = kHeaderBytes;
    pl.off_roi = pl.off_peaks + align16((uint64_t)pl.n_peaks * 6);
    pl.off_len = pl.off_roi + align16((uint64_t)pl.n_peaks * roi_h * roi_w * 4);
    pl.off_cidx = pl.off_len + align16(di.nsym);
    pl.off_lo = pl.off_cidx + align16((uint64_t)p.n_chunks * 4);
    pl.off_pq = pl.off_lo + align16((uint64_t)pl.n_lo * 8);
    pl.off_bits = pl.off_pq + align16((uint64_t)pl.n_pq * 8);
    pl.total = pl.off_bits + align16((uint64_t)pl.n_words * 4);
    if (pl.total != total || di.base + pl.total > a.in_bytes) ok = 0;
  }
  __syncthreads();
  if (!ok) {
    if (threadIdx.x == 0) {
      s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
      s.dec_info[f] = di;
    }
    return;
  }
  // canonical decoding tables: count per length, first code per length, index
  // of the first symbol of each length in the (length, symbol) order.
  const uint8_t* len = a.in + di.base + di.pl.off_len;
  uint32_t* tab = s.dec_table + (size_t)f * kDecTableWords;
  if (threadIdx.x < 34) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) nsym_s = di.nsym;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < di.nsym; k += blockDim.x) {
    const uint32_t L = len[k];
    if (L > 32) ok = 0;
    else if (L > 0) atomicAdd(&cnt[L], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t c = 0;
    uint32_t prev = 0, idx = 0;
    uint64_t kraft = 0;  // sum of 2^(32 - L): a complete code sums to 2^32
    for (uint32_t L = 1; L <= 32; ++L) {
      tab[L] = cnt[L];
      tab[34 + L] = 0;
      tab[68 + L] = idx;
      if (cnt[L]) {
        c = prev == 0 ? 0 : (c + cnt[prev]) << (L - prev);
        tab[34 + L] = (uint32_t)c;
        prev = L;
        kraft += (uint64_t)cnt[L] << (32 - L);
      }
      idx += cnt[L];
    }
    tab[0] = 0;
    // a code with one symbol of length 1 is allowed (kraft = 2^31)
    const bool single = idx == 1 && cnt[1] == 1;
    if (idx == 0 || (kraft != (1ull << 32) && !single)) ok = 0;
  }
  __syncthreads();
  // symbols in (length, symbol) order: rank among same-length smaller symbols
  for (uint32_t k = threadIdx.x; k < nsym_s; k += blockDim.x) {
    const uint32_t L = len[k];
    if (L == 0 || L > 32) continue;
    uint32_t rank = 0;
    for (uint32_t j = 0; j < k; ++j) rank += len[j] == L;
    tab[102 + tab[68 + L] + rank] = k;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
    else s.status[f] = ROIBIN_OK;
    s.dec_info[f] = di;
  }
}

// decode: one thread per chunk (block = 64 chunks of one frame).
constexpr int kDecThreads = 64;
__global__ void __launch_bounds__(kDecThreads) k_dec_decode(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t tab[kDecTableWords];
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  for (uint32_t i = threadIdx.x; i < kDecTableWords; i += kDecThreads)
    tab[i] = s.dec_table[(size_t)f * kDecTableWords + i];
  __syncthreads();
  const uint32_t k = blockIdx.x * kDecThreads + threadIdx.x;
  if (k >= p.n_chunks) return;
  const DecInfo di = s.dec_info[f];
  const uint8_t* base = a.in + di.base;
  const uint32_t* cidx = reinterpret_cast<const uint32_t*>(base + di.pl.off_cidx);
  const uint32_t* words = reinterpret_cast<const uint32_t*>(base + di.pl.off_bits);
  const uint32_t w0 = cidx[k];
  const uint32_t w1 = k + 1 < p.n_chunks ? cidx[k + 1] : di.pl.n_words;
  if (w0 > w1 || w1 > di.pl.n_words) {
    mark_corrupt(s, f);
    return;
  }
  const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
  uint64_t bit = 0;
  const uint32_t s0 = k * kChunk, s1 = min(p.M, s0 + kChunk);
  int32_t* dq = s.dq + (size_t)f * p.M;
  uint32_t zeros = 0;
  // bit reader: `cur` holds the next up-to-32 bits, MSB first
  uint32_t wi = w0;
  uint64_t buf = 0;
  int nbuf = 0;
  for (uint32_t i = s0; i < s1; ++i) {
    if (nbuf < 32) {
      const uint32_t w = wi < w1 ? words[wi] : 0u;
      ++wi;
      buf |= (uint64_t)w << (32 - nbuf);
      nbuf += 32;
    }
    // canonical decode: extend the code one bit at a time
    uint32_t code = 0;
    int sym = -1;
    for (uint32_t L = 1; L <= 32; ++L) {
      code = (code << 1) | (uint32_t)(buf >> (63 - (L - 1)) & 1u);
      const uint32_t n = tab[L];
      if (n && code - tab[34 + L] < n && code >= tab[34 + L]) {
        sym = (int)tab[102 + tab[68 + L] + (code - tab[34 + L])];
        buf <<= L;
        nbuf -= (int)L;
        bit += L;
        break;
      }
    }
    if (sym < 0 || bit > bit_end) {
      mark_corrupt(s, f);
      return;
    }
    if (sym == 0) {
      dq[i] = kSentinel;
      ++zeros;
    } else {
      dq[i] = sym - di.R;
    }
  }
  if ((bit + 31) / 32 != (uint64_t)(w1 - w0)) mark_corrupt(s, f);
  if (zeros) atomicAdd(s.dec_zero + f, zeros);
}

// lorenzo: scatter the Lorenzo-outlier deltas (must land on code-0 bins, in
// strictly ascending order).
__global__ void k_dec_lorenzo(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const DecInfo& di = s.dec_info[f];
  if (blockIdx.x == 0 && threadIdx.x == 0 && s.dec_zero[f] != di.pl.n_lo) mark_corrupt(s, f);
  const uint2* lo = reinterpret_cast<const uint2*>(a.in + di.base + di.pl.off_lo);
  int32_t* dq = s.dq + (size_t)f * p.M;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < di.pl.n_lo; e += gridDim.x * blockDim.x) {
    const uint2 v = lo[e];
    const bool ordered = e == 0 || lo[e - 1].x < v.x;
    if (v.x >= p.M || !ordered || dq[v.x] != kSentinel) {
      mark_corrupt(s, f);
      continue;
    }
    dq[v.x] = (int32_t)v.y;
  }
}

// rows: inclusive prefix sum along each binned row (one warp per row).
__global__ void k_dec_rows(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const uint32_t row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= p.P * p.Hb) return;
  uint32_t* r = reinterpret_cast<uint32_t*>(s.dq + (size_t)f * p.M + (size_t)row * p.Wb);
  uint32_t carry = 0;  // unsigned: wraps instead of overflowing on corrupt input
  for (uint32_t j0 = 0; j0 < p.Wb; j0 += 32) {
    const uint32_t j = j0 + lane_id();
    const uint32_t v = j < p.Wb ? r[j] : 0u;
    const uint32_t inc = warp_incl_scan(v) + carry;
    if (j < p.Wb) r[j] = inc;
    carry = __shfl_sync(0xffffffffu, inc, 31);
  }
}

// cols: prefix sum down each column of a binned panel, then b^ = fl(q * 2eb).
__global__ void k_dec_cols(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.P * p.Wb) return;
  const uint32_t pn = t / p.Wb, j = t - pn * p.Wb;
  const float two_eb = s.dec_info[f].two_eb;
  const uint32_t* dq = reinterpret_cast<const uint32_t*>(s.dq + (size_t)f * p.M + (size_t)pn * p.Hb * p.Wb);
  float* bh = s.bhat + (size_t)f * p.M + (size_t)pn * p.Hb * p.Wb;
  uint32_t q = 0;
  for (uint32_t i = 0; i < p.Hb; ++i) {
    q += dq[(size_t)i * p.Wb + j];
    bh[(size_t)i * p.Wb + j] = __fmul_rn((float)(int32_t)q, two_eb);
  }
}

// pq: prequantisation outliers overwrite b^ with their stored bits.
__global__ void k_dec_pq(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const DecInfo& di = s.dec_info[f];
  const uint2* pq = reinterpret_cast<const uint2*>(a.in + di.base + di.pl.off_pq);
  float* bh = s.bhat + (size_t)f * p.M;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < di.pl.n_pq; e += gridDim.x * blockDim.x) {
    const uint2 v = pq[e];
    const bool ordered = e == 0 || pq[e - 1].x < v.x;
    if (v.x >= p.M || !ordered) {
      mark_corrupt(s, f);
      continue;
    }
    bh[v.x] = __uint_as_float(v.y);
  }
}

// upsample: every pixel takes its bin's value.
__global__ void k_dec_upsample(DevParams p, Scratch s, DecArgs a, int vec4) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const float* bh = s.bhat + (size_t)f * p.M;
  float* out = a.out + (size_t)f * p.frame_px;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  if (vec4) {  // bin 2 x 2, W % 4 == 0: 4 pixels = 2 bins
    const uint64_t n4 = p.frame_px / 4;
    const uint32_t W4 = p.W / 4;
    for (uint64_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += stride) {
      const uint32_t rowg = (uint32_t)(e / W4), c4 = (uint32_t)(e - (uint64_t)rowg * W4);
      const uint32_t pn = rowg / p.H, r = rowg - pn * p.H;
      const float2 v = *reinterpret_cast<const float2*>(bh + ((size_t)pn * p.Hb + r / 2) * p.Wb + 2 * c4);
      reinterpret_cast<float4*>(out)[e] = make_float4(v.x, v.x, v.y, v.y);
    }
    return;
  }
  for (uint64_t e = blockIdx.x * blockDim.x + threadIdx.x; e < p.frame_px; e += stride) {
    const uint32_t rowg = (uint32_t)(e / p.W), c = (uint32_t)(e - (uint64_t)rowg * p.W);
    const uint32_t pn = rowg / p.H, r = rowg - pn * p.H;
    out[e] = bh[((size_t)pn * p.Hb + r / p.bh) * p.Wb + c / p.bw];
  }
}

// roi: restore every in-panel ROI pixel from the stream (one warp per peak).
__global__ void k_dec_roi(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const DecInfo& di = s.dec_info[f];
  const uint8_t* base = a.in + di.base;
  const uint16_t* pk = reinterpret_cast<const uint16_t*>(base + di.pl.off_peaks);
  const float* roi = reinterpret_cast<const float*>(base + di.pl.off_roi);
  const uint32_t win = (uint32_t)(di.roi_h * di.roi_w);
  const uint32_t wpb = blockDim.x >> 5;
  for (uint32_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < di.pl.n_peaks; k += gridDim.x * wpb) {
    const uint32_t pn = pk[3 * k], r = pk[3 * k + 1], c = pk[3 * k + 2];
    if (pn >= p.P || r >= p.H || c >= p.W) {
      if (lane_id() == 0) mark_corrupt(s, f);
      continue;
    }
    float* panel = a.out + (size_t)f * p.frame_px + (size_t)pn * p.H * p.W;
    const int r0 = (int)r - di.roi_h / 2, c0 = (int)c - di.roi_w / 2;
    for (uint32_t e = lane_id(); e < win; e += 32) {
      const int rr = r0 + (int)(e / di.roi_w), cc = c0 + (int)(e % di.roi_w);
      if (rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W)
        panel[(size_t)rr * p.W + cc] = roi[(size_t)k * win + e];
    }
  }
}

__global__ void k_dec_finish(Scratch s, int32_t* status, uint32_t n) {
  const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) status[f] = s.status[f];
}

// ROI mask: u8 per pixel, 1 on every in-panel pixel of some peak's window.
__global__ void k_roi_mask_set(DevParams p, const uint16_t* peaks, const uint32_t* npeaks, uint8_t* mask) {
  const uint32_t f = blockIdx.y;
  const uint32_t n = min(npeaks[f], p.max_peaks);
  const uint32_t k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= n) return;
  const uint16_t* pk = peaks + ((size_t)f * p.max_peaks + k) * 3;
  const uint32_t pn = pk[0], r = pk[1], c = pk[2];
  if (pn >= p.P || r >= p.H || c >= p.W) return;
  uint8_t* m = mask + (size_t)f * p.frame_px + (size_t)pn * p.H * p.W;
  const int r0 = (int)r - p.roi_h / 2, c0 = (int)c - p.roi_w / 2;
  const uint32_t win = (uint32_t)(p.roi_h * p.roi_w);
  for (uint32_t e = lane_id(); e < win; e += 32) {
    const int rr = r0 + (int)(e / p.roi_w), cc = c0 + (int)(e % p.roi_w);
    if (rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W) m[(size_t)rr * p.W + cc] = 1;
  }
}

// pack: copy each frame's stream from its strided slot to its packed offset.
__global__ void k_pack(const uint8_t* src, uint64_t stride, const uint64_t* sizes,
                       const uint64_t* offsets, uint8_t* dst) {
  const uint32_t f = blockIdx.y;
  const uint64_t n16 = sizes[f] / 16;
  const uint4* s4 = reinterpret_cast<const uint4*>(src + (size_t)f * stride);
  uint4* d4 = reinterpret_cast<uint4*>(dst + offsets[f]);
  for (uint64_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n16; e += (uint64_t)gridDim.x * blockDim.x)
    d4[e] = s4[e];
}

// ---------------------------------------------------------------------------
cudaError_t launch_dec_parse(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  k_dec_parse<<<a.n_frames, 256, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_decode(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(ceil_div(p.n_chunks, kDecThreads), a.n_frames);
  k_dec_decode<<<grid, kDecThreads, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_lorenzo(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(64, a.n_frames);
  k_dec_lorenzo<<<grid, 256, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_rows(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(ceil_div(p.P * p.Hb, 8), a.n_frames);
  k_dec_rows<<<grid, 256, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_cols(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(ceil_div(p.P * p.Wb, 128), a.n_frames);
  k_dec_cols<<<grid, 128, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_pq(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(16, a.n_frames);
  k_dec_pq<<<grid, 256, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_upsample(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  const bool vec4 = p.bh == 2 && p.bw == 2 && (p.W % 4) == 0 && (p.Wb % 2) == 0 &&
                    (reinterpret_cast<uintptr_t>(a.out) % 16) == 0;
  dim3 grid(ceil_div((uint32_t)(p.frame_px / 4 / 256), 4) + 1, a.n_frames);
  k_dec_upsample<<<grid, 256, 0, st>>>(p, s, a, vec4 ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_dec_roi(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  dim3 grid(64, a.n_frames);
  k_dec_roi<<<grid, 256, 0, st>>>(p, s, a);
  if (cudaGetLastError() != cudaSuccess) return cudaGetLastError();
  k_dec_finish<<<ceil_div(a.n_frames, 256), 256, 0, st>>>(s, a.frame_status, a.n_frames);
  return cudaGetLastError();
}
cudaError_t launch_roi_mask(const DevParams& p, const uint16_t* peaks, const uint32_t* npeaks, uint32_t n,
                            uint8_t* mask, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(mask, 0, (size_t)n * p.frame_px, st);
  if (e != cudaSuccess || p.max_peaks == 0) return e;
  dim3 grid(ceil_div(p.max_peaks, 8), n);
  k_roi_mask_set<<<grid, 256, 0, st>>>(p, peaks, npeaks, mask);
  return cudaGetLastError();
}
cudaError_t launch_pack(const uint8_t* src, uint64_t stride, const uint64_t* sizes, const uint64_t* offsets,
                        uint32_t n, uint8_t* dst, cudaStream_t st) {
  dim3 grid(64, n);
  k_pack<<<grid, 256, 0, st>>>(src, stride, sizes, offsets, dst);
  return cudaGetLastError();
}

}  // namespace roibin
