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

#include <algorithm>

#include "roibin_internal.cuh"

namespace roibin {

constexpr int32_t kSentinel = INT32_MIN;  // delta of a code-0 bin until its outlier arrives
constexpr uint32_t kDecSparseMax = 1024;  // other symbols per chunk at most, for a sparse frame

__device__ __forceinline__ void mark_corrupt(Scratch& s, uint32_t f) {
  s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
}

// The fields of a stream's header (24 words), checked against the context's
// geometry and each other as the oracle checks them; the stream's layout.
__device__ bool read_header(const uint32_t* hdr, const DevParams& p, uint64_t base, uint64_t in_bytes, DecInfo& di) {
  di = DecInfo{};
  di.base = base;
  const uint32_t roi_h = hdr[5] & 0xFFFFu, roi_w = hdr[5] >> 16;
  const uint32_t bh = hdr[6] & 0xFFFFu, bw = hdr[6] >> 16;
  di.eb = __uint_as_float(hdr[7]);
  di.two_eb = __fmul_rn(2.0f, di.eb);
  di.R = (int32_t)hdr[8];
  di.roi_h = (int32_t)roi_h;
  di.roi_w = (int32_t)roi_w;
  di.nsym = 2u * hdr[8];
  FramePlan& pl = di.pl;
  di.roi_coding = hdr[19];
  di.roi_bytes = hdr[20];
  di.roi_words = hdr[21];
  di.back_ref = hdr[22];
  pl.n_peaks = hdr[9];
  pl.n_lo = hdr[10];
  pl.n_pq = hdr[11];
  pl.n_words = hdr[15];
  const uint64_t total = (uint64_t)hdr[16] | ((uint64_t)hdr[17] << 32);
  bool ok = !(hdr[0] != kMagic || hdr[1] != kVersion || hdr[2] != p.P || hdr[3] != p.H || hdr[4] != p.W ||
              bh != (uint32_t)p.bh || bw != (uint32_t)p.bw || roi_h < 1 || roi_h > 63 || roi_w < 1 ||
              roi_w > 63 || hdr[8] < 2 || hdr[8] > 512 || hdr[12] != p.M || hdr[13] != kChunk ||
              hdr[14] != p.n_chunks || pl.n_lo > p.M || pl.n_pq > p.M || pl.n_words > p.M ||
              pl.n_peaks > 65535u || !(di.eb > 0.0f) || !isfinite(di.two_eb) ||
              hdr[18] != (p.dims == 2 ? 0u : (uint32_t)p.dims) ||  // the context's Lorenzo dimension
              di.roi_coding > 2 || (di.roi_coding == 0 && (di.roi_bytes | di.roi_words) != 0) ||
              di.back_ref > 63);  // a chunk holds at most 64 frames
  pl.off_peaks = kHeaderBytes;
  pl.off_roi = pl.off_peaks + align16((uint64_t)pl.n_peaks * 6);
  pl.off_len = pl.off_roi + (di.roi_coding == 0 ? align16((uint64_t)pl.n_peaks * roi_h * roi_w * 4) : 0);
  pl.off_cidx = pl.off_len + (di.back_ref == 0 ? align16(di.nsym) : 0);  // lengths: a chunk's head only
  pl.off_lo = pl.off_cidx + align16((uint64_t)p.n_chunks * 4);
  pl.off_pq = pl.off_lo + align16((uint64_t)pl.n_lo * 8);
  pl.off_bits = pl.off_pq + align16((uint64_t)pl.n_pq * 8);
  pl.total = pl.off_bits + align16((uint64_t)pl.n_words * 4);
  di.off_roi_sec = pl.total;  // the ROI section after the bitstream (roi coding 1, 2)
  pl.total += di.roi_bytes;
  if (pl.total != total || base + pl.total > in_bytes) ok = false;
  return ok;
}

// parse: one block per frame.  Reads the header and the code lengths (its own,
// or those of its chunk's head, back_ref frames earlier in the call), builds
// the canonical decoding tables and the prefix table, checks that both outlier
// lists are strictly ascending and inside the frame, and records where each
// panel's outliers start in them.
__global__ void __launch_bounds__(256) k_dec_parse(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t hdr[24], hhdr[24];
  __shared__ int ok;
  __shared__ uint64_t len_at;  // byte offset of the code lengths in the input
  __shared__ uint32_t cnt[34], first[34], idx0[34];
  __shared__ uint8_t lens[kMaxSymbols];
  __shared__ uint16_t order[kMaxSymbols];
  __shared__ uint32_t nsym_s;
  __shared__ int sparse;
  const uint32_t f = blockIdx.x;
  DecInfo di = {};
  if (threadIdx.x == 0) {
    s.dec_zero[f] = 0;
    ok = 1;
    const uint64_t base = a.offsets[f];
    if ((base & 15u) != 0 || base + kHeaderBytes > a.in_bytes) ok = 0;
    if (ok) {
      const uint32_t* h = reinterpret_cast<const uint32_t*>(a.in + base);
      for (int i = 0; i < 24; ++i) hdr[i] = h[i];
      ok = read_header(hdr, p, base, a.in_bytes, di) ? 1 : 0;
      len_at = base + di.pl.off_len;
    }
    // a stream without code lengths takes its chunk head's: the frame back_ref
    // earlier in this call, which must be a valid stream keeping its own
    // lengths, with the same alphabet
    if (ok && di.back_ref != 0) {
      DecInfo hd;
      const uint64_t hb = di.back_ref <= f ? a.offsets[f - di.back_ref] : 0;
      ok = di.back_ref <= f && (hb & 15u) == 0 && hb + kHeaderBytes <= a.in_bytes;
      if (ok) {
        const uint32_t* h = reinterpret_cast<const uint32_t*>(a.in + hb);
        for (int i = 0; i < 24; ++i) hhdr[i] = h[i];
        ok = read_header(hhdr, p, hb, a.in_bytes, hd) && hd.back_ref == 0 && hd.R == di.R;
        len_at = hb + hd.pl.off_len;
      }
    }
    if (!ok) {
      s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
      s.dec_info[f] = di;
    }
  }
  __syncthreads();
  if (!ok) return;
  if (threadIdx.x != 0) read_header(hdr, p, a.offsets[f], a.in_bytes, di);  // every thread's copy
  __syncthreads();
  // canonical decoding tables: count per length, first code per length, index
  // of the first symbol of each length in the (length, symbol) order.
  const uint8_t* base = a.in + di.base;
  uint32_t* tab = s.dec_table + (size_t)f * kDecTableWords;
  if (threadIdx.x < 34) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) nsym_s = di.nsym;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < di.nsym; k += blockDim.x) {
    const uint32_t L = a.in[len_at + k];
    lens[k] = (uint8_t)L;
    if (L > 32) ok = 0;
    else if (L > 0) atomicAdd(&cnt[L], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t c = 0;
    uint32_t prev = 0, idx = 0;
    uint64_t kraft = 0;  // sum of 2^(32 - L): a complete code sums to 2^32
    first[0] = idx0[0] = 0;
    for (uint32_t L = 1; L <= 32; ++L) {
      first[L] = 0;
      idx0[L] = idx;
      if (cnt[L]) {
        c = prev == 0 ? 0 : (c + cnt[prev]) << (L - prev);
        first[L] = (uint32_t)c;
        prev = L;
        kraft += (uint64_t)cnt[L] << (32 - L);
      }
      idx += cnt[L];
    }
    // a code with one symbol of length 1 is allowed (kraft = 2^31)
    const bool single = idx == 1 && cnt[1] == 1;
    if (idx == 0 || (kraft != (1ull << 32) && !single)) ok = 0;
    sparse = cnt[1] != 0;
  }
  __syncthreads();
  // sparse frame: with a length-1 code every other code takes 2 bits or more,
  // so a chunk of n symbols in w words holds at most 32 w - n other symbols
  if (sparse) {
    const uint32_t* cidx = reinterpret_cast<const uint32_t*>(base + di.pl.off_cidx);
    for (uint32_t k = threadIdx.x; k < p.n_chunks; k += blockDim.x) {
      const uint32_t w0 = cidx[k], w1 = k + 1 < p.n_chunks ? cidx[k + 1] : di.pl.n_words;
      const uint32_t n = min(p.M, k * kChunk + kChunk) - k * kChunk;
      if (w1 < w0 || 32ull * (w1 - w0) > (uint64_t)n + kDecSparseMax) sparse = 0;
    }
  }
  if (threadIdx.x <= 32) {
    const uint32_t L = threadIdx.x;
    tab[L] = L ? cnt[L] : 0;
    tab[34 + L] = first[L];
    tab[68 + L] = idx0[L];
  }
  // symbols in (length, symbol) order: rank among same-length smaller symbols
  for (uint32_t k = threadIdx.x; k < nsym_s; k += blockDim.x) {
    const uint32_t L = lens[k];
    if (L == 0 || L > 32) continue;
    uint32_t rank = 0;
    for (uint32_t j = 0; j < k; ++j) rank += lens[j] == L;
    tab[102 + idx0[L] + rank] = k;
    order[idx0[L] + rank] = (uint16_t)k;
  }
  __syncthreads();
  // prefix table: the shortest code that matches the top bits of the entry,
  // as the bit-serial decoder would find it
  if (ok) {
    for (uint32_t w = threadIdx.x; w < kDecLutWords; w += blockDim.x) {
      uint32_t word = 0;
      for (uint32_t h = 0; h < 2; ++h) {
        const uint32_t e = 2 * w + h;
        uint32_t ent = 0;
        for (uint32_t L = 1; L <= kDecLutBits; ++L) {
          const uint32_t code = e >> (kDecLutBits - L);
          if (cnt[L] && code >= first[L] && code - first[L] < cnt[L]) {
            ent = (L << 10) | order[idx0[L] + code - first[L]];
            break;
          }
        }
        word |= ent << (16 * h);
      }
      tab[kDecCanonWords + w] = word;
    }
  }
  // outlier lists: strictly ascending bin indices below M; the first entry of
  // each panel's run goes to the panel's start slot
  const uint32_t Mp = p.Hb * p.Wb;
  for (int list = 0; list < 2; ++list) {
    const uint2* v = reinterpret_cast<const uint2*>(base + (list == 0 ? di.pl.off_lo : di.pl.off_pq));
    const uint32_t n = list == 0 ? di.pl.n_lo : di.pl.n_pq;
    uint32_t* start = (list == 0 ? reinterpret_cast<uint32_t*>(s.dq) : reinterpret_cast<uint32_t*>(s.bhat)) +
                      (size_t)f * p.M;
    if (n == 0)
      for (uint32_t q = threadIdx.x; q < p.P; q += blockDim.x) start[q] = 0;
    for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
      const uint32_t x = v[e].x;
      const uint32_t px = e ? v[e - 1].x : 0u;
      if (x >= p.M || (e > 0 && px >= x)) {
        ok = 0;
        continue;
      }
      const uint32_t q1 = x / Mp;
      for (uint32_t q = e ? px / Mp + 1 : 0; q <= q1; ++q) start[q] = e;
      if (e == n - 1)
        for (uint32_t q = q1 + 1; q < p.P; ++q) start[q] = n;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) s.status[f] = ROIBIN_ERR_CORRUPT_STREAM;
    else s.status[f] = ROIBIN_OK;
    di.sparse = sparse ? 1u : 0u;
    s.dec_info[f] = di;
  }
}

// decode: one thread per chunk (block = 64 chunks of one frame).
constexpr int kDecThreads = 64;
// Other blocks of the frame may mark it corrupt while this one starts, so the
// go/no-go decision is read once and shared before any barrier.
__global__ void __launch_bounds__(kDecThreads) k_dec_decode(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t tab[kDecCanonWords];
  __shared__ int go;
  const uint32_t f = blockIdx.y;
  if (threadIdx.x == 0) go = s.status[f] == ROIBIN_OK;
  __syncthreads();
  if (!go) return;
  for (uint32_t i = threadIdx.x; i < kDecCanonWords; i += kDecThreads)
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

// cols: prefix sum down each column of a binned panel, then b^ = fl(q * 2eb)
// (dequant), or the sums back in place for the 3-D inverse (k_dec_stack).
__global__ void k_dec_cols(DevParams p, Scratch s, DecArgs a, int dequant) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.P * p.Wb) return;
  const uint32_t pn = t / p.Wb, j = t - pn * p.Wb;
  const float two_eb = s.dec_info[f].two_eb;
  uint32_t* dq = reinterpret_cast<uint32_t*>(s.dq + (size_t)f * p.M + (size_t)pn * p.Hb * p.Wb);
  float* bh = s.bhat + (size_t)f * p.M + (size_t)pn * p.Hb * p.Wb;
  uint32_t q = 0;
  for (uint32_t i = 0; i < p.Hb; ++i) {
    q += dq[(size_t)i * p.Wb + j];
    if (dequant) bh[(size_t)i * p.Wb + j] = __fmul_rn((float)(int32_t)q, two_eb);
    else dq[(size_t)i * p.Wb + j] = q;
  }
}

// stack (3-D inverse, last axis): prefix sum across the panels at each binned
// position of the 2-D sums, then b^ = fl(q * 2eb).  The three axes' prefix
// sums commute, so rows, columns, then panels inverts the 3-D predictor.
__global__ void k_dec_stack(DevParams p, Scratch s, DecArgs a) {
  const uint32_t f = blockIdx.y;
  if (s.status[f] != ROIBIN_OK) return;
  const uint32_t plane = p.Hb * p.Wb;
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= plane) return;
  const float two_eb = s.dec_info[f].two_eb;
  const uint32_t* dq = reinterpret_cast<const uint32_t*>(s.dq + (size_t)f * p.M);
  float* bh = s.bhat + (size_t)f * p.M;
  uint32_t q = 0;
  for (uint32_t pn = 0; pn < p.P; ++pn) {
    q += dq[(size_t)pn * plane + t];
    bh[(size_t)pn * plane + t] = __fmul_rn((float)(int32_t)q, two_eb);
  }
}

// chain (1-D inverse): after the row sums, every binned row adds the sum of
// all rows before it in the frame's row-major order.  One block per frame
// walks the rows in tiles of blockDim.x, scanning the tile's row totals.
constexpr uint32_t kChainThreads = 1024;
__global__ void __launch_bounds__(kChainThreads) k_dec_chain(DevParams p, Scratch s, DecArgs a) {
  __shared__ uint32_t carry[kChainThreads];
  __shared__ uint32_t warp_sum[kChainThreads / 32];
  const uint32_t f = blockIdx.x;
  if (s.status[f] != ROIBIN_OK) return;
  const float two_eb = s.dec_info[f].two_eb;
  const uint32_t* dq = reinterpret_cast<const uint32_t*>(s.dq + (size_t)f * p.M);
  float* bh = s.bhat + (size_t)f * p.M;
  const uint32_t rows = p.P * p.Hb, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  uint32_t base = 0;  // sum of every row before the tile (unsigned: wraps like the stream's int32)
  for (uint32_t r0 = 0; r0 < rows; r0 += kChainThreads) {
    const uint32_t r = r0 + tid;
    const uint32_t total = r < rows ? dq[(size_t)r * p.Wb + p.Wb - 1] : 0u;  // the row's inclusive sum
    const uint32_t inc = warp_incl_scan(total);
    if (lane == 31) warp_sum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = warp_incl_scan(warp_sum[lane]);
      warp_sum[lane] = w;
    }
    __syncthreads();
    carry[tid] = base + (warp ? warp_sum[warp - 1] : 0u) + inc - total;  // exclusive
    const uint32_t tile_sum = warp_sum[31];
    __syncthreads();
    const uint32_t n = min(kChainThreads, rows - r0);
    for (uint32_t k = warp; k < n; k += kChainThreads / 32) {
      const size_t row = (size_t)(r0 + k) * p.Wb;
      const uint32_t c = carry[k];
      for (uint32_t j = lane; j < p.Wb; j += 32)
        bh[row + j] = __fmul_rn((float)(int32_t)(dq[row + j] + c), two_eb);
    }
    base += tile_sum;
    __syncthreads();
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
  const uint32_t n_in_place = di.roi_coding == 0 ? di.pl.n_peaks : 0u;  // else k_dec_roi_coded
  for (uint32_t k = blockIdx.x * wpb + (threadIdx.x >> 5); k < n_in_place; k += gridDim.x * wpb) {
    const uint32_t pn = pk[3 * k], r = pk[3 * k + 1], c = pk[3 * k + 2];
    if (pn >= p.P || r >= p.H || c >= p.W) {
      if (lane_id() == 0) mark_corrupt(s, f);
      continue;
    }
    float* panel = a.out + (size_t)f * p.frame_px + (size_t)pn * p.H * p.W;
    const int r0 = (int)r - di.roi_h / 2, c0 = (int)c - di.roi_w / 2;
    if (!RB_CHECK(s, di.pl.off_roi + (uint64_t)(k + 1) * win * 4 <= di.pl.total, ROIBIN_CHECK_STREAM_READ)) continue;
    for (uint32_t e = lane_id(); e < win; e += 32) {
      const int rr = r0 + (int)(e / di.roi_w), cc = c0 + (int)(e % di.roi_w);
      if (rr >= 0 && rr < (int)p.H && cc >= 0 && cc < (int)p.W)
        panel[(size_t)rr * p.W + cc] = roi[(size_t)k * win + e];
    }
  }
}

// ---------------------------------------------------------------------------
// The panel path.
//
// The panel path's decoders: one thread per chunk, up to kDecMaxThreads chunks
// of one frame per block, like k_dec_decode, with two shortcuts.
//   - When a code of length 1 exists it is the all-zero code, so a run of z zero
//     bits is z copies of its symbol, taken in one step (count of leading zeros).
//   - Other codes: the next 12 bits index the prefix table (codes of up to 12
//     bits resolve in one lookup; longer ones continue bit by bit from length 13).
// A frame the parse step marked sparse (a length-1 code, and each chunk's bit
// count leaves room for at most kDecSparseMax other symbols) takes
// k_dec_decode_sparse, which lists only each chunk's other symbols (dec_list):
// the panel kernel fills the rest with the length-1 code's symbol, so the
// frame's symbols never go through device memory.  Other frames take
// k_dec_decode_dense, which writes every symbol to the [n][n_chunks * kChunk]
// u16 symbol array: it stages kDecRound symbols per thread in shared memory and
// has the warp store its 32 slots together, instead of each thread storing into
// its own cache lines.  Corrupt-stream checks are those of k_dec_decode.
constexpr uint32_t kDecRound = 32;                     // symbols per thread and round (dense)
constexpr uint32_t kDecSlotWords = kDecRound / 2 + 4;  // 64 bytes + 16 bytes of bank skew
constexpr uint32_t kDecMaxThreads = 256;

// Reads a chunk's words [w0, w1) in aligned 16-byte groups, one group ahead of
// the one being consumed; words at or past w1 read as 0.  The bitstream section
// starts 16-byte aligned and is padded to 16 bytes, so every group read lies
// inside it.
struct WordReader {
  const uint4* g4;
  uint32_t gi, ci, w1;
  uint4 cur, nxt;
  __device__ __forceinline__ uint4 group(uint32_t g) const {
    return 4 * g < w1 ? g4[g] : make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ void init(const uint32_t* words, uint32_t w0, uint32_t w1_) {
    g4 = reinterpret_cast<const uint4*>(words);
    w1 = w1_;
    gi = w0 >> 2;
    ci = w0 & 3u;
    cur = group(gi);
    nxt = group(gi + 1);
  }
  __device__ __forceinline__ uint32_t next() {
    uint32_t w = ci == 0 ? cur.x : ci == 1 ? cur.y : ci == 2 ? cur.z : cur.w;
    if (4 * gi + ci >= w1) w = 0;
    if (++ci == 4) {
      ci = 0;
      ++gi;
      cur = nxt;
      nxt = group(gi + 1);
    }
    return w;
  }
};

// One code from the top of `buf` (at least 32 valid bits): its length, 0 when
// no code of up to 32 bits matches; the symbol in `sym`.
__device__ __forceinline__ uint32_t decode_one(const uint32_t* tab, const uint16_t* lut, uint64_t buf,
                                               uint32_t& sym) {
  const uint32_t ent = lut[(uint32_t)(buf >> (64 - kDecLutBits))];
  sym = ent & 1023u;
  if (ent >> 10) return ent >> 10;
  uint32_t code = (uint32_t)(buf >> (64 - kDecLutBits));
  for (uint32_t L = kDecLutBits + 1; L <= 32; ++L) {
    code = (code << 1) | (uint32_t)(buf >> (63 - (L - 1)) & 1u);
    const uint32_t n = tab[L];
    if (n && code >= tab[34 + L] && code - tab[34 + L] < n) {
      sym = tab[102 + tab[68 + L] + (code - tab[34 + L])];
      return L;
    }
  }
  return 0;
}

// A sparse frame's symbols, as the decoder leaves them for the panel kernel:
// chunk k lists its symbols other than the length-1 code's, in order, as
// (position in the chunk << 16) | symbol, in the first half of the chunk's slot
// of the symbol array; the count per chunk goes to the [n][n_chunks] array the
// compressor uses for its per-chunk outlier offsets (free while decompressing).
__device__ __forceinline__ uint32_t* dec_list(const Scratch& s, const DevParams& p, uint32_t f, uint32_t k) {
  return reinterpret_cast<uint32_t*>(s.codes + ((size_t)f * p.n_chunks + k) * kChunk);
}
__device__ __forceinline__ uint32_t* dec_list_count(const Scratch& s, const DevParams& p, uint32_t f) {
  return s.chunk_lo + (size_t)f * p.n_chunks;
}
static_assert(kDecSparseMax * 4 <= kChunk * 2, "a chunk's list fits its slot of the symbol array");

// The frame's decoding tables into shared memory; false when the frame is not
// this kernel's (or not OK).  Read once by thread 0 and shared, since other
// blocks of the frame may mark it corrupt meanwhile.
__device__ __forceinline__ bool dec_load_tables(const Scratch& s, uint32_t f, bool want_sparse, uint32_t* tab,
                                                int* go) {
  if (threadIdx.x == 0) *go = s.status[f] == ROIBIN_OK && (s.dec_info[f].sparse != 0) == want_sparse;
  __syncthreads();
  if (!*go) return false;
  const uint4* src = reinterpret_cast<const uint4*>(s.dec_table + (size_t)f * kDecTableWords);
  uint4* dst = reinterpret_cast<uint4*>(tab);
  static_assert(kDecTableWords % 4 == 0, "table copied in 16-byte pieces");
  for (uint32_t i = threadIdx.x; i < kDecTableWords / 4; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kDecMaxThreads) k_dec_decode_sparse(DevParams p, Scratch s, DecArgs a) {
  __shared__ __align__(16) uint32_t tab[kDecTableWords];
  __shared__ int go;
  const uint32_t f = blockIdx.y;
  if (!dec_load_tables(s, f, true, tab, &go)) return;
  const uint16_t* lut = reinterpret_cast<const uint16_t*>(tab + kDecCanonWords);
  // the length-1 code is code 0: its symbol comes first in the (length, symbol) order
  const uint32_t zsym = tab[102];
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.n_chunks) return;
  const DecInfo& di = s.dec_info[f];
  const uint8_t* base = a.in + di.base;
  const uint32_t n_words = di.pl.n_words;
  const uint32_t* cidx = reinterpret_cast<const uint32_t*>(base + di.pl.off_cidx);
  const uint32_t* words = reinterpret_cast<const uint32_t*>(base + di.pl.off_bits);
  const uint32_t w0 = cidx[k];
  const uint32_t w1 = k + 1 < p.n_chunks ? cidx[k + 1] : n_words;
  uint32_t* count = dec_list_count(s, p, f) + k;
  if (w0 > w1 || w1 > n_words) {
    *count = 0;
    mark_corrupt(s, f);
    return;
  }
  const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
  const uint32_t n_sym = min(p.M, k * kChunk + kChunk) - k * kChunk;
  uint32_t* list = dec_list(s, p, f, k);
  WordReader rd;
  rd.init(words, w0, w1);
  uint64_t buf = 0;  // next bits, MSB first; nbuf of them are valid
  uint32_t nbuf = 0, pos = 0, zeros = 0, n_list = 0;
  uint64_t bit = 0;
  bool bad = false;
  while (pos < n_sym) {
    if (nbuf < 32) {
      buf |= (uint64_t)rd.next() << (32 - nbuf);
      nbuf += 32;
    }
    if ((buf >> 63) == 0) {
      const uint32_t z = min(min((uint32_t)__clzll(buf), nbuf), n_sym - pos);
      pos += z;
      buf <<= z;
      nbuf -= z;
      bit += z;
      if (zsym == 0) zeros += z;
    } else {
      uint32_t sym;
      const uint32_t L = decode_one(tab, lut, buf, sym);
      if (L == 0 || n_list == kDecSparseMax) {
        bad = true;
        break;
      }
      list[n_list++] = (pos << 16) | sym;
      ++pos;
      buf <<= L;
      nbuf -= L;
      bit += L;
      zeros += sym == 0;
    }
    if (bit > bit_end) {
      bad = true;
      break;
    }
  }
  *count = bad ? 0u : n_list;
  if (bad || (bit + 31) / 32 != (uint64_t)(w1 - w0)) mark_corrupt(s, f);
  if (zeros) atomicAdd(s.dec_zero + f, zeros);
}

struct SymbolWriter {  // eight u16 symbols per 16-byte shared-memory store
  uint16_t* slot;      // this thread's slot (16-byte aligned)
  uint32_t pos = 0;    // symbols emitted in the chunk
  uint64_t lo = 0, hi = 0;
  __device__ __forceinline__ void flush() {
    *reinterpret_cast<uint4*>(slot + ((pos - 8) & (kDecRound - 1))) =
        make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
    lo = hi = 0;
  }
  __device__ __forceinline__ void put(uint32_t sym) {
    const uint32_t k = pos & 7u;
    if (k < 4) lo |= (uint64_t)sym << (16 * k);
    else hi |= (uint64_t)sym << (16 * (k - 4));
    ++pos;
    if ((pos & 7u) == 0) flush();
  }
  __device__ __forceinline__ void run(uint32_t sym, uint32_t z) {
    while (z && (pos & 7u)) {
      put(sym);
      --z;
    }
    const uint64_t rep = (uint64_t)sym * 0x0001000100010001ull;
    for (; z >= 8; z -= 8) {
      pos += 8;
      lo = hi = rep;
      flush();
    }
    while (z) {
      put(sym);
      --z;
    }
  }
  __device__ __forceinline__ void finish() {  // the chunk's last partial group
    const uint32_t k = pos & 7u, b = (pos - k) & (kDecRound - 1);
#pragma unroll
    for (uint32_t h = 0; h < 7; ++h)
      if (h < k) slot[b + h] = (uint16_t)((h < 4 ? lo >> (16 * h) : hi >> (16 * (h - 4))) & 0xFFFFu);
  }
};

__global__ void __launch_bounds__(kDecMaxThreads) k_dec_decode_dense(DevParams p, Scratch s, DecArgs a) {
  __shared__ __align__(16) uint32_t tab[kDecTableWords];
  __shared__ __align__(16) uint32_t slots[kDecMaxThreads * kDecSlotWords];
  __shared__ int go;
  const uint32_t f = blockIdx.y;
  if (!dec_load_tables(s, f, false, tab, &go)) return;
  const uint16_t* lut = reinterpret_cast<const uint16_t*>(tab + kDecCanonWords);
  const uint32_t lane = lane_id();
  const uint32_t warp0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);  // chunk of lane 0
  if (warp0 >= p.n_chunks) return;  // whole warp past the last chunk
  const uint32_t k = warp0 + lane;
  const bool live = k < p.n_chunks;
  const DecInfo& di = s.dec_info[f];
  const uint8_t* base = a.in + di.base;
  const uint32_t n_words = di.pl.n_words;
  const uint32_t* cidx = reinterpret_cast<const uint32_t*>(base + di.pl.off_cidx);
  const uint32_t* words = reinterpret_cast<const uint32_t*>(base + di.pl.off_bits);
  uint32_t w0 = 0, w1 = 0, n_sym = 0;
  bool bad = false;
  if (live) {
    w0 = cidx[k];
    w1 = k + 1 < p.n_chunks ? cidx[k + 1] : n_words;
    n_sym = min(p.M, k * kChunk + kChunk) - k * kChunk;
    if (w0 > w1 || w1 > n_words) bad = true;
  }
  const uint64_t bit_end = (uint64_t)(w1 - w0) * 32;
  // the length-1 code, when there is one, is code 0: its symbol comes first
  // in the (length, symbol) order
  const bool zrun = tab[1] != 0;
  const uint32_t zsym = tab[102];
  uint32_t* warp_slots = slots + (threadIdx.x & ~31u) * kDecSlotWords;
  SymbolWriter wr;
  wr.slot = reinterpret_cast<uint16_t*>(warp_slots + lane * kDecSlotWords);
  uint16_t* out = s.codes + (size_t)f * p.n_chunks * kChunk;
  const uint32_t n_warp = min(32u, p.n_chunks - warp0);  // live lanes
  WordReader rd;  // a lane with a bad chunk index reads nothing
  rd.init(words, w0, live && !bad ? w1 : 0u);
  uint64_t bit = 0;
  uint32_t zeros = 0;
  uint64_t buf = 0;  // next bits, MSB first; nbuf of them are valid
  uint32_t nbuf = 0;
  for (uint32_t r0 = 0; r0 < kChunk; r0 += kDecRound) {
    const uint32_t target = min(n_sym, r0 + kDecRound);
    while (!bad && wr.pos < target) {
      if (nbuf < 32) {
        buf |= (uint64_t)rd.next() << (32 - nbuf);
        nbuf += 32;
      }
      if (zrun && (buf >> 63) == 0) {
        const uint32_t z = min(min((uint32_t)__clzll(buf), nbuf), target - wr.pos);
        wr.run(zsym, z);
        buf <<= z;
        nbuf -= z;
        bit += z;
        if (zsym == 0) zeros += z;
      } else {
        uint32_t sym;
        const uint32_t L = decode_one(tab, lut, buf, sym);
        if (L == 0) {
          bad = true;
          break;
        }
        wr.put(sym);
        buf <<= L;
        nbuf -= L;
        bit += L;
        zeros += sym == 0;
      }
      if (bit > bit_end) bad = true;
    }
    if (!bad && wr.pos == n_sym && (n_sym & 7u)) wr.finish();
    __syncwarp();
    // the warp writes the round out: lanes 0-15 one slot, lanes 16-31 the next
    for (uint32_t b0 = 0; b0 < n_warp; b0 += 2) {
      const uint32_t b = b0 + (lane >> 4), w = lane & 15u;
      if (b < n_warp) {
        const uint32_t kb = warp0 + b;
        const uint32_t cnt = min(p.M, kb * kChunk + kChunk) - kb * kChunk;  // symbols of chunk kb
        const uint32_t i = r0 + 2 * w;                                       // first symbol of the word
        const uint32_t v = warp_slots[b * kDecSlotWords + w];
        uint16_t* dst = out + (size_t)kb * kChunk + i;
        if (i + 1 < cnt) *reinterpret_cast<uint32_t*>(dst) = v;
        else if (i < cnt) *dst = (uint16_t)v;
      }
    }
    __syncwarp();
  }
  if (live) {
    if (bad || (bit + 31) / 32 != (uint64_t)(w1 - w0)) mark_corrupt(s, f);
    if (zeros) atomicAdd(s.dec_zero + f, zeros);
  }
}

// Places the outliers of one strip.  The run of the list that belongs to the
// panel is ascending, so the strip's entries are the first ones still unplaced:
// thread t takes entry cur + t, and the count of threads that found theirs in
// the strip advances the cursor for everyone.  `place(bin, value)` returns false
// on a corrupt entry.
template <class F>
__device__ __forceinline__ uint32_t place_strip_outliers(const uint2* v, uint32_t cur, uint32_t end, uint32_t sb1,
                                                         F place, bool& bad) {
  for (;;) {
    const uint32_t e = cur + threadIdx.x;
    bool in = false;
    if (e < end) {
      const uint2 x = v[e];
      in = x.x < sb1;
      if (in && !place(x.x, x.y)) bad = true;
    }
    const uint32_t n_in = (uint32_t)__syncthreads_count(in);
    cur += n_in;
    if (n_in < blockDim.x) return cur;
  }
}

// panel: one block per (panel, frame).  Strip by strip (sb binned rows):
//   symbols -> deltas in shared memory (code 0: sentinel), Lorenzo outliers in;
//   column prefix sums carried from the strip above (thread per column);
//   row prefix sums (thread per row segment: a sequential scan of its segment,
//   then the segment totals scanned across the lanes of the row);
//   b^ = fl(q * 2eb), prequantisation outliers in;
//   the strip's output rows (every pixel takes its bin's value).
// After the last strip, the panel's ROI windows overwrite their in-panel pixels.
// The 2-D prefix sum wraps modulo 2^32 in any order, so column-then-row equals
// the row-then-column definition.
// The symbols of the next strip arrive by a 1-D TMA bulk copy (a 16-byte
// aligned superset of the strip) while the block works on the current one.
constexpr int kPanelThreads = 256;
constexpr uint32_t kPanelMaxWb = 4096;  // widest binned row the panel path takes
// carry[Wb] + tile[sb][Wb] (u32); the symbol buffer (u16, + 32 bytes of
// alignment slack) starts 16-byte aligned, as a bulk copy's destination must;
// then the mbarrier
__host__ __device__ inline uint32_t panel_sym_offset(uint32_t Wb, uint32_t sb) { return (4 * Wb * (sb + 1) + 15) & ~15u; }
__host__ __device__ inline uint32_t panel_sym_bytes(uint32_t Wb, uint32_t sb) { return (2 * Wb * sb + 32 + 15) & ~15u; }
__host__ __device__ inline uint32_t panel_smem_bytes(uint32_t Wb, uint32_t sb) {
  return panel_sym_offset(Wb, sb) + panel_sym_bytes(Wb, sb) + 16;
}
__global__ void __launch_bounds__(kPanelThreads, 8) k_dec_panel(DevParams p, Scratch s, DecArgs a, uint32_t sb,
                                                                uint32_t lg_seg, int vec4) {
  extern __shared__ __align__(16) int32_t sm[];  // carry[Wb], tile[sb][Wb], symbols, mbarrier
  __shared__ int go;
  const uint32_t pn = blockIdx.x, f = blockIdx.y;
  const uint32_t Wb = p.Wb, Hb = p.Hb, Mp = Hb * Wb, W = p.W, H = p.H, bh = p.bh;
  if (threadIdx.x == 0) {
    go = s.status[f] == ROIBIN_OK && s.dec_zero[f] == s.dec_info[f].pl.n_lo;
    // a code-0 count that differs from the Lorenzo-outlier count
    if (!go && s.status[f] == ROIBIN_OK) mark_corrupt(s, f);
    // the bulk copy's destination must be 16-byte aligned
    if ((smem_u32(reinterpret_cast<uint8_t*>(sm) + panel_sym_offset(Wb, sb)) & 15u) != 0) {
      go = 0;
      s.status[f] = ROIBIN_ERR_CUDA;
    }
  }
  __syncthreads();
  if (!go) return;
  const DecInfo& di = s.dec_info[f];
  const uint32_t pb = pn * Mp;
  const int32_t R = di.R;
  const float two_eb = di.two_eb;
  const uint8_t* base = a.in + di.base;
  const uint2* lo = reinterpret_cast<const uint2*>(base + di.pl.off_lo);
  const uint2* pq = reinterpret_cast<const uint2*>(base + di.pl.off_pq);
  const uint32_t* lo_start = reinterpret_cast<const uint32_t*>(s.dq) + (size_t)f * p.M;
  const uint32_t* pq_start = reinterpret_cast<const uint32_t*>(s.bhat) + (size_t)f * p.M;
  uint32_t lo_cur = lo_start[pn], pq_cur = pq_start[pn];
  const uint32_t lo_end = pn + 1 < p.P ? lo_start[pn + 1] : di.pl.n_lo;
  const uint32_t pq_end = pn + 1 < p.P ? pq_start[pn + 1] : di.pl.n_pq;
  uint32_t* carry = reinterpret_cast<uint32_t*>(sm);
  uint32_t* tile = carry + Wb;
  float* tilef = reinterpret_cast<float*>(tile);
  uint8_t* symbuf = reinterpret_cast<uint8_t*>(sm) + panel_sym_offset(Wb, sb);
  uint64_t* bar = reinterpret_cast<uint64_t*>(symbuf + panel_sym_bytes(Wb, sb));
  // the frame's symbols start 16-byte aligned (chunks of kChunk u16)
  const uint8_t* fsym = reinterpret_cast<const uint8_t*>(s.codes + (size_t)f * p.n_chunks * kChunk);
  const uint64_t policy = evict_first_policy();
  // strip r0's symbols: bytes [2 (pb + r0 Wb), 2 (pb + (r0 + nr) Wb)) of fsym,
  // copied from the 16-byte boundary below to the one above
  auto fetch = [&](uint32_t r0) {
    const uint32_t nr = min(sb, Hb - r0);
    const uint32_t b0 = 2 * (pb + r0 * Wb), b1 = 2 * (pb + (r0 + nr) * Wb);
    const uint32_t a0 = b0 & ~15u, a1 = (b1 + 15) & ~15u;
    fence_proxy_async();
    mbar_expect_tx(bar, a1 - a0);
    tma_load_1d(symbuf, fsym + a0, a1 - a0, bar, policy);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  // a sparse frame's strips are filled with the length-1 code's delta and its
  // listed symbols scattered in; a dense frame's symbols come by bulk copy
  const bool sparse = di.sparse != 0;
  const uint32_t zsym = s.dec_table[(size_t)f * kDecTableWords + 102];
  const uint32_t fillv = zsym ? (uint32_t)((int32_t)zsym - R) : (uint32_t)kSentinel;
  const uint32_t* counts = dec_list_count(s, p, f);
  if (threadIdx.x == 0 && !sparse) fetch(0);
  uint32_t phase = 0;
  bool timed_out = false;  // uniform: set after a barrier
  float* panel = a.out + (size_t)f * p.frame_px + (size_t)pn * H * W;
  // row-segment role: row seg_row of the strip, segment seg of 2^lg_seg
  const uint32_t G = 1u << lg_seg, seg_row = threadIdx.x >> lg_seg, seg = threadIdx.x & (G - 1);
  const uint32_t seg_len = ceil_div(Wb, G);
  const uint32_t sj0 = min(Wb, seg * seg_len), sj1 = min(Wb, sj0 + seg_len);
  // output role (vec4): float4 column c4 of bin row orow, advanced by (dr, dc)
  const uint32_t W4 = W / 4;
  const uint32_t dr = vec4 ? blockDim.x / W4 : 0, dc = vec4 ? blockDim.x - dr * W4 : 0;
  bool bad = false;
  for (uint32_t j = threadIdx.x; j < Wb; j += blockDim.x) carry[j] = 0;
  for (uint32_t r0 = 0; r0 < Hb; r0 += sb) {
    const uint32_t nr = min(sb, Hb - r0), nb = nr * Wb;
    const uint32_t sb0 = pb + r0 * Wb, sb1 = sb0 + nb;
    // symbols -> deltas (code 0: sentinel until its outlier arrives)
    if (sparse) {
      for (uint32_t e = threadIdx.x; e < nb; e += blockDim.x) tile[e] = fillv;
      __syncthreads();
      // the strip's bins lie in chunks sb0 / kChunk .. (sb1 - 1) / kChunk
      for (uint32_t k = sb0 / kChunk; k <= (sb1 - 1) / kChunk; ++k) {
        const uint32_t* list = dec_list(s, p, f, k);
        const uint32_t cnt = min(counts[k], kDecSparseMax), kb = k * kChunk;
        for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
          const uint32_t v = list[e], x = kb + (v >> 16), u = v & 0xFFFFu;
          if (x >= sb0 && x < sb1) tile[x - sb0] = u ? (uint32_t)((int32_t)u - R) : (uint32_t)kSentinel;
        }
      }
      __syncthreads();
    } else {
      const bool late = !mbar_wait(bar, phase);
      phase ^= 1u;
      if (!late) {
        const uint16_t* u16 = reinterpret_cast<const uint16_t*>(symbuf) + ((2 * (pb + r0 * Wb)) & 15u) / 2;
        for (uint32_t e = threadIdx.x; e < nb; e += blockDim.x) {
          const uint32_t u = u16[e];
          tile[e] = u ? (uint32_t)((int32_t)u - R) : (uint32_t)kSentinel;
        }
      }
      if (__syncthreads_or(late)) {
        // a copy that did not land in time: wait for it once more (bounded), then stop
        if (threadIdx.x == 0) mbar_wait(bar, phase ^ 1u);
        timed_out = true;
        break;
      }
      // the buffer is free: the next strip's symbols come in behind this one
      if (threadIdx.x == 0 && r0 + sb < Hb) fetch(r0 + sb);
    }
    lo_cur = place_strip_outliers(lo, lo_cur, lo_end, sb1, [&](uint32_t x, uint32_t y) {
      if (x < sb0 || tile[x - sb0] != (uint32_t)kSentinel) return false;
      tile[x - sb0] = y;
      return true;
    }, bad);
    // column prefix sums, carried from the strip above (unsigned: wraps instead
    // of overflowing on corrupt input)
    for (uint32_t j = threadIdx.x; j < Wb; j += blockDim.x) {
      uint32_t q = carry[j];
      for (uint32_t i = 0; i < nr; ++i) {
        q += tile[i * Wb + j];
        tile[i * Wb + j] = q;
      }
      carry[j] = q;
    }
    __syncthreads();
    // row prefix sums and b^ = fl(q * 2eb)
    {
      const bool mine = seg_row < nr;
      uint32_t* row = tile + seg_row * Wb;
      uint32_t run = 0;
      if (mine)
        for (uint32_t j = sj0; j < sj1; ++j) {
          run += row[j];
          row[j] = run;
        }
      // exclusive scan of the segment totals across the G lanes of the row
      uint32_t incl = run;
      for (uint32_t d = 1; d < G; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d, G);
        if (seg >= d) incl += v;
      }
      const uint32_t excl = incl - run;
      if (mine)
        for (uint32_t j = sj0; j < sj1; ++j)
          tilef[seg_row * Wb + j] = __fmul_rn((float)(int32_t)(row[j] + excl), two_eb);
    }
    __syncthreads();
    pq_cur = place_strip_outliers(pq, pq_cur, pq_end, sb1, [&](uint32_t x, uint32_t y) {
      if (x < sb0) return false;
      tilef[x - sb0] = __uint_as_float(y);
      return true;
    }, bad);
    // output rows of the strip: bin row i covers pixel rows (r0 + i) * bh ...
    // (streaming stores: the kernel never reads these pixels back)
    if (vec4) {  // bin width 2, W % 4 == 0: one float4 = 2 bins, stored on each of its rows
      const uint32_t n2 = nr * W4;
      uint32_t i = threadIdx.x / W4, c4 = threadIdx.x - i * W4;
      for (uint32_t e = threadIdx.x; e < n2; e += blockDim.x) {
        const float2 v = *reinterpret_cast<const float2*>(tilef + i * Wb + 2 * c4);
        const float4 o = make_float4(v.x, v.x, v.y, v.y);
        const uint32_t pr0 = (r0 + i) * bh, pr1 = min(H, pr0 + bh);
        for (uint32_t pr = pr0; pr < pr1; ++pr) __stcs(reinterpret_cast<float4*>(panel + (size_t)pr * W) + c4, o);
        i += dr;
        c4 += dc;
        if (c4 >= W4) {
          c4 -= W4;
          ++i;
        }
      }
    } else {
      const uint32_t ro0 = r0 * bh, ro1 = min(H, (r0 + nr) * bh);
      const uint32_t n1 = (ro1 - ro0) * W;
      for (uint32_t e = threadIdx.x; e < n1; e += blockDim.x) {
        const uint32_t rr = e / W, c = e - rr * W;
        __stcs(panel + (size_t)ro0 * W + e, tilef[((ro0 + rr) / bh - r0) * Wb + c / p.bw]);
      }
    }
    __syncthreads();
  }
  if (lo_cur != lo_end || pq_cur != pq_end) bad = true;
  if (timed_out) {
    if (threadIdx.x == 0) s.status[f] = ROIBIN_ERR_TIMEOUT;
    return;
  }
  // ROI windows of this panel's peaks (every block checks every peak's place);
  // a ROI section after the bitstream is restored by k_dec_roi_coded instead
  const uint16_t* pk = reinterpret_cast<const uint16_t*>(base + di.pl.off_peaks);
  const float* roi = reinterpret_cast<const float*>(base + di.pl.off_roi);
  const uint32_t win = (uint32_t)(di.roi_h * di.roi_w);
  const uint32_t n_in_place = di.roi_coding == 0 ? di.pl.n_peaks : 0u;
  for (uint32_t k = threadIdx.x >> 5; k < n_in_place; k += blockDim.x >> 5) {
    const uint32_t kp = pk[3 * k], r = pk[3 * k + 1], c = pk[3 * k + 2];
    if (kp >= p.P || r >= H || c >= W) {
      bad = true;
      continue;
    }
    if (kp != pn) continue;
    const int r0 = (int)r - di.roi_h / 2, c0 = (int)c - di.roi_w / 2;
    for (uint32_t e = lane_id(); e < win; e += 32) {
      const int rr = r0 + (int)(e / di.roi_w), cc = c0 + (int)(e % di.roi_w);
      if (rr >= 0 && rr < (int)H && cc >= 0 && cc < (int)W) panel[(size_t)rr * W + cc] = roi[(size_t)k * win + e];
    }
  }
  if (bad) mark_corrupt(s, f);
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
cudaError_t launch_dec_cols(const DevParams& p, const Scratch& s, const DecArgs& a, bool dequant, cudaStream_t st) {
  dim3 grid(ceil_div(p.P * p.Wb, 128), a.n_frames);
  k_dec_cols<<<grid, 128, 0, st>>>(p, s, a, dequant ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_dec_carry(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  if (p.dims == 3) {
    dim3 grid(ceil_div(p.Hb * p.Wb, 256), a.n_frames);
    k_dec_stack<<<grid, 256, 0, st>>>(p, s, a);
  } else {
    k_dec_chain<<<a.n_frames, kChainThreads, 0, st>>>(p, s, a);
  }
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
  return cudaGetLastError();
}
cudaError_t launch_dec_finish(const Scratch& s, const DecArgs& a, cudaStream_t st) {
  k_dec_finish<<<ceil_div(a.n_frames, 256), 256, 0, st>>>(s, a.frame_status, a.n_frames);
  return cudaGetLastError();
}
uint32_t dec_panel_rows(const DevParams& p) {
  if (p.Wb > kPanelMaxWb) return 0;
  // the most rows (up to 32) that fit 24 KB, so that 8 blocks share an SM
  // (at least one row, in up to 48 KB), then evened out over the strips
  uint32_t most = 1;
  while (most < 32 && most < p.Hb && panel_smem_bytes(p.Wb, most + 1) <= 24576) ++most;
  const uint32_t strips = ceil_div(p.Hb, most);
  return ceil_div(p.Hb, strips);
}
cudaError_t launch_dec_decoders(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  // a thread per chunk, in whole warps; a frame's chunks in as few blocks as fit
  const uint32_t threads = std::min<uint32_t>(kDecMaxThreads, ceil_div(p.n_chunks, 32) * 32);
  dim3 grid(ceil_div(p.n_chunks, threads), a.n_frames);
  k_dec_decode_sparse<<<grid, threads, 0, st>>>(p, s, a);
  if (cudaGetLastError() != cudaSuccess) return cudaGetLastError();
  k_dec_decode_dense<<<grid, threads, 0, st>>>(p, s, a);
  return cudaGetLastError();
}
cudaError_t launch_dec_panel(const DevParams& p, const Scratch& s, const DecArgs& a, cudaStream_t st) {
  const uint32_t sb = dec_panel_rows(p);
  if (sb == 0) return cudaErrorInvalidValue;
  const bool vec4 = p.bw == 2 && (p.W % 4) == 0 && (reinterpret_cast<uintptr_t>(a.out) % 16) == 0;
  const size_t smem = panel_smem_bytes(p.Wb, sb);
  // row segments: the most lanes per row that still give every row of a strip
  // its own lanes (sb <= 32, so at least 8)
  uint32_t lg_seg = 5;
  while (lg_seg > 0 && (sb << lg_seg) > (uint32_t)kPanelThreads) --lg_seg;
  dim3 grid(p.P, a.n_frames);
  k_dec_panel<<<grid, kPanelThreads, smem, st>>>(p, s, a, sb, lg_seg, vec4 ? 1 : 0);
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
