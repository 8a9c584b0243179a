// fused_jobs.cu - one persistent launch over several batches of frames, each
// with its own geometry and parameters (the stream of a facility whose
// detectors differ, §4.1 and §5.3.5: the work of many events spread over the
// device at once).  The batches' work items share one ticket counter, cut
// into slices: slice k holds the k-th run of tickets of every batch (one
// slice by default: each batch's tickets in one run, so the next batch fills
// the previous one's tail instead of a gap between launches).  A CTA runs
// each ticket with its batch's parameters, scratch and shape and the code of
// k_fused, so every frame's bytes are those of compressing its batch alone.  A batch's
// own tickets are handed out in their order, and a CTA only waits for work of
// its own batch handed out at an earlier ticket, so the argument that every
// wait ends is the one for a single batch.
#include "fused_device.cuh"

namespace roibin {

// The job table is a kernel parameter read in place (__grid_constant__, no
// copy).  The CTAs per SM and ring slots are common to every job (the ring
// barriers are set up once per CTA), so the control words and barriers sit at
// the same offsets for every job.  Built for 3 CTAs per SM (80 registers):
// one body runs every job's geometry and peak variant, and at 4 CTAs per SM
// (64 registers) it spilled 528 bytes; on a CSPAD + epix10k + 8 x 512 x 1024
// batch the launch took 6.75 ms at 3 CTAs and 4 ring slots, 7.11 ms at 4 CTAs
// and 7.94 ms at 2.
__global__ void __launch_bounds__(kPT, 3) k_fused_jobs(const __grid_constant__ FusedJobs m) {
  extern __shared__ __align__(128) unsigned char sm[];
  const FusedShape& sh0 = m.job[0].sh;
  fused_cta_init(sm, sh0);
  uint32_t ring_iter = 0;  // ring stages consumed so far (the same in every thread)
  for (;;) {
    const uint32_t t = fused_next_ticket(sm, sh0, m.ticket);
    if (t >= m.total) break;
    const uint32_t k = t / m.slice, o = t - k * m.slice;
    uint32_t j = 0;
    while (o >= m.job[j].cend) ++j;
    const FusedJob& J = m.job[j];
    const uint32_t u = k * J.chunk + (o - J.cbegin);  // the job's own ticket
    if (u >= J.tickets) continue;                      // past the job's last one
    const SyncWords sw = sync_words(J.s, J.a.n_frames);
    // one copy of the item code per column-group count; dense peaks (sh.dense) at run time
    const bool worked = J.sh.kG > 1 ? fused_ticket<false, kMaxG, true>(J.p, J.s, J.a, J.sh, sw, sm, u, ring_iter)
                                    : fused_ticket<false, 1, true>(J.p, J.s, J.a, J.sh, sw, sm, u, ring_iter);
    if (worked) __syncthreads();
  }
}

bool fused_jobs_plan(FusedJobs* m, const FusedShape* tuned, int num_sms, uint32_t* smem, uint32_t* grid) {
  if (m->n_jobs < 1 || m->n_jobs > kMaxFusedJobs) return false;
  // (CTAs per SM, ring slots), the measured default first
  static const uint32_t kCandidates[][2] = {{3, 4}, {3, 3}, {3, 2}, {2, 2}, {2, 1}, {1, 1}};
  for (const auto& c : kCandidates) {
    const uint32_t ctas = c[0], stages = c[1];
    bool ok = true;
    uint32_t need = 0;
    for (uint32_t i = 0; ok && i < m->n_jobs; ++i) {
      FusedJob& J = m->job[i];
      FusedShape sh;
      ok = fused_shape_for(J.p, ctas, 2, stages, &sh) && sh.ctas_per_sm == ctas;  // two binned rows per step
      if (!ok) break;
      sh.wait_limit = tuned[i].wait_limit;
      sh.dense = J.dense;
      J.sh = sh;
      const uint32_t bytes = J.dense ? sh.smem_dense : sh.smem;
      need = bytes > need ? bytes : need;
    }
    if (!ok) continue;
    if (cudaFuncSetAttribute(k_fused_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_jobs, kPT, need) != cudaSuccess ||
        per_sm < (int)ctas) {
      cudaGetLastError();
      continue;
    }
    uint64_t most = 0;
    for (uint32_t i = 0; i < m->n_jobs; ++i) {
      FusedJob& J = m->job[i];
      const uint32_t n = J.a.n_frames;
      J.sh.lag1 = n < kLagSize ? n : kLagSize;
      J.sh.lag2 = n < kLagWrite ? n : kLagWrite;
      const uint64_t t = fused_tickets(J.sh, n);
      if (t >= (1ull << 31)) return false;
      J.tickets = (uint32_t)t;
      most = t > most ? t : most;
    }
    const uint64_t slices = most < kJobSlices ? most : kJobSlices;
    uint64_t slice = 0;
    for (uint32_t i = 0; i < m->n_jobs; ++i) {
      FusedJob& J = m->job[i];
      J.chunk = (uint32_t)((J.tickets + slices - 1) / slices);
      J.cbegin = (uint32_t)slice;
      slice += J.chunk;
      J.cend = (uint32_t)slice;
    }
    const uint64_t total = slices * slice;
    if (total + ctas * (uint64_t)num_sms >= (1ull << 32)) return false;  // every CTA's last ticket stays below 2^32
    m->total = (uint32_t)total;
    m->slice = (uint32_t)slice;
    *smem = need;
    const uint64_t ctas_all = (uint64_t)ctas * (uint64_t)num_sms;
    *grid = (uint32_t)(total < ctas_all ? total : ctas_all);
    return true;
  }
  return false;
}

cudaError_t launch_fused_jobs(const FusedJobs& m, uint32_t smem, uint32_t grid, cudaStream_t st) {
  const cudaError_t e = cudaFuncSetAttribute(k_fused_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_fused_jobs<<<grid, kPT, smem, st>>>(m);
  return cudaGetLastError();
}

}  // namespace roibin
