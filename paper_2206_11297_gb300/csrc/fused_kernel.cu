// fused_kernel.cu - the persistent cluster kernel (one launch per batch).
#include <cuda_runtime.h>

#include "roibin_internal.cuh"

namespace roibin {

bool fused_supported(const DevParams& p, int device) {
  (void)p;
  (void)device;
  return false;
}

uint64_t fused_scratch_bytes_per_frame(const DevParams& p) {
  (void)p;
  return 0;
}

cudaError_t launch_fused(const DevParams& p, const Scratch& s, const PlainArgs& a, cudaStream_t st,
                         int num_sms) {
  (void)p;
  (void)s;
  (void)a;
  (void)st;
  (void)num_sms;
  return cudaErrorNotSupported;
}

}  // namespace roibin
