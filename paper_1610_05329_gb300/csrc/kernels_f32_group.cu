// FP32 grouped steps: the step kernels of same-shaped condensates launched once for the
// whole group (GroupLaunch in dgpe_device.cuh), compiled apart from kernels_f32.cu so that
// the two build in parallel.
#include "dgpe_device.cuh"

namespace dgpe {
cudaError_t group_init_f32() { return GroupLaunch<float>::init(); }
cudaError_t group_step_f32(const KArgs &a, const KArgs *ga, int n, int renorm, cudaStream_t st) {
  return GroupLaunch<float>::step(a, ga, n, renorm, st);
}
}  // namespace dgpe
