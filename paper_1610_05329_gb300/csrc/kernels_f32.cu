// FP32 instantiation of the SSCN kernels (complex64 psi and spectrum; the norm, mu and
// energy sums stay FP64 in both precisions).
#include "dgpe_device.cuh"

namespace dgpe {
const KernelSet *kernels_f32() { return Impl<float>::set(); }
}  // namespace dgpe
