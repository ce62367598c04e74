// FP64 instantiation of the SSCN kernels (complex128 psi and spectrum).
#include "dgpe_device.cuh"

namespace dgpe {
const KernelSet *kernels_f64() { return Impl<double>::set(); }
}  // namespace dgpe
