// Double-float instantiation of the SSCN kernels: psi and the spectrum hold pairs of FP32
// numbers (hi + lo, about 48 significant bits) and every operation runs on the FP32 pipe.
#include "dgpe_device.cuh"

namespace dgpe {
const KernelSet *kernels_df64() { return Impl<df>::set(); }
}  // namespace dgpe
