// Hopping kernels with eight-real links (LF = 2, FP32 single-RHS Wilson
// launches): explicit instantiation of hop_kernels.cuh, compiled apart.
#include "hop_kernels.cuh"

namespace wl {
template struct HopKernels<kClNone, 2>;
}  // namespace wl
