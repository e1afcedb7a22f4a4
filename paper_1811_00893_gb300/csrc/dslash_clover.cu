// Instantiation of the hopping kernels with the clover term of Eq. 2 fused
// into their epilogue (the kernels are in hop_kernels.cuh; the Wilson ones
// are instantiated in dslash.cu).
#include "hop_kernels.cuh"

namespace wl {

template struct HopKernels<kClX2>;
template struct HopKernels<kClOut>;

}  // namespace wl
