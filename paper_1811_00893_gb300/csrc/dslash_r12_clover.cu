// Instantiation of the hopping kernels on compressed links (LF = 1) with the
// clover term of Eq. 2 in the epilogue.  The kernels are in hop_kernels.cuh.
#include "hop_kernels.cuh"

namespace wl {

template struct HopKernels<kClX2, 1>;
template struct HopKernels<kClOut, 1>;

}  // namespace wl
