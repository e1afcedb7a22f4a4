// Instantiation of the hopping kernels on compressed links (LF = 1: two
// rows of each SU(3) matrix stored, the third rebuilt in the kernel; FP32 and
// FP16), without the clover term.  The kernels are in hop_kernels.cuh.
#include "hop_kernels.cuh"

namespace wl {

template struct HopKernels<kClNone, 1>;

}  // namespace wl
