// Instantiation of the hopping kernels with the clover term of Eq. 2 applied
// to the epilogue's result (out = C (x1 + b1 x2 + a H in): the A_oo^-1 H_oe
// half of the clover Schur operator and the x_o reconstruction).  The kernels
// are in hop_kernels.cuh.
#include "hop_kernels.cuh"

namespace wl {

template struct HopKernels<kClOut, 0>;

}  // namespace wl
