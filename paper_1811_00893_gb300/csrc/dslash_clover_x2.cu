// Instantiation of the hopping kernels with the clover term of Eq. 2 applied
// to the x2 operand of the epilogue (out = x1 + b1 A x2 + a H in: the A_ee x
// term of the clover Schur operator and of D_clov).  The kernels are in
// hop_kernels.cuh; each clover mode has its own translation unit so that the
// library's units compile in parallel.
#include "hop_kernels.cuh"

namespace wl {

template struct HopKernels<kClX2, 0>;

}  // namespace wl
