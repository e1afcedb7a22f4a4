// Kernels of the domain-decomposed hopping term with the clover term of Eq. 2
// in the epilogue (both modes), full links: explicit instantiation of
// dd_kernels.cuh.
#include "dd_kernels.cuh"

namespace wl {
template struct DDKernels<0, kClX2>;
template struct DDKernels<0, kClOut>;
}  // namespace wl
