// Kernels of the domain-decomposed hopping term with the clover term of Eq. 2
// in the epilogue (both modes), two-row compressed links: explicit
// instantiation of dd_kernels.cuh.
#include "dd_kernels.cuh"

namespace wl {
template struct DDKernels<1, kClX2>;
template struct DDKernels<1, kClOut>;
}  // namespace wl
