// Kernels of the domain-decomposed hopping term with full links (LF = 0):
// explicit instantiation of dd_kernels.cuh, compiled apart from the
// compressed-link variant (dd_hop_r12.cu).
#include "dd_kernels.cuh"

namespace wl {
template struct DDKernels<0>;
}  // namespace wl
