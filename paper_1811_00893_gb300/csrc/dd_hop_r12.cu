// Kernels of the domain-decomposed hopping term with two-row compressed
// links (LF = 1, FP32 / FP16), no clover term: explicit instantiation of
// dd_kernels.cuh.
#include "dd_kernels.cuh"

namespace wl {
template struct DDKernels<1, kClNone>;
}  // namespace wl
