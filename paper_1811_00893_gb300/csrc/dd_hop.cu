// Kernels of the domain-decomposed hopping term with full links (LF = 0) and
// no clover term, and the face-packing launcher: explicit instantiation of
// dd_kernels.cuh, compiled apart from the other families.
#include "dd_kernels.cuh"

namespace wl {

template struct DDKernels<0, kClNone>;

void dd_pack(int prec, bool dagger, const DDPackArgs& A, dim3 grid, cudaStream_t s)
{
    auto go = [&](auto pc) {
        constexpr int PP = decltype(pc)::value;
        if (dagger) dd_pack_kernel<PP, true><<<grid, kDDBlock, 0, s>>>(A);
        else dd_pack_kernel<PP, false><<<grid, kDDBlock, 0, s>>>(A);
    };
    if (prec == WL_F32) go(std::integral_constant<int, WL_F32>());
    else if (prec == WL_F16) go(std::integral_constant<int, WL_F16>());
    else if (prec == WL_F64) go(std::integral_constant<int, WL_F64>());
    else go(std::integral_constant<int, WL_DF64>());
}

}  // namespace wl
