// Instantiation helpers for the per-dtype translation units.
#pragma once

#include "launch.h"
#include "plain.cuh"
#include "tb.cuh"

namespace jac {

template <class TR, int V, int NW, int T, int MODE, int NS>
constexpr size_t tb_smem_bytes() {
    return TBLayout<V, NW, T, NS, typename TR::S, rho_slots<MODE, NS, T>()>::bytes();
}

template <class TR, int V, int NW, int T, int MODE, int NS, int EMU>
cudaError_t tb_launch(const CUtensorMap& map, const CUtensorMap& map_rho, const TBArgs& a,
                      dim3 grid, cudaStream_t st) {
    constexpr size_t smem = tb_smem_bytes<TR, V, NW, T, MODE, NS>();
    tb_sweep_kernel<TR, V, NW, T, MODE, NS, EMU><<<grid, NW * 32, smem, st>>>(map, map_rho, a);
    return cudaGetLastError();
}

template <class TR, int V, int WY, int NEMU>
cudaError_t plain_launch(const void* A, void* B, const Geom& g, int kchunk, dim3 grid,
                         const int* fast, cudaStream_t st) {
    using S = typename TR::S;
    if constexpr (NEMU >= 48)
        plain_sweep_kernel_capped<TR, V, WY, NEMU><<<grid, dim3(32, WY), 0, st>>>(
            static_cast<const S*>(A), static_cast<S*>(B), g, kchunk, fast, 1u);
    else
        plain_sweep_kernel<TR, V, WY, NEMU><<<grid, dim3(32, WY), 0, st>>>(
            static_cast<const S*>(A), static_cast<S*>(B), g, kchunk, fast, 1u);
    return cudaGetLastError();
}

template <class TR, int V, int WY, int NEMU>
const void* plain_kernel_ptr() {
    if constexpr (NEMU >= 48)
        return reinterpret_cast<const void*>(&plain_sweep_kernel_capped<TR, V, WY, NEMU>);
    else
        return reinterpret_cast<const void*>(&plain_sweep_kernel<TR, V, WY, NEMU>);
}

}  // namespace jac

#define JAC_TBE(TR, V, NW, T, MODE, NS, EMU)                                          \
    {TR::kDtype, MODE, V, NW, T, NS, ::jac::tb_smem_bytes<TR, V, NW, T, MODE, NS>(), EMU, \
     &::jac::tb_launch<TR, V, NW, T, MODE, NS, EMU>,                                \
     reinterpret_cast<const void*>(&::jac::tb_sweep_kernel<TR, V, NW, T, MODE, NS, EMU>)}

#define JAC_TB(TR, V, NW, T, MODE, NS) JAC_TBE(TR, V, NW, T, MODE, NS, 0)

#define JAC_PLAIN(TR, V, WY, NEMU) \
    {TR::kDtype, V, WY, NEMU, &::jac::plain_launch<TR, V, WY, NEMU>, \
     ::jac::plain_kernel_ptr<TR, V, WY, NEMU>()}

#define JAC_TABLE(NAME, ARR)                                  \
    const TBEntry* NAME(int* n) {                             \
        *n = (int)(sizeof(ARR) / sizeof(ARR[0]));             \
        return ARR;                                           \
    }
