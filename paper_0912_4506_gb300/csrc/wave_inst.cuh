// Instantiation helper of the pipelined (wavefront) kernel.
#pragma once

#include "launch.h"
#include "wave.cuh"

namespace jac {

template <class TR, int V, int WY, int NEMU, int MINB, int TMA>
constexpr size_t wave_smem_bytes() {
    return TMA ? WaveTma<typename TR::S, V, WY>::bytes() : 0;
}

template <class TR, int V, int WY, int NEMU, int MINB, int TMA>
cudaError_t wave_launch(const WaveArgs& a, const CUtensorMap& map_src,
                        const CUtensorMap& map_ring, int ctas, cudaStream_t st) {
    constexpr size_t smem = wave_smem_bytes<TR, V, WY, NEMU, MINB, TMA>();
    wave_kernel<TR, V, WY, NEMU, MINB, TMA><<<ctas, dim3(32, WY + 1), smem, st>>>(a, map_src,
                                                                                 map_ring);
    return cudaGetLastError();
}

}  // namespace jac

// MINB: resident CTAs per SM the register allocation must allow; TMA: 1 for the
// TMA-staged march
#define JAC_WAVE(TR, V, WY, NEMU, MINB, TMA)                                            \
    {TR::kDtype, V, WY, NEMU, TMA, ::jac::wave_smem_bytes<TR, V, WY, NEMU, MINB, TMA>(), \
     &::jac::wave_launch<TR, V, WY, NEMU, MINB, TMA>,                                    \
     reinterpret_cast<const void*>(&::jac::wave_kernel<TR, V, WY, NEMU, MINB, TMA>)}
