// Instantiation helper of the pipelined (wavefront) kernel.
#pragma once

#include "launch.h"
#include "wave.cuh"

namespace jac {

template <class TR, int V, int WY, int NEMU, int MINB>
cudaError_t wave_launch(const WaveArgs& a, int ctas, cudaStream_t st) {
    wave_kernel<TR, V, WY, NEMU, MINB><<<ctas, dim3(32, WY + 1), 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace jac

// MINB: resident CTAs per SM the register allocation must allow
#define JAC_WAVE(TR, V, WY, NEMU, MINB)                                          \
    {TR::kDtype, V, WY, NEMU, &::jac::wave_launch<TR, V, WY, NEMU, MINB>,       \
     reinterpret_cast<const void*>(&::jac::wave_kernel<TR, V, WY, NEMU, MINB>)}
