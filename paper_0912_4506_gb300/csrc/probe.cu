// Pipe-rate probes: kernels that do nothing but one kind of arithmetic from
// registers, so that the roofline of the sweeps can be stated against measured
// per-GPU rates instead of nominal ones.  Each thread runs kChains independent
// dependency chains of `iters` operations; the chains' values are written out
// so the work cannot be removed.  Operations per launch:
// blocks * threads * iters * kChains.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/jacobi.h"
#include "emu.cuh"
#include "emusum.cuh"

namespace jac {

constexpr int kChains = JAC_PROBE_CHAINS;

__device__ __forceinline__ uint32_t lop3_96(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t r;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

template <int KIND>
__global__ void __launch_bounds__(256) pipe_probe_kernel(double* out, int iters, uint32_t seed) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if constexpr (KIND == JAC_PROBE_DADD) {
        double x[kChains];
        const double y = 1.0 + (double)(seed & 7) * 0x1p-40;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1.0 + (double)(tid + c) * 0x1p-30;
#pragma unroll 1
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __dadd_rn(x[c], y);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    } else if constexpr (KIND == JAC_PROBE_FADD) {
        float x[kChains];
        const float y = 1.0f + (float)(seed & 7) * 0x1p-20f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1.0f + (float)(tid + c) * 0x1p-20f;
#pragma unroll 1
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fadd_rn(x[c], y);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    } else if constexpr (KIND == JAC_PROBE_LOP3) {
        uint32_t x[kChains];
        const uint32_t y = seed * 2654435761u, z = seed ^ 0x9E3779B9u;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = tid * 747796405u + c;
#pragma unroll 1
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = lop3_96(x[c], y, z + c);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += (double)x[c];
    } else if constexpr (KIND == JAC_PROBE_IMAD) {
        uint32_t x[kChains];
        const uint32_t y = seed | 1u, z = seed ^ 0x9E3779B9u;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = tid * 747796405u + c;
#pragma unroll 1
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = mad_lo(x[c], y, z + c);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += (double)x[c];
    } else if constexpr (KIND == JAC_PROBE_ACC_ADD) {
        // the FP64 sweeps' unpacked running sum: additions of an operand whose
        // exponent is at most 9 below the sum's (reset into [1, 2) every 64)
        const emusum::Mul km = emusum::make_mul(seed);
        emusum::Words a[kChains];
        const emusum::UnpW y = emusum::unpack_w(0.75 + (double)(seed & 7) * 0x1p-40, km);
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            a[c] = emusum::first_w(emusum::unpack_w(1.0 + (double)(tid + c) * 0x1p-30, km), y, km);
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) emusum::add_w(a[c], y, km);
            if ((i & 63) == 63) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) a[c].e = 1023u;
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += emusum::pack_w(a[c], km) + (double)a[c].bad;
    } else {  // JAC_PROBE_EMU_ADD: the sweep's exact binary64 addition on integer pipes
        double x[kChains];
        // operands of similar magnitude, as in a sweep: the running sum doubles
        // its exponent only rarely, so reset it into [1, 2) every 64 additions
        const double y = 0.75 + (double)(seed & 7) * 0x1p-40;
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1.0 + (double)(tid + c) * 0x1p-30;
#pragma unroll 1
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = add_pos_exact_f(x[c], y, seed >> 31 | 1u);
            if ((i & 63) == 63) {
#pragma unroll
                for (int c = 0; c < kChains; ++c)
                    x[c] = __longlong_as_double((__double_as_longlong(x[c]) &
                                                 0x000FFFFFFFFFFFFFll) |
                                                0x3FF0000000000000ll);
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    }
    out[tid] = acc;
}

}  // namespace jac

extern "C" int jacobi_pipe_probe(int kind, double* out, int blocks, int threads, int iters,
                                 void* stream) {
    if (!out || blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 1)
        return JAC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t seed = 1u;  // a runtime 1 in the integer-pipe additions
    switch (kind) {
        case JAC_PROBE_DADD:
            jac::pipe_probe_kernel<JAC_PROBE_DADD><<<blocks, threads, 0, st>>>(out, iters, seed);
            break;
        case JAC_PROBE_FADD:
            jac::pipe_probe_kernel<JAC_PROBE_FADD><<<blocks, threads, 0, st>>>(out, iters, seed);
            break;
        case JAC_PROBE_LOP3:
            jac::pipe_probe_kernel<JAC_PROBE_LOP3><<<blocks, threads, 0, st>>>(out, iters, seed);
            break;
        case JAC_PROBE_IMAD:
            jac::pipe_probe_kernel<JAC_PROBE_IMAD><<<blocks, threads, 0, st>>>(out, iters, seed);
            break;
        case JAC_PROBE_ACC_ADD:
            jac::pipe_probe_kernel<JAC_PROBE_ACC_ADD><<<blocks, threads, 0, st>>>(out, iters,
                                                                                   seed);
            break;
        case JAC_PROBE_EMU_ADD:
            jac::pipe_probe_kernel<JAC_PROBE_EMU_ADD><<<blocks, threads, 0, st>>>(out, iters,
                                                                                   seed);
            break;
        default:
            return JAC_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? JAC_OK : JAC_ECUDA;
}
