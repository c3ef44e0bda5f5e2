// Host-side registry of the compiled kernels, shared by the translation units of
// the library (one per dtype/mode group, compiled in parallel) and the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace jac {

struct TBArgs;

// map: the grid read by the pass; map_rho: the right-hand side (correction
// sweeps; any valid map otherwise)
using TBLaunchFn = cudaError_t (*)(const CUtensorMap& map, const CUtensorMap& map_rho,
                                   const TBArgs& a, dim3 grid, cudaStream_t st);

// One instantiation of the temporally-blocked kernel.
struct TBEntry {
    int dtype;      // 0 f64, 1 f32, 2 bf16
    int mode;       // MODE_PLAIN, MODE_RHS, MODE_ADJ
    int V;          // x cells per lane (extended tile width 32*V)
    int NW;         // warps = rows of the extended tile
    int T;          // temporal-blocking depth
    int NS;         // TMA ring slots
    size_t smem;    // dynamic shared memory bytes
    int emu;        // FP64: additions on the integer pipes when the range check passes
    TBLaunchFn launch;
    const void* kernel;
};

using PlainLaunchFn = cudaError_t (*)(const void* A, void* B, const Geom& g, int kchunk,
                                      dim3 grid, const int* fast, cudaStream_t st);

struct PlainEntry {
    int dtype;
    int V;     // cells per lane
    int WY;    // warps (rows) per CTA
    int nemu;  // additions done on the integer pipes when `fast` is set (FP64)
    PlainLaunchFn launch;
    const void* kernel;
};

struct WaveArgs;
// map_src: the source grid, map_ring: the rings (TMA-staged entries only)
using WaveLaunchFn = cudaError_t (*)(const WaveArgs& a, const CUtensorMap& map_src,
                                     const CUtensorMap& map_ring, int ctas, cudaStream_t st);

// One instantiation of the pipelined (wavefront) kernel: tiles of 32*V x WY cells.
struct WaveEntry {
    int dtype;
    int V;
    int WY;
    int nemu;     // FP64: integer-pipe additions code (0: all on the FP64 unit)
    int tma;      // 1: planes staged in shared memory by TMA (boxes of 32V + 2*16B x WY+2)
    size_t smem;  // dynamic shared memory bytes
    WaveLaunchFn launch;
    const void* kernel;
};

// Tables provided by the per-dtype translation units.
const TBEntry* tb_entries_f64(int* n);
const TBEntry* tb_entries_f64_deep(int* n);
const TBEntry* tb_entries_f32(int* n);
const TBEntry* tb_entries_f32_rhs(int* n);
const TBEntry* tb_entries_bf16(int* n);
const TBEntry* tb_entries_bf16_rhs(int* n);
const PlainEntry* plain_entry_f64();
const PlainEntry* plain_entries_f64(int* n);  // all emulation variants
const PlainEntry* plain_entry_f32();
const PlainEntry* plain_entry_bf16();
const WaveEntry* wave_entries_f64(int* n);
const WaveEntry* wave_entries_f32(int* n);
const WaveEntry* wave_entries_bf16(int* n);

// Auxiliary kernels (aux.cu).
cudaError_t launch_boundary_copy(int dtype, const void* A, void* B, const Geom& g,
                                 cudaStream_t st);
cudaError_t launch_face_reduce(int dtype, void* grad, const Geom& g, const void* fbuf,
                               long long fstride, int nsweeps, cudaStream_t st);
// Face values of one adjoint pass of depth T (band.cu): FP64 or FP32, T in 1..8
// (cudaErrorInvalidValue otherwise).
cudaError_t launch_face_band(int dtype, const void* src, const Geom& g, void* fbuf,
                             long long fstride, int sweep0, int T, cudaStream_t st);
cudaError_t launch_range_check(const double* A, const Geom& g, int* flag, cudaStream_t st);
cudaError_t launch_residual(const double* u_in, double* u_out, const Geom& gu,
                            const void* e, void* rho, int lo_dtype, const Geom& glo,
                            cudaStream_t st);

}  // namespace jac
