// Device side of the batched Jacobi kernel (see batch.cu for the host side).
#pragma once

#include "tb.cuh"

namespace jac {

// Every CTA has 32 warps (one row each); a grid's tiles are 64 (V = 2, depths
// 1-6) or 128 (V = 4, depths 1-2) cells wide -- deeper 128-wide tiles need more
// registers than 1024-thread CTAs of this kernel have (they spill).
constexpr int kBatchNW = 32, kBatchTMax = 6, kBatchTMaxWide = 2;

struct BatchPassGeom {
    int t, v, ox, x0_first, ntx, nty, kz, nchunk;
};

struct BatchGridDesc {
    Geom g;
    void* a;
    void* b;
    int npass;
    BatchPassGeom full;  // passes 0 .. npass-2 (and the last one if it is full)
    BatchPassGeom last;  // the last pass
};

struct BatchItem {
    int g, pass, tile, wait;  // wait: completed tiles of grid g needed first
};

struct BatchArgs {
    const BatchItem* items;
    int nitems;
    const BatchGridDesc* grids;
    const CUtensorMap* maps;  // 2 per grid: source A (even passes), source B (odd)
    int* done;                // per grid: completed tiles
    int* head;                // next item
    int* status;
    unsigned long long wait_ns;
};

template <class Tr, int V, int T>
__device__ __forceinline__ void batch_tile(const CUtensorMap* map, const TBArgs& a, int bx,
                                           int by, int bz, unsigned char* smem, int* s_abort) {
    if (tile_inside_xy<V, kBatchNW, T>(a, bx, by))
        tb_tile<Tr, V, kBatchNW, T, MODE_PLAIN, true>(map, nullptr, a, bx, by, bz, smem, s_abort);
    else
        tb_tile<Tr, V, kBatchNW, T, MODE_PLAIN, false>(map, nullptr, a, bx, by, bz, smem,
                                                       s_abort);
}

template <class Tr>
__global__ void __launch_bounds__(kBatchNW * 32, 1) tb_batch_kernel(const BatchArgs ba) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int s_abort, s_item;
    const int tid = threadIdx.x;
    if (tid == 0) s_abort = 0;
#pragma unroll 1
    while (true) {
        if (tid == 0) s_item = atomicAdd(ba.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= ba.nitems || s_abort) break;
        const BatchItem item = ba.items[it];
        const BatchGridDesc& G = ba.grids[item.g];
        if (tid == 0) {
            // wait for the previous pass of this grid (bounded)
            if (ld_acquire(ba.done + item.g) < item.wait) {
                const uint64_t t0 = global_ns();
                while (ld_acquire(ba.done + item.g) < item.wait) {
                    if (global_ns() - t0 > ba.wait_ns) {
                        atomicOr(ba.status, kStatusTimeout);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(200);
                }
            }
            fence_proxy_async_global();
        }
        __syncthreads();
        if (s_abort) break;
        const bool is_last = item.pass == G.npass - 1;
        const BatchPassGeom& pg = is_last ? G.last : G.full;
        TBArgs a;
        a.g = G.g;
        a.dst = (item.pass & 1) ? G.a : G.b;
        a.grad = nullptr;
        a.ox = pg.ox;
        a.x0_first = pg.x0_first;
        a.kz = pg.kz;
        a.status = ba.status;
        a.fast = nullptr;
        a.one = 1u;
        const int bx = item.tile % pg.ntx;
        const int by = (item.tile / pg.ntx) % pg.nty;
        const int bz = item.tile / (pg.ntx * pg.nty);
        const CUtensorMap* map = ba.maps + 2 * item.g + (item.pass & 1);
        if (pg.v == 4) {
            switch (pg.t) {
                case 1: batch_tile<Tr, 4, 1>(map, a, bx, by, bz, smem, &s_abort); break;

                default: batch_tile<Tr, 4, 2>(map, a, bx, by, bz, smem, &s_abort); break;
            }
        } else {
            switch (pg.t) {
                case 1: batch_tile<Tr, 2, 1>(map, a, bx, by, bz, smem, &s_abort); break;
                case 2: batch_tile<Tr, 2, 2>(map, a, bx, by, bz, smem, &s_abort); break;
                case 3: batch_tile<Tr, 2, 3>(map, a, bx, by, bz, smem, &s_abort); break;
                case 4: batch_tile<Tr, 2, 4>(map, a, bx, by, bz, smem, &s_abort); break;
                case 5: batch_tile<Tr, 2, 5>(map, a, bx, by, bz, smem, &s_abort); break;
                default: batch_tile<Tr, 2, 6>(map, a, bx, by, bz, smem, &s_abort); break;
            }
        }
        // publish: every thread's stores of this tile are made visible at GPU
        // scope before the one release on the grid's completion counter
        __threadfence();
        __syncthreads();
        if (tid == 0 && !s_abort) atomicAdd(ba.done + item.g, 1);
    }
}

}  // namespace jac

namespace jac {
cudaError_t launch_batch_f32(const BatchArgs& a, int ctas, size_t smem, cudaStream_t st);
cudaError_t launch_batch_bf16(const BatchArgs& a, int ctas, size_t smem, cudaStream_t st);
const void* batch_kernel_f32();
const void* batch_kernel_bf16();
}  // namespace jac
