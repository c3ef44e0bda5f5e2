// Batched Jacobi (host side): many independent grids of different shapes, each with its own
// sweep count and temporal-blocking depth, in one persistent launch.
//
// The host flattens every grid's passes into work items (grid, pass, tile),
// ordered by pass round, so an item only ever depends on items that come
// earlier in the queue: the tiles of the same grid's previous pass.  The
// persistent CTAs pull items from a global counter; before a tile of pass p of
// grid g starts, its CTA waits (bounded) until the per-grid completion counter
// says every tile of passes < p is done, and after finishing it publishes its
// own completion (release / acquire on the counter, then a proxy fence so the
// TMA loads of the next pass see the generic stores of the previous one).  Any
// item that has been taken is held by a running CTA, so the waits always end
// unless a producer is missing; then the bounded wait records a timeout in the
// status word and every CTA leaves.  The per-tile work is the same tb_tile
// routine as the single-grid kernel, dispatched on the item's depth.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/jacobi.h"
#include "batch_kernel.cuh"
#include "launch.h"
#include "plan.h"


using namespace jac;

struct jacobi_batch_s {
    int count = 0, dtype = 0, device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    std::vector<BatchGridDesc> host_desc;
    std::vector<int> final_b, t_used, passes, tile_x;
    int nitems = 0, ctas = 0;
    size_t smem = 0;
    BatchGridDesc* d_desc = nullptr;
    CUtensorMap* d_maps = nullptr;
    BatchItem* d_items = nullptr;
    int* d_counters = nullptr;  // done[count], head, status
    BatchArgs args{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
};

namespace {

// Tile geometry of a pass of depth t; the k-chunk count keeps chunks >= 8t planes
// (many grids share the GPU, so no grid needs whole waves of its own).
BatchPassGeom pass_geom(const Geom& g, int dtype, int t, int v, int nchunk_req) {
    const int nchunk = nchunk_req > 0 ? nchunk_req : std::max(1, g.nz / std::max(8 * t, 32));
    const TileGeom tg = tile_geom(dtype, g, v, kBatchNW, t, 1, nchunk);
    BatchPassGeom p{};
    p.t = t;
    p.v = v;
    p.ox = tg.ox;
    p.x0_first = tg.x0_first;
    p.ntx = tg.ntx;
    p.nty = tg.nty;
    p.kz = tg.kz;
    p.nchunk = tg.nchunk;
    return p;
}

const void* batch_kernel_ptr(int dtype) {
    return dtype == JAC_F32 ? batch_kernel_f32() : batch_kernel_bf16();
}

cudaError_t launch_batch(const jacobi_batch_s* b, cudaStream_t st) {
    return b->dtype == JAC_F32 ? launch_batch_f32(b->args, b->ctas, b->smem, st)
                               : launch_batch_bf16(b->args, b->ctas, b->smem, st);
}

void free_batch(jacobi_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_desc);
    cudaFree(b->d_maps);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    delete b;
}

// Enqueue one run: reset the counters, then the persistent kernel.
cudaError_t enqueue_run(jacobi_batch_s* b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * (b->count + 2), st);
    if (e != cudaSuccess) return e;
    return launch_batch(b, st);
}

}  // namespace

extern "C" {

int jacobi_batch_create(jacobi_batch_t* out, int count, const int* dims,
                        const long long* pitches, void* const* grids_a, void* const* grids_b,
                        const int* nsweeps, const int* t, const int* tile_x, const int* nchunk,
                        int dtype,
                        void* stream, int flags, double wait_limit_s) {
    if (!out) return JAC_EINVAL;
    *out = nullptr;
    if (count < 1 || !dims || !pitches || !grids_a || !grids_b || !nsweeps) return JAC_EINVAL;
    if (dtype != JAC_F32 && dtype != JAC_BF16) return JAC_EUNSUPPORTED;
    if (flags & ~(JAC_BATCH_NO_GRAPH | JAC_BATCH_TEST_MISSING_PRODUCER)) return JAC_EINVAL;
    const int es = elem_size(dtype);
    jacobi_batch_s* b = new (std::nothrow) jacobi_batch_s();
    if (!b) return JAC_ENOMEM;
    b->count = count;
    b->dtype = dtype;
    b->stream = static_cast<cudaStream_t>(stream);
    b->use_graph = !(flags & JAC_BATCH_NO_GRAPH);
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) !=
            cudaSuccess) {
        delete b;
        return JAC_ECUDA;
    }
    std::vector<BatchItem> items;
    std::vector<CUtensorMap> maps(2 * count);
    b->host_desc.resize(count);
    b->final_b.resize(count);
    b->t_used.resize(count);
    b->passes.resize(count);
    b->tile_x.resize(count);
    int max_pass = 0;
    for (int i = 0; i < count; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        const long long px = pitches[i];
        if (nx < 1 || ny < 1 || nz < 1 || px < nx + 2 || (px * es) % 16 || nsweeps[i] < 0 ||
            !grids_a[i] || !grids_b[i] || grids_a[i] == grids_b[i] ||
            (reinterpret_cast<uintptr_t>(grids_a[i]) & 15) ||
            (reinterpret_cast<uintptr_t>(grids_b[i]) & 15)) {
            delete b;
            return JAC_EINVAL;
        }
        Geom g{nx, ny, nz, px, px * (ny + 2)};
        if (t && t[i] > kBatchTMax) {
            delete b;
            return JAC_EUNSUPPORTED;  // deeper than the batched kernel's deepest depth
        }
        int ti = (t && t[i] > 0) ? t[i] : 4;
        ti = std::min(ti, std::max(1, nsweeps[i]));
        // tile width: the caller's (64 or 128), else 128 where the depth allows it
        const int tx = (tile_x && tile_x[i] > 0) ? tile_x[i] : (ti <= kBatchTMaxWide ? 128 : 64);
        if ((tx != 64 && tx != 128) || (tx == 128 && ti > kBatchTMaxWide)) {
            delete b;
            return JAC_EUNSUPPORTED;  // no kernel for this tile width and depth
        }
        const int vi = tx / 32;
        const int nc = nchunk ? nchunk[i] : 0;
        BatchGridDesc& d = b->host_desc[i];
        d.g = g;
        d.a = grids_a[i];
        d.b = grids_b[i];
        const int n = nsweeps[i];
        d.npass = (n + ti - 1) / ti;
        const int rem = n - (d.npass - 1) * ti;
        d.full = pass_geom(g, dtype, ti, vi, nc);
        d.last = pass_geom(g, dtype, n > 0 ? rem : ti, vi, nc);
        b->final_b[i] = d.npass & 1;
        b->t_used[i] = ti;
        b->tile_x[i] = tx;
        b->passes[i] = d.npass;
        max_pass = std::max(max_pass, d.npass);
        if (!encode_grid_map(&maps[2 * i], dtype, g, grids_a[i], tx, kBatchNW) ||
            !encode_grid_map(&maps[2 * i + 1], dtype, g, grids_b[i], tx, kBatchNW)) {
            delete b;
            return JAC_ECUDA;
        }
    }
    // work items by pass round; inside a round, bigger grids first
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        const Geom& gx = b->host_desc[x].g;
        const Geom& gy = b->host_desc[y].g;
        return (long long)gx.nx * gx.ny * gx.nz > (long long)gy.nx * gy.ny * gy.nz;
    });
    std::vector<int> done_before(count, 0);
    for (int p = 0; p < max_pass; ++p)
        for (int i : order) {
            const BatchGridDesc& d = b->host_desc[i];
            if (p >= d.npass) continue;
            const BatchPassGeom& pg = (p == d.npass - 1) ? d.last : d.full;
            const int tiles = pg.ntx * pg.nty * pg.nchunk;
            for (int k = 0; k < tiles; ++k) items.push_back({i, p, k, done_before[i]});
            done_before[i] += tiles;
        }
    if (flags & JAC_BATCH_TEST_MISSING_PRODUCER) {
        // test hook: one extra item waiting for a tile that no item produces
        items.push_back({0, b->host_desc[0].npass, 0, done_before[0] + 1});
    }
    b->nitems = (int)items.size();

    const void* kern = batch_kernel_ptr(dtype);
    // shared memory: the larger of the two tile families' deepest layouts
    b->smem = (dtype == JAC_F32)
                  ? std::max(TBLayout<2, kBatchNW, kBatchTMax, kRing, float>::bytes(),
                             TBLayout<4, kBatchNW, kBatchTMaxWide, kRing, float>::bytes())
                  : std::max(TBLayout<2, kBatchNW, kBatchTMax, kRing, uint16_t>::bytes(),
                             TBLayout<4, kBatchNW, kBatchTMaxWide, kRing, uint16_t>::bytes());
    int occ = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBatchNW * 32, b->smem) !=
            cudaSuccess) {
        delete b;
        return JAC_ECUDA;
    }
    b->ctas = std::max(1, occ) * b->num_sms;

    const size_t bytes_desc = sizeof(BatchGridDesc) * count;
    const size_t bytes_maps = sizeof(CUtensorMap) * 2 * count;
    const size_t bytes_items = sizeof(BatchItem) * std::max(1, b->nitems);
    if (cudaMalloc(&b->d_desc, bytes_desc) != cudaSuccess ||
        cudaMalloc(&b->d_maps, bytes_maps) != cudaSuccess ||
        cudaMalloc(&b->d_items, bytes_items) != cudaSuccess ||
        cudaMalloc(&b->d_counters, sizeof(int) * (count + 2)) != cudaSuccess) {
        free_batch(b);
        return JAC_ENOMEM;
    }
    if (cudaMemcpy(b->d_desc, b->host_desc.data(), bytes_desc, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_maps, maps.data(), bytes_maps, cudaMemcpyHostToDevice) != cudaSuccess ||
        (b->nitems &&
         cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * b->nitems,
                    cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemset(b->d_counters, 0, sizeof(int) * (count + 2)) != cudaSuccess) {
        free_batch(b);
        return JAC_ECUDA;
    }
    b->args.items = b->d_items;
    b->args.nitems = b->nitems;
    b->args.grids = b->d_desc;
    b->args.maps = b->d_maps;
    b->args.done = b->d_counters;
    b->args.head = b->d_counters + count;
    b->args.status = b->d_counters + count + 1;
    b->args.wait_ns = (unsigned long long)((wait_limit_s > 0 ? wait_limit_s : 2.0) * 1e9);

    // the B grids need A's boundary layer
    for (int i = 0; i < count; ++i)
        if (launch_boundary_copy(dtype, grids_a[i], grids_b[i], b->host_desc[i].g, b->stream) !=
            cudaSuccess) {
            free_batch(b);
            return JAC_ECUDA;
        }

    if (b->use_graph) {
        // record reset + persistent kernel into a graph (captured on a private stream)
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            free_batch(b);
            return JAC_ECUDA;
        }
        bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaError_t e1 = cudaMemsetAsync(b->d_counters + count, 0, 2 * sizeof(int), cap);
            cudaError_t e2 = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * count, cap);
            cudaError_t e3 = launch_batch(b, cap);
            ok = cudaStreamEndCapture(cap, &b->graph) == cudaSuccess && e1 == cudaSuccess &&
                 e2 == cudaSuccess && e3 == cudaSuccess;
        }
        cudaStreamDestroy(cap);
        if (!ok || cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
            free_batch(b);
            return JAC_ECUDA;
        }
    }
    *out = b;
    return JAC_OK;
}

int jacobi_batch_run(jacobi_batch_t b, int* final_is_b) {
    if (!b) return JAC_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) return JAC_ECUDA;
    cudaError_t e = b->use_graph ? cudaGraphLaunch(b->exec, b->stream) : enqueue_run(b, b->stream);
    if (e != cudaSuccess) return JAC_ECUDA;
    if (final_is_b)
        for (int i = 0; i < b->count; ++i) final_is_b[i] = b->final_b[i];
    return JAC_OK;
}

int jacobi_batch_info(jacobi_batch_t b, int* t_used, int* tile_x, int* passes, int* items,
                      int* ctas) {
    if (!b) return JAC_EINVAL;
    for (int i = 0; i < b->count; ++i) {
        if (t_used) t_used[i] = b->t_used[i];
        if (tile_x) tile_x[i] = b->tile_x[i];
        if (passes) passes[i] = b->passes[i];
    }
    if (items) *items = b->nitems;
    if (ctas) *ctas = b->ctas;
    return JAC_OK;
}

int jacobi_batch_check(jacobi_batch_t b) {
    if (!b) return JAC_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) return JAC_ECUDA;
    int st = 0;
    if (cudaMemcpyAsync(&st, b->args.status, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return JAC_ECUDA;
    return st ? JAC_ETIMEOUT : JAC_OK;
}

int jacobi_batch_destroy(jacobi_batch_t b) {
    if (!b) return JAC_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return JAC_OK;
}

}  // extern "C"
