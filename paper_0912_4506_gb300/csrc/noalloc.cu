// jacobi_sweep_noalloc: the sweep for callers that cannot allocate device
// memory.  Everything the sweep needs beyond the caller's grid - the second
// ping-pong grid and the device status word - lives in one static device array
// in this file, so the call itself performs no allocation of any kind (no
// cudaMalloc/cudaFree, no allocating library routine, no host heap use).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/jacobi.h"
#include "launch.h"
#include "plan.h"
#include "tb.cuh"

namespace {

using namespace jac;

// the first 256 bytes hold the status word (int 0) and the FP64 range flag
// (int 16); the scratch grid starts after them
constexpr size_t kStatusBytes = 256;
constexpr size_t kScratchBytes = JAC_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code its name is only a host-side stand-in, not a
// device address: kernels get the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (with that device current).
int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return JAC_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return JAC_ECUDA;
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return JAC_OK;
}

}  // namespace

extern "C" int jacobi_sweep_noalloc(int nx, int ny, int nz, int dtype, void* grid,
                                    long long row_pitch, int nsweeps, int t, void* stream,
                                    int sync) {
    if (nx < 1 || ny < 1 || nz < 1 || dtype < JAC_F64 || dtype > JAC_BF16) return JAC_EINVAL;
    if (nsweeps < 0 || t < 0 || !grid || (reinterpret_cast<uintptr_t>(grid) & 15u))
        return JAC_EINVAL;
    const int es = elem_size(dtype);
    if (row_pitch < nx + 2 || (row_pitch * es) % 16 != 0) return JAC_EINVAL;
    const unsigned long long bytes =
        (unsigned long long)row_pitch * (ny + 2) * (unsigned long long)(nz + 2) * es;
    if (bytes > kScratchBytes - kStatusBytes) return JAC_EINVAL;  // too large for the scratch

    // the same plan as jacobi_sweep with the same arguments
    if (t == 0) t = default_t(dtype, MODE_PLAIN);
    const bool plain = (t == 1 && dtype == JAC_F64);
    DepthPlan dp{};
    if (!plain) {
        const int rc = plan_depths(dtype, MODE_PLAIN, nsweeps, t, &dp);
        if (rc != JAC_OK) return rc;
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return JAC_ECUDA;
    unsigned char* scratch = nullptr;
    int rc = scratch_address(device, &scratch);
    if (rc != JAC_OK) return rc;
    int* status = reinterpret_cast<int*>(scratch);  // sticky until a sync call reads it
    int* range_flag = status + 16;
    void* other = scratch + kStatusBytes;

    Geom g{nx, ny, nz, row_pitch, row_pitch * (ny + 2)};
    // what must start fresh: the scratch grid's boundary layer
    if (launch_boundary_copy(dtype, grid, other, g, st) != cudaSuccess) return JAC_ECUDA;

    int cur_other = 0;  // 0: current data in the caller's grid
    if (plain) {
        const PlainEntry* pe = plain_for(dtype);
        dim3 grid3;
        int kchunk = 0;
        plain_grid(pe, dtype, g, device, sms, &grid3, &kchunk);
        const int* fast = nullptr;
        if (pe->nemu > 0 && nsweeps > 0) {
            fast = range_flag;
            if (launch_range_check(static_cast<const double*>(grid), g, range_flag, st) !=
                cudaSuccess)
                return JAC_ECUDA;
        }
        for (int s = 0; s < nsweeps; ++s) {
            const void* src = cur_other ? other : grid;
            void* dst = cur_other ? grid : other;
            if (pe->launch(src, dst, g, kchunk, grid3, fast, st) != cudaSuccess) return JAC_ECUDA;
            cur_other ^= 1;
        }
    } else if (dp.passes() > 0) {
        const int* fast = nullptr;
        if (dtype == JAC_F64) {
            const TBEntry* e0 = tb_entry(dtype, MODE_PLAIN, dp.t_full);
            const TBEntry* e1 = dp.t_last > 0 ? tb_entry(dtype, MODE_PLAIN, dp.t_last) : nullptr;
            if ((e0 && e0->emu > 0) || (e1 && e1->emu > 0)) {
                fast = range_flag;
                if (launch_range_check(static_cast<const double*>(grid), g, range_flag, st) !=
                    cudaSuccess)
                    return JAC_ECUDA;
            }
        }
        int box_x = 0, box_y = 0;
        CUtensorMap map_grid, map_other;
        for (int p = 0; p < dp.passes(); ++p) {
            const TBEntry* e = tb_entry(dtype, MODE_PLAIN, dp.depth(p));
            if (!e) return JAC_EUNSUPPORTED;
            const TileGeom gm = tile_geom(dtype, g, e->V, e->NW, e->T,
                                          (long long)sms * tb_occupancy(*e, device), 0);
            if (!gm.ok) return JAC_EUNSUPPORTED;
            const int EX = 32 * e->V, EY = e->NW;
            if (EX != box_x || EY != box_y) {
                if (!encode_grid_map(&map_grid, dtype, g, grid, EX, EY) ||
                    !encode_grid_map(&map_other, dtype, g, other, EX, EY))
                    return JAC_ECUDA;
                box_x = EX;
                box_y = EY;
            }
            TBArgs a;
            a.g = g;
            a.dst = cur_other ? grid : other;
            a.grad = nullptr;
            a.ox = gm.ox;
            a.x0_first = gm.x0_first;
            a.kz = gm.kz;
            a.status = status;
            a.fast = fast;
            a.one = 1u;
            const CUtensorMap& m = cur_other ? map_other : map_grid;
            if (e->launch(m, m, a, dim3(gm.ntx, gm.nty, gm.nchunk), st) != cudaSuccess)
                return JAC_ECUDA;
            cur_other ^= 1;
        }
    }
    if (cur_other) {  // result in the scratch grid: copy the rows back (not the padding)
        if (cudaMemcpy2DAsync(grid, (size_t)row_pitch * es, other, (size_t)row_pitch * es,
                              (size_t)(nx + 2) * es, (size_t)(ny + 2) * (nz + 2),
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return JAC_ECUDA;
    }
    if (sync) {
        // the status word is sticky: a timeout of an earlier call made with sync = 0
        // is reported here, and the word is cleared once it has been read
        int h_status = 0;
        if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return JAC_ECUDA;
        if (h_status != 0) {
            if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return JAC_ECUDA;
            return JAC_ETIMEOUT;
        }
    }
    return JAC_OK;
}
