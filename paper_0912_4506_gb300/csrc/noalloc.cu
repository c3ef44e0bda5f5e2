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
#include "tb.cuh"

namespace {

using namespace jac;

constexpr size_t kStatusBytes = 256;  // first 256 bytes: the status word
constexpr size_t kScratchBytes = JAC_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

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

int esize(int dtype) { return dtype == JAC_F64 ? 8 : dtype == JAC_F32 ? 4 : 2; }

int fdiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool encode(CUtensorMap* map, int dtype, const Geom& g, void* base, int bx, int by) {
    auto fn = encoder();
    if (!fn) return false;
    const int es = esize(dtype);
    const CUtensorMapDataType dt = dtype == JAC_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : dtype == JAC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                      : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx + 2, (cuuint64_t)g.ny + 2, (cuuint64_t)g.nz + 2};
    cuuint64_t strides[2] = {(cuuint64_t)g.px * es, (cuuint64_t)g.plane * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Geometry of one blocked pass (same tiling rules as the handle-based planner).
struct Pass {
    const TBEntry* e;
    int ox, oy, x0_first, ntx, nty, kz, nchunk;
};

bool pass_geometry(const TBEntry* e, const Geom& g, int dtype, int sms, Pass* p) {
    const int A = 16 / esize(dtype);
    const int EX = 32 * e->V, EY = e->NW, T = e->T;
    p->e = e;
    p->ox = ((EX - 2 * T) / A) * A;
    p->oy = EY - 2 * T;
    if (p->ox < A || p->oy < 1) return false;
    p->x0_first = fdiv(1 - T, A) * A;
    p->ntx = (g.nx + 1 - (p->x0_first + T) + p->ox - 1) / p->ox;
    p->nty = (g.ny + p->oy - 1) / p->oy;
    int occ = 1;
    cudaFuncSetAttribute(e->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e->kernel, e->NW * 32, e->smem);
    if (occ < 1) occ = 1;
    const long long tiles = (long long)p->ntx * p->nty, slots = (long long)sms * occ;
    int best = 1;
    double best_score = -1.0;
    const int max_chunks = g.nz / ((4 * T > 8) ? 4 * T : 8);
    for (int c = 1; c <= (max_chunks > 1 ? max_chunks : 1); ++c) {
        const int kz = (g.nz + c - 1) / c;
        const long long ctas = tiles * ((g.nz + kz - 1) / kz);
        const long long waves = (ctas + slots - 1) / slots;
        const double score = (double)ctas / (double)(waves * slots) * kz / (double)(kz + 2 * T);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = c;
        }
    }
    p->kz = (g.nz + best - 1) / best;
    p->nchunk = (g.nz + p->kz - 1) / p->kz;
    return true;
}

const TBEntry* entry_for(int dtype, int T) {
    int n = 0;
    const TBEntry* tab = dtype == JAC_F64   ? tb_entries_f64(&n)
                         : dtype == JAC_F32 ? tb_entries_f32(&n)
                                            : tb_entries_bf16(&n);
    for (int i = 0; i < n; ++i)
        if (tab[i].mode == MODE_PLAIN && tab[i].T == T) return &tab[i];
    return nullptr;
}

// Deepest feasible depth <= want (0 if none).
int depth_at_most(int dtype, const Geom& g, int want) {
    for (int d = want; d >= 1; --d) {
        const TBEntry* e = entry_for(dtype, d);
        if (!e) continue;
        const int A = 16 / esize(dtype);
        if (((32 * e->V - 2 * d) / A) * A >= A && e->NW - 2 * d >= 1) return d;
    }
    return 0;
}

}  // namespace

extern "C" int jacobi_sweep_noalloc(int nx, int ny, int nz, int dtype, void* grid,
                                    long long row_pitch, int nsweeps, int t, void* stream,
                                    int sync) {
    if (nx < 1 || ny < 1 || nz < 1 || dtype < JAC_F64 || dtype > JAC_BF16) return JAC_EINVAL;
    if (nsweeps < 0 || t < 0 || !grid || (reinterpret_cast<uintptr_t>(grid) & 15u))
        return JAC_EINVAL;
    const int es = esize(dtype);
    if (row_pitch < nx + 2 || (row_pitch * es) % 16 != 0) return JAC_EINVAL;
    const unsigned long long bytes =
        (unsigned long long)row_pitch * (ny + 2) * (unsigned long long)(nz + 2) * es;
    if (bytes > kScratchBytes - kStatusBytes) return JAC_EINVAL;  // too large for the scratch

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return JAC_ECUDA;
    unsigned char* scratch = nullptr;
    int rc = scratch_address(device, &scratch);
    if (rc != JAC_OK) return rc;
    int* status = reinterpret_cast<int*>(scratch);
    void* other = scratch + kStatusBytes;

    Geom g{nx, ny, nz, row_pitch, row_pitch * (ny + 2)};
    // what must start fresh: the status word and the scratch grid's boundary layer
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess ||
        launch_boundary_copy(dtype, grid, other, g, st) != cudaSuccess)
        return JAC_ECUDA;

    if (t == 0) t = (dtype == JAC_F64) ? 1 : 4;
    int cur_other = 0;  // 0: current data in the caller's grid
    if (t == 1) {
        const PlainEntry* pe = dtype == JAC_F64   ? plain_entry_f64()
                               : dtype == JAC_F32 ? plain_entry_f32()
                                                  : plain_entry_bf16();
        const bool aligned_x1 = pe->V == 1 || dtype == JAC_F64;
        const int nvec = aligned_x1 ? (nx + pe->V - 1) / pe->V : nx / pe->V + 1;
        dim3 grid3((nvec + 31) / 32, (ny + pe->WY - 1) / pe->WY, 1);
        int kchunk = nz;
        for (int s = 0; s < nsweeps; ++s) {
            const void* src = cur_other ? other : grid;
            void* dst = cur_other ? grid : other;
            if (pe->launch(src, dst, g, kchunk, grid3, nullptr, st) != cudaSuccess) return JAC_ECUDA;
            cur_other ^= 1;
        }
    } else {
        const int tmax = depth_at_most(dtype, g, t);
        if (tmax == 0) return JAC_EUNSUPPORTED;
        int left = nsweeps;
        int box_x = 0, box_y = 0;
        CUtensorMap map_grid, map_other;
        while (left > 0) {
            const int d = depth_at_most(dtype, g, left < tmax ? left : tmax);
            Pass p;
            if (d == 0 || !pass_geometry(entry_for(dtype, d), g, dtype, sms, &p))
                return JAC_EUNSUPPORTED;
            const int EX = 32 * p.e->V, EY = p.e->NW;
            if (EX != box_x || EY != box_y) {
                if (!encode(&map_grid, dtype, g, grid, EX, EY) ||
                    !encode(&map_other, dtype, g, other, EX, EY))
                    return JAC_ECUDA;
                box_x = EX;
                box_y = EY;
            }
            TBArgs a;
            a.g = g;
            a.dst = cur_other ? grid : other;
            a.grad = nullptr;
            a.ox = p.ox;
            a.x0_first = p.x0_first;
            a.kz = p.kz;
            a.status = status;
            const CUtensorMap& m = cur_other ? map_other : map_grid;
            if (p.e->launch(m, m, a, dim3(p.ntx, p.nty, p.nchunk), st) != cudaSuccess)
                return JAC_ECUDA;
            cur_other ^= 1;
            left -= d;
        }
    }
    if (cur_other) {  // result in the scratch grid: copy the rows back (not the padding)
        if (cudaMemcpy2DAsync(grid, (size_t)row_pitch * es, other, (size_t)row_pitch * es,
                              (size_t)(nx + 2) * es, (size_t)(ny + 2) * (nz + 2),
                              cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return JAC_ECUDA;
    }
    if (sync) {
        int h_status = 0;
        if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return JAC_ECUDA;
        if (h_status != 0) return JAC_ETIMEOUT;
    }
    return JAC_OK;
}
