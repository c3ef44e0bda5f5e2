// C ABI of the Jacobi library (include/jacobi.h): argument checks, the launch
// planner, TMA descriptor set-up and the pass loop.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/jacobi.h"
#include "launch.h"
#include "tb.cuh"

using namespace jac;

namespace {
constexpr int kDefaultF64Emu = 6;  // half additions per plane (3 of 5)
}

struct jacobi_s {
    int dtype;
    Geom g;
    void* a;
    void* b;
    cudaStream_t stream;
    int device;
    int num_sms;
    int* status;          // device status word (owned); status[16]: FP64 range flag
    CUtensorMap map_a;    // TMA descriptors of A and B (box set per entry shape)
    CUtensorMap map_b;
    int map_box_x, map_box_y;
    CUtensorMap map_rho;  // right-hand side of the correction sweeps (last rho seen)
    const void* rho_ptr;
    int rho_box_x, rho_box_y;
};

namespace {

int elem_size(int dtype) { return dtype == JAC_F64 ? 8 : dtype == JAC_F32 ? 4 : 2; }

int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// 3D tensor map over the padded grid (nx+2, ny+2, nz+2) with a (bx, by, 1) box.
// Elements outside the padded grid (including the row padding) read as zero.
int make_map(CUtensorMap* map, const jacobi_s* h, void* base, int bx, int by) {
    auto fn = encode_fn();
    if (!fn) return JAC_ECUDA;
    const int es = elem_size(h->dtype);
    const CUtensorMapDataType dt = h->dtype == JAC_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : h->dtype == JAC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                         : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)h->g.nx + 2, (cuuint64_t)h->g.ny + 2,
                          (cuuint64_t)h->g.nz + 2};
    cuuint64_t strides[2] = {(cuuint64_t)h->g.px * es, (cuuint64_t)h->g.plane * es};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? JAC_OK : JAC_ECUDA;
}

const std::vector<TBEntry>& tb_table(int dtype, int mode) {
    static std::vector<TBEntry> tabs[3][3];
    static std::once_flag once;
    std::call_once(once, [] {
        auto add = [](const TBEntry* p, int n) {
            for (int i = 0; i < n; ++i) tabs[p[i].dtype][p[i].mode].push_back(p[i]);
        };
        int n;
        const TBEntry* p;
        p = tb_entries_f64(&n); add(p, n);
        p = tb_entries_f32(&n); add(p, n);
        p = tb_entries_f32_rhs(&n); add(p, n);
        p = tb_entries_f32_adj(&n); add(p, n);
        p = tb_entries_bf16(&n); add(p, n);
        p = tb_entries_bf16_rhs(&n); add(p, n);
        for (auto& d : tabs)
            for (auto& v : d)
                std::sort(v.begin(), v.end(),
                          [](const TBEntry& x, const TBEntry& y) { return x.T < y.T; });
    });
    return tabs[dtype][mode];
}

// Allow every kernel of a table its dynamic shared memory on the current device
// (needed before occupancy queries and launches; done once per device).
void ensure_attrs(const std::vector<TBEntry>& tab, int device) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& e : tab) {
        bool seen = false;
        for (const auto& d : done)
            if (d.first == e.kernel && d.second == device) seen = true;
        if (seen) continue;
        cudaFuncSetAttribute(e.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem);
        done.emplace_back(e.kernel, device);
    }
}

// Additions the FP64 plain sweep does on the integer pipes when the range check
// allows it, in half additions per plane (0..8); JACOBI_F64_EMU overrides.
int f64_emu_count() {
    static int n = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        n = kDefaultF64Emu;
        if (const char* e = getenv("JACOBI_F64_EMU")) {
            const int v = atoi(e);
            if (v >= 0 && v <= 8) n = v;
        }
    });
    return n;
}

const PlainEntry* plain_for(int dtype) {
    if (dtype == JAC_F64) {
        int n = 0;
        const PlainEntry* tab = plain_entries_f64(&n);
        const int want = f64_emu_count();
        for (int i = 0; i < n; ++i)
            if (tab[i].nemu == want) return &tab[i];
        return plain_entry_f64();
    }
    return dtype == JAC_F32 ? plain_entry_f32() : plain_entry_bf16();
}

// Geometry of one temporally-blocked pass for an entry.
struct TBGeom {
    int ox, oy, x0_first, ntx, nty, kz, nchunk;
    bool ok;
};

// Choose the number of k-chunks: enough CTAs to fill whole waves, but chunks
// long enough that the 2T-plane pipeline fill/drain of each chunk stays small.
int pick_chunks(int nz, int T, long long tiles, int slots) {
    int best = 1;
    double best_score = -1.0;
    const int max_chunks = std::max(1, nz / std::max(4 * T, 8));
    for (int c = 1; c <= max_chunks; ++c) {
        const int kz = (nz + c - 1) / c;
        const long long ctas = tiles * (long long)((nz + kz - 1) / kz);
        const long long waves = (ctas + slots - 1) / slots;
        const double fill = (double)ctas / (double)(waves * slots);
        const double zeff = (double)kz / (double)(kz + 2 * T);
        const double score = fill * zeff;
        if (score > best_score + 1e-9) {
            best_score = score;
            best = c;
        }
    }
    return best;
}

TBGeom tb_geom(const jacobi_s* h, const TBEntry& e) {
    TBGeom r{};
    const int A = 16 / elem_size(h->dtype);
    const int EX = 32 * e.V, EY = e.NW, T = e.T;
    r.ox = ((EX - 2 * T) / A) * A;
    r.oy = EY - 2 * T;
    r.ok = r.ox >= A && r.oy >= 1;
    if (!r.ok) return r;
    r.x0_first = floor_div(1 - T, A) * A;
    r.ntx = (h->g.nx + 1 - (r.x0_first + T) + r.ox - 1) / r.ox;
    r.nty = (h->g.ny + r.oy - 1) / r.oy;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.kernel, e.NW * 32, e.smem);
    occ = std::max(occ, 1);
    r.nchunk = pick_chunks(h->g.nz, T, (long long)r.ntx * r.nty, h->num_sms * occ);
    r.kz = (h->g.nz + r.nchunk - 1) / r.nchunk;
    r.nchunk = (h->g.nz + r.kz - 1) / r.kz;
    return r;
}

int plain_chunks(const jacobi_s* h, const PlainEntry* pe, dim3* grid, int* kchunk) {
    // interior-aligned kernels (V == 1, or FP64) start at x = 1; vector kernels at 0
    const bool aligned_x1 = pe->V == 1 || h->dtype == JAC_F64;
    const int nvec = aligned_x1 ? (h->g.nx + pe->V - 1) / pe->V : h->g.nx / pe->V + 1;
    grid->x = (nvec + 31) / 32;
    grid->y = (h->g.ny + pe->WY - 1) / pe->WY;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pe->kernel, 32 * pe->WY, 0);
    occ = std::max(occ, 1);
    const long long tiles = (long long)grid->x * grid->y;
    const int c = pick_chunks(h->g.nz, 1, tiles, h->num_sms * occ);
    *kchunk = (h->g.nz + c - 1) / c;
    grid->z = (h->g.nz + *kchunk - 1) / *kchunk;
    return JAC_OK;
}

// The pass depths for n sweeps at requested depth t with the available entries:
// full passes of the deepest depth <= t, the remainder split greedily.
bool split_passes(const std::vector<TBEntry>& tab, const jacobi_s* h, int n, int t,
                  std::vector<int>* depths) {
    std::vector<int> avail;
    for (const auto& e : tab)
        if (tb_geom(h, e).ok) avail.push_back(e.T);
    if (avail.empty()) return false;
    int tmax = 0;
    for (int d : avail)
        if (d <= t) tmax = std::max(tmax, d);
    if (tmax == 0) tmax = avail.front();
    int left = n;
    while (left > 0) {
        int d = 0;
        for (int a : avail)
            if (a <= std::min(left, tmax)) d = std::max(d, a);
        if (d == 0) return false;
        depths->push_back(d);
        left -= d;
    }
    return true;
}

const TBEntry* find_entry(const std::vector<TBEntry>& tab, int T) {
    for (const auto& e : tab)
        if (e.T == T) return &e;
    return nullptr;
}

int check_grid_args(int nx, int ny, int nz, int dtype, long long pitch) {
    if (nx < 1 || ny < 1 || nz < 1) return JAC_EINVAL;
    if (dtype < JAC_F64 || dtype > JAC_BF16) return JAC_EINVAL;
    if (pitch < nx + 2) return JAC_EINVAL;
    if ((pitch * elem_size(dtype)) % 16 != 0) return JAC_EINVAL;
    if ((long long)(ny + 2) * pitch * (nz + 2) > (1LL << 40)) return JAC_EINVAL;
    return JAC_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Depth used when the caller leaves it to the planner (t = 0), the fastest
// measured at 512^3 on GB300: FP64 is bound by the FP64 pipe, so blocking cannot
// help it (plain streaming kernel); plain FP32/bf16 sweeps peak at depth 3
// (128 x 32 tiles), FP32 correction sweeps at 4 (tied with 3), bf16 correction
// sweeps at 2, adjoint sweeps at 4.
int default_t(int dtype, int mode) {
    if (dtype == JAC_F64) return 1;
    if (mode == MODE_PLAIN) return 3;
    if (mode == MODE_RHS) return dtype == JAC_BF16 ? 2 : 4;
    return 4;
}

// Run nsweeps of `mode` as a sequence of passes.  kernel: JAC_KERNEL_*.
int run_passes(jacobi_s* h, int mode, int nsweeps, int t, int kernel, const void* rho,
               void* grad, int* final_is_b, jacobi_plan_info* info_only) {
    if (!h || nsweeps < 0 || t < 0) return JAC_EINVAL;
    if (kernel < JAC_KERNEL_AUTO || kernel > JAC_KERNEL_TB) return JAC_EINVAL;
    if (t == 0) t = default_t(h->dtype, mode);
    // depth 1: FP64 takes the register-march streaming kernel (FP64-pipe bound, with
    // the integer-pipe additions); FP32/bf16 take the TMA-ring kernel at depth 1
    // (128 x 12 tiles), which keeps more bytes in flight than the register march
    if (kernel == JAC_KERNEL_AUTO)
        kernel = (t == 1 && h->dtype == JAC_F64) ? JAC_KERNEL_PLAIN : JAC_KERNEL_TB;
    if (mode != MODE_PLAIN) kernel = JAC_KERNEL_TB;  // RHS/adjoint only exist blocked
    if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;

    if (kernel == JAC_KERNEL_PLAIN) {
        const PlainEntry* pe = plain_for(h->dtype);
        dim3 grid;
        int kchunk = 0;
        plain_chunks(h, pe, &grid, &kchunk);
        if (info_only) {
            std::memset(info_only, 0, sizeof(*info_only));
            info_only->kernel = JAC_KERNEL_PLAIN;
            info_only->emu_adds = pe->nemu;
            info_only->t = 1;
            info_only->passes = nsweeps;
            info_only->tile_x = 32 * pe->V;
            info_only->tile_y = pe->WY;
            info_only->ext_x = 32 * pe->V;
            info_only->ext_y = pe->WY;
            info_only->kchunk = kchunk;
            info_only->threads = 32 * pe->WY;
            info_only->grid_x = grid.x;
            info_only->grid_y = grid.y;
            info_only->grid_z = grid.z;
            return JAC_OK;
        }
        const int* fast = nullptr;
        if (pe->nemu > 0 && nsweeps > 0) {
            // the integer-pipe additions need every value positive and normal
            fast = h->status + 16;
            if (launch_range_check(static_cast<const double*>(h->a), h->g, h->status + 16,
                                   h->stream) != cudaSuccess)
                return JAC_ECUDA;
        }
        for (int s = 0; s < nsweeps; ++s) {
            const void* src = (s & 1) ? h->b : h->a;
            void* dst = (s & 1) ? h->a : h->b;
            if (pe->launch(src, dst, h->g, kchunk, grid, fast, h->stream) != cudaSuccess)
                return JAC_ECUDA;
        }
        if (final_is_b) *final_is_b = nsweeps & 1;
        return JAC_OK;
    }

    const auto& tab = tb_table(h->dtype, mode);
    if (tab.empty()) return JAC_EUNSUPPORTED;
    ensure_attrs(tab, h->device);
    std::vector<int> depths;
    if (nsweeps > 0 && !split_passes(tab, h, nsweeps, t, &depths)) return JAC_EUNSUPPORTED;

    if (info_only) {
        std::memset(info_only, 0, sizeof(*info_only));
        info_only->kernel = JAC_KERNEL_TB;
        info_only->passes = (int)depths.size();
        if (!depths.empty()) {
            const TBEntry* e = find_entry(tab, depths.front());
            const TBGeom gm = tb_geom(h, *e);
            info_only->t = depths.front();
            info_only->remainder_t = depths.back() != depths.front() ? depths.back() : 0;
            info_only->tile_x = gm.ox;
            info_only->tile_y = gm.oy;
            info_only->ext_x = 32 * e->V;
            info_only->ext_y = e->NW;
            info_only->kchunk = gm.kz;
            info_only->threads = e->NW * 32;
            info_only->smem_bytes = (int)e->smem;
            info_only->grid_x = gm.ntx;
            info_only->grid_y = gm.nty;
            info_only->grid_z = gm.nchunk;
        }
        return JAC_OK;
    }

    int cur_b = 0;  // 0: current data in A
    for (size_t p = 0; p < depths.size(); ++p) {
        const TBEntry* e = find_entry(tab, depths[p]);
        const TBGeom gm = tb_geom(h, *e);
        if (!gm.ok) return JAC_EUNSUPPORTED;
        const int EX = 32 * e->V, EY = e->NW;
        if (EX != h->map_box_x || EY != h->map_box_y) {
            if (make_map(&h->map_a, h, h->a, EX, EY) != JAC_OK) return JAC_ECUDA;
            if (make_map(&h->map_b, h, h->b, EX, EY) != JAC_OK) return JAC_ECUDA;
            h->map_box_x = EX;
            h->map_box_y = EY;
        }
        TBArgs args;
        args.g = h->g;
        args.dst = cur_b ? h->a : h->b;
        args.grad = grad;
        args.ox = gm.ox;
        args.x0_first = gm.x0_first;
        args.kz = gm.kz;
        args.status = h->status;
        if (mode == MODE_RHS &&
            (rho != h->rho_ptr || EX != h->rho_box_x || EY != h->rho_box_y)) {
            if (make_map(&h->map_rho, h, const_cast<void*>(rho), EX, EY) != JAC_OK)
                return JAC_ECUDA;
            h->rho_ptr = rho;
            h->rho_box_x = EX;
            h->rho_box_y = EY;
        }
        const CUtensorMap& map = cur_b ? h->map_b : h->map_a;
        const CUtensorMap& map_rho = mode == MODE_RHS ? h->map_rho : map;
        if (e->launch(map, map_rho, args, dim3(gm.ntx, gm.nty, gm.nchunk), h->stream) !=
            cudaSuccess)
            return JAC_ECUDA;
        cur_b ^= 1;
    }
    if (final_is_b) *final_is_b = cur_b;
    return JAC_OK;
}

}  // namespace

extern "C" {

int jacobi_create(jacobi_t* out, int nx, int ny, int nz, int dtype, void* grid_a, void* grid_b,
                  long long row_pitch, void* stream) {
    if (!out) return JAC_EINVAL;
    *out = nullptr;
    int rc = check_grid_args(nx, ny, nz, dtype, row_pitch);
    if (rc != JAC_OK) return rc;
    if (!grid_a || !grid_b || grid_a == grid_b || !aligned16(grid_a) || !aligned16(grid_b))
        return JAC_EINVAL;
    jacobi_s* h = new (std::nothrow) jacobi_s();
    if (!h) return JAC_ENOMEM;
    h->dtype = dtype;
    h->g.nx = nx;
    h->g.ny = ny;
    h->g.nz = nz;
    h->g.px = row_pitch;
    h->g.plane = row_pitch * (long long)(ny + 2);
    h->a = grid_a;
    h->b = grid_b;
    h->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess) {
        delete h;
        return JAC_ECUDA;
    }
    if (cudaMalloc(&h->status, 32 * sizeof(int)) != cudaSuccess) {
        delete h;
        return JAC_ENOMEM;
    }
    if (cudaMemsetAsync(h->status, 0, 32 * sizeof(int), h->stream) != cudaSuccess ||
        launch_boundary_copy(dtype, grid_a, grid_b, h->g, h->stream) != cudaSuccess) {
        cudaFree(h->status);
        delete h;
        return JAC_ECUDA;
    }
    *out = h;
    return JAC_OK;
}

int jacobi_sweep(jacobi_t h, int nsweeps, int t, int* final_is_b) {
    return run_passes(h, MODE_PLAIN, nsweeps, t, JAC_KERNEL_AUTO, nullptr, nullptr, final_is_b,
                      nullptr);
}

int jacobi_sweep_ex(jacobi_t h, int nsweeps, int t, int kernel, int* final_is_b) {
    return run_passes(h, MODE_PLAIN, nsweeps, t, kernel, nullptr, nullptr, final_is_b, nullptr);
}

int jacobi_plan(jacobi_t h, int nsweeps, int t, int kernel, jacobi_plan_info* info) {
    if (!info) return JAC_EINVAL;
    return run_passes(h, MODE_PLAIN, nsweeps, t, kernel, nullptr, nullptr, nullptr, info);
}

int jacobi_sweep_rhs(jacobi_t h, const void* rho, int nsweeps, int t, int* final_is_b) {
    if (!h || !rho || !aligned16(rho)) return JAC_EINVAL;
    if (h->dtype == JAC_F64) return JAC_EUNSUPPORTED;
    return run_passes(h, MODE_RHS, nsweeps, t, JAC_KERNEL_TB, rho, nullptr, final_is_b,
                      nullptr);
}

int jacobi_adjoint(jacobi_t h, void* grad_bdry, int nsweeps, int t, int* final_is_b) {
    if (!h || !grad_bdry || !aligned16(grad_bdry)) return JAC_EINVAL;
    if (h->dtype == JAC_BF16) return JAC_EUNSUPPORTED;
    if (grad_bdry == h->a || grad_bdry == h->b) return JAC_EINVAL;
    return run_passes(h, MODE_ADJ, nsweeps, t, JAC_KERNEL_TB, nullptr, grad_bdry, final_is_b,
                      nullptr);
}

int jacobi_residual_accumulate(int nx, int ny, int nz, const double* u_in, double* u_out,
                               long long u_pitch, const void* e, void* rho, int lo_dtype,
                               long long lo_pitch, void* stream) {
    if (check_grid_args(nx, ny, nz, JAC_F64, u_pitch) != JAC_OK) return JAC_EINVAL;
    if (check_grid_args(nx, ny, nz, lo_dtype, lo_pitch) != JAC_OK) return JAC_EINVAL;
    if (!u_in || !u_out || !e || !rho || u_in == u_out || e == rho) return JAC_EINVAL;
    if (!aligned16(u_in) || !aligned16(u_out) || !aligned16(e) || !aligned16(rho))
        return JAC_EINVAL;
    Geom gu{nx, ny, nz, u_pitch, u_pitch * (ny + 2)};
    Geom gl{nx, ny, nz, lo_pitch, lo_pitch * (ny + 2)};
    if (launch_residual(u_in, u_out, gu, e, rho, lo_dtype, gl,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return JAC_ECUDA;
    return JAC_OK;
}

static size_t grid_bytes(const jacobi_s* h) {
    return (size_t)h->g.plane * (size_t)(h->g.nz + 2) * (size_t)elem_size(h->dtype);
}

int jacobi_upload(jacobi_t h, const void* host) {
    if (!h || !host) return JAC_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;
    if (cudaMemcpyAsync(h->a, host, grid_bytes(h), cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess ||
        launch_boundary_copy(h->dtype, h->a, h->b, h->g, h->stream) != cudaSuccess)
        return JAC_ECUDA;
    return JAC_OK;
}

int jacobi_download(jacobi_t h, void* host, int from_b) {
    if (!h || !host) return JAC_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;
    if (cudaMemcpyAsync(host, from_b ? h->b : h->a, grid_bytes(h), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess)
        return JAC_ECUDA;
    return JAC_OK;
}

int jacobi_copy_planes(void* dst, const void* src, long long plane_elems, int elem_bytes,
                       int nplanes, void* stream) {
    if (!dst || !src || plane_elems < 1 || nplanes < 0 ||
        (elem_bytes != 2 && elem_bytes != 4 && elem_bytes != 8))
        return JAC_EINVAL;
    if (nplanes == 0) return JAC_OK;
    const size_t bytes = (size_t)plane_elems * (size_t)elem_bytes * (size_t)nplanes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice,
                           static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? JAC_OK
               : JAC_ECUDA;
}

int jacobi_check(jacobi_t h) {
    if (!h) return JAC_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;
    int st = 0;
    if (cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return JAC_ECUDA;
    if (st != 0) {
        cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
        cudaStreamSynchronize(h->stream);
        return JAC_ETIMEOUT;
    }
    return JAC_OK;
}

int jacobi_destroy(jacobi_t h) {
    if (!h) return JAC_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->status);
    delete h;
    return JAC_OK;
}

const char* jacobi_strerror(int code) {
    switch (code) {
        case JAC_OK: return "ok";
        case JAC_EINVAL: return "invalid argument (shape, pointer, pitch or alignment)";
        case JAC_ENOMEM: return "device allocation failed";
        case JAC_ECUDA: return "CUDA call failed";
        case JAC_ETIMEOUT: return "bounded device wait timed out";
        case JAC_EUNSUPPORTED: return "no kernel for this dtype/mode/configuration";
        default: return "unknown status";
    }
}

int jacobi_version(void) { return 100; }

}  // extern "C"
