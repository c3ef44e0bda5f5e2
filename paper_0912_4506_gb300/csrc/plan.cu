// Host-side launch planning shared by the entry points (see plan.h).
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "../../include/jacobi.h"
#include "plan.h"
#include "tb.cuh"

namespace jac {

namespace {

constexpr int kModes = 3;      // MODE_PLAIN, MODE_RHS, MODE_ADJ
constexpr int kCacheSlots = 64;

// Integer-pipe additions of the FP64 plain sweep when the range check allows
// them: 76 = 4 of the 5 additions through the unpacked accumulator, word form 3,
// register-capped kernel (the fastest measured, see tb_f64.cu); JACOBI_F64_EMU
// selects another entry (0: all on the FP64 unit, 6: per-addition routine,
// 16 + K + 8F: accumulator, +32: register-capped kernel).
constexpr int kDefaultF64Emu = 76;

std::mutex g_mu;

struct Tables {
    const TBEntry* e[3][kModes][kMaxDepth + 1];
    int max_t[3][kModes];
};

const Tables& tables() {
    static Tables t;
    static std::once_flag once;
    std::call_once(once, [] {
        for (auto& d : t.e)
            for (auto& m : d)
                for (auto& p : m) p = nullptr;
        // the first entry of a depth is its kernel; later ones are alternate tile
        // shapes, chosen only through JACOBI_TB_SHAPE (measurement runs)
        struct Want { int mode, T, V, NW; } want[16];
        int nwant = 0;
        if (const char* env = getenv("JACOBI_TB_SHAPE")) {
            // "mode,T,V,NW;mode,T,V,NW;..."
            const char* c = env;
            while (*c && nwant < 16) {
                Want w{};
                if (sscanf(c, "%d,%d,%d,%d", &w.mode, &w.T, &w.V, &w.NW) == 4) want[nwant++] = w;
                while (*c && *c != ';') ++c;
                if (*c == ';') ++c;
            }
        }
        auto add = [&](const TBEntry* p, int n) {
            for (int i = 0; i < n; ++i) {
                if (p[i].T < 1 || p[i].T > kMaxDepth) continue;
                const TBEntry*& slot = t.e[p[i].dtype][p[i].mode][p[i].T];
                if (!slot) slot = &p[i];
                for (int k = 0; k < nwant; ++k)
                    if (want[k].mode == p[i].mode && want[k].T == p[i].T && want[k].V == p[i].V &&
                        want[k].NW == p[i].NW)
                        slot = &p[i];
            }
        };
        int n = 0;
        const TBEntry* p;
        p = tb_entries_f64(&n); add(p, n);
        p = tb_entries_f64_deep(&n); add(p, n);
        p = tb_entries_f32(&n); add(p, n);
        p = tb_entries_f32_rhs(&n); add(p, n);
        p = tb_entries_bf16(&n); add(p, n);
        p = tb_entries_bf16_rhs(&n); add(p, n);
        // the deepest depth reachable without a gap (a table with a gap would
        // need a multi-depth remainder split; none is built that way)
        for (int d = 0; d < 3; ++d)
            for (int m = 0; m < kModes; ++m) {
                int mt = 0;
                while (mt + 1 <= kMaxDepth && t.e[d][m][mt + 1]) ++mt;
                t.max_t[d][m] = mt;
            }
    });
    return t;
}

// Small per-device cache of occupancy results keyed by kernel pointer.
struct OccSlot {
    const void* kernel;
    int device;
    int occ;
};
OccSlot g_occ[kCacheSlots];
int g_nocc = 0;

int cached_occupancy(const void* kernel, int device, int threads, size_t smem, bool set_smem) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < g_nocc; ++i)
        if (g_occ[i].kernel == kernel && g_occ[i].device == device) return g_occ[i].occ;
    if (set_smem)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) !=
        cudaSuccess)
        occ = 0;
    occ = std::max(occ, 1);
    if (g_nocc < kCacheSlots) g_occ[g_nocc++] = {kernel, device, occ};
    return occ;
}

}  // namespace

int elem_size(int dtype) { return dtype == JAC_F64 ? 8 : dtype == JAC_F32 ? 4 : 2; }

int floor_div(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

bool encode_grid_map(CUtensorMap* map, int dtype, const Geom& g, const void* base, int box_x,
                     int box_y) {
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
    if (!fn) return false;
    const int es = elem_size(dtype);
    const CUtensorMapDataType dt = dtype == JAC_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : dtype == JAC_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                      : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    cuuint64_t dims[3] = {(cuuint64_t)g.nx + 2, (cuuint64_t)g.ny + 2, (cuuint64_t)g.nz + 2};
    cuuint64_t strides[2] = {(cuuint64_t)g.px * es, (cuuint64_t)g.plane * es};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

const TBEntry* tb_entry(int dtype, int mode, int T) {
    if (dtype < 0 || dtype > 2 || mode < 0 || mode >= kModes || T < 1 || T > kMaxDepth)
        return nullptr;
    return tables().e[dtype][mode][T];
}

int max_depth(int dtype, int mode) {
    if (dtype < 0 || dtype > 2 || mode < 0 || mode >= kModes) return 0;
    return tables().max_t[dtype][mode];
}

int tb_occupancy(const TBEntry& e, int device) {
    return cached_occupancy(e.kernel, device, e.NW * 32, e.smem, true);
}

int pick_chunks(int nz, int T, long long tiles, long long slots) {
    int best = 1;
    double best_score = -1.0;
    slots = std::max<long long>(slots, 1);
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

TileGeom tile_geom(int dtype, const Geom& g, int V, int NW, int T, long long slots,
                   int nchunk_req) {
    TileGeom r{};
    const int A = 16 / elem_size(dtype);
    const int EX = 32 * V, EY = NW;
    r.ox = ((EX - 2 * T) / A) * A;
    r.oy = EY - 2 * T;
    r.ok = r.ox >= A && r.oy >= 1;
    if (!r.ok) return r;
    r.x0_first = floor_div(1 - T, A) * A;
    r.ntx = (g.nx + 1 - (r.x0_first + T) + r.ox - 1) / r.ox;
    r.nty = (g.ny + r.oy - 1) / r.oy;
    int nchunk = nchunk_req > 0 ? nchunk_req
                                : pick_chunks(g.nz, T, (long long)r.ntx * r.nty, slots);
    nchunk = std::max(1, std::min(nchunk, g.nz));
    r.kz = (g.nz + nchunk - 1) / nchunk;
    r.nchunk = (g.nz + r.kz - 1) / r.kz;
    return r;
}

// Measured fastest at 512^3 on GB300: FP64 is bound by its arithmetic pipes, so
// blocking (which adds halo recompute) cannot help the plain FP64 sweep; plain
// FP32/bf16 sweeps peak at depth 3 (128 x 32 tiles), FP32 correction sweeps at 4
// (tied with 3), bf16 correction sweeps at 2, adjoint sweeps at 3 (FP32) and 1
// (FP64).
int default_t(int dtype, int mode) {
    if (dtype == JAC_F64) return 1;
    if (mode == MODE_PLAIN) return 3;
    if (mode == MODE_RHS) return dtype == JAC_BF16 ? 2 : 4;
    return 3;
}

const PlainEntry* plain_for(int dtype) {
    if (dtype == JAC_F64) {
        static int want = -1;
        static std::once_flag once;
        std::call_once(once, [] {
            want = kDefaultF64Emu;
            if (const char* e = getenv("JACOBI_F64_EMU")) {
                const int v = atoi(e);
                if (v >= 0 && v <= 79) want = v;
            }
        });
        int n = 0;
        const PlainEntry* tab = plain_entries_f64(&n);
        for (int i = 0; i < n; ++i)
            if (tab[i].nemu == want) return &tab[i];
        return plain_entry_f64();
    }
    return dtype == JAC_F32 ? plain_entry_f32() : plain_entry_bf16();
}

void plain_grid(const PlainEntry* pe, int dtype, const Geom& g, int device, int num_sms,
                dim3* grid, int* kchunk) {
    // interior-aligned kernels (V == 1, or FP64) start at x = 1; vector kernels at 0
    const bool aligned_x1 = pe->V == 1 || dtype == JAC_F64;
    const int nvec = aligned_x1 ? (g.nx + pe->V - 1) / pe->V : g.nx / pe->V + 1;
    grid->x = (nvec + 31) / 32;
    grid->y = (g.ny + pe->WY - 1) / pe->WY;
    const int occ = cached_occupancy(pe->kernel, device, 32 * pe->WY, 0, false);
    const long long tiles = (long long)grid->x * grid->y;
    const int c = pick_chunks(g.nz, 1, tiles, (long long)num_sms * occ);
    *kchunk = (g.nz + c - 1) / c;
    grid->z = (g.nz + *kchunk - 1) / *kchunk;
}

int plan_depths(int dtype, int mode, int nsweeps, int t, DepthPlan* out) {
    out->t_full = out->n_full = out->t_last = 0;
    if (nsweeps < 0 || t < 0) return JAC_EINVAL;
    if (t == 0) t = default_t(dtype, mode);
    const int mt = max_depth(dtype, mode);
    if (mt == 0 || t > mt) return JAC_EUNSUPPORTED;
    if (nsweeps == 0) return JAC_OK;
    const int tf = std::min(t, nsweeps);
    out->t_full = tf;
    out->n_full = nsweeps / tf;
    out->t_last = nsweeps % tf;
    return JAC_OK;
}

const WaveEntry* wave_for(int dtype) {
    int n = 0;
    const WaveEntry* tab = dtype == JAC_F64   ? wave_entries_f64(&n)
                           : dtype == JAC_F32 ? wave_entries_f32(&n)
                                              : wave_entries_bf16(&n);
    int i = 0;
    if (const char* env = getenv("JACOBI_WAVE_VARIANT")) i = atoi(env);
    return (i >= 0 && i < n) ? &tab[i] : &tab[0];
}

int default_wave_t(int dtype) { return dtype == JAC_F64 ? 2 : 4; }

bool wave_plan(int dtype, const Geom& g, int t, const WaveEntry& e, int device, int num_sms,
               WavePlan* out) {
    WavePlan w{};
    if (t < 1 || t > kMaxWaveDepth) return false;
    w.t = t;
    // FP64 (register march): interior-aligned cells 1..; FP32/bf16: cells from x = 0
    const int cells = dtype == JAC_F64 ? g.nx : g.nx + 1;
    w.ntx = (cells + 32 * e.V - 1) / (32 * e.V);
    w.nty = (g.ny + e.WY - 1) / e.WY;
    const size_t plane_bytes = (size_t)g.plane * (size_t)elem_size(dtype);
    const size_t budget = (size_t)512 << 20;
    w.R = 4;
    w.sk = 2;
    w.kb = 1;
    for (int kb = 32; kb >= 1; kb /= 2)
        if ((size_t)(t - 1) * (size_t)w.R * (size_t)kb * plane_bytes <= budget) {
            w.kb = kb;
            break;
        }
    if (const char* env = getenv("JACOBI_WAVE")) {
        int kb = 0, R = 0, sk = 0;
        const int n = sscanf(env, "%d,%d,%d", &kb, &R, &sk);
        if (n >= 2 && kb >= 1 && kb <= 256 && R >= 3 && R <= 64) {
            if (n < 3) sk = std::min(2, R - 2);
            if (sk >= 1 && sk < R - 1) {
                w.kb = kb;
                w.R = R;
                w.sk = sk;
            }
        }
    }
    w.kb = std::min(w.kb, g.nz);
    w.rp = w.R * w.kb;
    w.nb = (g.nz + w.kb - 1) / w.kb;
    const long long nitems = (long long)t * w.nb * w.ntx * w.nty;
    if (nitems > (1LL << 30)) return false;
    w.nitems = (int)nitems;
    const int occ = cached_occupancy(e.kernel, device, 32 * (e.WY + 1), e.smem,
                                     e.smem > (size_t)48 * 1024);
    w.ctas = (int)std::min<long long>(nitems, (long long)num_sms * occ);
    w.ring_bytes = (size_t)(t - 1) * (size_t)w.rp * plane_bytes;
    w.flags = (size_t)t * w.ntx * w.nty * w.nb;
    *out = w;
    return true;
}

}  // namespace jac
