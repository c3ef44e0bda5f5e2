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
#include "plan.h"
#include "tb.cuh"
#include "wave.cuh"

using namespace jac;

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
    void* fbuf;           // adjoint: face values per sweep (owned, grown on demand)
    size_t fbuf_bytes;
    cudaStream_t side;    // adjoint: face bands run beside the passes (created on first use)
    cudaEvent_t ev_in, ev_band[3];  // ev_band[i]: last band that read grid i (A, B, C)
    void* c;              // adjoint: third grid of the rotation (owned, grown on demand)
    size_t c_bytes;
    CUtensorMap map_c;
    int map_c_box_x, map_c_box_y;
    int inplace;          // one grid (jacobi_create_inplace): b == nullptr
    void* wbuf;           // pipelined passes: rings and counters (owned, grown on demand)
    size_t wbuf_bytes;
};

namespace {

int check_grid_args(int nx, int ny, int nz, int dtype, long long pitch) {
    if (nx < 1 || ny < 1 || nz < 1) return JAC_EINVAL;
    if (dtype < JAC_F64 || dtype > JAC_BF16) return JAC_EINVAL;
    if (pitch < nx + 2) return JAC_EINVAL;
    if ((pitch * elem_size(dtype)) % 16 != 0) return JAC_EINVAL;
    if ((long long)(ny + 2) * pitch * (nz + 2) > (1LL << 40)) return JAC_EINVAL;
    return JAC_OK;
}

// Integer-pipe additions of a kernel variant in half additions per update (codes
// of 16 and above select the unpacked accumulator with (code - 16) mod 8 additions).
int emu_half_adds(int code) { return code >= 16 ? 2 * ((code - 16) & 7) : code; }  // K bits

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Grow the handle's device buffer `*buf` to at least `need` bytes (the stream
// is drained before an old buffer is released).
int grow_buffer(jacobi_s* h, void** buf, size_t* bytes, size_t need) {
    if (need <= *bytes) return JAC_OK;
    if (*buf) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return JAC_ECUDA;
        cudaFree(*buf);
        *buf = nullptr;
        *bytes = 0;
    }
    if (cudaMalloc(buf, need) != cudaSuccess) {
        *buf = nullptr;
        return JAC_ENOMEM;
    }
    *bytes = need;
    return JAC_OK;
}

// Pipelined (wavefront) passes: t updates per pass with no halo recompute; in
// place for a one-grid handle (every pass of depth >= 2).
int run_wave(jacobi_s* h, int nsweeps, int t, int* final_is_b, jacobi_plan_info* info_only) {
    const WaveEntry* we = wave_for(h->dtype);
    if (t == 0) t = default_wave_t(h->dtype);
    if (t > kMaxWaveDepth) return JAC_EUNSUPPORTED;
    DepthPlan dp{0, 0, 0};
    if (nsweeps > 0) {
        dp.t_full = std::min(t, nsweeps);
        dp.n_full = nsweeps / dp.t_full;
        dp.t_last = nsweeps % dp.t_full;
        if (h->inplace) {
            // an in-place pass needs depth >= 2 (its last level overwrites values
            // that its first level of the neighbouring tiles still reads otherwise)
            if (dp.t_full < 2) return JAC_EUNSUPPORTED;
            if (dp.t_last == 1) {
                dp.n_full -= 1;
                dp.t_last = dp.t_full + 1;
                if (dp.t_last > kMaxWaveDepth) return JAC_EUNSUPPORTED;
            }
        }
    }
    // handle buffer: the done flags, the ticket and the abort word first (cleared
    // once per call; pass p marks its flags with p + 1), the rings after them
    WavePlan wp[2];
    size_t flags = 0, rings = 0;
    for (int p = 0; p < 2; ++p) {
        const int d = p == 0 ? dp.t_full : dp.t_last;
        if (d == 0 || (p == 0 && dp.n_full == 0)) continue;
        if (!wave_plan(h->dtype, h->g, d, *we, h->device, h->num_sms, &wp[p]))
            return JAC_EUNSUPPORTED;
        flags = std::max(flags, wp[p].flags);
        rings = std::max(rings, wp[p].ring_bytes);
    }
    const size_t sync_bytes = ((flags + 2) * sizeof(int) + 255) & ~(size_t)255;
    const size_t need = sync_bytes + rings;
    if (info_only) {
        std::memset(info_only, 0, sizeof(*info_only));
        info_only->kernel = JAC_KERNEL_WAVE;
        info_only->passes = dp.passes();
        if (dp.passes() > 0) {
            const WavePlan& w = dp.n_full > 0 ? wp[0] : wp[1];
            info_only->t = w.t;
            info_only->remainder_t = dp.n_full > 0 ? dp.t_last : 0;
            info_only->tile_x = 32 * we->V;
            info_only->tile_y = we->WY;
            info_only->ext_x = 32 * we->V;
            info_only->ext_y = we->WY;
            info_only->kchunk = w.kb;
            info_only->threads = 32 * (we->WY + 1);
            info_only->grid_x = w.ctas;
            info_only->grid_y = 1;
            info_only->grid_z = 1;
            info_only->emu_adds = emu_half_adds(we->nemu);
        }
        return JAC_OK;
    }
    if (dp.passes() == 0) {
        if (final_is_b) *final_is_b = 0;
        return JAC_OK;
    }
    int rc = grow_buffer(h, &h->wbuf, &h->wbuf_bytes, need);
    if (rc != JAC_OK) return rc;
    const int* fast = nullptr;
    if (we->nemu > 0) {
        fast = h->status + 16;
        if (launch_range_check(static_cast<const double*>(h->a), h->g, h->status + 16,
                               h->stream) != cudaSuccess)
            return JAC_ECUDA;
    }
    // failure-detection tests: the items of the first block of level 1 are never
    // handed out, so the items that need them wait out a short limit and the
    // launch ends with the timeout status
    const char* hook = getenv("JACOBI_WAVE_TEST_MISSING_PRODUCER");
    const bool missing_producer = hook && hook[0] == '1';
    int* sync = static_cast<int*>(h->wbuf);
    if (cudaMemsetAsync(sync, 0, (flags + 2) * sizeof(int), h->stream) != cudaSuccess)
        return JAC_ECUDA;
    int cur_b = 0;
    for (int p = 0; p < dp.passes(); ++p) {
        const WavePlan& w = p < dp.n_full ? wp[0] : wp[1];
        if (p > 0 &&
            cudaMemsetAsync(sync + flags, 0, 2 * sizeof(int), h->stream) != cudaSuccess)
            return JAC_ECUDA;
        WaveArgs a;
        a.g = h->g;
        a.src = cur_b ? h->b : h->a;
        a.dst = h->inplace ? h->a : (cur_b ? h->a : h->b);
        a.ring = static_cast<char*>(h->wbuf) + sync_bytes;
        a.t = w.t;
        a.kb = w.kb;
        a.nb = w.nb;
        a.R = w.R;
        a.sk = w.sk;
        a.rp = w.rp;
        a.ntx = w.ntx;
        a.nty = w.nty;
        a.nitems = w.nitems;
        a.inplace = h->inplace;
        a.done = sync;
        a.epoch = p + 1;
        a.ticket = sync + flags;
        a.abort = sync + flags + 1;
        a.status = h->status;
        a.fast = fast;
        a.one = 1u;
        a.wait_ns = 2000000000ull;
        if (missing_producer) {
            const int first = w.ntx * w.nty;  // tickets of items (s = 1, b = 0, *)
            if (cudaMemcpyAsync(a.ticket, &first, sizeof(int), cudaMemcpyHostToDevice,
                                h->stream) != cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess)
                return JAC_ECUDA;
            a.wait_ns = 100000000ull;
        }
        // TMA-staged entries: boxes of the tile plus a 16-byte-aligned x halo and one
        // row above and below, over the source grid and over the rings (levels
        // 1..t-1 as one array of (t-1) rp planes in the grid's plane layout)
        CUtensorMap map_src{}, map_ring{};
        if (we->tma) {
            const int box_x = 32 * we->V + 2 * (16 / elem_size(h->dtype));
            const int box_y = we->WY + 2;
            if (!encode_grid_map(&map_src, h->dtype, h->g, a.src, box_x, box_y))
                return JAC_ECUDA;
            map_ring = map_src;
            if (w.t >= 2) {
                Geom gr = h->g;
                gr.nz = (w.t - 1) * w.rp - 2;
                if (!encode_grid_map(&map_ring, h->dtype, gr, a.ring, box_x, box_y))
                    return JAC_ECUDA;
            }
        }
        if (we->launch(a, map_src, map_ring, w.ctas, h->stream) != cudaSuccess)
            return JAC_ECUDA;
        if (!h->inplace) cur_b ^= 1;
    }
    if (final_is_b) *final_is_b = cur_b;
    return JAC_OK;
}

// Run nsweeps of `mode` as a sequence of passes.  kernel: JAC_KERNEL_*.
int run_passes(jacobi_s* h, int mode, int nsweeps, int t, int kernel, const void* rho,
               void* grad, int* final_is_b, jacobi_plan_info* info_only) {
    if (!h || nsweeps < 0 || t < 0) return JAC_EINVAL;
    if (kernel < JAC_KERNEL_AUTO || kernel > JAC_KERNEL_WAVE) return JAC_EINVAL;
    if (h->inplace) {
        // one grid: only the pipelined passes update it in place
        if (mode != MODE_PLAIN || (kernel != JAC_KERNEL_AUTO && kernel != JAC_KERNEL_WAVE))
            return JAC_EUNSUPPORTED;
        kernel = JAC_KERNEL_WAVE;
    }
    if (kernel == JAC_KERNEL_WAVE) {
        if (mode != MODE_PLAIN) return JAC_EUNSUPPORTED;
        if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;
        return run_wave(h, nsweeps, t, final_is_b, info_only);
    }
    if (t == 0) t = default_t(h->dtype, mode);
    // depth 1: FP64 takes the register-march streaming kernel (FP64-pipe bound, with
    // the integer-pipe additions); FP32/bf16 take the TMA-ring kernel at depth 1
    // (128 x 12 tiles), which keeps more bytes in flight than the register march
    if (kernel == JAC_KERNEL_AUTO)
        kernel = (t == 1 && h->dtype == JAC_F64) ? JAC_KERNEL_PLAIN : JAC_KERNEL_TB;
    if (mode == MODE_RHS) kernel = JAC_KERNEL_TB;  // correction sweeps only exist blocked
    if (cudaSetDevice(h->device) != cudaSuccess) return JAC_ECUDA;

    // adjoint: one row of face values per sweep, added to the gradient at the end;
    // the face bands run on a side stream beside the sweeps
    const long long fstride = 2LL * ((long long)h->g.ny * h->g.nz +
                                     (long long)h->g.nx * h->g.nz +
                                     (long long)h->g.nx * h->g.ny);
    if (mode == MODE_ADJ && nsweeps > 0 && !info_only) {
        const size_t need = (size_t)fstride * (size_t)nsweeps * (size_t)elem_size(h->dtype);
        int grc = grow_buffer(h, &h->fbuf, &h->fbuf_bytes, need);
        if (grc != JAC_OK) return grc;
        void* old_c = h->c;
        const size_t grid_bytes = (size_t)h->g.plane * (size_t)(h->g.nz + 2) *
                                  (size_t)elem_size(h->dtype);
        grc = grow_buffer(h, &h->c, &h->c_bytes, grid_bytes);
        if (grc != JAC_OK) return grc;
        if (h->c != old_c) h->map_c_box_x = h->map_c_box_y = 0;  // stale descriptor
        if (!h->side) {
            if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess)
                return JAC_ECUDA;
            for (int i = 0; i < 3; ++i)
                if (cudaEventCreateWithFlags(&h->ev_band[i], cudaEventDisableTiming) !=
                    cudaSuccess)
                    return JAC_ECUDA;
        }
        // the third grid carries A's boundary layer like B
        if (launch_boundary_copy(h->dtype, h->a, h->c, h->g, h->stream) != cudaSuccess)
            return JAC_ECUDA;
    }
    // Adjoint grids rotate through A, B and C: the face values of the levels
    // 0..T-1 of a pass come from its input (the band kernel on the side stream,
    // beside the pass, which only reads the same input), and a pass writes to the
    // grid that is neither its input nor the previous pass's input, so it waits
    // only for the band of the pass before last (the one that read its output
    // grid).  The last pass writes to A or B.  Other modes alternate A and B.
    void* const grids[3] = {h->a, h->b, h->c};
    bool band_pending[3] = {false, false, false};
    int cur = 0, prev = -1;  // grid of the current input, of the previous input
    auto band_before = [&](int sweep0, int T) -> bool {
        band_pending[cur] = true;
        return cudaEventRecord(h->ev_in, h->stream) == cudaSuccess &&
               cudaStreamWaitEvent(h->side, h->ev_in, 0) == cudaSuccess &&
               launch_face_band(h->dtype, grids[cur], h->g, h->fbuf, fstride, sweep0, T,
                                h->side) == cudaSuccess &&
               cudaEventRecord(h->ev_band[cur], h->side) == cudaSuccess;
    };
    auto band_wait = [&](int i) -> bool {
        if (!band_pending[i]) return true;
        band_pending[i] = false;
        return cudaStreamWaitEvent(h->stream, h->ev_band[i], 0) == cudaSuccess;
    };
    // the grid the next pass writes (waiting for a band still reading it)
    auto next_grid = [&](bool last) -> int {
        if (mode != MODE_ADJ) return cur ^ 1;
        int d = prev < 0 ? 1 : 3 - cur - prev;
        if (last && d == 2) d = prev;
        return d;
    };
    // all bands done, then the face rows into the gradient
    auto finish_adjoint = [&]() -> bool {
        return band_wait(0) && band_wait(1) && band_wait(2) &&
               launch_face_reduce(h->dtype, grad, h->g, h->fbuf, fstride, nsweeps,
                                  h->stream) == cudaSuccess;
    };

    if (kernel == JAC_KERNEL_PLAIN) {
        const PlainEntry* pe = plain_for(h->dtype);
        dim3 grid;
        int kchunk = 0;
        plain_grid(pe, h->dtype, h->g, h->device, h->num_sms, &grid, &kchunk);
        if (info_only) {
            std::memset(info_only, 0, sizeof(*info_only));
            info_only->kernel = JAC_KERNEL_PLAIN;
            info_only->emu_adds = emu_half_adds(pe->nemu);
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
            if (mode == MODE_ADJ && !band_before(s, 1)) return JAC_ECUDA;
            const int dst = next_grid(s + 1 == nsweeps);
            if (!band_wait(dst)) return JAC_ECUDA;
            if (pe->launch(grids[cur], grids[dst], h->g, kchunk, grid, fast, h->stream) !=
                cudaSuccess)
                return JAC_ECUDA;
            prev = cur;
            cur = dst;
        }
        if (mode == MODE_ADJ && nsweeps > 0 && !finish_adjoint()) return JAC_ECUDA;
        if (final_is_b) *final_is_b = cur;
        return JAC_OK;
    }

    // The adjoint sweep (transposed Eq. 1 on lambda with a zero boundary) is the
    // plain sweep on the handle's grids: it runs on the plain blocked kernels, and
    // its boundary-gradient face values come from launch_face_band per pass.
    const int kmode = mode == MODE_ADJ ? MODE_PLAIN : mode;
    DepthPlan dp;
    const int rc = plan_depths(h->dtype, kmode, nsweeps, t, &dp);
    if (rc != JAC_OK) return rc;
    const long long slots_per_sm = h->num_sms;

    if (info_only) {
        std::memset(info_only, 0, sizeof(*info_only));
        info_only->kernel = JAC_KERNEL_TB;
        info_only->passes = dp.passes();
        if (dp.passes() > 0) {
            const int t0 = dp.depth(0);
            const TBEntry* e = tb_entry(h->dtype, kmode, t0);
            const TileGeom gm = tile_geom(h->dtype, h->g, e->V, e->NW, e->T,
                                          slots_per_sm * tb_occupancy(*e, h->device), 0);
            info_only->t = t0;
            info_only->remainder_t = dp.n_full > 0 ? dp.t_last : 0;
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
            info_only->emu_adds = emu_half_adds(e->emu);
        }
        return JAC_OK;
    }

    // FP64 blocked passes with integer-pipe additions: one range check per call
    // (the sweep averages, so values stay in range for every later pass)
    const int* fast = nullptr;
    if (h->dtype == JAC_F64 && mode == MODE_PLAIN && dp.passes() > 0) {
        bool any_emu = false;
        for (int p = 0; p < 2; ++p) {
            const int d = p == 0 ? dp.t_full : dp.t_last;
            const TBEntry* e = d > 0 ? tb_entry(h->dtype, mode, d) : nullptr;
            any_emu = any_emu || (e && e->emu > 0);
        }
        if (any_emu) {
            fast = h->status + 16;
            if (launch_range_check(static_cast<const double*>(h->a), h->g, h->status + 16,
                                   h->stream) != cudaSuccess)
                return JAC_ECUDA;
        }
    }

    int sweep0 = 0;
    for (int p = 0; p < dp.passes(); ++p) {
        const TBEntry* e = tb_entry(h->dtype, kmode, dp.depth(p));
        if (!e) return JAC_EUNSUPPORTED;
        if (mode == MODE_ADJ && !band_before(sweep0, e->T)) return JAC_ECUDA;
        const TileGeom gm = tile_geom(h->dtype, h->g, e->V, e->NW, e->T,
                                      slots_per_sm * tb_occupancy(*e, h->device), 0);
        if (!gm.ok) return JAC_EUNSUPPORTED;
        const int EX = 32 * e->V, EY = e->NW;
        if (EX != h->map_box_x || EY != h->map_box_y) {
            if (!encode_grid_map(&h->map_a, h->dtype, h->g, h->a, EX, EY) ||
                !encode_grid_map(&h->map_b, h->dtype, h->g, h->b, EX, EY))
                return JAC_ECUDA;
            h->map_box_x = EX;
            h->map_box_y = EY;
        }
        if (cur == 2 && (EX != h->map_c_box_x || EY != h->map_c_box_y)) {
            if (!encode_grid_map(&h->map_c, h->dtype, h->g, h->c, EX, EY)) return JAC_ECUDA;
            h->map_c_box_x = EX;
            h->map_c_box_y = EY;
        }
        const int dst = next_grid(p + 1 == dp.passes());
        if (!band_wait(dst)) return JAC_ECUDA;
        TBArgs args;
        args.g = h->g;
        args.dst = grids[dst];
        args.grad = grad;
        args.ox = gm.ox;
        args.x0_first = gm.x0_first;
        args.kz = gm.kz;
        args.status = h->status;
        args.fast = fast;
        args.one = 1u;
        if (mode == MODE_RHS &&
            (rho != h->rho_ptr || EX != h->rho_box_x || EY != h->rho_box_y)) {
            if (!encode_grid_map(&h->map_rho, h->dtype, h->g, rho, EX, EY)) return JAC_ECUDA;
            h->rho_ptr = rho;
            h->rho_box_x = EX;
            h->rho_box_y = EY;
        }
        const CUtensorMap& map = cur == 0 ? h->map_a : cur == 1 ? h->map_b : h->map_c;
        const CUtensorMap& map_rho = mode == MODE_RHS ? h->map_rho : map;
        if (e->launch(map, map_rho, args, dim3(gm.ntx, gm.nty, gm.nchunk), h->stream) !=
            cudaSuccess)
            return JAC_ECUDA;
        prev = cur;
        cur = dst;
        sweep0 += e->T;
    }
    if (mode == MODE_ADJ && nsweeps > 0 && !finish_adjoint()) return JAC_ECUDA;
    if (final_is_b) *final_is_b = cur;
    return JAC_OK;
}

}  // namespace

extern "C" {

static int create_handle(jacobi_t* out, int nx, int ny, int nz, int dtype, void* grid_a,
                         void* grid_b, long long row_pitch, void* stream) {
    if (!out) return JAC_EINVAL;
    *out = nullptr;
    int rc = check_grid_args(nx, ny, nz, dtype, row_pitch);
    if (rc != JAC_OK) return rc;
    if (!grid_a || grid_a == grid_b || !aligned16(grid_a) || (grid_b && !aligned16(grid_b)))
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
    h->inplace = grid_b == nullptr;
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
        (grid_b && launch_boundary_copy(dtype, grid_a, grid_b, h->g, h->stream) != cudaSuccess)) {
        cudaFree(h->status);
        delete h;
        return JAC_ECUDA;
    }
    *out = h;
    return JAC_OK;
}

int jacobi_create(jacobi_t* out, int nx, int ny, int nz, int dtype, void* grid_a, void* grid_b,
                  long long row_pitch, void* stream) {
    if (!grid_b) {
        if (out) *out = nullptr;
        return JAC_EINVAL;
    }
    return create_handle(out, nx, ny, nz, dtype, grid_a, grid_b, row_pitch, stream);
}

int jacobi_create_inplace(jacobi_t* out, int nx, int ny, int nz, int dtype, void* grid,
                          long long row_pitch, void* stream) {
    return create_handle(out, nx, ny, nz, dtype, grid, nullptr, row_pitch, stream);
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
    return run_passes(h, MODE_ADJ, nsweeps, t, JAC_KERNEL_AUTO, nullptr, grad_bdry,
                      final_is_b, nullptr);
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
        (h->b && launch_boundary_copy(h->dtype, h->a, h->b, h->g, h->stream) != cudaSuccess))
        return JAC_ECUDA;
    return JAC_OK;
}

int jacobi_download(jacobi_t h, void* host, int from_b) {
    if (!h || !host || (from_b && !h->b)) return JAC_EINVAL;
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
    if (h->fbuf) cudaFree(h->fbuf);
    if (h->c) cudaFree(h->c);
    if (h->wbuf) cudaFree(h->wbuf);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaEventDestroy(h->ev_in);
        for (int i = 0; i < 3; ++i) cudaEventDestroy(h->ev_band[i]);
        cudaStreamDestroy(h->side);
    }
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
        case JAC_EUNSUPPORTED:
            return "no kernel for this dtype/operation/depth (jacobi_max_depth gives the deepest "
                   "depth built)";
        default: return "unknown status";
    }
}

int jacobi_max_depth(int dtype, int op) {
    if (dtype < JAC_F64 || dtype > JAC_BF16 || op < JAC_OP_SWEEP || op > JAC_OP_ADJOINT)
        return JAC_EINVAL;
    // the adjoint runs on the plain sweep's kernels (run_passes); bf16 has none
    if (op == JAC_OP_ADJOINT && dtype == JAC_BF16) return 0;
    const int mode = op == JAC_OP_RHS ? MODE_RHS : MODE_PLAIN;
    return max_depth(dtype, mode);
}

int jacobi_version(void) { return 300; }

}  // extern "C"
