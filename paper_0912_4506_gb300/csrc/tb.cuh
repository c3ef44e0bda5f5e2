// Temporally-blocked sweep: T successive sweeps of Eq. 1 in one pass over HBM.
//
// GPU restatement of the paper's temporal blocking (Sect. 1.3): a block of the
// grid is updated several times while it is held on chip, and every update
// covers a region one cell smaller on each side ("shifting the block by one
// cell", Fig. 1), so no boundary exchange is needed inside a pass.  Here the
// on-chip store is one CTA's shared memory and registers instead of a shared
// L3, and the pipeline of thread-team stages becomes a pipeline of time levels
// inside the CTA:
//
//  * the CTA owns an output tile (OX x OY cells, a chunk of k-planes) and loads
//    the extended tile (EX x EY = (32*V) x NW cells, a T-cell halo around the
//    output tile) plane by plane with TMA into a ring of NS shared-memory slots;
//  * it marches k.  At step m, level 0 is plane Zlo+m (just loaded), and level s
//    (1..T) computes plane Zlo+m-s from level s-1's planes Zlo+m-s-1..Zlo+m-s+1:
//    the k-neighbours come from the thread's own registers (a 3-plane rotation
//    per level), the x-neighbours by warp shuffles, the y-neighbours from a
//    double-buffered shared-memory plane per level written in the previous step;
//  * one __syncthreads per step; level T's planes inside the chunk are written
//    to global memory for the cells of the output tile.
//
// Every thread owns V consecutive x cells of one row (lane -> x, warp -> y).
// Level s is valid on rows [s, EY-s) and columns [s, EX-s) of the extended tile;
// warps outside that row range skip the level.  Cells off the interior (the
// boundary layer, the row padding and anything outside the array, which TMA
// fills with zeros) keep their level-0 value at every level, which is exactly
// the fixed Dirichlet boundary.  All arithmetic follows Eq. 1's operand order;
// a pass of depth T therefore returns bit for bit what T plain sweeps return.
//
// Modes: MODE_PLAIN (Eq. 1), MODE_RHS (the refinement's correction sweep, adds
// rho before the product), MODE_ADJ (the adjoint sweep on a zero boundary, and
// accumulation of RN(1/6)*lambda at the face-neighbouring interior cells into
// the boundary gradient).
#pragma once

#include "common.cuh"

namespace jac {

enum { MODE_PLAIN = 0, MODE_RHS = 1, MODE_ADJ = 2 };

struct TBArgs {
    Geom g;
    void* dst;          // output grid of the pass (level T)
    const void* rho;    // MODE_RHS: right-hand side grid (same layout)
    void* grad;         // MODE_ADJ: boundary gradient grid (same layout)
    int ox;             // output tile width (multiple of the TMA alignment)
    int x0_first;       // x origin of tile 0's extended tile (aligned, may be < 0)
    int kz;             // output k-planes per CTA
    int* status;        // device status word (timeouts)
};

template <int V, int NW, int T, int NS, class S>
struct TBLayout {
    static constexpr int EX = 32 * V;
    static constexpr int EY = NW;
    static constexpr int PLANE = EX * EY;
    static constexpr int NLB = (T > 1) ? 2 * (T - 1) : 0;  // level buffers
    static constexpr int HEADER = 1024;                      // mbarriers, aligned
    static constexpr size_t bytes() {
        return HEADER + (size_t)(NS + NLB) * PLANE * sizeof(S);
    }
};

template <class Tr, int V, int NW, int T, int MODE, int NS>
__global__ void __launch_bounds__(NW * 32, 1)
    tb_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const TBArgs a) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    using L = TBLayout<V, NW, T, NS, S>;
    constexpr int EX = L::EX, EY = L::EY, PLANE = L::PLANE;
    constexpr uint32_t kPlaneBytes = PLANE * sizeof(S);
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    S* ring = reinterpret_cast<S*>(smem + L::HEADER);
    S* lvl = ring + NS * PLANE;
    __shared__ int s_abort;

    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const Geom g = a.g;
    constexpr int OY = EY - 2 * T;
    const int X0 = a.x0_first + (int)blockIdx.x * a.ox;
    const int Y0 = 1 - T + (int)blockIdx.y * OY;
    const int ox0 = X0 + T, oy0 = Y0 + T;
    const int kz0 = 1 + (int)blockIdx.z * a.kz;
    const int kz1 = min(g.nz + 1, kz0 + a.kz);
    const int Zlo = kz0 - T;
    const int M = (kz1 - kz0) + 2 * T;
    const int gy = Y0 + w;
    const int gx0 = X0 + lane * V;

    bool inxy[V], outxy[V];
    bool all_out = true, all_in = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int x = gx0 + e;
        inxy[e] = (x >= 1) && (x <= g.nx) && (gy >= 1) && (gy <= g.ny);
        outxy[e] = inxy[e] && (x >= ox0) && (x < ox0 + a.ox) && (gy >= oy0) && (gy < oy0 + OY);
        all_out = all_out && outxy[e];
        all_in = all_in && inxy[e];
    }

    if (tid == 0) {
        s_abort = 0;
#pragma unroll 1
        for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();
    int issued = 0;  // planes issued so far (thread 0 only)
    if (tid == 0) {
#pragma unroll 1
        for (int i = 0; i < NS && i < M; ++i) {
            mbar_arrive_expect_tx(&bars[i], kPlaneBytes);
            tma_load_3d(ring + i * PLANE, &tmap, &bars[i], X0, Y0, Zlo + i);
        }
        issued = min(NS, M);
    }

    C r[T][3][V];  // per level s < T: planes (old, cur, new) of level s, own cells
    C rq[(MODE == MODE_RHS) ? T + 1 : 1][V];  // rho FIFO: rq[j] = rho at plane Zlo+m-j
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int e = 0; e < V; ++e) r[s][j][e] = C(0);
#pragma unroll
    for (int j = 0; j < ((MODE == MODE_RHS) ? T + 1 : 1); ++j)
#pragma unroll
        for (int e = 0; e < V; ++e) rq[j][e] = C(0);

    const C c6 = Tr::sixth();
    const S* rho = static_cast<const S*>(a.rho);
    S* dst = static_cast<S*>(a.dst);
    S* grad = static_cast<S*>(a.grad);
    const long long rowoff = (long long)gy * g.px + gx0;  // valid only when used

    // boundary-gradient accumulation of one level's plane p (MODE_ADJ)
    auto adj_acc = [&](const C (&v)[V], int p) {
        if (p < kz0 || p >= kz1) return;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (!outxy[e]) continue;
            const int x = gx0 + e;
            const C cv = Tr::mul(c6, v[e]);
            if (x == 1) {
                const long long o = g.lin(0, gy, p);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
            if (x == g.nx) {
                const long long o = g.lin(g.nx + 1, gy, p);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
            if (gy == 1) {
                const long long o = g.lin(x, 0, p);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
            if (gy == g.ny) {
                const long long o = g.lin(x, g.ny + 1, p);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
            if (p == 1) {
                const long long o = g.lin(x, gy, 0);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
            if (p == g.nz) {
                const long long o = g.lin(x, gy, g.nz + 1);
                grad[o] = Tr::st(Tr::add(Tr::ld(grad[o]), cv));
            }
        }
    };

    int m = 0;
#pragma unroll 1
    for (; m < M; ++m) {
        const int slot = m % NS;
        if (!mbar_wait_bounded(&bars[slot], (uint32_t)((m / NS) & 1))) {
            atomicOr(a.status, kStatusTimeout);
            s_abort = 1;
        }
        // ---- level 0: plane Zlo + m, own cells
        {
            const int p = Zlo + m;
            const bool zin = (p >= 1) && (p <= g.nz);
            const Vec<S, V> t =
                *reinterpret_cast<const Vec<S, V>*>(ring + slot * PLANE + w * EX + lane * V);
#pragma unroll
            for (int e = 0; e < V; ++e) r[0][2][e] = Tr::ld(t.v[e]);
            if (MODE == MODE_RHS) {
#pragma unroll
                for (int j = ((MODE == MODE_RHS) ? T : 0); j >= 1; --j)
#pragma unroll
                    for (int e = 0; e < V; ++e) rq[j][e] = rq[j - 1][e];
                if (zin && all_in) {
                    const Vec<S, V> q = ldg_vec<S, V>(rho + g.plane * p + rowoff);
#pragma unroll
                    for (int e = 0; e < V; ++e) rq[0][e] = Tr::ld(q.v[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        rq[0][e] = (zin && inxy[e]) ? Tr::ld(rho[g.plane * p + rowoff + e]) : C(0);
                }
            }
            if (MODE == MODE_ADJ && T > 0) adj_acc(r[0][2], p);
        }
        // ---- levels 1..T
#pragma unroll
        for (int s = 1; s <= T; ++s) {
            if (m < s) continue;                        // pipeline fill
            if (w < s || w >= EY - s) continue;         // row outside level s's region
            const int q = Zlo + m - s;
            const bool zin = (q >= 1) && (q <= g.nz);
            const S* nb = (s == 1) ? ring + ((m - 1) % NS) * PLANE
                                   : lvl + ((s - 2) * 2 + ((m - 1) & 1)) * PLANE;
            const Vec<S, V> vn = *reinterpret_cast<const Vec<S, V>*>(nb + (w - 1) * EX + lane * V);
            const Vec<S, V> vs = *reinterpret_cast<const Vec<S, V>*>(nb + (w + 1) * EX + lane * V);
            const C left = __shfl_up_sync(FULL, r[s - 1][1][V - 1], 1);
            const C right = __shfl_down_sync(FULL, r[s - 1][1][0], 1);
            C out[V];
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const C l = (e == 0) ? left : r[s - 1][1][e - 1];
                const C rr = (e == V - 1) ? right : r[s - 1][1][e + 1];
                C sum = Tr::add(l, rr);
                sum = Tr::add(sum, Tr::ld(vn.v[e]));
                sum = Tr::add(sum, Tr::ld(vs.v[e]));
                sum = Tr::add(sum, r[s - 1][0][e]);
                sum = Tr::add(sum, r[s - 1][2][e]);
                if (MODE == MODE_RHS) sum = Tr::add(sum, rq[s][e]);
                const C val = Tr::rnd(Tr::mul(sum, c6));
                out[e] = (inxy[e] && zin) ? val : r[s - 1][1][e];
            }
            if (s < T) {
                Vec<S, V> o;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    r[s < T ? s : 0][2][e] = out[e];
                    o.v[e] = Tr::st(out[e]);
                }
                *reinterpret_cast<Vec<S, V>*>(lvl + ((s - 1) * 2 + (m & 1)) * PLANE + w * EX +
                                              lane * V) = o;
                if (MODE == MODE_ADJ) adj_acc(out, q);
            } else if (q >= kz0 && q < kz1) {
                const long long o = g.plane * q + rowoff;
                if (all_out) {
                    Vec<S, V> ov;
#pragma unroll
                    for (int e = 0; e < V; ++e) ov.v[e] = Tr::st(out[e]);
                    *reinterpret_cast<Vec<S, V>*>(dst + o) = ov;
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (outxy[e]) dst[o + e] = Tr::st(out[e]);
                }
            }
        }
        // ---- rotate the per-level k window
#pragma unroll
        for (int s = 0; s < T; ++s)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                r[s][0][e] = r[s][1][e];
                r[s][1][e] = r[s][2][e];
            }
        __syncthreads();
        if (s_abort) break;
        // the slot of plane Zlo+m-1 is free now: refill it with plane Zlo+m-1+NS
        if (tid == 0 && m >= 1 && issued < M) {
            const int sl = (m - 1) % NS;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[sl], kPlaneBytes);
            tma_load_3d(ring + sl * PLANE, &tmap, &bars[sl], X0, Y0, Zlo + issued);
            ++issued;
        }
    }
    if (m < M && tid == 0) {
        // timed out: let the copies already in flight land before the CTA's shared
        // memory is released (each wait bounded again)
#pragma unroll 1
        for (int p = m + 1; p < issued; ++p)
            (void)mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), 500000000ull);
    }
}

}  // namespace jac
