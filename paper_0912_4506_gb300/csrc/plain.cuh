// Plain streaming sweep: one sweep of Eq. 1 per pass over HBM.
//
// Each thread owns V consecutive x cells of one row (a 16-byte vector for
// V > 1, the interior-aligned cell for V == 1) and marches k through a chunk of
// planes, keeping the k-1, k, k+1 values of its cells in registers (k-plane
// register rotation), so each plane of A is read from HBM once and each plane
// of B written once: 2 * sizeof(S) bytes per lattice-site update (Eq. 2 of the
// paper's baseline model counts 16 B/LUP for FP64).  In-plane neighbours: x via
// warp shuffles (global loads at the two warp edges), y via L1-cached loads of
// the rows above and below, which the neighbouring warps stream anyway.
#pragma once

#include "common.cuh"
#include "emu.cuh"
#include "emusum.cuh"

namespace jac {

// The sweep of one chunk for FP32/bf16 storage (arithmetic in FP32, Eq. 1's
// operand order).  The sweep is bound by HBM, so the march keeps several planes of
// loads in flight and spends few instructions per step: one base pointer at plane
// k+1 advances by a plane per step, and every load is that pointer plus a row,
// plane or element offset (the stream of plane k+3, the rows above and below of
// plane k+1, the two x-edge cells of plane k+1); values stay in storage format
// until used.  Loads past the last plane of the array are skipped (the stream
// runs ahead of the chunk by two planes).
template <class Tr, int V>
__device__ __forceinline__ void plain_march(const typename Tr::S* __restrict__ A,
                                            typename Tr::S* __restrict__ B, const Geom& g,
                                            int k0, int k1, int lane, bool loadable,
                                            const bool (&interior)[V], bool all_interior,
                                            bool left_ok, bool right_ok, long long row) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    using VS = Vec<S, V>;
    const unsigned FULL = 0xffffffffu;
    const C c6 = Tr::sixth();
    const long long plane = g.plane, px = g.px;
    const int ktop = g.nz + 1;  // last plane in the array
    const bool el_ok = lane == 0 && left_ok, er_ok = lane == 31 && right_ok;
    VS zero;
#pragma unroll
    for (int e = 0; e < V; ++e) zero.v[e] = S(0);
    auto ldv = [&](const S* p, bool ok) -> VS { return ok ? ldg_vec<S, V>(p) : zero; };
    auto lds = [&](const S* p, bool ok) -> S { return ok ? __ldg(p) : S(0); };

    // p1: (x0, y) of plane k+1 in A; planes k0-1 .. k0+2 and the in-plane
    // neighbours of plane k0 are loaded before the march
    const S* p1 = A + row + plane * k0;
    VS dn = ldv(p1 - plane, loadable);
    VS ct = ldv(p1, loadable);
    VS up = ldv(p1 + plane, loadable && k0 + 1 <= ktop);
    VS up2 = ldv(p1 + 2 * plane, loadable && k0 + 2 <= ktop);
    VS no = ldv(p1 - px, loadable);
    VS so = ldv(p1 + px, loadable);
    S el = lds(p1 - 1, el_ok), er = lds(p1 + V, er_ok);
    p1 += plane;
    S* pb = B + row + plane * k0;

#pragma unroll 2
    for (int k = k0; k <= k1; ++k) {
        // loads for the next steps first: stream plane k+3, neighbours of k+1
        const VS up3 = ldv(p1 + 2 * plane, loadable && k + 3 <= ktop);
        const bool n1 = loadable && k + 1 <= ktop;
        const VS no2 = ldv(p1 - px, n1);
        const VS so2 = ldv(p1 + px, n1);
        const S el2 = lds(p1 - 1, el_ok && k + 1 <= ktop);
        const S er2 = lds(p1 + V, er_ok && k + 1 <= ktop);

        C left = __shfl_up_sync(FULL, Tr::ld(ct.v[V - 1]), 1);
        C right = __shfl_down_sync(FULL, Tr::ld(ct.v[0]), 1);
        if (lane == 0) left = Tr::ld(el);
        if (lane == 31) right = Tr::ld(er);
        VS outv;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const C l = (e == 0) ? left : Tr::ld(ct.v[e - 1]);
            const C r = (e == V - 1) ? right : Tr::ld(ct.v[e + 1]);
            C s = Tr::add(l, r);
            s = Tr::add(s, Tr::ld(no.v[e]));
            s = Tr::add(s, Tr::ld(so.v[e]));
            s = Tr::add(s, Tr::ld(dn.v[e]));
            s = Tr::add(s, Tr::ld(up.v[e]));
            outv.v[e] = Tr::st(Tr::mul(s, c6));
        }
        if (all_interior) {
            *reinterpret_cast<VS*>(pb) = outv;
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (interior[e]) pb[e] = outv.v[e];
        }
        dn = ct;
        ct = up;
        up = up2;
        up2 = up3;
        no = no2;
        so = so2;
        el = el2;
        er = er2;
        p1 += plane;
        pb += plane;
    }
}

// FP64 variant of the march.  The FP64 sweep is bound by its arithmetic pipes
// (the FP64 unit and, for the emulated additions, the integer ALU), so this
// march saves instructions rather than latency: cells are interior-aligned
// (x0 = 1 + V*lane, no idle lanes at the row end), loaded as scalars, the pointers
// advance by one plane per step instead of being recomputed, and each plane is
// loaded one step ahead only (fewer registers, more resident warps).
template <class Tr, int V, int NEMU>
__device__ __forceinline__ void plain_march_shallow(const typename Tr::S* __restrict__ A,
                                            typename Tr::S* __restrict__ B, const Geom& g,
                                            int k0, int k1, int x0, int y, int lane,
                                            bool loadable, const bool (&interior)[V],
                                            bool all_interior, bool left_ok, bool right_ok,
                                            long long row, uint32_t one) {
    using C = typename Tr::C;
    const unsigned FULL = 0xffffffffu;
    const C c6 = Tr::sixth();
    auto add = [one](int idx, int nemu, C a, C b) -> C {
        if constexpr (NEMU > 0) {
            if (idx < nemu) return add_pos_exact_f(a, b, one);
        }
        return Tr::add(a, b);
    };
    // per cell: inside the row allocation (the cell past nx is the boundary value
    // that the neighbouring lane needs, so a partly outside vector still loads)
    bool okl[V];
#pragma unroll
    for (int e = 0; e < V; ++e) okl[e] = (x0 + e) < g.px;
    auto load = [&](const typename Tr::S* p, C (&out)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = okl[e] ? Tr::ld(__ldg(p + e)) : C(0);
    };

    const long long plane = g.plane, px = g.px;
    const typename Tr::S* pa = A + row + plane * k0;  // (x0, y, k) of A
    typename Tr::S* pb = B + row + plane * k0;        // (x0, y, k) of B
    C dn[V], ct[V], up[V], no[V], so[V];
    load(pa - plane, dn);
    load(pa, ct);

    auto plane_step = [&](int nemu) {
        load(pa + plane, up);
        load(pa - px, no);
        load(pa + px, so);
        C left = __shfl_up_sync(FULL, ct[V - 1], 1);
        C right = __shfl_down_sync(FULL, ct[0], 1);
        if (lane == 0) left = left_ok ? Tr::ld(__ldg(pa - 1)) : C(0);
        if (lane == 31) right = right_ok ? Tr::ld(__ldg(pa + V)) : C(0);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const C l = (e == 0) ? left : ct[e - 1];
            const C r = (e == V - 1) ? right : ct[e + 1];
            C sum = add(0, nemu, l, r);
            sum = add(1, nemu, sum, no[e]);
            sum = add(2, nemu, sum, so[e]);
            sum = add(3, nemu, sum, dn[e]);
            sum = add(4, nemu, sum, up[e]);
            if (interior[e]) pb[e] = Tr::st(Tr::mul(sum, c6));
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dn[e] = ct[e];
            ct[e] = up[e];
        }
        pa += plane;
        pb += plane;
    };
    constexpr int kEven = NEMU / 2, kOdd = (NEMU + 1) / 2;
    int k = k0;
#pragma unroll 1
    for (; k + 1 <= k1; k += 2) {
        plane_step(kEven);
        plane_step(kOdd);
    }
    if (k <= k1) plane_step(kEven);
    (void)all_interior;
    (void)loadable;
}

// NEMU >= kAccBase (FP64): NEMU = kAccBase + K + 8 F; the first K of the five additions of
// every update run through the unpacked exact accumulator of emusum.cuh; a warp
// with a lane whose exponent gaps leave that routine's window recomputes those
// additions on the FP64 unit.  The other additions and the product stay on the
// FP64 unit.  F selects the form of the word arithmetic (emusum.cuh).
constexpr int kAccBase = 16;

template <class Tr, int V, int K, int F>
__device__ __forceinline__ void plain_march_acc(const double* __restrict__ A,
                                                double* __restrict__ B, const Geom& g, int k0,
                                                int k1, int x0, int lane,
                                                const bool (&interior)[V], bool left_ok,
                                                bool right_ok, long long row, uint32_t one) {
    static_assert(K >= 1 && K <= 5, "1..5 additions on the integer pipes");
    const emusum::Mul km = emusum::make_mul(one);
    const unsigned FULL = 0xffffffffu;
    const double c6 = Tr::sixth();
    bool okl[V];
#pragma unroll
    for (int e = 0; e < V; ++e) okl[e] = (x0 + e) < g.px;
    auto load = [&](const double* p, double (&out)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = okl[e] ? __ldg(p + e) : 0.0;
    };
    const long long plane = g.plane, px = g.px;
    const double* pa = A + row + plane * k0;
    double* pb = B + row + plane * k0;
    double dn[V], ct[V], up[V], no[V], so[V];
    load(pa - plane, dn);
    load(pa, ct);
    // two planes per iteration: the two planes' integer-pipe chains interleave
    // (512^3: 208.9 GLUP/s against 201.9 with one plane per iteration, at the same
    // 48 registers)
#pragma unroll 2
    for (int k = k0; k <= k1; ++k) {
        load(pa + plane, up);
        load(pa - px, no);
        load(pa + px, so);
        double left = __shfl_up_sync(FULL, ct[V - 1], 1);
        double right = __shfl_down_sync(FULL, ct[0], 1);
        if (lane == 0) left = left_ok ? __ldg(pa - 1) : 0.0;
        if (lane == 31) right = right_ok ? __ldg(pa + V) : 0.0;
        double x[V][6];
        emusum::Words acc[V];
        uint32_t bad = 0;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            x[e][0] = (e == 0) ? left : ct[e - 1];
            x[e][1] = (e == V - 1) ? right : ct[e + 1];
            x[e][2] = no[e];
            x[e][3] = so[e];
            x[e][4] = dn[e];
            x[e][5] = up[e];
            acc[e] = emusum::first_w<F>(emusum::unpack_w(x[e][0], km),
                                        emusum::unpack_w(x[e][1], km), km);
#pragma unroll
            for (int i = 2; i <= K; ++i)
                emusum::add_w<F>(acc[e], emusum::unpack_w(x[e][i], km), km);
            // cells outside the interior are never stored: their gaps do not count
            if (interior[e]) bad |= acc[e].bad;
        }
        double s[V];
        if (__any_sync(FULL, bad != 0u)) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
                s[e] = __dadd_rn(x[e][0], x[e][1]);
#pragma unroll
                for (int i = 2; i <= K; ++i) s[e] = __dadd_rn(s[e], x[e][i]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) s[e] = emusum::pack_w(acc[e], km);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
#pragma unroll
            for (int i = K + 1; i <= 5; ++i) s[e] = __dadd_rn(s[e], x[e][i]);
            if (interior[e]) pb[e] = __dmul_rn(s[e], c6);
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dn[e] = ct[e];
            ct[e] = up[e];
        }
        pa += plane;
        pb += plane;
    }
}

// `fast` (FP64, NEMU > 0): device flag written by range_check_kernel; when it is
// set every value of A lies in [2^-1000, 2^1000], and by the maximum principle of
// the averaging sweep so does every later value, so the emulated additions are
// valid for the whole call.
template <class Tr, int V, int WY, int NEMU>
__device__ __forceinline__ void plain_sweep_body(const typename Tr::S* __restrict__ A,
                                                 typename Tr::S* __restrict__ B, const Geom& g,
                                                 const int kchunk, const int* __restrict__ fast,
                                                 const uint32_t one) {
    // FP64 and V == 1: interior-aligned cells (scalar loads); else 16-byte vectors
    constexpr int XOFF = (V == 1 || sizeof(typename Tr::S) == 8) ? 1 : 0;
    const int lane = threadIdx.x;
    const int x0 = XOFF + (int)(blockIdx.x * 32 + lane) * V;
    const int y = 1 + (int)(blockIdx.y * WY + threadIdx.y);
    if (y > g.ny) return;  // uniform over the warp
    const int k0 = 1 + (int)blockIdx.z * kchunk;
    if (k0 > g.nz) return;
    const int k1 = min(g.nz, k0 + kchunk - 1);

    // the lane's vector lies inside the row allocation (needed for shuffles even
    // when none of its cells is interior); the FP64 march loads cell by cell, so
    // there a vector that runs past the row still updates its interior cells
    const bool loadable = (x0 + V) <= g.px;
    constexpr bool kPerCellLoads = sizeof(typename Tr::S) == 8;
    bool interior[V];
    bool all_interior = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        interior[e] = (kPerCellLoads || loadable) && (x0 + e >= 1) && (x0 + e <= g.nx);
        all_interior = all_interior && interior[e];
    }
    const bool left_ok = (x0 >= 1);
    const bool right_ok = (x0 + V) < g.px;
    const long long row = g.lin(x0 < g.px ? x0 : 0, y, 0);

    if constexpr (sizeof(typename Tr::S) == 8 && NEMU >= kAccBase) {
        if (fast != nullptr && *fast)
            plain_march_acc<Tr, V, ((NEMU - kAccBase) & 7), (((NEMU - kAccBase) / 8) & 3)>(
                A, B, g, k0, k1, x0, lane, interior, left_ok, right_ok, row, one);
        else
            plain_march_shallow<Tr, V, 0>(A, B, g, k0, k1, x0, y, lane, loadable, interior,
                                          all_interior, left_ok, right_ok, row, one);
    } else if constexpr (sizeof(typename Tr::S) == 8) {
        if (NEMU > 0 && fast != nullptr && *fast)
            plain_march_shallow<Tr, V, NEMU>(A, B, g, k0, k1, x0, y, lane, loadable, interior,
                                             all_interior, left_ok, right_ok, row, one);
        else
            plain_march_shallow<Tr, V, 0>(A, B, g, k0, k1, x0, y, lane, loadable, interior,
                                          all_interior, left_ok, right_ok, row, one);
    } else {
        plain_march<Tr, V>(A, B, g, k0, k1, lane, loadable, interior, all_interior, left_ok,
                           right_ok, row);
    }
}

template <class Tr, int V, int WY, int NEMU>
__global__ void __launch_bounds__(32 * WY)
    plain_sweep_kernel(const typename Tr::S* __restrict__ A, typename Tr::S* __restrict__ B,
                       const Geom g, const int kchunk, const int* __restrict__ fast,
                       const uint32_t one) {
    plain_sweep_body<Tr, V, WY, NEMU>(A, B, g, kchunk, fast, one);
}

// The same sweep compiled for at least 1280 resident threads per SM (so at most
// 51 registers a thread): variant codes 48 and above, whose register demand
// otherwise costs resident warps (the accumulator forms).
template <class Tr, int V, int WY, int NEMU>
__global__ void __launch_bounds__(32 * WY, (1280 / (32 * WY) > 0 ? 1280 / (32 * WY) : 1))
    plain_sweep_kernel_capped(const typename Tr::S* __restrict__ A,
                              typename Tr::S* __restrict__ B, const Geom g, const int kchunk,
                              const int* __restrict__ fast, const uint32_t one) {
    plain_sweep_body<Tr, V, WY, NEMU>(A, B, g, kchunk, fast, one);
}

}  // namespace jac
