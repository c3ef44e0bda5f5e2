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

namespace jac {

template <class Tr, int V>
__device__ __forceinline__ void load_vec(const typename Tr::S* __restrict__ p, bool ok,
                                         typename Tr::C (&out)[V]) {
    using S = typename Tr::S;
    if (ok) {
        const Vec<S, V> t = ldg_vec<S, V>(p);
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = Tr::ld(t.v[e]);
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = 0;
    }
}

// The sweep of one chunk, with the first NEMU of the five additions done by
// add_pos_exact (FP64 only; NEMU = 0: all on the FP64 unit).  NEMU is counted in
// half additions: an odd NEMU does NEMU/2 on even planes and NEMU/2 + 1 on odd
// planes, which balances the FP64 and integer pipes between whole splits.
// Software-pipelined: while plane k is computed, plane k+3 (the stream from HBM)
// and the in-plane neighbours of plane k+1 are already being loaded, so each
// thread keeps two steps of loads in flight.
template <class Tr, int V, int NEMU>
__device__ __forceinline__ void plain_march(const typename Tr::S* __restrict__ A,
                                            typename Tr::S* __restrict__ B, const Geom& g,
                                            int k0, int k1, int x0, int y, int lane,
                                            bool loadable, const bool (&interior)[V],
                                            bool all_interior, bool left_ok, bool right_ok,
                                            long long row) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    const unsigned FULL = 0xffffffffu;
    const C c6 = Tr::sixth();
    auto add = [](int idx, int nemu, C a, C b) -> C {
        if constexpr (NEMU > 0) {
            if (idx < nemu) return add_pos_exact(a, b);
        }
        return Tr::add(a, b);
    };
    const int ktop = g.nz + 1;  // last plane in the array
    auto edge_l = [&](int k) -> C {
        return (lane == 0 && left_ok) ? Tr::ld(__ldg(A + row + g.plane * k - 1)) : C(0);
    };
    auto edge_r = [&](int k) -> C {
        return (lane == 31 && right_ok) ? Tr::ld(__ldg(A + row + g.plane * k + V)) : C(0);
    };

    // streamed values are kept in storage format (bf16 stays 16-bit) and
    // converted when used
    using VS = Vec<S, V>;
    auto ldv = [&](long long off) -> VS {
        if (loadable) return ldg_vec<S, V>(A + off);
        VS z;
#pragma unroll
        for (int e = 0; e < V; ++e) z.v[e] = S(0);
        return z;
    };
    VS dn = ldv(row + g.plane * (k0 - 1));
    VS ct = ldv(row + g.plane * k0);
    VS up = ldv(row + g.plane * min(k0 + 1, ktop));
    VS up2 = ldv(row + g.plane * min(k0 + 2, ktop));
    VS no = ldv(row + g.plane * k0 - g.px);
    VS so = ldv(row + g.plane * k0 + g.px);
    C el = edge_l(k0), er = edge_r(k0);

    auto plane_step = [&](int k, int nemu) {
        // loads for the next steps first
        const int kn = min(k + 1, ktop);
        const VS up3 = ldv(row + g.plane * min(k + 3, ktop));
        const VS no2 = ldv(row + g.plane * kn - g.px);
        const VS so2 = ldv(row + g.plane * kn + g.px);
        const C el2 = edge_l(kn), er2 = edge_r(kn);

        C left = __shfl_up_sync(FULL, Tr::ld(ct.v[V - 1]), 1);
        C right = __shfl_down_sync(FULL, Tr::ld(ct.v[0]), 1);
        if (lane == 0) left = el;
        if (lane == 31) right = er;
        VS outv;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const C l = (e == 0) ? left : Tr::ld(ct.v[e - 1]);
            const C r = (e == V - 1) ? right : Tr::ld(ct.v[e + 1]);
            C s = add(0, nemu, l, r);
            s = add(1, nemu, s, Tr::ld(no.v[e]));
            s = add(2, nemu, s, Tr::ld(so.v[e]));
            s = add(3, nemu, s, Tr::ld(dn.v[e]));
            s = add(4, nemu, s, Tr::ld(up.v[e]));
            outv.v[e] = Tr::st(Tr::mul(s, c6));
        }
        const long long base = row + g.plane * k;
        if (all_interior) {
            *reinterpret_cast<VS*>(B + base) = outv;
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (interior[e]) B[base + e] = outv.v[e];
        }
        dn = ct;
        ct = up;
        up = up2;
        up2 = up3;
        no = no2;
        so = so2;
        el = el2;
        er = er2;
    };
    constexpr int kEven = NEMU / 2, kOdd = (NEMU + 1) / 2;
    int k = k0;
#pragma unroll 1
    for (; k + 1 <= k1; k += 2) {
        plane_step(k, kEven);
        plane_step(k + 1, kOdd);
    }
    if (k <= k1) plane_step(k, kEven);
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

// `fast` (FP64, NEMU > 0): device flag written by range_check_kernel; when it is
// set every value of A lies in [2^-1000, 2^1000], and by the maximum principle of
// the averaging sweep so does every later value, so the emulated additions are
// valid for the whole call.
template <class Tr, int V, int WY, int NEMU>
__global__ void __launch_bounds__(32 * WY)
    plain_sweep_kernel(const typename Tr::S* __restrict__ A, typename Tr::S* __restrict__ B,
                       const Geom g, const int kchunk, const int* __restrict__ fast,
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
    // when none of its cells is interior)
    const bool loadable = (x0 + V) <= g.px;
    bool interior[V];
    bool all_interior = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        interior[e] = loadable && (x0 + e >= 1) && (x0 + e <= g.nx);
        all_interior = all_interior && interior[e];
    }
    const bool left_ok = (x0 >= 1);
    const bool right_ok = (x0 + V) < g.px;
    const long long row = g.lin(x0 < g.px ? x0 : 0, y, 0);

    if constexpr (sizeof(typename Tr::S) == 8) {
        if (NEMU > 0 && fast != nullptr && *fast)
            plain_march_shallow<Tr, V, NEMU>(A, B, g, k0, k1, x0, y, lane, loadable, interior,
                                             all_interior, left_ok, right_ok, row, one);
        else
            plain_march_shallow<Tr, V, 0>(A, B, g, k0, k1, x0, y, lane, loadable, interior,
                                          all_interior, left_ok, right_ok, row, one);
    } else {
        plain_march<Tr, V, 0>(A, B, g, k0, k1, x0, y, lane, loadable, interior, all_interior,
                              left_ok, right_ok, row);
    }
}

}  // namespace jac
