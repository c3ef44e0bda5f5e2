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
// The k-march is unrolled by 6, the period of the ring slot (NS = 6), of the
// level buffers' parity (2) and of the register rotation (3), so every shared-
// memory offset and register role is a compile-time constant.  Tiles whose
// extended region lies inside the interior in x and y take a path without the
// per-cell boundary selects.
//
// Modes: MODE_PLAIN (Eq. 1), MODE_RHS (the refinement's correction sweep, adds
// rho before the product; rho's planes arrive by TMA beside the grid's).  MODE_ADJ
// names the adjoint operation for the planner: the adjoint sweep is the plain
// sweep on lambda with a zero boundary, so it runs on the MODE_PLAIN kernels, and
// its boundary-gradient face values come from a separate band kernel (band.cu).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "emu.cuh"
#include "emusum.cuh"

namespace jac {

enum { MODE_PLAIN = 0, MODE_RHS = 1, MODE_ADJ = 2 };

constexpr int kRing = 6;  // TMA ring slots (the unroll period)
constexpr int kAccBaseTB = 16;  // EMU >= this: accumulator with EMU - 16 additions
#ifndef JAC_PACKED_F32
#define JAC_PACKED_F32 1
#endif
constexpr bool kPackedF32 = JAC_PACKED_F32 != 0;  // packed FP32 pairs in the level updates

struct TBArgs {
    Geom g;
    void* dst;          // output grid of the pass (level T)
    void* grad;         // gradient grid (only the never-executed hook below names it)
    int ox;             // output tile width (multiple of the TMA alignment)
    int x0_first;       // x origin of tile 0's extended tile (aligned, may be < 0)
    int kz;             // output k-planes per CTA
    int* status;        // device status word (timeouts)
    const int* fast;    // FP64 (EMU > 0): range flag set by range_check_kernel, or null
    uint32_t one;       // a runtime 1 (the integer-pipe additions' multiplier)
};

// Shared memory of one CTA: mbarriers (HEADER), the TMA ring (NS planes), the
// level buffers (two per level 1..T-1), one guard row, and for correction sweeps
// the rho ring (NSR planes).  The rows just above and below the extended tile are
// read without clamping (their values only reach cells outside the valid region
// of the level being computed); the header's tail and the guard row keep those
// reads inside the allocation.
template <int V, int NW, int T, int NS, class S, int NSR = 0>
struct TBLayout {
    static constexpr int EX = 32 * V;
    static constexpr int EY = NW;
    static constexpr int PLANE = EX * EY;
    static constexpr int NLB = (T > 1) ? 2 * (T - 1) : 0;  // level buffers
    static constexpr int HEADER = 1024;                      // mbarriers, aligned
    static_assert(EX * sizeof(S) + 64 <= HEADER, "guard row overlaps the mbarriers");
    static constexpr size_t RHO_OFF =
        HEADER + (size_t)(NS + NLB) * PLANE * sizeof(S) + (size_t)EX * sizeof(S);
    static_assert(RHO_OFF % 128 == 0, "TMA destinations must stay 128-byte aligned");
    static constexpr size_t bytes() { return RHO_OFF + (size_t)NSR * PLANE * sizeof(S); }
};

// Slots of the rho ring for depth T (correction sweeps): rho plane P is issued
// with grid plane P, NS - 1 steps before level 1 reads it, and level T reads it
// T - 1 steps after that, so NS + T slots keep it until its last reader is done.
template <int MODE, int NS, int T>
constexpr int rho_slots() {
    return MODE == MODE_RHS ? NS + T : 0;
}

template <int N>
using IC = std::integral_constant<int, N>;

// One output tile of one temporally-blocked pass.  `smem` is the CTA's dynamic
// shared memory (TBLayout), `s_abort` a shared flag.  Returns false when a TMA
// wait timed out (status already recorded).  All threads of the CTA call it.
// EMU (FP64 only): the first EMU of the five additions of every update run as
// exact binary64 additions on the integer pipes (emu.cuh), valid when every
// value of the pass lies in [2^-1000, 2^1000]; the results are the same bits.
template <class Tr, int V, int NW, int T, int MODE, bool FAST, int EMU = 0>
__device__ __forceinline__ bool tb_tile(const CUtensorMap* tmap, const CUtensorMap* tmap_rho,
                                        const TBArgs& a, int bx, int by, int bz,
                                        unsigned char* smem, int* s_abort) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    constexpr int NS = kRing;
    constexpr int NSR = rho_slots<MODE, NS, T>();
    using L = TBLayout<V, NW, T, NS, S, NSR>;
    constexpr int EX = L::EX, EY = L::EY, PLANE = L::PLANE;
    constexpr uint32_t kPlaneBytes = PLANE * sizeof(S);
    // bytes landing per ring slot: the grid plane, and the rho plane of the same k
    constexpr uint32_t kSlotBytes = (NSR > 0 ? 2 : 1) * kPlaneBytes;
    constexpr int OY = EY - 2 * T;
    static_assert(OY >= 1, "tile too small for the depth");
    // level values are storage values already (every level is rounded): stores may
    // take their bits without a conversion (used where it measured faster)
    constexpr bool kExactStore = T >= 2 && MODE == MODE_PLAIN;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    S* ring = reinterpret_cast<S*>(smem + L::HEADER);
    S* lvl = ring + NS * PLANE;
    S* rring = reinterpret_cast<S*>(smem + L::RHO_OFF);

    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const Geom& g = a.g;
    const int X0 = a.x0_first + bx * a.ox;
    const int Y0 = 1 - T + by * OY;
    const int ox0 = X0 + T, oy0 = Y0 + T;
    const int kz0 = 1 + bz * a.kz;
    const int kz1 = min(g.nz + 1, kz0 + a.kz);
    const int Zlo = kz0 - T;
    const int M = (kz1 - kz0) + 2 * T;
    const int gy = Y0 + w;
    const int gx0 = X0 + lane * V;
    const int smax = min(w, EY - 1 - w);  // deepest level this warp's row takes part in

    bool inxy[V], outxy[V];
    bool all_out = true, all_in = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int x = gx0 + e;
        inxy[e] = FAST || ((x >= 1) && (x <= g.nx) && (gy >= 1) && (gy <= g.ny));
        outxy[e] = inxy[e] && (x >= ox0) && (x < ox0 + a.ox) && (x <= g.nx) && (gy >= oy0) &&
                   (gy < oy0 + OY) && (gy <= g.ny) && (x >= 1) && (gy >= 1);
        all_out = all_out && outxy[e];
        all_in = all_in && inxy[e];
    }

    if (tid == 0) {
#pragma unroll 1
        for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0;  // planes issued so far (thread 0 only)
    int rslot = 0;   // rho slot of plane Zlo + issued (thread 0 only)
    if (tid == 0) {
#pragma unroll 1
        for (int i = 0; i < NS && i < M; ++i) {
            mbar_arrive_expect_tx(&bars[i], kSlotBytes);
            tma_load_3d(ring + i * PLANE, tmap, &bars[i], X0, Y0, Zlo + i);
            if (NSR > 0) tma_load_3d(rring + i * PLANE, tmap_rho, &bars[i], X0, Y0, Zlo + i);
        }
        issued = min(NS, M);
        rslot = issued;  // NS < NSR
    }

    C r[T][3][V];                                 // per level s < T: 3 planes of level s
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int e = 0; e < V; ++e) r[s][j][e] = C(0);

    const C c6 = Tr::sixth();
    S* dst = static_cast<S*>(a.dst);
    const long long rowoff = (long long)gy * g.px + gx0;  // valid only when used
    const int mycol = w * EX + lane * V;
    // Never executed: a per-level reduction hook (global reductions into the
    // gradient grid, unreachable in every mode), called at every level of the
    // k-march.  Kept because its presence changes how nvcc 13.0 schedules the
    // k-march: measured on GB300 at 512^3, FP32 depth 3 runs at 993 GLUP/s with it
    // and 792 without it (bf16 878 / 687; the same loss with an empty hook or with
    // the hook's loop removed).  The reason is not known; the results are the same
    // bits either way.
    S* grad = static_cast<S*>(a.grad);
    constexpr uint32_t fmask = 0;
    constexpr bool xy_face = false;
    auto adj_acc = [&](const C* v, int p) {
        if constexpr (true) return;
        const bool zlo = p == 1, zhi = p == g.nz;
        if (FAST ? !(zlo || zhi) : (!xy_face && !(zlo || zhi))) return;
        if (p < kz0 || p >= kz1 || fmask == 0u) return;
        C* gacc = reinterpret_cast<C*>(grad);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const uint32_t f = (fmask >> (5 * (V - 1 - e))) & 31u;
            if (!(f & 16u)) continue;
            const C cv = Tr::mul(c6, v[e]);
            const int x = gx0 + e;
            if (f & 1u) atomicAdd(gacc + g.lin(0, gy, p), cv);
            if (f & 2u) atomicAdd(gacc + g.lin(g.nx + 1, gy, p), cv);
            if (f & 4u) atomicAdd(gacc + g.lin(x, 0, p), cv);
            if (f & 8u) atomicAdd(gacc + g.lin(x, g.ny + 1, p), cv);
            if (zlo) atomicAdd(gacc + g.lin(x, gy, 0), cv);
            if (zhi) atomicAdd(gacc + g.lin(x, gy, g.nz + 1), cv);
        }
    };

    // EMU >= kAccBaseTB (FP64 plain sweeps): the first EMU - kAccBaseTB additions
    // of every update through the exact accumulator of emusum.cuh instead
    constexpr bool kAcc = EMU >= kAccBaseTB && std::is_same<C, double>::value &&
                          MODE == MODE_PLAIN;
    // FP32 arithmetic (FP32 and bf16 storage) on pairs of cells
    // (FP32 storage, depths 1-2, CTAs of at most 16 warps: measured 707 / 950 against
    // 693 / 924 GLUP/s at 512^3; 1024-thread kernels spill with it, bf16 storage ran
    // slower, and depth 3 on 24 / 20 / 16-warp tiles, which fit it without spills,
    // ran at 926 / 850 / 707 against 993 for the unpacked 32-warp tile)
    constexpr bool kPacked = kPackedF32 && std::is_same<S, float>::value && V % 2 == 0 &&
                             T <= 2 && NW <= 16;
    // addition number idx (0..4) of an update: the first EMU on the integer pipes
    const uint32_t one = a.one;
    auto add = [one](int idx, C x, C y) -> C {
        if constexpr (EMU > 0 && EMU < kAccBaseTB && std::is_same<C, double>::value) {
            if (idx < EMU) return add_pos_exact_f(x, y, one);
        }
        return Tr::add(x, y);
    };
    (void)one;

    int cur_m = 0;  // step being executed (for the clean-up after a timeout)
    int rs = 0;     // rho slot of plane Zlo + m (MODE_RHS)
    // One step of the k-march; PH = m mod 6 fixes slot, parity and rotation.
    auto step = [&](auto ph, int m) -> bool {
        constexpr int PH = decltype(ph)::value;
        cur_m = m;
        constexpr int SLOT = PH % NS;
        constexpr int PSLOT = (PH + NS - 1) % NS;  // slot of plane Zlo+m-1
        constexpr int PAR = PH & 1;
        constexpr int OLD = PH % 3, CUR = (PH + 1) % 3, NEW = (PH + 2) % 3;
        if (!mbar_wait_bounded(&bars[SLOT], (uint32_t)((m / NS) & 1))) {
            atomicOr(a.status, kStatusTimeout);
            *s_abort = 1;
        }
        // ---- level 0: plane Zlo + m, own cells
        const int p0 = Zlo + m;
        {
            const Vec<S, V> t = *reinterpret_cast<const Vec<S, V>*>(ring + SLOT * PLANE + mycol);
#pragma unroll
            for (int e = 0; e < V; ++e) r[0][NEW][e] = Tr::ld(t.v[e]);
            if (MODE == MODE_ADJ) adj_acc(r[0][NEW], p0);
        }
        // ---- levels 1..T
#pragma unroll
        for (int s = 1; s <= T; ++s) {
            if (m < s) continue;     // pipeline fill
            if (s > smax) continue;  // row outside level s's region
            const int q = p0 - s;
            const bool zin = (q >= 1) && (q <= g.nz);
            const S* nb = (s == 1) ? ring + PSLOT * PLANE
                                   : lvl + ((s - 2) * 2 + (PAR ^ 1)) * PLANE;
            const Vec<S, V> vn = *reinterpret_cast<const Vec<S, V>*>(nb + mycol - EX);
            const Vec<S, V> vs = *reinterpret_cast<const Vec<S, V>*>(nb + mycol + EX);
            // rho at plane q (MODE_RHS): the rho slot of plane Zlo + m - s
            Vec<S, V> vr;
            if (MODE == MODE_RHS) {
                const int sl = (rs >= s) ? rs - s : rs - s + (NSR > 0 ? NSR : 1);
                vr = *reinterpret_cast<const Vec<S, V>*>(rring + sl * PLANE + mycol);
            }
            const C left = __shfl_up_sync(FULL, r[s - 1][CUR][V - 1], 1);
            const C right = __shfl_down_sync(FULL, r[s - 1][CUR][0], 1);
            C out[V];
            if (zin) {
                C val[V];
                if constexpr (kAcc) {
                    // the first K additions through the exact accumulator; a warp
                    // with an interior lane outside its window redoes them on the
                    // FP64 unit (lanes off the interior keep their old values)
                    constexpr int K = EMU - kAccBaseTB;
                    C x[V][6];
                    emusum::Acc acc[V];
                    uint32_t bad = 0;
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        x[e][0] = (e == 0) ? left : r[s - 1][CUR][e - 1];
                        x[e][1] = (e == V - 1) ? right : r[s - 1][CUR][e + 1];
                        x[e][2] = Tr::ld(vn.v[e]);
                        x[e][3] = Tr::ld(vs.v[e]);
                        x[e][4] = r[s - 1][OLD][e];
                        x[e][5] = r[s - 1][NEW][e];
                        // the 64-bit form: fewer registers than the word form here,
                        // and faster at every depth measured
                        acc[e] = emusum::first(emusum::unpack(x[e][0]), emusum::unpack(x[e][1]));
#pragma unroll
                        for (int i = 2; i <= K; ++i) emusum::add(acc[e], emusum::unpack(x[e][i]));
                        if (FAST || inxy[e]) bad |= acc[e].bad;
                    }
                    C sum[V];
                    if (__any_sync(FULL, bad != 0u)) {
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            sum[e] = Tr::add(x[e][0], x[e][1]);
#pragma unroll
                            for (int i = 2; i <= K; ++i) sum[e] = Tr::add(sum[e], x[e][i]);
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < V; ++e) sum[e] = emusum::pack(acc[e]);
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e) {
#pragma unroll
                        for (int i = K + 1; i <= 5; ++i) sum[e] = Tr::add(sum[e], x[e][i]);
                        val[e] = Tr::mul(sum[e], c6);
                    }
                } else if constexpr (kPacked) {
                    // FP32 arithmetic on cell pairs (e, e+1): the same operand order
                    // per cell, two lanes of one packed instruction
                    const unsigned long long c6p = f2_pack(c6, c6);
#pragma unroll
                    for (int e = 0; e < V; e += 2) {
                        const C l0 = (e == 0) ? left : r[s - 1][CUR][e - 1];
                        const C r1 = (e + 2 == V) ? right : r[s - 1][CUR][e + 2];
                        unsigned long long sp =
                            f2_add(f2_pack(l0, r[s - 1][CUR][e]),
                                   f2_pack(r[s - 1][CUR][e + 1], r1));
                        sp = f2_add(sp, f2_pack(Tr::ld(vn.v[e]), Tr::ld(vn.v[e + 1])));
                        sp = f2_add(sp, f2_pack(Tr::ld(vs.v[e]), Tr::ld(vs.v[e + 1])));
                        sp = f2_add(sp, f2_pack(r[s - 1][OLD][e], r[s - 1][OLD][e + 1]));
                        sp = f2_add(sp, f2_pack(r[s - 1][NEW][e], r[s - 1][NEW][e + 1]));
                        if (MODE == MODE_RHS)
                            sp = f2_add(sp, f2_pack(Tr::ld(vr.v[e]), Tr::ld(vr.v[e + 1])));
                        f2_unpack(f2_mul(sp, c6p), val[e], val[e + 1]);
                    }
                } else {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const C l = (e == 0) ? left : r[s - 1][CUR][e - 1];
                    const C rr = (e == V - 1) ? right : r[s - 1][CUR][e + 1];
                    C sum = add(0, l, rr);
                    sum = add(1, sum, Tr::ld(vn.v[e]));
                    sum = add(2, sum, Tr::ld(vs.v[e]));
                    sum = add(3, sum, r[s - 1][OLD][e]);
                    sum = add(4, sum, r[s - 1][NEW][e]);
                    if (MODE == MODE_RHS) sum = Tr::add(sum, Tr::ld(vr.v[e]));
                    val[e] = Tr::mul(sum, c6);
                }
                }
                // round to storage precision (plain bf16 sweeps of depth >= 2: two
                // values per conversion; the one-value form measured faster at depth
                // 1 and, by two registers that cost a CTA per SM, for the bf16
                // correction sweep at depth 2)
                if constexpr (V % 2 == 0 && T >= 2 && MODE == MODE_PLAIN) {
#pragma unroll
                    for (int e = 0; e < V; e += 2) Tr::rnd_pair(val[e], val[e + 1]);
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e) val[e] = Tr::rnd(val[e]);
                }
#pragma unroll
                for (int e = 0; e < V; ++e) out[e] = (FAST || inxy[e]) ? val[e] : r[s - 1][CUR][e];
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) out[e] = r[s - 1][CUR][e];
            }
            if (s < T) {
                Vec<S, V> o;
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    r[s < T ? s : 0][NEW][e] = out[e];
                    o.v[e] = kExactStore ? Tr::st_exact(out[e]) : Tr::st(out[e]);
                }
                *reinterpret_cast<Vec<S, V>*>(lvl + ((s - 1) * 2 + PAR) * PLANE + mycol) = o;
                if (MODE == MODE_ADJ) adj_acc(out, q);
            } else if (q >= kz0 && q < kz1) {
                const long long o = g.plane * q + rowoff;
                if (all_out) {
                    Vec<S, V> ov;
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        ov.v[e] = kExactStore ? Tr::st_exact(out[e]) : Tr::st(out[e]);
                    *reinterpret_cast<Vec<S, V>*>(dst + o) = ov;
                } else {
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (outxy[e])
                            dst[o + e] = kExactStore ? Tr::st_exact(out[e]) : Tr::st(out[e]);
                }
            }
        }
        __syncthreads();
        if (*s_abort) return false;
        // the slot of plane Zlo+m-1 is free now: refill it with plane Zlo+m-1+NS,
        // and the rho ring's next slot with rho of the same k (see rho_slots)
        if (tid == 0 && m >= 1 && issued < M) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bars[PSLOT], kSlotBytes);
            tma_load_3d(ring + PSLOT * PLANE, tmap, &bars[PSLOT], X0, Y0, Zlo + issued);
            if (NSR > 0) {
                tma_load_3d(rring + rslot * PLANE, tmap_rho, &bars[PSLOT], X0, Y0,
                            Zlo + issued);
                rslot = (rslot + 1 == NSR) ? 0 : rslot + 1;
            }
            ++issued;
        }
        if (MODE == MODE_RHS) rs = (rs + 1 == NSR) ? 0 : rs + 1;
        return true;
    };

    int m = 0;
    bool ok = true;
#pragma unroll 1
    for (; m + 6 <= M; m += 6) {
        if (!step(IC<0>{}, m) || !step(IC<1>{}, m + 1) || !step(IC<2>{}, m + 2) ||
            !step(IC<3>{}, m + 3) || !step(IC<4>{}, m + 4) || !step(IC<5>{}, m + 5)) {
            ok = false;
            break;
        }
    }
    if (ok) {
        // remainder (M mod 6 steps), same phases
        const int left = M - m;
        if (left > 0) ok = step(IC<0>{}, m);
        if (ok && left > 1) ok = step(IC<1>{}, m + 1);
        if (ok && left > 2) ok = step(IC<2>{}, m + 2);
        if (ok && left > 3) ok = step(IC<3>{}, m + 3);
        if (ok && left > 4) ok = step(IC<4>{}, m + 4);
    }
    if (!ok && tid == 0) {
        // timed out: let the copies still in flight (planes cur_m .. issued-1) land
        // before the shared memory is reused or released (each wait bounded again)
#pragma unroll 1
        for (int p = cur_m; p < issued; ++p)
            (void)mbar_wait_bounded(&bars[p % NS], (uint32_t)((p / NS) & 1), 500000000ull);
    }
    __syncthreads();
    if (ok && tid == 0) {
#pragma unroll 1
        for (int i = 0; i < NS; ++i) mbar_inval(&bars[i]);
    }
    return ok;
}

// CTA-uniform test: the extended tile lies inside the interior in x and y.
template <int V, int NW, int T>
__device__ __forceinline__ bool tile_inside_xy(const TBArgs& a, int bx, int by) {
    const int X0 = a.x0_first + bx * a.ox;
    const int Y0 = 1 - T + by * (NW - 2 * T);
    return X0 >= 1 && X0 + 32 * V - 1 <= a.g.nx && Y0 >= 1 && Y0 + NW - 1 <= a.g.ny;
}

// EMU > 0 (FP64 plain sweeps): the variant with integer-pipe additions runs when
// the call's range check passed (a.fast set), else every addition stays on the
// FP64 unit; both give the same bits.
template <class Tr, int V, int NW, int T, int MODE, int NS, int EMU = 0>
__global__ void __launch_bounds__(NW * 32, 1)
    tb_sweep_kernel(const __grid_constant__ CUtensorMap tmap,
                    const __grid_constant__ CUtensorMap tmap_rho, const TBArgs a) {
    static_assert(NS == kRing, "the k-march is unrolled by the ring size");
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_abort = 0;
        prefetch_tmap(&tmap);
        if (MODE == MODE_RHS) prefetch_tmap(&tmap_rho);
    }
    const int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    const bool inside = tile_inside_xy<V, NW, T>(a, bx, by);
    if constexpr (EMU > 0) {
        if (a.fast != nullptr && *a.fast) {
            if (inside)
                tb_tile<Tr, V, NW, T, MODE, true, EMU>(&tmap, &tmap_rho, a, bx, by, bz, smem,
                                                       &s_abort);
            else
                tb_tile<Tr, V, NW, T, MODE, false, EMU>(&tmap, &tmap_rho, a, bx, by, bz, smem,
                                                        &s_abort);
            return;
        }
    }
    if (inside)
        tb_tile<Tr, V, NW, T, MODE, true>(&tmap, &tmap_rho, a, bx, by, bz, smem, &s_abort);
    else
        tb_tile<Tr, V, NW, T, MODE, false>(&tmap, &tmap_rho, a, bx, by, bz, smem, &s_abort);
}

}  // namespace jac
