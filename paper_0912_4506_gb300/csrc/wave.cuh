// Pipelined temporal blocking across CTAs: the GPU form of the paper's pipelined
// scheme with relaxed synchronisation (Sect. 1.3, Eq. 3).
//
// In the paper a team of threads shares one cache.  Every block of the grid is
// updated t times in turn, update s by thread s.  Thread s may start its next
// block when thread s-1 is at least d_l blocks ahead and thread s+1 at most d_u
// blocks behind (Eq. 3), which one progress counter per thread tells.  Nothing
// is recomputed: each of the t updates of a block is done once.
//
// Here the team is the whole GPU and the shared cache is the L2:
//  * A work item is one level s (1..t) of one block.  A block is an x-y tile of
//    32V x WY cells (one warp per row, V cells per lane) and kb planes in z.
//  * Levels 1..t-1 live in ring buffers of rp planes each (rp = R kb, full planes
//    in the grid's layout), 512 MB at most (the planner's budget; larger items
//    measured faster than rings held to the L2 size).  Level 0 is the
//    source grid.  Level t is the destination grid, or the source itself for
//    an in-place pass.
//  * One flag per (level, tile, block) marks it done (with the pass's number in
//    the call, so the flags are cleared once per call, not per pass).  An item
//    starts when three things hold.
//    Blocks b-1 .. b+1 of level s-1 of the 3 x 3 tile neighbourhood are done:
//    the lower distance of Eq. 3.  Level s+1 of the neighbourhood has finished
//    reading ring block b-R, whose slot this item overwrites (its readers are
//    blocks b-R-1 .. b-R+1): the upper distance of Eq. 3.  For an in-place pass
//    (s = t), level 1 of the neighbourhood has read every value of the block that
//    the item overwrites (blocks b-1 .. b+1 of level 1).  Counting blocks in z
//    order instead would make a finished item wait for its tile's previous
//    block before it could be marked.
//  * Items are handed out by one atomic ticket in the order (b + sk s, s, tile)
//    with a skew sk >= 1 and R > sk + 1.  In that order every item waits only
//    for items with smaller tickets (its input, level s-1 of block b+1, comes
//    sk - 1 diagonals earlier; the readers of its ring slot R - sk - 1
//    diagonals earlier; in place, level 1 of block b+1 earlier for t >= 2), so
//    a persistent grid of any size makes progress, and with sk = 2 an item's
//    input was handed out a whole diagonal of items before it.  Each wait is
//    bounded in time; a timeout sets the status word and the abort flag, and
//    every CTA leaves.
//  * Ring levels carry the boundary layer like the grids do.  A lane stores
//    every boundary value it loaded (its own non-interior cells, the row above
//    y = 1 and below y = ny, the x = 0 and x = nx+1 edge cells) to the same
//    place in the next level.  The boundary planes z = 0 and z = nz+1 of every
//    level are read from the source grid, whose boundary layer no pass writes.
//
// The levels are read either by TMA into a shared-memory ring (FP32/bf16, the
// default) or by the register march through the coherent path (ld.global.ca;
// FP64): the data was written during this launch by other CTAs, and the GPU-scope
// acquire of the counters makes it visible to every thread of the CTA after the
// job barrier (and to the TMA unit after a proxy fence).
// The arithmetic is Eq. 1 in its operand order, as in every other kernel, so
// results are bit-identical to a sequential sweep loop.
#pragma once

#include "common.cuh"
#include "emusum.cuh"

namespace jac {

struct WaveArgs {
    Geom g;
    const void* src;  // level 0
    void* dst;        // level t (== src for an in-place pass)
    void* ring;       // levels 1..t-1, rp planes each
    int t;            // updates per pass
    int kb;           // planes per block
    int nb;           // blocks along z
    int R;            // ring blocks per level (> sk + 1)
    int sk;           // skew of the ticket order
    int rp;           // ring planes per level (R * kb)
    int ntx, nty;     // tiles
    int nitems;       // t * nb * ntx * nty
    int inplace;
    int* done;        // [t][ntx * nty][nb]: == epoch once (level, tile, block) is done
    int epoch;        // this pass's mark: its index in the call + 1 (flags cleared per call)
    int* ticket;      // next work item
    int* abort;       // set by a wait that ran out
    int* status;      // handle status word (kStatusTimeout)
    const int* fast;  // FP64: the range flag of the integer-pipe additions
    uint32_t one;
    unsigned long long wait_ns;
};

// The plane sequence of the level read (s-1) and the level written (s).
template <class S>
struct WaveLevels {
    const S* sgrid;  // level 0, and the boundary planes of every level
    const S* sring;  // ring of level s-1 (s >= 2)
    S* dgrid;        // destination grid (s == t)
    S* dring;        // ring of level s (s < t)
    long long plane;
    int rp, nz;
    bool s_in_ring, d_in_ring;
    __device__ __forceinline__ const S* src(int k, int sl) const {
        return (s_in_ring && k >= 1 && k <= nz) ? sring + (long long)sl * plane
                                                 : sgrid + (long long)k * plane;
    }
    __device__ __forceinline__ S* dst(int k, int sl) const {
        return d_in_ring ? dring + (long long)sl * plane : dgrid + (long long)k * plane;
    }
    __device__ __forceinline__ int next(int sl) const { return sl + 1 == rp ? 0 : sl + 1; }
    __device__ __forceinline__ int prev(int sl) const { return sl == 0 ? rp - 1 : sl - 1; }
};

// Coherent loads (weak ld.global.ca): never the read-only path, whose cache is
// not kept coherent with stores made during the launch.
template <class S, int V>
__device__ __forceinline__ Vec<S, V> ldca_vec(const S* p) {
    using R = typename RawOf<sizeof(Vec<S, V>)>::T;
    const R r = __ldca(reinterpret_cast<const R*>(p));
    Vec<S, V> out;
    memcpy(&out, &r, sizeof(out));
    return out;
}

// One level of one block, FP32/bf16 storage (16-byte vectors of V cells, x
// origin 0).  The loads of the next step (plane k+2, the rows and edge cells of
// plane k+1) are issued before the arithmetic of step k.  (Loading two steps
// ahead, with the registers that takes, measured slower: the march is bound by
// its resident warps, not by the depth of its loads.)
template <class Tr, int V>
__device__ __forceinline__ void wave_march_vec(const WaveLevels<typename Tr::S>& L,
                                               const Geom& g, int k0, int k1, int x0, int y,
                                               int lane, bool loadable,
                                               const bool (&interior)[V], bool all_interior,
                                               bool left_ok, bool right_ok, long long row) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    using VS = Vec<S, V>;
    const unsigned FULL = 0xffffffffu;
    const C c6 = Tr::sixth();
    const long long px = g.px;
    const bool el_ok = lane == 0 && left_ok, er_ok = lane == 31 && right_ok;
    const bool to_ring = L.d_in_ring;
    const bool row_lo = to_ring && loadable && y == 1;
    const bool row_hi = to_ring && loadable && y == g.ny;
    const bool edge_lo = to_ring && el_ok && x0 == 1;          // cell x = 0
    const bool edge_hi = to_ring && er_ok && x0 + V == g.nx + 1;  // cell x = nx+1
    VS zero;
#pragma unroll
    for (int e = 0; e < V; ++e) zero.v[e] = S(0);
    auto ldv = [&](const S* p, bool ok) -> VS { return ok ? ldca_vec<S, V>(p) : zero; };
    auto lds = [&](const S* p, bool ok) -> S { return ok ? __ldca(p) : S(0); };

    int sl = (k0 - 1) % L.rp;  // ring slot of plane k
    int sln = L.next(sl);      // of plane k+1
    VS dn = ldv(L.src(k0 - 1, L.prev(sl)) + row, loadable);
    const S* pc = L.src(k0, sl) + row;
    VS ct = ldv(pc, loadable);
    VS no = ldv(pc - px, loadable);
    VS so = ldv(pc + px, loadable);
    S el = lds(pc - 1, el_ok), er = lds(pc + V, er_ok);
    const S* pn = L.src(k0 + 1, sln) + row;  // plane k+1
    VS up = ldv(pn, loadable);

#pragma unroll 1
    for (int k = k0; k <= k1; ++k) {
        const bool more = k < k1;  // planes k+1 <= nz and k+2 <= nz+1 exist
        const int sl2 = L.next(sln);
        const S* pn2 = L.src(k + 2, sl2) + row;
        const VS up2 = ldv(pn2, more && loadable);
        const VS no2 = ldv(pn - px, more && loadable);
        const VS so2 = ldv(pn + px, more && loadable);
        const S el2 = lds(pn - 1, more && el_ok);
        const S er2 = lds(pn + V, more && er_ok);

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
            outv.v[e] = interior[e] ? Tr::st(Tr::mul(s, c6)) : ct.v[e];
        }
        S* pd = L.dst(k, sl) + row;
        if (to_ring) {
            // the whole vector: computed cells and the boundary values passed on
            if (loadable) *reinterpret_cast<VS*>(pd) = outv;
            if (row_lo) *reinterpret_cast<VS*>(pd - px) = no;
            if (row_hi) *reinterpret_cast<VS*>(pd + px) = so;
            if (edge_lo) pd[-1] = el;
            if (edge_hi) pd[V] = er;
        } else if (all_interior) {
            *reinterpret_cast<VS*>(pd) = outv;
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (interior[e]) pd[e] = outv.v[e];
        }
        dn = ct;
        ct = up;
        up = up2;
        no = no2;
        so = so2;
        el = el2;
        er = er2;
        pn = pn2;
        sl = sln;
        sln = sl2;
    }
}

// One level of one block, FP64 (interior-aligned cells x0 = 1 + V lane, loaded
// cell by cell).  K > 0: the first K additions of every update go through the
// exact unpacked accumulator of emusum.cuh in word form F, with the same warp-vote
// fallback to the FP64 unit as the streaming sweep; K == 0: all on the FP64 unit.
template <class Tr, int V, int K, int F>
__device__ __forceinline__ void wave_march_f64(const WaveLevels<double>& L, const Geom& g,
                                               int k0, int k1, int x0, int y, int lane,
                                               const bool (&interior)[V], bool left_ok,
                                               bool right_ok, long long row, uint32_t one) {
    static_assert(K >= 0 && K <= 5, "0..5 additions on the integer pipes");
    const unsigned FULL = 0xffffffffu;
    const double c6 = Tr::sixth();
    const long long px = g.px;
    const bool to_ring = L.d_in_ring;
    bool okl[V];
#pragma unroll
    for (int e = 0; e < V; ++e) okl[e] = (x0 + e) < g.px;
    auto load = [&](const double* p, double (&out)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = okl[e] ? __ldca(p + e) : 0.0;
    };
    const bool row_lo = to_ring && y == 1, row_hi = to_ring && y == g.ny;
    const bool edge_lo = to_ring && lane == 0 && left_ok && x0 == 1;
    const bool edge_hi = to_ring && lane == 31 && right_ok && x0 + V == g.nx + 1;

    int sl = (k0 - 1) % L.rp;
    double dn[V], ct[V], up[V], no[V], so[V];
    load(L.src(k0 - 1, L.prev(sl)) + row, dn);
    load(L.src(k0, sl) + row, ct);
#pragma unroll 1
    for (int k = k0; k <= k1; ++k) {
        const int sln = L.next(sl);
        const double* pc = L.src(k, sl) + row;
        load(L.src(k + 1, sln) + row, up);
        load(pc - px, no);
        load(pc + px, so);
        double left = __shfl_up_sync(FULL, ct[V - 1], 1);
        double right = __shfl_down_sync(FULL, ct[0], 1);
        if (lane == 0) left = left_ok ? __ldca(pc - 1) : 0.0;
        if (lane == 31) right = right_ok ? __ldca(pc + V) : 0.0;
        double x[V][6];
#pragma unroll
        for (int e = 0; e < V; ++e) {
            x[e][0] = (e == 0) ? left : ct[e - 1];
            x[e][1] = (e == V - 1) ? right : ct[e + 1];
            x[e][2] = no[e];
            x[e][3] = so[e];
            x[e][4] = dn[e];
            x[e][5] = up[e];
        }
        double s[V];
        if constexpr (K > 0) {
            const emusum::Mul km = emusum::make_mul(one);
            emusum::Words acc[V];
            uint32_t bad = 0;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                acc[e] = emusum::first_w<F>(emusum::unpack_w(x[e][0], km),
                                            emusum::unpack_w(x[e][1], km), km);
#pragma unroll
                for (int i = 2; i <= K; ++i)
                    emusum::add_w<F>(acc[e], emusum::unpack_w(x[e][i], km), km);
                if (interior[e]) bad |= acc[e].bad;  // outside cells are not stored
            }
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
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) s[e] = __dadd_rn(x[e][0], x[e][1]);
        }
        constexpr int kFirstUnit = K > 0 ? K + 1 : 2;
        double* pd = L.dst(k, sl) + row;
#pragma unroll
        for (int e = 0; e < V; ++e) {
#pragma unroll
            for (int i = kFirstUnit; i <= 5; ++i) s[e] = __dadd_rn(s[e], x[e][i]);
            if (interior[e])
                pd[e] = __dmul_rn(s[e], c6);
            else if (to_ring && okl[e])
                pd[e] = ct[e];  // boundary value passed on
        }
        if (row_lo) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (okl[e]) pd[e - px] = no[e];
        }
        if (row_hi) {
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (okl[e]) pd[e + px] = so[e];
        }
        if (edge_lo) pd[-1] = left;
        if (edge_hi) pd[V] = right;
#pragma unroll
        for (int e = 0; e < V; ++e) {
            dn[e] = ct[e];
            ct[e] = up[e];
        }
        sl = sln;
    }
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Record a wait that ran out: the status word and the abort flag that ends
// every CTA's loop.
__device__ __forceinline__ void wave_fail(const WaveArgs& a) {
    atomicOr(a.status, kStatusTimeout);
    atomicExch(a.abort, 1);
}

// The start conditions of item (s, b, tile), watched by the control warp: lane
// 9c + n watches condition c of neighbour n of the 3 x 3 tiles, three blocks
// each: c = 0, the input: blocks b-1, b, b+1 of level s-1 (the planes k0-1 ..
// k1+1 the item reads); c = 1, the readers of the ring slot overwritten: blocks
// b-R-1 .. b-R+1 of level s+1; c = 2, in place: blocks b-1 .. b+1 of level 1,
// the readers of the level-0 block overwritten.  poll() reads the flags once
// with relaxed loads; after it succeeds, one fence makes the observation an
// acquire.
struct WaveDeps {
    const int* ptr;  // flag of the first block watched
    int nblk;        // blocks watched (0..3)
    __device__ __forceinline__ void init(const WaveArgs& a, int s, int b, int tile, int lane) {
        const int ntiles = a.ntx * a.nty;
        ptr = nullptr;
        nblk = 0;
        if (lane < 27) {
            const int c = lane / 9, nn = lane % 9;
            const int x = tile % a.ntx + nn % 3 - 1, y = tile / a.ntx + nn / 3 - 1;
            if (x >= 0 && x < a.ntx && y >= 0 && y < a.nty) {
                const int n = y * a.ntx + x;
                int lev = 0, mid = 0;  // level (1..t) and middle block watched
                if (c == 0 && s >= 2) {
                    lev = s - 1;
                    mid = b;
                } else if (c == 1 && s < a.t && b >= a.R) {
                    lev = s + 1;
                    mid = b - a.R;
                } else if (c == 2 && s == a.t && a.inplace) {
                    lev = 1;
                    mid = b;
                }
                if (lev > 0) {
                    const int b0 = max(mid - 1, 0), b1 = min(mid + 1, a.nb - 1);
                    ptr = a.done + ((long long)(lev - 1) * ntiles + n) * a.nb + b0;
                    nblk = b1 - b0 + 1;
                }
            }
        }
    }
    // a flag never reverts within a pass: a lane whose blocks are done stops reading
    __device__ __forceinline__ bool poll(int epoch) {
        bool ok = true;
        for (int i = 0; i < nblk; ++i) ok = ok && ld_relaxed(ptr + i) == epoch;
        if (ok) nblk = 0;
        return __all_sync(0xffffffffu, ok);
    }
};


// Named barriers: "job i published" from the control warp to the compute warps,
// one per job parity so that consecutive jobs never share a barrier generation.
// (Barrier numbers are immediates, so only barriers 0..3 are allocated; 3 is the
// compute warps' step barrier of the TMA-staged march.)
template <int ID, int N>
__device__ __forceinline__ void named_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory");
}
template <int ID, int N>
__device__ __forceinline__ void named_arrive() {
    asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void ready_sync(int i) {
    if (i & 1) named_sync<2, N>(); else named_sync<1, N>();
}
template <int N>
__device__ __forceinline__ void ready_arrive(int i) {
    if (i & 1) named_arrive<2, N>(); else named_arrive<1, N>();
}

// ---------------------------------------------------------------------------
// TMA-staged march (FP32/bf16).  The register march above needs a register for
// every load in flight, so its resident warps bound it.  Here the planes of an
// item reach shared memory by TMA: one box per source plane, the tile's rows
// y0-1 .. y0+WY and columns x0-XA .. x0+32V+XA-1 (XA cells = 16 bytes, so the box
// starts aligned), into a ring of NS slots with one "full" mbarrier each.  Warp 0
// issues the copies; after step m every compute warp passes a named barrier, and
// warp 0 then refills the slot of source plane m with plane m+NS.  Phases run on
// across items (a per-CTA count of the planes issued).  (Per-slot release
// mbarriers instead of the step barrier, so that no warp waits for another, with
// an 8-slot ring refilled two steps late, measured slower: FP32 558 / 446 GLUP/s
// at t = 1 / 4 against 606 / 484; the barrier's stall is mostly the slowest
// warp's copy.)
// 8 slots: 4 CTAs per SM in shared memory; against 6, bf16 +5 % and FP32 +3 % at
// depth 4 (512^3); 10 slots measured slower
constexpr int kWaveRing = 8;
constexpr int kBarStep = 3;  // named barrier among the compute warps

template <class S, int V, int WY>
struct WaveTma {
    static constexpr int XA = 16 / (int)sizeof(S);      // 16-byte alignment in cells
    static constexpr int EXB = 32 * V + 2 * XA;         // box width (cells)
    static constexpr int ROWS = WY + 2;                 // box height
    static constexpr int BOX_BYTES = EXB * ROWS * (int)sizeof(S);
    static constexpr int SLOT = (BOX_BYTES + 127) / 128 * 128;  // slot stride (bytes)
    static constexpr int HEADER = 128;                  // NS mbarriers
    static constexpr size_t bytes() { return HEADER + (size_t)kWaveRing * SLOT; }
    static_assert(EXB * (int)sizeof(S) % 16 == 0, "box rows are whole 16-byte units");
    static_assert(EXB <= 256 && ROWS <= 256, "TMA box dimensions");
};

// (FP64 keeps the register march: this march with the integer-pipe accumulator
// measured 75 GLUP/s against 142 at 512^3.)
template <class Tr, int V, int WY>
__device__ __forceinline__ void wave_march_tma(const WaveArgs& a, const CUtensorMap* map_src,
                                               const CUtensorMap* map_ring, int s, int k0,
                                               int k1, int tx, int ty, unsigned char* smem,
                                               uint32_t& issued) {
    using S = typename Tr::S;
    using C = typename Tr::C;
    using VS = Vec<S, V>;
    using Ly = WaveTma<S, V, WY>;
    constexpr int NS = kWaveRing;
    const Geom& g = a.g;
    const int lane = threadIdx.x, warp = threadIdx.y;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    unsigned char* ring = smem + Ly::HEADER;
    const C c6 = Tr::sixth();
    const long long px = g.px, plane = g.plane;

    const int xt = 32 * V * tx;                 // first cell of the tile (x)
    const int X0 = xt - Ly::XA, Y0 = ty * WY;   // box origin (x aligned, y = y0 - 1)
    const int M = k1 - k0 + 3;                  // source planes k0-1 .. k1+1
    const uint32_t first = issued;
    const bool producer = warp == 0 && lane == 0;
    auto issue = [&](int e) {  // source plane k0-1+e into the slot of entry first+e
        const uint32_t ge = first + (uint32_t)e;
        const int slot = (int)(ge % NS);
        const int z = k0 - 1 + e;
        mbar_arrive_expect_tx(&full[slot], Ly::BOX_BYTES);
        void* dst = ring + slot * Ly::SLOT;
        if (s == 1 || z == 0 || z == g.nz + 1)
            tma_load_3d(dst, map_src, &full[slot], X0, Y0, z);
        else
            tma_load_3d(dst, map_ring, &full[slot], X0, Y0, (s - 2) * a.rp + (z - 1) % a.rp);
    };
    if (producer) {
        // the item's inputs were acquired (control warp fence, then the job barrier)
        // through the generic proxy; TMA reads them through the async proxy
        fence_proxy_async_global();
        for (int e = 0; e < NS && e < M; ++e) issue(e);
    }
    issued = first + (uint32_t)M;

    const int y = 1 + ty * WY + warp;
    const int x0 = xt + V * lane;
    const bool row_ok = y <= g.ny;
    const bool loadable = x0 + V <= g.px;
    bool interior[V];
    bool all_interior = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        interior[e] = loadable && x0 + e >= 1 && x0 + e <= g.nx;
        all_interior = all_interior && interior[e];
    }
    const bool to_ring = s < a.t;
    const bool row_lo = to_ring && row_ok && loadable && y == 1;
    const bool row_hi = to_ring && row_ok && loadable && y == g.ny;
    const bool edge_lo = to_ring && row_ok && lane == 0 && x0 == 1;
    const bool edge_hi = to_ring && row_ok && lane == 31 && x0 + V == g.nx + 1 &&
                         x0 + V < g.px;
    S* dbase = to_ring ? static_cast<S*>(a.ring) + (long long)(s - 1) * a.rp * plane
                       : static_cast<S*>(a.dst);
    const long long row = g.lin(loadable ? x0 : 0, row_ok ? y : 1, 0);
    const int col = Ly::XA + V * lane;  // the lane's first cell in a box row
    auto at = [&](uint32_t ge, int r) -> const S* {
        return reinterpret_cast<const S*>(ring + (int)(ge % NS) * Ly::SLOT) + r * Ly::EXB + col;
    };
    // bounded; returns at once when another wait of the launch has run out
    auto wait = [&](uint32_t ge) {
        uint64_t* bar = &full[ge % NS];
        const uint32_t par = (ge / NS) & 1u;
        if (mbar_try_wait(bar, par)) return;
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(bar, par)) {
            if (ld_relaxed(a.abort) != 0) return;
            if (global_ns() - t0 > a.wait_ns) {
                wave_fail(a);
                return;
            }
        }
    };
    wait(first);
    wait(first + 1);
#pragma unroll 1
    for (int m = 0; m + 2 < M; ++m) {
        const uint32_t e0 = first + (uint32_t)m;  // plane k-1; e0+1: plane k; e0+2: plane k+1
        wait(e0 + 2);
        const int k = k0 + m;
        if (row_ok) {
            const int r = warp + 1;
            const VS dn = *reinterpret_cast<const VS*>(at(e0, r));
            const VS ct = *reinterpret_cast<const VS*>(at(e0 + 1, r));
            const VS up = *reinterpret_cast<const VS*>(at(e0 + 2, r));
            const VS no = *reinterpret_cast<const VS*>(at(e0 + 1, r - 1));
            const VS so = *reinterpret_cast<const VS*>(at(e0 + 1, r + 1));
            const S el = at(e0 + 1, r)[-1];
            const S er = at(e0 + 1, r)[V];
            VS outv;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const C l = Tr::ld(e == 0 ? el : ct.v[e - 1]);
                const C rr = Tr::ld(e == V - 1 ? er : ct.v[e + 1]);
                C sum = Tr::add(l, rr);
                sum = Tr::add(sum, Tr::ld(no.v[e]));
                sum = Tr::add(sum, Tr::ld(so.v[e]));
                sum = Tr::add(sum, Tr::ld(dn.v[e]));
                sum = Tr::add(sum, Tr::ld(up.v[e]));
                outv.v[e] = interior[e] ? Tr::st(Tr::mul(sum, c6)) : ct.v[e];
            }
            S* pd = dbase + (to_ring ? (long long)((k - 1) % a.rp) * plane
                                     : (long long)k * plane) + row;
            if (to_ring) {
                if (loadable) *reinterpret_cast<VS*>(pd) = outv;
                if (row_lo) *reinterpret_cast<VS*>(pd - px) = no;
                if (row_hi) *reinterpret_cast<VS*>(pd + px) = so;
                if (edge_lo) pd[-1] = el;
                if (edge_hi) pd[V] = er;
            } else if (all_interior) {
                *reinterpret_cast<VS*>(pd) = outv;
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (interior[e]) pd[e] = outv.v[e];
            }
        }
        // every compute warp is done with the slot of plane k-1: refill it
        named_sync<kBarStep, 32 * WY>();
        if (producer && m + NS < M) issue(m + NS);
    }
}

// NEMU (FP64): 0 = every addition on the FP64 unit; kAccBaseWave + K + 8F = K
// additions through the accumulator in word form F (when the range flag is set).
constexpr int kAccBaseWave = 16;

template <class Tr, int V, int WY, int NEMU>
__device__ __forceinline__ void wave_item(const WaveArgs& a, int s, int b, int tile, bool fast) {
    using S = typename Tr::S;
    constexpr bool kF64 = sizeof(S) == 8;
    constexpr int XOFF = kF64 ? 1 : 0;
    const Geom& g = a.g;
    const int lane = threadIdx.x;
    const int tx = tile % a.ntx, ty = tile / a.ntx;
    const int x0 = XOFF + (tx * 32 + lane) * V;
    const int y = 1 + ty * WY + (int)threadIdx.y;
    if (y > g.ny) return;  // uniform over the warp
    const int k0 = 1 + b * a.kb;
    const int k1 = min(g.nz, k0 + a.kb - 1);

    WaveLevels<S> L;
    L.plane = g.plane;
    L.rp = a.rp;
    L.nz = g.nz;
    L.sgrid = static_cast<const S*>(a.src);
    L.s_in_ring = s >= 2;
    L.sring = static_cast<const S*>(a.ring) + (long long)max(s - 2, 0) * a.rp * g.plane;
    L.d_in_ring = s < a.t;
    L.dgrid = static_cast<S*>(a.dst);
    L.dring = static_cast<S*>(a.ring) + (long long)max(s - 1, 0) * a.rp * g.plane;

    const bool loadable = (x0 + V) <= g.px;
    bool interior[V];
    bool all_interior = true;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        interior[e] = (kF64 || loadable) && (x0 + e >= 1) && (x0 + e <= g.nx);
        all_interior = all_interior && interior[e];
    }
    const bool left_ok = x0 >= 1;
    const bool right_ok = (x0 + V) < g.px;
    const long long row = g.lin(x0 < g.px ? x0 : 0, y, 0);
    if constexpr (kF64) {
        constexpr int K = NEMU >= kAccBaseWave ? ((NEMU - kAccBaseWave) & 7) : 0;
        constexpr int F = NEMU >= kAccBaseWave ? (((NEMU - kAccBaseWave) / 8) & 3) : 0;
        if (K > 0 && fast)
            wave_march_f64<Tr, V, K, F>(L, g, k0, k1, x0, y, lane, interior, left_ok, right_ok,
                                        row, a.one);
        else
            wave_march_f64<Tr, V, 0, 0>(L, g, k0, k1, x0, y, lane, interior, left_ok,
                                        right_ok, row, a.one);
    } else {
        wave_march_vec<Tr, V>(L, g, k0, k1, x0, y, lane, loadable, interior, all_interior,
                              left_ok, right_ok, row);
    }
}

// "job i computed": an mbarrier with one arrival per compute warp; phase i
// completes when job i is done.  Non-blocking test, so that the control warp
// can watch it while it polls the counters of the next job.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Persistent kernel: each CTA takes tickets until the pass is done.  Warps
// 0..WY-1 compute; warp WY is the control warp.  The control warp decodes the
// next ticket and polls that job's start conditions while the compute warps march
// earlier jobs; it publishes a job as soon as its conditions hold, so the compute
// warps find the next job waiting when they finish one.  At most two published
// jobs are unreleased at a time: job j is published only after job j-2 is seen
// done, which keeps the per-parity "job published" barriers and "job done"
// mbarriers from ever holding two generations.  Finished jobs are released in
// order from inside the same polling loop (a job may depend on the CTA's own
// earlier job).  Every wait is on a smaller ticket, so the pass makes progress
// for any number of CTAs.
// TMA = 1: the compute warps use the TMA-staged march (FP32/bf16) with the maps
// of the source grid and of the rings; TMA = 0: the register march (maps unused).
template <class Tr, int V, int WY, int NEMU, int MINB, int TMA>
__global__ void __launch_bounds__(32 * (WY + 1), MINB)
    wave_kernel(const WaveArgs a, const __grid_constant__ CUtensorMap map_src,
                const __grid_constant__ CUtensorMap map_ring) {
    const unsigned FULL = 0xffffffffu;
    constexpr int kThreads = 32 * (WY + 1);
    extern __shared__ __align__(1024) unsigned char wsmem[];
    __shared__ int s_job[2][4];  // s, b, tile, go
    __shared__ __align__(8) uint64_t s_done[2];  // job j done: s_done[j & 1]
    const int lane = threadIdx.x;
    const int ntiles = a.ntx * a.nty;
    if (threadIdx.y == WY && lane == 0) {
        mbar_init(&s_done[0], WY);
        mbar_init(&s_done[1], WY);
        if constexpr (TMA) {
            uint64_t* full = reinterpret_cast<uint64_t*>(wsmem);
            for (int i = 0; i < kWaveRing; ++i) mbar_init(&full[i], 1);
            prefetch_tmap(&map_src);
            prefetch_tmap(&map_ring);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (threadIdx.y == WY) {
        // ---- control warp
        int d = 1, base = 0;  // lane 0: diagonal b + sk s of the ticket, its first ticket
        int it = 0;           // lane 0: the next ticket
        if (lane == 0) it = atomicAdd(a.ticket, 1);
        int js[2] = {0, 0}, jb[2] = {0, 0}, jt[2] = {0, 0};  // published jobs, by parity
        int pub = 0, rel = 0;  // jobs < pub published, jobs < rel released
        auto done = [&](int j) -> bool {  // job j computed (lane 0 reads, all agree)
            int v = 0;
            if (lane == 0) v = mbar_test(&s_done[j & 1], (uint32_t)((j >> 1) & 1)) ? 1 : 0;
            return __shfl_sync(FULL, v, 0) != 0;
        };
        auto release = [&](int j) {  // the job's stores, then its flag
            if (lane == 0) {
                int* f = a.done + ((long long)(js[j & 1] - 1) * ntiles + jt[j & 1]) * a.nb +
                         jb[j & 1];
                __threadfence();
                atomicExch(f, a.epoch);
            }
            __syncwarp();
        };
        auto publish = [&](int s, int b, int tile, int go) {
            if (lane == 0) {
                s_job[pub & 1][0] = s;
                s_job[pub & 1][1] = b;
                s_job[pub & 1][2] = tile;
                s_job[pub & 1][3] = go;
            }
            js[pub & 1] = s;
            jb[pub & 1] = b;
            jt[pub & 1] = tile;
            __syncwarp();
            ready_arrive<kThreads>(pub);
            ++pub;
        };
        bool failed = false;
#pragma unroll 1
        while (true) {
            // decode the next ticket
            int s = 0, b = 0, tile = 0;
            if (lane == 0 && it < a.nitems) {
                while (true) {
                    // levels s of diagonal d: b = d - sk s in [0, nb)
                    const int over = d - (a.nb - 1);
                    const int lo = over <= 0 ? 1 : max(1, (over + a.sk - 1) / a.sk);
                    const int hi = min(a.t, d / a.sk);
                    const int cnt = hi >= lo ? (hi - lo + 1) * ntiles : 0;
                    if (it < base + cnt) {
                        s = lo + (it - base) / ntiles;
                        tile = (it - base) % ntiles;
                        break;
                    }
                    base += cnt;
                    ++d;
                }
                b = d - a.sk * s;
            }
            const bool valid = __shfl_sync(FULL, it, 0) < a.nitems;
            s = __shfl_sync(FULL, s, 0);
            b = __shfl_sync(FULL, b, 0);
            tile = __shfl_sync(FULL, tile, 0);
            WaveDeps deps;
            deps.init(a, s, b, tile, lane);
            bool deps_ok = !valid;
            uint64_t t0 = lane == 0 ? global_ns() : 0;
#pragma unroll 1
            while (true) {
                bool progressed = false;
                while (rel < pub && done(rel)) {
                    release(rel);
                    ++rel;
                    progressed = true;
                }
                if (!deps_ok) {
                    deps_ok = deps.poll(a.epoch);
                    if (deps_ok) __threadfence();  // acquire side of the counter polls
                }
                if (deps_ok && pub - rel < 2) break;
                if (progressed) {
                    if (lane == 0) t0 = global_ns();
                    continue;
                }
                int fail = 0;
                if (lane == 0) {
                    if (ld_relaxed(a.abort) != 0) {
                        fail = 1;
                    } else if (global_ns() - t0 > a.wait_ns) {
                        wave_fail(a);
                        fail = 1;
                    }
                }
                if (__shfl_sync(FULL, fail, 0)) {
                    failed = true;
                    break;
                }
                __nanosleep(64);
            }
            if (failed || !valid) break;
            publish(s, b, tile, 1);
            if (lane == 0) it = atomicAdd(a.ticket, 1);
        }
        // the stop job (go = 0) once at most one job is outstanding (jobs always
        // finish: the compute warps' own waits are bounded), then the last
        // releases; after a failed wait nothing more is released
#pragma unroll 1
        while (pub - rel >= 2) {
            const uint64_t t1 = global_ns();
            while (!done(rel) && global_ns() - t1 < a.wait_ns) __nanosleep(32);
            if (!failed) release(rel);
            ++rel;
        }
        publish(0, 0, 0, 0);
#pragma unroll 1
        while (rel < pub - 1) {
            const uint64_t t1 = global_ns();
            while (!done(rel) && global_ns() - t1 < a.wait_ns) __nanosleep(32);
            if (!failed) release(rel);
            ++rel;
        }
        return;
    }

    // ---- compute warps
    const bool fast = a.fast != nullptr && *a.fast != 0;
    uint32_t issued = 0;  // TMA march: source planes issued so far (mbarrier phases)
#pragma unroll 1
    for (int i = 0;; ++i) {
        ready_sync<kThreads>(i);
        if (!s_job[i & 1][3]) break;
        const int s = s_job[i & 1][0], b = s_job[i & 1][1], tile = s_job[i & 1][2];
        if constexpr (TMA) {
            const int k0 = 1 + b * a.kb;
            const int k1 = min(a.g.nz, k0 + a.kb - 1);
            static_assert(sizeof(typename Tr::S) < 8, "FP64 uses the register march");
            wave_march_tma<Tr, V, WY>(a, &map_src, &map_ring, s, k0, k1, tile % a.ntx,
                                      tile / a.ntx, wsmem, issued);
        } else {
            wave_item<Tr, V, WY, NEMU>(a, s, b, tile, fast);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_done[i & 1]);
    }
}

}  // namespace jac
