// Shared device-side pieces of the Jacobi library: element traits, the grid
// geometry, inline-PTX wrappers for mbarriers and TMA, and the bounded wait.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace jac {

// ---------------------------------------------------------------------------
// Element traits.  S is the storage type, C the compute type.  add/mul are
// single IEEE-754 round-to-nearest operations (no contraction into FMA).
// sixth is RN(1/6) in the compute precision: Eq. 1 multiplies the sum of the
// six neighbours by 1/6; the library multiplies by the rounded constant.
struct F64 {
    using S = double;
    using C = double;
    static constexpr int kDtype = 0;
    __device__ __forceinline__ static C ld(S v) { return v; }
    __device__ __forceinline__ static S st(C v) { return v; }
    __device__ __forceinline__ static C rnd(C v) { return v; }
    // storage form of a value already representable in S
    __device__ __forceinline__ static S st_exact(C v) { return v; }
    __device__ __forceinline__ static void rnd_pair(C& a, C& b) {}
    __device__ __forceinline__ static C add(C a, C b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static C mul(C a, C b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static C sixth() { return 0x1.5555555555555p-3; }
};

struct F32 {
    using S = float;
    using C = float;
    static constexpr int kDtype = 1;
    __device__ __forceinline__ static C ld(S v) { return v; }
    __device__ __forceinline__ static S st(C v) { return v; }
    __device__ __forceinline__ static C rnd(C v) { return v; }
    __device__ __forceinline__ static S st_exact(C v) { return v; }
    __device__ __forceinline__ static void rnd_pair(C& a, C& b) {}
    __device__ __forceinline__ static C add(C a, C b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static C mul(C a, C b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static C sixth() { return 0x1.555556p-3f; }
};

// bf16 storage as raw 16-bit patterns; FP32 arithmetic; every stored value is
// rounded to bf16 with round-to-nearest-even.
struct BF16 {
    using S = uint16_t;
    using C = float;
    static constexpr int kDtype = 2;
    __device__ __forceinline__ static C ld(S v) {
        return __uint_as_float(static_cast<uint32_t>(v) << 16);
    }
    __device__ __forceinline__ static S st(C v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    __device__ __forceinline__ static C rnd(C v) { return ld(st(v)); }
    // a float that is already a bf16 value: its high half
    __device__ __forceinline__ static S st_exact(C v) {
        return static_cast<S>(__float_as_uint(v) >> 16);
    }
    // round two floats to bf16 (nearest-even) with one packed conversion
    __device__ __forceinline__ static void rnd_pair(C& a, C& b) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
        const uint32_t u = *reinterpret_cast<const uint32_t*>(&p);
        a = __uint_as_float(u << 16);
        b = __uint_as_float(u & 0xFFFF0000u);
    }
    __device__ __forceinline__ static C add(C a, C b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static C mul(C a, C b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static C sixth() { return 0x1.555556p-3f; }
};

// Packed FP32 pairs (sm_100 family): two independent IEEE-754 round-to-nearest
// additions or multiplications in one instruction, bit for bit the results of
// the two scalar operations.
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long p, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Padded grid geometry: cell (i,j,k) at i + px * (j + (ny+2) * k).
struct Geom {
    int nx, ny, nz;
    long long px;      // row pitch (elements)
    long long plane;   // px * (ny + 2)
    __host__ __device__ __forceinline__ long long lin(int i, int j, int k) const {
        return (long long)i + px * (long long)j + plane * (long long)k;
    }
};

// Status word bits written by kernels into the handle's device status.
enum : int { kStatusTimeout = 1, kStatusBadLaunch = 2 };

// A vector of V storage elements, aligned so that it loads/stores as one access.
template <class S, int V>
struct alignas(V * sizeof(S) >= 16 ? 16 : V * sizeof(S)) Vec {
    S v[V];
};

template <int BYTES> struct RawOf;
template <> struct RawOf<16> { using T = uint4; };
template <> struct RawOf<8> { using T = uint2; };
template <> struct RawOf<4> { using T = unsigned int; };
template <> struct RawOf<2> { using T = unsigned short; };

// Read-only (non-coherent path) load of one vector.
template <class S, int V>
__device__ __forceinline__ Vec<S, V> ldg_vec(const S* p) {
    using R = typename RawOf<sizeof(Vec<S, V>)>::T;
    const R r = __ldg(reinterpret_cast<const R*>(p));
    Vec<S, V> out;
    memcpy(&out, &r, sizeof(out));
    return out;
}

// ---------------------------------------------------------------------------
// Inline PTX: mbarrier and TMA (cp.async.bulk.tensor), CTA scope.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Orders this thread's view of global memory (data acquired from other CTAs'
// ordinary stores) before its later TMA reads, which go through the async proxy.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// GPU-scope acquire load of a progress counter written by other CTAs.
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait for phase `parity` of `bar`, giving up after ~limit_ns of wall time.
// Returns false on timeout (the caller records it and leaves cleanly).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// 3D tiled TMA load of one box into shared memory, completion on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

}  // namespace jac
