// Auxiliary kernels: boundary-layer copy and the FP64 residual step of the
// mixed-precision iterative refinement.
#include <algorithm>

#include "../../include/jacobi.h"
#include "emu.cuh"
#include "emusum.cuh"
#include "launch.h"

namespace jac {

// Copy the boundary layer (all cells with an index 0 or n+1) of A into B.
template <class S>
__global__ void boundary_copy_kernel(const S* __restrict__ A, S* __restrict__ B, const Geom g) {
    const long long nxp = g.nx + 2, nyp = g.ny + 2;
    const long long n_planes = 2 * nxp * nyp;              // k = 0 and k = nz+1
    const long long n_rows = (long long)g.nz * 2 * nxp;      // j = 0, ny+1 for k in 1..nz
    const long long n_cols = (long long)g.nz * g.ny * 2;     // i = 0, nx+1
    const long long total = n_planes + n_rows + n_cols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (t < n_planes) {
            const long long pl = t / (nxp * nyp), r = t % (nxp * nyp);
            k = pl ? g.nz + 1 : 0;
            j = (int)(r / nxp);
            i = (int)(r % nxp);
        } else if (t < n_planes + n_rows) {
            const long long u = t - n_planes;
            k = 1 + (int)(u / (2 * nxp));
            const long long r = u % (2 * nxp);
            j = (r < nxp) ? 0 : g.ny + 1;
            i = (int)(r % nxp);
        } else {
            const long long u = t - n_planes - n_rows;
            k = 1 + (int)(u / (2 * g.ny));
            const long long r = u % (2 * g.ny);
            j = 1 + (int)(r / 2);
            i = (r & 1) ? g.nx + 1 : 0;
        }
        const long long o = g.lin(i, j, k);
        B[o] = A[o];
    }
}

cudaError_t launch_boundary_copy(int dtype, const void* A, void* B, const Geom& g,
                                 cudaStream_t st) {
    const int threads = 256, blocks = 1024;
    switch (dtype) {
        case 0:
            boundary_copy_kernel<double><<<blocks, threads, 0, st>>>(
                static_cast<const double*>(A), static_cast<double*>(B), g);
            break;
        case 1:
            boundary_copy_kernel<float><<<blocks, threads, 0, st>>>(
                static_cast<const float*>(A), static_cast<float*>(B), g);
            break;
        default:
            boundary_copy_kernel<uint16_t><<<blocks, threads, 0, st>>>(
                static_cast<const uint16_t*>(A), static_cast<uint16_t*>(B), g);
            break;
    }
    return cudaGetLastError();
}

// Validity test for the integer-pipe additions of the FP64 plain sweep: every
// cell of the padded grid (boundary layer included, row padding excluded) lies
// in [2^-1000, 2^1000].  *flag must be 1 on entry; any cell outside clears it.
__global__ void range_check_kernel(const double* __restrict__ A, const Geom g, int* flag) {
    const long long nxp = g.nx + 2, rows = (long long)(g.ny + 2) * (g.nz + 2);
    const unsigned long long lo = 0x0170000000000000ull;  // 2^-1000
    const unsigned long long hi = 0x7E70000000000000ull;  // 2^1000
    bool ok = true;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const double* row = A + r * g.px;
        for (long long i = threadIdx.x; i < nxp; i += blockDim.x) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(__ldg(row + i));
            ok = ok && v >= lo && v <= hi;
        }
    }
    if (!__syncthreads_and(ok) && threadIdx.x == 0) *flag = 0;
}

cudaError_t launch_range_check(const double* A, const Geom& g, int* flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flag, 0xFF, sizeof(int), st);  // nonzero = valid
    if (e != cudaSuccess) return e;
    range_check_kernel<<<1024, 256, 0, st>>>(A, g, flag);
    return cudaGetLastError();
}

// Elementwise emulated addition (verification entry point of add_pos_exact).
__global__ void emulated_add_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                    double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = a[i], y = b[i];
        const unsigned long long X = (unsigned long long)__double_as_longlong(x);
        const unsigned long long Y = (unsigned long long)__double_as_longlong(y);
        // positive normal operands with a finite sum take the integer path
        const bool ok = (X >> 52) >= 1 && (X >> 52) <= 2045 && (Y >> 52) >= 1 &&
                        (Y >> 52) <= 2045;
        out[i] = ok ? add_pos_exact(x, y) : __dadd_rn(x, y);
    }
}

// Boundary gradient of the adjoint sweeps: grad[b] += c * lambda_s[m_b] for every
// face cell b (interior neighbour m_b) and sweep s, added in sweep order (the
// reverse-mode order: the last forward sweep first) from the face buffer the
// blocked adjoint kernel fills.  One thread per face cell; the face buffer holds
// nsweeps rows of fstride values (x faces, y faces, z faces, low face first).
template <class S>
__global__ void face_reduce_kernel(S* __restrict__ grad, const Geom g,
                                   const S* __restrict__ fbuf, long long fstride, int nsweeps) {
    const long long fxs = (long long)g.ny * g.nz, fys = (long long)g.nx * g.nz;
    const long long fzs = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < fstride;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        if (i < 2 * fxs) {
            const long long f = i / fxs, r = i % fxs;
            z = (int)(r / g.ny) + 1;
            y = (int)(r % g.ny) + 1;
            x = f == 0 ? 0 : g.nx + 1;
        } else if (i < 2 * fxs + 2 * fys) {
            const long long f = (i - 2 * fxs) / fys, r = (i - 2 * fxs) % fys;
            z = (int)(r / g.nx) + 1;
            x = (int)(r % g.nx) + 1;
            y = f == 0 ? 0 : g.ny + 1;
        } else {
            const long long f = (i - 2 * fxs - 2 * fys) / fzs, r = (i - 2 * fxs - 2 * fys) % fzs;
            y = (int)(r / g.nx) + 1;
            x = (int)(r % g.nx) + 1;
            z = f == 0 ? 0 : g.nz + 1;
        }
        S acc = grad[g.lin(x, y, z)];
        for (int s = 0; s < nsweeps; ++s) acc = acc + fbuf[(long long)s * fstride + i];
        grad[g.lin(x, y, z)] = acc;
    }
}

cudaError_t launch_face_reduce(int dtype, void* grad, const Geom& g, const void* fbuf,
                               long long fstride, int nsweeps, cudaStream_t st) {
    const int threads = 256;
    const long long blocks = std::min<long long>((fstride + threads - 1) / threads, 8192);
    if (dtype == 0)
        face_reduce_kernel<double><<<(unsigned)blocks, threads, 0, st>>>(
            static_cast<double*>(grad), g, static_cast<const double*>(fbuf), fstride, nsweeps);
    else
        face_reduce_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(
            static_cast<float*>(grad), g, static_cast<const float*>(fbuf), fstride, nsweeps);
    return cudaGetLastError();
}

// Six-term sums through the exact accumulator (verification entry point of
// emusum.cuh): out[i] = ((((x0 + x1) + x2) + x3) + x4) + x5 with x_j =
// x[j * n + i], the additions done as the FP64 sweeps do them (all five through
// the accumulator; a warp with a lane outside its window, or with an operand
// that is not a positive normal double, on the FP64 unit).
__global__ void emulated_sum6_kernel(const double* __restrict__ x, double* __restrict__ out,
                                     long long n, uint32_t one) {
    const unsigned FULL = 0xffffffffu;
    const emusum::Mul km = emusum::make_mul(one);
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        const long long i = base + threadIdx.x;
        const bool live = i < n;
        double v[6];
        bool normal = true;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            v[j] = live ? x[j * n + i] : 1.0;
            const unsigned long long b = (unsigned long long)__double_as_longlong(v[j]);
            normal = normal && (b >> 52) >= 1 && (b >> 52) <= 2045;
        }
        emusum::Words a = emusum::first_w(emusum::unpack_w(v[0], km), emusum::unpack_w(v[1], km), km);
#pragma unroll
        for (int j = 2; j < 6; ++j) emusum::add_w(a, emusum::unpack_w(v[j], km), km);
        double s;
        if (__any_sync(FULL, a.bad != 0u || !normal)) {
            s = __dadd_rn(v[0], v[1]);
#pragma unroll
            for (int j = 2; j < 6; ++j) s = __dadd_rn(s, v[j]);
        } else {
            s = emusum::pack_w(a, km);
        }
        if (live) out[i] = s;
    }
}

// Exact widening of a float to double on the integer pipes (IEEE 754 binary32
// -> binary64: same sign, exponent rebiased by 1023 - 127, fraction shifted left
// by 29), for normal numbers and zeros; subnormals, infinities and NaNs take the
// conversion instruction.  Keeps the FP64 pipe, which bounds the residual step,
// for the arithmetic.
static __device__ __noinline__ double f32_to_f64_unit(float f) { return (double)f; }

__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t ex = (b >> 23) & 0xFFu;
    const bool zero = (b & 0x7FFFFFFFu) == 0u;
    const uint32_t hi = (b & 0x80000000u) |
                        (zero ? 0u : (((ex + 896u) << 20) | ((b & 0x7FFFFFu) >> 3)));
    const uint32_t lo = zero ? 0u : (b << 29);
    double r = __hiloint2double((int)hi, (int)lo);
    const bool special = !zero && (ex == 0u || ex == 0xFFu);
    if (__any_sync(__activemask(), special)) {
        if (special) r = f32_to_f64_unit(f);
    }
    return r;
}
__device__ __forceinline__ double widen(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double widen(double d) { return d; }

// Residual step of the refinement, fused and streaming in k.  For every interior
// cell, with u'(c) = u_in(c) + (double) e(c) on interior cells and u_in(c) on the
// boundary layer:
//     u_out = u'
//     rho   = ((((( u'[i-1] + u'[i+1]) + u'[j-1]) + u'[j+1]) + u'[k-1]) + u'[k+1]) - 6.0*u'
// in FP64 (product rounded before the subtraction), rho rounded to the low
// precision.  The kernel is bound by the FP64 pipe (2 ops/clk/SM on GB300), so
// every FP64 instruction a warp issues should produce cells: a CTA of
// RES_ROWS + 2 warps covers RES_ROWS rows plus one halo row above and below, and
// each warp's 32 lanes cover 32 consecutive columns of which the 30 inner ones
// are outputs (the two edge lanes supply the x-neighbours), so no lane forms a
// second u'.  Each warp forms u' for its row of the plane streaming in, keeps the
// k-1, k, k+1 values in registers, and shares the k plane through shared memory
// (y-neighbours) and shuffles (x); the halo warps only form u'.  Same bits as
// "accumulate everywhere, then take the residual" (u' of a cell is the same FP64
// sum wherever it is formed).
constexpr int RES_ROWS = 16;
constexpr int RES_OUT_X = 30;

template <class Lo>
__global__ void __launch_bounds__((RES_ROWS + 2) * 32)
    residual_kernel(const double* __restrict__ u_in, double* __restrict__ u_out, const Geom gu,
                    const typename Lo::S* __restrict__ e, typename Lo::S* __restrict__ rho,
                    const Geom gl, const int kchunk) {
    __shared__ double s_u[2][RES_ROWS + 2][32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;  // w = 0 and RES_ROWS+1: halo
    const int x = (int)blockIdx.x * RES_OUT_X + lane;          // lanes 0 and 31: halo
    const int y = (int)blockIdx.y * RES_ROWS + w;  // row of this warp (0 .. ny+1 possible)
    const int k0 = 1 + (int)blockIdx.z * kchunk;
    const int k1 = min(gu.nz, k0 + kchunk - 1);
    const int xc = min(x, gu.nx + 1);  // clamped column (loads stay inside the array)
    const int yc = min(y, gu.ny + 1);
    const bool cell_in = y >= 1 && y <= gu.ny && x >= 1 && x <= gu.nx;  // interior in x, y
    const bool compute = w >= 1 && w <= RES_ROWS && lane >= 1 && lane <= RES_OUT_X && cell_in;
    const int ktop = gu.nz + 1;
    const long long ou = gu.lin(xc, yc, 0), ol = gl.lin(xc, yc, 0);

    // u' of this lane's cell at plane kk (boundary planes and cells: u_in)
    auto uprime = [&](int kk) -> double {
        const double u = __ldg(u_in + ou + gu.plane * kk);
        const double d = widen(Lo::ld(__ldg(e + ol + gl.plane * kk)));
        const bool in = cell_in && kk >= 1 && kk <= gu.nz;
        return in ? __dadd_rn(u, d) : u;
    };
    double dn = uprime(k0 - 1);
    double ct = uprime(k0);
    double up = uprime(min(k0 + 1, ktop));
    int buf = 0;
    s_u[buf][w][lane] = ct;
    __syncthreads();
    for (int k = k0; k <= k1; ++k) {
        // next plane first (its loads overlap this step's arithmetic)
        const double up2 = uprime(min(k + 2, ktop));
        const double left = __shfl_up_sync(FULL, ct, 1);
        const double right = __shfl_down_sync(FULL, ct, 1);
        if (compute) {
            double s = __dadd_rn(left, right);
            s = __dadd_rn(s, s_u[buf][w - 1][lane]);
            s = __dadd_rn(s, s_u[buf][w + 1][lane]);
            s = __dadd_rn(s, dn);
            s = __dadd_rn(s, up);
            const double r = __dsub_rn(s, __dmul_rn(6.0, ct));
            u_out[ou + gu.plane * k] = ct;
            rho[ol + gl.plane * k] = Lo::st((typename Lo::C)r);
        }
        dn = ct;
        ct = up;
        up = up2;
        buf ^= 1;
        s_u[buf][w][lane] = ct;
        __syncthreads();
    }
}

cudaError_t launch_residual(const double* u_in, double* u_out, const Geom& gu, const void* e,
                            void* rho, int lo_dtype, const Geom& glo, cudaStream_t st) {
    const dim3 block((RES_ROWS + 2) * 32);
    // k-chunks of at least 16 planes, enough CTAs for several waves
    const int tx = (gu.nx + RES_OUT_X - 1) / RES_OUT_X, ty = (gu.ny + RES_ROWS - 1) / RES_ROWS;
    const long long tiles = (long long)tx * ty;
    int chunks = (int)std::max<long long>(1, std::min<long long>(gu.nz / 16, 8192 / tiles + 1));
    const int kchunk = (gu.nz + chunks - 1) / chunks;
    chunks = (gu.nz + kchunk - 1) / kchunk;
    const dim3 grid(tx, ty, chunks);
    if (lo_dtype == 1) {
        residual_kernel<F32><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                     static_cast<const float*>(e),
                                                     static_cast<float*>(rho), glo, kchunk);
    } else if (lo_dtype == 2) {
        residual_kernel<BF16><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                      static_cast<const uint16_t*>(e),
                                                      static_cast<uint16_t*>(rho), glo, kchunk);
    } else {
        residual_kernel<F64><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                     static_cast<const double*>(e),
                                                     static_cast<double*>(rho), glo, kchunk);
    }
    return cudaGetLastError();
}

}  // namespace jac

extern "C" int jacobi_emulated_add(const double* a, const double* b, double* out, long long n,
                                   void* stream) {
    if (n < 0 || (n > 0 && (!a || !b || !out))) return JAC_EINVAL;
    if (n == 0) return JAC_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    jac::emulated_add_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        a, b, out, n);
    return cudaGetLastError() == cudaSuccess ? JAC_OK : JAC_ECUDA;
}

extern "C" int jacobi_emulated_sum6(const double* x, double* out, long long n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return JAC_EINVAL;
    if (n == 0) return JAC_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    jac::emulated_sum6_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        x, out, n, 1u);
    return cudaGetLastError() == cudaSuccess ? JAC_OK : JAC_ECUDA;
}
