// Auxiliary kernels: boundary-layer copy and the FP64 residual step of the
// mixed-precision iterative refinement.
#include <algorithm>

#include "../../include/jacobi.h"
#include "emu.cuh"
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

// Residual step of the refinement, fused and streaming in k.  For every interior
// cell, with u'(c) = u_in(c) + (double) e(c) on interior cells and u_in(c) on the
// boundary layer:
//     u_out = u'
//     rho   = ((((( u'[i-1] + u'[i+1]) + u'[j-1]) + u'[j+1]) + u'[k-1]) + u'[k+1]) - 6.0*u'
// in FP64 (product rounded before the subtraction), rho rounded to the low
// precision.  u' of a neighbour is recomputed from u_in and e instead of being
// read back from u_out, so the kernel needs no grid-wide barrier and gives the
// same bits as "accumulate everywhere, then take the residual".
// Thread layout: lane -> x (interior-aligned, one cell), warp -> y, k marched.
template <class Lo>
__global__ void __launch_bounds__(256)
    residual_kernel(const double* __restrict__ u_in, double* __restrict__ u_out, const Geom gu,
                    const typename Lo::S* __restrict__ e, typename Lo::S* __restrict__ rho,
                    const Geom gl) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int x = 1 + (int)(blockIdx.x * 32 + lane);
    const int y = 1 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (y > gu.ny) return;  // uniform over the warp
    const bool act = x <= gu.nx;
    const int xc = act ? x : gu.nx;  // clamped for address arithmetic

    // u' at (xx, yy, kk); interior test per cell
    auto unew = [&](int xx, int yy, int kk) -> double {
        const double u = __ldg(u_in + gu.lin(xx, yy, kk));
        const bool in = (xx >= 1) && (xx <= gu.nx) && (yy >= 1) && (yy <= gu.ny) && (kk >= 1) &&
                        (kk <= gu.nz);
        if (!in) return u;
        return __dadd_rn(u, (double)Lo::ld(__ldg(e + gl.lin(xx, yy, kk))));
    };

    double dn = unew(xc, y, 0);
    double ct = unew(xc, y, 1);
    for (int k = 1; k <= gu.nz; ++k) {
        const double up = unew(xc, y, k + 1);
        const double no = unew(xc, y - 1, k);
        const double so = unew(xc, y + 1, k);
        double left = __shfl_up_sync(FULL, ct, 1);
        double right = __shfl_down_sync(FULL, ct, 1);
        if (lane == 0) left = unew(xc - 1, y, k);
        if (lane == 31 || x == gu.nx) right = unew(xc + 1, y, k);
        if (act) {
            double s = __dadd_rn(left, right);
            s = __dadd_rn(s, no);
            s = __dadd_rn(s, so);
            s = __dadd_rn(s, dn);
            s = __dadd_rn(s, up);
            const double six_u = __dmul_rn(6.0, ct);
            const double r = __dsub_rn(s, six_u);
            u_out[gu.lin(x, y, k)] = ct;
            rho[gl.lin(x, y, k)] = Lo::st((typename Lo::C)r);
        }
        dn = ct;
        ct = up;
    }
}

cudaError_t launch_residual(const double* u_in, double* u_out, const Geom& gu, const void* e,
                            void* rho, int lo_dtype, const Geom& glo, cudaStream_t st) {
    const dim3 block(32, 8);
    const dim3 grid((gu.nx + 31) / 32, (gu.ny + 7) / 8, 1);
    if (lo_dtype == 1) {
        residual_kernel<F32><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                     static_cast<const float*>(e),
                                                     static_cast<float*>(rho), glo);
    } else if (lo_dtype == 2) {
        residual_kernel<BF16><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                      static_cast<const uint16_t*>(e),
                                                      static_cast<uint16_t*>(rho), glo);
    } else {
        residual_kernel<F64><<<grid, block, 0, st>>>(u_in, u_out, gu,
                                                     static_cast<const double*>(e),
                                                     static_cast<double*>(rho), glo);
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
