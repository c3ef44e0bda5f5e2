// Face values of the adjoint passes: the levels 0..T-1 of a pass at the cells next
// to the six faces, for the boundary gradient (the transposed sweep's contribution
// c * lambda_s to every face cell, with c = RN(1/6)).
#include <algorithm>

#include "../../include/jacobi.h"
#include "launch.h"

namespace jac {
namespace {

constexpr int kBandTU = 32, kBandTV = 8;  // face cells of one CTA along u and v

// One 32 x 8 tile of the face cells of face `face` (normal axis AX; the low end of
// the axis for an even face, the high end for an odd one).  Level s on the face
// layer depends on the pass input within s cells of it, so a band of T layers along
// the normal with a T-1 halo along the face holds everything the tile needs.  The
// band is loaded once (every load of a thread issued before the first store to
// shared memory: the loops have compile-time trip counts), and the levels are
// computed in shared memory with the sweep's arithmetic (the six neighbours in
// Eq. 1's order of the absolute axes, then the product by RN(1/6); a zero
// boundary), so the values are bit-identical to the levels the pass computes.
// Level s of the face cells goes to row sweep0 + s of the face buffer (x faces,
// y faces, z faces, low face first; rows of the face's u extent).
template <class S, int T, int AX>
__device__ __forceinline__ void face_band_tile(const S* __restrict__ src, const Geom& g,
                                               S* __restrict__ fbuf, long long fstride,
                                               int sweep0, int face, S* cur, S* nxt) {
    constexpr int TU = kBandTU, TV = kBandTV;
    constexpr int H = T - 1, BU = TU + 2 * H, BV = TV + 2 * H;
    constexpr int layer = BU * BV;
    constexpr int JU = (BU + TU - 1) / TU, JV = (BV + TV - 1) / TV;
    const int tu = threadIdx.x, tv = threadIdx.y;
    const bool hi = (face & 1) != 0;
    // face extent: u = y (x faces) or x; v = y (z faces) or z; nn along the normal
    const int nu = AX == 0 ? g.ny : g.nx;
    const int nv = AX == 2 ? g.ny : g.nz;
    const int nn = AX == 0 ? g.nx : AX == 1 ? g.ny : g.nz;
    const int u0 = 1 + (int)blockIdx.x * TU, v0 = 1 + (int)blockIdx.y * TV;
    if (u0 > nu || v0 > nv) return;  // the whole CTA
    const S c6 = sizeof(S) == 8 ? S(0x1.5555555555555p-3) : S(0x1.555556p-3f);
    // grid offsets of one step along u, along v and inward along the normal
    const long long su = AX == 0 ? g.px : 1;
    const long long sv = AX == 2 ? g.px : g.plane;
    const long long sn_abs = AX == 0 ? 1 : AX == 1 ? g.px : g.plane;
    const long long sn = hi ? -sn_abs : sn_abs;
    const int w0 = hi ? nn : 1;  // the face layer along the normal
    const long long origin = AX == 0 ? g.lin(w0, 0, 0) : AX == 1 ? g.lin(0, w0, 0)
                                                                : g.lin(0, 0, w0);
    const long long fxs = (long long)g.ny * g.nz, fys = (long long)g.nx * g.nz;
    const long long fbase = AX == 0 ? face * fxs
                            : AX == 1 ? 2 * fxs + (face - 2) * fys
                                      : 2 * fxs + 2 * fys + (long long)(face - 4) * g.nx * g.ny;
    const int urow = AX == 0 ? g.ny : g.nx;  // face-buffer row length along u

    // level 0: band cell (n, iu, iv) lies n layers in from the face, u = u0 - H + iu;
    // cells outside the interior (boundary or beyond) are zero
    S val[T][JV][JU];
#pragma unroll
    for (int n = 0; n < T; ++n) {
#pragma unroll
        for (int jv = 0; jv < JV; ++jv) {
            const int iv = tv + jv * TV, v = v0 - H + iv;
            const bool vin = n < nn && iv < BV && v >= 1 && v <= nv;
            const S* row = src + origin + n * sn + (long long)v * sv;
#pragma unroll
            for (int ju = 0; ju < JU; ++ju) {
                const int iu = tu + ju * TU, u = u0 - H + iu;
                val[n][jv][ju] = (vin && iu < BU && u >= 1 && u <= nu) ? row[u * su] : S(0);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < T; ++n)
#pragma unroll
        for (int jv = 0; jv < JV; ++jv)
#pragma unroll
            for (int ju = 0; ju < JU; ++ju) {
                const int iv = tv + jv * TV, iu = tu + ju * TU;
                if (iv < BV && iu < BU) cur[n * layer + iv * BU + iu] = val[n][jv][ju];
            }
    __syncthreads();

    const int uo = u0 + tu, vo = v0 + tv;
    const bool owns = uo <= nu && vo <= nv;  // this thread's face cell exists
    S* fb = fbuf + (long long)sweep0 * fstride + fbase + (long long)(vo - 1) * urow + (uo - 1);
    auto store_face = [&](const S* lv, int s) {
        if (!owns) return;
        const S lam = lv[(H + tv) * BU + (H + tu)];  // layer 0
        fb[(long long)s * fstride] = sizeof(S) == 8
            ? S(__dmul_rn((double)c6, (double)lam)) : S(__fmul_rn((float)c6, (float)lam));
    };
    store_face(cur, 0);
#pragma unroll
    for (int s = 1; s < T; ++s) {
        // level s on layers 0..T-1-s, within s cells less of halo
        const int JVs = (BV - 2 * s + TV - 1) / TV, JUs = (BU - 2 * s + TU - 1) / TU;
#pragma unroll
        for (int n = 0; n < T - s; ++n) {
#pragma unroll
            for (int jv = 0; jv < JV; ++jv) {
                const int iv = s + tv + jv * TV, v = v0 - H + iv;
                const bool vin = jv < JVs && iv < BV - s && n < nn && v >= 1 && v <= nv;
#pragma unroll
                for (int ju = 0; ju < JU; ++ju) {
                    const int iu = s + tu + ju * TU, u = u0 - H + iu;
                    if (!(jv < JVs && ju < JUs && iv < BV - s && iu < BU - s)) continue;
                    const int c = n * layer + iv * BU + iu;
                    S out = S(0);
                    if (vin && u >= 1 && u <= nu) {
                        // neighbours along the normal (n - 1 beyond the face is the boundary)
                        const S nlo = n > 0 ? cur[c - layer] : S(0), nhi = cur[c + layer];
                        const S am = hi ? nhi : nlo, ap = hi ? nlo : nhi;  // axis -1, +1
                        const S um = cur[c - 1], up = cur[c + 1];
                        const S vm = cur[c - BU], vp = cur[c + BU];
                        // u, v and the normal as the absolute axes x, y, z
                        const S xm = AX == 0 ? am : um, xp = AX == 0 ? ap : up;
                        const S ym = AX == 0 ? um : AX == 1 ? am : vm;
                        const S yp = AX == 0 ? up : AX == 1 ? ap : vp;
                        const S zm = AX == 2 ? am : vm, zp = AX == 2 ? ap : vp;
                        if constexpr (sizeof(S) == 8) {
                            double acc = __dadd_rn(xm, xp);
                            acc = __dadd_rn(acc, ym);
                            acc = __dadd_rn(acc, yp);
                            acc = __dadd_rn(acc, zm);
                            acc = __dadd_rn(acc, zp);
                            out = __dmul_rn(acc, (double)c6);
                        } else {
                            float acc = __fadd_rn(xm, xp);
                            acc = __fadd_rn(acc, ym);
                            acc = __fadd_rn(acc, yp);
                            acc = __fadd_rn(acc, zm);
                            acc = __fadd_rn(acc, zp);
                            out = __fmul_rn(acc, (float)c6);
                        }
                    }
                    nxt[c] = out;
                }
            }
        }
        __syncthreads();
        store_face(nxt, s);
        S* tmp = cur;
        cur = nxt;
        nxt = tmp;
        __syncthreads();
    }
}

// Grid: (tiles of 32 cells along u, of 8 along v, 6 faces); face f has normal axis
// f / 2.  Block (32, 8).  Dynamic shared memory: two bands of T layers.
template <class S, int T>
__global__ void __launch_bounds__(256) face_band_kernel(const S* __restrict__ src, const Geom g,
                                                        S* __restrict__ fbuf, long long fstride,
                                                        int sweep0) {
    extern __shared__ __align__(16) unsigned char band_smem[];
    constexpr int vol = T * (kBandTU + 2 * (T - 1)) * (kBandTV + 2 * (T - 1));
    S* cur = reinterpret_cast<S*>(band_smem);
    S* nxt = cur + vol;
    const int face = (int)blockIdx.z;
    switch (face >> 1) {
        case 0: face_band_tile<S, T, 0>(src, g, fbuf, fstride, sweep0, face, cur, nxt); break;
        case 1: face_band_tile<S, T, 1>(src, g, fbuf, fstride, sweep0, face, cur, nxt); break;
        default: face_band_tile<S, T, 2>(src, g, fbuf, fstride, sweep0, face, cur, nxt); break;
    }
}

template <class S, int T>
cudaError_t launch_band_t(const void* src, const Geom& g, void* fbuf, long long fstride,
                          int sweep0, cudaStream_t st) {
    constexpr size_t smem =
        2 * (size_t)T * (kBandTU + 2 * (T - 1)) * (kBandTV + 2 * (T - 1)) * sizeof(S);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(face_band_kernel<S, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return cudaGetLastError();
    const dim3 grid((unsigned)((std::max(g.nx, g.ny) + kBandTU - 1) / kBandTU),
                    (unsigned)((std::max(g.ny, g.nz) + kBandTV - 1) / kBandTV), 6);
    face_band_kernel<S, T><<<grid, dim3(kBandTU, kBandTV), smem, st>>>(
        static_cast<const S*>(src), g, static_cast<S*>(fbuf), fstride, sweep0);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_band_s(const void* src, const Geom& g, void* fbuf, long long fstride,
                          int sweep0, int T, cudaStream_t st) {
    switch (T) {
        case 1: return launch_band_t<S, 1>(src, g, fbuf, fstride, sweep0, st);
        case 2: return launch_band_t<S, 2>(src, g, fbuf, fstride, sweep0, st);
        case 3: return launch_band_t<S, 3>(src, g, fbuf, fstride, sweep0, st);
        case 4: return launch_band_t<S, 4>(src, g, fbuf, fstride, sweep0, st);
        case 5: return launch_band_t<S, 5>(src, g, fbuf, fstride, sweep0, st);
        case 6: return launch_band_t<S, 6>(src, g, fbuf, fstride, sweep0, st);
        case 7: return launch_band_t<S, 7>(src, g, fbuf, fstride, sweep0, st);
        case 8: return launch_band_t<S, 8>(src, g, fbuf, fstride, sweep0, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_face_band(int dtype, const void* src, const Geom& g, void* fbuf,
                             long long fstride, int sweep0, int T, cudaStream_t st) {
    if (dtype == JAC_F64) return launch_band_s<double>(src, g, fbuf, fstride, sweep0, T, st);
    if (dtype == JAC_F32) return launch_band_s<float>(src, g, fbuf, fstride, sweep0, T, st);
    return cudaErrorInvalidValue;
}

}  // namespace jac
