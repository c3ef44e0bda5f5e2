/*
 * CPU oracle for the 3D 7-point Jacobi method (Wittmann, Hager, Wellein,
 * "Multicore-aware parallel temporal blocking of stencil codes for shared and
 * distributed memory", Sect. 1.1, Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, constant or helper with the CUDA path.
 *
 * Compile with -O2 -ffp-contract=off -fno-fast-math (see oracle/build.py):
 * every floating-point operation below is a single IEEE-754 round-to-nearest-
 * even operation in the order written.
 *
 * Grid layout (all functions): a padded array with a one-cell boundary layer,
 * interior cells 1..n per axis, boundary cells 0 and n+1.  Cell (i,j,k) lives at
 *     lin(i,j,k) = i + px * (j + py * k),   px >= nx+2, py >= ny+2,
 * i (x) contiguous.  The boundary layer holds the fixed Dirichlet data and is
 * never written by a sweep (Sect. 1.1 describes successive sweeps between two
 * grids A and B; the boundary values are the data of the boundary value problem).
 *
 * Parallelism: the optional OpenMP loop over k changes nothing numerically;
 * every interior cell is computed by one thread with the same operations.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LIN(i, j, k) ((size_t)(i) + (size_t)px * ((size_t)(j) + (size_t)py * (size_t)(k)))

/* The factor 1/6 of Eq. 1, rounded once to the storage precision.  Eq. 1 writes
 * the update as (1/6) * (sum); we multiply by the rounded constant and never
 * divide.  0x1.5555555555555p-3 is RN64(1/6). */
static const double ORACLE_SIXTH = 0x1.5555555555555p-3;

/* ---- bfloat16 storage: defined from its bit layout (the upper 16 bits of an
 *      IEEE binary32), rounding to nearest with ties to even.  Inputs are finite. */
static float bf16_to_f32(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static uint16_t f32_to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t keep = u >> 16;          /* truncated result            */
    uint32_t rest = u & 0xFFFFu;      /* the 16 bits that are dropped */
    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u)))
        keep += 1u;                   /* carries into the exponent correctly */
    return (uint16_t)keep;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1, one sweep, FP64: for every interior cell
 *   B = ((((( A[i-1] + A[i+1]) + A[j-1]) + A[j+1]) + A[k-1]) + A[k+1]) * RN(1/6)   */
static void sweep_f64(const double *A, double *B, int nx, int ny, int nz,
                      long px, long py, int nthreads)
{
    int k;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double s = A[LIN(i - 1, j, k)];
                s = s + A[LIN(i + 1, j, k)];
                s = s + A[LIN(i, j - 1, k)];
                s = s + A[LIN(i, j + 1, k)];
                s = s + A[LIN(i, j, k - 1)];
                s = s + A[LIN(i, j, k + 1)];
                B[LIN(i, j, k)] = s * ORACLE_SIXTH;
            }
}

static void sweep_f32(const float *A, float *B, int nx, int ny, int nz,
                      long px, long py, int nthreads)
{
    const float c = (float)ORACLE_SIXTH; /* RN32(1/6) */
    int k;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                float s = A[LIN(i - 1, j, k)];
                s = s + A[LIN(i + 1, j, k)];
                s = s + A[LIN(i, j - 1, k)];
                s = s + A[LIN(i, j + 1, k)];
                s = s + A[LIN(i, j, k - 1)];
                s = s + A[LIN(i, j, k + 1)];
                B[LIN(i, j, k)] = s * c;
            }
}

/* bf16 storage, f32 arithmetic, result rounded to bf16 after every sweep. */
static void sweep_bf16(const uint16_t *A, uint16_t *B, int nx, int ny, int nz,
                       long px, long py, int nthreads)
{
    const float c = (float)ORACLE_SIXTH;
    int k;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
    for (k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                float s = bf16_to_f32(A[LIN(i - 1, j, k)]);
                s = s + bf16_to_f32(A[LIN(i + 1, j, k)]);
                s = s + bf16_to_f32(A[LIN(i, j - 1, k)]);
                s = s + bf16_to_f32(A[LIN(i, j + 1, k)]);
                s = s + bf16_to_f32(A[LIN(i, j, k - 1)]);
                s = s + bf16_to_f32(A[LIN(i, j, k + 1)]);
                B[LIN(i, j, k)] = f32_to_bf16(s * c);
            }
}

/* n successive sweeps writing A and B in turn (Sect. 1.1).  The boundary layer of
 * B must equal that of A on entry; it is never written.  Returns 0 when the
 * result is in A (n even) and 1 when it is in B (n odd). */
int oracle_sweeps_f64(double *A, double *B, int nx, int ny, int nz,
                      long px, long py, int n, int nthreads)
{
    for (int s = 0; s < n; ++s) {
        if (s & 1) sweep_f64(B, A, nx, ny, nz, px, py, nthreads);
        else       sweep_f64(A, B, nx, ny, nz, px, py, nthreads);
    }
    return n & 1;
}

int oracle_sweeps_f32(float *A, float *B, int nx, int ny, int nz,
                      long px, long py, int n, int nthreads)
{
    for (int s = 0; s < n; ++s) {
        if (s & 1) sweep_f32(B, A, nx, ny, nz, px, py, nthreads);
        else       sweep_f32(A, B, nx, ny, nz, px, py, nthreads);
    }
    return n & 1;
}

int oracle_sweeps_bf16(uint16_t *A, uint16_t *B, int nx, int ny, int nz,
                       long px, long py, int n, int nthreads)
{
    for (int s = 0; s < n; ++s) {
        if (s & 1) sweep_bf16(B, A, nx, ny, nz, px, py, nthreads);
        else       sweep_bf16(A, B, nx, ny, nz, px, py, nthreads);
    }
    return n & 1;
}

/* ------------------------------------------------------------------------- */
/* Iterative refinement pieces.  With r = b - (I - J0) u the residual of the
 * discrete boundary value problem that the Jacobi method of Sect. 1.1 solves,
 * and rho = 6 r, one correction sweep is
 *     e' = (((((( e[i-1] + e[i+1]) + e[j-1]) + e[j+1]) + e[k-1]) + e[k+1]) + rho) * RN(1/6)
 * on a grid e whose boundary layer is zero.  Storage precision: f64, f32 or bf16
 * (bf16: f32 arithmetic, rounded to bf16 after every sweep). */
int oracle_rhs_sweeps_f64(double *E, double *E2, const double *rho, int nx, int ny,
                          int nz, long px, long py, int n)
{
    for (int s = 0; s < n; ++s) {
        const double *a = (s & 1) ? E2 : E;
        double *b = (s & 1) ? E : E2;
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    double v = a[LIN(i - 1, j, k)];
                    v = v + a[LIN(i + 1, j, k)];
                    v = v + a[LIN(i, j - 1, k)];
                    v = v + a[LIN(i, j + 1, k)];
                    v = v + a[LIN(i, j, k - 1)];
                    v = v + a[LIN(i, j, k + 1)];
                    v = v + rho[LIN(i, j, k)];
                    b[LIN(i, j, k)] = v * ORACLE_SIXTH;
                }
    }
    return n & 1;
}

int oracle_rhs_sweeps_f32(float *E, float *E2, const float *rho, int nx, int ny,
                          int nz, long px, long py, int n, int nthreads)
{
    const float c = (float)ORACLE_SIXTH;
    for (int s = 0; s < n; ++s) {
        const float *a = (s & 1) ? E2 : E;
        float *b = (s & 1) ? E : E2;
        int k;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
        for (k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    float v = a[LIN(i - 1, j, k)];
                    v = v + a[LIN(i + 1, j, k)];
                    v = v + a[LIN(i, j - 1, k)];
                    v = v + a[LIN(i, j + 1, k)];
                    v = v + a[LIN(i, j, k - 1)];
                    v = v + a[LIN(i, j, k + 1)];
                    v = v + rho[LIN(i, j, k)];
                    b[LIN(i, j, k)] = v * c;
                }
    }
    return n & 1;
}

int oracle_rhs_sweeps_bf16(uint16_t *E, uint16_t *E2, const uint16_t *rho, int nx,
                           int ny, int nz, long px, long py, int n, int nthreads)
{
    const float c = (float)ORACLE_SIXTH;
    for (int s = 0; s < n; ++s) {
        const uint16_t *a = (s & 1) ? E2 : E;
        uint16_t *b = (s & 1) ? E : E2;
        int k;
#pragma omp parallel for schedule(static) num_threads(nthreads) if (nthreads > 1)
        for (k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    float v = bf16_to_f32(a[LIN(i - 1, j, k)]);
                    v = v + bf16_to_f32(a[LIN(i + 1, j, k)]);
                    v = v + bf16_to_f32(a[LIN(i, j - 1, k)]);
                    v = v + bf16_to_f32(a[LIN(i, j + 1, k)]);
                    v = v + bf16_to_f32(a[LIN(i, j, k - 1)]);
                    v = v + bf16_to_f32(a[LIN(i, j, k + 1)]);
                    v = v + bf16_to_f32(rho[LIN(i, j, k)]);
                    b[LIN(i, j, k)] = f32_to_bf16(v * c);
                }
    }
    return n & 1;
}

/* Residual step of the refinement, in FP64:
 *   1. u += (double) e          on every interior cell;
 *   2. rho = s(u) - 6.0 * u     on every interior cell, with s(u) the six-
 *      neighbour sum of Eq. 1 in its order (boundary data included), the
 *      product rounded before the subtraction; rho stored in the low precision
 *      (elem = 4: f32, elem = 2: bf16, elem = 8: f64).
 * Step 1 finishes on the whole grid before step 2 starts. */
void oracle_residual_accumulate(double *u, const void *e, void *rho, int elem,
                                int nx, int ny, int nz, long px, long py)
{
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                size_t x = LIN(i, j, k);
                double ev;
                if (elem == 8)      ev = ((const double *)e)[x];
                else if (elem == 4) ev = (double)((const float *)e)[x];
                else                ev = (double)bf16_to_f32(((const uint16_t *)e)[x]);
                u[x] = u[x] + ev;
            }
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double s = u[LIN(i - 1, j, k)];
                s = s + u[LIN(i + 1, j, k)];
                s = s + u[LIN(i, j - 1, k)];
                s = s + u[LIN(i, j + 1, k)];
                s = s + u[LIN(i, j, k - 1)];
                s = s + u[LIN(i, j, k + 1)];
                double six_u = 6.0 * u[LIN(i, j, k)];
                double r = s - six_u;
                size_t x = LIN(i, j, k);
                if (elem == 8)      ((double *)rho)[x] = r;
                else if (elem == 4) ((float *)rho)[x] = (float)r;
                else                ((uint16_t *)rho)[x] = f32_to_bf16((float)r);
            }
}

/* ------------------------------------------------------------------------- */
/* Reverse-mode gradient of L = sum over all padded cells of W * A_n, where A_0
 * has interior X and boundary g and A_s = sweep(A_{s-1}) with the boundary held
 * at g.  The forward program is walked backwards operation by operation:
 *   B = sum * c          gives  lam_sum  = c * lam_B
 *   sum = sum' + x       gives  lam_x   += lam_sum, lam_sum' = lam_sum
 *   A_s[b] = g[b]        gives  grad_g[b] += lam_{A_s}[b]   (boundary copy)
 * The tape holds no values because every operation is linear; the operations
 * are replayed in reverse order (last sweep first, last cell first, last operand
 * first).  Output `grad` (padded): interior = dL/dX, boundary = dL/dg.  FP64.
 * Work space: two padded arrays `lam` and `lam2`, zeroed here. */
void oracle_grad_f64(const double *W, double *grad, double *lam, double *lam2,
                     int nx, int ny, int nz, long px, long py, int n)
{
    size_t total = (size_t)px * (size_t)py * (size_t)(nz + 2);
    memcpy(lam, W, total * sizeof(double));            /* lam_n = dL/dA_n = W */
    memset(grad, 0, total * sizeof(double));
    for (int s = n; s >= 1; --s) {
        memset(lam2, 0, total * sizeof(double));         /* lam_{s-1}          */
        /* boundary cells of A_s were copies of g */
        for (int k = 0; k <= nz + 1; ++k)
            for (int j = 0; j <= ny + 1; ++j)
                for (int i = 0; i <= nx + 1; ++i) {
                    int bnd = (i == 0 || i == nx + 1 || j == 0 || j == ny + 1 ||
                               k == 0 || k == nz + 1);
                    if (bnd) grad[LIN(i, j, k)] += lam[LIN(i, j, k)];
                }
        /* interior cells, last one first; operands of the sum last one first */
        for (int k = nz; k >= 1; --k)
            for (int j = ny; j >= 1; --j)
                for (int i = nx; i >= 1; --i) {
                    double lam_sum = ORACLE_SIXTH * lam[LIN(i, j, k)];
                    lam2[LIN(i, j, k + 1)] += lam_sum;
                    lam2[LIN(i, j, k - 1)] += lam_sum;
                    lam2[LIN(i, j + 1, k)] += lam_sum;
                    lam2[LIN(i, j - 1, k)] += lam_sum;
                    lam2[LIN(i + 1, j, k)] += lam_sum;
                    lam2[LIN(i - 1, j, k)] += lam_sum;
                }
        double *tmp = lam; lam = lam2; lam2 = tmp;
    }
    /* A_0: interior is X, boundary is g */
    for (int k = 0; k <= nz + 1; ++k)
        for (int j = 0; j <= ny + 1; ++j)
            for (int i = 0; i <= nx + 1; ++i) {
                int bnd = (i == 0 || i == nx + 1 || j == 0 || j == ny + 1 ||
                           k == 0 || k == nz + 1);
                if (bnd) grad[LIN(i, j, k)] += lam[LIN(i, j, k)];
                else     grad[LIN(i, j, k)] = lam[LIN(i, j, k)];
            }
}

/* Helpers exposed so that tests can check the storage conversions themselves. */
void oracle_f32_to_bf16(const float *in, uint16_t *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = f32_to_bf16(in[i]);
}

void oracle_bf16_to_f32(const uint16_t *in, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = bf16_to_f32(in[i]);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
