/*
 * jacobi.h — C ABI of the GB300 (sm_103a) temporally-blocked 3D 7-point Jacobi
 * library (libjacobi_gb300.so).
 *
 * Method: Wittmann, Hager, Wellein, "Multicore-aware parallel temporal blocking
 * of stencil codes for shared and distributed memory" (arXiv:0912.4506).
 *   Eq. 1 (Sect. 1.1)   one cell update: B_ijk = 1/6 (A_i-1 + A_i+1 + A_j-1 +
 *                       A_j+1 + A_k-1 + A_k+1);
 *   Sect. 1.1           successive sweeps write grids A and B in turn;
 *   Sect. 1.3           temporal blocking: several updates of a block while it
 *                       is held on chip, each update shifted by one cell.
 *
 * Arithmetic: the six neighbours are summed left to right in the order of Eq. 1
 * and the sum is multiplied by RN(1/6) of the compute precision (never divided),
 * with no fused multiply-add.  FP64 grids compute in FP64, FP32 grids in FP32,
 * bf16 grids load bf16, compute in FP32 and round to bf16 (nearest-even) after
 * every sweep, also inside a temporally-blocked pass.  Results are therefore
 * independent of the temporal-blocking depth and bit-identical to a plain
 * sequential sweep loop.
 *
 * Grid layout (every grid argument): a padded array with a one-cell boundary
 * layer.  Interior cells are 1..n per axis, boundary cells 0 and n+1.  Cell
 * (i,j,k) is element  i + row_pitch * (j + (ny+2) * k);  x (i) is contiguous.
 * row_pitch >= nx+2 and row_pitch * element_size must be a multiple of 16 bytes;
 * every device pointer must be 16-byte aligned.  Elements i >= nx+2 of a row are
 * padding: never read, never written.  The boundary layer holds fixed Dirichlet
 * data and is never written by a sweep.
 *
 * Ownership: the caller owns every grid, every device buffer and the stream.
 * The library owns only what a handle holds (plan, tensor-map descriptors, a
 * small device status word and, once a call needs them, the adjoint's face
 * buffer and third grid and the pipelined passes' rings), released by the
 * matching destroy call.
 *
 * Errors: every call returns JAC_OK (0) or a negative JAC_E* code; nothing is
 * thrown across the ABI.  Calls are asynchronous on the handle's stream: a
 * device-side fault or timeout surfaces at jacobi_check() (or at the caller's
 * next synchronisation).  Grids passed to one call must not alias.
 */
#ifndef JACOBI_GB300_H
#define JACOBI_GB300_H

#include <stddef.h>

#if defined(__GNUC__)
#define JAC_API __attribute__((visibility("default")))
#else
#define JAC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum jac_status {
    JAC_OK = 0,
    JAC_EINVAL = -1,       /* bad shape, pointer, alignment or argument            */
    JAC_ENOMEM = -2,       /* device allocation for the handle failed              */
    JAC_ECUDA = -3,        /* a CUDA runtime/driver call failed                    */
    JAC_ETIMEOUT = -4,     /* a bounded device-side wait ran out (status word)     */
    JAC_EUNSUPPORTED = -5  /* no kernel for this dtype/mode/config                 */
};

typedef enum { JAC_F64 = 0, JAC_F32 = 1, JAC_BF16 = 2 } jac_dtype;

/* Operations, for jacobi_max_depth(). */
typedef enum {
    JAC_OP_SWEEP = 0,      /* jacobi_sweep / jacobi_sweep_ex (Eq. 1)               */
    JAC_OP_RHS = 1,        /* jacobi_sweep_rhs (correction sweeps)                 */
    JAC_OP_ADJOINT = 2     /* jacobi_adjoint (transpose sweeps)                    */
} jac_op;

/* Kernel selection for jacobi_sweep_ex(). */
typedef enum {
    JAC_KERNEL_AUTO = 0,   /* planner: plain streaming or temporal blocking        */
    JAC_KERNEL_PLAIN = 1,  /* one sweep per pass over HBM (Eq. 1, 2*elem B/LUP)   */
    JAC_KERNEL_TB = 2,     /* temporally blocked passes of depth t (Sect. 1.3)     */
    JAC_KERNEL_WAVE = 3    /* pipelined passes of depth t, no halo recompute
                              (Sect. 1.3, relaxed synchronisation, Eq. 3)          */
} jac_kernel;

typedef struct jacobi_s *jacobi_t;

/* Description of the launch sequence a sweep call will use (jacobi_plan). */
typedef struct {
    int kernel;            /* JAC_KERNEL_PLAIN, JAC_KERNEL_TB or JAC_KERNEL_WAVE   */
    int t;                 /* depth of the full passes (1 for plain)              */
    int passes;            /* number of kernel launches                           */
    int remainder_t;       /* depth of the last pass (0 if all passes are full)   */
    int tile_x, tile_y;    /* output tile of one CTA (cells)                      */
    int ext_x, ext_y;      /* loaded tile including the t-cell halo              */
    int kchunk;            /* output k-planes per CTA (pipelined: per work item)   */
    int threads;           /* threads per CTA                                     */
    int smem_bytes;        /* dynamic shared memory per CTA                       */
    int grid_x, grid_y, grid_z;
    int emu_adds;          /* FP64 sweeps: additions done on the integer pipes when
                              the grid's values allow it (see jacobi_emulated_add and
                              jacobi_emulated_sum6), in half additions per update:
                              5 = 2 and 3 on alternate planes, 8 = 4 of the 5 */
} jacobi_plan_info;

/*
 * jacobi_create — bind two caller-owned device grids A and B (same dtype, shape,
 * row_pitch) of an nx x ny x nz interior to a handle.
 *   dtype      JAC_F64, JAC_F32 or JAC_BF16 (bf16: 16-bit bit patterns).
 *   grid_a/b   device pointers, 16-byte aligned, (nz+2)*(ny+2)*row_pitch elements.
 *   row_pitch  elements per row, >= nx+2, row_pitch*elem % 16 == 0.
 *   stream     cudaStream_t to launch on (NULL: legacy default stream).
 * Enqueues one copy of A's boundary layer into B, so only A needs the boundary
 * data on entry.  nx, ny, nz >= 1.  Returns JAC_EINVAL for bad arguments.
 */
JAC_API int jacobi_create(jacobi_t *out, int nx, int ny, int nz, int dtype, void *grid_a,
                  void *grid_b, long long row_pitch, void *stream);

/*
 * jacobi_create_inplace — bind ONE caller-owned device grid (layout as for
 * jacobi_create) to a handle whose sweeps update it in place: half the memory of
 * the two grids A and B, the aim of the paper's compressed grid (Sect. 1.3).  The
 * paper shifts every result by one cell so that a sequential sweep never
 * overwrites a value it still needs; here the pipelined passes' counters give the
 * same guarantee, so values stay where they are.  Sweeps on this handle run the
 * pipelined kernel only (JAC_KERNEL_AUTO or JAC_KERNEL_WAVE), every pass of depth
 * >= 2 (the last update of a pass must not overwrite values that the first
 * update of a neighbouring tile still reads): t == 1, or nsweeps == 1, returns
 * JAC_EUNSUPPORTED, and a remainder of one sweep is merged into the last pass
 * (depth t+1).  final_is_b is always 0.  jacobi_sweep_rhs and jacobi_adjoint
 * return JAC_EUNSUPPORTED; jacobi_download with from_b != 0 returns JAC_EINVAL.
 * Needs no boundary copy (there is no second grid).
 */
JAC_API int jacobi_create_inplace(jacobi_t *out, int nx, int ny, int nz, int dtype, void *grid,
                          long long row_pitch, void *stream);

/*
 * jacobi_sweep — nsweeps sweeps of Eq. 1, A -> B -> A ... (Sect. 1.1).
 *   t          temporal-blocking depth request (Sect. 1.3): 0 = planner's choice
 *              (FP64: 1, FP32/bf16: 3), 1 = one sweep per pass (FP64: the
 *              register-march streaming kernel; FP32/bf16: the TMA-ring kernel at
 *              depth 1), t >= 2 = passes of depth min(t, nsweeps) with a shallower
 *              last pass when t does not divide nsweeps.  A depth deeper than the
 *              deepest kernel built (jacobi_max_depth: 8 for every dtype) is
 *              rejected with JAC_EUNSUPPORTED before anything is launched: an
 *              extended tile of depth t needs more than 2t rows, and one warp per
 *              row caps a CTA at 32 rows, so depth 16 has no kernel.
 *   final_is_b set to 1 when the result is in B, else 0.  Every pass (one plain
 *              sweep, or one blocked pass of several sweeps) reads one grid and
 *              writes the other, so this is the parity of the number of passes.
 * nsweeps == 0 is a no-op.  The result values are bit-identical for every t.
 */
JAC_API int jacobi_sweep(jacobi_t h, int nsweeps, int t, int *final_is_b);

/* jacobi_sweep_ex — as jacobi_sweep, with the kernel family forced
 * (JAC_KERNEL_PLAIN: the register-march streaming kernel for every dtype;
 * JAC_KERNEL_TB with t == 1 runs the blocked kernel at depth 1).
 *
 * JAC_KERNEL_WAVE: pipelined passes (Sect. 1.3 with the relaxed synchronisation
 * of Eq. 3).  One persistent launch per pass of depth t (1 <= t <= 32; t == 0:
 * 2 for FP64, 4 for FP32/bf16).  Each work item is one of the t updates of an
 * x-y tile over a few planes, and it starts once the items it reads from and
 * the items that still read the buffer it overwrites are done, as the paper's
 * per-thread counters pace its team.  Updates 1..t-1 of a pass live in ring
 * buffers that the handle allocates on first use (kept until destroy, grown when
 * a deeper pass needs more; 512 MB at most), so no cell is recomputed and
 * each pass reads and writes the grid once.  Every wait on another item is
 * bounded (2 s); a wait that runs out ends the launch, and jacobi_check returns
 * JAC_ETIMEOUT.  Results are bit-identical to the other kernels.  For failure-
 * detection tests only, the environment variable
 * JACOBI_WAVE_TEST_MISSING_PRODUCER=1 withholds the first block of update 1 of
 * every tile (and shortens the wait limit to 0.1 s), so the call times out. */
JAC_API int jacobi_sweep_ex(jacobi_t h, int nsweeps, int t, int kernel, int *final_is_b);

/* jacobi_plan — fill *info with the plan jacobi_sweep_ex(h, nsweeps, t, kernel)
 * would execute, without launching anything (same return codes). */
JAC_API int jacobi_plan(jacobi_t h, int nsweeps, int t, int kernel, jacobi_plan_info *info);

/*
 * jacobi_sweep_rhs — nsweeps correction sweeps of the iterative refinement:
 *   e' = (((((( e[i-1] + e[i+1]) + e[j-1]) + e[j+1]) + e[k-1]) + e[k+1]) + rho) * RN(1/6)
 * on the handle's grids (A = e on entry, boundary layer zero), the Jacobi
 * iteration of (I - J0) e = rho/6 with J0 the sweep of Eq. 1 on a zero
 * boundary.  rho: device grid of the handle's dtype and layout (read only, not
 * written while the call's kernels run; 16-byte aligned, else JAC_EINVAL: it is
 * read through a TMA descriptor, which the handle caches for the last rho seen).
 * dtype JAC_F32 or JAC_BF16 (JAC_EUNSUPPORTED otherwise).  t, final_is_b as in
 * jacobi_sweep (t = 0: depth 4 for FP32, 2 for bf16).
 */
JAC_API int jacobi_sweep_rhs(jacobi_t h, const void *rho, int nsweeps, int t,
                     int *final_is_b);

/*
 * jacobi_residual_accumulate — the FP64 step of the iterative refinement, on an
 * nx x ny x nz interior:
 *   u_out = u_in + (double) e        on the interior;
 *   rho   = s(u_out) - 6.0 * u_out   on the interior, s = the six-neighbour sum
 *                                    of Eq. 1 in its order (boundary data of
 *                                    u_in included), product rounded first;
 * rho is stored in lo_dtype (JAC_F32 or JAC_BF16: RN to FP32, then nearest-even
 * to bf16; JAC_F64 also accepted).  Only interior cells of u_out and rho are
 * written: u_out's boundary layer must already hold the boundary data, rho's
 * boundary layer is never read by the correction sweep.  u_in/u_out: distinct
 * FP64 grids with row pitch u_pitch.  e/rho: lo_dtype grids with row pitch
 * lo_pitch.  Asynchronous on `stream` (cudaStream_t, NULL = default stream).
 */
JAC_API int jacobi_residual_accumulate(int nx, int ny, int nz, const double *u_in,
                               double *u_out, long long u_pitch, const void *e,
                               void *rho, int lo_dtype, long long lo_pitch,
                               void *stream);

/*
 * jacobi_adjoint — reverse sweeps for the gradient of L = sum(W * A_n) (A_n the
 * result of n forward sweeps of Eq. 1).  The handle's grids hold the adjoint
 * field: A = lambda_n (W on the interior, zero boundary layer) on entry.  Each
 * sweep applies the transpose of one forward sweep, which is the same stencil on
 * a zero boundary (it runs on the plain sweep's kernels: the streaming kernel for
 * FP64 at depth 1, the blocked kernels otherwise), and every face
 * cell b of the boundary layer receives RN(1/6) * lambda_s at its interior
 * neighbour: per pass, a band kernel recomputes the pass's levels along
 * the six faces (bit-identical values) and stores them per sweep in a face buffer
 * the handle owns (2*(ny*nz + nx*nz + nx*ny) elements per sweep, allocated on the
 * first call that needs more and kept until jacobi_destroy; JAC_ENOMEM if that
 * allocation fails); it runs on a second stream the handle creates on first use.
 * So that a band can run beside the next pass as well, the passes rotate through
 * A, B and a third grid of the same layout that the handle owns (allocated on
 * the first adjoint call, given A's boundary layer at every call, freed by
 * jacobi_destroy; JAC_ENOMEM if that allocation fails): a pass waits, by an
 * event, only for the band that read the grid it writes, the call stays ordered
 * on the handle's stream, and the last pass writes A or B (final_is_b says
 * which; the other grids' contents are unspecified).  One kernel at the end of the call adds
 * the rows into grad_bdry in sweep order (lambda_n's share first), so the result
 * is deterministic.  grad_bdry: a grid of the handle's layout and dtype, pre-set
 * by the caller (the direct term W on the boundary layer); only its face cells
 * are written.  After nsweeps the interior of the final grid is dL/dA_0 and
 * grad_bdry is dL/dg.  t as in jacobi_sweep (t = 0: depth 3 for FP32, 1 for
 * FP64; deepest 8).  dtype JAC_F32 or JAC_F64.
 */
JAC_API int jacobi_adjoint(jacobi_t h, void *grad_bdry, int nsweeps, int t,
                   int *final_is_b);

/*
 * jacobi_upload / jacobi_download — copy a whole padded grid between host memory
 * and the handle's grid A (upload) or the grid holding a result (download,
 * from_b = the final_is_b of the sweep call), asynchronously on the handle's
 * stream.  host: (nz+2)*(ny+2)*row_pitch elements, same layout as the device
 * grids; page-locked memory makes the copy asynchronous, pageable memory works
 * but synchronises.  Upload also refreshes B's boundary layer from A.
 */
JAC_API int jacobi_upload(jacobi_t h, const void *host);
JAC_API int jacobi_download(jacobi_t h, void *host, int from_b);

/*
 * Batched grids: many independent grids (different shapes, sweep counts and
 * depths) advanced by one persistent kernel launch, recorded once into a CUDA
 * graph and replayed by jacobi_batch_run.  Every grid's sweeps are the same
 * bit-exact sweeps as jacobi_sweep with the same depth.
 */
typedef struct jacobi_batch_s *jacobi_batch_t;

#define JAC_BATCH_NO_GRAPH 1               /* launch directly instead of a CUDA graph  */
#define JAC_BATCH_TEST_MISSING_PRODUCER 2  /* test hook: add one work item that waits
                                              for a tile no item produces, so the run
                                              ends in JAC_ETIMEOUT (bounded wait)      */

/*
 * jacobi_batch_create — plan a batch of `count` grids of one dtype (JAC_F32 or
 * JAC_BF16).  Per grid i: dims[3i..3i+2] = (nx, ny, nz), pitches[i] = row pitch
 * (elements, row a multiple of 16 bytes), grids_a[i]/grids_b[i] = caller-owned
 * device grids (A holds the initial grid and boundary layer; B receives A's
 * boundary layer here), nsweeps[i] >= 0, t[i] = depth (0 or t == NULL: 4;
 * at most 6), tile_x[i] = width of the loaded tile in cells, 64 or 128 (128 only
 * for depths up to 2; 0 or tile_x == NULL: 128 where the depth allows it, else
 * 64), nchunk[i] = k-chunks per pass (0 or nchunk == NULL: planner).  A depth or
 * width without a kernel gives JAC_EUNSUPPORTED.
 * Work items are (grid, pass, tile) in pass-round order; a CTA waits (bounded by
 * wait_limit_s, 0 = 2 s) for the previous pass of its grid.  The library owns the
 * descriptors, the work list and the counters (freed by jacobi_batch_destroy).
 */
JAC_API int jacobi_batch_create(jacobi_batch_t *out, int count, const int *dims,
                                const long long *pitches, void *const *grids_a,
                                void *const *grids_b, const int *nsweeps, const int *t,
                                const int *tile_x, const int *nchunk, int dtype, void *stream,
                                int flags, double wait_limit_s);

/* jacobi_batch_run — enqueue one run of the whole batch on the batch's stream
 * (every grid advances by its own sweep count from A).  final_is_b (count
 * entries, may be NULL) reports per grid whether the result is in B.  A run
 * starts from the current contents of each A, so a second run continues from
 * wherever the first left A (the result itself when it ended in A). */
JAC_API int jacobi_batch_run(jacobi_batch_t b, int *final_is_b);

/* jacobi_batch_info — per grid: depth used, tile width and number of passes;
 * totals: work items and persistent CTAs.  Any pointer may be NULL. */
JAC_API int jacobi_batch_info(jacobi_batch_t b, int *t_used, int *tile_x, int *passes,
                              int *items, int *ctas);

/* jacobi_batch_check — wait for the batch's stream; JAC_ETIMEOUT if a bounded
 * device wait ran out during a run. */
JAC_API int jacobi_batch_check(jacobi_batch_t b);

/* jacobi_batch_destroy — release the batch (not the grids).  NULL is accepted. */
JAC_API int jacobi_batch_destroy(jacobi_batch_t b);

/*
 * jacobi_sweep_noalloc — jacobi_sweep for callers that cannot allocate device
 * memory: code running where cudaMalloc is not allowed or not wanted, such as a
 * host framework that owns every device byte through its own pool allocator, or
 * a plug-in that must not grow the process's device footprint while it runs.
 * There is no counterpart in the paper; it is a deployment convenience.  No
 * handle is needed and the call allocates nothing: the second (ping-pong) grid,
 * the device status word and the FP64 range flag live in one static device
 * array of JAC_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU
 * that loads the library keeps until the process exits.
 *   grid       the caller's device grid (layout as above): input on entry,
 *              result on return (the library copies the result back when the
 *              last pass ends in the scratch grid).  Row padding is not touched.
 *   nsweeps, t as in jacobi_sweep; the call runs the kernels jacobi_sweep runs
 *              with the same arguments (same depths, tiles and FP64 additions).
 *   stream     cudaStream_t (NULL: legacy default stream).
 *   sync       0: return after enqueueing; nonzero: wait for the stream and
 *              report a device-side timeout as JAC_ETIMEOUT.
 * The padded grid, (nz+2)*(ny+2)*row_pitch elements, must fit in
 * JAC_NOALLOC_SCRATCH_BYTES - 256 bytes (about 4.1 M FP64 or 8.4 M FP32 cells);
 * larger grids are rejected with JAC_EINVAL before anything runs.
 * First call on a device: it looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current), which is also when the
 * driver commits the array's device memory (modules load lazily), so the first
 * call does reserve JAC_NOALLOC_SCRATCH_BYTES on that device; make that first
 * call before any stream capture.
 * Timeouts: the status word is sticky.  A call with sync = 0 does not report a
 * timeout of its own kernels; it stays recorded until the next call made with
 * sync != 0, which returns JAC_ETIMEOUT and clears it.
 * Every call shares the one scratch array, which keeps the previous call's
 * contents (each call re-initialises what it needs): calls that can overlap on
 * the GPU (different streams, or different threads) race, so serialise them.
 */
#define JAC_NOALLOC_SCRATCH_BYTES (32u << 20)
JAC_API int jacobi_sweep_noalloc(int nx, int ny, int nz, int dtype, void *grid,
                                 long long row_pitch, int nsweeps, int t, void *stream,
                                 int sync);

/*
 * jacobi_emulated_add — out[i] = a[i] + b[i] computed the way the FP64 plain
 * sweep computes its integer-pipe additions: exact IEEE-754 binary64 addition
 * with round-to-nearest-even, done with integer instructions for positive
 * normal operands whose exponents differ by at most 31 (the FP64 unit for every
 * other pair).  The results equal the FP64 unit's bit for bit; this entry point
 * lets tests check that on any set of pairs.  Device arrays of n doubles;
 * asynchronous on `stream`.
 */
JAC_API int jacobi_emulated_add(const double *a, const double *b, double *out, long long n,
                                void *stream);

/*
 * jacobi_emulated_sum6 — out[i] = ((((x0 + x1) + x2) + x3) + x4) + x5 with
 * x_j = x[j*n + i], each addition rounded to nearest even in binary64 (the
 * partial sums of Eq. 1), computed the way the FP64 sweeps compute them: an
 * unpacked running sum on the integer pipes, and the FP64 unit for every warp
 * that holds an operand which is not a positive normal double or an exponent gap
 * outside that routine's window.  The results equal the FP64 unit's sequential
 * sums bit for bit; this entry point lets tests check that on any set of
 * 6-tuples.  x: device array of 6*n doubles, out: n doubles; asynchronous on
 * `stream`.
 */
JAC_API int jacobi_emulated_sum6(const double *x, double *out, long long n, void *stream);

/*
 * jacobi_copy_planes — copy nplanes consecutive k-planes of one padded grid into
 * another of the same row pitch and ny (plane size plane_elems = row_pitch*(ny+2)
 * elements of elem_bytes each): the halo exchange of the z-slab decomposition
 * (multi-layer halos, Sect. 2.1).  dst/src point at the first plane to copy;
 * device memory; asynchronous on `stream`.  Planes of one slab grid must not
 * overlap the copied range of another.
 */
JAC_API int jacobi_copy_planes(void *dst, const void *src, long long plane_elems,
                               int elem_bytes, int nplanes, void *stream);

/* jacobi_check — wait for the handle's stream and report a device-side status
 * (JAC_ETIMEOUT when a bounded wait ran out) or a CUDA error (JAC_ECUDA).  The
 * status word is cleared. */
JAC_API int jacobi_check(jacobi_t h);

/* jacobi_destroy — release the handle (not the grids).  NULL is accepted. */
JAC_API int jacobi_destroy(jacobi_t h);

/* jacobi_strerror — static text for a status code. */
JAC_API const char *jacobi_strerror(int code);

/*
 * jacobi_pipe_probe — measurement kernels for the roofline of the sweeps (no
 * counterpart in the paper; the paper's own model, Sect. 1.4 Eq. 4-5, needs the
 * machine's rates as inputs).  Launches `blocks` x `threads` threads (threads a
 * multiple of 32, at most 256), each running JAC_PROBE_CHAINS independent
 * dependency chains of `iters` operations of one kind from registers:
 *   JAC_PROBE_DADD     FP64 additions (the FP64 unit)
 *   JAC_PROBE_FADD     FP32 additions
 *   JAC_PROBE_LOP3     3-input logic operations (the integer ALU pipe)
 *   JAC_PROBE_IMAD     32-bit integer multiply-adds (the FMA pipe)
 *   JAC_PROBE_EMU_ADD  exact binary64 additions on the integer pipes, one
 *                      packed addition at a time (see jacobi_emulated_add)
 *   JAC_PROBE_ACC_ADD  additions to the unpacked exact running sum the FP64
 *                      sweeps use (see jacobi_emulated_sum6)
 * so one launch performs blocks*threads*iters*JAC_PROBE_CHAINS operations; the
 * caller times it (CUDA events).  out: device array of blocks*threads doubles
 * that receives each thread's chain values.  Asynchronous on `stream`.
 */
#define JAC_PROBE_CHAINS 8
enum jac_probe {
    JAC_PROBE_DADD = 0,
    JAC_PROBE_FADD = 1,
    JAC_PROBE_LOP3 = 2,
    JAC_PROBE_IMAD = 3,
    JAC_PROBE_EMU_ADD = 4,
    JAC_PROBE_ACC_ADD = 5
};
JAC_API int jacobi_pipe_probe(int kind, double *out, int blocks, int threads, int iters,
                              void *stream);

/* jacobi_max_depth — the deepest temporal-blocking depth (Sect. 1.3) built for
 * dtype and op (jac_op); every depth from 1 to it exists.  JAC_EINVAL for an
 * unknown dtype or op; 0 when the operation has no kernel for the dtype. */
JAC_API int jacobi_max_depth(int dtype, int op);

/* jacobi_version — library version as 10000*major + 100*minor + patch. */
JAC_API int jacobi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI_GB300_H */
