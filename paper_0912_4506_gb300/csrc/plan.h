// Host-side launch planning shared by every entry point of the library (the
// handle-based sweeps, the batched grids and the allocation-free sweep): the
// tensor-map encoder, the kernel tables, the tile geometry of a temporally-
// blocked pass, the k-chunk choice and the split of n sweeps into passes.
//
// Nothing here allocates memory: tables and per-device caches are fixed-size
// static arrays, filled once under a mutex.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "launch.h"

namespace jac {

constexpr int kMaxDevices = 64;
constexpr int kMaxDepth = 8;  // deepest temporal-blocking depth any table holds

int elem_size(int dtype);
int floor_div(int a, int b);

// 3D TMA descriptor over the padded grid (nx+2, ny+2, nz+2) at `base` with a
// (box_x, box_y, 1) box.  Elements outside the padded grid (the row padding and
// anything beyond the array) read as zero.  False when the CUDA driver rejects it.
bool encode_grid_map(CUtensorMap* map, int dtype, const Geom& g, const void* base, int box_x,
                     int box_y);

// Blocked-kernel entry of (dtype, mode) for depth T, or nullptr when no kernel
// of that depth is built.  Every table holds the depths 1..max_depth without gaps.
const TBEntry* tb_entry(int dtype, int mode, int T);
int max_depth(int dtype, int mode);

// Resident CTAs per SM of a blocked kernel on `device` (its dynamic shared
// memory attribute is set there first, once per device and kernel).
int tb_occupancy(const TBEntry& e, int device);

// Number of k-chunks: enough CTAs to fill whole waves of `slots` resident CTAs,
// with chunks long enough that the 2T-plane pipeline fill of each stays small.
int pick_chunks(int nz, int T, long long tiles, long long slots);

// Tile geometry of one blocked pass with an extended tile of (32*V) x NW cells at
// depth T: output tile ox x oy (ox a multiple of the 16-byte TMA alignment), the
// aligned x origin of tile 0, the tile counts and the k-chunking (nchunk_req > 0:
// that many chunks; otherwise pick_chunks over `slots`).
struct TileGeom {
    int ox, oy, x0_first, ntx, nty, kz, nchunk;
    bool ok;  // false: the extended tile leaves no output cells at this depth
};
TileGeom tile_geom(int dtype, const Geom& g, int V, int NW, int T, long long slots,
                   int nchunk_req);

// Depth used when the caller leaves it to the planner (t = 0).
int default_t(int dtype, int mode);

// The plain streaming kernel of a dtype (FP64: the variant with the configured
// number of integer-pipe additions) and its launch grid.
const PlainEntry* plain_for(int dtype);
void plain_grid(const PlainEntry* pe, int dtype, const Geom& g, int device, int num_sms,
                dim3* grid, int* kchunk);

// Split of n sweeps at requested depth t into passes: n_full passes of depth
// t_full, then one pass of depth t_last (0: none).  JAC_EUNSUPPORTED when t is
// deeper than the deepest kernel built for (dtype, mode).
struct DepthPlan {
    int t_full, n_full, t_last;
    int passes() const { return n_full + (t_last > 0 ? 1 : 0); }
    int depth(int p) const { return p < n_full ? t_full : t_last; }
};
int plan_depths(int dtype, int mode, int nsweeps, int t, DepthPlan* out);

// Pipelined (wavefront) passes.  A pass of depth t keeps levels 1..t-1 in ring
// buffers of rp = R * kb planes each; kb (planes per work item) is the largest
// power of two up to 32 whose rings fit 512 MB (kb = 1 otherwise; larger items
// measured faster than rings held to the L2 size), R = 4,
// ticket skew sk = 2.  JACOBI_WAVE="kb,R" or "kb,R,sk" overrides them
// (measurement runs); sk defaults to min(2, R - 2) and must stay below R - 1.
constexpr int kMaxWaveDepth = 32;
// The pipelined kernel of a dtype (JACOBI_WAVE_VARIANT=i selects alternate i of
// its table, for measurement runs).
const WaveEntry* wave_for(int dtype);
struct WavePlan {
    int t, kb, R, sk, rp, nb, ntx, nty, nitems, ctas;
    size_t ring_bytes;   // (t-1) * rp planes
    size_t flags;        // t * ntiles * nb done flags
};
bool wave_plan(int dtype, const Geom& g, int t, const WaveEntry& e, int device, int num_sms,
               WavePlan* out);

// Default depth of the pipelined passes.
int default_wave_t(int dtype);

}  // namespace jac
