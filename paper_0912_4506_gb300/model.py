"""Performance model of a temporally-blocked pass: the paper's single-cache model
(Sect. 1.4, Eq. 4-5) restated for one GB300 and used to order the autotuner's
candidates.

The paper's Eq. 4 gives the time of t block updates of a thread team as the
memory transfer of one load and one store (16 B per update at the single-
thread memory bandwidth M_s,1) plus 2(t-1) cache transfers of 8 B at the shared
cache bandwidth M_c; Eq. 5 turns it into the speedup over the standard sweep,
    S = (M_s,1 / M_s) * t / (1 + (t - 1) * M_s,1 / M_c).
On the GPU the roles are: HBM for M_s (the TMA copies stream every plane once per
pass), the SM's shared memory for M_c (level planes of a CTA), and a third limit
the CPU model leaves out because a CPU core's load/store units do all of it: the
instruction issue of the level updates.  TMA, shared memory and the issue
scheduler are separate resources that overlap, so the GPU form takes the
largest of the three times instead of their sum:
    time per useful update = max(B_hbm / M_s, B_smem / M_c, I * r / R_issue),
with B_hbm the HBM bytes per useful update (the extended tile read once, the
output tile written once, the k-chunk's 2t-plane pipeline fill), B_smem the
shared-memory bytes (level 0 read from the ring, two neighbour rows read and one
row written per level below t), r the recompute factor of the shrinking levels
(every lane computes its whole row, valid or not), I the instructions per
computed cell update and R_issue the thread instructions the GPU issues per
second.  Every input is a number the caller measures (bench.py: MEASURED_PEAKS.json
and the pipe probes) or takes from a profile; nothing here is tuned to fit.
"""

# Shared-memory bandwidth of one SM (bytes per clock, 32 banks of 4 bytes) and the
# issue rate (thread instructions per clock: 4 schedulers x 32 lanes); both are
# architectural figures of the sm_100 family.
SMEM_BYTES_PER_CLK_PER_SM = 128
ISSUE_THREAD_INST_PER_CLK_PER_SM = 128


def eq5_speedup(t, ms1, ms, mc, teams=1):
    """Eq. 5 as printed: expected speedup of pipelined temporal blocking with t
    updates per team and `teams` teams over the standard in-memory sweep."""
    tt = t * teams
    return (ms1 / ms) * tt / (1.0 + (tt - 1) * ms1 / mc)


def eq4_time(t, ms1, mc, teams=1, word=8):
    """Eq. 4 as printed: time of t*teams block updates, 16 B from memory and
    2(tT-1) transfers of `word` bytes in the cache (seconds per byte-normalised
    update when bandwidths are in B/s)."""
    tt = t * teams
    return 2 * word / ms1 + 2 * (tt - 1) * word / mc


def tile(t, ex, ey, es, align_bytes=16):
    """Output tile (ox, oy) of an extended tile ex x ey at depth t: ox rounded
    down to the TMA alignment (16 bytes), as the planner does."""
    a = align_bytes // es
    ox = ((ex - 2 * t) // a) * a
    oy = ey - 2 * t
    return ox, oy


def recompute(t, ex, ey, es):
    """Computed cell updates per useful update: level s is computed on rows
    [s, ey-s) across the full tile width."""
    ox, oy = tile(t, ex, ey, es)
    computed = sum(ex * (ey - 2 * s) for s in range(1, t + 1))
    return computed / (t * ox * oy)


def hbm_bytes(t, ex, ey, es, kz=None):
    """HBM bytes per useful update of one pass (kz: output planes per CTA; the
    2t planes of pipeline fill are read once more per chunk)."""
    ox, oy = tile(t, ex, ey, es)
    per_plane = es * ex * ey + es * ox * oy
    fill = 1.0 if kz is None else (kz + 2 * t) / kz
    return per_plane * fill / (ox * oy * t)


def smem_bytes(t, ex, ey, es):
    """Shared-memory bytes per useful update: level 0 read once per cell from the
    ring; level s >= 1 reads two neighbour rows of level s-1 per cell and, below
    level t, writes its own row."""
    ox, oy = tile(t, ex, ey, es)
    total = es * ex * ey  # level 0 read
    for s in range(1, t + 1):
        cells = ex * (ey - 2 * s)
        total += es * cells * (2 + (1 if s < t else 0))
    return total / (ox * oy * t)


def predict(t, ex, ey, es, hbm_gbs, sm_mhz, sms, inst_per_update, kz=None, pipe_ops=0.0,
            pipe_gops=None, nxy=None):
    """Predicted useful lattice-site updates per second (GLUP/s) of a pass and
    the bound that sets it: max of the HBM, shared-memory and issue times, and of
    an arithmetic pipe's time when `pipe_ops` operations per computed update run
    on a pipe of `pipe_gops` measured operations per second (the FP64 unit).
    nxy = (nx, ny) charges the partial tiles at the grid's x and y ends to the
    computed updates.  A ceiling: every resource at its full rate."""
    clk = sm_mhz * 1e6
    r = recompute(t, ex, ey, es)
    if nxy is not None:
        # partial tiles at the x and y ends of a grid of nx x ny interior cells
        ox, oy = tile(t, ex, ey, es)
        nx, ny = nxy
        r *= (-(-nx // ox) * ox * -(-ny // oy) * oy) / (nx * ny)
    t_hbm = hbm_bytes(t, ex, ey, es, kz) / (hbm_gbs * 1e9)
    t_smem = smem_bytes(t, ex, ey, es) / (SMEM_BYTES_PER_CLK_PER_SM * sms * clk)
    t_issue = inst_per_update * r / (ISSUE_THREAD_INST_PER_CLK_PER_SM * sms * clk)
    times = {"hbm": t_hbm, "smem": t_smem, "issue": t_issue}
    if pipe_ops and pipe_gops:
        times["pipe"] = pipe_ops * r / (pipe_gops * 1e9)
    bound = max(times, key=times.get)
    return 1.0 / times[bound] / 1e9, bound


def order_candidates(cands, shape, es, hbm_gbs, sm_mhz, sms, inst_per_update, ey=32):
    """Batched-grid candidates (tile width, depth) sorted by predicted rate on a
    grid of `shape`, fastest first; a tile wider than the grid is charged for the
    columns it wastes."""
    nx, ny, nz = shape

    def rate(c):
        ex, t = c
        ox, oy = tile(t, ex, ey, es)
        ntx = -(-nx // ox)
        nty = -(-ny // oy)
        waste = (ntx * ox * nty * oy) / (nx * ny)
        g, _ = predict(t, ex, ey, es, hbm_gbs, sm_mhz, sms, inst_per_update, kz=nz)
        return g / waste

    return sorted(cands, key=rate, reverse=True)
