"""z-slab domain decomposition with multi-layer halos (Sect. 2.1 of the paper).

The global grid is cut into slabs along k.  Each slab keeps its own padded grid
covering its core planes plus h halo planes on each side (and one more plane
that acts as the slab grid's boundary layer).  Every pass of depth t <= h starts
with a halo exchange (h+1 planes from each neighbour's core, the paper's "h
layers exchanged every h updates", one message per side instead of one per
sweep), after which each slab runs an ordinary temporally-blocked pass on its
own grid: level s is exact on the slab's planes except the s outermost on each
side, so after t <= h levels the core is exact ("update number s covers a
domain that is h - s layers larger").  Only k is cut, so the dimension-by-
dimension exchange of the paper reduces to one axis and there are no edge or
corner messages.  The result is bit-identical to the single-grid sweep.

``SlabJacobi`` keeps every slab on one GPU (device copies through
jacobi_copy_planes); ``RankSlab`` is the same decomposition with one slab per
process and the halos exchanged by point-to-point messages, following the same
plan (``halo_plan``).
"""
import torch

from . import _lib, api


def slab_ranges(nz, nslabs):
    """Core planes (z0, z1), inclusive, 1-based, of each slab: near-equal cuts."""
    if nslabs < 1 or nslabs > nz:
        raise ValueError("need 1 <= nslabs <= nz")
    base, extra = divmod(nz, nslabs)
    out, z = [], 1
    for i in range(nslabs):
        size = base + (1 if i < extra else 0)
        out.append((z, z + size - 1))
        z += size
    return out


def slab_extent(z0, z1, nz, h):
    """Global planes [lo, hi] a slab grid holds: its core, h halo planes per side
    and one plane beyond them (the slab grid's boundary layer), clipped to the
    global grid [0, nz+1]."""
    return max(0, z0 - h - 1), min(nz + 1, z1 + h + 1)


def halo_plan(nz, nslabs, h):
    """Copies of one halo exchange: list of (dst_slab, dst_plane_global,
    src_slab, nplanes).  Slab i's planes below its core come from slab i-1's
    core, the planes above from slab i+1's core; every core needs >= h+1 planes."""
    ranges = slab_ranges(nz, nslabs)
    for z0, z1 in ranges:
        if z1 - z0 + 1 < h + 1 and nslabs > 1:
            raise ValueError("every slab core needs at least h+1 planes")
    plan = []
    for i, (z0, z1) in enumerate(ranges):
        lo, hi = slab_extent(z0, z1, nz, h)
        if i > 0 and lo < z0:        # below the core: from slab i-1
            plan.append((i, lo, i - 1, z0 - lo))
        if i < nslabs - 1 and hi > z1:  # above the core: from slab i+1
            plan.append((i, z1 + 1, i + 1, hi - z1))
    return plan


class SlabJacobi:
    """n sweeps of a global grid through nslabs z-slabs with h-plane halos."""

    def __init__(self, A, nslabs, h):
        nx, ny, nz, px = api.grid_geom(A)
        self.nx, self.ny, self.nz, self.px = nx, ny, nz, px
        self.h = h
        self.ranges = slab_ranges(nz, nslabs)
        self.plan = halo_plan(nz, nslabs, h)
        self.dtype = A.dtype
        self.device = A.device
        self.es = A.element_size()
        self.plane = px * (ny + 2)
        self.slabs = []
        for z0, z1 in self.ranges:
            lo, hi = slab_extent(z0, z1, nz, h)
            g0 = api.alloc_grid(nx, ny, hi - lo - 1, A.dtype, A.device, pitch=px)
            g0.copy_(A[lo:hi + 1])
            g1 = api.alloc_like(g0)
            # two handles with swapped roles, so a pass can start from either grid
            j0 = api.Jacobi(g0, g1)
            j1 = api.Jacobi(g1, g0)
            self.slabs.append({"lo": lo, "hi": hi, "z0": z0, "z1": z1, "grids": (g0, g1),
                               "jacs": (j0, j1), "cur": 0})

    def _cur(self, s):
        return s["grids"][s["cur"]]

    def exchange(self):
        """Copy every slab's halo planes from its neighbours' cores."""
        stream = torch.cuda.current_stream(self.device).cuda_stream
        for dst, gplane, src, n in self.plan:
            d, s = self.slabs[dst], self.slabs[src]
            dg, sg = self._cur(d), self._cur(s)
            _lib.jacobi_copy_planes(dg.data_ptr() + (gplane - d["lo"]) * self.plane * self.es,
                                    sg.data_ptr() + (gplane - s["lo"]) * self.plane * self.es,
                                    self.plane, self.es, n, stream)

    def sweep(self, nsweeps, t=None):
        """nsweeps sweeps: a halo exchange, then at most h sweeps per slab."""
        t = self.h if t is None else min(t, self.h)
        done = 0
        while done < nsweeps:
            d = min(t, nsweeps - done)
            self.exchange()
            for s in self.slabs:
                j = s["jacs"][s["cur"]]
                out = j.sweep(d, d, api.JAC_KERNEL_TB if d > 1 else api.JAC_KERNEL_PLAIN)
                if out is j.B:
                    s["cur"] ^= 1
            done += d
        return self

    def gather(self, out=None):
        """The global grid: every slab's core planes plus the global boundary."""
        out = api.alloc_grid(self.nx, self.ny, self.nz, self.dtype, self.device,
                             pitch=self.px) if out is None else out
        for i, s in enumerate(self.slabs):
            cur = self._cur(s)
            a = s["z0"] if i > 0 else 0
            b = s["z1"] if i < len(self.slabs) - 1 else self.nz + 1
            out[a:b + 1].copy_(cur[a - s["lo"]:b - s["lo"] + 1])
        return out

    def close(self):
        for s in self.slabs:
            for j in s["jacs"]:
                j.close()


class RankSlab:
    """This process's slab of a z-slab decomposition across processes (one slab
    per rank, Sect. 2.1's multi-layer halos between processes).

    ``slab`` holds global planes lo..hi (``slab_extent`` of this rank's core) of a
    padded grid of nx x ny x nz interior cells, as a tensor of shape
    (hi-lo+1, ny+2, row_pitch): a CUDA tensor swept by the library, or a CPU
    tensor swept by ``sweeper(array, d)`` (a callable returning the array after d
    sweeps; tests pass the oracle).  Every pass of depth d <= h starts with one
    halo exchange: h+1 planes to and from each neighbouring rank by point-to-point
    send/recv over ``torch.distributed`` (NCCL between GPUs, gloo between CPU
    processes), into and out of the slab's own memory; then a local pass of
    depth d.  The cores of all ranks together hold exactly the single-grid result.
    """

    def __init__(self, nx, ny, nz, h, slab, rank, world, sweeper=None, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.nx, self.ny, self.nz, self.h = nx, ny, nz, h
        self.rank, self.world, self.group = rank, world, group
        self.z0, self.z1 = slab_ranges(nz, world)[rank]
        self.lo, self.hi = slab_extent(self.z0, self.z1, nz, h)
        if slab.shape[0] != self.hi - self.lo + 1 or slab.shape[1] != ny + 2:
            raise ValueError("slab must hold planes lo..hi of the global grid")
        plan = halo_plan(nz, world, h)
        # (first global plane, planes, peer): my core planes to send, my halos to receive
        self.sends = [(gp, k, dst) for dst, gp, src, k in plan if src == rank]
        self.recvs = [(gp, k, src) for dst, gp, src, k in plan if dst == rank]
        self.sweeper = sweeper
        self.grids = [slab]
        self.cur = 0
        if slab.is_cuda and sweeper is None:
            g0 = api.as_grid(slab, nx)
            g1 = api.alloc_like(g0)
            self.grids = [slab, g1.as_strided(slab.shape, slab.stride())]
            # two handles with swapped roles, so a pass can start from either grid
            self.jacs = (api.Jacobi(g0, g1), api.Jacobi(g1, g0))
        elif sweeper is None:
            raise ValueError("a CPU slab needs a sweeper")

    def current(self):
        """The tensor that holds this slab's current planes lo..hi."""
        return self.grids[self.cur]

    def exchange(self):
        """Send my core planes to the neighbours' halos and receive my halos."""
        if self.world == 1:
            return
        dist, cur, lo = self.dist, self.current(), self.lo
        ops = [dist.P2POp(dist.isend, cur[gp - lo:gp - lo + k], peer, self.group)
               for gp, k, peer in self.sends]
        ops += [dist.P2POp(dist.irecv, cur[gp - lo:gp - lo + k], peer, self.group)
                for gp, k, peer in self.recvs]
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def local_pass(self, d, t=None):
        """d <= h sweeps on this slab alone (after an exchange): one blocked pass of
        depth d, or with t the library's choice at depth t (t = 1: d plain sweeps,
        the FP64 choice) in one call."""
        if self.sweeper is not None:
            self.grids[0] = self.sweeper(self.grids[0], d)
            return
        j = self.jacs[self.cur]
        if t is None:
            out = j.sweep(d, d, api.JAC_KERNEL_TB if d > 1 else api.JAC_KERNEL_PLAIN)
        else:
            out = j.sweep(d, min(t, d))
        if out is j.B:
            self.cur ^= 1

    def passes(self, nsweeps, t=None):
        """Sweeps between exchanges for nsweeps sweeps (each at most h)."""
        t = self.h if t is None else min(t, self.h)
        out, done = [], 0
        while done < nsweeps:
            out.append(min(t, nsweeps - done))
            done += out[-1]
        return out

    def sweep(self, nsweeps, t=None, kernel_t=None):
        """nsweeps sweeps: per exchange one halo exchange, then at most h sweeps
        (t: sweeps between exchanges, default h; kernel_t: depth of the library's
        passes inside, default one blocked pass; a single rank needs no exchange
        and sweeps in one call)."""
        if self.world == 1 and self.sweeper is None:
            self.local_pass(nsweeps, kernel_t if kernel_t is not None else t or self.h)
            return self
        for d in self.passes(nsweeps, t):
            self.exchange()
            self.local_pass(d, kernel_t)
        return self

    def core(self):
        """This rank's share of the global grid: its core planes, plus the global
        boundary plane below (rank 0) or above (last rank)."""
        a = self.z0 if self.rank > 0 else 0
        b = self.z1 if self.rank < self.world - 1 else self.nz + 1
        return self.current()[a - self.lo:b - self.lo + 1]

    def close(self):
        for j in getattr(self, "jacs", ()):
            j.close()
        self.jacs = ()


def exchange_in_process(slabs_):
    """The halo exchange of a list of RankSlab objects held by one process (one
    per rank, in rank order): the same planes as the point-to-point exchange,
    moved by tensor copies.  Cores and halos are disjoint, so the order of the
    copies does not matter."""
    for me in slabs_:
        for gp, k, peer in me.recvs:
            src = slabs_[peer]
            me.current()[gp - me.lo:gp - me.lo + k].copy_(
                src.current()[gp - src.lo:gp - src.lo + k])
