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

Here every slab lives on the same GPU (peer copies through jacobi_copy_planes);
the plan (``halo_plan``) is the same one a multi-process run uses, and
tests/test_slabs_gloo.py runs it across gloo ranks on the CPU oracle.
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
