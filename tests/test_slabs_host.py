"""Host logic of the z-slab decomposition (Sect. 2.1 multi-layer halos), no GPU:
the cores partition the interior planes, and one halo exchange fills exactly the
planes each slab holds outside its core, every plane copied from the core of the
slab that owns it."""
import itertools

import pytest

from paper_0912_4506_gb300 import slabs


@pytest.mark.parametrize("nz,nslabs,h", [(10, 1, 2), (10, 2, 2), (17, 3, 3), (64, 4, 4),
                                          (65, 5, 1), (40, 8, 4), (9, 3, 2)])
def test_halo_plan_covers_exactly_the_halo(nz, nslabs, h):
    ranges = slabs.slab_ranges(nz, nslabs)
    # cores partition 1..nz in order
    assert ranges[0][0] == 1 and ranges[-1][1] == nz
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert b0 == a1 + 1 and a0 <= a1
    plan = slabs.halo_plan(nz, nslabs, h)
    filled = {i: set() for i in range(nslabs)}
    for dst, plane, src, n in plan:
        z0, z1 = ranges[src]
        for p in range(plane, plane + n):
            assert z0 <= p <= z1, "copied plane lies in the source slab's core"
            assert p not in filled[dst], "no plane is copied twice"
            filled[dst].add(p)
    for i, (z0, z1) in enumerate(ranges):
        lo, hi = slabs.slab_extent(z0, z1, nz, h)
        # planes held outside the core and inside the interior: exactly the copies
        want = {p for p in itertools.chain(range(lo, z0), range(z1 + 1, hi + 1))
                if 1 <= p <= nz}
        assert filled[i] == want
        # the held region reaches h planes past the core (or the grid boundary)
        assert lo == max(0, z0 - h - 1) and hi == min(nz + 1, z1 + h + 1)


def test_cores_too_thin_for_the_halo_are_rejected():
    with pytest.raises(ValueError):
        slabs.halo_plan(10, 4, 3)
    with pytest.raises(ValueError):
        slabs.slab_ranges(5, 6)
