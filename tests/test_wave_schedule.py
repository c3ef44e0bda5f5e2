"""The schedule of the pipelined (wavefront) passes, on the CPU: a restatement of
the device's ticket decode (order (b + sk s, s, tile)) and of its three start
conditions (blocks b-1..b+1 of level s-1 of the 3 x 3 tiles; the three level-s+1
readers of ring block b-R; in place, blocks b-1..b+1 of level 1), checked for the
property the kernel's progress rests on: every item waits only for items with
smaller tickets when R > sk + 1 (and t >= 2 in place), so a persistent grid of
any number of CTAs, each taking tickets in order, finishes."""
import itertools

import pytest


def decode_all(t, nb, ntiles, sk):
    """Tickets in order -> (s, b, tile), as the control warp decodes them."""
    out = []
    d, base, it = 1, 0, 0
    total = t * nb * ntiles
    while it < total:
        over = d - (nb - 1)
        lo = 1 if over <= 0 else max(1, -(-over // sk))
        hi = min(t, d // sk)
        cnt = (hi - lo + 1) * ntiles if hi >= lo else 0
        if it < base + cnt:
            s = lo + (it - base) // ntiles
            tile = (it - base) % ntiles
            out.append((s, d - sk * s, tile))
            it += 1
        else:
            base += cnt
            d += 1
    return out


def deps(item, t, nb, ntx, nty, R, inplace):
    s, b, tile = item
    tx, ty = tile % ntx, tile // ntx
    res = []
    for dy, dx in itertools.product((-1, 0, 1), repeat=2):
        x, y = tx + dx, ty + dy
        if not (0 <= x < ntx and 0 <= y < nty):
            continue
        n = y * ntx + x
        conds = []
        if s >= 2:
            conds.append((s - 1, b))
        if s < t and b >= R:
            conds.append((s + 1, b - R))
        if s == t and inplace:
            conds.append((1, b))
        for lev, mid in conds:
            for bb in range(max(mid - 1, 0), min(mid + 1, nb - 1) + 1):
                res.append((lev, bb, n))
    return res


GEOMS = [(t, nb, ntx, nty) for t in (1, 2, 3, 5) for nb in (1, 2, 7) for ntx, nty in
         ((1, 1), (3, 2), (4, 5))]


@pytest.mark.parametrize("t,nb,ntx,nty", GEOMS)
def test_decode_enumerates_every_item_once(t, nb, ntx, nty):
    for sk in (1, 2, 3):
        items = decode_all(t, nb, ntx * nty, sk)
        assert sorted(items) == sorted((s, b, tile) for s in range(1, t + 1)
                                       for b in range(nb) for tile in range(ntx * nty))


@pytest.mark.parametrize("t,nb,ntx,nty", GEOMS)
def test_every_dependency_has_a_smaller_ticket(t, nb, ntx, nty):
    for sk, R in ((1, 3), (2, 4), (3, 5), (2, 6)):
        for inplace in (False, True):
            if inplace and t < 2:
                continue
            items = decode_all(t, nb, ntx * nty, sk)
            ticket = {it: k for k, it in enumerate(items)}
            for it in items:
                for dep in deps(it, t, nb, ntx, nty, R, inplace):
                    assert ticket[dep] < ticket[it], (sk, R, inplace, it, dep)


def test_ring_depth_below_skew_plus_two_breaks_the_order():
    """With R = sk + 1 some ring-slot reader is handed out after its writer: the
    planner's R > sk + 1 rule is needed."""
    t, nb, ntx, nty, sk, R = 3, 7, 2, 2, 2, 3
    items = decode_all(t, nb, ntx * nty, sk)
    ticket = {it: k for k, it in enumerate(items)}
    assert any(ticket[dep] > ticket[it] for it in items
               for dep in deps(it, t, nb, ntx, nty, R, False))


@pytest.mark.parametrize("workers", [1, 2, 5, 64])
def test_persistent_grid_finishes(workers):
    """Workers take tickets in order (up to three held each, as a CTA with its
    control warp does) and start an item once its dependencies are done; every
    item finishes, whatever the number of workers."""
    t, nb, ntx, nty, sk, R = 4, 6, 3, 3, 2, 4
    items = decode_all(t, nb, ntx * nty, sk)
    done, nxt = set(), 0
    held = [[] for _ in range(workers)]
    for _ in range(10 * len(items)):
        progressed = False
        for w in range(workers):
            while len(held[w]) < 3 and nxt < len(items):
                held[w].append(items[nxt])
                nxt += 1
            if held[w] and all(d in done for d in deps(held[w][0], t, nb, ntx, nty, R, True)):
                done.add(held[w].pop(0))
                progressed = True
        if len(done) == len(items):
            break
        assert progressed, "no worker can start its next item"
    assert len(done) == len(items)
