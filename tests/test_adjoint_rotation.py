"""The adjoint's grid rotation, on the CPU: a restatement of the host's choice of
output grid per pass (A, B and the handle's third grid C; a band kernel reads
each pass's input beside the pass) checked for what the call's correctness and
its overlap rest on: no pass writes its own input or a grid a band still reads
without waiting for that band, the last pass writes A or B, every band is waited
for before the face rows are reduced, and only the last pass ever waits for the
band of the pass just before it."""
import pytest

A, B, C = 0, 1, 2


def next_grid(cur, prev, last):
    """Output grid of a pass reading `cur` (the previous pass read `prev`)."""
    d = B if prev is None else 3 - cur - prev
    if last and d == C:
        d = prev
    return d


def simulate(passes):
    """Events of one call: ('band', grid), ('wait', grid), ('pass', src, dst),
    ('reduce',); the band of a pass reads its input grid."""
    ev, pending = [], set()
    cur, prev = A, None
    for p in range(passes):
        ev.append(("band", cur))
        pending.add(cur)
        dst = next_grid(cur, prev, p + 1 == passes)
        if dst in pending:
            ev.append(("wait", dst))
            pending.discard(dst)
        ev.append(("pass", cur, dst))
        prev, cur = cur, dst
    for g in sorted(pending):
        ev.append(("wait", g))
    ev.append(("reduce",))
    return ev, cur


@pytest.mark.parametrize("passes", range(1, 40))
def test_rotation_invariants(passes):
    ev, final = simulate(passes)
    assert final in (A, B)
    reading = set()  # grids a band reads that no wait has covered yet
    inputs = []
    for e in ev:
        if e[0] == "band":
            reading.add(e[1])
        elif e[0] == "wait":
            reading.discard(e[1])
        elif e[0] == "pass":
            _, src, dst = e
            assert dst != src
            assert dst not in reading, (passes, e)  # never overwrite a band's input
            inputs.append(src)
        else:
            assert not reading  # every band done before the reduction
    assert len(inputs) == passes and inputs[0] == A


@pytest.mark.parametrize("passes", range(2, 40))
def test_only_the_last_pass_waits_for_the_previous_band(passes):
    """Pass p + 1 writes a grid the band of pass p does not read, so that band
    overlaps the next pass; the last pass may be redirected from C to the grid the
    previous band reads, and then waits for it."""
    ev, _ = simulate(passes)
    bands, p, redirected = [], 0, False
    for e in ev:
        if e[0] == "band":
            bands.append(e[1])  # bands[p]: the grid pass p reads
        elif e[0] == "wait" and p < passes and p >= 1 and e[1] == bands[p - 1]:
            assert p == passes - 1, (passes, p)  # waits for the previous band
            redirected = True
        elif e[0] == "pass":
            p += 1
    # the redirect happens exactly when C would have been the last output
    assert redirected == (passes % 3 == 2)


def test_the_third_grid_is_used():
    ev, _ = simulate(6)
    assert [e[2] for e in ev if e[0] == "pass"] == [B, C, A, B, C, A]
    ev, final = simulate(5)
    assert [e[2] for e in ev if e[0] == "pass"] == [B, C, A, B, A] and final == A
