"""Host-side check of the work-item schedule of the halo-exchange FP32 kernel
(csrc/emd_halo.cu): the claim sequence, the ring of w tile slots and the
waits, restated here and run as a discrete-event simulation.

Each simulated CTA claims the next item of the sequence, waits until the
item's dependencies are met, runs for a random time and publishes. The test
asserts that every dependency of an item comes earlier in the claim sequence
(so no wait can deadlock with any number of CTAs), that the simulation never
stalls, that every adjoint item reads the w tiles of its own exposure and
neighbours, that no forward item overwrites a slot while a reader still
needs it, and that adjoint items of one tile run in exposure order. The
batch kernel's work list (several jobs' sequences merged round-robin or job
after job) is checked the same way."""
import random

import pytest


def plan(gx, gy, ne, cap):
    T = gx * gy
    dmax = (gx if gy > 1 else 0) + (1 if gx > 1 else 0)
    NT = ne * T
    L = min(NT, dmax + 2 * cap)
    R = min(NT, L + dmax + 1 + cap)
    return T, dmax, NT, L, R


def decode(sq, NT, L):
    if sq < L:
        return True, sq
    if sq < 2 * NT - L:
        j = sq - L
        return (True, L + j // 2) if j & 1 else (False, j // 2)
    return False, sq - NT


def neighbours(k, gx, gy):
    ti, tj = divmod(k, gx)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            a, b = ti + dy, tj + dx
            if 0 <= a < gy and 0 <= b < gx:
                yield a * gx + b


def deps(fwd, i, gx, gy, T, R):
    """(kind, id) items that must be finished before item (fwd, i) proceeds."""
    out = []
    if fwd:
        if i >= R:
            pe, pk = divmod(i - R, T)
            out += [("A", pe * T + k) for k in neighbours(pk, gx, gy)]
    else:
        e, k = divmod(i, T)
        out += [("F", e * T + k2) for k2 in neighbours(k, gx, gy)]
        if e > 0:
            out.append(("A", (e - 1) * T + k))
    return out


SHAPES = [(1, 1), (1, 3), (3, 1), (2, 2), (5, 4), (8, 8), (4, 9)]


@pytest.mark.parametrize("gx,gy", SHAPES)
@pytest.mark.parametrize("ne", [1, 2, 5])
@pytest.mark.parametrize("cap", [1, 3, 160, 320, 480, 640])
def test_dependencies_are_claimed_earlier(gx, gy, ne, cap):
    T, dmax, NT, L, R = plan(gx, gy, ne, cap)
    pos = {}
    for sq in range(2 * NT):
        fwd, i = decode(sq, NT, L)
        key = ("F" if fwd else "A", i)
        assert key not in pos
        pos[key] = sq
    assert len(pos) == 2 * NT  # every item exactly once
    for (kind, i), sq in pos.items():
        for d in deps(kind == "F", i, gx, gy, T, R):
            assert pos[d] < sq, ((kind, i), d)


def simulate(gx, gy, ne, cap, ctas, seed, ahead=True):
    """ahead: each CTA claims its next position when it starts an item (the
    kernel's claim-ahead, which prefetches that item's data meanwhile)."""
    T, dmax, NT, L, R = plan(gx, gy, ne, cap)
    rng = random.Random(seed)
    pending = [None] * ctas   # the claim taken ahead, not started yet
    done = set()
    ring = [None] * R         # F id whose w the slot holds
    readers = {}              # A id -> list of (slot, expected F id)
    next_sq = 0
    workers = [None] * ctas   # (kind, id, state, remaining time)
    adone_order = {}
    time = 0
    while len(done) < 2 * NT:
        progressed = False
        for wi in range(ctas):
            w = workers[wi]
            if w is None:
                sq = pending[wi]
                if sq is None:
                    sq, next_sq = next_sq, next_sq + 1
                pending[wi] = None
                if sq < 2 * NT:
                    fwd, i = decode(sq, NT, L)
                    workers[wi] = ["F" if fwd else "A", i, "wait", rng.randint(1, 5)]
                    if ahead:
                        pending[wi], next_sq = next_sq, next_sq + 1
                    progressed = True
                continue
            kind, i, state, rem = w
            if state == "wait":
                if all(d in done for d in deps(kind == "F", i, gx, gy, T, R)):
                    w[2] = "run"
                    progressed = True
                    if kind == "F":
                        slot = i % R
                        # nobody still needs the slot's previous tile
                        for a, lst in readers.items():
                            if ("A", a) not in done:
                                assert (slot, ring[slot]) not in lst or ring[slot] is None
                        ring[slot] = ("pending", i)
                    else:
                        e, k = divmod(i, T)
                        need = [((e * T + k2) % R, e * T + k2) for k2 in neighbours(k, gx, gy)]
                        for slot, fid in need:
                            assert ring[slot] == fid, (i, slot, ring[slot], fid)
                        readers[i] = need
                continue
            w[3] -= 1
            progressed = True
            if w[3] == 0:
                if kind == "F":
                    ring[i % R] = i
                else:
                    for slot, fid in readers[i]:
                        assert ring[slot] == fid  # not overwritten while being read
                    e, k = divmod(i, T)
                    assert adone_order.get(k, -1) == e - 1
                    adone_order[k] = e
                done.add((kind, i))
                workers[wi] = None
        time += 1
        assert progressed, "schedule stalled"
    return time


@pytest.mark.parametrize("gx,gy", SHAPES)
@pytest.mark.parametrize("ne", [1, 3])
@pytest.mark.parametrize("cap,ctas", [(1, 1), (1, 2), (2, 5), (3, 40)])
@pytest.mark.parametrize("ahead", [False, True])
def test_simulated_execution(gx, gy, ne, cap, ctas, ahead):
    for seed in range(3):
        simulate(gx, gy, ne, cap, ctas, seed, ahead)


def merged(jobs, order):
    """The batch step's work list: each job's claim positions in its own
    order, merged round-robin (order 0) or job after job (order 1)."""
    seqs = [[(j, sq) for sq in range(2 * plan(*jb)[2])] for j, jb in enumerate(jobs)]
    if order == 1:
        return [e for s in seqs for e in s]
    out, q = [], 0
    while len(out) < sum(len(s) for s in seqs):
        out += [s[q] for s in seqs if q < len(s)]
        q += 1
    return out


JOB_MIXES = [[(2, 2, 3, 2), (1, 1, 4, 2), (5, 3, 2, 1)],
             [(8, 8, 2, 3), (3, 1, 5, 2)],
             [(1, 3, 1, 1), (4, 4, 3, 2), (2, 1, 6, 1), (3, 3, 2, 3)]]


@pytest.mark.parametrize("jobs", JOB_MIXES)
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("ctas", [1, 3, 17])
def test_merged_batch_work_list(jobs, order, ctas):
    """Every dependency of an entry (same job) comes earlier in the merged
    list, and a simulated run with claim-ahead finishes, each adjoint item
    reading the ring slots its job's forward items filled."""
    lst = merged(jobs, order)
    pos = {}
    for p_, (j, sq) in enumerate(lst):
        NT, L = plan(*jobs[j])[2], plan(*jobs[j])[3]
        fwd, i = decode(sq, NT, L)
        pos[(j, "F" if fwd else "A", i)] = p_
    for (j, kind, i), p_ in pos.items():
        gx, gy = jobs[j][0], jobs[j][1]
        T, _, _, _, R = plan(*jobs[j])
        for d in deps(kind == "F", i, gx, gy, T, R):
            assert pos[(j,) + d] < p_
    rng = random.Random(len(lst) + ctas)
    done, ring = set(), {}
    workers, pending, nxt = [None] * ctas, [None] * ctas, 0
    steps = 0
    while len(done) < len(lst):
        progressed = False
        for w in range(ctas):
            if workers[w] is None:
                p_ = pending[w]
                if p_ is None:
                    p_, nxt = nxt, nxt + 1
                pending[w] = None
                if p_ < len(lst):
                    j, sq = lst[p_]
                    NT, L = plan(*jobs[j])[2], plan(*jobs[j])[3]
                    fwd, i = decode(sq, NT, L)
                    workers[w] = [j, "F" if fwd else "A", i, "wait", rng.randint(1, 4)]
                    pending[w], nxt = nxt, nxt + 1
                    progressed = True
                continue
            j, kind, i, state, rem = workers[w]
            gx, gy = jobs[j][0], jobs[j][1]
            T, _, _, _, R = plan(*jobs[j])
            if state == "wait":
                if all((j,) + d in done for d in deps(kind == "F", i, gx, gy, T, R)):
                    workers[w][3] = "run"
                    progressed = True
                    if kind == "A":
                        e, k = divmod(i, T)
                        for k2 in neighbours(k, gx, gy):
                            assert ring[(j, (e * T + k2) % R)] == e * T + k2
                continue
            workers[w][4] -= 1
            progressed = True
            if workers[w][4] == 0:
                if kind == "F":
                    ring[(j, i % R)] = i
                done.add((j, kind, i))
                workers[w] = None
        steps += 1
        assert progressed, "merged schedule stalled"
