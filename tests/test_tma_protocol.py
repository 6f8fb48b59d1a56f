"""Discrete model of the hand-off protocol of the TMA kernel (k_fused_tma), run over random
interleavings of its roles on the CPU.

Roles: producer (TMA loads), storer (TMA stores), compute warps, halo warp.  Per stage s:
mbarrier full[s] (the TMA bytes landed); named barriers RING(s) (producer bar.arrive, compute and
halo bar.sync), OUT_FULL(s) (compute bar.arrive, storer bar.sync), EMPTY(s) (storer and producer
bar.sync); COMP (the compute warps' own reductions).  A use k of stage k % S carries plane p; the
collided plane p - 1 goes into the stage just pulled and leaves it by the storer's tensor store.
The model checks: every run ends (no deadlock), no named barrier gets more arrivals than its count
(no role laps another), no stage is refilled before all its reads and its output store are done, no
output is written into a stage before its reads are done, no store reads an incomplete output, and
no psi ring plane is read other than the one the reader expects.  Timeouts and a stalled first copy
exercise the abort path (waits skipped, barrier sequence kept).  Broken variants of the protocol
must be caught.
"""
import random

import pytest


class Deadlock(Exception):
    pass


def programs(items, S, R, C, stall, mutation=None):
    prog = {}
    P, k = [], 0
    for z0, z1 in items:
        for _ in range(z0 - 1, z1 + 1):
            s = k % S
            if k >= S:
                P.append(("sync" if mutation != "producer_arrives_empty" else "arrive", "E%d" % s))
            P.append(("issue", s, k, stall and k == 0))
            P.append(("arrive", "R%d" % s))
            k += 1
    for q in range(max(k - S, 0), k):
        P.append(("sync" if mutation != "producer_arrives_empty" else "arrive", "E%d" % (q % S)))
    for q in range(max(k - S, 0), k):
        P.append(("drainfull", q % S, q))
    prog["producer"] = P
    St, k = [], 0
    for z0, z1 in items:
        for p in range(z0 - 1, z1 + 1):
            s = k % S
            St.append(("sync", "OF%d" % s))
            if p > z0:
                St.append(("storeread", s, k))
            St.append(("sync", "E%d" % s))
            k += 1
    prog["storer"] = St
    for c in range(C):
        Cp, k = [], 0
        for z0, z1 in items:
            def pull(out_after_ring=True):
                nonlocal k
                s = k % S
                Cp.append(("waitfull", s, k))
                Cp.append(("read", s, k))
                Cp.append(("ring_write", k % R, k))
                Cp.append(("sync", "R%d" % s))
                k += 1
            pull()
            Cp.append(("arrive", "OF%d" % ((k - 1) % S)))
            pull()
            Cp.append(("arrive", "OF%d" % ((k - 1) % S)))
            for _ in range(z0, z1):
                if mutation == "out_before_ring":
                    s = k % S
                    Cp.append(("waitfull", s, k))
                    Cp.append(("read", s, k))
                    Cp.append(("ring_write", k % R, k))
                    Cp.append(("write_out", s, k))
                    Cp.append(("sync", "R%d" % s))
                    k += 1
                else:
                    pull()
                for d in (3, 2, 1):
                    Cp.append(("ring_read", (k - d) % R, k - d))
                so = (k - 1) % S
                if mutation != "out_before_ring":
                    Cp.append(("write_out", so, k - 1))
                Cp.append(("arrive", "OF%d" % so))
            Cp.append(("sync", "COMP"))
        Cp.append(("sync", "COMP"))
        prog["compute%d" % c] = Cp
    H, k = [], 0
    for z0, z1 in items:
        for _ in range(z0 - 1, z1 + 1):
            s = k % S
            H.append(("waitfull", s, k))
            H.append(("read", s, k))
            H.append(("ring_write", k % R, k))
            H.append(("sync" if mutation != "halo_arrives_ring" else "arrive", "R%d" % s))
            k += 1
    prog["halo"] = H
    return prog


def run(items, S, R, C, stall, timeout_prob, seed, mutation=None):
    rnd = random.Random(seed)
    prog = programs(items, S, R, C, stall, mutation)
    counts = {"COMP": C}
    for s in range(S):
        counts["E%d" % s] = 2
        counts["R%d" % s] = C + 2
        counts["OF%d" % s] = C + 1
    pc = {w: 0 for w in prog}
    blocked = {}
    arrived = {i: [0, []] for i in counts}
    full_phase = [0] * S
    inflight = []
    stage = [None] * S            # ("in", k) | ("out", k, writers) | None while loading
    readers = [set() for _ in range(S)]
    stored = [True] * S
    ring = [None] * R
    abort = False
    stall_pending = False
    nreaders = C + 1
    for _ in range(3_000_000):
        runnable = [w for w in prog if pc[w] < len(prog[w]) and w not in blocked]
        events = (["land"] if inflight else []) + (["stall_end"] if stall_pending else [])
        if not runnable and not events:
            if all(pc[w] >= len(prog[w]) for w in prog):
                return
            raise Deadlock({w: prog[w][pc[w]] for w in prog if pc[w] < len(prog[w])})
        if events and (not runnable or rnd.random() < 0.3):
            if rnd.choice(events) == "land":
                s, k = inflight.pop(rnd.randrange(len(inflight)))
                stage[s] = ("in", k)
                full_phase[s] += 1
            else:                       # the producer's bounded wait on the stalled copy ran out
                stall_pending = False
                abort = True
                stage[0] = ("in", 0)
                full_phase[0] += 1
            continue
        w = rnd.choice(runnable)
        op = prog[w][pc[w]]
        kind = op[0]
        if kind == "issue":
            _, s, k, st = op
            if not abort and k >= S:
                assert len(readers[s]) == nreaders, ("refill before all reads", s, k)
                assert stored[s], ("refill before the store read the output", s, k)
            readers[s] = set()
            stored[s] = True
            if st:
                stall_pending = True
            elif abort:
                stage[s] = ("in", k)
                full_phase[s] += 1
            else:
                stage[s] = None
                inflight.append((s, k))
        elif kind == "drainfull":
            _, s, q = op
            if full_phase[s] <= q // S and not abort:
                assert any(x[0] == s for x in inflight) or stall_pending, ("drain waits forever", s, q)
                continue
        elif kind == "waitfull":
            _, s, k = op
            if not abort and full_phase[s] <= k // S:
                if timeout_prob and rnd.random() < timeout_prob:
                    abort = True
                else:
                    continue
        elif kind == "read":
            _, s, k = op
            if not abort:
                assert stage[s] == ("in", k), ("stage race", w, op, stage[s])
                readers[s].add(w)
        elif kind == "ring_write":
            ring[op[1]] = op[2]
        elif kind == "ring_read":
            if not abort:
                assert ring[op[1]] == op[2], ("ring race", w, op, ring[op[1]])
        elif kind == "write_out":
            _, s, k = op
            if not abort:
                assert len(readers[s]) == nreaders, ("output written before all reads", w, op)
                if stage[s] == ("in", k):
                    stage[s] = ("out", k, set())
                assert stage[s][:2] == ("out", k), ("output race", w, op, stage[s])
                stage[s][2].add(w)
                stored[s] = False
        elif kind == "storeread":
            _, s, k = op
            if not abort:
                assert stage[s][:2] == ("out", k) and len(stage[s][2]) == C, ("store of an incomplete output", op)
                stored[s] = True
        elif kind in ("sync", "arrive"):
            b = op[1]
            arrived[b][0] += 1
            assert arrived[b][0] <= counts[b], ("barrier lapped", b, w)
            if kind == "sync":
                arrived[b][1].append(w)
                blocked[w] = b
            if arrived[b][0] == counts[b]:
                for x in arrived[b][1]:
                    blocked.pop(x, None)
                arrived[b] = [0, []]
        pc[w] += 1
    raise Deadlock("step limit")


def _random_case(seed):
    rnd = random.Random(1000 + seed)
    items = []
    for _ in range(rnd.choice([1, 1, 2, 3])):
        z0 = rnd.randrange(0, 20)
        items.append((z0, z0 + rnd.choice([1, 2, 3, 4, 7])))
    return dict(items=items, S=rnd.choice([3, 4]), R=4, C=rnd.choice([1, 2, 3]),
                stall=rnd.random() < 0.25, timeout_prob=rnd.choice([0, 0, 0.001, 0.01]))


def test_protocol_random_interleavings():
    for seed in range(1500):
        run(seed=seed, **_random_case(seed))


@pytest.mark.parametrize("mutation", ["halo_arrives_ring", "producer_arrives_empty", "out_before_ring"])
def test_broken_protocols_are_caught(mutation):
    caught = 0
    for seed in range(400):
        case = dict(_random_case(seed), stall=False, timeout_prob=0)
        try:
            run(seed=seed, mutation=mutation, **case)
        except (AssertionError, Deadlock):
            caught += 1
    assert caught > 0, mutation
