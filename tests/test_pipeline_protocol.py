"""The dedispersion kernel's staging protocol (A5, Sec. 2.2.2), model-checked
on the CPU: consumer warps wait on a stage's "full" barrier, consume it and
arrive on its "empty" barrier; the stage's copies are issued either by a
producer warp running up to STAGES stages ahead, or (ALGO 6 and 7) by the
consumer warps in rotation, warp w issuing stages w, w + NCONS, ... LOOK
stages ahead of their use after waiting for the buffer's previous release.

Random schedules of the warps' steps are explored; every run must end with
every stage consumed by every warp (no deadlock), and no buffer may be
refilled before all warps released its previous stage nor consumed before it
was filled -- the properties the barriers' phases encode."""
import random

import pytest


def _run(nstage, nw, stages, look, rot, rng):
    """One random interleaving; returns the number of steps taken."""
    released = [[False] * nw for _ in range(nstage)]  # released[stage][warp]
    issued = [False] * nstage
    # buffer b holds stage owner[b] (the last one issued into it)
    owner = [None] * stages

    def free_for(j):
        # the buffer of stage j may be refilled once every warp released
        # stage j - stages (the barrier phase the issuing warp waits on)
        return j < stages or all(released[j - stages])

    def issue(j):
        b = j % stages
        prev = owner[b]
        assert prev is None or all(released[prev]), "buffer refilled before its release"
        assert not issued[j]
        owner[b] = j
        issued[j] = True

    # per-warp program counters
    if rot:
        pc = [dict(i=0, pro=0, phase="pro") for _ in range(nw)]
    else:
        pc = [dict(i=0, phase="wait") for _ in range(nw)]
        producer = dict(j=0)
    steps = 0
    while True:
        runnable = []
        for w in range(nw):
            p = pc[w]
            if p["phase"] == "done":
                continue
            if p["phase"] == "pro":
                # the prologue: stages w, w + nw, ... below look
                j = w + p["pro"] * nw
                if j >= min(look, nstage):
                    runnable.append((w, "enter"))
                else:
                    runnable.append((w, "pro"))  # j < look <= stages: no wait
            elif p["phase"] == "prod":
                j = p["i"] + look
                if free_for(j):
                    runnable.append((w, "prod"))
            elif p["phase"] == "wait":
                if issued[p["i"]]:
                    runnable.append((w, "consume"))
        if not rot and producer["j"] < nstage and free_for(producer["j"]):
            runnable.append((-1, "produce"))
        if not runnable:
            break
        w, act = rng.choice(runnable)
        steps += 1
        if act == "produce":
            issue(producer["j"])
            producer["j"] += 1
            continue
        p = pc[w]
        if act == "pro":
            issue(w + p["pro"] * nw)
            p["pro"] += 1
        elif act == "enter":
            p["phase"] = "start"
        elif act == "prod":
            issue(p["i"] + look)
            p["phase"] = "wait"
        elif act == "consume":
            i = p["i"]
            assert issued[i] and owner[i % stages] == i, "stage consumed before it was filled"
            released[i][w] = True
            p["i"] += 1
            p["phase"] = "start"
        if p["phase"] == "start":
            i = p["i"]
            if i >= nstage:
                p["phase"] = "done"
            elif rot and i + look < nstage and (i + look) % nw == w:
                p["phase"] = "prod"
            else:
                p["phase"] = "wait"
    assert all(p["phase"] == "done" for p in pc), "deadlock"
    assert all(all(r) for r in released)
    return steps


@pytest.mark.parametrize("nw,stages,look,rot", [
    (8, 6, 2, True),    # ALGO 6, 7 as built (8 consumer warps)
    (8, 8, 4, True),    # ALGO 12: four stages ahead over eight buffers
    (8, 5, 2, True),    # two CTAs per SM: one buffer fewer
    (12, 6, 2, True),   # 12 consumer warps
    (8, 6, 3, True),
    (8, 4, 3, True),    # one stage of slack: correct, only slower
    (2, 6, 2, True),    # fewer warps than stages issued ahead
    (1, 6, 2, True),
    (7, 4, 3, False),   # a producer warp, up to STAGES stages ahead
    (11, 4, 3, False),
])
def test_protocol_never_deadlocks_nor_overwrites(nw, stages, look, rot):
    rng = random.Random(nw * 100 + stages * 10 + look)
    for nstage in (1, 2, 3, 5, 9, 40):
        for _ in range(60):
            _run(nstage, nw, stages, look, rot, rng)
