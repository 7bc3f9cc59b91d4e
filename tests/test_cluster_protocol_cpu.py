"""The buffer-rotation protocol of the thread-block-cluster kernel, model-checked on the CPU.

A cluster of NR CTAs owns one unit u (a tile of NR x 2^TB words) at a time, with three
shared buffers per CTA.  Unit u's input S_u is loaded by TMA into buffer u mod 3; after
phases 1-2 have read it, the same buffer receives the pushes R_{u+1} of unit u+1 from every
CTA, which phase 3 of unit u+1 reads; then the load of S_{u+3} refills it.  Barriers per CTA
(three each, index = unit mod 3, phase parity (u / 3) & 1): tma (the CTA's own load, one
arrival), free (NR arrivals: every CTA's buffer for R_u may be written) and full (NR
arrivals: every CTA has pushed R_u).  Each CTA runs, in program order,

  LD(0) LD(1) AF(0)
  for k = 0..K:  [k >= 1]  WF(k-1) P3(k-1) [k+1 < K] LD(k+1)
                 [k <  K]  WT(k) P12(k) AF(k+1) WFr(k) PUSH(k) AFull(k)

where AF / AFull arrive on every CTA's free / full barrier, WF / WFr / WT wait on the CTA's
own full / free / tma barrier, P12 reads S_k, PUSH writes R_k into every CTA's buffer
(k + 2) mod 3 and P3 reads R_k from its own.  The test explores every interleaving of the
CTAs (atomic actions; a TMA load is in flight from LD to WT) and checks that

  * no state is stuck before every CTA finishes (every wait ends);
  * every barrier phase is made of arrivals for one unit only, and a wait passes exactly
    when the phase of its unit has completed (never one early, never one late);
  * each buffer holds one live item at a time (an input being loaded or not yet read, or
    a set of pushes not yet read), and phase 3 of unit k reads all NR pushes of R_k;

and that planted mistakes (two buffers, phase 3 without the full wait, the next load
issued before phase 3 has read the buffer) each fail a check.  It also shows that the free
handshake is implied by the full wait of the previous unit in this order.
"""

import pytest


def program(nr, units, variant):
    prog = [("LD", 0)] if units > 0 else []
    if units > 1:
        prog.append(("LD", 1))
    if units > 0:
        prog.append(("AF", 0))
    for k in range(units + 1):
        if k >= 1:
            finish = [("WF", k - 1), ("P3", k - 1)]
            if variant == "no_full_wait":
                finish = [("P3", k - 1)]
            if k + 1 < units:
                if variant == "load_before_phase3":
                    finish.insert(0, ("LD", k + 1))
                else:
                    finish.append(("LD", k + 1))
            prog += finish
        if k < units:
            body = [("WT", k), ("P12", k), ("AF", k + 1), ("WFr", k), ("PUSH", k), ("AFull", k)]
            if variant == "no_free_wait":
                body = [b for b in body if b[0] != "WFr"]
            prog += body
    return prog


def explore(nr, units, variant="kernel"):
    nbuf = 2 if variant == "two_buffers" else 3
    progs = [program(nr, units, variant) for _ in range(nr)]
    end = len(progs[0])
    index = [{a: i for i, a in enumerate(p)} for p in progs]
    problems = set()

    def did(c, pos, kind, n):
        i = index[c].get((kind, n))
        return i is not None and i < pos

    def completed(st, kind, idx):
        # phases completed on barrier `kind` index idx (arrivals go to every CTA alike)
        return sum(1 for u in range(units + 1) if u % nbuf == idx and all(did(c, st[c], kind, u) for c in range(nr)))

    def check_state(st):
        for kind in ("AF", "AFull"):  # a phase holds arrivals of one unit only
            for c in range(nr):
                for u in range(units + 1):
                    if did(c, st[c], kind, u) and u >= nbuf:
                        if not all(did(o, st[o], kind, u - nbuf) for o in range(nr)):
                            problems.add(f"{kind} of unit {u} arrives while unit {u - nbuf}'s phase is open")
        for j in range(nr):
            for b in range(nbuf):
                live = []
                for u in range(units):
                    if u % nbuf == b and did(j, st[j], "LD", u) and not did(j, st[j], "P12", u):
                        live.append(f"S{u}")
                    if (u + 2) % nbuf == b and any(did(i, st[i], "PUSH", u) for i in range(nr)) \
                            and not did(j, st[j], "P3", u):
                        live.append(f"R{u}")
                if len(live) > 1:
                    problems.add(f"CTA {j} buffer {b} holds {live} at once")

    seen = set()
    stack = [tuple([0] * nr)]
    while stack:
        st = stack.pop()
        if st in seen:
            continue
        seen.add(st)
        check_state(st)
        moved = False
        for c in range(nr):
            if st[c] == end:
                continue
            kind, n = progs[c][st[c]]
            if kind in ("WF", "WFr", "WT"):
                idx = n % nbuf
                if kind == "WT":
                    done = sum(1 for u in range(units) if u % nbuf == idx and did(c, st[c], "LD", u))
                else:
                    done = completed(st, "AFull" if kind == "WF" else "AF", idx)
                if done % 2 == (n // nbuf) & 1:
                    continue  # the phase of that parity has not completed
                if done != n // nbuf + 1:
                    problems.add(f"{kind} of unit {n} passed after {done} phases")
            if kind == "P3" and not all(did(i, st[i], "PUSH", n) for i in range(nr)):
                problems.add(f"phase 3 of unit {n} reads before every push landed")
            nxt = list(st)
            nxt[c] += 1
            stack.append(tuple(nxt))
            moved = True
        if not moved and st != tuple([end] * nr):
            problems.add(f"stuck at {st}")
    return problems, len(seen)


@pytest.mark.parametrize("nr,units", [(2, 1), (2, 2), (2, 4), (2, 7), (4, 3), (4, 4)])
def test_cluster_protocol_as_built_is_safe_and_live(nr, units):
    problems, states = explore(nr, units)
    assert not problems, sorted(problems)[:10]
    assert states > len(program(nr, units, "kernel"))


@pytest.mark.parametrize("variant", ["two_buffers", "no_full_wait", "load_before_phase3"])
def test_planted_protocol_mistakes_are_caught(variant):
    problems, _ = explore(2, 5, variant)
    assert problems, f"the model did not catch the {variant} mistake"


@pytest.mark.parametrize("nr,units", [(2, 5), (4, 3)])
def test_free_handshake_is_implied_by_the_previous_full_wait(nr, units):
    # In this order a CTA pushes R_k only after its wait on full for unit k-1, i.e. after
    # every CTA's AFull(k-1), which each CTA gives after its phases 1-2 of unit k-1 have
    # read the buffer R_k goes to.  So the free barrier adds a margin, not a requirement:
    # the protocol without its wait passes every check as well.
    problems, _ = explore(nr, units, "no_free_wait")
    assert not problems, sorted(problems)[:10]
