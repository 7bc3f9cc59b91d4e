"""The exchange protocol of the tensor-memory kernel over a pair of SMs (m = 17), model-checked
on the CPU.

Label bit 16 pairs values held by the two CTAs of a cluster.  For every output chunk n
(counted over the CTA's signals; both CTAs walk the same chunks) each CTA, in program order:

  S(n)  bulk-stores the half it gives away into its scratch slot (rank, n mod 2);
  A(n)  waits for that store to complete and arrives on the peer's barrier ready[n mod 2];
  W(n)  waits on its own ready[n mod 2] for phase parity (n >> 1) & 1;
  L(n)  issues the bulk load of the peer's slot (peer, n mod 2) into its exchange buffer,
        completing on its barrier load (one load per chunk);
  F(n)  waits on load for phase parity n & 1, then reads the buffer and finishes the chunk.

The store is in flight between S and A, the load between L and F.  This test explores every
interleaving of the two CTAs (the state is the pair of program positions; the barriers'
phase counts follow from it) with the hardware's parity rule for a wait: it returns once
the phase whose parity it names has completed, i.e. while the completed-phase count has
the other parity.  It checks that

  * no state is stuck before both CTAs finish (every wait ends);
  * a wait never returns early or late: when W(n) / F(n) passes, exactly (n >> 1) + 1 /
    n + 1 phases have completed (the parity is never ambiguous);
  * a load reads the peer's values of its own chunk (the slot's last completed store is
    chunk n, and no store to that slot is in flight while the load is);

and that the checks have teeth: a single scratch slot, or a store issued before the
previous chunk's finish, or waiting on parity n & 1 instead, each fails one of them.
"""

import itertools

import pytest

ACTIONS = ("S", "A", "W", "L", "F")


def program(chunks, variant):
    """One CTA's actions in program order: (kind, chunk)."""
    if variant == "store_before_finish":
        # S(n+1) hoisted above F(n): the buffer and the slot would be reused too early
        prog = []
        for n in range(chunks):
            prog += [("S", n), ("A", n), ("W", n), ("L", n)]
            if n > 0:
                prog.append(("F", n - 1))
        prog.append(("F", chunks - 1))
        return prog
    return [(a, n) for n in range(chunks) for a in ACTIONS]


def explore(chunks, variant="kernel"):
    slots = 1 if variant == "one_slot" else 2
    ready_parity = (lambda n: n & 1) if variant == "ready_parity_n" else (lambda n: (n >> 1) & 1)
    progs = [program(chunks, variant), program(chunks, variant)]
    end = len(progs[0])
    problems = set()

    def done(r, pos, kind, n):
        # whether CTA r has executed (kind, n) at program position pos
        return progs[r].index((kind, n)) < pos

    def count(r, pos, kind, cond=lambda n: True):
        return sum(1 for k, n in progs[r][:pos] if k == kind and cond(n))

    seen = set()
    stack = [(0, 0)]
    while stack:
        st = stack.pop()
        if st in seen:
            continue
        seen.add(st)
        moved = False
        for r in (0, 1):
            p = 1 - r
            pos, ppos = st[r], st[p]
            if pos == end:
                continue
            kind, n = progs[r][pos]
            if kind == "W":
                # arrivals on this CTA's ready[n mod 2] come from the peer's A(m), m = n mod 2
                c = count(p, ppos, "A", lambda m: m % slots == n % slots)
                if c % 2 == ready_parity(n):
                    continue  # the phase of that parity has not completed: blocked
                if c != (n >> 1) + 1 and slots == 2:
                    problems.add(f"ready wait of chunk {n} passed after {c} phases")
                if slots == 1 and c != n + 1:
                    problems.add(f"ready wait of chunk {n} passed after {c} phases")
            elif kind == "F":
                c = count(r, pos, "L")  # loads issued = loads completed by the time F may pass
                if c % 2 == (n & 1):
                    continue
                if c != n + 1:
                    problems.add(f"load wait of chunk {n} passed after {c} phases")
            elif kind == "L":
                # the peer's slot must hold chunk n: its last completed store to the slot is n
                last = [m for m in range(chunks) if m % slots == n % slots and done(p, ppos, "A", m)]
                if not last or max(last) != n:
                    problems.add(f"load of chunk {n} reads slot contents of chunk {max(last) if last else None}")
            nxt = list(st)
            nxt[r] += 1
            nxt = tuple(nxt)
            # in flight after the move: a peer store and a load on the same slot must not overlap
            for a, b in ((r, p), (p, r)):
                for m in range(chunks):
                    storing = done(a, nxt[a], "S", m) and not done(a, nxt[a], "A", m)
                    if not storing:
                        continue
                    for k in range(chunks):
                        loading = done(b, nxt[b], "L", k) and not done(b, nxt[b], "F", k)
                        if loading and k % slots == m % slots:
                            problems.add(f"store of chunk {m} overlaps the peer's load of chunk {k}")
            stack.append(nxt)
            moved = True
        if not moved and st != (end, end):
            problems.add(f"stuck at positions {st}")
    return problems, len(seen)


@pytest.mark.parametrize("chunks", [1, 2, 3, 4, 5, 8])
def test_exchange_protocol_as_built_is_safe_and_live(chunks):
    problems, states = explore(chunks)
    assert not problems, sorted(problems)
    assert states > 5 * chunks  # the two CTAs really interleave


@pytest.mark.parametrize("variant", ["one_slot", "store_before_finish", "ready_parity_n"])
def test_planted_protocol_mistakes_are_caught(variant):
    problems, _ = explore(5, variant)
    assert problems, f"the model did not catch the {variant} mistake"


def test_action_order_covers_every_step():
    prog = program(3, "kernel")
    assert [a for a, _ in prog[:5]] == list(ACTIONS)
    assert sorted(itertools.chain(prog)) == sorted((a, n) for a in ACTIONS for n in range(3))
