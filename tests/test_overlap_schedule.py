"""Model of the two-stream schedule of the checkpointed adjoint.

The checkpointed unsteady adjoint (`adjoint_impl` for one lattice, `enqueue_gradient`
for the batch) recomputes segment s - 1 on the handle's second stream while the
adjoint marches segment s on the caller's stream, with two segment stores used
alternately.  The host issues, in this order:

    record fork on main; aux waits fork
    recompute(last) on aux; record seg[last & 1] on aux
    for s = last .. 0:
        main waits seg[s & 1]
        if s > 0:
            if s < last: aux waits adj[(s + 1) & 1]
            recompute(s - 1) on aux; record seg[(s - 1) & 1] on aux
        march(s) on main; record adj[s & 1] on main
    record fork on aux; main waits fork          (the join, on every exit)
    flush of the sensitivity on main

A wait orders the waiting stream after the event's latest record at the time of
the call (CUDA's rule, the same under graph capture).  This test replays that
sequence for every segment count, builds the happens-before order, and checks
that each adjoint segment reads a store its own recompute has finished writing,
that no recompute overwrites a store an earlier-issued adjoint segment still
reads, and that the flush comes after everything on the second stream.
"""
import itertools

import pytest


def _replay(n_seg, aux_waits_adj=True):
    ops = []            # (stream, name); index = op id
    last_on = {}        # stream -> id of its last op
    edges = set()       # (a, b): a happens before b
    latest = {}         # event -> id of the op its latest record follows

    def op(stream, name):
        i = len(ops)
        ops.append((stream, name))
        if stream in last_on:
            edges.add((last_on[stream], i))
        last_on[stream] = i
        return i

    def record(ev, stream):
        latest[ev] = op(stream, f"record {ev}")

    def wait(stream, ev):
        i = op(stream, f"wait {ev}")
        if ev in latest:
            edges.add((latest[ev], i))

    last = n_seg - 1
    op("main", "forward")
    record("fork", "main")
    wait("aux", "fork")
    op("aux", f"recompute {last}")
    record(f"seg{last & 1}", "aux")
    for s in range(last, -1, -1):
        wait("main", f"seg{s & 1}")
        if s > 0:
            if s < last and aux_waits_adj:
                wait("aux", f"adj{(s + 1) & 1}")
            op("aux", f"recompute {s - 1}")
            record(f"seg{(s - 1) & 1}", "aux")
        op("main", f"march {s}")
        record(f"adj{s & 1}", "main")
    record("fork", "aux")
    wait("main", "fork")
    op("main", "flush")

    # transitive closure of the happens-before edges (the graphs are small)
    n = len(ops)
    succ = [set() for _ in range(n)]
    for a, b in edges:
        succ[a].add(b)
    reach = [None] * n
    for i in range(n - 1, -1, -1):
        r = set(succ[i])
        for j in succ[i]:
            r |= reach[j]
        reach[i] = r
    idx = {name: i for i, (_, name) in enumerate(ops)}
    return ops, idx, lambda a, b: b in reach[a]


@pytest.mark.parametrize("n_seg", [1, 2, 3, 4, 5, 8, 13])
def test_segment_stores_are_written_before_read_and_not_overwritten_while_read(n_seg):
    ops, idx, hb = _replay(n_seg)
    for s in range(n_seg):
        # the adjoint of segment s reads store s & 1 after its recompute wrote it
        assert hb(idx[f"recompute {s}"], idx[f"march {s}"]), s
        # the forward's snapshots exist before any recompute reads them
        assert hb(idx["forward"], idx[f"recompute {s}"]), s
    for s, t in itertools.product(range(n_seg), repeat=2):
        if s == t or (s & 1) != (t & 1):
            continue
        if t < s:
            # segment t is recomputed into the store that segment s's adjoint read:
            # that recompute must come after the adjoint is done with it
            assert hb(idx[f"march {s}"], idx[f"recompute {t}"]), (s, t)
    # the recomputes run in order on the second stream (they share the state
    # ping-pong), and the adjoint segments run in order on the caller's stream
    for s in range(n_seg - 1):
        assert hb(idx[f"recompute {s + 1}"], idx[f"recompute {s}"])
        assert hb(idx[f"march {s + 1}"], idx[f"march {s}"])
    # the join: the flush on the caller's stream follows all work on the second one
    for i, (stream, _) in enumerate(ops):
        if stream == "aux":
            assert hb(i, idx["flush"]), ops[i]


def test_recompute_overlaps_the_adjoint_of_the_next_segment():
    """The schedule leaves the recompute of segment s - 1 unordered with the adjoint of
    segment s: the two may run at the same time (that is the overlap)."""
    n_seg = 6
    ops, idx, hb = _replay(n_seg)
    for s in range(1, n_seg):
        a, b = idx[f"recompute {s - 1}"], idx[f"march {s}"]
        assert not hb(a, b) and not hb(b, a), s


def test_a_single_store_would_race():
    """Check the checker: with every segment in one store (seg[0] only), the recompute of
    segment s - 1 overwrites the store that segment s's adjoint is still reading."""
    n_seg = 4
    ops, idx, hb = _replay(n_seg)
    races = [s for s in range(1, n_seg) if not hb(idx[f"march {s}"], idx[f"recompute {s - 1}"])]
    assert races == list(range(1, n_seg))


def test_without_the_second_streams_wait_a_recompute_overwrites_a_store_in_use():
    """Check the checker: dropping the second stream's wait for the adjoint that last
    read a store lets the recompute of segment s - 1 overwrite segment s + 1's store
    while that adjoint may still read it."""
    n_seg = 5
    ops, idx, hb = _replay(n_seg, aux_waits_adj=False)
    unordered = [s for s in range(1, n_seg - 1) if not hb(idx[f"march {s + 1}"], idx[f"recompute {s - 1}"])]
    assert unordered == list(range(1, n_seg - 1))
