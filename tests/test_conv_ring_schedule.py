"""Schedule model of the tcgen05 convolution ring (host logic, no GPU).

conv_ring_kernel (csrc/evx_nn_tc.cu) walks work units of L output rows. Input
row i = 0 .. L+1 of a unit with first virtual row V is one MMA item k: it
accumulates into virtual rows V+i, V+i+1, V+i+2 and then commits row V+i (the
last item also commits rows V+L+2 and V+L+3). Each virtual row owns the
accumulator block blk(v) = (16 - v mod 16) mod 16 of a 16-block ring.

The synchronisation rests on ordering arguments, checked here over many unit
sequences:
  - claims: when row V+i+2 is not yet claimed, the MMA warp probes only the block
    of row V+i+9 for the phase in which row V+i-7 was freed. Every epilogue warp
    frees rows in order, so that phase implies all earlier rows are free. Rows up
    to V+i+9 then count as claimed;
  - slots: input slot k mod 5 is refilled once row V+i of item k-5 has been
    committed; the producer waits on that row's block barrier;
  - the epilogue waits on each row's block barrier in row order.
Each barrier wait names a parity. The model checks that the awaited phase is
the only one that can complete while the waiter is blocked, i.e. no wait could
pass on a later phase.
"""
import random

import pytest

NBLK, NS = 16, 5


def blk(v):
    return (NBLK - v % NBLK) % NBLK


def items_of(lengths):
    out, V, k = [], 0, 0
    for L in lengths:
        for i in range(L + 2):
            out.append((k, V, i, L))
            k += 1
        V += L + 4
    return out, V


def commits_of(item):
    k, V, i, L = item
    rows = [V + i]
    if i == L + 1:
        rows += [V + L + 2, V + L + 3]
    return rows


def check(lengths):
    items, nrows = items_of(lengths)
    committed = set()
    committed_upto = []  # committed_upto[k]: rows committed before item k starts
    vready = NBLK - 1
    freed_required = -1  # the epilogue has freed every row <= this at the latest claim
    for item in items:
        k, V, i, L = item
        committed_upto.append(set(committed))
        # the three target rows sit in adjacent blocks b0, b0+1, b0+2 (mod 16); a wrap splits
        # each MMA into N = 64 + 32 (b0 = 14) or 32 + 64 (b0 = 15)
        b0 = blk(V + i + 2)
        assert blk(V + i + 1) == (b0 + 1) % NBLK and blk(V + i) == (b0 + 2) % NBLK
        if V + i + 2 > vready:
            vc = V + i + 9
            need = vc - NBLK  # freed-row phase the single probe waits for
            assert need >= 0 and blk(vc) == blk(need)
            # the epilogue can free it: every row <= need was committed by an earlier item
            assert all(r in committed for r in range(need + 1)), (lengths, k)
            freed_required = max(freed_required, need)
            vready = vc
        for w in (V + i, V + i + 1, V + i + 2):
            assert w <= vready  # claimed
            assert w - NBLK <= freed_required  # its block's previous row has been freed
        # a later phase of a claimed block (row w + 16) cannot be written before row w is freed
        committed.update(commits_of(item))
    assert committed == set(range(nrows))  # every virtual row is committed once (and freed by the epilogue)
    # slots: item k refills slot k % NS after the commit of item k - NS's row; while the producer
    # waits, at most items < k have run, whose commits stay below that row + 16 (same parity
    # cannot recur), and the awaited commit is among them only once item k - NS has run
    for k in range(NS, len(items)):
        v_slot = items[k - NS][1] + items[k - NS][2]
        before = committed_upto[k]  # commits issued before item k starts
        assert max(before) < v_slot + NBLK, (lengths, k)  # the wait on parity (v_slot / 16) & 1 is unambiguous
    # epilogue: row v's wait on blk(v) parity (v / 16) & 1; row v + 16 is written only after the claim
    # that needs row v freed, so the barrier is at most one phase ahead of the waiter
    return nrows


@pytest.mark.parametrize("lengths", [
    [64] * 6,
    [128, 128, 128],
    [8, 8, 8, 8, 8, 8, 8, 8, 8, 8],
    [1] * 40,
    [2, 1, 3, 1, 2, 9, 1, 1, 30],
    [7, 3, 64, 2, 5, 100, 16, 15, 17],
])
def test_ring_schedule(lengths):
    assert check(lengths) == sum(L + 4 for L in lengths)


def test_ring_schedule_random_units():
    rnd = random.Random(7)
    for _ in range(200):
        lengths = [rnd.randint(1, 70) for _ in range(rnd.randint(1, 12))]
        check(lengths)


def test_claim_window_bound():
    """Before item k starts, rows up to V+i-1 are committed. So a claim reaching w rows
    ahead (up to V+i+w, needing row V+i+w-16 freed) cannot wait on itself for w <= 15.
    With w = 16 it would need row V+i, which only this item commits. The kernel uses
    w = 9, which leaves the epilogue 6 committed rows of slack at each claim."""
    for w, feasible in ((9, True), (15, True), (16, False)):
        items, _ = items_of([64, 64])
        committed, ok = set(), True
        for item in items:
            k, V, i, L = item
            need = V + i + w - NBLK
            if need >= 0 and need not in committed:
                ok = False
                break
            committed.update(commits_of(item))
        assert ok == feasible, w
