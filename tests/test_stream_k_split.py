"""Host restatement of the tensor-core TTM's stream-K work split (csrc/ttm_tc.cu).

The T x nkb (tile, 64-deep K block) iterations are cut into G contiguous ranges
[start(b), start(b+1)), start(b) = floor(b W / G), W = T nkb.  A CTA's range is a chain of
segments (consecutive K blocks of one tile).  A segment that is a whole tile is written
directly; otherwise it goes to the CTA's partial slot (2b for the CTA's first segment, 2b + 1
for a later one), the CTA bumps the arrival counter of the tile's first CTA b0, and the CTA
that arrives last (count b1 - b0) adds the slots of CTAs b0..b1 in K order.  These tests
restate that integer logic and check it over many shapes: every iteration is done exactly
once, no slot is written twice in one launch, the reader finds each part where its writer put
it, counters belong to one tile each, and no CTA ever waits for another."""
import itertools

import pytest


def start(b, W, G):
    return b * W // G


def cta_of(w, W, G):
    b = w * G // W
    while b + 1 < G and start(b + 1, W, G) <= w:
        b += 1
    while b > 0 and start(b, W, G) > w:
        b -= 1
    return b


def segments(b, W, G, nkb):
    """(tile, first K block, end K block, slot or None) of CTA b, in order."""
    w0, w1 = start(b, W, G), start(b + 1, W, G)
    out = []
    w = w0
    while w < w1:
        tile, a = divmod(w, nkb)
        e = min(nkb, a + (w1 - w))
        full = a == 0 and e == nkb
        out.append((tile, a, e, None if full else 2 * b + (0 if w == w0 else 1)))
        w += e - a
    return out


@pytest.mark.parametrize("T,nkb,G", list(itertools.product([1, 2, 7, 100, 1250, 2501], [1, 2, 7, 8], [1, 3, 96, 152])))
def test_stream_k_split_covers_each_iteration_once_and_matches_slots(T, nkb, G):
    W = T * nkb
    G = min(G, W)  # the launcher never starts more CTAs than iterations
    covered = [0] * W
    writers = {}  # tile -> {cta: slot}
    slots_used = set()
    for b in range(G):
        segs = segments(b, W, G, nkb)
        assert sum(1 for s in segs if s[3] is not None) <= 2
        for tile, a, e, slot in segs:
            for kb in range(a, e):
                covered[tile * nkb + kb] += 1
            if slot is not None:
                assert slot not in slots_used
                slots_used.add(slot)
                assert slot // 2 == b
                writers.setdefault(tile, {})[b] = slot
    assert covered == [1] * W
    counters = set()
    for tile, ws in writers.items():
        b0, b1 = cta_of(tile * nkb, W, G), cta_of(tile * nkb + nkb - 1, W, G)
        # the arrival count the last CTA sees is b1 - b0: every CTA of the tile writes one part
        assert sorted(ws) == list(range(b0, b1 + 1))
        for bb in range(b0, b1 + 1):
            reader_slot = 2 * bb + (1 if start(bb, W, G) < tile * nkb else 0)
            assert reader_slot == ws[bb]
        assert b0 not in counters
        counters.add(b0)
        # parts in K order
        kfirst = [max(start(bb, W, G), tile * nkb) for bb in range(b0, b1 + 1)]
        assert kfirst == sorted(kfirst)
    # the partial slots fit the workspace of 2 per CTA
    assert all(s < 2 * G for s in slots_used)


def test_cta_of_inverts_start():
    for W, G in [(7, 3), (700, 152), (8750, 152), (5, 5), (1, 1), (10 ** 9 + 7, 152)]:
        for b in range(G):
            s, e = start(b, W, G), start(b + 1, W, G)
            for w in {s, e - 1}:
                if s <= w < e:
                    assert cta_of(w, W, G) == b
