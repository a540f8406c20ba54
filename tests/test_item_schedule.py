"""The work-item schedule of the tensor-core item-index kernel, checked on
the CPU against its buffers.

The schedule is built on the device by two kernels (subset_tc.cu): a
one-block plan (items per (class, item group), the cost classes' sizes in
closed form, the CTA lists' offsets) and a one-thread-per-item placement
(each item's cost class, its sorted position, its slot in a CTA list dealt in
snake order).  This test restates that arithmetic in Python and checks, over
random and extreme group sizes, what the kernels rely on without checking:

* the item count never exceeds the host's bound on the items buffer;
* the plan's closed-form cost-class sizes equal the classes of the items the
  placement computes one by one, so sorted positions are a permutation;
* every item lands inside its CTA's list and every list slot is filled once;
* the items cover every (pattern, record) pair of every group exactly once,
  so the executed test count the plan reports is the index's.
"""
import numpy as np
import pytest

OWN_TILE = 128          # resident rows per half
STREAM_TILE = 128       # streamed rows per tile
BUCKETS = 64


def div_up(a, b):
    return -(-a // b)


def cost_bucket(b_tiles, own_count, per):
    cmax = 2 * per + 2
    cost = b_tiles * (2 if own_count > 128 else 1) + 2
    return (cmax - cost) * BUCKETS // (cmax + 1)


def host_bound(n_keyed, L, own_rows, G):
    return 16 * G + sum(div_up(n, own_rows) + L + 1 for n in n_keyed)


def plan(own, strm, own_rows, G):
    """own[c][l], strm[l]: group sizes -> (per, goff, hist, n_items, tests, cta_off)."""
    n_cls, L = len(own), len(strm)
    tiles, tests = 0, [0] * n_cls
    for l in range(L):
        for c in range(n_cls):
            no, ns = own[c][l], strm[l]
            if no and ns:
                tiles += div_up(no, own_rows) * div_up(ns, STREAM_TILE)
                tests[c] += no * ns
    per = max(1, tiles // (G * 8))
    counts, hist = [], [0] * BUCKETS
    for c in range(n_cls):
        for l in range(L):
            no, ns = own[c][l], strm[l]
            items = 0
            if no and ns:
                A, nb = div_up(no, own_rows), div_up(ns, STREAM_TILE)
                nbp = div_up(nb, per)
                items = A * nbp
                rem_o, rem_b = no - (A - 1) * own_rows, nb - (nbp - 1) * per
                if A > 1 and nbp > 1:
                    hist[cost_bucket(per, own_rows, per)] += (A - 1) * (nbp - 1)
                if A > 1:
                    hist[cost_bucket(rem_b, own_rows, per)] += A - 1
                if nbp > 1:
                    hist[cost_bucket(per, rem_o, per)] += nbp - 1
                hist[cost_bucket(rem_b, rem_o, per)] += 1
            counts.append(items)
    goff = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n_items = int(goff[-1])
    R, rem = n_items // G, n_items % G
    sizes = [R + ((g < rem) if R % 2 == 0 else (g >= G - rem)) for g in range(G)]
    cta_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return per, goff, hist, n_items, tests, cta_off


def place(own, strm, own_rows, G, per, goff, hist, n_items, cta_off):
    """Every item as the placement kernel builds it -> list slots and items."""
    L = len(strm)
    boff = np.concatenate([[0], np.cumsum(hist)[:-1]]).astype(np.int64)
    bcnt = [0] * BUCKETS
    slots = {}
    for k in range(n_items):
        g = int(np.searchsorted(goff, k, side="right")) - 1      # last goff[g] <= k
        c, l = g // L, g % L
        no, ns = own[c][l], strm[l]
        nb = div_up(ns, STREAM_TILE)
        nbp = div_up(nb, per)
        j = k - int(goff[g])
        a, bs = j // nbp, (j % nbp) * per
        item = (c, l, a * own_rows, min(own_rows, no - a * own_rows), bs * STREAM_TILE,
                min(per, nb - bs), min(per * STREAM_TILE, ns - bs * STREAM_TILE))
        bk = cost_bucket(item[5], item[3], per)
        sp = int(boff[bk]) + bcnt[bk]
        bcnt[bk] += 1
        rnd, kk = sp // G, sp % G
        cta = G - 1 - kk if rnd % 2 else kk
        slot = int(cta_off[cta]) + rnd
        assert cta_off[cta] <= slot < cta_off[cta + 1], "item outside its CTA's list"
        assert slot not in slots, "two items in one list slot"
        slots[slot] = item
    assert bcnt == list(hist), "closed-form cost classes differ from the items' classes"
    return slots


def check(own, strm, own_rows, G):
    n_keyed = [sum(o) for o in own]
    per, goff, hist, n_items, tests, cta_off = plan(own, strm, own_rows, G)
    assert n_items <= host_bound(n_keyed, len(strm), own_rows, G)
    slots = place(own, strm, own_rows, G, per, goff, hist, n_items, cta_off)
    assert sorted(slots) == list(range(n_items)) and cta_off[-1] == n_items
    # Coverage: per (class, group), the items tile the own x stream rectangle
    # exactly once.
    met = [0] * len(own)
    cover = {}
    for c, l, o0, oc, s0, bt, sc in slots.values():
        assert oc >= 1 and sc >= 1 and bt == div_up(sc, STREAM_TILE)
        met[c] += oc * sc
        cover.setdefault((c, l), []).append((o0, oc, s0, sc))
    assert met == tests
    for (c, l), parts in cover.items():
        # The own tiles partition [0, no), each one's stream ranges partition
        # [0, ns), and no (own tile, stream range) pair repeats.
        assert len(set(parts)) == len(parts)
        by_tile = {}
        for o0, oc, s0, sc in parts:
            by_tile.setdefault((o0, oc), []).append((s0, sc))
        edge = 0
        for o0, oc in sorted(by_tile):
            assert o0 == edge
            edge = o0 + oc
            end = 0
            for s0, sc in sorted(by_tile[(o0, oc)]):
                assert s0 == end
                end = s0 + sc
            assert end == strm[l]
        assert edge == own[c][l]
    return n_items


@pytest.mark.parametrize("seed", range(12))
def test_random_groups(seed):
    rng = np.random.default_rng(seed)
    n_cls = 1 + seed % 2
    own_rows = OWN_TILE * (2 if n_cls == 2 else 1)
    L = int(rng.choice([8, 64, 464]))
    G = int(rng.choice([1, 7, 152]))
    skew = rng.pareto(1.2, size=L)
    strm = (skew / skew.sum() * rng.integers(1, 40000)).astype(int)
    own = [(rng.pareto(1.5, size=L) * rng.integers(1, 300)).astype(int) for _ in range(n_cls)]
    for o in own:
        o[rng.random(L) < 0.3] = 0                        # groups without patterns
    strm[rng.random(L) < 0.1] = 0                         # groups without records
    check(own, list(strm), own_rows, G)


def test_extremes():
    # One huge group and many empty ones; a single row; more CTAs than
    # items; the largest index width.
    assert check([[0] * 9 + [5000]], [0] * 9 + [300000], OWN_TILE, 152) > 152
    # The 148k evidence shape: 464 groups, skewed, both classes, per > 1.
    rng = np.random.default_rng(148)
    w = rng.pareto(1.1, size=464)
    strm = list((w / w.sum() * 133200 * 41).astype(int))
    own = [list((rng.pareto(1.3, size=464) * 300).astype(int)) for _ in range(2)]
    assert check(own, strm, 2 * OWN_TILE, 152) > 8 * 152
    assert check([[1]], [1], OWN_TILE, 152) == 1
    assert check([[3] * 4, [0] * 4], [2] * 4, 2 * OWN_TILE, 152) == 4
    rng = np.random.default_rng(5)
    L = 1024
    check([list(rng.integers(0, 20, L)), list(rng.integers(0, 20, L))],
          list(rng.integers(0, 500, L)), 2 * OWN_TILE, 152)
    assert check([[0, 0], [0, 0]], [5, 5], 2 * OWN_TILE, 152) == 0
