"""Host model of the warp-level bit manipulation the binning kernels use, run on
the CPU (no GPU): the 32 x 32 bit transpose across a warp (five butterfly
exchanges), the search of an instance's owner lane in a non-decreasing
per-lane prefix, and the n-th set bit of a mask. Checked on random inputs
against plain definitions, and in the two enumerations built from them: the
cull numbers the (plane, Gaussian) pairs that pass its first test plane by
plane and hands them out 32 at a time, and the work list walks each lane's
own planes; both must visit every set bit exactly once."""
import numpy as np

MASKS = (0x0000FFFF, 0x00FF00FF, 0x0F0F0F0F, 0x33333333, 0x55555555)


def bit_transpose(rows):
    """Lane r holds row r (bit c = element (r, c)); after five exchanges with
    lane r ^ j (j = 16, 8, 4, 2, 1) lane c holds column c."""
    x = [int(v) for v in rows]
    for k, m in enumerate(MASKS):
        j = 16 >> k
        y = [x[lane ^ j] for lane in range(32)]
        x = [((x[lane] & ~m) | ((y[lane] >> j) & m)) & 0xFFFFFFFF if lane & j
             else ((x[lane] & m) | ((y[lane] & m) << j)) & 0xFFFFFFFF for lane in range(32)]
    return x


def owner_lane(pre, o):
    """Largest lane l with pre[l] <= o (pre non-decreasing), by halving steps."""
    lane = 0
    step = 16
    while step:
        if pre[lane + step] <= o:
            lane += step
        step >>= 1
    return lane


def nth_set_bit(m, n):
    pos = 0
    for w in (32, 16, 8, 4, 2, 1):
        c = bin(m & ((1 << w) - 1)).count("1")
        if n >= c:
            n -= c
            m >>= w
            pos += w
    return pos


def test_bit_transpose_is_the_transpose():
    rng = np.random.default_rng(0)
    for _ in range(200):
        rows = rng.integers(0, 1 << 32, 32, dtype=np.uint64)
        cols = bit_transpose(rows)
        for c in range(32):
            for r in range(32):
                assert (cols[c] >> r) & 1 == (int(rows[r]) >> c) & 1


def test_nth_set_bit():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        m = int(rng.integers(0, 1 << 63)) & int(rng.integers(0, 1 << 63))
        if m == 0:
            continue
        bits = [i for i in range(64) if (m >> i) & 1]
        n = int(rng.integers(0, len(bits)))
        assert nth_set_bit(m, n) == bits[n]


def test_cull_pair_enumeration_visits_every_pass_once():
    """32 lanes (Gaussians) x 32 planes of first-test results: the transposed
    masks give each plane's passing lanes; pair e (numbered plane by plane) is
    owned by the plane whose exclusive count prefix is the largest <= e, and its
    Gaussian is the (e - prefix)-th set bit of that plane's mask."""
    rng = np.random.default_rng(2)
    for density in (0.02, 0.13, 0.5, 1.0):
        for _ in range(50):
            passes = (rng.random((32, 32)) < density)  # [lane, plane]
            rows = [sum(int(passes[lane, q]) << q for q in range(32)) for lane in range(32)]
            pm = bit_transpose(rows)  # lane q: plane q's passing Gaussians
            cnt = [bin(x).count("1") for x in pm]
            excl = list(np.concatenate([[0], np.cumsum(cnt)[:-1]]))
            total = sum(cnt)
            seen = set()
            for rb in range(0, total, 32):
                for lane in range(32):
                    e = rb + lane
                    if e >= total:
                        continue
                    q = owner_lane(excl, e)
                    g = nth_set_bit(pm[q], e - excl[q])
                    assert passes[g, q]
                    assert (q, g) not in seen
                    seen.add((q, g))
            assert len(seen) == int(passes.sum())


def test_list_walk_visits_each_lanes_planes_in_order():
    """The work list: a chunk's candidate masks (one per plane, bit = Gaussian
    lane) transposed, so lane g holds the planes of its own candidates and
    walks them in ascending order; every candidate gets its record slot
    base[q] + (number of candidates of plane q in lower lanes)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        masks = [int(x) for x in rng.integers(0, 1 << 32, 32, dtype=np.uint64)]
        masks = [m & int(rng.integers(0, 1 << 32)) for m in masks]
        base = list(np.concatenate([[0], np.cumsum([bin(m).count("1") for m in masks])[:-1]]))
        mine = bit_transpose(masks)
        slots = []
        for g in range(32):
            planes = [q for q in range(32) if (mine[g] >> q) & 1]
            assert planes == sorted(planes)
            for q in planes:
                assert (masks[q] >> g) & 1
                slots.append(base[q] + bin(masks[q] & ((1 << g) - 1)).count("1"))
        assert sorted(slots) == list(range(sum(bin(m).count("1") for m in masks)))
