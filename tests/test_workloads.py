"""Input generators: batch concatenation keeps every box's data and maps
exclusion partners to batch-global indices inside the same box; a group's
exclusion subset; the prune radius (reading R9)."""
import numpy as np
import pytest

from paper_1306_1737_gb300 import workloads as w


def test_concat_offsets_and_exclusions():
    boxes = [w.water_box(40, 1.2, seed=1), w.water_box(25, 1.0, seed=2), w.water_box(33, 1.1, seed=3)]
    B = w.concat(boxes)
    off = B.offsets
    assert B.nbox == 3 and B.n == sum(b.n for b in boxes) and off[-1] == B.n
    assert B.excl_off.shape == (B.n + 1,) and B.excl_off[-1] == B.excl_idx.size
    for k, b in enumerate(boxes):
        sl = slice(int(off[k]), int(off[k + 1]))
        assert np.array_equal(B.xyz[sl], b.xyz) and np.array_equal(B.q[sl], b.q)
        assert np.array_equal(B.types[sl], b.types) and np.array_equal(B.boxes[k], b.box)
        for i in range(b.n):
            got = B.excl_idx[B.excl_off[off[k] + i]:B.excl_off[off[k] + i + 1]]
            want = b.excl_idx[b.excl_off[i]:b.excl_off[i + 1]] + off[k]
            assert np.array_equal(got, want)
            assert np.all((got >= off[k]) & (got < off[k + 1]))


def test_batch_sizes_range():
    s = w.batch_sizes(256, seed=1004)
    assert s.shape == (256,) and np.all(s % 3 == 0)
    assert s.min() >= 1497 and s.max() <= 60000
    # log-uniform: the median sits near the geometric mean of the bounds
    assert abs(np.log(np.median(s)) - 0.5 * (np.log(1500) + np.log(60000))) < 0.3


def test_prune_radius_reading():
    """R9: rc + 6 sigma of the relative displacement of two hydrogens over
    nstprune steps (sigma^2 = 2 kB T / m_H (dt)^2 nstprune), capped at rlist;
    about 1.06 nm for rc 1.0, rlist 1.1, five 2 fs steps at 300 K."""
    import math
    kT = 0.0083144626 * 300.0
    s = math.sqrt(2.0 * kT / 1.008) * 0.002 * math.sqrt(5)
    assert w.prune_radius(1.0, 1.1, 5) == pytest.approx(1.0 + 6.0 * s, rel=1e-6)
    assert abs(w.prune_radius(1.0, 1.1, 5) - 1.0597) < 1e-3
    assert w.prune_radius(1.0, 1.02, 5) == pytest.approx(1.02)          # capped at rlist
    assert w.prune_radius(1.0, 1.1, 20) > w.prune_radius(1.0, 1.1, 5)   # grows with the interval


def test_subset_exclusions_of_a_group_of_boxes():
    """The exclusion CSR of a subset of a batch's boxes, with partner indices
    renumbered to the subset's particles, equals the concatenation of the
    chosen boxes' own exclusion lists."""
    from paper_1306_1737_gb300.batch import _subset_csr
    boxes = [w.water_box(m, None, seed=910 + k) for k, m in enumerate([40, 70, 55])]
    B = w.concat(boxes)
    off = B.offsets
    for pick in ([1], [0, 2], [2, 1], [0, 1, 2]):
        eo, ei = _subset_csr(B.excl_off, B.excl_idx, off, pick)
        want = w.concat([boxes[k] for k in pick])
        assert np.array_equal(eo, want.excl_off) and np.array_equal(ei, want.excl_idx), pick
