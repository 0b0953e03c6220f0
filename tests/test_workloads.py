"""Input generators: batch concatenation keeps every box's data and maps
exclusion partners to batch-global indices inside the same box."""
import numpy as np

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
