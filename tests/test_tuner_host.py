"""The autotuner's host logic on the CPU, with the GPU timing of a candidate
group replaced by a synthetic cost: size classes cover every box once, the
fastest candidate wins each class (cluster size and list lifetime first,
then the prune interval), the winners are cached per batch and read back,
and the list radius of a lifetime follows the sqrt rule or the Appendix's
drift bound."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1306_1737_gb300 import batch, tuner  # noqa: E402


def _batch(n_boxes=12, seed=3):
    rng = np.random.default_rng(seed)
    counts = rng.integers(1500, 60000, n_boxes)
    boxes = np.stack([np.full(3, (c / 100.0) ** (1 / 3)) for c in counts])
    return counts, boxes


def test_classes_cover_every_box_once_by_size():
    counts, _ = _batch(13)
    cls = tuner._classes(counts, 4)
    flat = sorted(i for c in cls for i in c)
    assert flat == list(range(13))
    # classes are ordered by size: every box of a class is at most every box of the next
    for a, b in zip(cls, cls[1:]):
        assert counts[a].max() <= counts[b].min()


def test_key_changes_with_the_inputs():
    counts, boxes = _batch()
    p = {"elec": "ewald", "rc": 1.0, "beta": 3.12}
    k0 = tuner._key("gpu", counts, boxes, p, 1.1, 20, 5, 40)
    assert k0 == tuner._key("gpu", counts, boxes, dict(p), 1.1, 20, 5, 40)
    assert k0 != tuner._key("other gpu", counts, boxes, p, 1.1, 20, 5, 40)
    assert k0 != tuner._key("gpu", counts, boxes, dict(p, rc=0.9), 1.1, 20, 5, 40)
    assert k0 != tuner._key("gpu", counts, boxes, p, 1.1, 20, 2, 40)


def test_scaled_rlist_is_the_sqrt_rule():
    assert batch.scaled_rlist(1.0, 1.1, 20, 20) == pytest.approx(1.1)
    assert batch.scaled_rlist(1.0, 1.1, 20, 40) == pytest.approx(1.0 + 0.1 * math.sqrt(2.0))
    assert batch.scaled_rlist(1.0, 1.1, 20, 5) == pytest.approx(1.05)


def test_two_stage_choice_and_cache(tmp_path, monkeypatch):
    counts, boxes = _batch()
    n = int(counts.sum())
    frames = np.zeros((40, 1, 3), np.float32)          # only its length (the horizon) is read
    p = {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12}
    calls = []

    def fake_time(spec, *args, **kwargs):
        # cost per frame: C = 8 cheaper than C = 4, nstlist 20 best, then prune every 10 best
        calls.append((spec.C, spec.nstlist, spec.nstprune, tuple(spec.boxes)))
        size = float(counts[spec.boxes].sum())
        c = size * (1.0 if spec.C == 8 else 2.0) * {10: 1.2, 20: 1.0, 40: 1.1}[spec.nstlist]
        nsp = 5 if spec.nstprune is None else spec.nstprune
        return c * {2: 1.05, 5: 1.0, 10: 0.97}[nsp]

    monkeypatch.setattr(tuner, "time_group", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=0: "fake gpu")
    cache = str(tmp_path / "cache.json")
    args = (counts, boxes, np.zeros(n), np.zeros(n, np.int32), np.zeros((1, 2)), np.zeros(n + 1, np.int32),
            np.zeros(0, np.int32), frames, p, 5, 1.1, 20)
    groups, table = tuner.tune(*args, n_classes=3, cache_path=cache)
    assert len(table) == 3 and not any(t["cached"] for t in table)
    assert all(t["best"] == "8/20/10" for t in table)
    assert len(groups) == 1
    g = groups[0]
    assert (g.C, g.nstlist, g.nstprune) == (8, 20, 10)
    assert sorted(g.boxes) == list(range(len(counts)))
    assert g.rlist == pytest.approx(1.1)
    # first stage: 2 cluster sizes x 3 lifetimes per class; second: the other prune intervals
    # below the winning lifetime (2 and 10)
    assert len(calls) == 3 * (6 + 2)
    # a second call reads every class from the cache and times nothing
    calls.clear()
    groups2, table2 = tuner.tune(*args, n_classes=3, cache_path=cache)
    assert calls == [] and all(t["cached"] for t in table2)
    assert [(x.C, x.nstlist, x.nstprune, x.boxes) for x in groups2] == [(g.C, g.nstlist, g.nstprune, g.boxes)]


def test_particle_classes_and_appendix_rlist():
    pytest.importorskip("ctypes")
    import paper_1306_1737_gb300 as nb
    try:
        nb.load()
    except RuntimeError:
        pytest.skip("library not built")
    from paper_1306_1737_gb300 import workloads as w
    b = w.water_box(300, None, seed=11)
    cls = tuner.particle_classes(b.q, b.types, b.mass)
    assert sum(c[0] for c in cls) == b.n
    assert len(cls) == 2                                  # O and H sites
    p = {"elec": "ewald", "rc": 1.0, "beta": 3.12}
    table = nb.nb_lj_combine(b.sigma, b.eps)
    vol = float(np.prod(b.box))
    r = [tuner.appendix_rlist(cls, table, vol, p, nst) for nst in (10, 20, 40)]
    assert all(x > 1.0 for x in r)
    assert r[0] < r[1] < r[2]                             # a longer lifetime needs a larger buffer


def _tune_args(counts, boxes, frames_len=40):
    n = int(counts.sum())
    frames = np.zeros((frames_len, 1, 3), np.float32)
    p = {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12}
    return (counts, boxes, np.zeros(n), np.zeros(n, np.int32), np.zeros((1, 2)), np.zeros(n + 1, np.int32),
            np.zeros(0, np.int32), frames, p, 5, 1.1, 20)


def test_cache_file_in_the_working_directory(tmp_path, monkeypatch):
    counts, boxes = _batch(4)
    monkeypatch.setattr(tuner, "time_group", lambda spec, *a, **k: float(spec.C + spec.nstlist))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=0: "fake gpu")
    monkeypatch.chdir(tmp_path)
    groups, _ = tuner.tune(*_tune_args(counts, boxes), n_classes=2, cache_path="cache.json")
    assert (tmp_path / "cache.json").exists()
    assert [(g.C, g.nstlist) for g in groups] == [(4, 10)]


def test_no_candidate_fits_small_boxes(monkeypatch):
    """Boxes of 1.5 nm: every list radius (>= rc = 1.0 nm) reaches half a box
    edge, so nothing can be timed and the tuner says why."""
    counts = np.array([300, 330])
    boxes = np.full((2, 3), 1.5)
    monkeypatch.setattr(tuner, "time_group", lambda *a, **k: pytest.fail("nothing should be timed"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=0: "fake gpu")
    with pytest.raises(ValueError, match="no candidate fits"):
        tuner.tune(*_tune_args(counts, boxes), n_classes=1)
    # a horizon no list lifetime divides
    counts, boxes = _batch(2)
    with pytest.raises(ValueError, match="no candidate fits"):
        tuner.tune(*_tune_args(counts, boxes, frames_len=7), n_classes=1)


def test_every_candidate_failing_raises(monkeypatch):
    counts, boxes = _batch(3)
    monkeypatch.setattr(tuner, "time_group", lambda *a, **k: float("inf"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=0: "fake gpu")
    with pytest.raises(RuntimeError, match="failed"):
        tuner.tune(*_tune_args(counts, boxes), n_classes=1)


def test_batch_runner_refuses_a_horizon_a_lifetime_does_not_divide():
    """The check runs before any context is created (no device needed)."""
    counts, boxes = _batch(2)
    n = int(counts.sum())
    frames = np.zeros((30, n, 3), np.float32)
    with pytest.raises(ValueError, match="multiple"):
        batch.BatchRunner(counts, boxes, np.zeros(n), np.zeros(n, np.int32), np.zeros((1, 1, 2)),
                          np.zeros(n + 1, np.int32), np.zeros(0, np.int32), frames,
                          [batch.GroupSpec(8, 20, 1.1, [0, 1])], {"elec": "ewald", "rc": 1.0}, 5)
