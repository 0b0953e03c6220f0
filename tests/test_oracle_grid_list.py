"""Pins of the oracle's spatial clustering (Sec. 2.3), cluster-pair list
(Sec. 2.3, Fig. 3), exclusion masks (Sec. 2.4) and pruning (Sec. 2.3).

The list and masks are checked against a plain Python expansion to particle
pairs built from the minimum-image definition and the exclusion list."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def grid_invariants(b, g, C):
    n = b.n
    real = g.atom_of_slot[g.atom_of_slot >= 0]
    # a permutation of the particles, with its inverse
    assert np.array_equal(np.sort(real), np.arange(n))
    assert np.array_equal(g.atom_of_slot[g.slot_of_atom], np.arange(n))
    # wrapped coordinates in [0, L)
    L32 = b.box.astype(np.float32)
    assert np.all(g.wrapped >= 0) and np.all(g.wrapped < L32)
    # each particle sits in the column of its x/y cell (FP64 check away from
    # cell edges)
    fx = g.wrapped[:, 0].astype(np.float64) * g.nx / L32[0]
    fy = g.wrapped[:, 1].astype(np.float64) * g.ny / L32[1]
    ix = np.minimum(np.floor(fx), g.nx - 1).astype(int)
    iy = np.minimum(np.floor(fy), g.ny - 1).astype(int)
    away = (np.abs(fx - np.round(fx)) > 1e-5) & (np.abs(fy - np.round(fy)) > 1e-5)
    assert np.array_equal((ix * g.ny + iy)[away], g.col_of_atom[away])
    # columns in order, clusters consecutive, each column padded at its end
    cs = g.col_clu_start
    assert cs[0] == 0 and cs[-1] == g.nclu and np.all(np.diff(cs) >= 0)
    counts = np.bincount(g.col_of_atom, minlength=g.nx * g.ny)
    assert np.array_equal(np.diff(cs), (counts + C - 1) // C)
    for c in range(g.nx * g.ny):
        slots = np.arange(cs[c] * C, cs[c + 1] * C)
        atoms = g.atom_of_slot[slots]
        k = counts[c]
        assert np.all(atoms[:k] >= 0) and np.all(atoms[k:] < 0)
        assert np.all(g.col_of_atom[atoms[:k]] == c)
        z = g.wrapped[atoms[:k], 2]
        # sorted on z, ties by original index
        keys = list(zip(z.tolist(), atoms[:k].tolist()))
        assert keys == sorted(keys)
    # bounding boxes are exactly the extent of the real particles
    for cl in range(g.nclu):
        atoms = g.atom_of_slot[cl * C:(cl + 1) * C]
        atoms = atoms[atoms >= 0]
        assert atoms.size >= 1
        p = g.wrapped[atoms]
        assert np.array_equal(g.bb[cl, :3], p.min(0)) and np.array_equal(g.bb[cl, 3:], p.max(0))
    # slot data: coordinates, charges and types of the real particles
    s = g.slot_of_atom
    assert np.array_equal(g.xyzq[s, :3], g.wrapped)
    assert np.array_equal(g.xyzq[s, 3], b.q)
    assert np.array_equal(g.type_slot[s], b.types)
    # dummies: no charge, far from every particle and from each other
    d = np.nonzero(g.atom_of_slot < 0)[0]
    assert np.all(g.xyzq[d, 3] == 0)
    if d.size:
        G = oracle.dummy_spacing(b.box)
        assert G >= 4 * L32.max()
        assert np.all(g.xyzq[d, :3] <= -G)
        pos = g.xyzq[d, :3]
        assert np.unique(pos, axis=0).shape[0] == d.size


@pytest.mark.parametrize("C", [4, 8])
def test_grid_config1(cfg1, C):
    b, _ = cfg1
    g = oracle.grid(b.xyz, b.q, b.types, b.box, C)
    grid_invariants(b, g, C)
    # grid spacing (C / rho)^(1/3) (Sec. 2.3)
    s = (C * np.prod(b.box.astype(np.float32).astype(np.float64)) / b.n) ** (1 / 3)
    assert g.nx == max(1, int(np.floor(np.float32(b.box[0]) / s)))


def test_dummy_fraction_matches_paper_estimate():
    # Sec. 2.3: ~4% dummies with clusters of 8 and 10000 particles; the
    # estimate 1/2 (C/N)^(1/3) (reading of the garbled formula).
    b = w.water_box(3334, None, seed=12)
    g = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
    frac = (g.atom_of_slot < 0).mean()
    est = 0.5 * (8 / b.n) ** (1 / 3)
    assert frac == pytest.approx(GOLD["dummy_fraction_c8_n10000"]["value"], abs=0.015)
    assert 0.5 * est < frac < 1.5 * est


def test_grid_adversarial():
    # particles on cell edges, equal z, a wrap from both sides, empty columns,
    # fewer particles than a cluster
    L = np.array([2.0, 2.0, 2.0])
    xyz = np.array([[0.0, 0.0, 0.5], [1.0, 1.0, 0.5], [1.0, 1.0, 0.5], [-0.25, 1.999, 2.5],
                    [1.0, 0.0, 0.5], [0.5, 0.5, 1.9999999]], np.float32)
    q = np.arange(6, dtype=np.float32)
    t = np.zeros(6, np.int32)
    g = oracle.grid(xyz, q, t, L, 8)
    assert g.wrapped[3].tolist() == [np.float32(-0.25) + np.float32(2.0), np.float32(1.999),
                                     np.float32(0.5)]
    # equal z broken by original index: 1 before 2
    s1, s2 = g.slot_of_atom[1], g.slot_of_atom[2]
    assert g.col_of_atom[1] == g.col_of_atom[2] and s1 < s2

    class B:
        pass
    bb = B()
    bb.n, bb.box, bb.q, bb.types = 6, L, q, t
    grid_invariants(bb, g, 8)
    # one particle only
    g1 = oracle.grid(xyz[:1], q[:1], t[:1], L, 8)
    assert g1.nclu == 1 and (g1.atom_of_slot >= 0).sum() == 1
    # out of [-L, 2L) is an error
    with pytest.raises(ValueError):
        oracle.grid(np.array([[4.5, 0, 0]], np.float32), q[:1], t[:1], L, 8)


def expand_pairs(g, pl, excl_set):
    """Particle pairs (lo, hi, image shift) from the list keys: bit -> full,
    no bit -> correction (only meaningful for excluded pairs)."""
    C = g.C
    full, corr = {}, {}
    for a, b_, s, m in zip(pl.a.tolist(), pl.b.tolist(), pl.s.tolist(), pl.mask.tolist()):
        for i in range(C):
            pi = int(g.atom_of_slot[a * C + i])
            if pi < 0:
                continue
            for j in range(C):
                pj = int(g.atom_of_slot[b_ * C + j])
                if pj < 0 or pj == pi:
                    continue
                if a == b_ and s == 13 and j <= i:
                    continue
                key = (min(pi, pj), max(pi, pj), s if pi < pj else 26 - s)
                bit = (m >> (i * C + j)) & 1
                tgt = full if bit else corr
                tgt[key] = tgt.get(key, 0) + 1
    return full, corr


def min_image_pairs(xyz, L, r):
    out = {}
    x = xyz.astype(np.float64)
    n = x.shape[0]
    for i in range(n):
        d = x[i] - x[i + 1:]
        img = -np.round(d / L)
        d = d + img * L
        r2 = (d * d).sum(1)
        for k in np.nonzero(r2 < r * r)[0]:
            sv = img[k].astype(int)
            s = (sv[0] + 1) * 9 + (sv[1] + 1) * 3 + (sv[2] + 1)
            out[(i, i + 1 + int(k), s)] = math.sqrt(r2[k])
    return out


@pytest.mark.parametrize("nmol,L,C,rlist", [(100, 1.45, 8, 0.7), (60, 1.25, 4, 0.6),
                                            (512, 2.48, 8, 1.0), (70, 2.05, 8, 1.0)])
def test_list_covers_every_pair_once_with_correct_bits(nmol, L, C, rlist):
    # Small boxes (including ones where a cluster pair is in range under two
    # different shifts): expand the keys to particle pairs and compare with
    # the minimum-image pairs within rlist and the exclusion list.
    b = w.water_box(nmol, L, seed=nmol)
    g = oracle.grid(b.xyz, b.q, b.types, b.box, C)
    pl = oracle.pairlist(g, rlist, 0.0, b.excl_off, b.excl_idx)
    excl = set()
    for i in range(b.n):
        for j in b.excl_idx[b.excl_off[i]:b.excl_off[i + 1]]:
            excl.add((min(i, int(j)), max(i, int(j))))
    full, corr = expand_pairs(g, pl, excl)
    assert all(v == 1 for v in full.values())
    assert all(v == 1 for v in corr.values())
    within = min_image_pairs(g.wrapped, b.box.astype(np.float32).astype(np.float64), rlist)
    # every pair within rlist appears exactly once, with the right bit
    for (i, j, s), d in within.items():
        in_full = (i, j, s) in full
        in_corr = (i, j, s) in corr
        assert in_full != in_corr, (i, j, s, d)
        assert in_corr == ((i, j) in excl)
    # excluded pairs never carry a bit, under any shift
    assert not any((i, j) in excl for (i, j, _) in full)
    # every key has a particle pair within rlist (rBB = 0) and nothing else
    dm, db = oracle.key_distances(g, pl.a, pl.b, pl.s)
    assert np.all(dm < rlist) and np.all(db <= dm + 1e-12)
    assert np.all(pl.a <= pl.b)
    assert np.all((pl.a != pl.b) | (pl.s >= 13))
    cov = oracle.pair_cover(g, pl, rlist)
    assert cov[1] == 0 and cov[2] == 0 and cov[0] == len(within)


def test_list_rbb_shortcut_is_superset():
    # Fig. 3: with rBB > 0 cluster pairs whose bounding boxes are closer than
    # rBB skip the particle test; the list can only grow.
    b = w.water_box(200, None, seed=21)
    g = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
    p0 = oracle.pairlist(g, 0.8, 0.0, b.excl_off, b.excl_idx)
    p1 = oracle.pairlist(g, 0.8, 0.6, b.excl_off, b.excl_idx)
    k0, k1 = p0.keys(), p1.keys()
    assert k0 <= k1 and len(k1) > len(k0)
    dm, db = oracle.key_distances(g, p1.a, p1.b, p1.s)
    extra = np.array([k not in k0 for k in zip(p1.a.tolist(), p1.b.tolist(), p1.s.tolist())])
    assert np.all(db[extra] < 0.6) and np.all(dm[extra] >= 0.8)


def test_list_size_ratio_4x4_matches_paper():
    # Sec. 5 / Fig. 3: at 1 nm a 4x4 list holds 86% more particle pairs than
    # the sphere (3-site water at 100 nm^-3).
    b = w.water_box(3000, None, seed=5)
    g = oracle.grid(b.xyz, b.q, b.types, b.box, 4)
    pl = oracle.pairlist(g, 1.0, 0.0, b.excl_off, b.excl_idx)
    real = (g.atom_of_slot >= 0).reshape(-1, 4).sum(1)
    diag = (pl.a == pl.b) & (pl.s == 13)
    listed = np.where(diag, real[pl.a] * (real[pl.a] - 1) // 2, real[pl.a] * real[pl.b]).sum()
    ratio = listed / oracle.count_pairs_within(b.xyz, b.box, 1.0)
    assert ratio - 1 == pytest.approx(GOLD["extra_pairs_4x4_at_1nm"]["value"], rel=0.15)


def test_prune_keeps_every_pair_within_radius():
    # After moving particles, prune at r_prune: every pair closer than r_prune
    # is still in a kept key; keys dropped have no counted pair closer.
    b = w.water_box(512, 2.48, seed=3)
    g = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
    pl = oracle.pairlist(g, 1.0, 0.0, b.excl_off, b.excl_idx)
    disp = w.frame_displacements(b.mass, 3, seed=9).sum(0)
    xyz1 = b.xyz + disp
    x1 = oracle.slot_coords(g, xyz1)
    keep, dmin = oracle.prune(g, pl, 0.95, x1)
    assert 0 < keep.sum() < len(pl)
    assert np.all(dmin[keep] < 0.95) and np.all(dmin[~keep] >= 0.95)
    # the wrap offset is preserved: slot coordinates move by the displacement
    real = g.atom_of_slot >= 0
    mv = x1[real, :3].astype(np.float64) - g.xyzq[real, :3]
    assert np.abs(mv - disp[g.atom_of_slot[real]]).max() < 1e-5
    kept = oracle.PairList(pl.a[keep], pl.b[keep], pl.s[keep], pl.mask[keep])
    g1 = oracle.Grid(**{**g.__dict__, "wrapped": np.zeros_like(g.wrapped)})
    g1.wrapped[g.atom_of_slot[real]] = x1[real, :3]
    cov = oracle.pair_cover(g1, kept, 0.95)
    assert cov[1] == 0 and cov[2] == 0
    # the diagonal key of every cluster with two or more particles is kept
    nreal = real.reshape(-1, 8).sum(1)
    diag_keys = {(a, a, 13) for a in np.nonzero(nreal >= 2)[0].tolist()}
    assert diag_keys <= kept.keys()
