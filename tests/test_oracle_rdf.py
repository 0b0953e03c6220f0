"""Oracle pins for the pair-distance histogram (pair correlation function;
Sec. 1 names it as limited-range pair work, Sec. 2.3 gives its kernel form).

Closed forms on a simple cubic lattice of spacing a: every site has 6
neighbours at a, 12 at sqrt(2) a, 8 at sqrt(3) a and 6 at 2 a, so a box of N
sites holds 3N, 6N, 4N and 3N unordered pairs at those distances; on a
checkerboard colouring, neighbours at a and sqrt(3) a have opposite colours
and those at sqrt(2) a and 2 a equal colours.  Exclusions remove exactly the
excluded pairs.  The cell-list enumeration is pinned against the O(n^2)
double loop and against the independent brute-force pair count."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

A = 0.5
NS = 6                      # 6^3 = 216 sites, box 3 nm
N = NS ** 3
SHELLS = {1: 6, 2: 12, 3: 8, 4: 6}   # squared distance / a^2 -> coordination


def lattice():
    g = np.stack(np.meshgrid(np.arange(NS), np.arange(NS), np.arange(NS), indexing="ij"), -1).reshape(-1, 3)
    xyz = (g * A + 0.1).astype(np.float32)
    colour = (g.sum(1) % 2).astype(np.int32)
    return xyz, colour, np.full(3, NS * A)


def expected(r_max, nbins, per_shell):
    dr = r_max / nbins
    h = np.zeros(nbins, np.int64)
    for s2, cnt in per_shell.items():
        r = math.sqrt(s2) * A
        if r < r_max:
            h[int(r // dr)] += cnt
    return h


@pytest.mark.parametrize("brute", [False, True])
def test_cubic_lattice_shells(brute):
    xyz, colour, box = lattice()
    r_max, nbins = 2.21 * A, 17            # edges avoid a, sqrt2 a, sqrt3 a, 2 a
    h, _ = oracle.rdf(xyz, colour, box, r_max, nbins, brute=brute)
    want = expected(r_max, nbins, {s: N * z // 2 for s, z in SHELLS.items()})
    assert np.array_equal(h, want)
    assert h.sum() == (6 + 12 + 8 + 6) * N // 2


def test_checkerboard_type_selection():
    xyz, colour, box = lattice()
    r_max, nbins = 2.21 * A, 17
    same = {2: 12, 4: 6}                   # even shells: equal colours
    # type 0 with type 0: N/2 sites, each with 12 (6) same-colour neighbours
    h00, _ = oracle.rdf(xyz, colour, box, r_max, nbins, type_a=0, type_b=0)
    assert np.array_equal(h00, expected(r_max, nbins, {s: (N // 2) * z // 2 for s, z in same.items()}))
    h11, _ = oracle.rdf(xyz, colour, box, r_max, nbins, type_a=1, type_b=1)
    assert np.array_equal(h11, h00)
    # opposite colours: every odd-shell pair
    h01, _ = oracle.rdf(xyz, colour, box, r_max, nbins, type_a=0, type_b=1)
    h10, _ = oracle.rdf(xyz, colour, box, r_max, nbins, type_a=1, type_b=0)
    assert np.array_equal(h01, expected(r_max, nbins, {1: N * 6 // 2, 3: N * 8 // 2}))
    assert np.array_equal(h01, h10)
    hall, _ = oracle.rdf(xyz, colour, box, r_max, nbins)
    assert np.array_equal(hall, h00 + h11 + h01)


def test_exclusions_remove_exactly_the_excluded_pairs():
    xyz, colour, box = lattice()
    g = np.round((xyz - 0.1) / A).astype(int)
    idx = {tuple(v): i for i, v in enumerate(g)}
    # exclude each site's +x neighbour (periodic): N pairs at distance a
    nbr = [[] for _ in range(N)]
    for i, v in enumerate(g):
        j = idx[((v[0] + 1) % NS, v[1], v[2])]
        nbr[i].append(j)
        nbr[j].append(i)
    off = np.zeros(N + 1, np.int32)
    off[1:] = np.cumsum([len(x) for x in nbr])
    ex = np.array([j for x in nbr for j in sorted(x)], np.int32)
    r_max, nbins = 2.21 * A, 17
    h, _ = oracle.rdf(xyz, colour, box, r_max, nbins, off, ex)
    want = expected(r_max, nbins, {1: 2 * N, 2: 6 * N, 3: 4 * N, 4: 3 * N})
    assert np.array_equal(h, want)


def test_near_edge_counts():
    xyz, colour, box = lattice()
    # dr = a / 4: a and 2 a sit on edges 4 and 8 (the FP32 coordinates move
    # them by ~1e-7 nm to either side, so both neighbouring bins receive some)
    r_max, nbins = 2.25 * A, 9
    h, near = oracle.rdf(xyz, colour, box, r_max, nbins, delta=1e-6)
    want_near = np.zeros(nbins + 1, np.int64)
    want_near[4] = 3 * N
    want_near[8] = 3 * N
    assert np.array_equal(near, want_near)
    assert h.sum() == (6 + 12 + 8 + 6 + 24) * N // 2   # sqrt(5) a < 2.25 a: 24 neighbours more


def test_cells_match_brute_force_on_water():
    box = w.water_box(512, 2.48, seed=5)
    r_max, nbins = 1.2, 96
    for sel in ((-1, -1), (0, 0), (0, 1)):
        hc, nc = oracle.rdf(box.xyz, box.types, box.box, r_max, nbins, box.excl_off, box.excl_idx,
                            *sel, delta=2e-6)
        hb, nb = oracle.rdf(box.xyz, box.types, box.box, r_max, nbins, box.excl_off, box.excl_idx,
                            *sel, delta=2e-6, brute=True)
        assert np.array_equal(hc, hb) and np.array_equal(nc, nb)
    # all pairs, no exclusions: the total is the independent brute-force count
    h, _ = oracle.rdf(box.xyz, box.types, box.box, r_max, nbins)
    assert h.sum() == oracle.count_pairs_within(box.xyz, box.box, r_max)


def test_rejects_bad_arguments():
    xyz, colour, box = lattice()
    with pytest.raises(ValueError):
        oracle.rdf(xyz, colour, box, 1.6, 10)          # r_max above half the box
    with pytest.raises(ValueError):
        oracle.rdf(xyz, colour, box, 1.0, 10, delta=0.06)
