"""Seeded synthetic inputs shaped like the paper's water workloads.

This module only draws inputs: particle positions, charges, atom types,
per-type Lennard-Jones sigma/epsilon, force-field exclusions, masses and
per-frame thermal displacements.  It holds none of the method's arithmetic
(no gridding, no pair list, no interaction functions); both the CUDA path and
the FP64 oracle consume what it returns.

The paper measures on SPC/E-like 3-site water at 1 nm cut-off (Sec. 5,
Table 3; Fig. 3 uses a 3-site water model at number density 100 nm^-3).
No dataset is used; these boxes stand in for it.

Recipe (all FP64, rounded to FP32 at the end):
  * oxygen sites by random sequential addition (RSA) under periodic
    boundaries with a minimum O-O distance of 0.25 nm (candidates drawn from
    the seeded PCG64 stream, tested with a linked-cell list in gen_geom.c);
  * a uniform random orientation per molecule from a normalised 4-vector of
    standard normals (quaternion); O-H 0.1 nm, H-O-H 109.47 degrees;
  * a molecule whose hydrogen comes closer than 0.10 nm to a hydrogen of
    another molecule redraws its orientation (up to 100 rounds);
  * atom index 3*m + site (site 0 = O, 1 = H1, 2 = H2); charges O -0.82,
    H +0.41; LJ on O only (sigma 0.3166 nm, epsilon 0.650 kJ/mol);
  * exclusions: the three intramolecular pairs, listed both ways;
  * positions wrapped into [0, L) in FP64, then rounded to FP32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants used only to size thermal displacements.
KB_KJ_PER_MOL_K = 0.0083144626  # Boltzmann constant in kJ mol^-1 K^-1
MASS_O = 15.9994
MASS_H = 1.008

WATER_DENSITY_MOL_PER_NM3 = 33.43  # 1 g/cm^3 of water
OH_BOND_NM = 0.1
HOH_ANGLE_DEG = 109.47
Q_O = -0.82
Q_H = 0.41
SIGMA_O = 0.3166
EPS_O = 0.650
MIN_OO_NM = 0.25
MIN_HH_NM = 0.10

TYPE_O = 0
TYPE_H = 1


@dataclass
class Box:
    """One periodic box of particles (caller atom order)."""

    xyz: np.ndarray          # float32 [n, 3], wrapped into [0, L)
    q: np.ndarray            # float32 [n]
    types: np.ndarray        # int32 [n]
    sigma: np.ndarray        # float64 [ntypes]  per-type LJ sigma (nm)
    eps: np.ndarray          # float64 [ntypes]  per-type LJ epsilon (kJ/mol)
    mass: np.ndarray         # float64 [n]
    excl_off: np.ndarray     # int32 [n + 1]  CSR offsets of force-field exclusions
    excl_idx: np.ndarray     # int32 [nexcl]  excluded partner indices
    box: np.ndarray          # float64 [3]  edge lengths (nm)
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def ntypes(self) -> int:
        return int(self.sigma.shape[0])


def _uniform_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """k uniform random rotation matrices from normalised 4-normal quaternions."""
    qv = rng.standard_normal((k, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv[:, 0], qv[:, 1], qv[:, 2], qv[:, 3]
    r = np.empty((k, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def _h_offsets(rot: np.ndarray) -> np.ndarray:
    """Hydrogen offsets [k, 2, 3] from the oxygen for rotations rot [k, 3, 3]."""
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    local = np.array([[math.sin(half), math.cos(half), 0.0],
                      [-math.sin(half), math.cos(half), 0.0]]) * OH_BOND_NM
    return np.einsum("kab,hb->kha", rot, local)


def _cell_grid(L: np.ndarray, cell_min: float) -> np.ndarray:
    return np.maximum(1, np.floor(L / cell_min).astype(np.int64))


def _pairs_within_np(p: np.ndarray, L: np.ndarray, rcut: float):
    """All index pairs (i < j) with minimum-image distance < rcut (FP64).

    Generic geometry for input generation only (cell hashing with cells no
    smaller than rcut; needs rcut < L/3 per dimension for the 27-cell stencil
    to be free of duplicates, else falls back to all pairs).
    """
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    L = np.asarray(L, dtype=np.float64)
    nc = _cell_grid(L, rcut)
    if np.any(nc < 3) or n < 64:
        i, j = np.triu_indices(n, 1)
        d = p[i] - p[j]
        d -= L * np.round(d / L)
        keep = np.einsum("ij,ij->i", d, d) < rcut * rcut
        return i[keep], j[keep]
    c3 = np.minimum((p / (L / nc)).astype(np.int64), nc - 1)
    cid = (c3[:, 0] * nc[1] + c3[:, 1]) * nc[2] + c3[:, 2]
    order = np.argsort(cid, kind="stable")
    cid_sorted = cid[order]
    ncells = int(nc.prod())
    start = np.searchsorted(cid_sorted, np.arange(ncells + 1))
    cnt = start[1:] - start[:-1]
    maxocc = int(cnt.max())
    out_i, out_j = [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                nb = (((c3[:, 0] + ox) % nc[0]) * nc[1] + (c3[:, 1] + oy) % nc[1]) * nc[2] \
                    + (c3[:, 2] + oz) % nc[2]
                s = start[nb]
                m = cnt[nb]
                for k in range(maxocc):
                    valid = np.nonzero(k < m)[0]
                    jj = order[s[valid] + k]
                    ii = valid
                    keep = ii < jj
                    ii, jj = ii[keep], jj[keep]
                    d = p[ii] - p[jj]
                    d -= L * np.round(d / L)
                    close = np.einsum("ij,ij->i", d, d) < rcut * rcut
                    out_i.append(ii[close])
                    out_j.append(jj[close])
    i = np.concatenate(out_i) if out_i else np.zeros(0, np.int64)
    j = np.concatenate(out_j) if out_j else np.zeros(0, np.int64)
    return i, j


_geom = None


def _geom_lib():
    """The C geometry helper (gen_geom.c), built with gcc on first use."""
    global _geom
    if _geom is not None:
        return _geom
    import ctypes as C
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(here, "gen_geom.c")
    out = os.path.join(here, "_build", "libgengeom.so")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, out)
    lib = C.CDLL(out)
    P = C.c_void_p
    lib.gen_rsa_fill.argtypes = [P, C.c_double, P, P, P, P, P, C.c_int64, P, C.c_int64]
    lib.gen_rsa_fill.restype = C.c_int64
    lib.gen_close_pairs.argtypes = [P, C.c_double, C.c_int64, P, C.c_int64, P, P]
    lib.gen_close_pairs.restype = C.c_int64
    _geom = lib
    return lib


def pairs_within(p: np.ndarray, L: np.ndarray, rcut: float):
    """All index pairs (i < j) with minimum-image distance < rcut (FP64)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    if np.any(np.floor(L / rcut) < 3) or p.shape[0] < 64:
        return _pairs_within_np(p, L, rcut)
    lib = _geom_lib()
    cap = max(1024, 4 * p.shape[0])
    while True:
        oi = np.empty(cap, np.int64)
        oj = np.empty(cap, np.int64)
        n = lib.gen_close_pairs(L.ctypes.data, float(rcut), p.shape[0], p.ctypes.data, cap,
                                oi.ctypes.data, oj.ctypes.data)
        if n <= cap:
            return oi[:n], oj[:n]
        cap = int(n)


def rsa_points(n: int, L: np.ndarray, dmin: float, rng: np.random.Generator) -> np.ndarray:
    """n points in the periodic box L with pairwise minimum-image distance >= dmin.

    Random sequential addition: uniform candidates (drawn from rng in chunks)
    are accepted in order when no accepted point is closer than dmin.
    """
    import ctypes as C
    L = np.ascontiguousarray(L, dtype=np.float64)
    lib = _geom_lib()
    nc = np.maximum(1, np.floor(L / dmin)).astype(np.int32)
    head = np.full(int(np.prod(nc.astype(np.int64))), -1, np.int32)
    nxt = np.empty(max(n, 1), np.int32)
    pts = np.empty((max(n, 1), 3))
    npts = C.c_int64(0)
    while npts.value < n:
        chunk = max(4096, 4 * (n - npts.value))
        cand = np.ascontiguousarray(rng.random((chunk, 3)) * L)
        lib.gen_rsa_fill(L.ctypes.data, float(dmin), nc.ctypes.data, head.ctypes.data, nxt.ctypes.data,
                         pts.ctypes.data, C.byref(npts), n, cand.ctypes.data, chunk)
    return pts[:n].copy()


def water_box(n_mol: int, L: float | None = None, seed: int = 0,
              retype_frac: float = 0.0, n_extra_types: int = 0) -> Box:
    """A water-like box of n_mol 3-site molecules (see the module recipe).

    retype_frac > 0 picks that fraction of molecules (seeded) and re-types
    each of their sites uniformly among n_extra_types extra LJ types with
    sigma_k = 0.25 + 0.15 k/(n-1) nm and epsilon_k = 0.1 + 0.9 k/(n-1) kJ/mol
    (charges unchanged).
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    if L is None:
        L = (n_mol / WATER_DENSITY_MOL_PER_NM3) ** (1.0 / 3.0)
    Lv = np.array([L, L, L], dtype=np.float64)
    oxy = rsa_points(n_mol, Lv, MIN_OO_NM, rng)
    rot = _uniform_rotations(rng, n_mol)
    hoff = _h_offsets(rot)

    # redraw orientations with intermolecular H-H contacts below MIN_HH_NM
    min_hh = None
    for _ in range(100):
        hpos = (oxy[:, None, :] + hoff).reshape(-1, 3)
        i, j = pairs_within(hpos, Lv, MIN_HH_NM)
        inter = (i // 2) != (j // 2)
        i, j = i[inter], j[inter]
        if i.size == 0:
            break
        redo = np.unique(np.maximum(i // 2, j // 2))
        hoff[redo] = _h_offsets(_uniform_rotations(rng, redo.size))
    hpos = (oxy[:, None, :] + hoff).reshape(-1, 3)
    i, j = pairs_within(hpos, Lv, MIN_HH_NM)
    inter = (i // 2) != (j // 2)
    n_hh_close = int(inter.sum())

    n = 3 * n_mol
    xyz = np.empty((n_mol, 3, 3))
    xyz[:, 0] = oxy
    xyz[:, 1:] = oxy[:, None, :] + hoff
    xyz = xyz.reshape(n, 3)
    xyz = xyz - Lv * np.floor(xyz / Lv)
    xyz32 = xyz.astype(np.float32)
    # FP32 rounding can land exactly on L; fold those back to 0
    for d in range(3):
        col = xyz32[:, d]
        col[col >= np.float32(Lv[d])] = np.float32(0.0)

    q = np.tile(np.array([Q_O, Q_H, Q_H], dtype=np.float32), n_mol)
    types = np.tile(np.array([TYPE_O, TYPE_H, TYPE_H], dtype=np.int32), n_mol)
    sigma = [SIGMA_O, 0.0]
    eps = [EPS_O, 0.0]
    if n_extra_types > 0:
        for k in range(n_extra_types):
            f = k / max(n_extra_types - 1, 1)
            sigma.append(0.25 + 0.15 * f)
            eps.append(0.1 + 0.9 * f)
    if retype_frac > 0.0 and n_extra_types > 0:
        n_re = int(round(retype_frac * n_mol))
        mols = rng.choice(n_mol, size=n_re, replace=False)
        newt = rng.integers(0, n_extra_types, size=(n_re, 3)) + 2
        t3 = types.reshape(n_mol, 3)
        t3[mols] = newt.astype(np.int32)
        types = t3.reshape(n)
    mass = np.tile(np.array([MASS_O, MASS_H, MASS_H]), n_mol)

    # exclusions: each atom excludes the other two sites of its molecule
    excl_off = (np.arange(n + 1, dtype=np.int64) * 2).astype(np.int32)
    base = (np.arange(n) // 3) * 3
    site = np.arange(n) % 3
    other = np.stack([base + (site + 1) % 3, base + (site + 2) % 3], axis=1)
    other.sort(axis=1)
    excl_idx = other.reshape(-1).astype(np.int32)

    return Box(xyz=xyz32, q=q, types=types, sigma=np.array(sigma), eps=np.array(eps),
               mass=mass, excl_off=excl_off, excl_idx=excl_idx, box=Lv.copy(), seed=seed,
               meta={"n_mol": n_mol, "n_hh_close": n_hh_close})


def thermal_sigma(mass: np.ndarray, T: float = 300.0, dt: float = 0.002) -> np.ndarray:
    """Per-atom displacement standard deviation sqrt(kB T / m) * dt (nm)."""
    return np.sqrt(KB_KJ_PER_MOL_K * T / np.asarray(mass)) * dt


def frame_displacements(mass: np.ndarray, n_frames: int, seed: int,
                        T: float = 300.0, dt: float = 0.002) -> np.ndarray:
    """Independent Gaussian increments [n_frames, n, 3] (float32).

    Frame f's coordinates are the frame-0 coordinates plus the running sum of
    the first f increments (a random walk with per-step sigma sqrt(kT/m) dt).
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    s = thermal_sigma(mass, T, dt)
    d = rng.standard_normal((n_frames, mass.shape[0], 3)) * s[None, :, None]
    return d.astype(np.float32)


# ---------------------------------------------------------------------------
# The configurations (seed = 1000 + configuration index)

def config1() -> tuple[Box, dict]:
    """512 molecules (1,536 atoms), L = 2.48 nm, reaction field eps_rf = inf,
    rc 0.9 nm, rlist 1.0 nm; one list build and one force/energy evaluation."""
    b = water_box(512, 2.48, seed=1001)
    return b, {"elec": "rf", "rc": 0.9, "rlist": 1.0, "eps_rf": math.inf}


def config2() -> tuple[Box, dict]:
    """8,000 molecules (24,000 atoms), L = 6.21 nm, Ewald real space beta
    3.12 nm^-1, rc 1.0 nm, rlist 1.1 nm, 20 frames, prune every 5 frames."""
    b = water_box(8000, 6.21, seed=1002)
    return b, {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12,
               "nstlist": 20, "nstprune": 5}


def config3() -> tuple[Box, dict]:
    """1,000,000 molecules (3M atoms), L = 31.0 nm, same Ewald/LJ parameters,
    rlist 1.1 nm, nstlist 40, prune every 5; 10% of molecules re-typed among
    8 extra LJ types combined by Lorentz-Berthelot."""
    b = water_box(1_000_000, 31.0, seed=1003, retype_frac=0.1, n_extra_types=8)
    return b, {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12,
               "nstlist": 40, "nstprune": 5, "comb": "lb"}


def batch_sizes(n_boxes: int = 256, seed: int = 1004) -> np.ndarray:
    """Atom counts 3*round(exp(U(ln 1500, ln 60000))/3) for the batch of boxes."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    u = rng.uniform(math.log(1500.0), math.log(60000.0), size=n_boxes)
    return (3 * np.round(np.exp(u) / 3)).astype(np.int64)


def prune_radius(rc: float, rlist: float, nstprune: int, T: float = 300.0,
                 dt: float = 0.002, m_fast: float = MASS_H) -> float:
    """Inner (pruned) list radius: rc plus six standard deviations of the
    relative displacement of two hydrogens over nstprune steps, capped at
    rlist.  The paper prunes close to the cut-off without giving the radius."""
    s_pair = math.sqrt(2.0) * math.sqrt(KB_KJ_PER_MOL_K * T / m_fast) * dt * math.sqrt(nstprune)
    return rc + max(0.0, min(rlist - rc, 6.0 * s_pair))


@dataclass
class Batch:
    """Independent periodic boxes handled together.  Particle arrays are the
    boxes' arrays concatenated in box order; exclusion partner indices are
    shifted to batch-global indices.  All boxes share one LJ type table."""

    xyz: np.ndarray          # float32 [n, 3]
    q: np.ndarray            # float32 [n]
    types: np.ndarray        # int32 [n]
    sigma: np.ndarray        # float64 [ntypes]
    eps: np.ndarray          # float64 [ntypes]
    mass: np.ndarray         # float64 [n]
    excl_off: np.ndarray     # int32 [n + 1]
    excl_idx: np.ndarray     # int32 [nexcl], batch-global
    counts: np.ndarray       # int64 [nbox] particles per box
    boxes: np.ndarray        # float64 [nbox, 3] edge lengths
    members: list = field(default_factory=list)  # the Box of each box

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nbox(self) -> int:
        return int(self.counts.shape[0])

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)


def concat(boxes: list) -> Batch:
    """Concatenate boxes that share one LJ type table into a Batch."""
    if not boxes:
        raise ValueError("no boxes")
    s0, e0 = boxes[0].sigma, boxes[0].eps
    for b in boxes:
        if b.sigma.shape != s0.shape or not (np.array_equal(b.sigma, s0) and np.array_equal(b.eps, e0)):
            raise ValueError("boxes of a batch must share the LJ type table")
    counts = np.array([b.n for b in boxes], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(counts)])
    eo, ei = [np.zeros(1, np.int64)], []
    base_e = 0
    for k, b in enumerate(boxes):
        eo.append(b.excl_off[1:].astype(np.int64) + base_e)
        ei.append(b.excl_idx.astype(np.int64) + off[k])
        base_e += int(b.excl_off[-1])
    return Batch(xyz=np.concatenate([b.xyz for b in boxes]).astype(np.float32),
                 q=np.concatenate([b.q for b in boxes]).astype(np.float32),
                 types=np.concatenate([b.types for b in boxes]).astype(np.int32),
                 sigma=s0.copy(), eps=e0.copy(),
                 mass=np.concatenate([b.mass for b in boxes]),
                 excl_off=np.concatenate(eo).astype(np.int32),
                 excl_idx=(np.concatenate(ei) if ei else np.zeros(0)).astype(np.int32),
                 counts=counts, boxes=np.stack([b.box for b in boxes]), members=list(boxes))


def batch_boxes(n_boxes: int = 256, seed: int = 1004) -> Batch:
    """The batch of uneven water boxes: box k holds batch_sizes()[k] atoms
    (a whole number of molecules) at water density, drawn with seed
    seed * 1000 + k."""
    sizes = batch_sizes(n_boxes, seed)
    return concat([water_box(int(n) // 3, None, seed=seed * 1000 + k) for k, n in enumerate(sizes)])


def frame_walk(xyz: np.ndarray, mass: np.ndarray, n_frames: int, seed: int,
               T: float = 300.0, dt: float = 0.002):
    """Yield n_frames coordinate frames (float32 [n, 3]): frame 0 is xyz and
    each later frame adds one Gaussian increment per coordinate with sigma
    sqrt(kT/m) dt to the previous one (the random walk of frame_displacements,
    drawn one frame at a time to bound host memory)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    s = thermal_sigma(mass, T, dt).astype(np.float32)[:, None]
    x = np.array(xyz, dtype=np.float32, copy=True)
    yield x.copy()
    for _ in range(n_frames - 1):
        x += rng.standard_normal(x.shape, dtype=np.float32) * s
        yield x.copy()


def surrogate_samples(n: int = 1 << 20, r_min: float = 0.05, r_max: float = 1.0,
                      seed: int = 1005) -> np.ndarray:
    """Training distances for the Ewald-factor network: n draws of
    U[r_min, r_max] nm (FP64, seeded)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return rng.uniform(r_min, r_max, size=n)
