"""FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It builds ``oracle.c`` with gcc into
``oracle/_build/liboracle.so`` and wraps it with ctypes.  It shares no code
with the CUDA library and never imports it.

Functions (each follows the paper passage cited in ``oracle.c``):
  forces_brute   -- Tier A: O(N^2) minimum-image pair loop (Sec. 3.2 interactions)
  forces_cells   -- Tier B: the same through a cell list (linear cost)
  pair           -- one pair interaction (Sec. 3.2)
  grid           -- spatial clustering into columns and clusters (Sec. 2.3)
  pairlist       -- cluster-pair search by brute force over all cluster
                    pairs and shifts, with exclusion masks (Sec. 2.3, 2.4)
  prune          -- particle-pair distance pruning (Sec. 2.3)
  ewald_factor   -- the Ewald real-space force factor c(r) (Sec. 3.2)
  mlp_forward    -- the 1-32-32-1 SiLU network that may stand in for c(r)
  mlp_loss_grad  -- its weighted squared-error loss and parameter gradient
  buffer_drift_integral -- the Appendix's Verlet-buffer drift integral, by quadrature
  rdf            -- pair-distance histogram (pair correlation; Sec. 1, Sec. 2.3)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

ELEC_RF = 0
ELEC_EWALD = 1
COMB_LB = 0
COMB_GEOM = 1
FCOUL = 138.935458
SHIFT_CENTER = 13


class Params(C.Structure):
    _fields_ = [("elec", C.c_int), ("comb", C.c_int), ("rc", C.c_double),
                ("eps_rf", C.c_double), ("beta", C.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            i64 = C.c_int64
            L.or_num_threads.restype = C.c_int
            L.or_pair.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
            L.or_lj_pair_params.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_forces_brute.argtypes = [C.c_int, P, P, P, C.c_int, P, P, P, P, P,
                                          C.POINTER(Params), C.c_int, P, P, P, P]
            L.or_forces_brute.restype = C.c_int
            L.or_forces_cells.argtypes = L.or_forces_brute.argtypes
            L.or_forces_cells.restype = C.c_int
            L.or_count_pairs_within.argtypes = [C.c_int, P, P, C.c_double]
            L.or_count_pairs_within.restype = i64
            L.or_grid_dims.argtypes = [C.c_int, P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(i64)]
            L.or_dummy_spacing.argtypes = [P]
            L.or_dummy_spacing.restype = C.c_float
            L.or_grid.argtypes = [C.c_int, P, P, P, P, C.c_int, P, P, P, P, P, P, P, P]
            L.or_grid.restype = i64
            L.or_slot_coords.argtypes = [i64, P, P, P, P, P, P]
            L.or_pairlist.argtypes = [i64, C.c_int, P, P, P, P, C.c_double, C.c_double, P, P, i64,
                                      P, P, P, P]
            L.or_pairlist.restype = i64
            L.or_pairlist_cluster.argtypes = [i64, C.c_int, P, P, P, P, C.c_double, C.c_double, P, P,
                                              i64, i64, P, P, P, P]
            L.or_pairlist_cluster.restype = i64
            L.or_mask.argtypes = [C.c_int, P, P, P, i64, i64, C.c_int]
            L.or_mask.restype = C.c_uint64
            L.or_key_distances.argtypes = [C.c_int, P, P, P, P, i64, P, P, P, P, P]
            L.or_prune.argtypes = [C.c_int, P, P, P, C.c_double, i64, P, P, P, P, P]
            L.or_pair_cover.argtypes = [C.c_int, P, P, C.c_double, C.c_int, P, P, i64, P, P, P, P]
            L.or_ewald_factor.argtypes = [i64, P, C.c_double, P]
            L.or_mlp_forward.argtypes = [P, C.c_double, C.c_double, i64, P, P]
            L.or_mlp_loss_grad.argtypes = [P, C.c_double, C.c_double, i64, P, P, P, P]
            L.or_mlp_loss_grad.restype = C.c_double
            L.or_buffer_drift_integral.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            L.or_buffer_drift_integral.restype = C.c_double
            L.or_rdf.argtypes = [C.c_int, P, P, P, P, P, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_int, P, P]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(elec: str, rc: float, eps_rf: float = math.inf, beta: float = 0.0,
                comb: str = "lb") -> Params:
    return Params(ELEC_RF if elec == "rf" else ELEC_EWALD,
                  COMB_LB if comb == "lb" else COMB_GEOM,
                  float(rc), -1.0 if math.isinf(eps_rf) else float(eps_rf), float(beta))


def num_threads() -> int:
    return int(lib().or_num_threads())


def pair(params: Params, r: float, qq: float, c6: float, c12: float, excluded: bool = False):
    """(F/r, V_LJ, V_Coulomb) of one pair at distance r."""
    fs, vl, vc = C.c_double(), C.c_double(), C.c_double()
    lib().or_pair(C.byref(params), float(r), float(qq), float(c6), float(c12), int(excluded),
                  C.byref(fs), C.byref(vl), C.byref(vc))
    return fs.value, vl.value, vc.value


def lj_pair_params(comb: str, si: float, ei: float, sj: float, ej: float):
    c6, c12 = C.c_double(), C.c_double()
    lib().or_lj_pair_params(COMB_LB if comb == "lb" else COMB_GEOM, si, ei, sj, ej,
                            C.byref(c6), C.byref(c12))
    return c6.value, c12.value


def _forces(fn, xyz, q, types, sigma, eps, excl_off, excl_idx, box, params, sel, exact):
    if exact:
        xyz = _f64(xyz)
        box64 = _f64(box)
    else:
        xyz = _f32(xyz).astype(np.float64)
        box64 = _f32(box).astype(np.float64)
    n = xyz.shape[0]
    q = _f32(q)
    types = _i32(types)
    sigma = _f64(sigma)
    eps = _f64(eps)
    eo = _i32(excl_off) if excl_off is not None else None
    ei = _i32(excl_idx) if excl_idx is not None else None
    if sel is None:
        f = np.zeros((n, 3))
        e = np.zeros(2)
        vir = np.zeros(9)
        rc = fn(n, _p(xyz), _p(q), _p(types), sigma.shape[0], _p(sigma), _p(eps), _p(eo), _p(ei), _p(box64),
                C.byref(params), 0, None, _p(f), _p(e), _p(vir))
        if rc != 0:
            raise ValueError("cut-off must be below half the box")
        return f, e, vir.reshape(3, 3)
    sel = _i32(sel)
    f = np.zeros((sel.shape[0], 3))
    rc = fn(n, _p(xyz), _p(q), _p(types), sigma.shape[0], _p(sigma), _p(eps), _p(eo), _p(ei), _p(box64),
            C.byref(params), sel.shape[0], _p(sel), _p(f), None, None)
    if rc != 0:
        raise ValueError("cut-off must be below half the box")
    return f, None, None


def forces_brute(xyz, q, types, sigma, eps, excl_off, excl_idx, box, params: Params,
                 sel=None, exact: bool = False):
    """Tier A: brute-force FP64 forces [n or len(sel), 3], energies [2],
    virial [3, 3] (with sel: the selected particles' forces only).

    By default xyz and box are rounded to FP32 first (the precision the
    kernels receive) and promoted to FP64; exact=True passes FP64 values
    through unchanged (finite-difference checks).
    """
    return _forces(lib().or_forces_brute, xyz, q, types, sigma, eps, excl_off, excl_idx, box, params, sel,
                   exact)


def forces_cells(xyz, q, types, sigma, eps, excl_off, excl_idx, box, params: Params,
                 sel=None, exact: bool = False):
    """Tier B: the same quantities through an FP64 cell list (cost linear in
    the number of particles)."""
    return _forces(lib().or_forces_cells, xyz, q, types, sigma, eps, excl_off, excl_idx, box, params, sel,
                   exact)


def count_pairs_within(xyz, box, r: float) -> int:
    xyz = _f32(xyz).astype(np.float64)
    box64 = _f32(box).astype(np.float64)
    return int(lib().or_count_pairs_within(xyz.shape[0], _p(xyz), _p(box64), float(r)))


def grid_dims(n: int, box, C_: int):
    nx, ny, npm = C.c_int(), C.c_int(), C.c_int64()
    lib().or_grid_dims(int(n), _p(_f32(box)), int(C_), C.byref(nx), C.byref(ny), C.byref(npm))
    return nx.value, ny.value, npm.value


def dummy_spacing(box) -> float:
    return float(lib().or_dummy_spacing(_p(_f32(box))))


class Grid:
    """Canonical grid (Sec. 2.3) of one box."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def grid(xyz, q, types, box, C_: int = 8) -> Grid:
    xyz = _f32(xyz)
    n = xyz.shape[0]
    q = _f32(q)
    types = _i32(types)
    box32 = _f32(box)
    nx, ny, npm = grid_dims(n, box32, C_)
    wrapped = np.zeros((n, 3), np.float32)
    col_of_atom = np.zeros(n, np.int32)
    col_clu_start = np.zeros(nx * ny + 1, np.int32)
    atom_of_slot = np.full(npm, -2, np.int32)
    slot_of_atom = np.zeros(n, np.int32)
    xyzq = np.zeros((npm, 4), np.float32)
    type_slot = np.zeros(npm, np.int32)
    bb = np.zeros((max(npm // C_ + 1, 1), 6), np.float32)
    nclu = lib().or_grid(n, _p(xyz), _p(q), _p(types), _p(box32), int(C_), _p(wrapped),
                         _p(col_of_atom), _p(col_clu_start), _p(atom_of_slot), _p(slot_of_atom),
                         _p(xyzq), _p(type_slot), _p(bb))
    if nclu < 0:
        raise ValueError("coordinate outside [-L, 2L)")
    ns = nclu * C_
    return Grid(n=n, C=C_, nx=nx, ny=ny, nclu=int(nclu), box=box32, xyz_grid=xyz.copy(),
                wrapped=wrapped, col_of_atom=col_of_atom, col_clu_start=col_clu_start,
                atom_of_slot=atom_of_slot[:ns].copy(), slot_of_atom=slot_of_atom,
                xyzq=xyzq[:ns].copy(), type_slot=type_slot[:ns].copy(), bb=bb[:nclu].copy())


def slot_coords(g: Grid, xyz_new) -> np.ndarray:
    """Slot coordinates [nslots, 4] of a later frame (wrap offset kept)."""
    xyz_new = _f32(xyz_new)
    out = np.zeros_like(g.xyzq)
    lib().or_slot_coords(g.atom_of_slot.shape[0], _p(g.atom_of_slot), _p(xyz_new), _p(g.xyz_grid),
                         _p(g.wrapped), _p(g.xyzq), _p(out))
    return out


class PairList:
    def __init__(self, a, b, s, mask):
        self.a, self.b, self.s, self.mask = a, b, s, mask

    def __len__(self):
        return int(self.a.shape[0])

    def keys(self):
        return set(zip(self.a.tolist(), self.b.tolist(), self.s.tolist()))

    def key_mask(self):
        return dict(zip(zip(self.a.tolist(), self.b.tolist(), self.s.tolist()), self.mask.tolist()))


def pairlist(g: Grid, rlist: float, rbb: float = 0.0, excl_off=None, excl_idx=None,
             xyzq=None) -> PairList:
    """Full canonical cluster-pair list (brute force over all cluster pairs)."""
    xyzq = g.xyzq if xyzq is None else _f32(xyzq)
    eo = _i32(excl_off) if excl_off is not None else None
    ei = _i32(excl_idx) if excl_idx is not None else None
    args = (g.nclu, g.C, _p(xyzq), _p(g.atom_of_slot), _p(g.bb), _p(g.box), float(rlist), float(rbb),
            _p(eo), _p(ei))
    total = lib().or_pairlist(*args, 0, None, None, None, None)
    if total < 0:
        raise ValueError("rlist must be below half the box")
    a = np.zeros(total, np.int32)
    b = np.zeros(total, np.int32)
    s = np.zeros(total, np.int32)
    m = np.zeros(total, np.uint64)
    lib().or_pairlist(*args, total, _p(a), _p(b), _p(s), _p(m))
    return PairList(a, b, s, m)


def pairlist_cluster(g: Grid, c: int, rlist: float, rbb: float = 0.0, excl_off=None,
                     excl_idx=None) -> PairList:
    """Canonical keys that involve cluster c (sampled checks on large boxes)."""
    eo = _i32(excl_off) if excl_off is not None else None
    ei = _i32(excl_idx) if excl_idx is not None else None
    args = (g.nclu, g.C, _p(g.xyzq), _p(g.atom_of_slot), _p(g.bb), _p(g.box), float(rlist),
            float(rbb), _p(eo), _p(ei), int(c))
    total = lib().or_pairlist_cluster(*args, 0, None, None, None, None)
    a = np.zeros(total, np.int32)
    b = np.zeros(total, np.int32)
    s = np.zeros(total, np.int32)
    m = np.zeros(total, np.uint64)
    lib().or_pairlist_cluster(*args, total, _p(a), _p(b), _p(s), _p(m))
    return PairList(a, b, s, m)


def mask(g: Grid, a: int, b: int, s: int, excl_off, excl_idx) -> int:
    return int(lib().or_mask(g.C, _p(g.atom_of_slot), _p(_i32(excl_off)), _p(_i32(excl_idx)),
                             int(a), int(b), int(s)))


def key_distances(g: Grid, a, b, s, xyzq=None):
    """(min FP64 particle distance, FP64 bounding-box distance) per key."""
    xyzq = g.xyzq if xyzq is None else _f32(xyzq)
    a, b, s = _i32(a), _i32(b), _i32(s)
    dm = np.zeros(a.shape[0])
    db = np.zeros(a.shape[0])
    lib().or_key_distances(g.C, _p(xyzq), _p(g.atom_of_slot), _p(g.bb), _p(g.box), a.shape[0],
                           _p(a), _p(b), _p(s), _p(dm), _p(db))
    return dm, db


def prune(g: Grid, pl: PairList, r_prune: float, xyzq=None):
    """(keep flags, minimum counted-pair distance) per key of pl."""
    xyzq = g.xyzq if xyzq is None else _f32(xyzq)
    k = len(pl)
    keep = np.zeros(k, np.uint8)
    dmin = np.zeros(k)
    lib().or_prune(g.C, _p(xyzq), _p(g.atom_of_slot), _p(g.box), float(r_prune), k,
                   _p(_i32(pl.a)), _p(_i32(pl.b)), _p(_i32(pl.s)), _p(keep), _p(dmin))
    return keep.astype(bool), dmin


def pair_cover(g: Grid, pl: PairList, r: float):
    """(pairs within r covered once, not covered, covered more than once)."""
    cov = np.zeros(3, np.int64)
    lib().or_pair_cover(g.n, _p(g.wrapped), _p(g.box), float(r), g.C, _p(g.atom_of_slot),
                        _p(g.slot_of_atom), len(pl), _p(_i32(pl.a)), _p(_i32(pl.b)),
                        _p(_i32(pl.s)), _p(cov))
    return tuple(int(v) for v in cov)


def shift_index_to_vec(s: int):
    return (s // 9 - 1, (s // 3) % 3 - 1, s % 3 - 1)


MLP_HIDDEN = 32
MLP_NPARAMS = 32 + 32 + 32 * 32 + 32 + 32 + 1


def ewald_factor(r, beta: float) -> np.ndarray:
    """c(r) = erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2), FP64."""
    r = _f64(r).reshape(-1)
    out = np.empty_like(r)
    lib().or_ewald_factor(r.size, _p(r), float(beta), _p(out))
    return out


def mlp_forward(params, r_min: float, r_max: float, r) -> np.ndarray:
    p = _f64(params).reshape(-1)
    assert p.size == MLP_NPARAMS
    r = _f64(r).reshape(-1)
    y = np.empty_like(r)
    lib().or_mlp_forward(_p(p), float(r_min), float(r_max), r.size, _p(r), _p(y))
    return y


def mlp_loss_grad(params, r_min: float, r_max: float, r, t, w=None):
    """(loss, gradient [1153]) of (1/n) sum w (y(r) - t)^2."""
    p = _f64(params).reshape(-1)
    assert p.size == MLP_NPARAMS
    r = _f64(r).reshape(-1)
    t = _f64(t).reshape(-1)
    wv = None if w is None else _f64(w).reshape(-1)
    g = np.empty(MLP_NPARAMS)
    loss = lib().or_mlp_loss_grad(_p(p), float(r_min), float(r_max), r.size, _p(r), _p(t), _p(wv), _p(g))
    return float(loss), g


def buffer_drift_integral(v1: float, v2: float, rb: float, sigma: float) -> float:
    """The Appendix's double integral of [V'(rc)(rt - rc) + V''(rc)(rt - rc)^2/2]
    over rt < rc, r0 > rc + rb with a Gaussian of width sigma in rt - r0."""
    return float(lib().or_buffer_drift_integral(float(v1), float(v2), float(rb), float(sigma)))


def rdf(xyz, types, box, r_max: float, nbins: int, excl_off=None, excl_idx=None, type_a: int = -1,
        type_b: int = -1, delta: float = 0.0, brute: bool = False):
    """(hist int64 [nbins], near int64 [nbins + 1]): counts of selected
    unordered pairs per distance bin of width r_max / nbins (FP64 minimum-image
    distances of the FP32 coordinates), and per bin edge the selected pairs
    within delta of it.  Force-field-excluded pairs are not counted."""
    xyz = _f32(xyz).astype(np.float64).reshape(-1, 3)
    t = _i32(types)
    box64 = _f32(box).astype(np.float64)
    eo = None if excl_off is None else _i32(excl_off)
    ei = None if excl_idx is None else _i32(excl_idx)
    if ei is not None and ei.size == 0:
        ei = np.zeros(1, np.int32)
    hist = np.zeros(int(nbins), np.int64)
    near = np.zeros(int(nbins) + 1, np.int64)
    rc = lib().or_rdf(xyz.shape[0], _p(xyz), _p(t), _p(eo), _p(ei), _p(box64), float(r_max), int(nbins),
                      int(type_a), int(type_b), float(delta), 1 if brute else 0, _p(hist), _p(near))
    if rc != 0:
        raise ValueError("rdf: r_max + delta must be below half the box, nbins >= 1, delta < dr / 2")
    return hist, near
