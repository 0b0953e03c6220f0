"""Python binding of libnbcluster (the C ABI in include/nbcluster.h).

Argument marshalling only: every function forwards to the C entry point of
the same name; device arrays are torch CUDA tensors (their data_ptr is
passed), streams default to torch's current stream.  All the computation runs
in the library's CUDA kernels; there is no CPU fallback.  If the library has
not been built (``__graft_entry__.build()`` or ``python -m
paper_1306_1737_gb300.build``), loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnbcluster.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "nbcluster.h")

NB_OK = 0
NB_ERR_ARG = 1
NB_ERR_BOX = 2
NB_ERR_CAPACITY = 3
NB_ERR_CUDA = 4
NB_ERR_STATE = 5
NB_ERR_TIMEOUT = 6
NB_ERR_COORD = 7

NB_ELEC_RF = 0
NB_ELEC_EWALD = 1
NB_ELEC_EWALD_MLP = 2
NB_ELEC_EWALD_TAB = 3
NB_MLP_NPARAMS = 1153
NB_COMB_LB = 0
NB_COMB_GEOM = 1

NB_KERNEL_GRID = 0
NB_KERNEL_SEARCH = 1
NB_KERNEL_PRUNE = 2
NB_KERNEL_FORCE = 3
NB_KERNEL_FORCE_1X1 = 4
NB_KERNEL_RDF = 5
NB_KERNEL_FORCE_PRUNE = 6
NB_KERNEL_FINALIZE = 7
NB_KERNEL_COORDS = 8
NB_RDF_MAX_BINS = 2048

_lock = threading.Lock()
_lib = None


class nb_options(C.Structure):
    _fields_ = [("cluster_size", C.c_int), ("device", C.c_int)]


class nb_params(C.Structure):
    _fields_ = [("elec", C.c_int), ("want_energy", C.c_int), ("rc", C.c_float),
                ("eps_rf", C.c_float), ("beta", C.c_float)]


class nb_info(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("n_clusters", C.c_int),
                ("n_ientries", C.c_int64), ("n_jentries", C.c_int64),
                ("n_jentries_pruned", C.c_int64), ("ient_capacity", C.c_int64),
                ("jent_capacity", C.c_int64), ("n_pairs_rc", C.c_int64),
                ("n_cluster_pairs", C.c_int64), ("n_cluster_pairs_pruned", C.c_int64),
                ("n_superclusters", C.c_int), ("super_size", C.c_int), ("n_launches", C.c_int64),
                ("flags", C.c_uint32), ("n_boxes", C.c_int), ("atom_offset", C.c_int)]


class nb_frames(C.Structure):
    _fields_ = [("n_frames", C.c_int), ("n_atoms", C.c_int), ("n_boxes", C.c_int),
                ("x_host", C.c_void_p), ("f_host", C.c_void_p), ("energy_frames_host", C.c_void_p),
                ("e_host", C.c_void_p), ("vir_host", C.c_void_p),
                ("x_dev", C.c_void_p * 2), ("f_dev", C.c_void_p * 2), ("e_dev", C.c_void_p * 2),
                ("vir_dev", C.c_void_p * 2), ("build", C.c_int), ("boxes_host", C.c_void_p),
                ("rlist", C.c_float), ("rbb", C.c_float), ("excl_off_dev", C.c_void_p),
                ("excl_idx_dev", C.c_void_p), ("first_frame", C.c_int), ("nstprune", C.c_int),
                ("r_prune", C.c_float)]


class nb_particle_class(C.Structure):
    _fields_ = [("count", C.c_double), ("mass", C.c_double), ("charge", C.c_double), ("type", C.c_int)]


class NbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def load():
    """Load libnbcluster.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1306_1737_gb300.build)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        i = C.c_int
        st = C.c_int
        sig = {
            "nb_create": ([C.POINTER(P), C.POINTER(nb_options)], st),
            "nb_destroy": ([P], st),
            "nb_last_error": ([P], C.c_char_p),
            "nb_status_string": ([i], C.c_char_p),
            "nb_lj_combine": ([i, P, P, i, P], st),
            "nb_workspace_query": ([P, i, P, C.c_double, i, C.c_double, C.POINTER(C.c_size_t)], st),
            "nb_workspace_query_boxes": ([P, i, P, P, C.c_double, i, C.c_double,
                                          C.POINTER(C.c_size_t)], st),
            "nb_workspace_bytes": ([i, i, P, P, C.c_double, i, C.c_double, C.POINTER(C.c_size_t)], st),
            "nb_set_workspace": ([P, P, C.c_size_t], st),
            "nb_set_atoms": ([P, i, P, P, i, P, P], st),
            "nb_grid_put": ([P, P, P, P], st),
            "nb_pairlist_build": ([P, C.c_float, C.c_float, P, P, P], st),
            "nb_set_coords": ([P, P, P], st),
            "nb_prune": ([P, P, C.c_float, P], st),
            "nb_compute": ([P, C.POINTER(nb_params), P, P, P, P, P], st),
            "nb_check": ([P, P, C.POINTER(nb_info)], st),
            "nb_box_info": ([P, i, C.POINTER(nb_info)], st),
            "nb_get_grid": ([P, P, P, P, P, P, P, P, P, P], st),
            "nb_get_list": ([P, i, P, P, P, P], st),
            "nb_profile": ([P, i], st),
            "nb_profile_read": ([P, P, P, i, C.POINTER(C.c_int)], st),
            "nb_grid_put_noalloc": ([i, P, P, P, i, P, i, P, P, P, P, P, P, i, i, P], st),
            "nb_ewald_factor": ([P, C.c_int64, C.c_double, P, P], st),
            "nb_mlp_forward": ([P, C.c_float, C.c_float, P, C.c_int64, P, P], st),
            "nb_mlp_packed_bytes": ([], C.c_size_t),
            "nb_mlp_pack": ([P, C.c_float, C.c_float, P, P], st),
            "nb_mlp_forward_tc": ([P, P, C.c_int64, P, P], st),
            "nb_mlp_loss_grad": ([P, C.c_float, C.c_float, P, P, P, C.c_int64, P, P, P], st),
            "nb_mlp_train": ([P, P, C.c_float, C.c_float, P, P, P, C.c_int64, i, i, i, i, C.c_float,
                              C.c_float, P, P], st),
            "nb_set_surrogate": ([P, P, C.c_float, C.c_float, P], st),
            "nb_pairlist_1x1": ([P, C.c_float, i, P, P, P], st),
            "nb_buffer_drift": ([i, P, i, P, C.c_double, C.POINTER(nb_params), C.c_double, C.c_double,
                                 C.c_double, C.POINTER(C.c_double)], st),
            "nb_buffer_size": ([i, P, i, P, C.c_double, C.POINTER(nb_params), C.c_double, C.c_double,
                                C.c_double, C.POINTER(C.c_double)], st),
            "nb_compute_1x1": ([P, C.POINTER(nb_params), P, P, P, i, P, P], st),
            "nb_rdf": ([P, C.c_float, i, i, i, i, P, P], st),
            "nb_prune_compute": ([P, C.POINTER(nb_params), P, C.c_float, P, P, P, P], st),
            "nb_run_frames": ([P, C.POINTER(nb_params), C.POINTER(nb_frames), P, P], st),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def exported_symbols():
    """Names declared in include/nbcluster.h (for the ABI test)."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:nb_status|const char\*|size_t)\s+(nb_\w+)\s*\(", txt, re.M)))


def status_name(s: int) -> str:
    return load().nb_status_string(int(s)).decode()


_F32, _F64, _I32, _U64 = ("float32",), ("float64",), ("int32",), ("int64", "uint64")


_DTYPE_NAMES = {}   # torch dtype -> its name (memoised: the check runs on every call)


def _ptr(x, dtypes=None):
    """Device pointer of a torch tensor (or an int / None).  A tensor must be
    a contiguous CUDA tensor: every pointer the library takes addresses a
    dense device array; dtypes, where given, lists the element types the C
    declaration reads."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError("the library takes device memory: pass a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("the library takes dense arrays: pass a contiguous tensor")
    if dtypes is not None:
        name = _DTYPE_NAMES.get(x.dtype)
        if name is None:
            name = _DTYPE_NAMES.setdefault(x.dtype, str(x.dtype).replace("torch.", ""))
        if name not in dtypes:
            raise ValueError(f"expected a {' or '.join(dtypes)} tensor, got {x.dtype}")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, s):
    if s != NB_OK:
        msg = load().nb_last_error(ctx).decode() if ctx else ""
        raise NbError(s, msg)


# --- entry points (same names as the C ABI) --------------------------------

def nb_create(cluster_size: int = 8, device: int = 0):
    h = C.c_void_p()
    opt = nb_options(cluster_size, device)
    _check(None, load().nb_create(C.byref(h), C.byref(opt)))
    return h


def nb_destroy(ctx):
    _check(None, load().nb_destroy(ctx))


def nb_last_error(ctx) -> str:
    return load().nb_last_error(ctx).decode()


def nb_lj_combine(sigma, eps, comb: int = NB_COMB_LB):
    """Host LJ pair table float32 [nt, nt, 2] from per-type sigma/epsilon."""
    import numpy as np
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    nt = s.shape[0]
    out = np.zeros((nt, nt, 2), np.float32)
    _check(None, load().nb_lj_combine(nt, s.ctypes.data, e.ctypes.data, int(comb), out.ctypes.data))
    return out


def nb_workspace_query(ctx, n_atoms: int, box, rlist_max: float, ntypes: int,
                       list_factor: float = 0.0) -> int:
    b = (C.c_double * 3)(*[float(v) for v in box])
    nbytes = C.c_size_t()
    _check(ctx, load().nb_workspace_query(ctx, int(n_atoms), b, float(rlist_max), int(ntypes),
                                          float(list_factor), C.byref(nbytes)))
    return nbytes.value


def _boxes(boxes):
    """double [nbox][3] host array from one box (3 numbers) or a list of boxes."""
    import numpy as np
    b = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
    return b


def nb_workspace_query_boxes(ctx, n_atoms, boxes, rlist_max: float, ntypes: int,
                             list_factor: float = 0.0) -> int:
    import numpy as np
    n = np.ascontiguousarray(n_atoms, dtype=np.int32).reshape(-1)
    b = _boxes(boxes)
    if b.shape[0] != n.shape[0]:
        raise ValueError("one box per particle count")
    nbytes = C.c_size_t()
    _check(ctx, load().nb_workspace_query_boxes(ctx, int(n.shape[0]), n.ctypes.data, b.ctypes.data,
                                                float(rlist_max), int(ntypes), float(list_factor),
                                                C.byref(nbytes)))
    return nbytes.value


def nb_workspace_bytes(cluster_size, n_atoms, boxes, rlist_max: float, ntypes: int,
                       list_factor: float = 0.0) -> int:
    """Workspace bytes of a plan, computed on the host (no context, no device)."""
    import numpy as np
    n = np.ascontiguousarray(n_atoms, dtype=np.int32).reshape(-1)
    b = _boxes(boxes)
    if b.shape[0] != n.shape[0]:
        raise ValueError("one box per particle count")
    nbytes = C.c_size_t()
    s = load().nb_workspace_bytes(int(cluster_size), int(n.shape[0]), n.ctypes.data, b.ctypes.data,
                                  float(rlist_max), int(ntypes), float(list_factor), C.byref(nbytes))
    if s != NB_OK:
        raise NbError(s, "workspace plan refused")
    return nbytes.value


def nb_set_workspace(ctx, ws, nbytes: int):
    _check(ctx, load().nb_set_workspace(ctx, _ptr(ws), int(nbytes)))


def nb_set_atoms(ctx, n, q, types, ntypes, c6c12, stream=None):
    _check(ctx, load().nb_set_atoms(ctx, int(n), _ptr(q, _F32), _ptr(types, _I32), int(ntypes), _ptr(c6c12, _F32),
                                    _stream(stream)))


def nb_grid_put(ctx, xyz, boxes, stream=None):
    """boxes: the edges of one box (3 numbers) or of every box ([nbox][3])."""
    b = _boxes(boxes)
    _check(ctx, load().nb_grid_put(ctx, _ptr(xyz, _F32), b.ctypes.data, _stream(stream)))


def nb_pairlist_build(ctx, rlist, rbb=0.0, excl_off=None, excl_idx=None, stream=None):
    _check(ctx, load().nb_pairlist_build(ctx, float(rlist), float(rbb), _ptr(excl_off, _I32),
                                         _ptr(excl_idx, _I32), _stream(stream)))


def nb_set_coords(ctx, xyz, stream=None):
    _check(ctx, load().nb_set_coords(ctx, _ptr(xyz, _F32), _stream(stream)))


def nb_prune(ctx, xyz, r_prune, stream=None):
    _check(ctx, load().nb_prune(ctx, _ptr(xyz, _F32), float(r_prune), _stream(stream)))


def make_params(elec: str, rc: float, eps_rf: float = float("inf"), beta: float = 0.0,
                want_energy: bool = True) -> nb_params:
    """elec: "rf", "ewald", "ewald_mlp" (the network from nb_set_surrogate) or
    "ewald_tab" (tabulated force factor)."""
    code = {"rf": NB_ELEC_RF, "ewald": NB_ELEC_EWALD, "ewald_mlp": NB_ELEC_EWALD_MLP,
            "ewald_tab": NB_ELEC_EWALD_TAB}[elec]
    return nb_params(code, int(bool(want_energy)), float(rc), float(eps_rf), float(beta))


def nb_compute(ctx, params: nb_params, xyz, f, e=None, vir=None, stream=None):
    _check(ctx, load().nb_compute(ctx, C.byref(params), _ptr(xyz, _F32), _ptr(f, _F32), _ptr(e, _F64),
                                  _ptr(vir, _F64), _stream(stream)))


def nb_check(ctx, stream=None, raise_on_error: bool = True) -> nb_info:
    info = nb_info()
    s = load().nb_check(ctx, _stream(stream), C.byref(info))
    if raise_on_error:
        _check(ctx, s)
    info.status = s
    return info


def nb_box_info(ctx, box: int) -> nb_info:
    info = nb_info()
    _check(ctx, load().nb_box_info(ctx, int(box), C.byref(info)))
    return info


def nb_get_grid(ctx, atom_of_slot=None, slot_of_atom=None, col_clu_start=None, xyzq=None,
                type_slot=None, bb=None, col_of_atom=None, sc_info=None, stream=None):
    _check(ctx, load().nb_get_grid(ctx, _ptr(atom_of_slot, _I32), _ptr(slot_of_atom, _I32),
                                   _ptr(col_clu_start, _I32), _ptr(xyzq, _F32), _ptr(type_slot, _I32),
                                   _ptr(bb, _F32), _ptr(col_of_atom, _I32), _ptr(sc_info, _I32), _stream(stream)))


def nb_get_list(ctx, which, ient=None, cj=None, mask=None, stream=None):
    _check(ctx, load().nb_get_list(ctx, int(which), _ptr(ient, _I32), _ptr(cj, _I32), _ptr(mask, _U64),
                                   _stream(stream)))


def nb_profile(ctx, enable=True, keep=False):
    """enable: record spans; keep: spans survive reads (timing graph replays)."""
    _check(ctx, load().nb_profile(ctx, 2 if (enable and keep) else int(bool(enable))))


def nb_profile_read(ctx, max_spans=256):
    """[(kind, ms), ...] of the spans recorded since the last read."""
    kinds = (C.c_int * max_spans)()
    ms = (C.c_float * max_spans)()
    cnt = C.c_int()
    _check(ctx, load().nb_profile_read(ctx, kinds, ms, int(max_spans), C.byref(cnt)))
    return [(kinds[k], ms[k]) for k in range(cnt.value)]


def _need(x, count, name):
    """Raise if tensor x holds fewer than count elements (the C entry point
    trusts the sizes it is given; raw integer pointers are the caller's
    responsibility)."""
    if x is not None and not isinstance(x, int) and x.numel() < count:
        raise ValueError(f"{name} holds {x.numel()} elements, the call needs at least {count}")


def nb_grid_put_noalloc(n, xyz, q, types, ntypes, box, cluster_size, atom_of_slot, xyzq, type_slot,
                        bb, col_clu_start, info, max_slots, max_columns, stream=None):
    """Gridding into caller-provided outputs with no device allocation
    anywhere (scratch in a fixed array inside the library); see the header.
    Tensor arguments are checked against n, max_slots and max_columns first,
    since the library writes up to those sizes."""
    n, ms, mc, cs = int(n), int(max_slots), int(max_columns), int(cluster_size)
    if n > 0:
        _need(xyz, 3 * n, "xyz")
        _need(q, n, "q")
        _need(types, n, "types")
    if ms > 0:
        _need(atom_of_slot, ms, "atom_of_slot")
        _need(type_slot, ms, "type_slot")
        _need(xyzq, 4 * ms, "xyzq")
        if cs in (4, 8):
            _need(bb, 8 * (ms // cs), "bb")
    if mc > 0:
        _need(col_clu_start, mc + 1, "col_clu_start")
    _need(info, 2, "info")
    b = (C.c_double * 3)(*[float(v) for v in box])
    s = load().nb_grid_put_noalloc(int(n), _ptr(xyz, _F32), _ptr(q, _F32), _ptr(types, _I32), int(ntypes), b,
                                   int(cluster_size), _ptr(atom_of_slot, _I32), _ptr(xyzq, _F32),
                                   _ptr(type_slot, _I32), _ptr(bb, _F32), _ptr(col_clu_start, _I32),
                                   _ptr(info, _I32), int(max_slots),
                                   int(max_columns), _stream(stream))
    _check(None, s)


def _status(s, what):
    if s != NB_OK:
        raise NbError(s, what)


def nb_ewald_factor(r, beta, out, stream=None):
    _status(load().nb_ewald_factor(_ptr(r, _F64), int(r.numel()), float(beta), _ptr(out, _F64), _stream(stream)),
            "nb_ewald_factor")


def nb_mlp_forward(params, r_min, r_max, r, y, stream=None):
    _status(load().nb_mlp_forward(_ptr(params, _F32), float(r_min), float(r_max), _ptr(r, _F32), int(r.numel()),
                                  _ptr(y, _F32), _stream(stream)), "nb_mlp_forward")


def nb_mlp_packed_bytes() -> int:
    return int(load().nb_mlp_packed_bytes())


def nb_mlp_pack(params, r_min, r_max, packed, stream=None):
    _status(load().nb_mlp_pack(_ptr(params, _F32), float(r_min), float(r_max), _ptr(packed), _stream(stream)),
            "nb_mlp_pack")


def nb_mlp_forward_tc(packed, r, y, stream=None):
    _status(load().nb_mlp_forward_tc(_ptr(packed), _ptr(r, _F32), int(r.numel()), _ptr(y, _F32), _stream(stream)),
            "nb_mlp_forward_tc")


def nb_mlp_loss_grad(params, r_min, r_max, r, t, w, grad, loss=None, stream=None):
    _status(load().nb_mlp_loss_grad(_ptr(params, _F32), float(r_min), float(r_max), _ptr(r, _F32), _ptr(t, _F32),
                                    _ptr(w, _F32), int(r.numel()), _ptr(grad, _F32), _ptr(loss, _F32),
                                    _stream(stream)), "nb_mlp_loss_grad")


def nb_mlp_train(params, state, r_min, r_max, r, t, w, batch, steps, step0, total_steps, lr_max, lr_min,
                 loss=None, stream=None):
    _status(load().nb_mlp_train(_ptr(params, _F32), _ptr(state, _F32), float(r_min), float(r_max), _ptr(r, _F32),
                                _ptr(t, _F32), _ptr(w, _F32),
                                int(r.numel()), int(batch), int(steps), int(step0), int(total_steps),
                                float(lr_max), float(lr_min), _ptr(loss, _F32), _stream(stream)), "nb_mlp_train")


def _classes(classes):
    """[(count, mass, charge, type), ...] -> ctypes array of nb_particle_class."""
    arr = (nb_particle_class * len(classes))()
    for k, (cnt, m, q, t) in enumerate(classes):
        arr[k] = nb_particle_class(float(cnt), float(m), float(q), int(t))
    return arr


def nb_buffer_drift(classes, c6c12, volume, params, rb, t_ps, temperature):
    """Drift bound (kJ/mol/ps per particle) of buffer rb; classes as
    [(count, mass, charge, LJ type)], c6c12 host [nt, nt, 2]."""
    import numpy as np
    t = np.ascontiguousarray(c6c12, dtype=np.float32)
    out = C.c_double()
    arr = _classes(classes)
    _status(load().nb_buffer_drift(len(classes), arr, int(t.shape[0]), t.ctypes.data, float(volume),
                                   C.byref(params), float(rb), float(t_ps), float(temperature), C.byref(out)),
            "nb_buffer_drift")
    return out.value


def nb_buffer_size(classes, c6c12, volume, params, t_ps, temperature, tolerance):
    """Smallest buffer (nm) whose drift bound is at most tolerance."""
    import numpy as np
    t = np.ascontiguousarray(c6c12, dtype=np.float32)
    out = C.c_double()
    arr = _classes(classes)
    _status(load().nb_buffer_size(len(classes), arr, int(t.shape[0]), t.ctypes.data, float(volume),
                                  C.byref(params), float(t_ps), float(temperature), float(tolerance),
                                  C.byref(out)), "nb_buffer_size")
    return out.value


def nb_pairlist_1x1(ctx, rlist, max_nbr, nbr, count, stream=None):
    _check(ctx, load().nb_pairlist_1x1(ctx, float(rlist), int(max_nbr), _ptr(nbr, _I32), _ptr(count, _I32),
                                       _stream(stream)))


def nb_compute_1x1(ctx, params, xyz, nbr, count, max_nbr, f, stream=None):
    _check(ctx, load().nb_compute_1x1(ctx, C.byref(params), _ptr(xyz, _F32), _ptr(nbr, _I32), _ptr(count, _I32),
                                      int(max_nbr), _ptr(f, _F32), _stream(stream)))


def nb_prune_compute(ctx, params, xyz, r_prune, f, e=None, vir=None, stream=None):
    _check(ctx, load().nb_prune_compute(ctx, C.byref(params), _ptr(xyz, _F32), float(r_prune), _ptr(f, _F32),
                                        _ptr(e, _F64), _ptr(vir, _F64), _stream(stream)))


def _host_ptr(x, dtype, name):
    """Address of a contiguous host (CPU) tensor of the given torch dtype."""
    if x is None:
        return None
    if x.is_cuda:
        raise ValueError(f"{name} must be a host tensor (page-locked for overlapped copies)")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if str(x.dtype).replace("torch.", "") != dtype:
        raise ValueError(f"{name} must be {dtype}, got {x.dtype}")
    return x.data_ptr()


class RunFrames:
    """The marshalled arguments of nb_run_frames, for repeated runs over the
    same buffers: built (and checked) once, each call is then the C call
    alone.  Arguments as nb_run_frames; the host and device tensors, the
    energy flags and the boxes are kept referenced for the object's life."""

    def __init__(self, ctx, params, x_host, f_host, x_dev, f_dev, nbox=1, energy_frames=None, e_host=None,
                 vir_host=None, e_dev=None, vir_dev=None, build=False, boxes=None, rlist=0.0, rbb=0.0,
                 excl_off=None, excl_idx=None, first_frame=0, nstprune=0, r_prune=0.0):
        import numpy as np
        if x_host.dim() != 3 or x_host.shape[2] != 3 or tuple(f_host.shape) != tuple(x_host.shape):
            raise ValueError("x_host and f_host must both be [n_frames, n, 3]")
        nf, n = int(x_host.shape[0]), int(x_host.shape[1])
        fr = nb_frames()
        fr.n_frames, fr.n_atoms, fr.n_boxes = nf, n, int(nbox)
        fr.x_host = _host_ptr(x_host, "float32", "x_host")
        fr.f_host = _host_ptr(f_host, "float32", "f_host")
        self._ef = None
        if energy_frames is not None:
            ef = np.ascontiguousarray(np.asarray(energy_frames, dtype=bool).astype(np.uint8).reshape(-1))
            if ef.shape[0] != nf:
                raise ValueError("one energy flag per frame")
            fr.energy_frames_host = ef.ctypes.data
            self._ef = ef
        for name, h, d, w in (("e", e_host, e_dev, 2), ("vir", vir_host, vir_dev, 9)):
            if h is None:
                continue
            if h.numel() < nf * nbox * w:
                raise ValueError(f"{name}_host holds {h.numel()} values, needs {nf * nbox * w}")
            if d is None or len(d) != 2:
                raise ValueError(f"{name}_host needs two device buffers {name}_dev")
            setattr(fr, f"{name}_host", _host_ptr(h, "float64", f"{name}_host"))
            arr = getattr(fr, f"{name}_dev")
            for k in range(2):
                _need(d[k], nbox * w, f"{name}_dev[{k}]")
                arr[k] = _ptr(d[k], _F64)
        if len(x_dev) != 2 or len(f_dev) != 2:
            raise ValueError("two device buffers each for coordinates and forces")
        for k in range(2):
            _need(x_dev[k], 3 * n, f"x_dev[{k}]")
            _need(f_dev[k], 3 * n, f"f_dev[{k}]")
            fr.x_dev[k] = _ptr(x_dev[k], _F32)
            fr.f_dev[k] = _ptr(f_dev[k], _F32)
        self._boxes = None
        if build:
            self._boxes = _boxes(boxes)
            fr.build, fr.boxes_host = 1, self._boxes.ctypes.data
            fr.rlist, fr.rbb = float(rlist), float(rbb)
            fr.excl_off_dev, fr.excl_idx_dev = _ptr(excl_off, _I32), _ptr(excl_idx, _I32)
        fr.first_frame, fr.nstprune, fr.r_prune = int(first_frame), int(nstprune), float(r_prune)
        self.ctx, self.params, self.fr = ctx, params, fr
        self._keep = (x_host, f_host, x_dev, f_dev, e_host, vir_host, e_dev, vir_dev, excl_off, excl_idx)
        self._fn = load().nb_run_frames

    def __call__(self, stream=None, copy_stream=None):
        if copy_stream is None:
            raise ValueError("copy_stream: a second stream for the transfers")
        _check(self.ctx, self._fn(self.ctx, C.byref(self.params), C.byref(self.fr), _stream(stream),
                                  _stream(copy_stream)))


def nb_run_frames(ctx, params, x_host, f_host, x_dev, f_dev, nbox=1, energy_frames=None, e_host=None,
                  vir_host=None, e_dev=None, vir_dev=None, build=False, boxes=None, rlist=0.0, rbb=0.0,
                  excl_off=None, excl_idx=None, first_frame=0, nstprune=0, r_prune=0.0, stream=None,
                  copy_stream=None):
    """Frames from host memory through the calls of a list lifetime (see the
    header).  x_host, f_host: host float32 [n_frames, n, 3] (page-locked for
    overlap); x_dev, f_dev: two device float32 [n, 3] buffers each;
    energy_frames: per-frame flags (or None); e_host [n_frames, nbox, 2] and
    vir_host [n_frames, nbox, 9] host float64 with e_dev / vir_dev two device
    float64 buffers of [nbox, 2] / [nbox, 9].  The host tensors must stay
    alive until the streams finish.  (RunFrames marshals these once for
    repeated runs.)"""
    RunFrames(ctx, params, x_host, f_host, x_dev, f_dev, nbox, energy_frames, e_host, vir_host, e_dev, vir_dev,
              build, boxes, rlist, rbb, excl_off, excl_idx, first_frame, nstprune, r_prune)(stream, copy_stream)


def nb_rdf(ctx, r_max, nbins, type_a, type_b, accumulate, hist, stream=None):
    _check(ctx, load().nb_rdf(ctx, float(r_max), int(nbins), int(type_a), int(type_b), int(accumulate),
                              _ptr(hist, _U64), _stream(stream)))


def nb_set_surrogate(ctx, params, r_min, r_max, stream=None):
    _check(ctx, load().nb_set_surrogate(ctx, _ptr(params, _F32), float(r_min), float(r_max), _stream(stream)))


# --- convenience: boxes with their torch-allocated workspace ----------------

class Context:
    """A context for one box (n particles, box = 3 edges) or a batch of boxes
    (n = particles per box, box = [nbox][3] edges; particle arrays are the
    boxes' ranges concatenated): allocates the workspace with torch and keeps
    the per-particle inputs on the device."""

    def __init__(self, n, box, rlist_max, q, types, c6c12, cluster_size=8, device=0,
                 list_factor=0.0, stream=None):
        import numpy as np
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        counts = np.atleast_1d(np.asarray(n, dtype=np.int64))
        self.counts = counts
        self.nbox = int(counts.shape[0])
        self.n = int(counts.sum())
        self.C = cluster_size
        self.ctx = nb_create(cluster_size, device)
        nt = int(c6c12.shape[0])
        self.ws_bytes = nb_workspace_query_boxes(self.ctx, counts, box, rlist_max, nt, list_factor)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.dev)
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        nb_set_workspace(self.ctx, aligned, self.ws_bytes)
        self.q = torch.as_tensor(q, dtype=torch.float32).to(self.dev).contiguous()
        self.types = torch.as_tensor(types, dtype=torch.int32).to(self.dev).contiguous()
        self.c6c12 = torch.as_tensor(c6c12, dtype=torch.float32).to(self.dev).contiguous()
        nb_set_atoms(self.ctx, self.n, self.q, self.types, nt, self.c6c12, stream)

    def close(self):
        if self.ctx is not None:
            nb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
