"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/nbcluster.h declares (no compute calls)."""
import ctypes
import re
import subprocess

import pytest

import paper_1306_1737_gb300 as nb
from paper_1306_1737_gb300 import build as nbbuild


@pytest.fixture(scope="module")
def lib():
    nbbuild.build()
    return nb.load()


def test_header_declares_the_hot_path(lib):
    names = nb.exported_symbols()
    for required in ("nb_grid_put", "nb_pairlist_build", "nb_prune", "nb_compute", "nb_create",
                     "nb_destroy", "nb_workspace_query", "nb_set_workspace", "nb_set_atoms",
                     "nb_check", "nb_set_coords"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", nb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (nb_\w+)$", out, re.M))
    for name in nb.exported_symbols():
        assert name in exported, name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_status_strings_and_host_helpers(lib):
    assert nb.status_name(nb.NB_OK) == "NB_OK"
    assert nb.status_name(nb.NB_ERR_CAPACITY) == "NB_ERR_CAPACITY"
    t = nb.nb_lj_combine([0.3166, 0.0], [0.65, 0.0])
    # C6 = 4 eps sigma^6, C12 = 4 eps sigma^12 for the O-O pair
    assert t[0, 0, 0] == pytest.approx(4 * 0.65 * 0.3166 ** 6, rel=1e-6)
    assert t[0, 0, 1] == pytest.approx(4 * 0.65 * 0.3166 ** 12, rel=1e-6)
    assert (t[1] == 0).all() and (t[:, 1] == 0).all()
    with pytest.raises(nb.NbError):
        nb.nb_lj_combine([0.3], [0.5], comb=7)


def test_null_context_is_rejected(lib):
    assert lib.nb_destroy(None) == nb.NB_ERR_ARG
    assert lib.nb_grid_put(None, None, None, None) == nb.NB_ERR_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises: there is no CPU path."""
    monkeypatch.setattr(nb, "LIB_PATH", str(tmp_path / "libnbcluster.so"))
    monkeypatch.setattr(nb, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        nb.load()
    with pytest.raises(RuntimeError, match="missing"):
        nb.nb_lj_combine([0.3], [0.5])
    with pytest.raises(RuntimeError, match="missing"):
        nb.nb_create(8, 0)


def test_binding_refuses_host_tensors():
    """Pointers handed to the library address device memory: a CPU tensor is
    refused before any call (ints and None pass through unchanged)."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="CUDA tensor"):
        nb._ptr(torch.zeros(3))
    assert nb._ptr(None) is None and nb._ptr(4096) == 4096


def test_binding_checks_element_types():
    """The typed pointer arguments of the hot-path calls accept only the
    element type their C declaration reads (a stand-in object reports itself
    as a CUDA tensor, so no device is needed)."""
    torch = pytest.importorskip("torch")

    class DeviceArray:
        is_cuda = True

        def __init__(self, dtype, contiguous=True):
            self.dtype, self._c = dtype, contiguous

        def is_contiguous(self):
            return self._c

        def data_ptr(self):
            return 4096

    assert nb._ptr(DeviceArray(torch.float32), nb._F32) == 4096
    assert nb._ptr(DeviceArray(torch.int64), nb._U64) == 4096
    with pytest.raises(ValueError, match="float32"):
        nb._ptr(DeviceArray(torch.float64), nb._F32)
    with pytest.raises(ValueError, match="int32"):
        nb._ptr(DeviceArray(torch.int64), nb._I32)
    with pytest.raises(ValueError, match="contiguous"):
        nb._ptr(DeviceArray(torch.float32, contiguous=False), nb._F32)


def test_noalloc_binding_checks_sizes_before_the_call():
    """The binding compares each output tensor with n, max_slots and
    max_columns before handing pointers to the library, which writes up to
    those sizes (CPU tensors: the size check fires before the device check)."""
    torch = pytest.importorskip("torch")
    import paper_1306_1737_gb300 as nb
    n, ms, mc, C = 100, 400, 50, 8

    def args(**over):
        a = dict(xyz=torch.zeros(3 * n), q=torch.zeros(n), types=torch.zeros(n, dtype=torch.int32),
                 atom_of_slot=torch.zeros(ms, dtype=torch.int32), xyzq=torch.zeros(4 * ms),
                 type_slot=torch.zeros(ms, dtype=torch.int32), bb=torch.zeros(8 * (ms // C)),
                 col_clu_start=torch.zeros(mc + 1, dtype=torch.int32), info=torch.zeros(2, dtype=torch.int32))
        a.update(over)
        return a

    def call(a):
        nb.nb_grid_put_noalloc(n, a["xyz"], a["q"], a["types"], 1, [2.0, 2.0, 2.0], C, a["atom_of_slot"],
                               a["xyzq"], a["type_slot"], a["bb"], a["col_clu_start"], a["info"], ms, mc)

    for name, short in [("xyz", torch.zeros(3 * n - 1)), ("q", torch.zeros(n - 1)),
                        ("types", torch.zeros(n - 1, dtype=torch.int32)),
                        ("atom_of_slot", torch.zeros(ms - 1, dtype=torch.int32)),
                        ("xyzq", torch.zeros(4 * ms - 1)), ("type_slot", torch.zeros(ms - 1, dtype=torch.int32)),
                        ("bb", torch.zeros(8 * (ms // C) - 1)),
                        ("col_clu_start", torch.zeros(mc, dtype=torch.int32)),
                        ("info", torch.zeros(1, dtype=torch.int32))]:
        with pytest.raises(ValueError, match=name):
            call(args(**{name: short}))
    with pytest.raises(ValueError, match="CUDA"):
        call(args())


def test_run_frames_binding_checks_shapes_before_the_call():
    """nb_run_frames' binding: host frames and forces of one shape [F, n, 3],
    host tensors on the host, energy flags one per frame and two staging
    buffers of sufficient size, all checked before the library is called
    (which trusts the sizes against the context's particle count)."""
    torch = pytest.importorskip("torch")
    import paper_1306_1737_gb300 as nb
    prm = nb.make_params("ewald", 1.0, beta=3.12, want_energy=False)
    x = torch.zeros((4, 10, 3))
    with pytest.raises(ValueError, match="n_frames, n, 3"):
        nb.nb_run_frames(None, prm, x, torch.zeros((4, 11, 3)), [None, None], [None, None])
    with pytest.raises(ValueError, match="n_frames, n, 3"):
        nb.nb_run_frames(None, prm, torch.zeros((4, 10, 2)), torch.zeros((4, 10, 2)), [None, None],
                         [None, None])
    with pytest.raises(ValueError, match="one energy flag per frame"):
        nb.nb_run_frames(None, prm, x, torch.zeros_like(x), [None, None], [None, None], energy_frames=[1, 0])
    with pytest.raises(ValueError, match="two device buffers e_dev"):
        nb.nb_run_frames(None, prm, x, torch.zeros_like(x), [None, None], [None, None],
                         e_host=torch.zeros((4, 1, 2), dtype=torch.float64))
    with pytest.raises(ValueError, match="x_dev"):
        nb.nb_run_frames(None, prm, x, torch.zeros_like(x), [torch.zeros(29), torch.zeros(30)],
                         [torch.zeros(30), torch.zeros(30)])
