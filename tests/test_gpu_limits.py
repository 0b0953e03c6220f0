"""Limits and state checks of the C ABI.  The workspace plan (host code
behind a device context): a j-entry word holds a 27-bit cluster index, list
and slot indices are 32-bit, the grid has at most 2^15 columns along x and
y, and box edges are finite; plans beyond a limit are refused with a status
instead of being laid out with wrapped indices (no workspace is allocated for
them).  Particle types out of range are flagged on the device, and the 1 x 1
list is refused for coordinates its cluster list was not built from."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    return nb


def _status(nb, fn, *args):
    try:
        fn(*args)
    except nb.NbError as e:
        return e.status
    return nb.NB_OK


@pytest.mark.parametrize("C", [8, 4])
def test_realistic_plans_are_accepted(nb, C):
    ctx = nb.nb_create(C)
    try:
        for n, L in ((24000, 6.21), (3000000, 31.07)):
            assert nb.nb_workspace_query(ctx, n, [L, L, L], 1.1, 2) > 0
    finally:
        nb.nb_destroy(ctx)


def test_more_clusters_than_a_jword_holds(nb):
    """1.1e9 particles at 0.05 per nm^3 with clusters of 8: the slot, i-entry
    and j-entry counts stay below 2^31, the cluster count (1.38e8) does not
    fit 27 bits."""
    ctx = nb.nb_create(8)
    try:
        L = (1.1e9 / 0.05) ** (1.0 / 3.0)
        assert _status(nb, nb.nb_workspace_query, ctx, 1_100_000_000, [L, L, L], 1.1, 2) == nb.NB_ERR_CAPACITY
        assert "2^27" in nb.nb_last_error(ctx)
    finally:
        nb.nb_destroy(ctx)


def test_degenerate_and_oversized_boxes(nb):
    ctx = nb.nb_create(8)
    try:
        # a slab far thinner than the column spacing: the column count is capped, the slots overflow
        assert _status(nb, nb.nb_workspace_query, ctx, 1000, [2.2e6, 2.2e6, 2e-12], 1.1, 2) == nb.NB_ERR_CAPACITY
        assert _status(nb, nb.nb_workspace_query, ctx, 10, [1e31, 1.0, 1.0], 1.1, 2) == nb.NB_ERR_BOX
        assert _status(nb, nb.nb_workspace_query, ctx, 10, [0.0, 1.0, 1.0], 1.1, 2) == nb.NB_ERR_BOX
        # more than 2^31 - 1 particles over the boxes
        assert _status(nb, nb.nb_workspace_query_boxes, ctx, [1_500_000_000, 1_500_000_000],
                       [[1e3, 1e3, 1e3], [1e3, 1e3, 1e3]], 1.1, 2) == nb.NB_ERR_ARG
        # the context still plans a valid box afterwards
        assert nb.nb_workspace_query(ctx, 24000, [6.21, 6.21, 6.21], 1.1, 2) > 0
    finally:
        nb.nb_destroy(ctx)


def test_type_out_of_range_is_flagged(nb):
    """A particle type outside 0 .. ntypes - 1 is used as type 0 by the grid
    and raises the box's NB_ERR_ARG flag; correct types clear it."""
    import numpy as np
    import torch
    from paper_1306_1737_gb300 import workloads as w
    b = w.water_box(600, None, seed=7600)
    c6c12 = nb.nb_lj_combine(b.sigma, b.eps)
    nt = int(c6c12.shape[0])
    bad = np.asarray(b.types, dtype=np.int32).copy()
    bad[3], bad[11] = nt, -1
    cx = nb.Context(b.n, b.box, 1.0, b.q, bad, c6c12)
    try:
        ctx, dev = cx.ctx, cx.dev
        x = torch.as_tensor(b.xyz, device=dev)
        nb.nb_grid_put(ctx, x, b.box)
        info = nb.nb_check(ctx, raise_on_error=False)
        assert info.status == nb.NB_ERR_ARG
        assert "type" in nb.nb_last_error(ctx)
        good = torch.as_tensor(np.asarray(b.types, dtype=np.int32), device=dev)
        nb.nb_set_atoms(ctx, b.n, cx.q, good, nt, cx.c6c12)
        nb.nb_grid_put(ctx, x, b.box)
        assert nb.nb_check(ctx, raise_on_error=False).status == nb.NB_OK
    finally:
        cx.close()


def test_pairlist_1x1_needs_the_list_coordinates(nb):
    """The 1 x 1 list holds every pair within rlist only for the coordinates
    the cluster list was built from: after new coordinates it is refused
    until the next build."""
    import numpy as np
    import gpu_path
    from paper_1306_1737_gb300 import workloads as w
    b, p = w.config1()
    gb = gpu_path.GpuBox(b, p["rlist"])
    torch = gb.torch
    try:
        gb.grid()
        rl = float(np.float32(p["rlist"]))
        gb.build(rl)
        nbr = torch.zeros((b.n, 768), dtype=torch.int32, device=gb.dev)
        cnt = torch.zeros(b.n, dtype=torch.int32, device=gb.dev)
        nb.nb_set_coords(gb.ctx, torch.as_tensor(b.xyz).to(gb.dev))
        assert _status(nb, nb.nb_pairlist_1x1, gb.ctx, rl, 768, nbr, cnt) == nb.NB_ERR_STATE
        gb.build(rl)
        nb.nb_pairlist_1x1(gb.ctx, rl, 768, nbr, cnt)
        nb.nb_check(gb.ctx)
        assert int(cnt.sum().item()) > 0
    finally:
        gb.close()
