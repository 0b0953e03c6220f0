"""nb_grid_put_noalloc: gridding for callers that cannot allocate device
memory (its scratch is a fixed array inside the library, so no context and
no workspace are needed).  Through the C ABI, two calls in a row on
different boxes must give exactly what nb_grid_put + nb_get_grid give
(the grid is compared bit for bit, as everywhere in these tests).

Kept in a file of its own that collects last."""
import numpy as np
import pytest

from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    from paper_1306_1737_gb300 import build as nbbuild
    nbbuild.build()
    nb.load()
    return torch, nb


def reference_grid(torch, nb, b, C):
    dev = torch.device("cuda", 0)
    cx = nb.Context(b.n, b.box, 1.0, b.q, b.types, nb.nb_lj_combine(b.sigma, b.eps), cluster_size=C)
    try:
        nb.nb_grid_put(cx.ctx, torch.as_tensor(b.xyz, device=dev), b.box)
        info = nb.nb_check(cx.ctx)
        ns = info.n_clusters * C
        aos = torch.zeros(ns, dtype=torch.int32, device=dev)
        ccs = torch.zeros(info.nx * info.ny + 1, dtype=torch.int32, device=dev)
        xyzq = torch.zeros((ns, 4), dtype=torch.float32, device=dev)
        ts = torch.zeros(ns, dtype=torch.int32, device=dev)
        bb = torch.zeros((info.n_clusters, 6), dtype=torch.float32, device=dev)
        nb.nb_get_grid(cx.ctx, aos, None, ccs, xyzq, ts, bb, None)
        torch.cuda.synchronize()
        return dict(nclu=info.n_clusters, ncol=info.nx * info.ny, aos=aos.cpu().numpy(),
                    ccs=ccs.cpu().numpy(), xyzq=xyzq.cpu().numpy(), ts=ts.cpu().numpy(),
                    bb=bb.cpu().numpy())
    finally:
        cx.close()


def noalloc_grid(torch, nb, b, C, max_slots=40000, max_columns=2048):
    dev = torch.device("cuda", 0)
    aos = torch.full((max_slots,), -7, dtype=torch.int32, device=dev)
    xyzq = torch.zeros((max_slots, 4), dtype=torch.float32, device=dev)
    ts = torch.zeros(max_slots, dtype=torch.int32, device=dev)
    bb = torch.zeros((max_slots // C, 8), dtype=torch.float32, device=dev)
    ccs = torch.zeros(max_columns + 1, dtype=torch.int32, device=dev)
    info = torch.zeros(2, dtype=torch.int32, device=dev)
    nb.nb_grid_put_noalloc(b.n, torch.as_tensor(b.xyz, device=dev), torch.as_tensor(b.q, device=dev),
                           torch.as_tensor(b.types, device=dev), b.ntypes, b.box, C, aos, xyzq, ts, bb,
                           ccs, info, max_slots, max_columns)
    torch.cuda.synchronize()
    nclu, flags = info.cpu().numpy().tolist()
    ns = nclu * C
    return dict(nclu=nclu, flags=flags, aos=aos.cpu().numpy()[:ns], ccs=ccs.cpu().numpy(),
                xyzq=xyzq.cpu().numpy()[:ns], ts=ts.cpu().numpy()[:ns],
                bb=bb.cpu().numpy()[:nclu][:, [0, 1, 2, 4, 5, 6]])


def same(ref, got):
    assert got["flags"] == 0
    assert got["nclu"] == ref["nclu"]
    assert np.array_equal(got["ccs"][: ref["ncol"] + 1], ref["ccs"])
    assert np.array_equal(got["aos"], ref["aos"])
    assert np.array_equal(got["ts"], ref["ts"])
    assert np.array_equal(got["xyzq"].view(np.uint32), ref["xyzq"].view(np.uint32))
    assert np.array_equal(got["bb"].view(np.uint32), ref["bb"].view(np.uint32))


def test_noalloc_grid_matches_grid_put_twice(env):
    torch, nb = env
    big = w.water_box(512, 2.48, seed=1001)       # 1,536 particles
    small = w.water_box(101, 1.5, seed=77)        # 303 particles: stale scratch would show
    ref_big = reference_grid(torch, nb, big, 8)
    ref_small = reference_grid(torch, nb, small, 8)
    same(ref_big, noalloc_grid(torch, nb, big, 8))
    same(ref_small, noalloc_grid(torch, nb, small, 8))


def test_noalloc_limits_and_cluster_size_4(env):
    torch, nb = env
    b = w.water_box(300, None, seed=5)
    same(reference_grid(torch, nb, b, 4), noalloc_grid(torch, nb, b, 4))
    with pytest.raises(nb.NbError) as ei:       # output arrays too small
        noalloc_grid(torch, nb, b, 8, max_slots=100)
    assert ei.value.status == nb.NB_ERR_CAPACITY
    big = w.water_box(11000, None, seed=6)      # 33,000 particles: above the fixed maximum
    with pytest.raises(nb.NbError) as ei:
        noalloc_grid(torch, nb, big, 8, max_slots=70000, max_columns=8192)
    assert ei.value.status == nb.NB_ERR_CAPACITY
