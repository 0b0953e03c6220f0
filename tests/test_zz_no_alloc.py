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
    nb.load()
    return torch, nb


def reference_grid(torch, nb, b, C, rlist=1.0, device=0):
    dev = torch.device("cuda", device)
    cx = nb.Context(b.n, b.box, rlist, b.q, b.types, nb.nb_lj_combine(b.sigma, b.eps), cluster_size=C,
                    device=device)
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


def noalloc_grid(torch, nb, b, C, max_slots=40000, max_columns=2048, device=0):
    dev = torch.device("cuda", device)
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


class _Slab:
    """n uniform random particles (one LJ type, no charge) in a thin slab whose
    grid has exactly 64 x 64 = 4,096 columns for clusters of C: the column
    spacing (C a^2 h / n)^(1/3) is a / 64 for the height h = a n / (64^3 C)
    (a = the slab's edge), and just below it for 0.99 of that height."""

    def __init__(self, n, C, a=12.8, seed=3):
        rng = np.random.default_rng(seed)
        h = 0.99 * a * n / (64.0 ** 3 * C)
        self.n = n
        self.box = np.array([a, a, h])
        self.xyz = (rng.random((n, 3)) * self.box).astype(np.float32)
        self.q = np.zeros(n, np.float32)
        self.types = np.zeros(n, np.int32)
        self.ntypes = 1
        self.sigma = np.array([0.3])
        self.eps = np.array([0.5])


@pytest.mark.parametrize("C", [8, 4])
def test_noalloc_at_its_limits(env, C):
    """32,768 particles on a 4,096-column grid (for C = 8 that is 61,440
    slots, the fixed maximum) grid exactly as nb_grid_put grids them."""
    torch, nb = env
    b = _Slab(32768, C)
    ref = reference_grid(torch, nb, b, C, rlist=0.05)   # list capacity for a slab 0.2-0.4 nm thick
    assert ref["ncol"] == 4096
    got = noalloc_grid(torch, nb, b, C, max_slots=61440, max_columns=4096)
    same(ref, got)


def test_noalloc_flags_an_overlong_column(env):
    """A column with more than 8,192 particles is flagged (1 << NB_ERR_CAPACITY
    in info[1]); its particles get no slot and every other particle does."""
    torch, nb = env
    rng = np.random.default_rng(9)
    b = _Slab(16384, 8)
    b.box = np.array([8.0, 8.0, 8.0])
    xyz = rng.random((b.n, 3)) * b.box
    crowd = np.arange(9000)
    xyz[crowd, 0] = rng.random(crowd.size) * 0.3     # one grid column (spacing 0.63 nm)
    xyz[crowd, 1] = rng.random(crowd.size) * 0.3
    b.xyz = xyz.astype(np.float32)
    got = noalloc_grid(torch, nb, b, 8, max_slots=40000, max_columns=2048)
    assert got["flags"] & (1 << nb.NB_ERR_CAPACITY)
    placed = got["aos"][got["aos"] >= 0]
    assert len(np.unique(placed)) == placed.size
    assert not np.isin(crowd, placed).any()
    others = np.setdiff1d(np.arange(b.n), crowd)
    in_crowd_column = (np.floor(b.xyz[others, 0] * np.float32(12 / 8.0)) == 0) & \
                      (np.floor(b.xyz[others, 1] * np.float32(12 / 8.0)) == 0)
    assert np.isin(others[~in_crowd_column], placed).all()


def test_second_device_after_the_first(env):
    """The large shared-memory opt-ins of the gridding kernels are made per
    device: gridding through a context and without one on device 1, after
    device 0 has been used in the same process, gives device 0's grid bit
    for bit (skipped with one visible device)."""
    torch, nb = env
    if torch.cuda.device_count() < 2:
        pytest.skip("one CUDA device visible")
    b = w.water_box(512, 2.48, seed=1001)
    ref0 = reference_grid(torch, nb, b, 8)
    with torch.cuda.device(1):
        ref1 = reference_grid(torch, nb, b, 8, device=1)
        got1 = noalloc_grid(torch, nb, b, 8, device=1)
    same(ref0, dict(ref1, flags=0))
    same(ref0, got1)
