"""nb_run_frames: frames from host memory through a list lifetime (list built
on the first frame, pruned every nstprune frames, Sec. 2.3), copies on a
second stream.  Against the same calls made frame by frame on the device,
and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4   # max |dF| / RMS |F| against the oracle
SAME_TOL = 1e-5    # the same calls: equal up to the order of FP32 additions


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    return torch, torch.device("cuda", 0), nb


def _frames(b, n_frames, seed):
    disp = w.frame_displacements(b.mass, n_frames, seed=seed)
    x = b.xyz[None] + np.concatenate([np.zeros((1, b.n, 3), np.float32), np.cumsum(disp, 0)[:-1]])
    return x.astype(np.float32)


def test_run_frames_matches_calls_and_oracle(env):
    """Twelve frames of a 6,000-particle Ewald box: one call building the list
    on frame 0 and pruning every 2 frames (energies on frames 0 and 7), then a
    continuation call on 4 more frames of the same list (first_frame 8).
    Every frame's forces, energies and virial equal those of the per-frame
    calls; the first and last frames match the oracle."""
    torch, dev, nb = env
    b = w.water_box(2000, None, seed=7100)
    rc, rl, beta, nstprune = 1.0, 1.1, 3.12, 2
    rlf = float(np.float32(rl))
    rp = float(np.float32(w.prune_radius(rc, rl, 5)))
    x = _frames(b, 12, seed=7101)
    c6c12 = nb.nb_lj_combine(b.sigma, b.eps)
    prm = nb.make_params("ewald", rc, beta=beta, want_energy=False)
    eo = torch.as_tensor(b.excl_off, device=dev)
    ei = torch.as_tensor(b.excl_idx, device=dev)
    efr = np.zeros(8, bool)
    efr[[0, 7]] = True

    # the run from host memory
    cx = nb.Context(b.n, b.box, rl, b.q, b.types, c6c12)
    ref = nb.Context(b.n, b.box, rl, b.q, b.types, c6c12)
    try:
        xh = torch.as_tensor(x).pin_memory()
        fh = torch.full((12, b.n, 3), float("nan"), dtype=torch.float32).pin_memory()
        eh = torch.zeros((8, 1, 2), dtype=torch.float64).pin_memory()
        vh = torch.zeros((8, 1, 9), dtype=torch.float64).pin_memory()
        xd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        fd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        ed = [torch.empty((1, 2), dtype=torch.float64, device=dev) for _ in range(2)]
        vd = [torch.empty((1, 9), dtype=torch.float64, device=dev) for _ in range(2)]
        cs = torch.cuda.Stream(device=dev)
        main = torch.cuda.current_stream()
        nb.nb_run_frames(cx.ctx, prm, xh[:8], fh[:8], xd, fd, energy_frames=efr, e_host=eh, vir_host=vh,
                         e_dev=ed, vir_dev=vd, build=True, boxes=b.box, rlist=rlf, rbb=0.8, excl_off=eo,
                         excl_idx=ei, nstprune=nstprune, r_prune=rp, stream=main, copy_stream=cs)
        nb.nb_run_frames(cx.ctx, prm, xh[8:], fh[8:], xd, fd, first_frame=8, nstprune=nstprune, r_prune=rp,
                         stream=main, copy_stream=cs)
        main.synchronize()
        nb.nb_check(cx.ctx)
        F = fh.numpy().astype(np.float64)
        assert np.isfinite(F).all()

        # the same calls frame by frame
        f = torch.zeros((b.n, 3), dtype=torch.float32, device=dev)
        e = torch.zeros((1, 2), dtype=torch.float64, device=dev)
        v = torch.zeros((1, 9), dtype=torch.float64, device=dev)
        prm_e = nb.make_params("ewald", rc, beta=beta, want_energy=True)
        for k in range(12):
            xk = torch.as_tensor(x[k], device=dev)
            en = k < 8 and efr[k]
            q = prm_e if en else prm
            if k == 0:
                nb.nb_grid_put(ref.ctx, xk, b.box)
                nb.nb_pairlist_build(ref.ctx, rlf, 0.8, eo, ei)
                xk = None
            if k > 0 and k % nstprune == 0:
                nb.nb_prune_compute(ref.ctx, q, xk, rp, f, e if en else None, v if en else None)
            else:
                nb.nb_compute(ref.ctx, q, xk, f, e if en else None, v if en else None)
            fr = f.cpu().numpy().astype(np.float64)
            rms = np.sqrt((fr ** 2).sum(1).mean())
            assert np.abs(F[k] - fr).max() <= SAME_TOL * rms, k
            if en:
                er, vr = e.cpu().numpy()[0], v.cpu().numpy()[0]
                assert np.abs(eh.numpy()[k, 0] - er).max() <= 1e-6 * np.abs(er).max(), k
                assert np.abs(vh.numpy()[k, 0] - vr).max() <= 1e-6 * np.abs(vr).max(), k
        nb.nb_check(ref.ctx)
        assert not eh.numpy()[1:7].any() and not vh.numpy()[1:7].any()   # only the energy frames

        # the oracle on the first and last frames
        oprm = oracle.make_params("ewald", float(np.float32(rc)), beta=beta)
        for k in (0, 11):
            fo, eo_, vo = oracle.forces_cells(x[k], b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx,
                                              b.box, oprm)
            rms = np.sqrt((fo ** 2).sum(1).mean())
            assert np.sqrt(((F[k] - fo) ** 2).sum(1)).max() < FORCE_TOL * rms, k
            if k == 0:
                assert np.abs(eh.numpy()[0, 0] - eo_).max() / np.abs(eo_).max() < 1e-5
                assert np.abs(vh.numpy()[0, 0] - vo.reshape(-1)).max() / np.abs(vo).max() < 1e-5
    finally:
        cx.close()
        ref.close()


def test_run_frames_errors(env):
    """Refused: a particle count not the context's and a copy stream equal to
    the compute stream (before any work), no list to continue (at frame 0,
    after that frame's coordinates were queued for copying)."""
    torch, dev, nb = env
    b = w.water_box(300, None, seed=7102)
    cx = nb.Context(b.n, b.box, 1.0, b.q, b.types, nb.nb_lj_combine(b.sigma, b.eps))
    try:
        prm = nb.make_params("ewald", 0.9, beta=3.12, want_energy=False)
        x = torch.as_tensor(_frames(b, 2, seed=7103)).pin_memory()
        f = torch.zeros_like(x).pin_memory()
        xd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        fd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream(device=dev)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_run_frames(cx.ctx, prm, x[:, :-3].contiguous(), f[:, :-3].contiguous(), xd, fd, stream=main,
                             copy_stream=cs)
        assert ei.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NbError) as ei:
            nb.nb_run_frames(cx.ctx, prm, x, f, xd, fd, build=True, boxes=b.box, rlist=1.0, stream=main,
                             copy_stream=main)
        assert ei.value.status == nb.NB_ERR_ARG
        with pytest.raises(nb.NbError) as ei:
            nb.nb_run_frames(cx.ctx, prm, x, f, xd, fd, stream=main, copy_stream=cs)
        assert ei.value.status == nb.NB_ERR_STATE
        torch.cuda.synchronize()
    finally:
        cx.close()


@pytest.mark.parametrize("C", [8, 4])
def test_run_frames_batch(env, C):
    """Two boxes of uneven size in one context (C = 8: fused prune; C = 4:
    prune kernel then force kernel), six frames, a prune every 3 frames,
    energies and virial per box on frames 0 and 5: equal to the calls made
    frame by frame."""
    torch, dev, nb = env
    B = w.concat([w.water_box(700, None, seed=7110), w.water_box(1300, None, seed=7111)])
    rc, rl, beta, nstprune, nf = 1.0, 1.1, 3.12, 3, 6
    rlf = float(np.float32(rl))
    rp = float(np.float32(w.prune_radius(rc, rl, nstprune)))
    disp = w.frame_displacements(B.mass, nf, seed=7112)
    x = (B.xyz[None] + np.concatenate([np.zeros((1, B.n, 3), np.float32), np.cumsum(disp, 0)[:-1]]))
    x = x.astype(np.float32)
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    prm = nb.make_params("ewald", rc, beta=beta, want_energy=False)
    prm_e = nb.make_params("ewald", rc, beta=beta, want_energy=True)
    eo = torch.as_tensor(B.excl_off, device=dev)
    ei = torch.as_tensor(B.excl_idx, device=dev)
    nbx = B.nbox
    efr = np.array([1, 0, 0, 0, 0, 1], bool)
    cx = nb.Context(B.counts, B.boxes, rl, B.q, B.types, c6c12, cluster_size=C)
    ref = nb.Context(B.counts, B.boxes, rl, B.q, B.types, c6c12, cluster_size=C)
    try:
        xh = torch.as_tensor(x).pin_memory()
        fh = torch.zeros((nf, B.n, 3), dtype=torch.float32).pin_memory()
        eh = torch.zeros((nf, nbx, 2), dtype=torch.float64).pin_memory()
        vh = torch.zeros((nf, nbx, 9), dtype=torch.float64).pin_memory()
        xd = [torch.empty((B.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        fd = [torch.empty((B.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        ed = [torch.empty((nbx, 2), dtype=torch.float64, device=dev) for _ in range(2)]
        vd = [torch.empty((nbx, 9), dtype=torch.float64, device=dev) for _ in range(2)]
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream(device=dev)
        nb.nb_run_frames(cx.ctx, prm, xh, fh, xd, fd, nbox=nbx, energy_frames=efr, e_host=eh, vir_host=vh,
                         e_dev=ed, vir_dev=vd, build=True, boxes=B.boxes, rlist=rlf, rbb=0.8, excl_off=eo,
                         excl_idx=ei, nstprune=nstprune, r_prune=rp, stream=main, copy_stream=cs)
        main.synchronize()
        nb.nb_check(cx.ctx)
        f = torch.zeros((B.n, 3), dtype=torch.float32, device=dev)
        e = torch.zeros((nbx, 2), dtype=torch.float64, device=dev)
        v = torch.zeros((nbx, 9), dtype=torch.float64, device=dev)
        for k in range(nf):
            xk = torch.as_tensor(x[k], device=dev)
            q = prm_e if efr[k] else prm
            if k == 0:
                nb.nb_grid_put(ref.ctx, xk, B.boxes)
                nb.nb_pairlist_build(ref.ctx, rlf, 0.8, eo, ei)
                xk = None
            ev = (e, v) if efr[k] else (None, None)
            if k > 0 and k % nstprune == 0:
                nb.nb_prune_compute(ref.ctx, q, xk, rp, f, *ev)
            else:
                nb.nb_compute(ref.ctx, q, xk, f, *ev)
            fr = f.cpu().numpy().astype(np.float64)
            rms = np.sqrt((fr ** 2).sum(1).mean())
            assert np.abs(fh.numpy()[k] - fr).max() <= SAME_TOL * rms, k
            if efr[k]:
                er, vr = e.cpu().numpy(), v.cpu().numpy()
                assert np.abs(eh.numpy()[k] - er).max() <= 1e-6 * np.abs(er).max(), k
                assert np.abs(vh.numpy()[k] - vr).max() <= 1e-6 * np.abs(vr).max(), k
        nb.nb_check(ref.ctx)
    finally:
        cx.close()
        ref.close()


def test_run_frames_replay(env):
    """Identical runs: the first made call by call, the second captured in a
    CUDA graph, later ones replayed.  Every run's forces agree with the
    first's; a replay reads the host frames anew (new coordinates written
    into the same buffer give their own forces, against the oracle); a run
    with other arguments in between (another prune interval) is made call by
    call, and the original arguments afterwards are right again."""
    torch, dev, nb = env
    b = w.water_box(1500, None, seed=7120)
    rc, rl, beta = 1.0, 1.1, 3.12
    rlf = float(np.float32(rl))
    rp = float(np.float32(w.prune_radius(rc, rl, 5)))
    xa = _frames(b, 6, seed=7121)
    xb = _frames(b, 6, seed=7122)
    c6c12 = nb.nb_lj_combine(b.sigma, b.eps)
    prm = nb.make_params("ewald", rc, beta=beta, want_energy=False)
    eo = torch.as_tensor(b.excl_off, device=dev)
    ei = torch.as_tensor(b.excl_idx, device=dev)
    cx = nb.Context(b.n, b.box, rl, b.q, b.types, c6c12)
    try:
        xh = torch.as_tensor(xa).pin_memory()
        fh = torch.zeros((6, b.n, 3), dtype=torch.float32).pin_memory()
        xd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        fd = [torch.empty((b.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        cs = torch.cuda.Stream(device=dev)
        main = torch.cuda.current_stream()

        def run(nstprune=2):
            fh.zero_()
            nb.nb_run_frames(cx.ctx, prm, xh, fh, xd, fd, build=True, boxes=b.box, rlist=rlf, rbb=0.8,
                             excl_off=eo, excl_idx=ei, nstprune=nstprune, r_prune=rp, stream=main,
                             copy_stream=cs)
            main.synchronize()
            nb.nb_check(cx.ctx)
            return fh.numpy().astype(np.float64).copy()

        first = run()
        rms = np.sqrt((first ** 2).sum(-1).mean())
        for _ in range(4):   # call by call, captured, then replays
            assert np.abs(run() - first).max() <= SAME_TOL * rms
        oprm = oracle.make_params("ewald", float(np.float32(rc)), beta=beta)

        def check(F, x):
            for k in (0, 3, 5):
                fo, _, _ = oracle.forces_cells(x[k], b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx,
                                               b.box, oprm)
                r = np.sqrt((fo ** 2).sum(1).mean())
                assert np.sqrt(((F[k] - fo) ** 2).sum(1)).max() < FORCE_TOL * r, k

        check(first, xa)
        xh.copy_(torch.as_tensor(xb))
        check(run(), xb)                 # a replay with new coordinates in the same buffer
        other = run(nstprune=3)          # other arguments: call by call
        check(other, xb)
        check(run(), xb)                 # the original arguments again
        check(run(), xb)
        check(run(), xb)
    finally:
        cx.close()
