"""The learned Ewald force factor on the GPU, against the FP64 oracle.

1. FP64 targets c(r) from the library equal the oracle's.
2. FP32 forward, tensor-core forward and the loss gradient of the library's
   kernels equal the oracle's network and gradient (random parameters).
3. Training on the GPU (Adam, the library's forward/backward kernels) on 2^20
   distances with oracle targets fits c(r): the trained network's error on
   held-out distances and on the pair distances of the 24,000-atom box is
   small, and far below the untrained network's.
4. In the force kernel (8 x 8 tiles on the tensor cores) the surrogate's
   forces on the 24,000-atom box are within 5e-4 of the RMS force of the
   oracle; the analytic kernel's error and both kernels' times are reported
   beside it.
5. What the trained network gains over the method without it (the analytic
   kernel that runs when no network is installed), on the same list and
   GPU: its accuracy and time gains are measured and asserted as found --
   on this hardware both are below one (the analytic rational fit is more
   accurate and cheaper); the trained network's gain over the untrained one
   is also measured."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

BETA = 3.12
R_MIN, R_MAX = 0.05, 1.0
SURROGATE_FORCE_TOL = 5e-4
TRAIN_STEPS = 60000


@pytest.fixture(scope="module")
def env():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    return torch, torch.device("cuda", 0), nb


def test_ewald_factor_targets(env):
    torch, dev, nb = env
    r = w.surrogate_samples(1 << 16, R_MIN, R_MAX, seed=11)
    out = torch.empty(r.size, dtype=torch.float64, device=dev)
    nb.nb_ewald_factor(torch.as_tensor(r, device=dev), BETA, out)
    ref = oracle.ewald_factor(r, BETA)
    rel = np.abs(out.cpu().numpy() - ref) / np.abs(ref)
    assert rel.max() < 1e-13, rel.max()


def test_forward_and_gradient_match_oracle(env):
    torch, dev, nb = env
    rng = np.random.default_rng(21)
    p = (rng.standard_normal(nb.NB_MLP_NPARAMS) * 0.4).astype(np.float32)
    r = w.surrogate_samples(4099, R_MIN, R_MAX, seed=12)      # a ragged last tile
    t = oracle.ewald_factor(r, BETA)
    wt = rng.uniform(0.5, 2.0, r.size)
    pd = torch.as_tensor(p, device=dev)
    rd = torch.as_tensor(r.astype(np.float32), device=dev)
    # the oracle sees the FP32 values the GPU sees
    r32 = r.astype(np.float32).astype(np.float64)
    y_ref = oracle.mlp_forward(p.astype(np.float64), R_MIN, R_MAX, r32)
    y = torch.empty(r.size, dtype=torch.float32, device=dev)
    nb.nb_mlp_forward(pd, R_MIN, R_MAX, rd, y)
    err = np.abs(y.cpu().numpy() - y_ref)
    assert err.max() < 2e-5 * max(1.0, np.abs(y_ref).max()), err.max()
    packed = torch.empty(nb.nb_mlp_packed_bytes() // 4, dtype=torch.float32, device=dev)
    nb.nb_mlp_pack(pd, R_MIN, R_MAX, packed)
    ytc = torch.empty_like(y)
    nb.nb_mlp_forward_tc(packed, rd, ytc)
    err_tc = np.abs(ytc.cpu().numpy() - y_ref)
    assert err_tc.max() < 1e-4 * max(1.0, np.abs(y_ref).max()), err_tc.max()
    # weighted loss and gradient
    g = torch.empty(nb.NB_MLP_NPARAMS, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    nb.nb_mlp_loss_grad(pd, R_MIN, R_MAX, rd, torch.as_tensor(t.astype(np.float32), device=dev),
                        torch.as_tensor(wt.astype(np.float32), device=dev), g, loss)
    l_ref, g_ref = oracle.mlp_loss_grad(p.astype(np.float64), R_MIN, R_MAX, r32,
                                        t.astype(np.float32).astype(np.float64),
                                        wt.astype(np.float32).astype(np.float64))
    assert abs(loss.item() - l_ref) < 1e-5 * l_ref
    gd = g.cpu().numpy()
    assert np.abs(gd - g_ref).max() < 1e-4 * np.abs(g_ref).max(), np.abs(gd - g_ref).max()


@pytest.fixture(scope="module")
def trained(env):
    torch, dev, nb = env
    from paper_1306_1737_gb300 import surrogate
    r = w.surrogate_samples(1 << 20, R_MIN, R_MAX, seed=1005)
    t = oracle.ewald_factor(r, BETA)            # targets from the oracle
    t0 = time.perf_counter()
    p, losses = surrogate.train(r, BETA, t=t, steps=TRAIN_STEPS)
    dt = time.perf_counter() - t0
    return p, losses, dt


def _pair_distances_config2(n_pairs=1 << 16):
    """Distances of seeded random particle pairs of the 24,000-atom box that
    lie in [R_MIN, rc): the distance distribution the kernel meets."""
    b, _ = w.config2()
    rng = np.random.default_rng(31)
    i = rng.integers(0, b.n, 1 << 22)
    j = rng.integers(0, b.n, 1 << 22)
    d = b.xyz[i].astype(np.float64) - b.xyz[j]
    d -= b.box * np.round(d / b.box)
    r = np.sqrt((d * d).sum(1))
    r = r[(r >= R_MIN) & (r < 1.0)]
    return r[:n_pairs]


def test_training_fits_ewald_factor(env, trained):
    torch, dev, nb = env
    from paper_1306_1737_gb300 import surrogate
    p, losses, dt = trained
    assert np.all(np.isfinite(losses)) and losses[-1000:].mean() < 1e-2 * losses[:100].mean()
    held = np.concatenate([w.surrogate_samples(1 << 16, R_MIN, R_MAX, seed=99), _pair_distances_config2()])
    ref = oracle.ewald_factor(held, BETA)
    packed = torch.empty(nb.nb_mlp_packed_bytes() // 4, dtype=torch.float32, device=dev)
    nb.nb_mlp_pack(p, R_MIN, R_MAX, packed)
    y = torch.empty(held.size, dtype=torch.float32, device=dev)
    nb.nb_mlp_forward_tc(packed, torch.as_tensor(held.astype(np.float32), device=dev), y)
    err = np.abs(y.cpu().numpy() - ref)
    # the same network untrained
    p0 = torch.as_tensor(surrogate.init_params(0), device=dev)
    nb.nb_mlp_pack(p0, R_MIN, R_MAX, packed)
    nb.nb_mlp_forward_tc(packed, torch.as_tensor(held.astype(np.float32), device=dev), y)
    err0 = np.abs(y.cpu().numpy() - ref)
    print(f"\ntrained {TRAIN_STEPS} steps in {dt:.2f} s: max |dc| {err.max():.2e}, rms {np.sqrt((err**2).mean()):.2e}"
          f"; untrained max {err0.max():.2e}")
    assert err.max() < 1e-3
    assert err.max() < 1e-3 * err0.max()


def test_surrogate_forces_24k_box(env, trained):
    torch, dev, nb = env
    import gpu_path
    p, _, _ = trained
    b, prm = w.config2()
    gb = gpu_path.GpuBox(b, prm["rlist"])
    try:
        gb.grid()
        gb.build(float(np.float32(prm["rlist"])))
        nb.nb_set_surrogate(gb.ctx, p, R_MIN, R_MAX)
        fo, eo, _ = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box,
                                        oracle.make_params("ewald", float(np.float32(prm["rc"])), beta=BETA))
        res = {}
        for mode in ("ewald", "ewald_mlp"):
            pr = nb.make_params(mode, prm["rc"], beta=BETA, want_energy=False)
            f, _, _ = gb.compute(pr)
            emax, erms, rms = gpu_path.force_errors(f, fo)
            # device time of the force evaluation
            for _ in range(3):
                nb.nb_compute(gb.ctx, pr, None, gb.f)
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(10):
                nb.nb_compute(gb.ctx, pr, None, gb.f)
            z.record()
            z.synchronize()
            res[mode] = (emax, erms, a.elapsed_time(z) / 10)
        print("\n" + "; ".join(f"{k}: max|dF|/rms {v[0]:.2e}, rms {v[1]:.2e}, {v[2]:.3f} ms" for k, v in res.items()))
        assert res["ewald"][0] < 1e-4
        assert res["ewald_mlp"][0] < SURROGATE_FORCE_TOL, res["ewald_mlp"]
        # with energies requested the analytic kernel runs: energies equal the analytic ones
        f_e, e_e, _ = gb.compute(nb.make_params("ewald_mlp", prm["rc"], beta=BETA, want_energy=True))
        assert np.abs(e_e - eo).max() / np.abs(eo).max() < 1e-5
        # no network set on a fresh context: refused
    finally:
        gb.close()


def test_surrogate_needs_a_network(env, cfg1):
    torch, dev, nb = env
    import gpu_path
    b, prm = cfg1
    gb = gpu_path.GpuBox(b, prm["rlist"])
    try:
        gb.grid()
        gb.build(float(np.float32(prm["rlist"])))
        with pytest.raises(nb.NbError) as ei:
            nb.nb_compute(gb.ctx, nb.make_params("ewald_mlp", 0.9, beta=BETA, want_energy=False), None, gb.f)
        assert ei.value.status == nb.NB_ERR_STATE
    finally:
        gb.close()


def _spans_ms(nb, ctx, fn, kind, reps=10):
    """Mean device time (CUDA-event spans around the kernel) of reps calls."""
    import statistics
    fn()
    nb.nb_profile(ctx, True)
    nb.nb_profile_read(ctx)
    for _ in range(reps):
        fn()
    ms = [m for k, m in nb.nb_profile_read(ctx) if k == kind]
    nb.nb_profile(ctx, False)
    return statistics.mean(ms)


def test_what_the_network_gains_over_the_analytic_path(env, trained):
    """Gains of the trained network over the method without it, on the
    24,000-atom box: accuracy gain = (analytic max error) / (network max
    error) against the FP64 oracle, speed gain = (analytic kernel time) /
    (network kernel time).  Both are measured and asserted as they are on
    this GPU: the network loses on both (the rational fit reaches the FP32
    limit with ten multiply-adds and one reciprocal per pair, the network
    spends about two thousand operations per pair), while staying inside its
    5e-4 bound.  Against the untrained network the training gains at least
    a factor 100 in accuracy."""
    torch, dev, nb = env
    import gpu_path
    from paper_1306_1737_gb300 import surrogate
    p, _, _ = trained
    b, prm = w.config2()
    gb = gpu_path.GpuBox(b, prm["rlist"])
    try:
        gb.grid()
        gb.build(float(np.float32(prm["rlist"])))
        fo, _, _ = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box,
                                       oracle.make_params("ewald", float(np.float32(prm["rc"])), beta=BETA))
        err, ms = {}, {}
        for name, params in (("analytic", None), ("trained", p), ("untrained", surrogate.init_params(0))):
            mode = "ewald" if params is None else "ewald_mlp"
            if params is not None:
                nb.nb_set_surrogate(gb.ctx, torch.as_tensor(params, device=dev), R_MIN, R_MAX)
            pr = nb.make_params(mode, prm["rc"], beta=BETA, want_energy=False)
            f, _, _ = gb.compute(pr)
            err[name] = gpu_path.force_errors(f, fo)[0]
            ms[name] = _spans_ms(nb, gb.ctx, lambda: nb.nb_compute(gb.ctx, pr, None, gb.f), nb.NB_KERNEL_FORCE)
        acc_gain = err["analytic"] / err["trained"]
        speed_gain = ms["analytic"] / ms["trained"]
        train_gain = err["untrained"] / err["trained"]
        print(f"\nmax|dF|/rms: analytic {err['analytic']:.2e}, network {err['trained']:.2e} "
              f"(untrained {err['untrained']:.2e}); force kernel: analytic {ms['analytic']:.3f} ms, "
              f"network {ms['trained']:.3f} ms; gains of the network: accuracy x{acc_gain:.3f}, "
              f"speed x{speed_gain:.3f}; of training: accuracy x{train_gain:.0f}")
        assert err["analytic"] < 1e-4 and err["trained"] < SURROGATE_FORCE_TOL
        assert acc_gain < 1.0 and speed_gain < 1.0
        assert train_gain > 100.0
    finally:
        gb.close()
