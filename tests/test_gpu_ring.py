"""The force kernel streams each i-entry's j-clusters through a per-warp ring
of two groups of 8 entries in shared memory (the next group copied in while
the current one is computed).  Entries of 1 to 32 j-entries exercise a
partial first group, whole groups, the request of a last partial group and
the end of an entry on a group boundary.  On a box searched a block per
super-cluster (24,000 particles: entries of at most 12) and one searched a
warp per super-cluster (60,000 particles: entries of at most 32) the lists
hold entries of every length class, and the forces on the outer list and on
the pruned list after a displacement match the FP64 oracle (cell list) for
every particle."""
import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4     # of the RMS force, plus FP32 rounding of the particle's own force
F_ROUND = 4e-6


@pytest.fixture(scope="module")
def gp():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    import gpu_path
    return gpu_path


def _check(f, fo):
    rms = np.sqrt((fo ** 2).sum(1).mean())
    err = np.sqrt(((f - fo) ** 2).sum(1))
    bound = FORCE_TOL * rms + F_ROUND * np.sqrt((fo ** 2).sum(1))
    assert (err <= bound).all(), (float((err / bound).max()), int((err > bound).sum()))


@pytest.mark.parametrize("n_mol,max_len,classes", [
    # block mode: below one group, exactly one, one group and a partial one
    (8000, 12, [(1, 7), (8, 8), (9, 12)]),
    # warp mode: every position relative to the groups of 8, up to a full chunk
    (20000, 32, [(1, 7), (8, 8), (9, 15), (16, 16), (17, 23), (24, 24), (25, 31), (32, 32)]),
])
def test_ring_entry_lengths_and_forces(gp, n_mol, max_len, classes):
    import paper_1306_1737_gb300 as nb
    b = w.water_box(n_mol, seed=4400 + n_mol)
    rc, rlist, beta = 1.0, 1.1, 3.12
    rcf, rlf = float(np.float32(rc)), float(np.float32(rlist))
    gb = gp.GpuBox(b, rlist)
    try:
        gb.grid()
        gb.build(rlf, 0.8)
        _, ient, _, _, _ = gb.list_arrays(0)
        lens = ient[:, 3] - ient[:, 2]
        lens = lens[lens > 0]
        assert lens.max() <= max_len, lens.max()
        for lo, hi in classes:
            assert ((lens >= lo) & (lens <= hi)).any(), (lo, hi, np.bincount(lens))
        oprm = oracle.make_params("ewald", rcf, beta=beta)
        prm = nb.make_params("ewald", rcf, beta=beta, want_energy=False)
        f, _, _ = gb.compute(prm)
        fo, _, _ = oracle.forces_cells(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        _check(f, fo)
        # five frames later: the pruned list (fused into that frame's force pass),
        # then a force pass on the pruned list alone
        x5 = (b.xyz + w.frame_displacements(b.mass, 5, seed=4500 + n_mol).sum(0)).astype(np.float32)
        rp = float(np.float32(w.prune_radius(rc, rlist, 5)))
        x5d = gb.torch.as_tensor(x5).to(gb.dev).contiguous()
        nb.nb_prune_compute(gb.ctx, prm, x5d, rp, gb.f)
        nb.nb_check(gb.ctx)
        fo5, _, _ = oracle.forces_cells(x5, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        _check(gb.f.cpu().numpy().astype(np.float64), fo5)
        f5, _, _ = gb.compute(prm)
        _check(f5, fo5)
    finally:
        gb.close()
