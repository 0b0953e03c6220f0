"""Helpers for the GPU tests: drive the C ABI through the Python binding and
read results back as numpy; compare with the oracle's canonical forms."""
from __future__ import annotations

import math

import numpy as np

import paper_1306_1737_gb300 as nb


def torch_dev():
    import torch
    return torch, torch.device("cuda", 0)


class GpuBox:
    """One box on the GPU through the C ABI."""

    def __init__(self, b, rlist_max, C=8, comb=nb.NB_COMB_LB, list_factor=0.0):
        torch, dev = torch_dev()
        self.torch, self.dev, self.b, self.C = torch, dev, b, C
        self.c6c12 = nb.nb_lj_combine(b.sigma, b.eps, comb)
        self.cx = nb.Context(b.n, b.box, rlist_max, b.q, b.types, self.c6c12, cluster_size=C,
                             list_factor=list_factor)
        self.ctx = self.cx.ctx
        self.xyz = torch.as_tensor(b.xyz).to(dev).contiguous()
        self.excl_off = torch.as_tensor(b.excl_off).to(dev)
        self.excl_idx = torch.as_tensor(b.excl_idx).to(dev)
        self.f = torch.zeros((b.n, 3), dtype=torch.float32, device=dev)
        self.e = torch.zeros(2, dtype=torch.float64, device=dev)
        self.vir = torch.zeros(9, dtype=torch.float64, device=dev)

    def grid(self, xyz=None):
        x = self.xyz if xyz is None else self.torch.as_tensor(xyz).to(self.dev).contiguous()
        nb.nb_grid_put(self.ctx, x, self.b.box)
        return nb.nb_check(self.ctx)

    def build(self, rlist, rbb=0.0, excl=True):
        excl = excl and self.b.excl_idx.size > 0      # an empty CSR is passed as no exclusions
        nb.nb_pairlist_build(self.ctx, rlist, rbb, self.excl_off if excl else None,
                             self.excl_idx if excl else None)
        return nb.nb_check(self.ctx)

    def prune(self, r_prune, xyz=None):
        x = None if xyz is None else self.torch.as_tensor(xyz).to(self.dev).contiguous()
        nb.nb_prune(self.ctx, x, r_prune)
        return nb.nb_check(self.ctx)

    def compute(self, params, xyz=None):
        x = None if xyz is None else self.torch.as_tensor(xyz).to(self.dev).contiguous()
        nb.nb_compute(self.ctx, params, x, self.f, self.e, self.vir)
        nb.nb_check(self.ctx)
        return (self.f.cpu().numpy().astype(np.float64), self.e.cpu().numpy(),
                self.vir.cpu().numpy().reshape(3, 3))

    def grid_arrays(self):
        torch = self.torch
        info = nb.nb_check(self.ctx)
        ns = info.n_clusters * self.C
        ncol = info.nx * info.ny
        aos = torch.zeros(ns, dtype=torch.int32, device=self.dev)
        soa = torch.zeros(self.b.n, dtype=torch.int32, device=self.dev)
        ccs = torch.zeros(ncol + 1, dtype=torch.int32, device=self.dev)
        xyzq = torch.zeros((ns, 4), dtype=torch.float32, device=self.dev)
        ts = torch.zeros(ns, dtype=torch.int32, device=self.dev)
        bb = torch.zeros((info.n_clusters, 6), dtype=torch.float32, device=self.dev)
        coa = torch.zeros(self.b.n, dtype=torch.int32, device=self.dev)
        sci = torch.zeros((max(info.n_superclusters, 1), 2), dtype=torch.int32, device=self.dev)
        nb.nb_get_grid(self.ctx, aos, soa, ccs, xyzq, ts, bb, coa, sci)
        torch.cuda.synchronize()
        return dict(info=info, atom_of_slot=aos.cpu().numpy(), slot_of_atom=soa.cpu().numpy(),
                    col_clu_start=ccs.cpu().numpy(), xyzq=xyzq.cpu().numpy(),
                    type_slot=ts.cpu().numpy(), bb=bb.cpu().numpy(), col_of_atom=coa.cpu().numpy(),
                    sc_info=sci.cpu().numpy()[: info.n_superclusters])

    def list_arrays(self, which=0):
        """(info, i-entries [ni, 4], j-words [nj], masks [S, nj], super-cluster
        table [nsc, 2]) of the outer (0) or pruned (1) list."""
        torch = self.torch
        info = nb.nb_check(self.ctx)
        ni, nj, S = int(info.n_ientries), int(info.n_jentries), int(info.super_size)
        ient = torch.zeros((max(ni, 1), 4), dtype=torch.int32, device=self.dev)
        cj = torch.zeros(max(nj, 1), dtype=torch.int32, device=self.dev)
        mask = torch.zeros((S, max(nj, 1)), dtype=torch.int64, device=self.dev)
        nb.nb_get_list(self.ctx, which, ient, cj, mask)
        sci = torch.zeros((max(info.n_superclusters, 1), 2), dtype=torch.int32, device=self.dev)
        nb.nb_get_grid(self.ctx, sc_info=sci)
        torch.cuda.synchronize()
        masks = mask.cpu().numpy().view(np.uint64)
        if nj < masks.shape[1]:
            masks = masks[:, :nj]
        return info, ient.cpu().numpy()[:ni], cj.cpu().numpy()[:nj], masks, \
            sci.cpu().numpy()[: info.n_superclusters]

    def close(self):
        self.cx.close()


SUPER_SHIFT = 27


def expand_keys(ient, cj, masks, sc_info):
    """GPU super-cluster list -> arrays (a, b, s, mask) of cluster-pair keys."""
    lens = ient[:, 3] - ient[:, 2]
    starts = np.cumsum(lens) - lens
    idx = np.arange(int(lens.sum())) - np.repeat(starts, lens) + np.repeat(ient[:, 2], lens)
    q = np.repeat(ient[:, 0], lens)
    s = np.repeat(ient[:, 1], lens)
    w = cj[idx].astype(np.int64) & 0xFFFFFFFF
    b = (w & ((1 << SUPER_SHIFT) - 1)).astype(np.int64)
    bits = w >> SUPER_SHIFT
    g0 = sc_info[q, 0].astype(np.int64)
    A, B, Sh, M = [], [], [], []
    for k in range(masks.shape[0]):
        on = ((bits >> k) & 1).astype(bool)
        A.append(g0[on] + k)
        B.append(b[on])
        Sh.append(s[on])
        M.append(masks[k][idx[on]])
    return (np.concatenate(A), np.concatenate(B), np.concatenate(Sh), np.concatenate(M))


def canonical_keys(ient, cj, masks, sc_info):
    """GPU list -> ({(a, b, s): mask} with a <= b, number of duplicate keys)."""
    a, b, s, m = expand_keys(ient, cj, masks, sc_info)
    assert np.all(a <= b)
    keys = list(zip(a.tolist(), b.tolist(), s.tolist()))
    out = dict(zip(keys, m.tolist()))
    return out, len(keys) - len(out)


def force_errors(f_gpu, f_ref):
    rms = math.sqrt((f_ref ** 2).sum(1).mean())
    d = np.sqrt(((f_gpu - f_ref) ** 2).sum(1))
    return d.max() / rms, math.sqrt((d ** 2).mean()) / rms, rms
