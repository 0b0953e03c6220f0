"""Training and installing the learned Ewald force factor (argument
marshalling only: targets, training steps and evaluation run in the
library's kernels).

The network (1 -> 32 -> 32 -> 1, SiLU) stands in for
c(r) = erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2), the factor of
the real-space Ewald force f qq c(r) / r^2 (Sec. 3.2).  Training minimises
the weighted squared error with weights 1 / max(r, 0.1 nm)^2, which tracks
the pair force error f qq dc / r^2 at the distances where pairs occur.
"""
from __future__ import annotations

import math

import numpy as np

import paper_1306_1737_gb300 as nb

R_MIN = 0.05
R_MAX = 1.0
H = 32


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters: layer 1 spread over the input range
    (W1 ~ N(0, 3^2), b1 ~ U(-3, 3)), layers 2 and 3 ~ N(0, 1/32), zero
    biases."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    p = np.zeros(nb.NB_MLP_NPARAMS, np.float32)
    p[0:H] = rng.standard_normal(H) * 3.0
    p[H:2 * H] = rng.uniform(-3.0, 3.0, H)
    p[2 * H:2 * H + H * H] = rng.standard_normal(H * H) / math.sqrt(H)
    p[2 * H + H * H + H:2 * H + H * H + 2 * H] = rng.standard_normal(H) / math.sqrt(H)
    return p


def loss_weights(r: np.ndarray) -> np.ndarray:
    w = 1.0 / np.maximum(r, 0.1) ** 2
    return (w / w.mean()).astype(np.float32)


def train(r, beta: float, t=None, steps: int = 60000, batch: int = 8192, lr_max: float = 3e-3,
          lr_min: float = 1e-5, seed: int = 0, device: int = 0, r_min: float = R_MIN, r_max: float = R_MAX,
          params=None):
    """Train on distances r (host array).  t: targets (host array); None
    computes c(r) in FP64 on the GPU.  Returns (params [1153] float32 device
    tensor, per-step minibatch losses as a host array)."""
    import torch
    dev = torch.device("cuda", device)
    r64 = torch.as_tensor(np.asarray(r, dtype=np.float64), device=dev)
    if t is None:
        t64 = torch.empty_like(r64)
        nb.nb_ewald_factor(r64, beta, t64)
        t32 = t64.float()
    else:
        t32 = torch.as_tensor(np.asarray(t, dtype=np.float32), device=dev)
    r32 = r64.float()
    w32 = torch.as_tensor(loss_weights(np.asarray(r, dtype=np.float64)), device=dev)
    p = torch.as_tensor(init_params(seed) if params is None else np.asarray(params, np.float32), device=dev).clone()
    state = torch.zeros(3 * nb.NB_MLP_NPARAMS, dtype=torch.float32, device=dev)
    losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    nb.nb_mlp_train(p, state, r_min, r_max, r32, t32, w32, batch, steps, 0, steps, lr_max, lr_min, losses)
    torch.cuda.synchronize()
    return p, losses.cpu().numpy()[:steps]
