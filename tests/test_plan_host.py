"""The workspace plan on the host (nb_workspace_bytes: no context, no
device): sizes grow with the particles, the list radius and the capacity
factor; a batch needs at least what its boxes need alone; plans beyond the
32-bit indices, the 27-bit cluster field of a j-entry word, the grid's
column limit or with unusable box edges are refused with their status."""
import pytest

import paper_1306_1737_gb300 as nb
from paper_1306_1737_gb300 import build as nbbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    nbbuild.build()
    return nb.load()


def _status(*args, **kw):
    try:
        nb.nb_workspace_bytes(*args, **kw)
    except nb.NbError as e:
        return e.status
    return nb.NB_OK


@pytest.mark.parametrize("C", [8, 4])
def test_sizes_grow_with_the_plan(C):
    L = [6.21] * 3
    base = nb.nb_workspace_bytes(C, 24000, L, 1.1, 2)
    assert base > 0 and base % 256 == 0
    assert nb.nb_workspace_bytes(C, 24000, L, 1.1, 2) == base          # deterministic
    assert nb.nb_workspace_bytes(C, 30000, L, 1.1, 2) > base
    assert nb.nb_workspace_bytes(C, 24000, L, 1.3, 2) > base
    assert nb.nb_workspace_bytes(C, 24000, L, 1.1, 2, list_factor=3.0) > base
    # a batch of one is the single box; two boxes need at least each alone
    assert nb.nb_workspace_bytes(C, [24000], [L], 1.1, 2) == base
    other = nb.nb_workspace_bytes(C, 5000, [3.7] * 3, 1.1, 2)
    assert nb.nb_workspace_bytes(C, [24000, 5000], [L, [3.7] * 3], 1.1, 2) >= max(base, other)


def test_clusters_of_four_hold_longer_lists():
    # the 4x4 list has more j-entries per particle than the 8x8 one (Sec. 2.2, Table 1)
    assert nb.nb_workspace_bytes(4, 24000, [6.21] * 3, 1.1, 2) > nb.nb_workspace_bytes(8, 24000, [6.21] * 3, 1.1, 2)


def test_refused_plans():
    L = (1.1e9 / 0.05) ** (1.0 / 3.0)
    # 1.1e9 particles at 0.05 nm^-3, clusters of 8: 1.38e8 clusters do not fit 27 bits
    assert _status(8, 1_100_000_000, [L, L, L], 1.1, 2) == nb.NB_ERR_CAPACITY
    # the same at clusters of 4: more than 2^31 list entries
    assert _status(4, 600_000_000, [L, L, L], 1.1, 2) == nb.NB_ERR_CAPACITY
    # a slab far thinner than the column spacing
    assert _status(8, 1000, [2.2e6, 2.2e6, 2e-12], 1.1, 2) == nb.NB_ERR_CAPACITY
    assert _status(8, 10, [1e31, 1.0, 1.0], 1.1, 2) == nb.NB_ERR_BOX
    assert _status(8, 10, [0.0, 1.0, 1.0], 1.1, 2) == nb.NB_ERR_BOX
    assert _status(8, 10, [float("nan"), 1.0, 1.0], 1.1, 2) == nb.NB_ERR_BOX
    assert _status(8, [1_500_000_000] * 2, [[1e3] * 3] * 2, 1.1, 2) == nb.NB_ERR_ARG
    assert _status(8, [10] * 4097, [[2.0] * 3] * 4097, 1.1, 2) == nb.NB_ERR_ARG     # at most 4096 boxes
    assert _status(8, 10, [2.0] * 3, 1.1, 65) == nb.NB_ERR_ARG                      # at most 64 LJ types
    assert _status(8, 10, [2.0] * 3, 0.0, 2) == nb.NB_ERR_ARG
    assert _status(8, 10, [2.0] * 3, 1.1, 2, list_factor=0.5) == nb.NB_ERR_ARG
    assert _status(8, -1, [2.0] * 3, 1.1, 2) == nb.NB_ERR_ARG
    assert _status(6, 10, [2.0] * 3, 1.1, 2) == nb.NB_ERR_ARG
