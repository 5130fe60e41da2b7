"""GPU parity of the patch compaction (Sec. 3: the patches assembled from the
Step 3.1 labels before Step 3.2): the per-patch tile and node lists against
lists formed here from the oracle's node kinds, and the per-patch node counts
against the oracle's own counts.

- Exact, element by element: patch j's node list is every free node (oracle
  kind FREE) with GPU label j, ordered by tile and x fastest inside a tile;
  its tile list is the sorted set of those tiles with their node counts.
- Against the oracle's counts: gpu_count[j] - oracle_count[j] equals the
  number of free nodes labelled j by the GPU and not by the oracle minus the
  reverse (zero when the labels agree); the labels themselves follow the
  comparison rule of tests/_labels.py.
- Every patch retired with its FP64 sup-norm change at most tol.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._labels import assert_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    return P


def _expected_lists(p, free, lab, R):
    side = 8 if p.dim == 3 else 32
    n = [int(v) for v in p.n[: p.dim]]
    idx = np.arange(int(np.prod(n)))
    coords = []
    rest = idx
    for a in range(p.dim):
        coords.append(rest % n[a])
        rest = rest // n[a]
    nt = [(n[a] - 2 + side - 1) // side for a in range(p.dim)]
    tc = [(coords[a] - 1) // side for a in range(p.dim)]
    lc = [(coords[a] - 1) % side for a in range(p.dim)]
    tile = tc[0] + nt[0] * tc[1] + (nt[0] * nt[1] * tc[2] if p.dim == 3 else 0)
    local = lc[0] + side * lc[1] + (side * side * lc[2] if p.dim == 3 else 0)
    out = []
    for j in range(R):
        sel = np.nonzero(free & (lab == j))[0]
        order = np.lexsort((local[sel], tile[sel]))
        nodes = sel[order]
        tiles, counts = np.unique(tile[nodes], return_counts=True)
        out.append((nodes, tiles, counts))
    return out


def _check(pkg, p, dirichlet=False):
    flags = pkg.HJBP_FLAG_DIRICHLET if dirichlet else 0
    with pkg.Plan(p, flags=flags) as plan:
        assert plan.solve() == 0
        lab = plan.labels()
        st = plan.stats()
        L = plan.patch_lists()
    R = p.n_patches
    kind, _, _ = oracle.setup(p)
    free = kind == oracle.FREE
    exp = _expected_lists(p, free, lab, R)
    to, no = L["tile_offsets"], L["node_offsets"]
    assert to[0] == 0 and no[0] == 0 and np.all(np.diff(to) >= 0) and np.all(np.diff(no) >= 0)
    for j, (nodes, tiles, counts) in enumerate(exp):
        assert np.array_equal(L["node_ids"][no[j]:no[j + 1]], nodes), f"node list of patch {j}"
        assert np.array_equal(L["tile_ids"][to[j]:to[j + 1]], tiles), f"tile list of patch {j}"
        assert np.array_equal(L["tile_nodes"][to[j]:to[j + 1]], counts), f"tile counts of patch {j}"
        assert st["patch_nodes"][j] == nodes.size and st["patch_tiles"][j] == tiles.size
        assert st["residual_patch"][j] <= p.tol
    # against the oracle's own per-patch counts
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=dirichlet)
    assert_labels(lab, ref, p)
    for j in range(R):
        gain = int(np.sum(free & (lab == j) & (ref.labels != j)))
        loss = int(np.sum(free & (ref.labels == j) & (lab != j)))
        assert st["patch_nodes"][j] - ref.stats["patch_nodes"][j] == gain - loss


@pytest.mark.parametrize("seed,n,nc,R,radius", [(0, 129, 33, 4, 0.2), (2, 257, 33, 4, 0.05)])
def test_patch_lists_2d(pkg, seed, n, nc, R, radius):
    _check(pkg, W.sincos2d(seed, n=n, n_coarse=nc, n_targets=R, radius=radius))


def test_patch_lists_2d_obstacles_dirichlet(pkg):
    _check(pkg, W.eikonal_obstacles(n=161, n_coarse=41, parts=8), dirichlet=True)


def test_patch_lists_2d_non_square(pkg):
    p = W.sincos2d(2, n=129, n_coarse=33, n_targets=2, radius=0.12).with_(
        n=(129, 81, 1), hi=(2.0, 1.5, 0.0), lo=(-2.0, -1.0, 0.0), n_coarse=(33, 21, 1),
        targets=np.array([[1.0, 0.5, 0.12], [-0.8, -0.3, 0.12]]))
    _check(pkg, p)


def test_patch_lists_3d(pkg):
    _check(pkg, W.sin3d(0, n=41, n_coarse=11, n_targets=4, radius=0.12))


def test_patch_lists_64_patches(pkg):
    _check(pkg, W.eikonal_sectors(n=129, n_coarse=33, parts=64))


def test_patch_lists_before_a_solve_is_an_error(pkg):
    p = W.sincos2d(0, n=65, n_coarse=17, n_targets=2, radius=0.2)
    with pkg.Plan(p) as plan:
        with pytest.raises(pkg.HjbpError) as ei:
            plan.patch_lists()
        assert ei.value.status == pkg.HJBP_ESTATE
