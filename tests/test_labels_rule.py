"""CPU checks of the label comparison rule used by the GPU parity tests
(tests/_labels.py): a disagreement is allowed only at a tie node of the
oracle's solve that is next to a patch boundary of the oracle's labels."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._labels import assert_labels, boundary_adjacent, grid_shape, tie_mask


def test_boundary_adjacency_on_a_hand_made_map():
    lab = np.array([[-1, -1, -1, -1, -1],
                    [-1, 0, 0, 1, -1],
                    [-1, 0, 0, 1, -1],
                    [-1, 0, 0, 0, -1],
                    [-1, -1, -1, -1, -1]], np.int8)
    near = boundary_adjacent(lab.reshape(-1), lab.shape).reshape(lab.shape)
    want = np.array([[0, 0, 0, 0, 0],
                     [0, 0, 1, 1, 0],
                     [0, 0, 1, 1, 0],
                     [0, 0, 1, 1, 0],
                     [0, 0, 0, 0, 0]], bool)
    # the ghost ring (-1) is not a patch; diagonal neighbours count (3x3 stencil)
    assert np.array_equal(near, want)


def test_boundary_adjacency_3d():
    lab = np.zeros((4, 4, 4), np.int8)
    lab[2:, :, :] = 1
    near = boundary_adjacent(lab.reshape(-1), lab.shape).reshape(lab.shape)
    assert near[1].all() and near[2].all() and not near[0].any() and not near[3].any()


@pytest.fixture(scope="module")
def solved():
    p = W.sincos2d(1, n=65, n_coarse=17, n_targets=3, radius=0.2)
    return p, oracle.patchy_solve(p, tol=1e-12, keep_phi=True)


def test_rule_accepts_identical_labels(solved):
    p, ref = solved
    agree, nbad = assert_labels(ref.labels.copy(), ref, p)
    assert agree == 1.0 and nbad == 0


def test_rule_rejects_a_flip_inside_a_patch(solved):
    p, ref = solved
    near = boundary_adjacent(ref.labels, grid_shape(p))
    inner = np.nonzero((ref.labels >= 0) & ~near)[0]
    lab = ref.labels.copy()
    lab[inner[len(inner) // 2]] = (lab[inner[len(inner) // 2]] + 1) % p.n_patches
    with pytest.raises(AssertionError, match="not tie nodes"):
        assert_labels(lab, ref, p)


def test_rule_rejects_a_flip_at_a_boundary_node_that_is_not_a_tie(solved):
    p, ref = solved
    near = boundary_adjacent(ref.labels, grid_shape(p))
    tie = tie_mask(ref, p)
    cand = np.nonzero(near & ~tie)[0]
    assert cand.size > 0
    lab = ref.labels.copy()
    i = cand[0]
    lab[i] = (lab[i] + 1) % p.n_patches
    with pytest.raises(AssertionError, match="not tie nodes"):
        assert_labels(lab, ref, p)


def test_rule_accepts_a_flip_at_a_tie_next_to_a_boundary():
    # two equal disks mirrored about x1 = 0 with c = 1: the colours tie (1/2
    # each) on the bisector, which is the patch boundary
    p = W.sincos2d(0, n=65, n_coarse=17, n_targets=2, amplitude=0.0).with_(
        targets=np.array([[-1.0, 0.3, 0.2], [1.0, 0.3, 0.2]]))
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    near = boundary_adjacent(ref.labels, grid_shape(p))
    tie = tie_mask(ref, p)
    cand = np.nonzero(near & tie)[0]
    assert cand.size > 0
    lab = ref.labels.copy()
    i = cand[0]
    lab[i] = (lab[i] + 1) % p.n_patches
    assert_labels(lab, ref, p)


def test_rule_rejects_too_many_disagreements(solved):
    p, ref = solved
    lab = ref.labels.copy()
    idx = np.nonzero(lab >= 0)[0][: max(2, lab.size // 500)]
    lab[idx] = (lab[idx] + 1) % p.n_patches
    with pytest.raises(AssertionError, match="agreement"):
        assert_labels(lab, ref, p)


@pytest.mark.parametrize("family", ["sincos2d", "brockett3d"])
def test_restated_feedback_chain_reproduces_the_oracle_colours(family):
    """The chain the tie rule walks (tests/_labels.py: feet of the oracle's
    feedback, Q1 weights) is the one of Eq. (HJBridotta_discreta): its
    absorption probabilities, from a direct sparse solve, are the oracle's
    colours."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    from tests._labels import feedback_graph, reaches

    p = W.sincos2d(2, n=129, n_coarse=33) if family == "sincos2d" else W.brockett3d(n=21, n_coarse=11)
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    src, dst, N, w = feedback_graph(p, ref.astar)
    kind, part, _ = oracle.setup(p)
    for j in range(p.n_patches):
        tgt = (kind == oracle.TARGET) & (part == j)
        live = reaches(src, dst, N, tgt) & ~tgt
        ids = np.nonzero(live)[0]
        phi = np.where(tgt, 1.0, 0.0)
        if ids.size:
            P = sp.csr_matrix((w, (src, dst)), shape=(N, N))[ids]
            A = sp.identity(ids.size, format="csc") - P[:, ids].tocsc()
            b = np.asarray(P[:, np.nonzero(tgt)[0]].sum(axis=1)).ravel()
            phi[ids] = spl.spsolve(A, b)
        free = ref.astar >= 0
        assert np.abs(phi[free] - ref.phi[j][free]).max() < 1e-8


def test_hit_probability_on_a_small_chain():
    from tests._labels import hit_probability

    # 0 -> 1 (1/2), 0 -> 2 (1/2); 1 -> 3 (seed); 2 -> 2 (trap); 4 isolated
    src = np.array([0, 0, 1, 2])
    dst = np.array([1, 2, 3, 2])
    w = np.array([0.5, 0.5, 1.0, 1.0])
    seeds = np.array([False, False, False, True, False])
    pi = hit_probability(src, dst, 5, w, seeds)
    assert np.allclose(pi, [0.5, 1.0, 0.0, 1.0, 0.0])
