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
    tie = tie_mask(ref)
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
    tie = tie_mask(ref)
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
