"""The label comparison of the parity tests (Step 3.1, Eq. (proiezionecolore)
and Remark 3.1), shared by every test that compares patch labels with the
oracle's.

Rule: labels agree on at least 99.9 % of the nodes, and every node where they
disagree is BOTH a tie node of the oracle's solve (reading c10: the coarse
feedback's two best controls within 1e-9 max(1, U0), or max_j phi^j within
1e-6 of 1/2, or the two largest colours within 1e-6) AND adjacent to a patch
boundary of the oracle's label map (a node of another patch in its 3^d
neighbourhood).  The ghost ring and unreachable nodes (label -1) are not a
patch.
"""
import numpy as np


def tie_mask(ref) -> np.ndarray:
    """Tie nodes of an oracle patchy solve run with ``keep_phi=True``."""
    if ref.phi is None:
        raise ValueError("the oracle solve needs keep_phi=True for the tie mask")
    u0 = np.where(np.isfinite(ref.u0), ref.u0, 1.0)
    tie = ref.gap < 1e-9 * np.maximum(1.0, u0)
    phimax = ref.phi.max(axis=0)
    tie |= np.abs(phimax - 0.5) < 1e-6
    if ref.phi.shape[0] >= 2:
        srt = np.sort(ref.phi, axis=0)
        tie |= (srt[-1] - srt[-2]) < 1e-6
    return tie


def grid_shape(p):
    """numpy shape of a node array (x1 fastest)."""
    return tuple(int(v) for v in reversed(p.n[: p.dim]))


def boundary_adjacent(labels: np.ndarray, shape) -> np.ndarray:
    """Nodes with a patch label (>= 0) whose 3^d neighbourhood holds a node of
    another patch."""
    lab = labels.reshape(shape).astype(np.int16)
    d = lab.ndim
    pad = np.pad(lab, 1, constant_values=-1)
    out = np.zeros(lab.shape, bool)
    for off in np.ndindex(*([3] * d)):
        if all(o == 1 for o in off):
            continue
        sl = tuple(slice(o, o + s) for o, s in zip(off, lab.shape))
        nb = pad[sl]
        out |= (nb >= 0) & (lab >= 0) & (nb != lab)
    return out.reshape(-1)


def check_labels(lab: np.ndarray, ref_labels: np.ndarray, tie: np.ndarray, shape, min_agree: float = 0.999):
    """Assert the rule; returns (agreement, disagreements)."""
    bad = lab != ref_labels
    agree = 1.0 - bad.mean()
    assert agree >= min_agree, f"label agreement {agree:.6f} < {min_agree}"
    if bad.any():
        near = boundary_adjacent(ref_labels, shape)
        ok = tie & near
        assert np.all(ok[bad]), (
            f"{int(np.sum(bad & ~ok))} of {int(bad.sum())} label disagreements are not tie nodes next to a patch "
            f"boundary (not tie: {int(np.sum(bad & ~tie))}, not adjacent: {int(np.sum(bad & ~near))})")
    return agree, int(bad.sum())


def assert_labels(lab: np.ndarray, ref, p, min_agree: float = 0.999):
    """The rule against an oracle patchy solve of problem ``p`` (keep_phi=True)."""
    return check_labels(lab, ref.labels, tie_mask(ref), grid_shape(p), min_agree)
