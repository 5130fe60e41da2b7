"""The label comparison of the parity tests (Step 3.1, Eq. (proiezionecolore)
and Remark 3.1), shared by every test that compares patch labels with the
oracle's.

Rule: labels agree on at least 99.9 % of the nodes, and every node where they
disagree is BOTH a tie node of the oracle's solve AND adjacent to a patch
boundary of the oracle's label map (a node of another patch in its 3^d
neighbourhood).  The ghost ring and unreachable nodes (label -1) are not a
patch.

Tie nodes (reading c10): the coarse feedback's two best controls within
1e-9 max(1, U0) (a feedback tie: Eq. feedbackcontrol's argmin is decided by
rounding), max_j phi^j within 1e-6 of 1/2 or the two largest colours within
1e-6 (a projection tie), and every node whose colours a feedback tie can
reorder.  The colours of Eq. (HJBridotta_discreta) at node i are absorption
probabilities of the feedback chain started at i; if pi_i is the probability
that the chain passes through a feedback-tie node, the tied choice moves each
colour at i by at most pi_i, so the label at i is decided by the method only
where its two largest colours differ by more than 2 pi_i (+ 1e-6).
"""
import numpy as np


def feedback_graph(p, astar):
    """Edges i -> j of the feedback chain with their Q1 weights: j a
    positive-weight corner of the foot x_i + k f(x_i, a*_i)/|f| of a node
    with a defined feedback (restated here: unit direction of f per
    dynamics, grid coordinates).  Returns (src, dst, N, weights)."""
    from tests import _indep as I

    n = np.array(p.n[: p.dim], np.int64)
    N = int(np.prod(n))
    nodes = np.nonzero(astar >= 0)[0]
    a = astar[nodes]
    idx = np.stack([(nodes // int(np.prod(n[:d]))) % n[d] for d in range(p.dim)], axis=1)
    if p.dyn == "brockett":
        x = np.array(p.lo[: p.dim]) + idx * p.spacing
        ctl = np.asarray(p.controls, float)[a]
        f = np.stack([ctl[:, 0], ctl[:, 1], x[:, 0] * ctl[:, 1] - x[:, 1] * ctl[:, 0]], axis=1)
        d = f / np.linalg.norm(f, axis=1)[:, None]
        d[np.abs(d) < 1e-15] = 0.0
    else:
        dirs, _ = I.control_steps(p)
        d = dirs[a]
    xi = idx + d
    base = np.clip(np.floor(xi).astype(np.int64), 0, n - 2)
    t = xi - base
    src, dst, wts = [], [], []
    for bits in range(1 << p.dim):
        w = np.ones(nodes.size)
        j = np.zeros(nodes.size, np.int64)
        mul = 1
        for dd in range(p.dim):
            b = (bits >> dd) & 1
            w *= t[:, dd] if b else 1.0 - t[:, dd]
            j += (base[:, dd] + b) * mul
            mul *= int(n[dd])
        pos = w > 0
        src.append(nodes[pos])
        dst.append(j[pos])
        wts.append(w[pos])
    return np.concatenate(src), np.concatenate(dst), N, np.concatenate(wts)


def reaches(src, dst, N, seeds) -> np.ndarray:
    """Nodes from which the graph src -> dst reaches a seed node."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order

    seeds = np.nonzero(seeds)[0]
    out = np.zeros(N, bool)
    if seeds.size == 0:
        return out
    # reversed edges dst -> src, plus a source node N with an edge to every seed
    rows = np.concatenate([dst, np.full(seeds.size, N)])
    cols = np.concatenate([src, seeds])
    g = sp.csr_matrix((np.ones(rows.size, np.int8), (rows, cols)), shape=(N + 1, N + 1))
    order = breadth_first_order(g, N, directed=True, return_predecessors=False)
    out[order[order < N]] = True
    return out


def hit_probability(src, dst, N, w, seeds) -> np.ndarray:
    """pi_i = P(the chain src -> dst with weights w, started at i, visits a
    seed node): 1 on the seeds, pi = P pi elsewhere, 0 where no seed is
    reachable (solved directly on the nodes that reach a seed)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    pi = np.zeros(N)
    live = reaches(src, dst, N, seeds) & ~seeds
    pi[seeds] = 1.0
    if not live.any():
        return pi
    loc = -np.ones(N, np.int64)
    ids = np.nonzero(live)[0]
    loc[ids] = np.arange(ids.size)
    rows = live[src]
    P = sp.csr_matrix((w[rows], (loc[src[rows]], dst[rows])), shape=(ids.size, N))
    A = sp.identity(ids.size, format="csr") - P[:, ids]
    b = np.asarray(P[:, np.nonzero(seeds)[0]].sum(axis=1)).ravel()
    pi[ids] = np.clip(spl.spsolve(A.tocsc(), b), 0.0, 1.0)
    return pi


def tie_mask_from(p, u0, gap, astar, phi) -> np.ndarray:
    """Tie nodes from the oracle's U_P^(0), feedback gap, feedback and colours."""
    u0f = np.where(np.isfinite(u0), u0, 1.0)
    tie_a = (gap < 1e-9 * np.maximum(1.0, u0f)) & (astar >= 0)
    phimax = phi.max(axis=0)
    tie = tie_a | (np.abs(phimax - 0.5) < 1e-6)
    srt = np.sort(phi, axis=0) if phi.shape[0] >= 2 else None
    top2 = (srt[-1] - srt[-2]) if srt is not None else np.ones(phi.shape[1])
    tie |= top2 < 1e-6
    if tie_a.any():
        src, dst, N, w = feedback_graph(p, astar)
        pi = hit_probability(src, dst, N, w, tie_a)
        tie |= top2 <= 2.0 * pi + 1e-6
    return tie


def tie_mask(ref, p) -> np.ndarray:
    """Tie nodes of an oracle patchy solve of problem p run with ``keep_phi=True``."""
    if ref.phi is None:
        raise ValueError("the oracle solve needs keep_phi=True for the tie mask")
    return tie_mask_from(p, ref.u0, ref.gap, ref.astar, ref.phi)


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
    return check_labels(lab, ref.labels, tie_mask(ref, p), grid_shape(p), min_agree)
