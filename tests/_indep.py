"""Independent numpy restatements used by the oracle pins.

Nothing here imports the oracle.  These helpers restate the problem
definition (speed fields, node kinds, h = k / c) and the Q1 transition
weights so that the pins can check the oracle with a *different* algorithm
(Dijkstra, policy iteration with exact linear solves, absorption
probabilities) rather than by re-running its own code.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def speed_np(p, x: np.ndarray) -> np.ndarray:
    """c(x) for x of shape (M, dim)."""
    q = p.speed_params
    if p.speed == "one":
        return np.ones(x.shape[0])
    if p.speed == "sincos2d":
        return 1.0 + q[0] * np.sin(2 * math.pi * x[:, 0]) * np.cos(2 * math.pi * x[:, 1])
    if p.speed == "sin3d":
        return 1.0 + q[0] * np.sin(math.pi * x[:, 0]) * np.sin(math.pi * x[:, 1]) * np.sin(math.pi * x[:, 2])
    if p.speed == "fan":
        return np.abs(q[0] + q[1] * x[:, 0] + q[2] * x[:, 1] + (q[3] * x[:, 2] if x.shape[1] > 2 else 0.0))
    if p.speed == "fourier2d":
        a = q[:16].reshape(4, 4)
        th = q[16:32].reshape(4, 4)
        ps = q[32:48].reshape(4, 4)
        g = np.zeros(x.shape[0])
        for i in range(4):
            for j in range(4):
                g += a[i, j] * np.cos(math.pi * i * x[:, 0] / 2 + th[i, j]) * np.cos(math.pi * j * x[:, 1] / 2 + ps[i, j])
        return 1.0 + 0.5 * g / np.abs(a).sum()
    raise ValueError(p.speed)


def node_grid(p):
    """Integer node indices (N, dim) with i1 fastest, and coordinates."""
    rng = [range(p.n[d]) for d in range(p.dim)]
    idx = np.array([t[::-1] for t in itertools.product(*reversed(rng))], dtype=np.int64)
    x = np.array(p.lo[: p.dim]) + idx * p.spacing
    return idx, x


def linear(p, idx):
    idx = np.atleast_2d(idx)
    out = idx[:, 0].copy()
    mul = p.n[0]
    for d in range(1, p.dim):
        out += idx[:, d] * mul
        mul *= p.n[d]
    return out


def target_parts(p, x):
    """Target part of each point (-1 outside): balls, one ball in R angular
    sectors, or the slab |x1 - v| <= r in R pieces along x2."""
    N = x.shape[0]
    part = np.full(N, -1)
    if p.target_kind == "balls":
        for j in range(p.n_targets - 1, -1, -1):
            c, r = p.targets[j, : p.dim], p.targets[j, p.dim]
            part[np.linalg.norm(x - c, axis=1) <= r] = j
        return part
    R = p.n_parts
    t = p.targets[0]
    if p.target_kind == "sectors":
        off = x[:, :2] - t[:2]
        inside = np.linalg.norm(x - t[: p.dim], axis=1) <= t[p.dim]
        th = np.mod(np.arctan2(off[:, 1], off[:, 0]), 2 * math.pi)
        j = np.floor(R * th / (2 * math.pi) + 1e-9).astype(int) % R
        part[inside] = j[inside]
        return part
    if p.target_kind == "orthants":
        inside = np.linalg.norm(x - t[: p.dim], axis=1) <= t[p.dim]
        j = sum(((x[:, d] >= t[d]).astype(int) << d) for d in range(p.dim))
        part[inside] = j[inside]
        return part
    inside = np.abs(x[:, 0] - t[0]) <= t[p.dim]
    j = np.clip(np.floor(R * (x[:, 1] - p.lo[1]) / (p.hi[1] - p.lo[1]) + 1e-9).astype(int), 0, R - 1)
    part[inside] = j[inside]
    return part


def in_obstacles(p, x):
    """Points inside a closed obstacle ball or box."""
    out = np.zeros(x.shape[0], bool)
    obs = getattr(p, "obstacles", None)
    if obs is None:
        return out
    for row in np.asarray(obs, float):
        if row[0] == 0.0:
            out |= np.sum((x - row[1: 1 + p.dim]) ** 2, axis=1) <= row[4] ** 2
        else:
            out |= np.all((x >= row[1: 1 + p.dim]) & (x <= row[4: 4 + p.dim]), axis=1)
    return out


def kinds(p):
    """0 free, 1 target (part >= 0), 2 ghost (ring, obstacle, or a node whose
    speed vanishes); h = k / c(x)."""
    idx, x = node_grid(p)
    N = idx.shape[0]
    part = target_parts(p, x)
    ring = np.zeros(N, bool)
    for d in range(p.dim):
        ring |= (idx[:, d] == 0) | (idx[:, d] == p.n[d] - 1)
    c = speed_np(p, x)
    stopped = ~(c > 1e-12)
    kind = np.where(part >= 0, 1, np.where(ring | stopped | in_obstacles(p, x), 2, 0))
    with np.errstate(divide="ignore"):
        h = np.where(stopped, np.inf, p.spacing / np.where(stopped, 1.0, c))
    return kind, part, h


def control_steps(p):
    """Per control: the unit direction of f and the factor g with
    h_{i,a} = g * h_i (h_i = k / c(x_i) for f = c(x) a, g = 1; for the drift
    f = s a + w: h_i = k and g = 1 / |s a + w|)."""
    a = np.asarray(p.controls, float)
    if p.dyn == "speed":
        return a, np.ones(a.shape[0])
    s, w = p.drift[0], np.asarray(p.drift[1: 1 + p.dim])
    f = s * a + w
    nf = np.linalg.norm(f, axis=1)
    dirs = f / nf[:, None]
    dirs[np.abs(dirs) < 1e-15] = 0.0
    return dirs, 1.0 / nf


def node_control_steps(p, x):
    """Per node (rows of x) and control: the unit direction of f and the time
    step h = k / |f| (+inf where f = 0).  Brockett's f = (a1, a2, x1 a2 -
    x2 a1); otherwise the per-control steps of control_steps times h_i."""
    a = np.asarray(p.controls, float)
    if p.dyn != "brockett":
        dirs, g = control_steps(p)
        _, _, h = kinds(p)
        return np.broadcast_to(dirs, (x.shape[0],) + dirs.shape), h[:, None] * g[None, :]
    f = np.stack([np.broadcast_to(a[:, 0], (x.shape[0], a.shape[0])),
                  np.broadcast_to(a[:, 1], (x.shape[0], a.shape[0])),
                  x[:, 0:1] * a[None, :, 1] - x[:, 1:2] * a[None, :, 0]], axis=2)
    nf = np.linalg.norm(f, axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        dirs = np.where(nf[..., None] > 1e-15, f / nf[..., None], 0.0)
        h = np.where(nf > 1e-15, p.spacing / nf, np.inf)
    dirs[np.abs(dirs) < 1e-15] = 0.0
    return dirs, h


def q1_corners(p, node_idx, a):
    """Corners and bilinear/trilinear weights of the foot node_idx + a (grid
    coordinates); zero weights dropped."""
    xi = np.asarray(node_idx, float) + np.asarray(a, float)
    base = np.clip(np.floor(xi).astype(int), 0, np.array(p.n[: p.dim]) - 2)
    t = xi - base
    out = []
    for bits in itertools.product((0, 1), repeat=p.dim):
        w = 1.0
        for d, b in enumerate(bits):
            w *= t[d] if b else 1.0 - t[d]
        if w > 0:
            out.append((int(linear(p, base + np.array(bits))[0]), w))
    return out
