"""Seeded synthetic inputs for the volume-potential workloads.

This module prepares inputs only: quadtrees (uniform, or refined on the
resolution of the source and then 2:1 balanced), the tensor Gauss-Legendre
node coordinates at which the source is sampled, and the source functions.
It holds none of the volume-potential arithmetic, so both the oracle and the
CUDA path can consume what it produces.

Geometry conventions shared by every consumer (they define the input format):

* root box: centre (cx, cy), side length ``side``;
* a leaf is (level, ix, iy): side h = side / 2**level, lower-left corner
  (cx - side/2 + ix*h, cy - side/2 + iy*h);
* each leaf carries p x p Gauss-Legendre nodes; the node with x-index i and
  y-index j has flat index j*p + i within the leaf, and leaves are stored in
  the order given, so a field has shape [n_leaves * p * p].

The quadtree is level-restricted (adjacent leaves differ by at most one
level), as the paper's fast-summation section requires of its trees.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

KERNEL_MHELMHOLTZ = 0   # G1(r) = K0(alpha r) / (2 pi)
KERNEL_MBIHARMONIC = 1  # G2(r) = (K0(alpha r) + log r) / (2 pi alpha^2)


@dataclasses.dataclass
class Tree:
    """Leaf list of a level-restricted quadtree over a square root box."""
    cx: float
    cy: float
    side: float
    level: np.ndarray  # int32 [n_leaves]
    ix: np.ndarray     # int32 [n_leaves]
    iy: np.ndarray     # int32 [n_leaves]

    @property
    def n_leaves(self) -> int:
        return int(self.level.shape[0])

    @property
    def max_level(self) -> int:
        return int(self.level.max()) if self.n_leaves else 0

    def leaf_boxes(self):
        """(x0, y0, h) arrays: lower-left corners and sides of the leaves."""
        h = self.side / (2.0 ** self.level.astype(np.float64))
        x0 = self.cx - self.side / 2 + self.ix * h
        y0 = self.cy - self.side / 2 + self.iy * h
        return x0, y0, h


@dataclasses.dataclass
class Workload:
    """One volume-potential problem: kernel, alpha, p, tree and sampled source."""
    name: str
    kernel: int
    alpha: float
    p: int
    tree: Tree
    f: np.ndarray          # float64 [n_leaves * p * p]
    source: Callable | None = None

    @property
    def n_nodes(self) -> int:
        return self.tree.n_leaves * self.p * self.p


def gl_nodes(p: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (ascending)."""
    x, w = np.polynomial.legendre.leggauss(p)
    return x, w


def node_coords(tree: Tree, p: int):
    """Coordinates (x, y) of every leaf node, in the storage order above."""
    xi, _ = gl_nodes(p)
    x0, y0, h = tree.leaf_boxes()
    t = (xi + 1.0) / 2.0
    X = x0[:, None, None] + h[:, None, None] * t[None, None, :]   # [L, j, i]
    Y = y0[:, None, None] + h[:, None, None] * t[None, :, None]
    X = np.broadcast_to(X, (tree.n_leaves, p, p))
    Y = np.broadcast_to(Y, (tree.n_leaves, p, p))
    return np.ascontiguousarray(X).reshape(-1), np.ascontiguousarray(Y).reshape(-1)


# --------------------------------------------------------------------------
# trees

def uniform_tree(depth: int, cx=0.0, cy=0.0, side=2.0) -> Tree:
    n = 1 << depth
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return Tree(cx, cy, side,
                np.full(n * n, depth, np.int32),
                ii.reshape(-1).astype(np.int32), jj.reshape(-1).astype(np.int32))


def _children(l, x, y):
    return [(l + 1, 2 * x + a, 2 * y + b) for b in (0, 1) for a in (0, 1)]


def balance_21(leaves: set) -> set:
    """Refine leaves until adjacent leaves differ by at most one level."""
    leaves = set(leaves)
    while True:
        internal = set()
        for (l, x, y) in leaves:
            while l > 0:
                l, x, y = l - 1, x >> 1, y >> 1
                if (l, x, y) in internal:
                    break
                internal.add((l, x, y))
        to_split = []
        for (l, x, y) in leaves:
            n1 = 1 << (l + 1)
            bx, by = 2 * x, 2 * y
            hit = False
            for a in (-1, 0, 1, 2):
                for b in (-1, 0, 1, 2):
                    if 0 <= a <= 1 and 0 <= b <= 1:
                        continue
                    X, Y = bx + a, by + b
                    if 0 <= X < n1 and 0 <= Y < n1 and (l + 1, X, Y) in internal:
                        hit = True
                        break
                if hit:
                    break
            if hit:
                to_split.append((l, x, y))
        if not to_split:
            return leaves
        for b in to_split:
            leaves.discard(b)
            leaves.update(_children(*b))


def legendre_tail(F: np.ndarray, p: int) -> np.ndarray:
    """Largest tensor Legendre coefficient with i+j >= p-2, per leaf.

    F has shape [L, p(j), p(i)] holding samples at the Gauss-Legendre nodes.
    """
    x, w = gl_nodes(p)
    k = np.arange(p)
    Pk = np.polynomial.legendre.legvander(x, p - 1)          # [node, k]
    A = (Pk * w[:, None]).T * ((2 * k + 1) / 2.0)[:, None]   # [k, node]
    C = np.einsum("ai,lji,bj->lba", A, F, A)                  # [L, kj, ki]
    mask = (k[:, None] + k[None, :]) >= p - 2
    return np.abs(C[:, mask]).max(axis=1)


def adaptive_tree(fn, p: int, cx: float, cy: float, side: float, tol: float,
                  max_depth: int, min_depth: int = 2, fscale: float | None = None) -> Tree:
    """Refine until every leaf's Legendre tail / ||f||_inf is below tol, then 2:1 balance."""
    xi, _ = gl_nodes(p)
    t = (xi + 1.0) / 2.0
    active = [(min_depth, x, y) for y in range(1 << min_depth) for x in range(1 << min_depth)]
    done = []
    if fscale is None:
        n = 512
        g = cx - side / 2 + side * (np.arange(n) + 0.5) / n
        GX, GY = np.meshgrid(g, g)
        fscale = float(np.abs(fn(GX, GY)).max()) or 1.0
    while active:
        arr = np.array(active, dtype=np.int64)
        l, x, y = arr[:, 0], arr[:, 1], arr[:, 2]
        h = side / (2.0 ** l)
        x0 = cx - side / 2 + x * h
        y0 = cy - side / 2 + y * h
        X = x0[:, None, None] + h[:, None, None] * t[None, None, :]
        Y = y0[:, None, None] + h[:, None, None] * t[None, :, None]
        F = fn(np.broadcast_to(X, (len(active), p, p)), np.broadcast_to(Y, (len(active), p, p)))
        tail = legendre_tail(F, p) / fscale
        nxt = []
        for k, b in enumerate(active):
            if tail[k] > tol and b[0] < max_depth:
                nxt.extend(_children(*b))
            else:
                done.append(b)
        active = nxt
    leaves = balance_21(set(done))
    return tree_from_set(leaves, cx, cy, side)


def tree_from_set(leaves, cx, cy, side) -> Tree:
    arr = np.array(sorted(leaves), dtype=np.int64)
    return Tree(cx, cy, side, arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32),
                arr[:, 2].astype(np.int32))


def random_balanced_tree(rng: np.random.Generator, n_splits: int, max_depth: int,
                         cx=0.0, cy=0.0, side=2.0, min_depth=1) -> Tree:
    """A randomly refined, 2:1-balanced tree (for list and parity tests)."""
    leaves = {(min_depth, x, y) for y in range(1 << min_depth) for x in range(1 << min_depth)}
    for _ in range(n_splits):
        cand = [b for b in leaves if b[0] < max_depth]
        if not cand:
            break
        b = cand[rng.integers(len(cand))]
        leaves.discard(b)
        leaves.update(_children(*b))
        leaves = balance_21(leaves)
    return tree_from_set(leaves, cx, cy, side)


# --------------------------------------------------------------------------
# sources

def gaussian_sum(centers, widths, amps):
    """f(x) = sum_k a_k exp(-|x - c_k|^2 / w_k^2)  (width read as in exp(-r^2/w^2))."""
    centers = np.asarray(centers, np.float64)
    widths = np.asarray(widths, np.float64)
    amps = np.asarray(amps, np.float64)

    def fn(X, Y):
        out = np.zeros(np.broadcast(X, Y).shape)
        for (c, w, a) in zip(centers, widths, amps):
            out = out + a * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2) / (w * w))
        return out
    return fn


def smooth_step(s):
    """C-infinity step: 1 for s <= 0, 0 for s >= 1, built from exp(-1/t)."""
    s = np.asarray(s, np.float64)
    a = np.clip(1.0 - s, 0.0, 1.0)
    b = np.clip(s, 0.0, 1.0)
    with np.errstate(divide="ignore"):
        pa = np.where(a > 0, np.exp(-1.0 / np.where(a > 0, a, 1.0)), 0.0)
        pb = np.where(b > 0, np.exp(-1.0 / np.where(b > 0, b, 1.0)), 0.0)
    return pa / (pa + pb)


def star_source(rng: np.random.Generator, n_gauss=20, blend=0.05, amp_star=0.3, k_star=5):
    """Smooth field inside r(t) = 1 + 0.3 cos(5t + phi), blended to zero outside
    over a radial band of width ``blend``, plus narrow seeded Gaussians inside."""
    phi = rng.uniform(0.0, 2 * np.pi)
    th = rng.uniform(0.0, 2 * np.pi, n_gauss)
    frac = np.sqrt(rng.uniform(0.0, 1.0, n_gauss)) * 0.8
    rr = frac * (1.0 + amp_star * np.cos(k_star * th + phi))
    centers = np.stack([rr * np.cos(th), rr * np.sin(th)], axis=1)
    widths = rng.uniform(0.01, 0.05, n_gauss)
    amps = rng.uniform(-1.0, 1.0, n_gauss)
    gs = gaussian_sum(centers, widths, amps)

    def fn(X, Y):
        r = np.hypot(X, Y)
        t = np.arctan2(Y, X)
        rb = 1.0 + amp_star * np.cos(k_star * t + phi)
        chi = smooth_step((r - rb) / blend)
        return chi * (np.cos(2 * X) * np.sin(3 * Y) + 0.5 + gs(X, Y))
    return fn


# --------------------------------------------------------------------------
# the workloads

def small_gaussian_workload(seed=1, depth=3, p=8, alpha=10.0, kernel=KERNEL_MHELMHOLTZ,
                            n_gauss=3, side=2.0) -> Workload:
    """Box [-1,1]^2, uniform depth-3 tree (64 leaves), p=8 (4096 nodes), alpha=10,
    f = sum of 3 Gaussians with centres U[-0.5,0.5]^2, widths U[0.1,0.3], amplitudes U[-1,1]."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.5, 0.5, (n_gauss, 2))
    w = rng.uniform(0.1, 0.3, n_gauss)
    a = rng.uniform(-1.0, 1.0, n_gauss)
    fn = gaussian_sum(c, w, a)
    tree = uniform_tree(depth, side=side)
    X, Y = node_coords(tree, p)
    return Workload(f"gauss3_uniform_d{depth}_p{p}_a{alpha:g}", kernel, alpha, p, tree, fn(X, Y), fn)


def star_adaptive_workload(seed=2, alpha=300.0, p=16, tol=1e-11, max_depth=10, n_gauss=20,
                           kernel=KERNEL_MBIHARMONIC, side=3.0) -> Workload:
    """Box [-1.5,1.5]^2, modified-biharmonic kernel, p=16, tree refined until the
    leaf Legendre tail is below tol (max depth 10), source = star blend + 20 Gaussians."""
    rng = np.random.default_rng(seed)
    fn = star_source(rng, n_gauss=n_gauss)
    tree = adaptive_tree(fn, p, 0.0, 0.0, side, tol, max_depth, min_depth=2)
    X, Y = node_coords(tree, p)
    return Workload(f"star_adaptive_p{p}_a{alpha:g}", kernel, alpha, p, tree, fn(X, Y), fn)


def batched_workloads(seed=4, n_trees=64, nmin=1e4, nmax=5e5, amin=10.0, amax=1000.0,
                      p_choices=(8, 12, 16), side=2.0):
    """64 independent trees: node counts log-uniform in [1e4, 5e5], alpha log-uniform
    in [10, 1000], p from {8, 12, 16}, 3-10 seeded Gaussians each; leaves are refined
    around the Gaussian centres until the node count reaches its target, then balanced."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_trees):
        target = float(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        alpha = float(np.exp(rng.uniform(np.log(amin), np.log(amax))))
        p = int(rng.choice(p_choices))
        ng = int(rng.integers(3, 11))
        c = rng.uniform(-0.6, 0.6, (ng, 2))
        w = rng.uniform(0.02, 0.2, ng)
        a = rng.uniform(-1.0, 1.0, ng)
        fn = gaussian_sum(c, w, a)
        leaves = {(2, x, y) for y in range(4) for x in range(4)}
        n_target_leaves = max(16, int(target / (p * p)))
        while len(leaves) < n_target_leaves:
            # split the leaves nearest to any centre, largest first
            arr = np.array(sorted(leaves), dtype=np.int64)
            h = side / (2.0 ** arr[:, 0])
            xc = -side / 2 + (arr[:, 1] + 0.5) * h
            yc = -side / 2 + (arr[:, 2] + 0.5) * h
            d = np.min(np.hypot(xc[:, None] - c[None, :, 0], yc[:, None] - c[None, :, 1]) / w[None, :], axis=1)
            score = h / (1.0 + d)
            order = np.argsort(-score)
            n_split = max(1, min(len(order), (n_target_leaves - len(leaves)) // 3 + 1))
            for idx in order[:n_split]:
                b = tuple(int(v) for v in arr[idx])
                if b[0] >= 12:
                    continue
                leaves.discard(b)
                leaves.update(_children(*b))
            leaves = balance_21(leaves)
        tree = tree_from_set(leaves, 0.0, 0.0, side)
        X, Y = node_coords(tree, p)
        out.append(Workload(f"batch{k}_p{p}_a{alpha:.1f}", KERNEL_MHELMHOLTZ, alpha, p, tree, fn(X, Y), fn))
    return out


def moving_stokeslets(seed=5, n_sources=5, radius=(1.6, 2.1)):
    """Seeded exterior forcing for a sequence of boundary-value problems: stokeslets on circles
    outside the star (radius 1.6..2.1 > 1.3), each rotating with its own angular speed, with
    strengths oscillating in time. Returns a function t -> (sources [K][2], strengths [K][2])."""
    rng = np.random.default_rng(seed)
    rad = rng.uniform(radius[0], radius[1], n_sources)
    ang0 = rng.uniform(0, 2 * np.pi, n_sources)
    om = rng.uniform(-2.0, 2.0, n_sources)
    f0 = rng.uniform(-1, 1, (n_sources, 2))
    f1 = rng.uniform(-0.5, 0.5, (n_sources, 2))
    nu = rng.uniform(1.0, 4.0, (n_sources, 2))
    ph = rng.uniform(0, 2 * np.pi, (n_sources, 2))

    def at(t):
        a = ang0 + om * t
        src = np.stack([rad * np.cos(a), rad * np.sin(a)], axis=1)
        f = f0 + f1 * np.sin(nu * t + ph)
        return src, f
    return at


@dataclasses.dataclass
class StepWorkload:
    """A sequence of modified Stokes problems in the star r(t) = 1 + 0.3 cos(5t + phi) (one per
    time step): a vorticity source on a uniform volume tree and a moving exterior forcing that sets
    the boundary velocity."""
    name: str
    alpha: float
    dt: float
    p: int
    tree: Tree
    phi: float
    source: Callable      # (X, Y, t) -> source values, torch tensors on any device
    boundary: Callable    # t -> (stokeslet positions [K][2], strengths [K][2])


def step_workload(seed=5, depth=7, p=16, re=100.0, dt=1e-3, n_gauss=3, blend=0.05, side=3.0) -> StepWorkload:
    """Star domain of the star-source workload (phase seeded), alpha = sqrt(Re / dt) (about 316 at
    Re = 100, dt = 1e-3), box [-1.5, 1.5]^2, uniform depth-7 tree with p = 16 (4.19M nodes).
    Source: the smooth star field of the adaptive workload times the C-infinity radial blend,
    plus n_gauss Gaussians (widths U[0.1, 0.3], amplitudes U[-1, 1]) whose centres rotate about
    the origin at radius <= 0.56 (inside the star for every phase) with angular speeds U[-2, 2];
    the background field drifts with t. Boundary forcing: moving_stokeslets(seed)."""
    rng = np.random.default_rng(seed)
    phi = float(rng.uniform(0.0, 2 * np.pi))
    rad = np.sqrt(rng.uniform(0.0, 1.0, n_gauss)) * 0.56
    ang0 = rng.uniform(0.0, 2 * np.pi, n_gauss)
    om = rng.uniform(-2.0, 2.0, n_gauss)
    widths = rng.uniform(0.1, 0.3, n_gauss)
    amps = rng.uniform(-1.0, 1.0, n_gauss)

    def source(X, Y, t):
        import torch
        r = torch.hypot(X, Y)
        th = torch.atan2(Y, X)
        s = (r - (1.0 + 0.3 * torch.cos(5 * th + phi))) / blend
        a = torch.clamp(1.0 - s, 0.0, 1.0)
        b = torch.clamp(s, 0.0, 1.0)
        pa = torch.where(a > 0, torch.exp(-1.0 / torch.where(a > 0, a, torch.ones_like(a))), torch.zeros_like(a))
        pb = torch.where(b > 0, torch.exp(-1.0 / torch.where(b > 0, b, torch.ones_like(b))), torch.zeros_like(b))
        chi = pa / (pa + pb)
        val = torch.cos(2 * X + 0.3 * t) * torch.sin(3 * Y - 0.2 * t) + 0.5
        for k in range(n_gauss):
            cx = rad[k] * math.cos(ang0[k] + om[k] * t)
            cy = rad[k] * math.sin(ang0[k] + om[k] * t)
            val = val + amps[k] * torch.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (widths[k] ** 2))
        return chi * val

    return StepWorkload(f"star_steps_uniform_d{depth}_p{p}_re{re:g}_dt{dt:g}", math.sqrt(re / dt), dt, p,
                        uniform_tree(depth, side=side), phi, source, moving_stokeslets(seed))


# --------------------------------------------------------------------------- periodic flows

def periodic_grid(n: int, side: float = 2 * np.pi):
    """Uniform n x n grid of the periodic box [0, side)^2: X[j][i] = x_i, Y[j][i] = y_j."""
    x = np.arange(n) * side / n
    return np.meshgrid(x, x, indexing="xy")


def taylor_green(n: int):
    """The Taylor-Green vortex on [0, 2 pi)^2 at t = 0: u = (sin x cos y, -cos x sin y), its gradient
    [a][m] = d u_a / d x_m and Laplacian -2 u, each [component][row j][column i]. It solves the
    Navier-Stokes equations with u(t) = u(0) exp(-2 t / Re)."""
    X, Y = periodic_grid(n)
    u = np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)])
    g = np.stack([np.stack([np.cos(X) * np.cos(Y), -np.sin(X) * np.sin(Y)]),
                  np.stack([np.sin(X) * np.sin(Y), -np.cos(X) * np.cos(Y)])])
    return u, g, -2.0 * u


INTERACTING_MODES = ((1, 2, 0.7, 0.3), (2, 1, -0.5, 1.1), (3, 1, 0.4, 2.0), (1, 3, 0.3, -0.7))


def interacting_modes(n: int, modes=INTERACTING_MODES):
    """A divergence-free field on [0, 2 pi)^2, u = (d psi / dy, -d psi / dx) for the stream function
    psi = sum a cos(kx x + ky y + phase) over modes (kx, ky, a, phase), with its gradient and Laplacian
    in closed form. The modes interact: (u . grad) u is not a gradient."""
    X, Y = periodic_grid(n)
    u = np.zeros((2, n, n)); g = np.zeros((2, 2, n, n)); lap = np.zeros((2, n, n))
    for kx, ky, a, ph in modes:
        th = kx * X + ky * Y + ph
        s, c = np.sin(th), np.cos(th)
        u[0] += -a * ky * s; u[1] += a * kx * s
        g[0, 0] += -a * ky * kx * c; g[0, 1] += -a * ky * ky * c
        g[1, 0] += a * kx * kx * c; g[1, 1] += a * kx * ky * c
        k2 = kx * kx + ky * ky
        lap[0] += a * ky * s * k2; lap[1] += -a * kx * s * k2
    return u, g, lap
