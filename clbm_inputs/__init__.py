"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the lattice Boltzmann method itself: it
only builds the wall-normal cell edges of the paper's grids (App. C linear
contraction, a geometric stretch, polar radii), the node positions of
general (non-separable) grids, picks the azimuthal size of the circular
cases, and draws seeded random fields.  Both the CUDA library's
callers and the oracle take their grids and random perturbations from here.
"""
import math

import numpy as np

DEFAULT_SEED = 20230105


def uniform_edges(n, step=1.0, origin=0.0):
    """n+1 equally spaced edges."""
    return origin + step * np.arange(n + 1, dtype=np.float64)


def linear_contraction_edges(N, CR, length, origin=0.0):
    """Edges x'_0..x'_N of the App. C linearly contracting grid.

    The step grows linearly from each wall to the middle; CR is the contraction
    ratio (avg - first step)/avg, so the contraction parameter is
    a = 2 CR / (N/2 - 1).  N must be even.
    """
    N = int(N)
    if N % 2 or N < 2:
        raise ValueError("N must be even")
    dbar = length / N
    if N == 2:
        if CR != 0:
            raise ValueError("N=2 admits no contraction")
        return origin + dbar * np.arange(3, dtype=np.float64)
    a = 2.0 * CR / (N / 2 - 1)
    if not (0.0 <= a <= 2.0 / (N / 2 - 1) + 1e-15):
        raise ValueError("CR out of range [0, 1]")
    e = np.empty(N + 1)
    for i in range(N + 1):
        if i <= N // 2:
            e[i] = dbar * i * (1.0 + 0.5 * a * (i - N / 2))
        else:
            e[i] = dbar * (N / 2 + (i - N / 2) * (1.0 + 0.5 * a * (N - i)))
    return origin + e


def geometric_stretch_edges(N, ratio, length, origin=0.0):
    """Edges of a grid whose step grows by ``ratio`` per cell from each wall to
    the middle (symmetric about the centre line), scaled to ``length``."""
    N = int(N)
    half = N // 2
    steps = ratio ** np.arange(half, dtype=np.float64)
    if N % 2:
        mid = ratio ** half
        full = np.concatenate([steps, [mid], steps[::-1]])
    else:
        full = np.concatenate([steps, steps[::-1]])
    full *= length / full.sum()
    e = np.concatenate([[0.0], np.cumsum(full)])
    e[-1] = length
    return origin + e


GHOST = 4  # node layers beyond each wall and each periodic end in a node array


def _node_q(n):
    """Node coordinates q = k - 1/2 for k = -3 .. n + 4 (1-based node index)."""
    return np.arange(1 - GHOST, n + GHOST + 1, dtype=np.float64) - 0.5


def mapped_nodes(fun, n1, n2, ghosts="mirror"):
    """Node positions of a general grid, shape (n1 + 8, n2 + 8, 2): nodes
    i = -3 .. n1 + 4 (wall-normal) by j = -3 .. n2 + 4 (periodic) at
    x = fun(q1, q2), q = (i - 1/2, j - 1/2).  fun takes arrays and returns
    (x, y); it must give the periodic images itself (fun(q1, q2 + n2) = fun(q1,
    q2) shifted by the period).  Rows beyond a wall: ghosts="extend" evaluates
    fun there too; ghosts="mirror" reflects the first four rows inside through
    the wall, which must be a straight line (the wall node positions fun(0, q2)
    and fun(n1, q2) each lie on one line)."""
    q1, q2 = np.meshgrid(_node_q(n1), _node_q(n2), indexing="ij")
    x, y = fun(q1, q2)
    P = np.stack([np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64)], axis=-1)
    if ghosts == "extend":
        return np.ascontiguousarray(P)
    if ghosts != "mirror":
        raise ValueError("ghosts must be 'mirror' or 'extend'")
    for lo in (True, False):
        qw = 0.0 if lo else float(n1)
        w = np.stack(fun(np.full(n2 + 2 * GHOST, qw), _node_q(n2)), axis=-1)
        a, b = w[0], w[-1]
        t = (b - a) / np.linalg.norm(b - a)          # wall direction
        nrm = np.array([-t[1], t[0]])
        for k in range(1, GHOST + 1):
            gi = GHOST - k if lo else GHOST + n1 + k - 1          # ghost row index
            mi = GHOST + k - 1 if lo else GHOST + n1 - k          # mirrored interior row
            d = P[mi] - a
            P[gi] = P[mi] - 2.0 * (d @ nrm)[:, None] * nrm[None, :]
    return np.ascontiguousarray(P)


def sheared_channel(n1, n2, h=1.0, L2=1.0, shear=0.3):
    """Affine map with parallelogram cells: x = q1 h, y = q2 L2 + shear q1 h."""
    return lambda q1, q2: (q1 * h, q2 * L2 + shear * q1 * h)


def wavy_channel(n1, n2, h=1.0, L2=1.0, amp=0.2):
    """Non-separable map between straight walls x = 0 and x = n1 h:
    x = h (q1 + amp sin(pi q1 / n1) sin(2 pi q2 / n2)), y = q2 L2."""
    return lambda q1, q2: (h * (q1 + amp * np.sin(np.pi * q1 / n1) * np.sin(2.0 * np.pi * q2 / n2)),
                           q2 * L2)


def polar_edges(R1, R2, Nr, CR=0.0):
    """Radial edges r'_0..r'_Nr from R1 to R2, App. C contraction of ratio CR."""
    if CR == 0.0:
        return R1 + uniform_edges(Nr, (R2 - R1) / Nr)
    return linear_contraction_edges(Nr, CR, R2 - R1, origin=R1)


def n_theta(Nr, R1, R2):
    """Azimuthal size giving near-square cells at the inner wall (Sec. 3.3)."""
    return int(round(Nr * 2.0 * math.pi * R1 / (R2 - R1)))


def smooth_field(shape, seed=DEFAULT_SEED, modes=3, amplitude=1.0):
    """Seeded smooth random field over the last two axes of ``shape``.

    A sum of a few low sine/cosine modes per leading index, periodic in the
    last axis; values lie within +-amplitude.
    """
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    lead = int(np.prod(shape[:-2])) if len(shape) > 2 else 1
    n1, n2 = shape[-2], shape[-1]
    x = (np.arange(n1) + 0.5) / n1
    y = (np.arange(n2) + 0.5) / n2
    out = np.zeros((lead, n1, n2))
    for k in range(lead):
        acc = np.zeros((n1, n2))
        for _ in range(modes):
            kx = rng.integers(1, 4)
            ky = rng.integers(0, 4)
            ph1, ph2 = rng.uniform(0, 2 * np.pi, 2)
            amp = rng.uniform(-1, 1)
            acc += amp * np.sin(np.pi * kx * x + ph1)[:, None] * np.cos(2 * np.pi * ky * y + ph2)[None, :]
        out[k] = acc / modes
    return (amplitude * out).reshape(shape)


def white_field(shape, seed=DEFAULT_SEED, amplitude=1.0):
    """Seeded uniform noise in [-amplitude, amplitude]."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.uniform(-1.0, 1.0, size=shape)
