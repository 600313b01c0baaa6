"""Seeded synthetic media and sources.

The paper's experiments (Section 5) use homogeneous media, smoothly and
sharply varying 2D velocity models and a 3D geophysical model with an
absorbing layer of increasing attenuation towards the boundary.  The
generators here produce inputs of the same shape, range and structure from a
seed; they stand in for the paper's models, which are not reproduced.

Array convention: an n-node-per-axis grid is a numpy array of shape (n, n) in
2D or (n, n, n) in 3D, indexed [y, x] or [z, y, x], so the flattened C-order
index is x + n*(y + n*z) (x fastest).  The grid is nodal on [0, 1]^d with
h = 1/(n-1).  Depth is the slowest axis (y in 2D, z in 3D).
"""
from __future__ import annotations

import numpy as np


def omega_for_ppw(ppw: float, h: float, v_min: float = 1.5) -> float:
    """Angular frequency giving `ppw` grid points per wavelength at velocity v_min.

    The wavelength is 2*pi*v/omega; requiring it to span ppw cells of size h
    gives omega = 2*pi*v_min/(ppw*h) (Section 5 uses 10 points per wavelength).
    """
    return 2.0 * np.pi * v_min / (ppw * h)


def homogeneous_kappa(n: int, dim: int, kappa: float = 1.0) -> np.ndarray:
    """Constant slowness on an n^dim nodal grid."""
    return np.full((n,) * dim, float(kappa))


def _correlated_noise(shape, rng: np.random.Generator, corr_cells: float) -> np.ndarray:
    """White N(0,1) noise smoothed by a Gaussian of std `corr_cells` cells.

    The filter is applied in Fourier space (periodic), then the field is
    normalised to zero mean and unit standard deviation.
    """
    white = rng.standard_normal(shape)
    spec = np.fft.rfftn(white)
    k2 = np.zeros(spec.shape)
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            k = np.fft.rfftfreq(n) * 2.0 * np.pi
        else:
            k = np.fft.fftfreq(n) * 2.0 * np.pi
        sh = [1] * len(shape)
        sh[ax] = k.size
        k2 = k2 + (k.reshape(sh)) ** 2
    spec *= np.exp(-0.5 * corr_cells ** 2 * k2)
    field = np.fft.irfftn(spec, s=shape, axes=list(range(len(shape))))
    field -= field.mean()
    std = field.std()
    return field / std if std > 0 else field


def _ramp_smooth(profile: np.ndarray, ramp_cells: int) -> np.ndarray:
    """Moving average over ramp_cells+1 nodes: a step becomes a linear ramp of
    ramp_cells cells.  Ends are padded by repetition."""
    win = ramp_cells + 1
    pad = win // 2
    p = np.concatenate([np.full(pad, profile[0]), profile, np.full(win - 1 - pad, profile[-1])])
    c = np.cumsum(np.concatenate([[0.0], p]))
    return (c[win:] - c[:-win]) / win


def layered_kappa_2d(n: int, seed: int, v_min: float = 1.5, v_max: float = 4.5,
                     layers=(8, 12), ramp_cells: int = 4, noise: float = 0.05,
                     corr_cells: float = 16.0) -> np.ndarray:
    """Seeded layered 2D velocity model; returns the slowness kappa = 1/v.

    K ~ U{layers}; K-1 interfaces at sorted uniform depths; each layer's
    velocity ~ U[v_min, v_max]; interfaces smoothed into linear ramps of
    `ramp_cells` cells; then v <- v*(1 + noise*N) with N a unit-std Gaussian-
    correlated field of correlation length `corr_cells`; clipped to
    [v_min, v_max].
    """
    rng = np.random.default_rng(seed)
    K = int(rng.integers(layers[0], layers[1] + 1))
    interfaces = np.sort(rng.uniform(0.0, n - 1.0, size=K - 1))
    v_layer = rng.uniform(v_min, v_max, size=K)
    depth = np.arange(n, dtype=np.float64)
    prof = v_layer[np.searchsorted(interfaces, depth)]
    prof = _ramp_smooth(prof, ramp_cells)
    v = np.repeat(prof[:, None], n, axis=1)
    v = v * (1.0 + noise * _correlated_noise((n, n), rng, corr_cells))
    v = np.clip(v, v_min, v_max)
    return 1.0 / v


def geophysical_kappa_3d(n: int, seed: int, v_top: float = 1.5, v_bottom: float = 4.0,
                         v_inclusion: float = 4.5, noise: float = 0.03,
                         corr_cells: float = 16.0) -> np.ndarray:
    """Seeded 3D geophysical-like model; returns the slowness kappa = 1/v.

    Linear velocity gradient v_top -> v_bottom with depth (z), one ellipsoidal
    high-velocity inclusion (centre in [0.3, 0.7]^3, semi-axes in
    [0.08, 0.2], both from the seed) set to v_inclusion, then multiplicative
    Gaussian-correlated noise of relative size `noise`, clipped to
    [v_top, v_inclusion].
    """
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, n)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    v = v_top + (v_bottom - v_top) * z
    c = rng.uniform(0.3, 0.7, size=3)
    ax = rng.uniform(0.08, 0.2, size=3)
    inside = ((x - c[0]) / ax[0]) ** 2 + ((y - c[1]) / ax[1]) ** 2 + ((z - c[2]) / ax[2]) ** 2 <= 1.0
    v[inside] = v_inclusion
    v = v * (1.0 + noise * _correlated_noise((n, n, n), rng, corr_cells))
    v = np.clip(v, v_top, v_inclusion)
    return 1.0 / v


def absorbing_gamma(shape, omega: float, gamma_over_omega: float = 0.01,
                    layer_cells: int = 0) -> np.ndarray:
    """Attenuation gamma per node: background gamma0 = omega*gamma_over_omega
    plus an absorbing layer of `layer_cells` cells of increasing attenuation
    towards the boundary (Section 5 uses a 20-cell layer).

    Inside the layer gamma = gamma0 + omega*(d/L)^2, where d is the depth into
    the layer from its inner edge, d = max(0, L - dist), dist = the node's
    distance in cells to the nearest boundary, L = layer_cells.  At the
    outer boundary gamma/omega = gamma_over_omega + 1.
    """
    shape = tuple(shape)
    g0 = omega * gamma_over_omega
    gamma = np.full(shape, g0)
    if layer_cells <= 0:
        return gamma
    dist = None
    for ax, n in enumerate(shape):
        i = np.arange(n)
        d_ax = np.minimum(i, n - 1 - i)
        sh = [1] * len(shape)
        sh[ax] = n
        d_ax = d_ax.reshape(sh)
        dist = d_ax if dist is None else np.minimum(dist, d_ax)
    dist = np.broadcast_to(dist, shape)
    depth = np.maximum(0, layer_cells - dist).astype(np.float64)
    return gamma + omega * (depth / layer_cells) ** 2


def point_source(shape, node_xyz, h: float) -> np.ndarray:
    """Unit point source q = delta/h^d at the node with coordinates (x, y[, z])."""
    shape = tuple(shape)
    q = np.zeros(shape, dtype=np.complex128)
    idx = tuple(reversed(tuple(int(v) for v in node_xyz)))
    q[idx] = 1.0 / h ** len(shape)
    return q


def random_interior_nodes(n: int, dim: int, count: int, seed: int, margin: int = 8):
    """`count` seeded node coordinates (x, y[, z]) uniform in [margin, n-1-margin]^dim."""
    rng = np.random.default_rng(seed)
    pts = rng.integers(margin, n - margin, size=(count, dim))
    return [tuple(int(v) for v in p) for p in pts]
