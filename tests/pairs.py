"""Matched oracle / CUDA problems on the same seeded inputs (test helper)."""
from __future__ import annotations

import numpy as np

import workloads
from oracle import solver as osolver


def medium(dim, n, seed=0, layer=0, ppw=10.0, kind="layered"):
    """(h, omega, kappa, gamma) of a seeded medium on an n^dim grid."""
    h = 1.0 / (n - 1)
    if kind == "homogeneous":
        kappa = workloads.homogeneous_kappa(n, dim, 1.0)
        vmin = 1.0
    elif dim == 2:
        kappa = workloads.layered_kappa_2d(n, seed)
        vmin = 1.5
    else:
        kappa = workloads.geophysical_kappa_3d(n, seed)
        vmin = 1.5
    omega = workloads.omega_for_ppw(ppw, h, vmin)
    gamma = workloads.absorbing_gamma(kappa.shape, omega, 0.01, layer)
    return h, omega, kappa.ravel(), gamma.ravel()


def make_pair(dim, n, levels, patch, scheme, precision="fp64", alpha=0.25, seed=0, layer=0,
              kind="layered", patch_coarse=None, tol=1e-7, ppw=10.0, cycle="V", stencil="second"):
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    h, omega, kappa, gamma = medium(dim, n, seed, layer, ppw, kind)
    shape = (n,) * dim
    orc = osolver.Problem(shape, h, kappa, omega, gamma, alpha, levels, patch, scheme,
                          patch_coarse=patch_coarse, cycle=cycle, stencil=stencil)
    gpu = HelmholtzSolver(dim, [n] * dim, kappa, omega, gamma, alpha, levels, patch=patch,
                          intergrid=scheme, precision=precision, tol=tol, patch_coarse=patch_coarse,
                          cycle=cycle, stencil=stencil)
    return orc, gpu


def oracle_planes(A, shape_xyz, offsets):
    """Entries of sparse A as planes [len(offsets), N]: A[p, p + off] (0 outside)."""
    N = A.shape[0]
    d = len(shape_xyz)
    grids = np.meshgrid(*[np.arange(m) for m in reversed(shape_xyz)], indexing="ij")
    co = [g.ravel() for g in reversed(grids)]
    out = np.zeros((len(offsets), N), dtype=np.complex128)
    idx = np.arange(N)
    for s, off in enumerate(offsets):
        ok = np.ones(N, dtype=bool)
        nb = np.zeros(N, dtype=np.int64)
        stride = 1
        for a in range(d):
            c = co[a] + off[a]
            ok &= (c >= 0) & (c < shape_xyz[a])
            nb += np.where(ok, c, 0) * stride
            stride *= shape_xyz[a]
        out[s, ok] = np.asarray(A[idx[ok], nb[ok]]).ravel()
    return out


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# Solution agreement with the oracle (relative L2): the GPU solution must match
# the oracle's solution of the same problem at the same tolerance within these
# bounds; the error against an oracle solve to 1e-10 (about the exact discrete
# solution) is reported beside it.
AGREE = {"fp64": 1e-6, "mixed": 1e-5}


def l2_rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def check_agreement(p, p_tol, p_ref, precision, label=""):
    """Assert |p - p_tol| / |p_tol| <= AGREE[precision], p_tol the oracle's
    solution at the same tolerance; returns (error vs p_tol, error vs p_ref).
    The tight-solve error is a second, reported number: it may exceed the bound
    by the oracle's own error at the tolerance."""
    e_tol = l2_rel(p, p_tol)
    e_ref = l2_rel(p, p_ref) if p_ref is not None else float("nan")
    print(f"agreement {label} {precision}: vs oracle at tol {e_tol:.3e}, vs tight oracle {e_ref:.3e}")
    assert e_tol <= AGREE[precision], (label, precision, e_tol, e_ref)
    return e_tol, e_ref
