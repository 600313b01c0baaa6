"""Pins for the oracle's additive Vanka smoother (Sections 3.2, 3.3, 4.1).

- Patch sizes stated in Section 3.2 and boundary patch sizes stated in
  Section 3.3 (golden fixture).
- Interior weights are 1/N; the weights form a partition of unity.
- The assembled M r equals a brute-force loop over an independently
  enumerated patch list, each patch solved by dense LU (scipy lu_solve).
- Special cases: the RB patch on a 5-point stencil is damped Jacobi exactly
  (its patch matrices are diagonal); one whole-domain patch gives
  S = (1 - w) I.
- The constant-coefficient patch matrices of the compact 9-point stencil
  equal the matrices printed in Eqs. (4lfa, 5lfa, skew5lfa), and the stencil
  symbol equals Eq. (Hsymbol).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from conftest import read_golden
from oracle import lfa, operator, vanka


def _problem(shape, seed=0, alpha=0.3):
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    h = 1.0 / (shape[0] - 1)
    omega = 9.0
    A = operator.helmholtz(shape, h, 0.6 + 0.5 * rng.random(N), omega, 0.3 * rng.random(N))
    return operator.shifted(A, shape, omega, alpha)


def test_patch_sizes_and_boundary_patches():
    for kind, dim, interior, corner, edge in read_golden("patch_sizes.txt"):
        dim, interior, corner, edge = int(dim), int(interior), int(corner), int(edge)
        assert len(vanka.patch_offsets(kind, dim)) == interior
        if corner < 0:
            continue
        n = 6
        table = vanka.patch_index_table((n,) * dim, kind)
        sizes = (table >= 0).sum(axis=1)
        # anchors in the same flattened order as the nodes
        co = np.stack(np.meshgrid(*[np.arange(n)] * dim, indexing="ij"), -1).reshape(-1, dim)
        onb = ((co == 0) | (co == n - 1)).sum(axis=1)
        assert set(sizes[onb == dim]) == {corner}
        assert set(sizes[onb == 1]) == {edge}
        assert set(sizes[onb == 0]) == {interior}


@pytest.mark.parametrize("kind", ["element", "plus", "rb", "full", "jacobi"])
@pytest.mark.parametrize("dim", [2, 3])
def test_weights(kind, dim):
    shape = (7,) * dim
    table = vanka.patch_index_table(shape, kind)
    N = int(np.prod(shape))
    wt = vanka.node_weights(table, N)
    co = np.stack(np.meshgrid(*[np.arange(7)] * dim, indexing="ij"), -1).reshape(-1, dim)
    interior = np.all((co > 1) & (co < 5), axis=1)
    assert np.allclose(wt[interior], 1.0 / len(vanka.patch_offsets(kind, dim)))
    # partition of unity: sum_i V_i^T W_i V_i = I
    acc = np.zeros(N)
    for row in table:
        for j in row[row >= 0]:
            acc[j] += wt[j]
    assert np.allclose(acc, 1.0)


def _brute_force_patches(shape, kind):
    """Independent enumeration of the patches as lists of flat indices."""
    d = len(shape)
    if kind == "element":
        offs = list(itertools.product((0, 1), repeat=d))
    elif kind == "plus":
        offs = [o for o in itertools.product((-1, 0, 1), repeat=d) if sum(map(abs, o)) <= 1]
    elif kind == "rb":
        offs = [o for o in itertools.product((-1, 0, 1), repeat=d) if sum(map(abs, o)) % 2 == 0]
    elif kind == "full":
        offs = list(itertools.product((-1, 0, 1), repeat=d))
    else:
        offs = [(0,) * d]
    patches = []
    for anchor in itertools.product(*[range(n) for n in shape]):
        if kind == "element" and any(a == n - 1 for a, n in zip(anchor, shape)):
            continue
        nodes = []
        for o in offs:
            p = [a + b for a, b in zip(anchor, o)]
            if all(0 <= p[k] < shape[k] for k in range(d)):
                flat = 0
                for k in reversed(range(d)):
                    flat = flat * shape[k] + p[k]
                nodes.append(flat)
        patches.append(nodes)
    return patches


@pytest.mark.parametrize("kind", ["element", "plus", "rb", "full", "jacobi"])
@pytest.mark.parametrize("shape", [(5, 5), (4, 6), (4, 4, 3)])
def test_assembled_sum_matches_patchwise_dense_lu(kind, shape):
    A = _problem(shape)
    M = vanka.smoother_matrix(A, shape, kind)
    N = A.shape[0]
    rng = np.random.default_rng(3)
    r = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    patches = _brute_force_patches(shape, kind)
    count = np.zeros(N)
    for nodes in patches:
        count[nodes] += 1
    out = np.zeros(N, complex)
    Ad = A.toarray()
    for nodes in patches:
        Hi = Ad[np.ix_(nodes, nodes)]
        e = sla.lu_solve(sla.lu_factor(Hi), r[nodes])
        out[nodes] += e / count[nodes]
    assert np.allclose(M @ r, out, rtol=1e-12, atol=1e-12 * np.abs(out).max())


@pytest.mark.parametrize("shape", [(9, 9), (5, 6, 7)])
def test_rb_patch_on_second_order_stencil_is_jacobi(shape):
    A = _problem(shape)
    M = vanka.smoother_matrix(A, shape, "rb")
    J = vanka.smoother_matrix(A, shape, "jacobi")
    assert abs(M - J).max() <= 1e-14 * abs(J).max()
    assert np.allclose(J.diagonal(), 1.0 / A.diagonal(), rtol=1e-14)


def test_jacobi_fine_element_coarse_hierarchy():
    """The combined smoother of the heterogeneous 3D experiments (Section 5.5):
    damped Jacobi on the finest level only, element Vanka on every coarser
    smoothed level.  The Galerkin operators do not depend on the smoother, so
    each level must match the single-smoother hierarchy it takes its patch from."""
    from oracle import defaults, multigrid
    shape = (9, 9, 9)
    A = _problem(shape)
    mix = multigrid.build_hierarchy(A, shape, 3, ["jacobi", "element"], "linear")
    jac = multigrid.build_hierarchy(A, shape, 3, "jacobi", "linear")
    ele = multigrid.build_hierarchy(A, shape, 3, "element", "linear")
    assert abs(mix[0].M - jac[0].M).max() == 0 and mix[0].w == defaults.damping(3, "jacobi", 0)
    assert np.allclose(mix[0].M.diagonal(), 1.0 / A.diagonal(), rtol=1e-14) and mix[0].M.nnz == A.shape[0]
    assert abs(mix[1].M - ele[1].M).max() == 0 and mix[1].w == defaults.damping(3, "element", 1)
    assert mix[1].M.nnz > 8 * mix[1].A.shape[0]                    # true patches, not a diagonal
    for a, b in zip(mix, ele):
        assert abs(a.A - b.A).max() == 0


def test_whole_domain_patch_gives_one_minus_w():
    shape = (5, 4)
    A = _problem(shape)
    N = A.shape[0]
    table = np.arange(N)[None, :]
    (rows, slots, H), = vanka.patch_matrices(A, table)
    Minv = np.linalg.inv(H[0])                        # W = I: every node in one patch
    w = 0.7
    S = np.eye(N) - w * Minv @ A.toarray()
    assert np.allclose(S, (1 - w) * np.eye(N), atol=1e-11)


def test_lfa_patch_matrices_match_printed():
    a, b, c = 3.7 - 0.2j, -0.9 + 0.05j, -0.31
    h = 1.0
    # choose sigma so the compact stencil has centre a and edge b: a = 10/3 - 2s/3, b = -2/3 - s/12
    sigma = (10 / 3 - a) * 3 / 2
    st = operator.compact9_stencil(h, sigma)
    a_, b_, c_ = st[(0, 0)], st[(1, 0)], st[(1, 1)]
    assert np.isclose(c_, -1 / 6)
    sym = {"a": a_, "b": b_, "c": c_, "0": 0.0}
    rows = read_golden("lfa_patch_matrices.txt")
    i = 0
    while i < len(rows):
        kind = rows[i][0]
        N = len(rows[i + 1])
        printed = np.array([[sym[t] for t in rows[i + 1 + k]] for k in range(N)])
        got = lfa.patch_matrix(st, lfa.PATCHES_2D[kind])
        assert np.allclose(got, printed, rtol=0, atol=1e-14), kind
        i += N + 1
    # Eq. (Hsymbol)
    th = np.random.default_rng(0).uniform(-np.pi, np.pi, (50, 2))
    ref = a_ + 2 * b_ * np.cos(th[:, 0]) + 2 * b_ * np.cos(th[:, 1]) + 4 * c_ * np.cos(th[:, 0]) * np.cos(th[:, 1])
    assert np.allclose(lfa.symbol(st, th), ref, atol=1e-12)
