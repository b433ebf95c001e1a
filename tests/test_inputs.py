"""Pins of the seeded problem generators (the synthetic stand-ins for the
paper's matrices) against what their definitions fix: Kronecker-sum forms of
the constant-coefficient operators, the textbook trilinear (Q1) stiffness
stencil, symmetry / definiteness, the finite-volume transmissibilities, the
layered block system's structure and the smoothed field's moments."""
import itertools

import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")


def dense(d, off, A):
    """Assemble a stencil matrix [n][ns] (scalar) densely, x slowest."""
    n = d[0] * d[1] * d[2]
    M = np.zeros((n, n))
    A = np.asarray(A).reshape(n, len(off))
    for i, j, k in itertools.product(range(d[0]), range(d[1]), range(d[2])):
        p = (i * d[1] + j) * d[2] + k
        for e, (a, b, c) in enumerate(off):
            if 0 <= i + a < d[0] and 0 <= j + b < d[1] and 0 <= k + c < d[2]:
                M[p, ((i + a) * d[1] + j + b) * d[2] + k + c] += A[p, e]
            else:
                assert A[p, e] == 0.0  # zero padding off the grid
    return M


def tridiag(n, lo, mid, hi):
    return np.diag(np.full(n, mid)) + np.diag(np.full(n - 1, lo), -1) + np.diag(np.full(n - 1, hi), 1)


def test_laplace7_is_the_kronecker_sum():
    d = (4, 3, 5)
    T = [tridiag(t, -1.0, 2.0, -1.0) for t in d]
    E = [np.eye(t) for t in d]
    ref = np.kron(np.kron(T[0], E[1]), E[2]) + np.kron(np.kron(E[0], T[1]), E[2]) + np.kron(np.kron(E[0], E[1]), T[2])
    assert np.array_equal(dense(d, I.OFF7, I.laplace7(d).numpy()), ref)


def test_fv7_unit_coefficient_is_laplace7_and_transmissibility_is_harmonic():
    d = (5, 4, 3)
    assert np.array_equal(I.fv7(d, torch.ones(60)).numpy(), I.laplace7(d).numpy())
    kap = torch.rand(60, generator=torch.Generator().manual_seed(3), dtype=torch.float64) * 9 + 1
    A = I.fv7(d, kap).numpy()
    M = dense(d, I.OFF7, A)
    assert np.abs(M - M.T).max() < 1e-15 * np.abs(M).max()
    k = kap.numpy().reshape(d)
    # the face between cells (1,2,1) and (2,2,1): -2 k1 k2 / (k1 + k2)
    p, q = (1 * 4 + 2) * 3 + 1, (2 * 4 + 2) * 3 + 1
    assert abs(M[p, q] + 2 * k[1, 2, 1] * k[2, 2, 1] / (k[1, 2, 1] + k[2, 2, 1])) < 1e-15 * M[p, p]
    # rows of interior cells sum to zero; a cell with one boundary face keeps
    # that face's kappa in its row sum
    rs = M.sum(axis=1).reshape(d)
    assert abs(rs[2, 2, 1]) < 1e-13 * M.max()
    assert abs(rs[2, 2, 0] - k[2, 2, 0]) < 1e-13 * M.max()


@pytest.mark.parametrize("aniso", [(1.0, 1.0, 1.0), (1.0, 1.0, 1e-3), (1e-3, 1e-3, 1.0), (0.5, 2.0, 3.0)])
def test_q1_constant_coefficient_stencil_is_the_q1_kronecker_form(aniso):
    """kappa = 1 (std 0): every interior stencil is kx K(x)M(x)M + ky M(x)K(x)M +
    kz M(x)M(x)K with the assembled 1-D Q1 operators K = [-1, 2, -1] and
    M = [1, 4, 1]/6 -- for isotropic k the textbook centre 8/3, faces 0,
    edges -1/6, corners -1/12."""
    d = (5, 6, 4)
    A = I.q1_aniso27(d, 0, std=0.0, aniso=aniso).numpy().reshape(*d, 27)
    K = {-1: -1.0, 0: 2.0, 1: -1.0}
    Mm = {-1: 1 / 6, 0: 4 / 6, 1: 1 / 6}
    kx, ky, kz = aniso
    for e, (a, b, c) in enumerate(I.OFF27):
        ref = kx * K[a] * Mm[b] * Mm[c] + ky * Mm[a] * K[b] * Mm[c] + kz * Mm[a] * Mm[b] * K[c]
        for i, j, k in itertools.product(range(1, d[0] - 1), range(1, d[1] - 1), range(1, d[2] - 1)):
            assert abs(A[i, j, k, e] - ref) < 1e-15
    if aniso == (1.0, 1.0, 1.0):
        c = A[2, 2, 2]
        assert abs(c[13] - 8 / 3) < 1e-15 and abs(c[4]) < 1e-15 and abs(c[1] + 1 / 6) < 1e-15
        assert abs(c[0] + 1 / 12) < 1e-15


def test_q1_variable_coefficient_is_spd():
    d = (5, 4, 6)
    M = dense(d, I.OFF27, I.q1_aniso27(d, 7).numpy())
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0


def test_smoothed_field_moments_and_smoothness():
    g = I.smoothed_field((32, 24, 20), 5, sigma=4.0, std=1.5).numpy()
    assert abs(g.mean()) < 1e-12 and abs(g.std(ddof=1) - 1.5) < 1e-12
    # neighbouring cells are strongly correlated (iid noise would give ~0)
    a, b = g[:, :, :-1].ravel(), g[:, :, 1:].ravel()
    assert np.corrcoef(a, b)[0, 1] > 0.9
    assert np.array_equal(g, I.smoothed_field((32, 24, 20), 5, sigma=4.0, std=1.5).numpy())  # seeded


def test_block7_layered_structure():
    d = (4, 3, 16)
    A = I.block7_layered(d, 2).numpy()  # [n, 7, 3, 3]
    C = np.array(I.COUPLING3)
    assert np.abs(C.sum(axis=1)).max() < 1e-15
    S = A[:, :, 0, 0].copy()  # the scalar finite-volume part (off the diagonal)
    S[:, 3] = A[:, 3, 0, 0] / (1.0 + C[0, 0])  # the sum of the cell's face transmissibilities
    for e in range(7):
        if e == 3:
            assert np.abs(A[:, 3] - S[:, 3, None, None] * (np.eye(3) + C)).max() < 1e-12 * np.abs(S).max()
        else:
            assert np.abs(A[:, e] - S[:, e, None, None] * np.eye(3)).max() == 0.0
    # interior cells: the face sum is the negated sum of the off-diagonal entries
    Sg = S.reshape(*d, 7)
    assert abs(Sg[1, 1, 5, 3] + (Sg[1, 1, 5].sum() - Sg[1, 1, 5, 3])) < 1e-12 * Sg[1, 1, 5, 3]
    # permeability is constant on 8-cell z-layers: the x-face transmissibilities
    # agree within a layer and differ between layers
    Sx = S[:, 6].reshape(d)  # +x face transmissibility
    for z0 in (0, 8):
        layer = Sx[:-1, :, z0:z0 + 8]
        assert np.abs(layer - layer[0, 0, 0]).max() == 0.0
    assert Sx[0, 0, 0] != Sx[0, 0, 8]


def test_rhs_is_seeded_uniform():
    b = I.rhs(100000, 11).numpy()
    assert b.min() >= -1.0 and b.max() <= 1.0 and abs(b.mean()) < 0.01 and abs(b.var() - 1 / 3) < 0.01
    assert np.array_equal(b, I.rhs(100000, 11).numpy()) and not np.array_equal(b, I.rhs(100000, 12).numpy())
