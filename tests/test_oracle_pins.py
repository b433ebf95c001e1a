"""Pins of the CPU oracle against facts it does not compute itself: dense linear
algebra on assembled matrices, closed forms, invariants and the values the
paper prints.  A wrong sign, index, operand order or dropped term in the oracle
must fail at least one of these."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2506_21932_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rnd_matrix(d, off, seed, B=1, spd_shift=None):
    """Random stencil matrix with zero off-grid padding (not necessarily SPD)."""
    rng = np.random.default_rng(seed)
    n = d[0] * d[1] * d[2]
    A = rng.uniform(-1, 1, size=(n, len(off), B, B))
    ec = list(map(tuple, off)).index((0, 0, 0))
    A[:, ec] += (spd_shift if spd_shift is not None else 2.0 * len(off)) * np.eye(B)
    A = A.reshape(n, len(off) * B * B) if B > 1 else A.reshape(n, len(off))
    import torch
    At = torch.from_numpy(A.reshape(n, len(off), B, B) if B > 1 else A)
    return I._zero_offgrid(At.clone(), tuple(d), [tuple(o) for o in off]).numpy()


def sym_random(d, off, seed):
    """Random structurally symmetric, numerically symmetric, diagonally dominant
    stencil matrix: assembled dense, symmetrised, written back."""
    from oracle import oracle as orc
    A = rnd_matrix(d, off, seed)
    M = orc.assemble_dense(d, off, A)
    M = 0.5 * (M + M.T)
    n = M.shape[0]
    out = np.zeros_like(A)
    for i, j, k in itertools.product(range(d[0]), range(d[1]), range(d[2])):
        p = (i * d[1] + j) * d[2] + k
        for e, o in enumerate(off):
            a, b, c = i + o[0], j + o[1], k + o[2]
            if 0 <= a < d[0] and 0 <= b < d[1] and 0 <= c < d[2]:
                out[p, e] = M[p, (a * d[1] + b) * d[2] + c]
    ec = list(map(tuple, off)).index((0, 0, 0))
    out[:, ec] = np.abs(out).sum(axis=1) + 1.0
    assert n == out.shape[0]
    return out


# --------------------------------------------------------------------------- #
# SpMV: closed-form eigenpairs of the 7-point Laplacian                         #
# --------------------------------------------------------------------------- #

def test_spmv_laplace_eigenvectors(orc):
    """-Delta_h with Dirichlet: prod_d sin(p_d pi x_d/(n_d+1)) is an eigenvector
    with eigenvalue sum_d 4 sin^2(p_d pi / (2(n_d+1)))."""
    d = (9, 7, 11)
    A = I.laplace7(d).numpy()
    x = [np.arange(1, t + 1) for t in d]
    for pv in [(1, 1, 1), (3, 5, 2), (9, 7, 11)]:
        v = np.einsum("i,j,k->ijk", *[np.sin(pv[t] * np.pi * x[t] / (d[t] + 1)) for t in range(3)]).ravel()
        lam = sum(4 * math.sin(pv[t] * math.pi / (2 * (d[t] + 1))) ** 2 for t in range(3))
        y = orc.spmv(d, I.OFF7, A, v)
        assert np.max(np.abs(y - lam * v)) < 1e-13 * lam


def test_spmv_matches_dense(orc):
    d = (4, 5, 3)
    for off, B in [(I.OFF27, 1), (I.OFF7, 3), (I.OFF19, 1)]:
        A = rnd_matrix(d, off, 3, B=B)
        M = orc.assemble_dense(d, off, A, B=B)
        x = np.random.default_rng(1).normal(size=M.shape[0])
        assert np.allclose(orc.spmv(d, off, A, x, B=B), M @ x, rtol=0, atol=1e-13)
        b = np.random.default_rng(2).normal(size=M.shape[0])
        assert np.allclose(orc.residual(d, off, A, b, x, B=B), b - M @ x, rtol=0, atol=1e-13)


def test_dense_assembly_by_hand(orc):
    """One entry of the assembled matrix checked by hand: row of point (1,2,0)
    at neighbour (0,3,1) is the coefficient of offset (-1,+1,+1)."""
    d = (3, 4, 2)
    A = rnd_matrix(d, I.OFF27, 5)
    M = orc.assemble_dense(d, I.OFF27, A)
    p = (1 * 4 + 2) * 2 + 0
    q = (0 * 4 + 3) * 2 + 1
    assert M[p, q] == A[p, I.OFF27.index((-1, 1, 1))]
    assert np.count_nonzero(M) == np.count_nonzero(A)


def test_laplace_condition_number_closed_form():
    """Table 3 lists cond ~2e4 for Laplace at 16.8M dof (256^3); the closed form
    lambda_max/lambda_min of the 7-point operator on 256^3 is ~2.7e4, the same
    order (the printed figure is an estimate)."""
    n = 256
    lmin = 3 * 4 * math.sin(math.pi / (2 * (n + 1))) ** 2
    lmax = 3 * 4 * math.sin(n * math.pi / (2 * (n + 1))) ** 2
    c = lmax / lmin
    assert 2.0e4 < c < 3.0e4


# --------------------------------------------------------------------------- #
# Gauss-Seidel = dense triangular solves (Sec. 4.4 formulas)                   #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("off,B,w", [(I.OFF27, 1, 1.0), (I.OFF7, 1, 1.0), (I.OFF7, 1, 1.3), (I.OFF7, 3, 1.0),
                                     (I.OFF19, 1, 0.8)])
def test_gs_sweeps_are_triangular_solves(orc, off, B, w):
    d = (4, 3, 5)
    A = rnd_matrix(d, off, 11, B=B)
    M = orc.assemble_dense(d, off, A, B=B)
    n = M.shape[0]
    D = np.zeros_like(M)
    for p in range(n // B):
        D[p * B:(p + 1) * B, p * B:(p + 1) * B] = M[p * B:(p + 1) * B, p * B:(p + 1) * B]
    L = np.tril(M) - np.tril(D)
    U = np.triu(M) - np.triu(D)
    Dinv = orc.diag_inverse(d, off, A, B=B)
    rng = np.random.default_rng(7)
    b, u0 = rng.normal(size=n), rng.normal(size=n)
    # GS-Forward: u + w (D + wL)^{-1} (b - A u)
    ref_f = u0 + w * np.linalg.solve(D + w * L, b - M @ u0)
    got_f = orc.gs_forward(d, off, A, Dinv, b, u0, w=w, B=B)
    assert np.max(np.abs(got_f - ref_f)) < 1e-11 * max(1, np.abs(ref_f).max())
    ref_b = got_f + w * np.linalg.solve(D + w * U, b - M @ got_f)
    got_b = orc.gs_backward(d, off, A, Dinv, b, got_f, w=w, B=B)
    assert np.max(np.abs(got_b - ref_b)) < 1e-11 * max(1, np.abs(ref_b).max())


def test_gs_zero_guess_uses_lower_terms_only(orc):
    """From u = 0 the forward sweep is (D+L)^{-1} b: the upper part never enters."""
    d = (5, 6, 7)
    A = rnd_matrix(d, I.OFF27, 4)
    M = orc.assemble_dense(d, I.OFF27, A)
    Dinv = orc.diag_inverse(d, I.OFF27, A)
    b = np.random.default_rng(0).normal(size=M.shape[0])
    got = orc.gs_forward(d, I.OFF27, A, Dinv, b, np.zeros_like(b))
    ref = sla.solve_triangular(np.tril(M), b, lower=True)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


# --------------------------------------------------------------------------- #
# ILU(0)                                                                        #
# --------------------------------------------------------------------------- #

def _dense_lu_from_stencil(orc, d, off, LU):
    M = orc.assemble_dense(d, off, LU)
    L = np.tril(M, -1) + np.eye(M.shape[0])
    U = np.triu(M)
    return L, U


@pytest.mark.parametrize("off", [I.OFF7, I.OFF27, I.OFF19])
def test_ilu0_defining_property(orc, off):
    """(L U)_{pq} = a_{pq} on every position of the mask (ILU(0) definition),
    with L unit lower and U upper triangular."""
    d = (5, 4, 6)
    A = sym_random(d, off, 3)
    LU = orc.ilu0_factor(d, off, A)
    L, U = _dense_lu_from_stencil(orc, d, off, LU)
    M = orc.assemble_dense(d, off, A)
    pattern = orc.assemble_dense(d, off, np.ones_like(A)) != 0
    prod = L @ U
    assert np.max(np.abs((prod - M)[pattern])) < 1e-12 * np.abs(M).max()
    # and the factors really live on the pattern
    assert not np.any(L[~pattern & ~np.eye(len(M), dtype=bool)])


def test_ilu0_tridiagonal_is_exact(orc):
    """On a 1x1xn grid the 7-point mask is tridiagonal: ILU(0) has no dropped
    fill, equals the exact LU and one application solves the system."""
    d = (1, 1, 40)
    A = sym_random(d, I.OFF7, 9)
    M = orc.assemble_dense(d, I.OFF7, A)
    LU = orc.ilu0_factor(d, I.OFF7, A)
    udinv = 1.0 / LU[:, 3]
    b = np.random.default_rng(3).normal(size=40)
    x = orc.ilu0_apply(d, I.OFF7, LU, udinv, b)
    assert np.max(np.abs(M @ x - b)) < 1e-12


def test_ilu0_apply_is_two_triangular_solves(orc):
    d = (4, 5, 3)
    A = sym_random(d, I.OFF27, 1)
    LU = orc.ilu0_factor(d, I.OFF27, A)
    L, U = _dense_lu_from_stencil(orc, d, I.OFF27, LU)
    r = np.random.default_rng(4).normal(size=L.shape[0])
    ref = sla.solve_triangular(U, sla.solve_triangular(L, r, lower=True, unit_diagonal=True))
    got = orc.ilu0_apply(d, I.OFF27, LU, 1.0 / LU[:, 13], r)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


def test_ilu0_breakdown_reported(orc):
    d = (3, 3, 3)
    A = I.laplace7(d).numpy()
    A[:, 3] = -6.0  # negative pivots: not SPD
    with pytest.raises(ArithmeticError):
        orc.ilu0_factor(d, I.OFF7, A)


# --------------------------------------------------------------------------- #
# Transfers                                                                     #
# --------------------------------------------------------------------------- #

def test_restriction_is_adjoint_of_prolongation(orc):
    """R = P^T / 8 for full weighting and R = P^T for 3d8c, checked through the
    two independent routines: <R r, e> = c <r, P e>."""
    rng = np.random.default_rng(5)
    for transfer, c in [(orc.FW27V, 1 / 8), (orc.PC8C, 1.0)]:
        for fd in [(8, 6, 4), (10, 8, 6)]:
            for B in (1, 3):
                nf = np.prod(fd) * B
                nc = np.prod(orc.coarse_dims(fd)) * B
                r, e = rng.normal(size=nf), rng.normal(size=nc)
                lhs = orc.restrict(transfer, fd, r, B=B) @ e
                rhs = c * (r @ orc.prolong_add(transfer, fd, e, np.zeros(nf), B=B))
                assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))


def test_trilinear_interpolation_reproduces_linear_functions(orc):
    """3d27v interpolation is exact for (tri)linear functions on fine points
    whose two enclosing coarse points both exist: coarse I lives at fine 2I+1,
    so fine 0 and fine n-1 (next to the Dirichlet boundary) are excluded."""
    fd = (12, 10, 8)
    cd = orc.coarse_dims(fd)
    a, b, c, e0 = 0.3, -1.1, 0.7, 2.0
    ec = np.array([a * (2 * i + 1) + b * (2 * j + 1) + c * (2 * k + 1) + e0
                   for i in range(cd[0]) for j in range(cd[1]) for k in range(cd[2])])
    uf = orc.prolong_add(orc.FW27V, fd, ec, np.zeros(np.prod(fd))).reshape(fd)
    for i, j, k in itertools.product(range(1, fd[0] - 1), range(1, fd[1] - 1), range(1, fd[2] - 1)):
        assert abs(uf[i, j, k] - (a * i + b * j + c * k + e0)) < 1e-12
    # piecewise constant 3d8c reproduces constants everywhere
    uf = orc.prolong_add(orc.PC8C, fd, np.full(np.prod(cd), 3.5), np.zeros(np.prod(fd)))
    assert np.all(uf == 3.5)


# --------------------------------------------------------------------------- #
# Galerkin coarse operator, Eq. 4-5                                             #
# --------------------------------------------------------------------------- #

def _dense_transfer(orc, transfer, fd, B=1):
    """Assemble P column by column from the prolongation routine."""
    nc = np.prod(orc.coarse_dims(fd)) * B
    nf = np.prod(fd) * B
    P = np.zeros((nf, nc))
    for j in range(nc):
        e = np.zeros(nc)
        e[j] = 1.0
        P[:, j] = orc.prolong_add(transfer, fd, e, np.zeros(nf), B=B)
    return P


def _coarse_stencil_to_dense(orc, cd, Ac27, B=1):
    ns27 = np.array(I.OFF27)
    return orc.assemble_dense(cd, ns27, Ac27.reshape(len(Ac27), -1) if B == 1 else Ac27, B=B)


@pytest.mark.parametrize("fd,off,transfer,B", [
    ((8, 6, 4), I.OFF7, 0, 1), ((6, 6, 6), I.OFF27, 0, 1), ((8, 6, 4), I.OFF27, 0, 1),
    ((6, 8, 4), I.OFF19, 0, 1), ((8, 6, 4), I.OFF7, 1, 1), ((6, 6, 6), I.OFF27, 1, 1), ((8, 4, 6), I.OFF7, 1, 3)])
def test_rap_equals_assembled_triple_product(orc, fd, off, transfer, B):
    """Pin of the brute-force chain sum: A^C = R A^F P as dense matrix products,
    with R and P assembled from the restriction / prolongation routines."""
    A = rnd_matrix(fd, off, 21, B=B)
    Ac27, present = orc.rap27(transfer, fd, off, A, B=B)
    cd = orc.coarse_dims(fd)
    M = orc.assemble_dense(fd, off, A, B=B)
    P = _dense_transfer(orc, transfer, fd, B=B)
    scale = 1 / 8 if transfer == 0 else 1.0
    ref = scale * P.T @ M @ P
    got = _coarse_stencil_to_dense(orc, cd, Ac27, B=B)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()


def test_rap_galerkin_operator_identity(orc):
    """A^C e = R A^F P e for random e through spmv / restrict / prolong."""
    fd = (10, 8, 6)
    A = I.q1_aniso27(fd, 3).numpy()
    Ac27, present = orc.rap27(orc.FW27V, fd, I.OFF27, A)
    cd = orc.coarse_dims(fd)
    e = np.random.default_rng(8).normal(size=np.prod(cd))
    lhs = orc.spmv(cd, I.OFF27, Ac27.reshape(-1, 27), e)
    rhs = orc.restrict(orc.FW27V, fd, orc.spmv(fd, I.OFF27, A, orc.prolong_add(orc.FW27V, fd, e, np.zeros(np.prod(fd)))))
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.abs(lhs).max()


def test_rap_laplace_closed_form_kronecker_sum(orc):
    """Constant 7-point Laplacian = T(x)I(x)I + I(x)T(x)I + I(x)I(x)T with T =
    tridiag(-1,2,-1).  With 3d27v transfers the Galerkin product factorises per
    dimension: R1 T P1 = [-1,2,-1]/4 and R1 P1 = [1/8, 3/4, 1/8], so every
    interior coarse stencil is the Kronecker sum of those 1-D stencils."""
    fd = (16, 16, 16)
    A = I.laplace7(fd).numpy()
    Ac27, present = orc.rap27(orc.FW27V, fd, I.OFF7, A)
    t = {-1: -0.25, 0: 0.5, 1: -0.25}
    m = {-1: 0.125, 0: 0.75, 1: 0.125}
    cd = orc.coarse_dims(fd)
    assert present.sum() == 27
    for I0 in range(1, cd[0] - 2):
        for I1 in (1, 3):
            for I2 in (2, 4):
                P = (I0 * cd[1] + I1) * cd[2] + I2
                for e, (a, b, c) in enumerate(I.OFF27):
                    ref = t[a] * m[b] * m[c] + m[a] * t[b] * m[c] + m[a] * m[b] * t[c]
                    assert abs(Ac27[P, e, 0, 0] - ref) < 1e-15
    assert abs(0.5 * 0.75 ** 2 * 3 - 0.84375) < 1e-16  # centre value
    # row sums vanish in the interior (constants are in the kernel of the PDE)
    P = (3 * cd[1] + 3) * cd[2] + 3
    assert abs(Ac27[P].sum()) < 1e-15


def test_rap_cell_transfer_keeps_7pt_laplacian_times_4(orc):
    """3d8c restriction and interpolation of the 7-point Laplacian: the coarse
    operator is 4 x the same 7-point stencil in the interior (Table 2, 3d8c/
    3d7/3d8c keeps the pattern; Table 5 lists C_O = C_G for oil-4C)."""
    fd = (12, 12, 12)
    A = I.laplace7(fd).numpy()
    Ac27, present = orc.rap27(orc.PC8C, fd, I.OFF7, A)
    assert [I.OFF27[o] for o in range(27) if present[o]] == I.OFF7
    cd = orc.coarse_dims(fd)
    P = (2 * cd[1] + 3) * cd[2] + 2
    for e, o in enumerate(I.OFF27):
        ref = 24.0 if o == (0, 0, 0) else (-4.0 if o in I.OFF7 else 0.0)
        assert Ac27[P, e, 0, 0] == ref


def test_rap_preserves_symmetry(orc):
    fd = (8, 8, 6)
    A = I.q1_aniso27(fd, 5).numpy()
    for transfer in (orc.FW27V, orc.PC8C):
        Ac27, _ = orc.rap27(transfer, fd, I.OFF27, A)
        M = _coarse_stencil_to_dense(orc, orc.coarse_dims(fd), Ac27)
        assert np.max(np.abs(M - M.T)) < 1e-14 * np.abs(M).max()


# --------------------------------------------------------------------------- #
# Hierarchy: level planning and complexities (Eq. 2, Table 5)                  #
# --------------------------------------------------------------------------- #

def test_level_plans_for_the_workloads(orc):
    assert orc.plan_levels((32, 32, 32)) == [(32, 32, 32), (16, 16, 16), (8, 8, 8), (4, 4, 4)]
    assert len(orc.plan_levels((256,) * 3)) == 7 and orc.plan_levels((256,) * 3)[-1] == (4, 4, 4)
    assert orc.plan_levels((384,) * 3)[-1] == (6, 6, 6) and len(orc.plan_levels((384,) * 3)) == 7
    p4 = orc.plan_levels((128, 128, 64))
    assert len(p4) == 5 and p4[-1] == (8, 8, 4)
    assert orc.plan_levels((10, 12, 14)) == [(10, 12, 14), (5, 6, 7)]


def test_complexities_match_table5(orc):
    gold = json.load(open(os.path.join(GOLD, "complexity.json")))
    d = (32, 32, 32)
    mg = orc.MG(d, I.OFF7, I.laplace7(d).numpy(), smoother=orc.SGS)
    n = [np.prod(mg.level_info(l)[0]) for l in range(mg.nlevels)]
    z = [np.prod(mg.level_info(l)[0]) * len(mg.level_info(l)[1]) for l in range(mg.nlevels)]
    cg, co = sum(n) / n[0], sum(z) / z[0]
    assert round(cg, 2) == gold["laplace_3d7_full_coarsening"]["C_G"]
    assert round(co, 2) == gold["laplace_3d7_full_coarsening"]["C_O"]
    d = (32, 32, 16)
    A = I.block7_layered(d, 0).numpy()
    mg = orc.MG(d, I.OFF7, A, B=3, smoother=orc.SGS, transfer=orc.PC8C)
    n = [np.prod(mg.level_info(l)[0]) for l in range(mg.nlevels)]
    z = [np.prod(mg.level_info(l)[0]) * len(mg.level_info(l)[1]) for l in range(mg.nlevels)]
    assert round(sum(n) / n[0], 2) == gold["oil4c_3d7_cell_3d8"]["C_G"]
    assert round(sum(z) / z[0], 2) == gold["oil4c_3d7_cell_3d8"]["C_O"]


# --------------------------------------------------------------------------- #
# V-cycle                                                                       #
# --------------------------------------------------------------------------- #

def _dense_sgs_from_zero(M, f):
    u = sla.solve_triangular(np.tril(M), f, lower=True)
    return u + sla.solve_triangular(np.triu(M), f - M @ u, lower=False)


def _dense_sgs(M, f, u):
    u = u + sla.solve_triangular(np.tril(M), f - M @ u, lower=True)
    return u + sla.solve_triangular(np.triu(M), f - M @ u, lower=False)


def test_two_level_vcycle_matches_dense_algebra(orc):
    """Two-level V(1,1) with symmetric GS written with dense matrices:
    u = S f; u += P A_c^{-1} R (f - A u); u = S(u)."""
    fd = (10, 8, 8)
    A = I.q1_aniso27(fd, 1).numpy()
    mg = orc.MG(fd, I.OFF27, A, smoother=orc.SGS, max_levels=2)
    assert mg.nlevels == 2
    M = orc.assemble_dense(fd, I.OFF27, A)
    P = _dense_transfer(orc, orc.FW27V, fd)
    R = P.T / 8
    Ac = R @ M @ P
    f = np.random.default_rng(2).normal(size=M.shape[0])
    u = _dense_sgs_from_zero(M, f)
    u = u + P @ np.linalg.solve(Ac, R @ (f - M @ u))
    u = _dense_sgs(M, f, u)
    z = mg.vcycle(f)
    assert np.max(np.abs(z - u)) < 1e-11 * np.abs(u).max()


def test_two_level_ilu_vcycle_matches_dense_algebra(orc):
    fd = (8, 10, 8)
    A = I.q1_aniso27(fd, 2).numpy()
    mg = orc.MG(fd, I.OFF27, A, smoother=orc.ILU0, max_levels=2)
    assert mg.nlevels == 2
    M = orc.assemble_dense(fd, I.OFF27, A)
    L, U = _dense_lu_from_stencil(orc, fd, I.OFF27, orc.ilu0_factor(fd, I.OFF27, A))
    S = lambda r: sla.solve_triangular(U, sla.solve_triangular(L, r, lower=True, unit_diagonal=True))
    P = _dense_transfer(orc, orc.FW27V, fd)
    R = P.T / 8
    f = np.random.default_rng(3).normal(size=M.shape[0])
    u = S(f)
    u = u + P @ np.linalg.solve(R @ M @ P, R @ (f - M @ u))
    u = u + S(f - M @ u)
    z = mg.vcycle(f)
    assert np.max(np.abs(z - u)) < 1e-11 * np.abs(u).max()


@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycle_is_symmetric_for_spd(orc, smoother):
    """SGS pre/post and ILU(0) of an SPD matrix give a symmetric preconditioner
    (needed by PCG): <M x, y> = <x, M y>."""
    d = (16, 16, 16)
    A = I.q1_aniso27(d, 4).numpy()
    mg = orc.MG(d, I.OFF27, A, smoother=smoother)
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=4096), rng.normal(size=4096)
    a, b = mg.vcycle(x) @ y, x @ mg.vcycle(y)
    assert abs(a - b) < 1e-12 * abs(a)


def test_vcycle_contracts_as_stationary_iteration(orc):
    """Manufactured solution: u_{k+1} = u_k + M^{-1}(b - A u_k) converges."""
    d = (32, 32, 32)
    A = I.laplace7(d).numpy()
    mg = orc.MG(d, I.OFF7, A, smoother=orc.SGS)
    xs = np.random.default_rng(1).normal(size=32 ** 3)
    b = orc.spmv(d, I.OFF7, A, xs)
    u = np.zeros_like(b)
    errs = []
    for _ in range(6):
        u = u + mg.vcycle(b - orc.spmv(d, I.OFF7, A, u))
        errs.append(np.linalg.norm(u - xs))
    rates = [errs[t + 1] / errs[t] for t in range(len(errs) - 1)]
    assert max(rates[1:]) < 0.2


# --------------------------------------------------------------------------- #
# Krylov                                                                        #
# --------------------------------------------------------------------------- #

def test_pcg_with_exact_preconditioner_takes_one_step(orc):
    """A one-level hierarchy is the dense direct solve: M^{-1} = A^{-1}."""
    d = (6, 5, 4)
    A = I.q1_aniso27(d, 1).numpy()
    mg = orc.MG(d, I.OFF27, A, smoother=orc.SGS, max_levels=1)
    b = I.rhs(120, 3).numpy()
    x, rc, it, rr, _ = mg.pcg(b, tol=1e-12)
    assert rc == 0 and it == 1 and rr < 1e-13
    x, rc, it, rr, _ = mg.fgmres(b, tol=1e-12)
    assert rc == 0 and it == 1 and rr < 1e-13


def test_pcg_manufactured_solution(orc):
    d = (24, 24, 24)
    A = I.q1_aniso27(d, 2).numpy()
    xs = np.random.default_rng(4).normal(size=24 ** 3)
    b = orc.spmv(d, I.OFF27, A, xs)
    for sm in (orc.SGS, orc.ILU0):
        mg = orc.MG(d, I.OFF27, A, smoother=sm)
        x, rc, it, rr, hist = mg.pcg(b, tol=1e-10)
        assert rc == 0 and rr < 1e-10 and it < 60
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6
        assert np.all(np.diff(np.log(hist)) < 0.5)


def test_flexible_pcg_equals_pcg_for_fixed_preconditioner(orc):
    """With a fixed symmetric M, r_{k+1} is M-orthogonal to r_k in exact
    arithmetic, so the Polak-Ribiere beta equals Fletcher-Reeves and both
    variants take the same number of iterations."""
    d = (16, 16, 16)
    A = I.laplace7(d).numpy()
    mg = orc.MG(d, I.OFF7, A, smoother=orc.SGS)
    b = I.rhs(4096, 0).numpy()
    _, _, it1, rr1, _ = mg.pcg(b, tol=1e-9)
    _, _, it2, rr2, _ = mg.pcg(b, tol=1e-9, flexible=True)
    assert it1 == it2 and rr1 < 1e-9 and rr2 < 1e-9


def test_fgmres_block_system(orc):
    d = (16, 16, 16)
    A = I.block7_layered(d, 1).numpy()
    mg = orc.MG(d, I.OFF7, A, B=3, smoother=orc.SGS, transfer=orc.PC8C)
    xs = np.random.default_rng(6).normal(size=3 * 16 ** 3)
    b = orc.spmv(d, I.OFF7, A, xs, B=3)
    x, rc, it, rr, hist = mg.fgmres(b, tol=1e-10, restart=30, maxit=300)
    assert rc == 0 and rr < 1e-10
    M = orc.assemble_dense((4, 4, 4), I.OFF7, I.block7_layered((4, 4, 4), 1).numpy(), B=3)
    assert np.abs(M - M.T).max() > 1e-2 * np.abs(M).max()  # the block system really is nonsymmetric


# --------------------------------------------------------------------------- #
# Reduced precision                                                             #
# --------------------------------------------------------------------------- #

def _bf16_neighbours(x):
    """The two bf16 values around x (bf16 = float32 with the low 16 bits zero)."""
    f = np.array([x], dtype=np.float32)
    bits = f.view(np.uint32)[0] & np.uint32(0xFFFF0000)
    lo = np.array([bits], dtype=np.uint32).view(np.float32)[0]
    hi = np.array([bits + np.uint32(0x10000)], dtype=np.uint32).view(np.float32)[0]
    return float(lo), float(hi), int(bits >> 16)


def test_bf16_rounding_nearest_even(orc):
    rng = np.random.default_rng(0)
    xs = list(rng.normal(size=2000) * 10.0 ** rng.integers(-8, 8, size=2000))
    xs += [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 255.5, 1.0 - 2 ** -10]
    for x in xs:
        ax = abs(x)
        lo, hi, lobits = _bf16_neighbours(ax)
        # float32 rounding of x may have crossed lo; pick the true neighbours
        if lo > ax:
            hi = lo
            lo = float(np.array([(np.float32(lo).view(np.uint32) - np.uint32(0x10000))], dtype=np.uint32).view(np.float32)[0])
            lobits -= 1
        dl, dh = ax - lo, hi - ax
        ref = lo if (dl < dh or (dl == dh and lobits % 2 == 0)) else hi
        got = orc.bf16_round(x)
        assert got == math.copysign(ref, x), (x, got, ref)


def test_mixed_precision_vcycles_track_fp64(orc):
    d = (16, 16, 16)
    A = I.q1_aniso27(d, 6).numpy()
    r = I.rhs(4096, 1).numpy()
    for sm in (orc.SGS, orc.ILU0):
        z64 = orc.MG(d, I.OFF27, A, smoother=sm).vcycle(r)
        z32 = orc.MG(d, I.OFF27, A, smoother=sm, precision=orc.FP32).vcycle(r)
        zbf = orc.MG(d, I.OFF27, A, smoother=sm, precision=orc.BF16).vcycle(r)
        e32 = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
        ebf = np.linalg.norm(zbf - z64) / np.linalg.norm(z64)
        assert 1e-9 < e32 < 1e-4
        assert e32 < ebf < 0.1


def test_lowered_matrix_row_scaling(orc):
    d = (8, 8, 8)
    A = I.q1_aniso27(d, 7).numpy()
    mg = orc.MG(d, I.OFF27, A, smoother=orc.SGS, precision=orc.BF16)
    vals = mg.level_array(0, 3).reshape(-1, 27)
    sc = mg.level_array(0, 4)
    assert np.all(sc == np.abs(A).max(axis=1).astype(np.float32))
    for p in (0, 100, 511):
        for e in range(27):
            assert vals[p, e] == orc.bf16_round(A[p, e] / float(sc[p]))
    assert np.all(np.abs(vals) <= 1.0)


def test_bf16_block_hierarchy_is_rejected(orc):
    """Row-scaled BF16 exists for scalar problems only; a block problem with a
    BF16 hierarchy must be refused, not silently mis-sized (FP32 blocks are
    supported, see test_oracle_mixed_pins.py)."""
    from paper_2506_21932_gb300 import inputs as I
    d = (8, 8, 8)
    A = I.block7_layered(d, 1).numpy()
    with pytest.raises(ValueError):
        orc.MG(d, I.OFF7, A, B=3, transfer=orc.PC8C, precision=2)
