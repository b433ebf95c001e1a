"""Pins of the oracle's cell-centred transfer pair: 3d64c (trilinear, cell
centred) interpolation with 3d8c restriction, the combination of Table 2's
columns 3d8c / 3d19 / 3d64c and 3d8c / 3d27 / 3d64c and of the Table 8
settings for rhd-3T and solid-3D.  Each pin checks the oracle against
something it does not compute itself: exactness on linear functions, dense
matrix products of the separately assembled R, A and P, a hand-derived
Kronecker-sum closed form, and dense two-level algebra."""
import itertools

import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I
from tests.test_oracle_pins import _dense_lu_from_stencil, _dense_sgs, _dense_sgs_from_zero, rnd_matrix

sla = pytest.importorskip("scipy.linalg")


def _dense_P(orc, transfer, fd, B=1):
    nc = int(np.prod(orc.coarse_dims(fd))) * B
    nf = int(np.prod(fd)) * B
    P = np.zeros((nf, nc))
    for j in range(nc):
        e = np.zeros(nc)
        e[j] = 1.0
        P[:, j] = orc.prolong_add(transfer, fd, e, np.zeros(nf), B=B)
    return P


def _dense_R(orc, transfer, fd, B=1):
    nc = int(np.prod(orc.coarse_dims(fd))) * B
    nf = int(np.prod(fd)) * B
    R = np.zeros((nc, nf))
    for q in range(nf):
        e = np.zeros(nf)
        e[q] = 1.0
        R[:, q] = orc.restrict(transfer, fd, e, B=B)
    return R


def test_cell_interpolation_reproduces_linear_functions(orc):
    """Fine cell v has its centre at v + 1/2 and coarse cell I at 2I + 1 (in
    fine cell widths).  Linear interpolation between cell centres is exact for
    linear functions wherever both coarse neighbours of a fine cell exist, i.e.
    everywhere but the first and last fine cell of each line."""
    fd = (12, 10, 8)
    cd = orc.coarse_dims(fd)
    a, b, c, e0 = 0.5, -1.25, 0.75, 2.0
    ec = np.array([a * (2 * i + 1) + b * (2 * j + 1) + c * (2 * k + 1) + e0
                   for i in range(cd[0]) for j in range(cd[1]) for k in range(cd[2])])
    uf = orc.prolong_add(orc.C64C, fd, ec, np.zeros(np.prod(fd))).reshape(fd)
    for i, j, k in itertools.product(range(1, fd[0] - 1), range(1, fd[1] - 1), range(1, fd[2] - 1)):
        assert abs(uf[i, j, k] - (a * (i + .5) + b * (j + .5) + c * (k + .5) + e0)) < 1e-12


def test_cell_interpolation_weights_and_boundary_reading(orc):
    """Per dimension the weights are 3/4 (own coarse cell) and 1/4 (the
    neighbour on the side of the fine cell); a neighbour off the grid is
    dropped, so a constant is reproduced inside and scaled by 3/4 per boundary
    face that the fine cell touches."""
    fd = (8, 8, 8)
    cd = orc.coarse_dims(fd)
    uf = orc.prolong_add(orc.C64C, fd, np.ones(np.prod(cd)), np.zeros(np.prod(fd))).reshape(fd)
    for i, j, k in itertools.product(range(8), repeat=3):
        faces = sum(t in (0, 7) for t in (i, j, k))
        assert uf[i, j, k] == 0.75 ** faces
    # a single coarse unit value at J = (1,1,1) spreads over fine 2J + {-1,0,1,2}^3
    e = np.zeros(np.prod(cd))
    e[(1 * cd[1] + 1) * cd[2] + 1] = 1.0
    uf = orc.prolong_add(orc.C64C, fd, e, np.zeros(np.prod(fd))).reshape(fd)
    w = {1: 0.25, 2: 0.75, 3: 0.75, 4: 0.25}
    for i, j, k in itertools.product(range(8), repeat=3):
        ref = w.get(i, 0.0) * w.get(j, 0.0) * w.get(k, 0.0)
        assert uf[i, j, k] == ref
    assert np.count_nonzero(uf) == 64


def test_cell64_restriction_is_the_3d8c_sum(orc):
    rng = np.random.default_rng(0)
    for fd in [(8, 6, 4), (6, 10, 8)]:
        for B in (1, 3):
            r = rng.normal(size=int(np.prod(fd)) * B)
            a = orc.restrict(orc.C64C, fd, r, B=B)
            assert np.array_equal(a, orc.restrict(orc.PC8C, fd, r, B=B))
            f = r.reshape(*fd, B)
            ref = sum(f[x::2, y::2, z::2] for x, y, z in itertools.product((0, 1), repeat=3))
            assert np.max(np.abs(a - ref.reshape(-1))) < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("fd,off,B", [
    ((8, 6, 4), I.OFF7, 1), ((6, 6, 6), I.OFF27, 1), ((6, 8, 4), I.OFF19, 1), ((8, 4, 6), I.OFF7, 3)])
def test_cell64_rap_equals_assembled_triple_product(orc, fd, off, B):
    """Brute-force chain sum against R A P with R and P assembled from the
    restriction and interpolation routines."""
    A = rnd_matrix(fd, off, 31, B=B)
    Ac27, present = orc.rap27(orc.C64C, fd, off, A, B=B)
    M = orc.assemble_dense(fd, off, A, B=B)
    ref = _dense_R(orc, orc.C64C, fd, B) @ M @ _dense_P(orc, orc.C64C, fd, B)
    cd = orc.coarse_dims(fd)
    got = orc.assemble_dense(cd, np.array(I.OFF27), Ac27.reshape(len(Ac27), -1) if B == 1 else Ac27, B=B)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()
    assert present.sum() == 27


def test_cell64_rap_laplace_closed_form(orc):
    """Constant 7-point Laplacian = T(x)I(x)I + I(x)T(x)I + I(x)I(x)T with
    T = tridiag(-1,2,-1).  By hand, in 1-D: P e_J = (1/4, 3/4, 3/4, 1/4) on
    fine cells 2J-1..2J+2, so R1 P1 = [1/4, 3/2, 1/4] and R1 T P1 = [-1/2, 1,
    -1/2].  Every interior coarse stencil is therefore the Kronecker sum
    K'(x)M'(x)M' + M'(x)K'(x)M' + M'(x)M'(x)K' with centre 3 * (3/2)^2 = 6.75
    and face value -1/2 (3/2)^2 + 2 (1/4)(3/2) = -3/8."""
    fd = (16, 16, 16)
    A = I.laplace7(fd).numpy()
    Ac27, present = orc.rap27(orc.C64C, fd, I.OFF7, A)
    t = {-1: -0.5, 0: 1.0, 1: -0.5}
    m = {-1: 0.25, 0: 1.5, 1: 0.25}
    cd = orc.coarse_dims(fd)
    assert present.sum() == 27
    for I0, I1, I2 in itertools.product(range(1, cd[0] - 1), (1, 4, 6), (2, 5)):
        P = (I0 * cd[1] + I1) * cd[2] + I2
        for e, (a, b, c) in enumerate(I.OFF27):
            ref = t[a] * m[b] * m[c] + m[a] * t[b] * m[c] + m[a] * m[b] * t[c]
            assert abs(Ac27[P, e, 0, 0] - ref) < 1e-14
        assert abs(Ac27[P, 13, 0, 0] - 6.75) < 1e-14 and abs(Ac27[P, 4, 0, 0] + 0.375) < 1e-14
        assert abs(Ac27[P].sum()) < 1e-13


def test_cell64_coarse_operator_is_nonsymmetric(orc):
    """R is not a multiple of P^T, so a variable-coefficient symmetric fine
    operator gets a nonsymmetric coarse operator (the reason the pair is run
    under flexible or nonsymmetric Krylov methods here)."""
    fd = (8, 8, 6)
    A = I.varcoef7(fd, 3)[0].numpy()
    M = orc.assemble_dense(fd, I.OFF7, A)
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    Ac27, _ = orc.rap27(orc.C64C, fd, I.OFF7, A)
    C = orc.assemble_dense(orc.coarse_dims(fd), np.array(I.OFF27), Ac27.reshape(len(Ac27), -1))
    assert np.abs(C - C.T).max() > 1e-3 * np.abs(C).max()


@pytest.mark.parametrize("smoother", [0, 1])
def test_two_level_cell64_vcycle_matches_dense_algebra(orc, smoother):
    """Two-level V(1,1) with the cell-centred pair, written with dense
    matrices: u = S f; u += P A_c^{-1} R (f - A u); u = S'(f, u)."""
    fd = (8, 10, 8)
    A = I.varcoef7(fd, 2)[0].numpy()
    mg = orc.MG(fd, I.OFF7, A, smoother=smoother, transfer=orc.C64C, max_levels=2)
    assert mg.nlevels == 2
    M = orc.assemble_dense(fd, I.OFF7, A)
    P, R = _dense_P(orc, orc.C64C, fd), _dense_R(orc, orc.C64C, fd)
    f = np.random.default_rng(7).normal(size=M.shape[0])
    if smoother == 0:
        u = _dense_sgs_from_zero(M, f)
        u = u + P @ np.linalg.solve(R @ M @ P, R @ (f - M @ u))
        u = _dense_sgs(M, f, u)
    else:
        L, U = _dense_lu_from_stencil(orc, fd, I.OFF7, orc.ilu0_factor(fd, I.OFF7, A))
        S = lambda r: sla.solve_triangular(U, sla.solve_triangular(L, r, lower=True, unit_diagonal=True))
        u = S(f)
        u = u + P @ np.linalg.solve(R @ M @ P, R @ (f - M @ u))
        u = u + S(f - M @ u)
    z = mg.vcycle(f)
    assert np.max(np.abs(z - u)) < 1e-11 * np.abs(u).max()


def test_cell64_hierarchy_solves_with_flexible_and_gmres(orc):
    """Manufactured solution on a heterogeneous cell-centred problem: FPCG and
    FGMRES preconditioned by the cell-centred hierarchy reach the tolerance,
    and the stationary V-cycle iteration contracts."""
    d = (16, 16, 16)
    A = I.varcoef7(d, 1)[0].numpy()
    xs = np.random.default_rng(9).normal(size=16 ** 3)
    b = orc.spmv(d, I.OFF7, A, xs)
    for sm in (orc.SGS, orc.ILU0):
        mg = orc.MG(d, I.OFF7, A, smoother=sm, transfer=orc.C64C)
        x, rc, it, rr, _ = mg.pcg(b, tol=1e-10, flexible=True, maxit=200)
        assert rc == 0 and rr < 1e-10 and it < 60
        x, rc, it, rr, _ = mg.fgmres(b, tol=1e-10, restart=30, maxit=200)
        assert rc == 0 and rr < 1e-10 and it < 60
        u = np.zeros_like(b)
        errs = []
        for _ in range(5):
            u = u + mg.vcycle(b - orc.spmv(d, I.OFF7, A, u))
            errs.append(np.linalg.norm(u - xs))
        assert errs[-1] < 0.5 * errs[-2]


def test_cell64_mg_rejects_unknown_transfer(orc):
    d = (8, 8, 8)
    with pytest.raises(Exception):
        orc.MG(d, I.OFF7, I.laplace7(d).numpy(), transfer=4)
