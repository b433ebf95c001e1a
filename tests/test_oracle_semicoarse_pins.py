"""Pins of the oracle's 2-D semi-coarsening (transfer 3: x and y coarsened,
z kept; restriction = 2 x 2 cell sum, interpolation = cell-centred bilinear
in x and y, the 2d4c / 2d16c pair of Table 8's weather setting), run with
the z-line smoother.  Checked against: the level plan, exactness of the
interpolation on bilinear-in-(x, y) functions of any z profile, the dense
R A P of the separately assembled operators, a hand-derived Kronecker-sum
closed form of the coarse 7-point Laplacian, and dense two-level algebra."""
import itertools

import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I
from tests.test_oracle_lgs_pins import _column_split
from tests.test_oracle_pins import rnd_matrix

T3 = 3


def _dense_P(orc, fd, B=1):
    cd = orc.coarse_dims(fd, T3)
    nc, nf = int(np.prod(cd)) * B, int(np.prod(fd)) * B
    P = np.zeros((nf, nc))
    for j in range(nc):
        e = np.zeros(nc)
        e[j] = 1.0
        P[:, j] = orc.prolong_add(T3, fd, e, np.zeros(nf), B=B)
    return P


def _dense_R(orc, fd, B=1):
    cd = orc.coarse_dims(fd, T3)
    nc, nf = int(np.prod(cd)) * B, int(np.prod(fd)) * B
    R = np.zeros((nc, nf))
    for q in range(nf):
        e = np.zeros(nf)
        e[q] = 1.0
        R[:, q] = orc.restrict(T3, fd, e, B=B)
    return R


def test_semicoarsening_level_plan(orc):
    assert orc.plan_levels((256, 256, 64), transfer=T3) == [(256 >> l, 256 >> l, 64) for l in range(7)]
    assert orc.plan_levels((16, 24, 15), transfer=T3) == [(16, 24, 15), (8, 12, 15), (4, 6, 15)]
    assert orc.plan_levels((16, 18, 8), transfer=T3) == [(16, 18, 8), (8, 9, 8)]  # odd y stops
    assert orc.plan_levels((16, 16, 16)) == [(16, 16, 16), (8, 8, 8), (4, 4, 4)]  # full coarsening unchanged


def test_semicoarse_interpolation_is_bilinear_per_layer(orc):
    """(a x + b y + c) g(z) is reproduced wherever both coarse neighbours of
    a fine cell exist in x and in y; a coarse unit value spreads over the
    4 x 4 fine cells of its own layer only, with 3/4, 1/4 weights."""
    fd = (12, 10, 5)
    cd = orc.coarse_dims(fd, T3)
    assert cd == [6, 5, 5]
    g = np.array([0.3, -1.0, 2.0, 0.5, 1.5])
    a, b, c = 0.5, -1.25, 2.0
    ec = np.array([(a * (2 * i + 1) + b * (2 * j + 1) + c) * g[k]
                   for i in range(cd[0]) for j in range(cd[1]) for k in range(cd[2])])
    uf = orc.prolong_add(T3, fd, ec, np.zeros(np.prod(fd))).reshape(fd)
    for i, j, k in itertools.product(range(1, fd[0] - 1), range(1, fd[1] - 1), range(fd[2])):
        assert abs(uf[i, j, k] - (a * (i + .5) + b * (j + .5) + c) * g[k]) < 1e-12
    e = np.zeros(np.prod(cd))
    e[(2 * cd[1] + 1) * cd[2] + 3] = 1.0
    uf = orc.prolong_add(T3, fd, e, np.zeros(np.prod(fd))).reshape(fd)
    w = {3: 0.25, 4: 0.75, 5: 0.75, 6: 0.25}
    wy = {1: 0.25, 2: 0.75, 3: 0.75, 4: 0.25}
    for i, j, k in itertools.product(range(fd[0]), range(fd[1]), range(fd[2])):
        assert uf[i, j, k] == (w.get(i, 0.0) * wy.get(j, 0.0) if k == 3 else 0.0)


def test_semicoarse_restriction_is_the_2x2_sum(orc):
    rng = np.random.default_rng(1)
    for fd, B in [((8, 6, 5), 1), ((6, 10, 4), 3)]:
        r = rng.normal(size=int(np.prod(fd)) * B)
        got = orc.restrict(T3, fd, r, B=B)
        f = r.reshape(*fd, B)
        ref = f[0::2, 0::2] + f[0::2, 1::2] + f[1::2, 0::2] + f[1::2, 1::2]
        assert np.max(np.abs(got - ref.reshape(-1))) < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("fd,off,B", [((8, 6, 5), I.OFF7, 1), ((6, 6, 4), I.OFF27, 1), ((6, 8, 3), I.OFF19, 1),
                                      ((8, 4, 3), I.OFF7, 3)])
def test_semicoarse_rap_equals_assembled_triple_product(orc, fd, off, B):
    A = rnd_matrix(fd, off, 41, B=B)
    Ac27, present = orc.rap27(T3, fd, off, A, B=B)
    M = orc.assemble_dense(fd, off, A, B=B)
    ref = _dense_R(orc, fd, B) @ M @ _dense_P(orc, fd, B)
    cd = orc.coarse_dims(fd, T3)
    got = orc.assemble_dense(cd, np.array(I.OFF27), Ac27.reshape(len(Ac27), -1) if B == 1 else Ac27, B=B)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()


def test_semicoarse_rap_laplace_closed_form(orc):
    """7-point Laplacian = T(x)I(x)I + I(x)T(x)I + I(x)I(x)T.  In x and y the
    cell pair gives R1 T P1 = [-1/2, 1, -1/2] and R1 P1 = [1/4, 3/2, 1/4] (as
    for 3d64c); z is untouched.  So every coarse stencil away from the x-y
    boundary is K'(a) M'(b) d(c) + M'(a) K'(b) d(c) + M'(a) M'(b) T(c): centre
    1.5 + 1.5 + 2.25 * 2 = 7.5, z-neighbours -2.25, x-neighbours -0.5, x-y
    diagonals -0.25, x-z diagonals -0.375, corners -0.0625."""
    fd = (16, 12, 6)
    A = I.laplace7(fd).numpy()
    Ac27, present = orc.rap27(T3, fd, I.OFF7, A)
    kx = {-1: -0.5, 0: 1.0, 1: -0.5}
    mx = {-1: 0.25, 0: 1.5, 1: 0.25}
    tz = {-1: -1.0, 0: 2.0, 1: -1.0}
    dz = {-1: 0.0, 0: 1.0, 1: 0.0}
    cd = orc.coarse_dims(fd, T3)
    for I0, I1, I2 in itertools.product(range(1, cd[0] - 1), range(1, cd[1] - 1), range(1, cd[2] - 1)):
        P = (I0 * cd[1] + I1) * cd[2] + I2
        for e, (a, b, c) in enumerate(I.OFF27):
            ref = kx[a] * mx[b] * dz[c] + mx[a] * kx[b] * dz[c] + mx[a] * mx[b] * tz[c]
            assert abs(Ac27[P, e, 0, 0] - ref) < 1e-14
        assert abs(Ac27[P, 13, 0, 0] - 7.5) < 1e-14 and abs(Ac27[P, 12, 0, 0] + 2.25) < 1e-14
        assert abs(Ac27[P, 26, 0, 0] + 0.0625) < 1e-14 and abs(Ac27[P].sum()) < 1e-13


def test_two_level_semicoarse_lgs_vcycle_matches_dense_algebra(orc):
    fd = (8, 10, 6)
    A = I.q1_aniso27(fd, 3, aniso=(1e-2, 1e-2, 1.0)).numpy()
    mg = orc.MG(fd, I.OFF27, A, smoother=orc.LGS, transfer=T3, max_levels=2)
    assert mg.nlevels == 2 and tuple(mg.level_info(1)[0]) == (4, 5, 6)
    M = orc.assemble_dense(fd, I.OFF27, A)
    D, L, U = _column_split(fd, M)
    fwd = lambda f, u: np.linalg.solve(D + L, f - U @ u)
    bwd = lambda f, u: np.linalg.solve(D + U, f - L @ u)
    P, R = _dense_P(orc, fd), _dense_R(orc, fd)
    f = np.random.default_rng(2).normal(size=M.shape[0])
    u = bwd(f, fwd(f, np.zeros_like(f)))
    u = u + P @ np.linalg.solve(R @ M @ P, R @ (f - M @ u))
    u = bwd(f, fwd(f, u))
    z = mg.vcycle(f)
    assert np.max(np.abs(z - u)) < 1e-11 * np.abs(u).max()


def test_semicoarse_lgs_solves_z_anisotropy(orc):
    """Strong z coupling, x-y semi-coarsening with z-line smoothing: FGMRES
    and flexible PCG reach 1e-10 in a handful of iterations."""
    d = (32, 32, 24)
    A = I.q1_aniso27(d, 2, aniso=(1e-3, 1e-3, 1.0)).numpy()
    xs = np.random.default_rng(3).normal(size=int(np.prod(d)))
    b = orc.spmv(d, I.OFF27, A, xs)
    mg = orc.MG(d, I.OFF27, A, smoother=orc.LGS, transfer=T3)
    x, rc, it, rr, _ = mg.fgmres(b, tol=1e-10, restart=30, maxit=100)
    assert rc == 0 and rr < 1e-10 and it <= 12
    x, rc, it2, rr, _ = mg.pcg(b, tol=1e-10, flexible=True, maxit=100)
    assert rc == 0 and rr < 1e-10 and it2 <= 15
