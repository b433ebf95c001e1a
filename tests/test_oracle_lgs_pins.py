"""Pins of the oracle's line Gauss-Seidel smoother (LGS along z, Sec. 4.4:
the points of a column are updated together, the off-column couplings form
the right-hand side and the column's tridiagonal system is solved by the
Thomas algorithm).  Checked against dense block-triangular algebra on the
assembled matrix, exactness for decoupled columns, symmetry of the V-cycle
and the line smoother's known advantage on grid-aligned anisotropy
(Sec. 5.4: LGS is the better smoother when the strong direction is the
line direction)."""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I
from tests.test_oracle_pins import _dense_transfer, rnd_matrix, sym_random

sla = pytest.importorskip("scipy.linalg")


def _column_split(d, M):
    """Split the dense matrix by z-column index c = i*ny + j of row and column:
    in-column block diagonal D, earlier columns L, later columns U."""
    c = np.repeat(np.arange(d[0] * d[1]), d[2])
    same = c[:, None] == c[None, :]
    lower = c[:, None] > c[None, :]
    return np.where(same, M, 0.0), np.where(lower, M, 0.0), np.where(~same & ~lower, M, 0.0)


@pytest.mark.parametrize("off,d", [(I.OFF7, (4, 5, 6)), (I.OFF27, (5, 4, 7)), (I.OFF19, (3, 6, 5))])
def test_lgs_sweeps_are_block_triangular_solves(orc, off, d):
    """Forward LGS = (D + L)^{-1} (b - U u), backward LGS = (D + U)^{-1} (b - L u)
    with the column blocks of the assembled matrix."""
    A = rnd_matrix(d, off, 4)
    M = orc.assemble_dense(d, off, A)
    D, L, U = _column_split(d, M)
    rng = np.random.default_rng(1)
    b, u = rng.normal(size=(2, M.shape[0]))
    got = orc.lgs_forward(d, off, A, b, u)
    ref = np.linalg.solve(D + L, b - U @ u)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()
    got = orc.lgs_backward(d, off, A, b, u)
    ref = np.linalg.solve(D + U, b - L @ u)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


def test_lgs_column_solve_is_exact_for_decoupled_columns(orc):
    """With only the (0,0,+-1) couplings every column is independent and one
    sweep solves A u = b exactly (the Thomas algorithm is exact elimination)."""
    d = (3, 4, 50)
    A = rnd_matrix(d, I.OFF7, 8)
    for e, o in enumerate(I.OFF7):
        if o[0] != 0 or o[1] != 0:
            A[:, e] = 0.0
    M = orc.assemble_dense(d, I.OFF7, A)
    b = np.random.default_rng(2).normal(size=M.shape[0])
    u = orc.lgs_forward(d, I.OFF7, A, b, np.full(M.shape[0], 7.0))
    assert np.max(np.abs(M @ u - b)) < 1e-12 * np.abs(b).max()
    # one column alone against the banded solver
    col = M[:50, :50]
    ab = np.zeros((3, 50))
    ab[0, 1:], ab[1], ab[2, :-1] = np.diag(col, 1), np.diag(col), np.diag(col, -1)
    assert np.max(np.abs(u[:50] - sla.solve_banded((1, 1), ab, b[:50]))) < 1e-12 * np.abs(u[:50]).max()


def test_lgs_zero_guess_equals_lower_columns_only(orc):
    """From u = 0 the forward sweep is (D + L)^{-1} b: the later columns add
    nothing (ZeroGuess)."""
    d = (4, 4, 5)
    A = rnd_matrix(d, I.OFF27, 5)
    M = orc.assemble_dense(d, I.OFF27, A)
    D, L, _ = _column_split(d, M)
    b = np.random.default_rng(3).normal(size=M.shape[0])
    got = orc.lgs_forward(d, I.OFF27, A, b, np.zeros_like(b))
    assert np.max(np.abs(got - np.linalg.solve(D + L, b))) < 1e-12 * np.abs(got).max()


def test_lgs_pivot_check(orc):
    d = (8, 8, 8)
    A = I.laplace7(d).numpy()
    assert orc.lgs_check(d, I.OFF7, A) == orc.ORC_OK
    B = A.copy()
    B[(0 * 8 + 1) * 8 + 0, 3] = 0.0  # first pivot of column (0, 1) vanishes
    assert orc.lgs_check(d, I.OFF7, B) == orc.ORC_EBREAKDOWN
    with pytest.raises(ValueError):
        orc.MG(d, I.OFF7, B, smoother=orc.LGS)
    with pytest.raises(ValueError):
        orc.MG(d, I.OFF7, A, smoother=orc.LGS, w=1.2)  # line smoothing takes weight 1 only


def test_two_level_lgs_vcycle_matches_dense_algebra(orc):
    """u = S_b S_f(0); u += P A_c^{-1} R (f - A u); u = S_b S_f(u) with the
    block-triangular sweeps written densely."""
    fd = (8, 10, 8)
    A = I.q1_aniso27(fd, 2, aniso=(1e-2, 1e-2, 1.0)).numpy()
    mg = orc.MG(fd, I.OFF27, A, smoother=orc.LGS, max_levels=2)
    assert mg.nlevels == 2
    M = orc.assemble_dense(fd, I.OFF27, A)
    D, L, U = _column_split(fd, M)
    fwd = lambda f, u: np.linalg.solve(D + L, f - U @ u)
    bwd = lambda f, u: np.linalg.solve(D + U, f - L @ u)
    P = _dense_transfer(orc, orc.FW27V, fd)
    R = P.T / 8
    f = np.random.default_rng(5).normal(size=M.shape[0])
    u = bwd(f, fwd(f, np.zeros_like(f)))
    u = u + P @ np.linalg.solve(R @ M @ P, R @ (f - M @ u))
    u = bwd(f, fwd(f, u))
    z = mg.vcycle(f)
    assert np.max(np.abs(z - u)) < 1e-11 * np.abs(u).max()


def test_lgs_vcycle_is_symmetric_for_spd(orc):
    """Forward then backward block GS is a symmetric smoother for SPD A, so the
    V-cycle can precondition plain PCG."""
    d = (16, 16, 16)
    A = sym_random(d, I.OFF27, 6)
    mg = orc.MG(d, I.OFF27, A, smoother=orc.LGS)
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=(2, 4096))
    a, b = mg.vcycle(x) @ y, x @ mg.vcycle(y)
    assert abs(a - b) < 1e-12 * abs(a)


def test_lgs_wins_on_z_aligned_anisotropy(orc):
    """Strong coupling along the lines (k_z = 1, k_x = k_y = 1e-3): the line
    smoother removes the anisotropy that point GS cannot (cf. the LGS column
    of Table 6), and it stays competitive on the isotropic Laplacian."""
    d = (24, 24, 24)
    A = I.q1_aniso27(d, 1, aniso=(1e-3, 1e-3, 1.0)).numpy()
    b = I.rhs(24 ** 3, 4).numpy()
    it = {}
    for sm in (orc.SGS, orc.LGS):
        x, rc, it[sm], rr, _ = orc.MG(d, I.OFF27, A, smoother=sm).pcg(b, tol=1e-9, maxit=500)
        assert rc == 0 and rr < 1e-9
    assert it[orc.LGS] <= 10 and it[orc.SGS] >= 5 * it[orc.LGS]
    A = I.laplace7(d).numpy()
    x, rc, itl, rr, _ = orc.MG(d, I.OFF7, A, smoother=orc.LGS).pcg(b, tol=1e-9)
    assert rc == 0 and itl <= 8
