"""Pins of the oracle's reduced-precision (FP32 / BF16) cycle against facts
it does not compute itself.

The reduced-precision hierarchy is not in the paper: its definition (every
level array cast to FP32, or BF16 values with one FP32 row scale applied to
the finished row sum; all level arithmetic and accumulation in FP32; the
coarsest solve in FP64) is the build's.  Two kinds of pins hold the oracle to
that definition:

* Exactness pins.  On small-integer data with unit or power-of-two scales,
  every FP32 and BF16 operation is exact, so each reduced-precision
  operation -- and a whole V-cycle -- must equal the FP64 operation
  bit for bit.  A wrong array (L for U, A for the factors), a wrong row
  scale, a wrong transfer weight or a dropped term breaks the equality.
* Rounding pins.  A row whose sum provably rounds in FP32 (2^24 + 1) must
  give the FP32 result, not the FP64 one: they catch accumulation in double,
  a row scale applied before the sum instead of after it, and a correction
  added in double.

Matrices of the exactness pins couple points only inside 2x2x2 cells, so a
Gauss-Seidel or triangular-solve chain is at most 8 points long and the
integers stay small (each test checks that precondition)."""
import itertools

import numpy as np
import pytest
import torch

from paper_2506_21932_gb300 import inputs as I

OFF27 = I.OFF27
EC = OFF27.index((0, 0, 0))


def oidx(o):
    return (o[0] + 1) * 9 + (o[1] + 1) * 3 + (o[2] + 1)


def cells(d):
    """The 2x2x2 cells of an even grid: lists of 8 point indices in
    lexicographic (= sweep) order."""
    out = []
    for a, b, c in itertools.product(range(0, d[0], 2), range(0, d[1], 2), range(0, d[2], 2)):
        pts = [((a + x) * d[1] + (b + y)) * d[2] + (c + z) for x, y, z in itertools.product((0, 1), repeat=3)]
        out.append((pts, [(a + x, b + y, c + z) for x, y, z in itertools.product((0, 1), repeat=3)]))
    return out


def cell_matrix(d, seed, B=1, kind="antisym", density=0.5):
    """Identity diagonal (blocks) plus integer couplings in {-1, 0, 1} inside
    each 2x2x2 cell.  kind "antisym": a_uv = -a_vu, so every cell's entries sum
    to 8 I and the 3d8c coarse operator is 8 I.  kind "lower": only couplings
    to earlier points of the cell, half +1 and half -1 per cell (the matrix is
    its own unit-lower ILU(0) factor, and the cell sums are again 8 I)."""
    rng = np.random.default_rng(seed)
    n = d[0] * d[1] * d[2]
    A = np.zeros((n, 27, B, B))
    A[:, EC] = np.eye(B)
    for pts, coords in cells(d):
        pairs = [(s, t) for s in range(8) for t in range(s + 1, 8)]
        if kind == "antisym":
            for s, t in pairs:
                if rng.random() < density:
                    C = rng.integers(-1, 2, size=(B, B)).astype(float)
                    o = tuple(coords[t][q] - coords[s][q] for q in range(3))
                    A[pts[s], oidx(o)] = C
                    A[pts[t], oidx(tuple(-v for v in o))] = -C
        elif kind == "lu":
            # A_cell = L U with unit-lower L (entries +-1) and unit-upper U
            # (entries +-2): ILU(0) keeps every intra-cell entry, so its
            # factors are exactly L and U, with lower row scale 1, upper 2
            Lc, Uc = np.eye(8), np.eye(8)
            for s, t in pairs:
                if rng.random() < 0.3:
                    Lc[t, s] = rng.choice([-1.0, 1.0])
                if rng.random() < 0.3:
                    Uc[s, t] = rng.choice([-2.0, 2.0])
            Ac = Lc @ Uc
            for s, t in itertools.product(range(8), repeat=2):
                if Ac[t, s] != 0.0:
                    o = tuple(coords[s][q] - coords[t][q] for q in range(3))
                    A[pts[t], oidx(o)] = Ac[t, s] * np.eye(B)
        else:
            m = 2 * int(rng.integers(1, 5))
            chosen = rng.choice(len(pairs), size=m, replace=False)
            for q, c in enumerate(chosen):
                s, t = pairs[c]
                o = tuple(coords[s][r] - coords[t][r] for r in range(3))  # from the later point t to s
                A[pts[t], oidx(o)] = (1.0 if q < m // 2 else -1.0) * np.eye(B)
    return A.reshape(n, -1) if B == 1 else A.reshape(n, 27 * B * B)


def small_ints(n, seed, lim):
    return np.random.default_rng(seed).integers(-lim, lim + 1, size=n).astype(np.float64)


def exact_ints(x, bound=2 ** 20):
    """The precondition of an exactness pin: integer values well inside FP32."""
    x = np.asarray(x, dtype=np.float64)
    return np.all(np.abs(x) < bound) and np.all(x == np.round(x))


D8 = (8, 8, 8)
N8 = 512


# --------------------------------------------------------------------------- #
# single operations, exact data                                               #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("prec", [1, 2])
def test_residual_exact_equals_fp64(orc, prec):
    """r = b - s (sum_e v_e x_e) equals the FP64 residual when the row maxima
    are powers of two (BF16 values a/s exact) and the data are integers."""
    rng = np.random.default_rng(3)
    A = np.zeros((N8, 27))
    A[:, EC] = 4.0
    mask = rng.random((N8, 27)) < 0.4
    A[mask] = rng.integers(-3, 4, size=mask.sum())
    A[:, EC] = 4.0
    A = I._zero_offgrid(torch.from_numpy(A), D8, OFF27).numpy()
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, precision=prec, max_levels=2)
    assert np.all(mg.level_array(0, 4) == (4.0 if prec == 2 else 1.0))
    x, b = small_ints(N8, 1, 8), small_ints(N8, 2, 50)
    r32 = mg.level_apply32(0, 0, x=x, b=b, y=np.zeros(N8))
    r64 = orc.residual(D8, OFF27, A, b, x)
    assert exact_ints(r64) and np.array_equal(r32.astype(np.float64), r64)


@pytest.mark.parametrize("prec,B", [(1, 1), (2, 1), (1, 3)])
def test_gauss_seidel_sweeps_exact_equal_fp64(orc, prec, B):
    """Forward and backward FP32 / BF16 sweeps (scalar and 3x3 blocks) equal
    the FP64 sweeps on cell-coupled integer data with unit diagonals."""
    A = cell_matrix(D8, 5, B=B)
    mg = orc.MG(D8, OFF27, A, B=B, smoother=orc.SGS, transfer=orc.PC8C, precision=prec, max_levels=2)
    Dinv = orc.diag_inverse(D8, OFF27, A, B=B)
    b, u0 = small_ints(N8 * B, 7, 20), small_ints(N8 * B, 8, 20)
    f64 = orc.gs_forward(D8, OFF27, A, Dinv, b, u0, B=B)
    f32 = mg.level_apply32(0, 1, x=u0, b=b)
    assert exact_ints(f64) and np.array_equal(f32.astype(np.float64), f64)
    g64 = orc.gs_backward(D8, OFF27, A, Dinv, b, f64, B=B)
    g32 = mg.level_apply32(0, 2, x=f32, b=b)
    assert exact_ints(g64) and np.array_equal(g32.astype(np.float64), g64)


@pytest.mark.parametrize("prec,B", [(1, 1), (2, 1), (1, 3)])
def test_weighted_gauss_seidel_sweeps_exact_equal_fp64(orc, prec, B):
    """With w = 1/2 the Sec. 4.4 update (1 - w) u_p + w v only halves, so on
    the cell-coupled integer data the weighted FP32 / BF16 sweeps equal the
    weighted FP64 sweeps bit for bit; a dropped or misplaced weight breaks
    the equality (the weight changes the result, checked below)."""
    A = cell_matrix(D8, 5, B=B)
    mg = orc.MG(D8, OFF27, A, B=B, smoother=orc.SGS, transfer=orc.PC8C, w=0.5, precision=prec, max_levels=2)
    Dinv = orc.diag_inverse(D8, OFF27, A, B=B)
    b, u0 = small_ints(N8 * B, 7, 20), small_ints(N8 * B, 8, 20)
    f64 = orc.gs_forward(D8, OFF27, A, Dinv, b, u0, w=0.5, B=B)
    assert not np.array_equal(f64, orc.gs_forward(D8, OFF27, A, Dinv, b, u0, B=B))
    f32 = mg.level_apply32(0, 1, x=u0, b=b)
    assert np.array_equal(f64.astype(np.float32).astype(np.float64), f64)  # every value exact in FP32
    assert np.array_equal(f32.astype(np.float64), f64)
    g64 = orc.gs_backward(D8, OFF27, A, Dinv, b, f64, w=0.5, B=B)
    g32 = mg.level_apply32(0, 2, x=f32, b=b)
    assert np.array_equal(g64.astype(np.float32).astype(np.float64), g64)
    assert np.array_equal(g32.astype(np.float64), g64)


@pytest.mark.parametrize("prec", [1, 2])
def test_ilu_apply_exact_equals_fp64(orc, prec):
    """The FP32 / BF16 ILU(0) application (L solve with the lower row scale,
    U solve with the upper one and 1/u_pp) equals the FP64 one on a matrix
    that is its own unit-lower factor, on integer data."""
    A = cell_matrix(D8, 9, kind="lu")
    # (the vertex transfer: a cell sum of L U may vanish, which would make the
    # 3d8c coarse operator singular; this pin only uses level 0)
    mg = orc.MG(D8, OFF27, A, smoother=orc.ILU0, transfer=orc.FW27V, precision=prec, max_levels=2)
    LU = orc.ilu0_factor(D8, OFF27, A)
    assert np.all(LU[:, EC] == 1.0) and exact_ints(LU)  # unit pivots, integer factors
    if prec == 2:  # the two triangles carry different scales
        assert set(np.unique(mg.level_array(0, 6))) == {1.0} and 2.0 in set(np.unique(mg.level_array(0, 8)))
    r = small_ints(N8, 10, 30)
    x64 = orc.ilu0_apply(D8, OFF27, LU, np.ones(N8), r)
    x32 = mg.level_apply32(0, 3, b=r, y=np.zeros(N8))
    assert exact_ints(x64) and np.array_equal(x32.astype(np.float64), x64)


@pytest.mark.parametrize("transfer", [0, 1, 2, 3])
@pytest.mark.parametrize("B", [1, 3])
def test_transfers_exact_equal_fp64(orc, transfer, B):
    """FP32 restriction and prolongation equal the FP64 ones on integer data
    (every weight is a dyadic fraction, exact in FP32)."""
    if B == 3 and transfer not in (1, 2):
        pytest.skip("block problems use the cell-centred transfers")
    A = cell_matrix(D8, 11, B=B)
    mg = orc.MG(D8, OFF27, A, B=B, smoother=orc.SGS, transfer=transfer, precision=1, max_levels=2)
    nc = int(np.prod(orc.coarse_dims(D8, transfer))) * B
    rf = small_ints(N8 * B, 12, 1000)
    fc64 = orc.restrict(transfer, D8, rf, B=B)
    fc32 = mg.level_apply32(0, 4, x=rf, y=np.zeros(nc))
    assert np.all(np.abs(fc64) < 2 ** 14) and np.array_equal(fc32.astype(np.float64), fc64)
    ec, uf = small_ints(nc, 13, 1000), small_ints(N8 * B, 14, 1000)
    up64 = orc.prolong_add(transfer, D8, ec, uf, B=B)
    up32 = mg.level_apply32(0, 5, x=ec, y=uf)
    assert np.array_equal(up32.astype(np.float64), up64)


# --------------------------------------------------------------------------- #
# rounding: sums that provably round in FP32                                  #
# --------------------------------------------------------------------------- #
# 2^24 + 1 is not a float; it rounds to 2^24 (ties to even).  An FP64 sum keeps
# the 1, so each quantity below differs between the two definitions.

T24 = float(2 ** 24)


def pidx(i, j, k, d=D8):
    return (i * d[1] + j) * d[2] + k


def test_residual_accumulates_in_fp32(orc):
    """r_p = b_p - (2^24 + 1) with b_p = 1: FP32 gives -16777215, an FP64
    accumulation -16777216."""
    A = np.zeros((N8, 27))
    A[:, EC] = 1.0
    p = pidx(3, 3, 3)
    A[p, oidx((0, 0, -1))] = A[p, oidx((0, 0, 1))] = 1.0
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, transfer=orc.PC8C, precision=1, max_levels=2)
    x, b = np.zeros(N8), np.zeros(N8)
    x[p - 1], x[p + 1], b[p] = T24, 1.0, 1.0
    r = mg.level_apply32(0, 0, x=x, b=b, y=np.zeros(N8))
    assert r[p] == -16777215.0
    assert orc.residual(D8, OFF27, A, b, x)[p] == -16777216.0


def test_bf16_row_scale_multiplies_the_finished_sum(orc):
    """BF16 row p = 3 (1, 1, 1) (scale 3, values 1): r_p = -3 fl(2^24 + 1) =
    -50331648.  Scaling each term before the sum (3 * 2^24 + 3 -> -50331652)
    or summing in FP64 (3 * 16777217 -> -50331652) would not give it."""
    A = np.zeros((N8, 27))
    A[:, EC] = 1.0
    p = pidx(3, 3, 3)
    A[p, oidx((0, 0, -1))] = A[p, EC] = A[p, oidx((0, 0, 1))] = 3.0
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, transfer=orc.PC8C, precision=2, max_levels=2)
    assert mg.level_array(0, 4)[p] == 3.0
    x = np.zeros(N8)
    x[p - 1], x[p + 1] = T24, 1.0
    r = mg.level_apply32(0, 0, x=x, b=np.zeros(N8), y=np.zeros(N8))
    assert r[p] == -50331648.0


def test_gauss_seidel_accumulates_in_fp32(orc):
    """u_p = (1 - (u_{p-1} + u_{p+1})) with the new u_{p-1} = 2^24 and the old
    u_{p+1} = 1: FP32 gives -16777215."""
    A = np.zeros((N8, 27))
    A[:, EC] = 1.0
    p = pidx(3, 3, 3)
    A[p, oidx((0, 0, -1))] = A[p, oidx((0, 0, 1))] = 1.0
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, transfer=orc.PC8C, precision=1, max_levels=2)
    b, u0 = np.zeros(N8), np.zeros(N8)
    b[p - 1], b[p], u0[p + 1] = T24, 1.0, 1.0
    u = mg.level_apply32(0, 1, x=u0, b=b)
    assert u[p - 1] == T24 and u[p] == -16777215.0
    u64 = orc.gs_forward(D8, OFF27, A, np.ones(N8), b, u0)
    assert u64[p] == -16777216.0


def test_ilu_lower_solve_accumulates_in_fp32(orc):
    """Unit-lower L (= A, U = I): y_p = r_p - (y_{p-nz} + y_{p-1}) with
    y_{p-nz} = 1, y_{p-1} = 2^24, r_p = 1: FP32 gives -16777215."""
    A = np.zeros((N8, 27))
    A[:, EC] = 1.0
    p = pidx(3, 3, 3)
    A[p, oidx((0, -1, 0))] = A[p, oidx((0, 0, -1))] = 1.0
    mg = orc.MG(D8, OFF27, A, smoother=orc.ILU0, transfer=orc.PC8C, precision=1, max_levels=2)
    r = np.zeros(N8)
    r[p - D8[2]], r[p - 1], r[p] = 1.0, T24, 1.0
    x = mg.level_apply32(0, 3, b=r, y=np.zeros(N8))
    assert x[p] == -16777215.0
    assert orc.ilu0_apply(D8, OFF27, A, np.ones(N8), r)[p] == -16777216.0


def test_prolongation_sums_then_adds_in_fp32(orc):
    """Fine point v = (2J0+1, 2J1+1, 2J2+2) takes 1/2 of coarse J and 1/2 of
    J + e_z (vertex transfer): with e = 2^25 and 2 the interpolated value
    rounds to 2^24 in FP32, and 1 + 2^24 rounds again: uf_v = 2^24.  FP64
    gives 2^24 + 2."""
    A = cell_matrix(D8, 21)
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, transfer=orc.FW27V, precision=1, max_levels=2)
    cd = orc.coarse_dims(D8, 0)
    ec = np.zeros(int(np.prod(cd)))
    J = (1, 1, 1)
    ec[pidx(*J, d=cd)] = 2.0 ** 25
    ec[pidx(J[0], J[1], J[2] + 1, d=cd)] = 2.0
    v = pidx(2 * J[0] + 1, 2 * J[1] + 1, 2 * J[2] + 2)
    uf = np.zeros(N8)
    uf[v] = 1.0
    up = mg.level_apply32(0, 5, x=ec, y=uf)
    assert up[v] == T24
    assert orc.prolong_add(0, D8, ec, uf)[v] == T24 + 2


def test_restriction_accumulates_in_fp32_in_support_order(orc):
    """Coarse I gathers the fine corner 2I (weight 1/64), the centre 2I+1
    (1/8) and the corner 2I+2 (1/64) in support order: 1, then 2^24 (the sum
    rounds to 2^24), then 1 (rounds again).  FP32: 2^24; FP64: 2^24 + 2."""
    A = cell_matrix(D8, 22)
    mg = orc.MG(D8, OFF27, A, smoother=orc.SGS, transfer=orc.FW27V, precision=1, max_levels=2)
    cd = orc.coarse_dims(D8, 0)
    I0 = (1, 1, 1)
    rf = np.zeros(N8)
    rf[pidx(2 * I0[0], 2 * I0[1], 2 * I0[2])] = 64.0
    rf[pidx(2 * I0[0] + 1, 2 * I0[1] + 1, 2 * I0[2] + 1)] = 2.0 ** 27
    rf[pidx(2 * I0[0] + 2, 2 * I0[1] + 2, 2 * I0[2] + 2)] = 64.0
    fc = mg.level_apply32(0, 4, x=rf, y=np.zeros(int(np.prod(cd))))
    assert fc[pidx(*I0, d=cd)] == T24
    assert orc.restrict(0, D8, rf)[pidx(*I0, d=cd)] == T24 + 2


# --------------------------------------------------------------------------- #
# whole cycles                                                                #
# --------------------------------------------------------------------------- #

@pytest.mark.parametrize("prec,B,sm", [(1, 1, "sgs"), (2, 1, "sgs"), (1, 3, "sgs"), (1, 1, "ilu"), (2, 1, "ilu")])
def test_reduced_precision_vcycle_exact_equals_fp64(orc, prec, B, sm):
    """A whole FP32 / BF16 V-cycle (3d8c transfers, coarse operator 8 I) on
    integer data equals the FP64 V-cycle bit for bit: the smoothers, the
    residual, both transfers, the casts around the FP64 coarsest solve and the
    arrays each step uses are all pinned at once."""
    kind = "lower" if sm == "ilu" else "antisym"
    A = cell_matrix(D8, 31 + B, B=B, kind=kind, density=0.5 if B == 1 else 0.2)  # blocks grow faster
    smoother = orc.ILU0 if sm == "ilu" else orc.SGS
    r = small_ints(N8 * B, 32, 16)
    z64 = orc.MG(D8, OFF27, A, B=B, smoother=smoother, transfer=orc.PC8C).vcycle(r)
    z32 = orc.MG(D8, OFF27, A, B=B, smoother=smoother, transfer=orc.PC8C, precision=prec).vcycle(r)
    assert np.all(np.abs(z64) < 2 ** 20) and np.all(z64 * 8 == np.round(z64 * 8))  # eighths: 23 bits, exact in FP32
    assert np.array_equal(z32, z64)


def test_fp32_block_vcycle_tracks_fp64(orc):
    """On the layered 3-unknown system the FP32 block cycle differs from the
    FP64 one by FP32 rounding only, and its FGMRES solve reaches the
    tolerance with an FP64 outer iteration."""
    d = (16, 16, 16)
    A = I.block7_layered(d, 1).numpy()
    r = I.rhs(3 * 16 ** 3, 2).numpy()
    m64 = orc.MG(d, I.OFF7, A, B=3, smoother=orc.SGS, transfer=orc.PC8C)
    m32 = orc.MG(d, I.OFF7, A, B=3, smoother=orc.SGS, transfer=orc.PC8C, precision=1)
    z64, z32 = m64.vcycle(r), m32.vcycle(r)
    e = np.linalg.norm(z32 - z64) / np.linalg.norm(z64)
    assert 1e-9 < e < 1e-4
    x, rc, it, rr, _ = m32.fgmres(r, tol=1e-8, restart=30, maxit=200)
    _, rc64, it64, _, _ = m64.fgmres(r, tol=1e-8, restart=30, maxit=200)
    assert rc == 0 and rc64 == 0 and rr < 1e-8 and abs(it - it64) <= 2
