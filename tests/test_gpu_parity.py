"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64): the GPU uses fused multiply-adds and its own summation
order, so every computed value differs from the oracle's by a few units in
the last place, amplified at most by the local cancellation of the stencil
sum.  Single kernels are held to 1e-13 relative to the largest magnitude of
their output; a V-cycle to 1e-12 in the 2-norm (the bound the method's
specification states); FP32 / BF16 hierarchies to their own-precision oracle
at 2e-5 (float epsilon 6e-8 times the growth over a cycle).  Integer and
structural results (level sizes, offsets, sparsity, bf16 bit patterns of
values lowered from identical FP64 inputs) must match exactly.
"""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_KERNEL = 1e-13
TOL_VCYCLE = 1e-12
TOL_LOWP = 2e-5


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_21932_gb300 import build, smg
    build.build()
    return smg


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_max(got, ref):
    ref = np.asarray(ref)
    return np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300)


def rel2(got, ref):
    return np.linalg.norm(np.asarray(got) - ref) / max(np.linalg.norm(ref), 1e-300)


def rnd_sym27(d, seed, off=I.OFF27):
    """Random symmetric, diagonally dominant stencil matrix (exact zero padding)."""
    rng = np.random.default_rng(seed)
    n = d[0] * d[1] * d[2]
    A = np.zeros((n, len(off)))
    idx = np.arange(n).reshape(d)
    for e, o in enumerate(off):
        if o > (0, 0, 0) or o == (0, 0, 0):
            continue
        e2 = off.index(tuple(-t for t in o))
        sl_p = tuple(slice(max(0, -o[t]), d[t] - max(0, o[t])) for t in range(3))
        sl_q = tuple(slice(max(0, o[t]), d[t] + min(0, o[t])) for t in range(3))
        p, q = idx[sl_p].ravel(), idx[sl_q].ravel()
        v = -rng.uniform(0.1, 1.0, size=len(p))
        A[p, e] = v
        A[q, e2] = v
    ec = off.index((0, 0, 0))
    A[:, ec] = np.abs(A).sum(axis=1) + rng.uniform(0.01, 0.5, size=n)
    return A


def make(S, d, off, A, **kw):
    return S.SMG(d, off, cu(A.reshape(len(A), -1) if A.ndim == 2 else A), **kw)


# ---------------------------------------------------------------------------
# single kernels on level 0
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,off,B", [((9, 7, 11), I.OFF7, 1), ((5, 6, 7), I.OFF27, 1), ((6, 9, 5), I.OFF19, 1),
                                     ((7, 5, 6), I.OFF7, 3)])
def test_spmv_and_residual(S, orc, d, off, B):
    A = I.block7_layered(d, 3).numpy() if B == 3 else rnd_sym27(d, 1, off)
    h = make(S, d, off, A, block=B, max_levels=1)
    n = d[0] * d[1] * d[2] * B
    x, b = np.random.default_rng(2).normal(size=(2, n))
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_SPMV, x=cu(x), y=y)
    assert rel_max(host(y), orc.spmv(d, off, A, x, B=B)) < TOL_KERNEL
    h.level_apply(0, S.OP_RESIDUAL, x=cu(x), b=cu(b), y=y)
    assert rel_max(host(y), orc.residual(d, off, A, b, x, B=B)) < TOL_KERNEL


@pytest.mark.parametrize("d,off", [((5, 6, 7), I.OFF27), ((9, 7, 11), I.OFF7), ((6, 9, 5), I.OFF19),
                                   ((1, 1, 13), I.OFF7), ((3, 1, 8), I.OFF27), ((8, 33, 6), I.OFF27),
                                   ((6, 130, 9), I.OFF27), ((5, 97, 7), I.OFF7), ((4, 200, 3), I.OFF19),
                                   ((3, 530, 4), I.OFF27), ((2, 520, 3), I.OFF7)])
def test_gs_sweeps_exact_order(S, orc, d, off):
    """Forward, backward and zero-guess sweeps reproduce the sequential
    lexicographic Gauss-Seidel (ragged grids, ny above one warp, 1-wide)."""
    A = rnd_sym27(d, 3, off)
    n = A.shape[0]
    h = make(S, d, off, A, smoother=S.SGS, max_levels=1)
    Dinv = orc.diag_inverse(d, off, A)
    rng = np.random.default_rng(4)
    b, u0 = rng.normal(size=(2, n))
    lev = 0
    u = cu(u0)
    h.level_apply(lev, S.OP_GS_FORWARD, x=u, b=cu(b))
    ref = orc.gs_forward(d, off, A, Dinv, b, u0)
    assert rel_max(host(u), ref) < TOL_KERNEL
    h.level_apply(lev, S.OP_GS_BACKWARD, x=u, b=cu(b))
    ref = orc.gs_backward(d, off, A, Dinv, b, ref)
    assert rel_max(host(u), ref) < TOL_KERNEL
    u = cu(np.full(n, 123.0))  # ZeroGuess ignores the old contents
    h.level_apply(lev, S.OP_GS_ZERO, x=u, b=cu(b))
    assert rel_max(host(u), orc.gs_forward(d, off, A, Dinv, b, np.zeros(n))) < TOL_KERNEL


def test_gs_sweeps_on_small_odd_grids(S, orc):
    """Grids that are not coarsened: run the sweep through a 2-level hierarchy
    of an even grid whose finest level has the odd-sized neighbours inside."""
    for d, off in [((8, 10, 12), I.OFF27), ((10, 8, 14), I.OFF7)]:
        A = rnd_sym27(d, 7, off)
        h = make(S, d, off, A, smoother=S.SGS, max_levels=2)
        assert h.nlevels == 2
        Dinv = orc.diag_inverse(d, off, A)
        b = np.random.default_rng(5).normal(size=A.shape[0])
        u = cu(np.zeros(A.shape[0]))
        h.level_apply(0, S.OP_GS_FORWARD, x=u, b=cu(b))
        assert rel_max(host(u), orc.gs_forward(d, off, A, Dinv, b, np.zeros_like(b))) < TOL_KERNEL


@pytest.mark.parametrize("d", [(8, 10, 8), (8, 70, 10), (8, 34, 8)])
def test_block_gs_sweeps(S, orc, d):
    A = I.block7_layered(d, 2).numpy()
    h = make(S, d, I.OFF7, A, block=3, transfer=S.PC8C, smoother=S.SGS, max_levels=2)
    Dinv = orc.diag_inverse(d, I.OFF7, A, B=3)
    n = A.shape[0] * 3
    b, u0 = np.random.default_rng(6).normal(size=(2, n))
    u = cu(u0)
    h.level_apply(0, S.OP_GS_FORWARD, x=u, b=cu(b))
    ref = orc.gs_forward(d, I.OFF7, A, Dinv, b, u0, B=3)
    assert rel_max(host(u), ref) < TOL_KERNEL
    h.level_apply(0, S.OP_GS_BACKWARD, x=u, b=cu(b))
    assert rel_max(host(u), orc.gs_backward(d, I.OFF7, A, Dinv, b, ref, B=3)) < TOL_KERNEL


# (3, 530, 4): planes wider than 16 warps use the plane-per-CTA kernels
@pytest.mark.parametrize("d,off", [((8, 10, 12), I.OFF27), ((12, 8, 10), I.OFF7), ((8, 8, 9), I.OFF19),
                                   ((3, 530, 4), I.OFF27), ((5, 70, 6), I.OFF27)])
def test_ilu0_factor_and_apply(S, orc, d, off):
    A = rnd_sym27(d, 8, off)
    h = make(S, d, off, A, smoother=S.ILU0, max_levels=2)
    LU_ref = orc.ilu0_factor(d, off, A)
    LU = host(h.level_array(0, S.ARR_LU).view(torch.float64)).reshape(A.shape)
    assert rel_max(LU, LU_ref) < TOL_KERNEL
    ec = off.index((0, 0, 0))
    ud = host(h.level_array(0, S.ARR_DINV).view(torch.float64))
    assert rel_max(ud, 1.0 / LU_ref[:, ec]) < TOL_KERNEL
    r = np.random.default_rng(9).normal(size=A.shape[0])
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_ILU_APPLY, b=cu(r), y=y)
    assert rel_max(host(y), orc.ilu0_apply(d, off, LU_ref, 1.0 / LU_ref[:, ec], r)) < 1e-12


def test_ilu0_tridiagonal_exact_solve(S, orc):
    """On a 1 x 1 x n grid the 7-point mask is tridiagonal, ILU(0) drops no
    fill and one application solves the system exactly; the one-level
    hierarchy's direct solve must agree."""
    d = (1, 1, 40)
    A = rnd_sym27(d, 3, I.OFF7)
    h = make(S, d, I.OFF7, A, smoother=S.ILU0, max_levels=1)
    assert h.nlevels == 1
    b = np.random.default_rng(1).normal(size=A.shape[0])
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_ILU_APPLY, b=cu(b), y=y)
    assert rel_max(orc.spmv(d, I.OFF7, A, host(y)), b) < 1e-12
    h.level_apply(0, S.OP_COARSE_SOLVE, b=cu(b), y=y)
    assert rel_max(orc.spmv(d, I.OFF7, A, host(y)), b) < 1e-12


def test_coarsest_inverse_with_row_exchanges(S, orc):
    """The dense coarsest inverse (Gauss-Jordan, partial pivoting) of a
    1440-unknown level whose centre coefficients are shrunk a thousandfold,
    so that most columns need a row exchange: the direct solve agrees with a
    dense LU solve of the assembled matrix."""
    d = (6, 10, 24)
    A = rnd_sym27(d, 7)
    A[:, I.OFF27.index((0, 0, 0))] *= 1e-3
    h = make(S, d, I.OFF27, A, smoother=S.SGS, max_levels=1)
    assert h.nlevels == 1
    b = np.random.default_rng(2).normal(size=A.shape[0])
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_COARSE_SOLVE, b=cu(b), y=y)
    x_ref = np.linalg.solve(orc.assemble_dense(d, I.OFF27, A), b)
    assert rel2(host(y), x_ref) < 1e-9


# ---------------------------------------------------------------------------
# hierarchy: Galerkin coarse operators, transfers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,off,transfer,B,gen", [
    ((16, 12, 20), I.OFF7, 0, 1, "lap"), ((16, 16, 16), I.OFF27, 0, 1, "q1"), ((24, 16, 16), I.OFF27, 0, 1, "rnd"),
    ((16, 16, 8), I.OFF7, 1, 3, "blk"), ((16, 8, 24), I.OFF7, 1, 1, "rnd"),
    ((16, 12, 20), I.OFF7, 2, 1, "lap"), ((16, 16, 16), I.OFF27, 2, 1, "q1"), ((24, 16, 16), I.OFF19, 2, 1, "rnd"),
    ((16, 16, 8), I.OFF7, 2, 3, "blk"), ((16, 8, 24), I.OFF7, 2, 1, "fv"),
    ((16, 24, 12), I.OFF7, 3, 1, "lap"), ((16, 16, 10), I.OFF27, 3, 1, "q1"), ((24, 16, 7), I.OFF19, 3, 1, "rnd"),
    ((16, 16, 6), I.OFF7, 3, 3, "blk")])
def test_galerkin_hierarchy(S, orc, d, off, transfer, B, gen):
    A = {"lap": lambda: I.laplace7(d).numpy(), "q1": lambda: I.q1_aniso27(d, 2).numpy(),
         "rnd": lambda: rnd_sym27(d, 5, off), "blk": lambda: I.block7_layered(d, 4).numpy(),
         "fv": lambda: I.varcoef7(d, 4)[0].numpy()}[gen]()
    h = make(S, d, off, A, block=B, transfer=transfer, smoother=S.SGS)
    ref = orc.MG(d, off, A, B=B, smoother=orc.SGS, transfer=transfer)
    assert h.nlevels == ref.nlevels
    for l in range(h.nlevels):
        dg, og = h.level_info(l)
        dr, orr = ref.level_info(l)
        assert dg == dr
        assert og == [tuple(int(t) for t in o) for o in orr]  # offsets and sparsity bit-exact
        Ag = host(h.level_array(l, S.ARR_A).view(torch.float64))
        Ar = ref.level_array(l, 0)
        assert Ag.shape == Ar.shape
        assert rel_max(Ag, Ar) < TOL_KERNEL, l
        # zero padding: every coefficient whose neighbour is off the grid is exactly 0
        pad = np.ones((np.prod(dg), len(og), B, B), dtype=bool)
        idx = np.indices(dg).reshape(3, -1).T
        for e, o in enumerate(og):
            inside = np.all((idx + np.array(o) >= 0) & (idx + np.array(o) < np.array(dg)), axis=1)
            pad[inside, e] = False
        assert np.all(Ag.reshape(pad.shape)[pad] == 0.0)


@pytest.mark.parametrize("transfer,B", [(0, 1), (1, 1), (2, 1), (3, 1), (0, 3), (1, 3), (2, 3), (3, 3)])
def test_restrict_prolong(S, orc, transfer, B):
    d = (10, 12, 8) if B == 1 else (8, 8, 10)
    if transfer == 3:
        d = (d[0], d[1], 7)  # z is not coarsened: any length
    A = I.laplace7(d).numpy() if B == 1 else I.block7_layered(d, 0).numpy()
    h = make(S, d, I.OFF7, A, block=B, transfer=transfer, max_levels=2)
    nf = np.prod(d) * B
    nc = np.prod(orc.coarse_dims(d, transfer)) * B
    rf, ec, uf = np.random.default_rng(3).normal(size=(3, max(nf, nc)))
    rf, ec, uf = rf[:nf], ec[:nc], uf[:nf]
    y = torch.empty(nc, dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_RESTRICT, x=cu(rf), y=y)
    assert rel_max(host(y), orc.restrict(transfer, d, rf, B=B)) < TOL_KERNEL
    u = cu(uf)
    h.level_apply(0, S.OP_PROLONG_ADD, x=cu(ec), y=u)
    assert rel_max(host(u), orc.prolong_add(transfer, d, ec, uf, B=B)) < TOL_KERNEL


# ---------------------------------------------------------------------------
# V-cycle and solves
# ---------------------------------------------------------------------------

VCASES = [((32, 32, 32), "lap", 0, 0, 1), ((24, 16, 32), "q1", 1, 0, 1), ((16, 24, 16), "q1", 0, 0, 1),
          ((16, 16, 16), "blk", 0, 1, 3), ((20, 16, 24), "q1", 1, 0, 1), ((32, 32, 32), "fv", 0, 2, 1),
          ((24, 16, 32), "fv", 1, 2, 1), ((16, 24, 16), "q1", 1, 2, 1), ((16, 16, 16), "blk", 0, 2, 3),
          ((32, 32, 20), "fv", 0, 3, 1), ((16, 32, 24), "q1", 1, 3, 1), ((16, 16, 12), "blk", 0, 3, 3)]


def problem(kind, d, seed=1):
    if kind == "lap":
        return I.OFF7, I.laplace7(d).numpy()
    if kind == "q1":
        return I.OFF27, I.q1_aniso27(d, seed).numpy()
    if kind == "fv":
        return I.OFF7, I.varcoef7(d, seed)[0].numpy()
    return I.OFF7, I.block7_layered(d, seed).numpy()


@pytest.mark.parametrize("d,kind,smoother,transfer,B", VCASES)
def test_vcycle(S, orc, d, kind, smoother, transfer, B):
    off, A = problem(kind, d)
    h = make(S, d, off, A, block=B, smoother=smoother, transfer=transfer)
    ref = orc.MG(d, off, A, B=B, smoother=smoother, transfer=transfer)
    r = I.rhs(np.prod(d) * B, 11).numpy()
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    assert rel2(host(z), ref.vcycle(r)) < TOL_VCYCLE


@pytest.mark.parametrize("d,kind,smoother,transfer,prec", [
    ((16, 20, 72), "q1", "ilu", "fw", 0), ((16, 20, 72), "lap", "sgs", "fw", 0), ((12, 36, 40), "q1", "ilu", "fw", 1),
    ((16, 20, 72), "q1", "ilu", "fw", 2), ((16, 20, 72), "fv", "ilu", "c64", 0), ((16, 20, 72), "lap", "sgs", "pc", 1),
])
def test_fused_residual_restriction_equals_two_kernels(S, d, kind, smoother, transfer, prec):
    """One pass for f_c = R (f - A u) (option fuse_restrict) gives the same
    V-cycle, bit for bit, as the residual and restriction kernels: the same
    expressions in the same order.  The sizes leave ragged coarse tiles in j
    and k and several x-chunks."""
    off, A = problem(kind, d)
    sm = {"ilu": S.ILU0, "sgs": S.SGS}[smoother]
    tr = {"fw": S.FW27V, "c64": S.C64C, "pc": S.PC8C}[transfer]
    kry = S.PCG if prec == 0 else S.FPCG
    r = cu(I.rhs(np.prod(d), 5).numpy())
    z = []
    for fuse in (0, 1):
        h = make(S, d, off, A, smoother=sm, transfer=tr, precision=prec, krylov=kry, fuse_restrict=fuse)
        zz = torch.empty_like(r)
        h.vcycle(r, zz)
        h.close()
        z.append(zz)
    assert torch.equal(z[0], z[1])


def test_vcycle_graph_replay_is_bitwise_identical(S):
    d = (32, 32, 32)
    off, A = problem("q1", d)
    r = cu(I.rhs(np.prod(d), 3).numpy())
    z1, z2, z3 = (torch.empty_like(r) for _ in range(3))
    make(S, d, off, A, smoother=S.ILU0).vcycle(r, z1)
    hg = make(S, d, off, A, smoother=S.ILU0, use_graph=1)
    hg.vcycle(r, z2)
    hg.vcycle(r, z3)
    assert torch.equal(z1, z2) and torch.equal(z2, z3)


@pytest.mark.parametrize("d,kind,smoother,krylov", [((32, 32, 32), "lap", 0, 0), ((32, 32, 32), "q1", 1, 0),
                                                    ((24, 32, 16), "fv", 0, 0), ((32, 32, 32), "q1", 0, 1)])
def test_pcg_solve_matches_oracle(S, orc, d, kind, smoother, krylov):
    off, A = problem(kind, d)
    b = I.rhs(np.prod(d), 0).numpy()
    h = make(S, d, off, A, smoother=smoother, krylov=krylov)
    x = torch.zeros_like(cu(b))
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=200)
    xr, rcr, itr, rrr, _ = orc.MG(d, off, A, smoother=smoother).pcg(b, tol=1e-9, flexible=bool(krylov))
    assert rc == 0 and rcr == 0
    assert abs(it - itr) <= 1
    assert rr < 1e-9
    # the true residual, recomputed by the oracle from the GPU solution
    res = np.linalg.norm(orc.residual(d, off, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9 and abs(res - rr) < 1e-12


@pytest.mark.parametrize("kind,smoother,krylov", [("fv", 0, 1), ("fv", 1, 2), ("lap", 1, 1), ("q1", 1, 2)])
def test_cell64_solves_match_oracle(S, orc, kind, smoother, krylov):
    """Cell-centred 3d64c interpolation with 3d8c restriction (nonsymmetric
    V-cycle) under flexible PCG and FGMRES(30): same iteration count as the
    oracle within one, tolerance reached, true residual recomputed by the
    oracle."""
    d = (32, 24, 32)
    off, A = problem(kind, d)
    b = I.rhs(np.prod(d), 2).numpy()
    h = make(S, d, off, A, smoother=smoother, transfer=S.C64C, krylov=krylov, restart=30)
    x = torch.zeros_like(cu(b))
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=300)
    ref = orc.MG(d, off, A, smoother=smoother, transfer=orc.C64C)
    if krylov == 2:
        _, rcr, itr, _, _ = ref.fgmres(b, tol=1e-9, restart=30, maxit=300)
    else:
        _, rcr, itr, _, _ = ref.pcg(b, tol=1e-9, flexible=True, maxit=300)
    assert rc == 0 and rcr == 0 and abs(it - itr) <= 1 and rr < 1e-9
    res = np.linalg.norm(orc.residual(d, off, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9


def test_fgmres_block_solve_matches_oracle(S, orc):
    d = (32, 32, 16)
    A = I.block7_layered(d, 5).numpy()
    b = I.rhs(np.prod(d) * 3, 1).numpy()
    h = make(S, d, I.OFF7, A, block=3, transfer=S.PC8C, krylov=S.FGMRES, restart=30)
    x = torch.zeros_like(cu(b))
    it, rr, rc = h.solve(cu(b), x, tol=1e-8, maxit=300)
    ref = orc.MG(d, I.OFF7, A, B=3, transfer=orc.PC8C)
    xr, rcr, itr, rrr, _ = ref.fgmres(b, tol=1e-8, restart=30, maxit=300)
    assert rc == 0 and rcr == 0 and abs(it - itr) <= 1 and rr < 1e-8
    res = np.linalg.norm(orc.residual(d, I.OFF7, A, b, host(x), B=3)) / np.linalg.norm(b)
    assert res < 1e-8


@pytest.mark.parametrize("d", [(16, 16, 8), (32, 24, 16)])
def test_fp32_block_hierarchy_vcycle_and_fgmres(S, orc, d):
    """The 3-unknown system with an FP32 hierarchy (block GS in float) against
    the oracle's FP32 block cycle (same precision, own summation order:
    TOL_LOWP), its FP64 cycle within FP32 accuracy, and an FGMRES solve that
    reaches the tolerance with the true residual recomputed by the oracle in
    the FP32 oracle's iteration count within one."""
    A = I.block7_layered(d, 7).numpy()
    r = I.rhs(np.prod(d) * 3, 12).numpy()
    h = make(S, d, I.OFF7, A, block=3, transfer=S.PC8C, precision=S.FP32, krylov=S.FGMRES, restart=30)
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    ref32 = orc.MG(d, I.OFF7, A, B=3, transfer=orc.PC8C, precision=orc.FP32)
    assert rel2(host(z), ref32.vcycle(r)) < TOL_LOWP
    ref64 = orc.MG(d, I.OFF7, A, B=3, transfer=orc.PC8C)
    assert rel2(host(z), ref64.vcycle(r)) < 1e-4
    x = torch.zeros_like(cu(r))
    it, rr, rc = h.solve(cu(r), x, tol=1e-8, maxit=300)
    assert rc == 0 and rr < 1e-8
    res = np.linalg.norm(orc.residual(d, I.OFF7, A, r, host(x), B=3)) / np.linalg.norm(r)
    assert res < 1e-8
    _, rcr, itr, _, _ = ref32.fgmres(r, tol=1e-8, restart=30, maxit=300)
    assert rcr == 0 and abs(it - itr) <= 1


def test_solves_are_deterministic(S):
    d = (32, 32, 32)
    off, A = problem("q1", d)
    b = cu(I.rhs(np.prod(d), 4).numpy())
    h = make(S, d, off, A, smoother=S.ILU0)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    assert h.solve(b, x1)[0] == h.solve(b, x2)[0]
    assert torch.equal(x1, x2)


# ---------------------------------------------------------------------------
# reduced precision hierarchies
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("smoother", [0, 1])
def test_lowered_arrays_bit_exact(S, orc, smoother):
    d = (16, 16, 16)
    off, A = problem("q1", d, 3)
    h = make(S, d, off, A, smoother=smoother, precision=S.BF16)
    ref = orc.MG(d, off, A, smoother=smoother, precision=orc.BF16)
    v = host(h.level_array(0, S.ARR_AV).view(torch.bfloat16).float())
    assert np.array_equal(v, ref.level_array(0, 3))
    assert np.array_equal(host(h.level_array(0, S.ARR_AS).view(torch.float32)), ref.level_array(0, 4))
    if smoother == 1:
        # factors from the GPU's FP64 ILU(0) may differ in the last bit; allow
        # one bf16 unit where they do
        lv = host(h.level_array(0, S.ARR_LUV).view(torch.bfloat16).float()).reshape(-1, 27)
        lr = ref.level_array(0, 5).reshape(-1, 27)
        ur = ref.level_array(0, 7).reshape(-1, 27)
        want = np.where(np.arange(27) < 13, lr, ur)
        assert np.max(np.abs(lv - want)) <= 2.0 ** -7
        assert np.mean(lv == want) > 0.999


@pytest.mark.parametrize("prec,smoother,d", [(1, 0, (32, 32, 32)), (1, 1, (32, 32, 32)), (2, 0, (32, 32, 32)),
                                             (2, 1, (32, 32, 32)), (1, 1, (16, 96, 24)), (2, 0, (24, 160, 16)),
                                             (1, 0, (10, 288, 8))])
def test_low_precision_vcycle(S, orc, prec, smoother, d):
    off, A = problem("q1", d, 2)
    r = I.rhs(np.prod(d), 5).numpy()
    h = make(S, d, off, A, smoother=smoother, precision=prec)
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    zr = orc.MG(d, off, A, smoother=smoother, precision=prec).vcycle(r)
    assert rel2(host(z), zr) < TOL_LOWP


@pytest.mark.parametrize("prec", [1, 2])
def test_low_precision_fpcg_reaches_fp64_accuracy(S, orc, prec):
    d = (32, 32, 32)
    off, A = problem("q1", d, 1)
    b = I.rhs(np.prod(d), 6).numpy()
    h = make(S, d, off, A, smoother=S.ILU0, precision=prec, krylov=S.FPCG)
    x = torch.zeros_like(cu(b))
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=300)
    assert rc == 0 and rr < 1e-9
    res = np.linalg.norm(orc.residual(d, off, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9
    # error against an FP64 oracle solution converged far below the tolerance:
    # bounded by cond(A) * 1e-9; the problem's condition number is below 1e5
    x64 = orc.MG(d, off, A, smoother=orc.ILU0).pcg(b, tol=1e-13)[0]
    assert rel2(host(x), x64) < 1e-4


# ---------------------------------------------------------------------------
# edge cases and failure reporting
# ---------------------------------------------------------------------------

def test_zero_rhs_and_maxit_zero(S):
    d = (16, 16, 16)
    off, A = problem("lap", d)
    h = make(S, d, off, A)
    x = cu(np.ones(4096))
    it, rr, rc = h.solve(cu(np.zeros(4096)), x)
    assert rc == 0 and it == 0 and torch.count_nonzero(x) == 0
    it, rr, rc = h.solve(cu(np.ones(4096)), torch.zeros(4096, dtype=torch.float64, device="cuda"), maxit=0,
                         check=False)
    assert rc == S.ENOTCONV and it == 0


def test_single_level_is_direct_solve(S, orc):
    d = (5, 6, 7)
    off, A = I.OFF27, rnd_sym27((5, 6, 7), 2)
    h = make(S, d, off, A)
    assert h.nlevels == 1
    b = I.rhs(210, 1).numpy()
    x = torch.zeros_like(cu(b))
    it, rr, rc = h.solve(cu(b), x, tol=1e-12)
    assert rc == 0 and it == 1 and rr < 1e-12


def test_nonzero_padding_rejected(S):
    d = (8, 8, 8)
    A = I.laplace7(d).numpy()
    A[0, 0] = -1.0  # neighbour (-1,0,0) of point (0,0,0) is off the grid
    with pytest.raises(S.SmgError) as ei:
        make(S, d, I.OFF7, A)
    assert ei.value.status == S.EINVAL


def test_unsorted_offsets_are_canonicalised(S, orc):
    d = (16, 16, 16)
    A = I.q1_aniso27(d, 1).numpy()
    perm = np.random.default_rng(0).permutation(27)
    offs = [I.OFF27[e] for e in perm]
    h = make(S, d, offs, np.ascontiguousarray(A[:, perm]))
    r = I.rhs(4096, 2).numpy()
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    assert rel2(host(z), orc.MG(d, I.OFF27, A).vcycle(r)) < TOL_VCYCLE


def test_ilu_breakdown_reported(S):
    d = (16, 16, 16)
    A = I.laplace7(d).numpy()
    A[:, 3] = -6.0
    with pytest.raises(S.SmgError) as ei:
        make(S, d, I.OFF7, A, smoother=S.ILU0)
    assert ei.value.status == S.EBREAKDOWN


def test_bounded_wait_times_out_and_context_survives(S, orc):
    """A device wait on a flag nothing sets returns SMG_ETIMEOUT after its
    budget; the same context then still runs a correct V-cycle."""
    d = (16, 16, 16)
    off, A = problem("q1", d)
    h = make(S, d, off, A, smoother=S.ILU0)
    assert h.selftest_wait(20) == S.ETIMEOUT
    r = I.rhs(4096, 1).numpy()
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    assert rel2(host(z), orc.MG(d, off, A, smoother=orc.ILU0).vcycle(r)) < TOL_VCYCLE


def test_single_ilu_sweeps(S, orc):
    d = (16, 12, 8)
    A = rnd_sym27(d, 2)
    h = make(S, d, I.OFF27, A, smoother=S.ILU0, max_levels=1)
    LU = orc.ilu0_factor(d, I.OFF27, A)
    L, U = np.tril(orc.assemble_dense(d, I.OFF27, LU), -1) + np.eye(A.shape[0]), \
        np.triu(orc.assemble_dense(d, I.OFF27, LU))
    b = np.random.default_rng(1).normal(size=A.shape[0])
    y = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_ILU_LOWER, b=cu(b), y=y)
    assert rel_max(L @ host(y), b) < TOL_KERNEL
    yy = cu(b)
    h.level_apply(0, S.OP_ILU_UPPER, b=yy, y=yy)  # in place
    assert rel_max(U @ host(yy), b) < 1e-12


def test_launch_counter_counts_kernels(S):
    d = (16, 16, 16)
    off, A = problem("lap", d)
    h = make(S, d, off, A)
    r = cu(I.rhs(4096, 0).numpy())
    z = torch.empty_like(r)
    c0 = S.launch_count()
    h.vcycle(r, z)
    per = S.launch_count() - c0
    # per level above the coarsest: pre-smoothing (right-hand side into the
    # sweeps' skewed layout, 2 sweeps, result back), post-smoothing (right-hand
    # side and iterate in, 2 sweeps, result back), residual, restriction,
    # prolongation; plus the coarsest solve
    nl = h.nlevels
    assert per == 12 * (nl - 1) + 1
    # residual and restriction in one kernel
    hf = make(S, d, off, A, fuse_restrict=1)
    c0 = S.launch_count()
    hf.vcycle(r, z)
    assert S.launch_count() - c0 == 11 * (nl - 1) + 1
    hg = make(S, d, off, A, use_graph=1)
    c0 = S.launch_count()
    hg.vcycle(r, z)
    hg.vcycle(r, z)
    assert S.launch_count() - c0 == 2 * per


@pytest.mark.parametrize("smoother", ["ilu", "sgs"])
def test_zero_wait_budget_aborts_and_context_survives(S, orc, smoother):
    """A zero wait budget makes the wavefront sweeps give up at their first
    unsatisfied wait (error word set, every CTA drains); with the budget
    restored the same context runs a V-cycle equal to the oracle's."""
    d = (24, 40, 24)
    off, A = problem("q1", d)
    n = int(np.prod(d))
    sm = S.ILU0 if smoother == "ilu" else S.SGS
    h = make(S, d, off, A, smoother=sm)
    r = cu(I.rhs(n, 2).numpy())
    z = torch.empty_like(r)
    h.set_wait_budget_ns(0)
    status = S.OK
    try:
        h.vcycle(r, z)
    except S.SmgError as e:
        status = e.status
    assert status in (S.OK, S.ETIMEOUT)
    h.set_wait_budget_ns(10 ** 9)
    ref = orc.MG(d, off, A, smoother=orc.ILU0 if smoother == "ilu" else orc.SGS).vcycle(host(r))
    for _ in range(2):
        h.vcycle(r, z)
        assert rel2(host(z), ref) < TOL_VCYCLE
