"""Parity at the full size of the headline workload (27-point anisotropic Q1
diffusion, 256^3, ILU(0) V-cycle, PCG), in the launch configuration the
benchmark times (default options).  The oracle cannot run a whole 256^3
hierarchy in test time, so it checks what it can compute directly at this
size: the SpMV everywhere, the ILU(0) factorisation of the finest level
and one full ILU(0) application (exact lexicographic solves over all 16.8 M
points), the Galerkin coarse operator at sampled coarse points (brute force
per point), and the solve through the property that holds at any size --
the true residual recomputed by the oracle is below the tolerance.  The
extension workloads are checked at 256^3 too: one full line Gauss-Seidel
sweep (c7), the x-y semi-coarsened Galerkin operator at sampled points (c8)
and the cell-centred transfers (c6).  Tolerances as in the other parity
tests (FMA and summation order only)."""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D = (256, 256, 256)


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


@pytest.fixture(scope="module")
def problem(S):
    A = I.q1_aniso27(D, 0, device="cuda").contiguous()
    h = S.SMG(D, I.OFF27, A, smoother=S.ILU0)
    return A, A.cpu().numpy(), h


def rel_max(got, ref):
    return np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300)


def test_full_size_spmv_and_ilu(S, orc, problem):
    A_d, A, h = problem
    n = A.shape[0]
    rng = np.random.default_rng(0)
    x = rng.normal(size=n)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_SPMV, x=torch.from_numpy(x).cuda(), y=y)
    assert rel_max(y.cpu().numpy(), orc.spmv(D, I.OFF27, A, x)) < 1e-13
    LU = orc.ilu0_factor(D, I.OFF27, A)
    LUg = h.level_array(0, S.ARR_LU).view(torch.float64).cpu().numpy().reshape(A.shape)
    assert rel_max(LUg, LU) < 1e-13
    ud = 1.0 / LU[:, I.OFF27.index((0, 0, 0))]
    r = rng.normal(size=n)
    h.level_apply(0, S.OP_ILU_APPLY, b=torch.from_numpy(r).cuda(), y=y)
    assert rel_max(y.cpu().numpy(), orc.ilu0_apply(D, I.OFF27, LU, ud, r)) < 1e-12


def test_full_size_coarse_operator_at_sampled_points(S, orc, problem):
    _, A, h = problem
    dc, offc = h.level_info(1)
    Ac = h.level_array(1, S.ARR_A).view(torch.float64).cpu().numpy().reshape(-1, len(offc))
    nc = Ac.shape[0]
    pts = np.unique(np.concatenate([np.random.default_rng(1).integers(0, nc, size=400),
                                    [0, nc - 1, dc[1] * dc[2] - 1, nc // 2]]))
    ref = orc.rap27_at(0, D, I.OFF27, A, pts)[:, :, 0, 0]
    lex = [(o[0] + 1) * 9 + (o[1] + 1) * 3 + (o[2] + 1) for o in offc]
    assert rel_max(Ac[pts], ref[:, lex]) < 1e-13
    # every offset the oracle reaches is one of the GPU's, the others are zero
    missing = [t for t in range(27) if t not in lex]
    assert np.all(ref[:, missing] == 0.0)


def test_full_size_solve_reaches_the_tolerance(S, orc, problem):
    A_d, A, h = problem
    n = A.shape[0]
    b = I.rhs(n, 1000, device="cuda")
    x = torch.zeros_like(b)
    it, rr, rc = h.solve(b, x, tol=1e-9, maxit=500)
    assert rc == 0 and rr < 1e-9
    bh = b.cpu().numpy()
    res = np.linalg.norm(orc.residual(D, I.OFF27, A, bh, x.cpu().numpy())) / np.linalg.norm(bh)
    assert res < 1e-9


# ---------------------------------------------------------------------------
# the extension workloads at their full size (256^3)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def zproblem(S):
    A = I.q1_aniso27(D, 0, aniso=(1e-3, 1e-3, 1.0), device="cuda").contiguous()
    return A, A.cpu().numpy()


def test_full_size_line_sweep(S, orc, zproblem):
    """One forward line Gauss-Seidel sweep over all 65536 z-columns of the
    256^3 z-anisotropic matrix (the c7 workload's level 0), element by
    element against the oracle's Thomas sweep."""
    A_d, A = zproblem
    h = S.SMG(D, I.OFF27, A_d, smoother=S.LGS)
    n = A.shape[0]
    rng = np.random.default_rng(5)
    b, u0 = rng.normal(size=n), rng.normal(size=n)
    x = torch.from_numpy(u0).cuda()
    h.level_apply(0, S.OP_LGS_FORWARD, x=x, b=torch.from_numpy(b).cuda())
    assert rel_max(x.cpu().numpy(), orc.lgs_forward(D, I.OFF27, A, b, u0)) < 1e-12
    h.close()


def test_full_size_semicoarse_operator_at_sampled_points(S, orc, zproblem):
    """The x-y semi-coarsened Galerkin operator of the c8 workload (level 1,
    128 x 128 x 256) at sampled coarse points, brute force per point."""
    A_d, A = zproblem
    h = S.SMG(D, I.OFF27, A_d, smoother=S.LGS, transfer=S.C16XY)
    dc, offc = h.level_info(1)
    assert dc == (128, 128, 256)
    Ac = h.level_array(1, S.ARR_A).view(torch.float64).cpu().numpy().reshape(-1, len(offc))
    nc = Ac.shape[0]
    pts = np.unique(np.concatenate([np.random.default_rng(2).integers(0, nc, size=300), [0, nc - 1, 255, nc // 2]]))
    ref = orc.rap27_at(S.C16XY, D, I.OFF27, A, pts)[:, :, 0, 0]
    lex = [(o[0] + 1) * 9 + (o[1] + 1) * 3 + (o[2] + 1) for o in offc]
    assert rel_max(Ac[pts], ref[:, lex]) < 1e-13
    h.close()


def test_full_size_cell_transfers(S, orc):
    """3d8c restriction and 3d64c interpolation between 256^3 and 128^3 (the
    c6 workload's level 0), element by element."""
    A = I.varcoef7(D, 0, device="cuda")[0].contiguous()
    h = S.SMG(D, I.OFF7, A, smoother=S.ILU0, transfer=S.C64C)
    n, nc = 256 ** 3, 128 ** 3
    rng = np.random.default_rng(6)
    rf, ec, uf = rng.normal(size=n), rng.normal(size=nc), rng.normal(size=n)
    y = torch.empty(nc, dtype=torch.float64, device="cuda")
    h.level_apply(0, S.OP_RESTRICT, x=torch.from_numpy(rf).cuda(), y=y)
    assert rel_max(y.cpu().numpy(), orc.restrict(S.C64C, D, rf)) < 1e-13
    u = torch.from_numpy(uf).cuda()
    h.level_apply(0, S.OP_PROLONG_ADD, x=torch.from_numpy(ec).cuda(), y=u)
    assert rel_max(u.cpu().numpy(), orc.prolong_add(S.C64C, D, ec, uf)) < 1e-13
    h.close()
