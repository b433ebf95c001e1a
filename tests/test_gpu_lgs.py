"""Parity of the GPU line Gauss-Seidel smoother (LGS along z) with the
oracle's Thomas-algorithm line sweeps, through the C ABI.

The GPU solves each column by a partitioned elimination (128 chunks, parallel
cyclic reduction on the chunk interface) instead of the serial Thomas
recurrence: the same solution in exact arithmetic, with a different rounding
order.  The column systems here are diagonally dominant (condition numbers
up to a few hundred for the z-anisotropic problems), so single sweeps are
held to 1e-12 relative to the output's largest magnitude and V-cycles to
1e-12 in the 2-norm, as the point smoothers."""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_SWEEP = 1e-12
TOL_VCYCLE = 1e-12


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
    return np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300)


def rel2(got, ref):
    return np.linalg.norm(np.asarray(got) - ref) / max(np.linalg.norm(ref), 1e-300)


def zaniso(d, seed):
    return I.q1_aniso27(d, seed, aniso=(1e-3, 1e-3, 1.0)).numpy()


def problem(kind, d, seed=1):
    if kind == "lap":
        return I.OFF7, I.laplace7(d).numpy()
    if kind == "fv":
        return I.OFF7, I.varcoef7(d, seed)[0].numpy()
    if kind == "q1":
        return I.OFF27, I.q1_aniso27(d, seed).numpy()
    if kind == "q1z":
        return I.OFF27, zaniso(d, seed)
    A = I.q1_aniso27(d, seed, aniso=(1e-2, 1e-2, 1.0)).numpy()  # "q1z19": 19-point cut of the same matrix
    keep = [e for e, o in enumerate(I.OFF27) if sum(map(abs, o)) <= 2]
    A = A[:, keep].copy()
    A[:, I.OFF19.index((0, 0, 0))] += 1.0  # keep it diagonally dominant
    return I.OFF19, A


# grids: ragged nz (several chunk sizes, padded chunks), nz < 64 (two rows
# per chunk), a single plane, the largest supported column
@pytest.mark.parametrize("d,kind", [((6, 7, 45), "q1z"), ((5, 9, 100), "fv"), ((7, 5, 33), "q1z19"),
                                    ((4, 6, 1), "lap"), ((1, 3, 70), "q1"), ((2, 3, 1024), "q1z"),
                                    ((3, 40, 64), "q1")])
def test_line_sweeps_match_oracle(S, orc, d, kind):
    off, A = problem(kind, d)
    n = int(np.prod(d))
    h = S.SMG(d, off, cu(A), smoother=S.LGS, max_levels=1)
    rng = np.random.default_rng(3)
    b, u0 = rng.normal(size=(2, n))
    for op, ref in [(S.OP_LGS_FORWARD, orc.lgs_forward(d, off, A, b, u0)),
                    (S.OP_LGS_BACKWARD, orc.lgs_backward(d, off, A, b, u0)),
                    (S.OP_LGS_ZERO, orc.lgs_forward(d, off, A, b, np.zeros(n)))]:
        x = cu(u0)  # the zero-guess sweep must ignore what x holds
        h.level_apply(0, op, x=x, b=cu(b))
        assert rel_max(host(x), ref) < TOL_SWEEP, op


@pytest.mark.parametrize("d,kind,transfer", [((32, 32, 32), "q1z", 0), ((16, 24, 40), "fv", 0),
                                             ((24, 16, 32), "q1", 2), ((16, 16, 16), "lap", 1),
                                             ((32, 32, 24), "q1z", 3), ((16, 32, 45), "q1z19", 3)])
def test_lgs_vcycle_matches_oracle(S, orc, d, kind, transfer):
    off, A = problem(kind, d)
    h = S.SMG(d, off, cu(A), smoother=S.LGS, transfer=transfer)
    ref = orc.MG(d, off, A, smoother=orc.LGS, transfer=transfer)
    assert h.nlevels == ref.nlevels
    r = I.rhs(int(np.prod(d)), 5).numpy()
    z = torch.empty_like(cu(r))
    h.vcycle(cu(r), z)
    assert rel2(host(z), ref.vcycle(r)) < TOL_VCYCLE


def test_lgs_pcg_solve_matches_oracle(S, orc):
    """z-aligned anisotropy: the line smoother's case.  Same iteration count as
    the oracle within one, and far fewer than point GS on the same matrix."""
    d = (32, 32, 48)
    off, A = problem("q1z", d, seed=2)
    b = I.rhs(int(np.prod(d)), 7).numpy()
    x = torch.zeros_like(cu(b))
    h = S.SMG(d, off, cu(A), smoother=S.LGS)
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=300)
    _, rcr, itr, _, _ = orc.MG(d, off, A, smoother=orc.LGS).pcg(b, tol=1e-9, maxit=300)
    assert rc == 0 and rcr == 0 and abs(it - itr) <= 1 and rr < 1e-9
    res = np.linalg.norm(orc.residual(d, off, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9
    x.zero_()
    its, _, rcs = S.SMG(d, off, cu(A), smoother=S.SGS).solve(cu(b), x, tol=1e-9, maxit=500)
    assert rcs == 0 and its > 4 * it


@pytest.mark.parametrize("krylov", [1, 2])
def test_semicoarse_lgs_solve_matches_oracle(S, orc, krylov):
    """x-y semi-coarsening with z-line smoothing (Table 8, weather setting)
    under flexible PCG and FGMRES(30): iterations within one of the oracle's,
    tolerance reached, true residual recomputed by the oracle."""
    d = (32, 48, 40)
    off, A = problem("q1z", d, seed=4)
    b = I.rhs(int(np.prod(d)), 8).numpy()
    x = torch.zeros_like(cu(b))
    h = S.SMG(d, off, cu(A), smoother=S.LGS, transfer=S.C16XY, krylov=krylov, restart=30)
    assert h.nlevels == 4 and h.level_info(3)[0] == (4, 6, 40)
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=300)
    ref = orc.MG(d, off, A, smoother=orc.LGS, transfer=orc.C16XY)
    if krylov == 2:
        _, rcr, itr, _, _ = ref.fgmres(b, tol=1e-9, restart=30, maxit=300)
    else:
        _, rcr, itr, _, _ = ref.pcg(b, tol=1e-9, flexible=True, maxit=300)
    assert rc == 0 and rcr == 0 and abs(it - itr) <= 1 and rr < 1e-9
    res = np.linalg.norm(orc.residual(d, off, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9


def test_lgs_argument_checks_and_breakdown(S):
    d = (8, 8, 16)
    A = I.laplace7(d).numpy()
    for kw in [dict(precision=S.FP32), dict(relax_w=1.2)]:
        with pytest.raises(S.SmgError) as e:
            S.SMG(d, I.OFF7, cu(A), smoother=S.LGS, **kw)
        assert e.value.status == S.EINVAL
    dz = (2, 2, 1026)  # columns longer than the supported 1024 points
    with pytest.raises(S.SmgError) as e:
        S.SMG(dz, I.OFF7, cu(I.laplace7(dz).numpy()), smoother=S.LGS)
    assert e.value.status == S.EINVAL
    B = A.copy()
    B[(2 * 8 + 3) * 16 + 0, 3] = 0.0  # first Thomas pivot of column (2, 3)
    with pytest.raises(S.SmgError) as e:
        S.SMG(d, I.OFF7, cu(B), smoother=S.LGS)
    assert e.value.status == S.EBREAKDOWN
    # a sweep of another smoother's hierarchy is refused
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS)
    with pytest.raises(S.SmgError):
        h.level_apply(0, S.OP_LGS_FORWARD, x=torch.zeros(1024, dtype=torch.float64, device="cuda"),
                      b=torch.zeros(1024, dtype=torch.float64, device="cuda"))


def test_lgs_vcycle_graph_replay_and_determinism(S):
    """The line sweeps replay inside a captured V-cycle graph and give the
    same bits as the eager V-cycle, run after run."""
    d = (32, 32, 40)
    off, A = problem("q1z", d)
    r = cu(I.rhs(int(np.prod(d)), 3).numpy())
    z1, z2, z3 = (torch.empty_like(r) for _ in range(3))
    S.SMG(d, off, cu(A), smoother=S.LGS).vcycle(r, z1)
    hg = S.SMG(d, off, cu(A), smoother=S.LGS, use_graph=1)
    hg.vcycle(r, z2)
    hg.vcycle(r, z3)
    assert torch.equal(z1, z2) and torch.equal(z2, z3)


def test_lgs_abort_path_drains_and_the_context_survives(S, orc):
    """With a zero wait budget, every dependency wait of the line sweep that
    is not satisfied at once gives up: the sweep takes its abort path, which
    must drain the column copies it issued.  With the budget restored the same
    context then sweeps exactly as the oracle, twice in a row."""
    d = (8, 12, 64)  # even nz: the column data are staged by bulk copies; n <= 8192 (one level)
    off, A = problem("q1z", d)
    n = int(np.prod(d))
    h = S.SMG(d, off, cu(A), smoother=S.LGS, max_levels=1)
    b = cu(I.rhs(n, 5).numpy())
    h.set_wait_budget_ns(0)
    status = S.OK
    try:
        h.level_apply(0, S.OP_LGS_FORWARD, x=torch.zeros_like(b), b=b)
    except S.SmgError as e:
        status = e.status
    assert status in (S.OK, S.ETIMEOUT)
    h.set_wait_budget_ns(10 ** 9)
    ref = orc.lgs_forward(d, off, A, host(b), np.zeros(n))
    for _ in range(2):
        x = torch.zeros_like(b)
        h.level_apply(0, S.OP_LGS_FORWARD, x=x, b=b)
        assert rel_max(host(x), ref) < TOL_SWEEP
