"""The two-warp wavefront sweeps (option sweep_warps = 2) against the one-warp
kernel and the oracle.

The two-warp kernel hands the early partial sum of every point, formed in the
same order as the one-warp kernel's, from a helper warp to the warp that
finishes the point, so a V-cycle must come out bit for bit the same with
either kernel.  The cases cover 19- and 27-point masks, ILU(0) and symmetric
Gauss-Seidel (with and without a weight), the three hierarchy precisions,
one to twelve 32-column strips per plane with a ragged last strip, one and
two planes per CTA, and a zero wait budget.
"""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def rel2(got, ref):
    return np.linalg.norm(np.asarray(got) - ref) / max(np.linalg.norm(ref), 1e-300)


def rnd_sym(d, seed, off):
    """Random symmetric, diagonally dominant stencil matrix (exact zero padding)."""
    rng = np.random.default_rng(seed)
    n = d[0] * d[1] * d[2]
    A = np.zeros((n, len(off)))
    idx = np.arange(n).reshape(d)
    for e, o in enumerate(off):
        if o >= (0, 0, 0):
            continue
        e2 = off.index(tuple(-t for t in o))
        sl_p = tuple(slice(max(0, -o[t]), d[t] - max(0, o[t])) for t in range(3))
        sl_q = tuple(slice(max(0, o[t]), d[t] + min(0, o[t])) for t in range(3))
        p, q = idx[sl_p].ravel(), idx[sl_q].ravel()
        v = -rng.uniform(0.1, 1.0, size=len(p))
        A[p, e] = v
        A[q, e2] = v
    A[:, off.index((0, 0, 0))] = np.abs(A).sum(axis=1) + rng.uniform(0.01, 0.5, size=n)
    return A


def problem(mask, d):
    if mask == 27:
        return I.OFF27, I.q1_aniso27(d, 2).numpy()
    return I.OFF19, rnd_sym(d, 3, I.OFF19)


# (dims, mask, smoother, precision, relax_w); every hierarchy ends on a
# coarsest level of at most 1024 unknowns
CASES = [
    ((16, 20, 72), 27, "ilu", 0, 1.0), ((16, 20, 72), 27, "ilu", 1, 1.0), ((16, 20, 72), 27, "ilu", 2, 1.0),
    ((16, 80, 32), 27, "ilu", 0, 1.0), ((16, 80, 32), 27, "ilu", 1, 1.0), ((16, 80, 32), 27, "ilu", 2, 1.0),
    ((16, 256, 16), 27, "ilu", 0, 1.0), ((16, 160, 16), 27, "ilu", 1, 1.0), ((16, 160, 16), 27, "sgs", 2, 1.0),
    ((16, 80, 32), 27, "sgs", 0, 1.0), ((16, 80, 32), 27, "sgs", 1, 1.0), ((16, 80, 32), 27, "sgs", 1, 0.8),
    ((16, 44, 24), 19, "ilu", 0, 1.0), ((16, 44, 24), 19, "ilu", 1, 1.0), ((16, 44, 24), 19, "sgs", 2, 1.0),
    ((16, 44, 24), 19, "sgs", 0, 0.8),
    # 9 to 12 strips: FP64 ILU(0) on the 832-thread instantiation, the rest on one warp
    ((16, 384, 16), 27, "ilu", 0, 1.0), ((16, 384, 16), 27, "ilu", 1, 1.0), ((16, 352, 16), 27, "ilu", 2, 1.0),
    ((16, 384, 16), 27, "sgs", 2, 1.0), ((16, 352, 16), 27, "sgs", 1, 0.8), ((16, 320, 16), 19, "ilu", 0, 1.0),
]


@pytest.mark.parametrize("d,mask,smoother,prec,w", CASES)
def test_two_warp_vcycle_equals_one_warp_and_oracle(S, orc, d, mask, smoother, prec, w):
    off, A = problem(mask, d)
    sm = S.ILU0 if smoother == "ilu" else S.SGS
    r = cu(I.rhs(int(np.prod(d)), 7).numpy())
    z = {}
    for warps in (1, 2, 0):
        h = S.SMG(d, off, cu(A), smoother=sm, precision=prec, relax_w=w, sweep_warps=warps)
        ops = (S.OP_ILU_LOWER, S.OP_ILU_UPPER) if smoother == "ilu" else (S.OP_GS_ZERO, S.OP_GS_FORWARD)
        got = [h.level_sweep_warps(0, op) for op in ops]
        if warps == 1:
            assert got == [1, 1]
        else:  # 2, and the library's choice (0), which takes two warps where they apply
            # FP64 Gauss-Seidel with old values stays on one warp (it would
            # spill); planes of more than 8 strips take two warps only for the
            # FP64 ILU(0) solves
            wide = (d[1] + 31) // 32 > 8
            if wide:
                assert got == ([2, 2] if smoother == "ilu" and prec == 0 else [1, 1])
            else:
                assert got == ([2, 2] if smoother == "ilu" else [2, 1 if prec == 0 else 2])
        zz = torch.empty_like(r)
        h.vcycle(r, zz)
        z[warps] = zz
        h.close()
    assert torch.equal(z[1], z[2]) and torch.equal(z[0], z[2])
    ref = orc.MG(d, off, A, smoother=orc.ILU0 if smoother == "ilu" else orc.SGS, precision=prec,
                 w=w).vcycle(host(r))
    assert rel2(host(z[2]), ref) < (TOL_VCYCLE if prec == 0 else TOL_LOWP)


def test_two_warp_single_sweeps_in_place(S, orc):
    """The level operations run the same kernel: an in-place ILU(0) upper
    solve after the lower one reproduces the dense triangular solves."""
    d = (8, 40, 8)
    off, A = problem(27, d)
    h = S.SMG(d, off, cu(A), smoother=S.ILU0, max_levels=1, sweep_warps=2)
    assert h.level_sweep_warps(0, S.OP_ILU_LOWER) == 2
    LU = orc.ilu0_factor(d, off, A)
    L = np.tril(orc.assemble_dense(d, off, LU), -1) + np.eye(A.shape[0])
    U = np.triu(orc.assemble_dense(d, off, LU))
    b = np.random.default_rng(4).normal(size=A.shape[0])
    y = cu(b)
    h.level_apply(0, S.OP_ILU_LOWER, b=y, y=y)
    h.level_apply(0, S.OP_ILU_UPPER, b=y, y=y)
    x = np.linalg.solve(U, np.linalg.solve(L, b))
    assert rel2(host(y), x) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_two_warp_zero_wait_budget_aborts_and_context_survives(S, orc, prec):
    """With a zero wait budget the helper and main warps give up at their
    first unsatisfied wait (error word set, every CTA drains); with the
    budget restored the same context runs the oracle's V-cycle."""
    d = (24, 40, 24)
    off, A = problem(27, d)
    h = S.SMG(d, off, cu(A), smoother=S.ILU0, precision=prec, sweep_warps=2)
    r = cu(I.rhs(int(np.prod(d)), 2).numpy())
    z = torch.empty_like(r)
    h.set_wait_budget_ns(0)
    status = S.OK
    try:
        h.vcycle(r, z)
    except S.SmgError as e:
        status = e.status
    assert status in (S.OK, S.ETIMEOUT)
    h.set_wait_budget_ns(10 ** 9)
    ref = orc.MG(d, off, A, smoother=orc.ILU0, precision=prec).vcycle(host(r))
    for _ in range(2):
        h.vcycle(r, z)
        assert rel2(host(z), ref) < (TOL_VCYCLE if prec == 0 else TOL_LOWP)


def test_sweep_warps_query_rejects_bad_arguments(S):
    d = (8, 8, 8)
    off, A = problem(27, d)
    h = S.SMG(d, off, cu(A), smoother=S.ILU0, sweep_warps=2)
    with pytest.raises(S.SmgError):
        h.level_sweep_warps(0, S.OP_SPMV)
    with pytest.raises(S.SmgError):
        h.level_sweep_warps(99, S.OP_ILU_LOWER)
    assert h.level_sweep_warps(0, S.OP_GS_ZERO) == 0  # not this hierarchy's smoother
