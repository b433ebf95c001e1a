"""The allocation-free sweep entry point (smg_sweep_noalloc).

It is meant for callers that cannot let a library allocate device memory --
applications whose device memory is owned by their own pool, fixed-budget
real-time callers, plug-ins whose host forbids cudaMalloc.  It keeps its
scratch in a fixed device array, so these checks run it twice in a row on
the same array and compare every result with the context-based entry point
(smg_level_apply), which runs the same sweep kernel, with the same operation order, on the
hierarchy's own data: the results must be bit-identical.  This file is
collected last on purpose.
"""
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")



@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_21932_gb300 import build, smg
    build.build()
    return smg


def same(a, b):
    return torch.equal(a, b)


@pytest.mark.gpu
@pytest.mark.parametrize("d,off", [((24, 20, 16), I.OFF27), ((20, 33, 12), I.OFF7), ((2, 600, 5), I.OFF7)])
def test_noalloc_gauss_seidel_matches_context_sweeps(S, d, off):
    A = (I.q1_aniso27(d, 1) if len(off) == 27 else I.varcoef7(d, 2)[0]).cuda().contiguous()
    n = d[0] * d[1] * d[2]
    h = S.SMG(d, off, A, smoother=S.SGS, max_levels=1)
    dinv = h.level_array(0, S.ARR_DINV).view(torch.float64)
    b = I.rhs(n, 3).cuda()
    u_ref = I.rhs(n, 4).cuda()
    u = u_ref.clone()
    # two calls in a row on the same scratch: forward then backward
    h.level_apply(0, S.OP_GS_FORWARD, x=u_ref, b=b)
    assert S.sweep_noalloc(S.OP_GS_FORWARD, d, off, A, dinv, b, u) == S.OK
    assert same(u, u_ref)
    h.level_apply(0, S.OP_GS_BACKWARD, x=u_ref, b=b)
    assert S.sweep_noalloc(S.OP_GS_BACKWARD, d, off, A, dinv, b, u) == S.OK
    assert same(u, u_ref)
    # ZeroGuess ignores the old iterate
    z_ref = torch.zeros_like(u)
    h.level_apply(0, S.OP_GS_ZERO, x=z_ref, b=b)
    z = torch.full_like(u, 7.0)
    assert S.sweep_noalloc(S.OP_GS_ZERO, d, off, A, dinv, b, z) == S.OK
    assert same(z, z_ref)


@pytest.mark.gpu
def test_noalloc_ilu_solves_match_context_sweeps(S):
    d = (16, 24, 20)
    A = I.q1_aniso27(d, 5).cuda().contiguous()
    n = d[0] * d[1] * d[2]
    h = S.SMG(d, I.OFF27, A, smoother=S.ILU0, max_levels=1)
    LU = h.level_array(0, S.ARR_LU).view(torch.float64)
    udinv = h.level_array(0, S.ARR_DINV).view(torch.float64)
    r = I.rhs(n, 6).cuda()
    y_ref = torch.empty_like(r)
    h.level_apply(0, S.OP_ILU_LOWER, b=r, y=y_ref)
    for _ in range(2):  # twice in a row, separate output, then in place
        y = torch.empty_like(r)
        assert S.sweep_noalloc(S.OP_ILU_LOWER, d, I.OFF27, LU, None, r, y) == S.OK
        assert same(y, y_ref)
    x_ref = y_ref.clone()
    h.level_apply(0, S.OP_ILU_UPPER, b=x_ref, y=x_ref)
    x = y_ref.clone()
    assert S.sweep_noalloc(S.OP_ILU_UPPER, d, I.OFF27, LU, udinv, x, x) == S.OK
    assert same(x, x_ref)


@pytest.mark.gpu
def test_noalloc_rejects_what_it_cannot_hold(S):
    def vecs(d, ns):
        n = d[0] * d[1] * d[2]
        z = lambda m: torch.zeros(m, dtype=torch.float64, device="cuda")
        return z(n * ns), z(n), z(n), z(n)

    d_big = (4097, 4, 4)  # one progress counter per x-plane: 4096 planes at most
    assert S.sweep_noalloc(S.OP_GS_FORWARD, d_big, I.OFF7, *vecs(d_big, 7)) == S.EINVAL
    d_wide = (2, 1025, 2)  # one thread per y-column: 1024 columns at most
    assert S.sweep_noalloc(S.OP_GS_FORWARD, d_wide, I.OFF7, *vecs(d_wide, 7)) == S.EINVAL
    unsorted = [I.OFF7[e] for e in (3, 0, 1, 2, 4, 5, 6)]
    assert S.sweep_noalloc(S.OP_GS_FORWARD, (4, 4, 4), unsorted, *vecs((4, 4, 4), 7)) == S.EINVAL
    M, dv, b, u = vecs((4, 4, 4), 7)
    assert S.sweep_noalloc(S.OP_ILU_UPPER, (4, 4, 4), I.OFF7, M, None, b, u) == S.EINVAL
    # the binding refuses tensors that do not hold the grid before any call
    with pytest.raises(ValueError):
        S.sweep_noalloc(S.OP_GS_FORWARD, (4, 4, 4), I.OFF7, M[:-1], dv, b, u)
    with pytest.raises(ValueError):
        S.sweep_noalloc(S.OP_GS_FORWARD, (4, 4, 4), I.OFF7, M, dv.float(), b, u)
