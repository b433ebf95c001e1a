"""Parity of the learned post-smoother's CUDA path (through the C ABI) with
the FP64 network oracle, and a training run that shows its effect.

Tolerances.  The kernels round operands to BF16 and accumulate in FP32.  The
oracle's bf16 mode rounds at the same points and accumulates in FP64, so what
remains is the FP32 accumulation (at most 432 products per output, relative
error ~432 * 2^-24 = 2.6e-5 of the sum of magnitudes) and the rare hidden
activation whose BF16 rounding flips because of it (one BF16 ulp, 2^-8, on a
small fraction of activations): 2e-3 in the 2-norm.  Against the plain FP64
oracle the BF16 roundings themselves count (unit roundoff 2^-9 per rounding,
several roundings on every path through the network): 2e-2.  Adam runs in
FP32 on both FP32 inputs: 1e-5 relative.
"""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_EMU = 2e-3
TOL_FP64 = 2e-2


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_21932_gb300 import build, smg
    build.build()
    return smg


@pytest.fixture(scope="module")
def C():
    from oracle import cnn_oracle
    return cnn_oracle


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel2(got, ref):
    return np.linalg.norm(np.asarray(got) - ref) / max(np.linalg.norm(ref), 1e-300)


def rel_max(got, ref):
    return np.max(np.abs(np.asarray(got) - ref)) / max(np.max(np.abs(ref)), 1e-300)


# several 2 x 4 x 32 output bricks with a ragged tail in every direction
DIMS = [(5, 9, 45), (2, 4, 32), (1, 1, 7), (6, 13, 70)]


@pytest.mark.parametrize("d", DIMS)
def test_forward_matches_oracle(S, C, d):
    theta = I.cnn_theta(11)
    theta[880 - 16:880] = torch.linspace(-0.2, 0.2, 16)  # nonzero biases
    theta[-1] = 0.05
    x = I.cnn_volume(d, 2, seed=12)
    n = x.shape[1]
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ws = S.cnn_workspace(d)
    S.cnn_forward(d, cu(theta.numpy()), cu(x.numpy()), out, ws)
    got = out.cpu().numpy().astype(np.float64)
    params = C.unflatten(theta.numpy())
    xo = x.numpy().astype(np.float64).reshape((2,) + d)
    ref_emu = C.forward(params, xo, bf=True)[0].ravel()
    ref64 = C.forward(params, xo)[0].ravel()
    assert rel2(got, ref_emu) < TOL_EMU
    assert rel_max(got, ref_emu) < 5 * TOL_EMU
    assert rel2(got, ref64) < TOL_FP64


@pytest.mark.parametrize("d", [(5, 9, 45), (6, 13, 70)])
def test_loss_and_gradients_match_oracle(S, C, d):
    theta = I.cnn_theta(21)
    theta[880 - 16:880] = 0.05
    x = I.cnn_volume(d, 2, seed=22)
    tgt = I.cnn_volume(d, 1, seed=23, scale=0.5)
    ws = S.cnn_workspace(d)
    grad = torch.zeros(I.CNN_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    S.cnn_loss_grad(d, cu(theta.numpy()), cu(x.numpy()), cu(tgt.numpy()), grad, loss, ws)
    torch.cuda.synchronize()
    params = C.unflatten(theta.numpy())
    xo = x.numpy().astype(np.float64).reshape((2,) + d)
    to = tgt.numpy().astype(np.float64).reshape((1,) + d)
    g = grad.cpu().numpy().astype(np.float64)
    for bf, tol in ((True, TOL_EMU), (False, TOL_FP64)):
        lref, gref = C.mse_loss_and_grads(params, xo, to, bf=bf)
        assert abs(loss.item() - lref) <= tol * lref
        gflat = C.flatten(gref)
        o = 0
        for l, (W, b) in enumerate(params):
            nw = W.size
            assert rel2(g[o:o + nw], gflat[o:o + nw]) < 2 * tol, (bf, l, "W")
            assert rel2(g[o + nw:o + nw + b.size], gflat[o + nw:o + nw + b.size]) < 2 * tol, (bf, l, "b")
            o += nw + b.size
    # gradients and loss accumulate across calls
    S.cnn_loss_grad(d, cu(theta.numpy()), cu(x.numpy()), cu(tgt.numpy()), grad, loss, ws)
    assert rel2(grad.cpu().numpy(), 2 * g) < 1e-6


def test_adam_matches_oracle(S, C):
    rng = np.random.default_rng(31)
    th = rng.normal(size=I.CNN_PARAMS).astype(np.float32)
    m = (rng.normal(size=I.CNN_PARAMS) * 1e-2).astype(np.float32)
    v = (rng.uniform(size=I.CNN_PARAMS) * 1e-4).astype(np.float32)
    g = rng.normal(size=I.CNN_PARAMS).astype(np.float32)
    tt, mm, vv = cu(th), cu(m), cu(v)
    S.cnn_adam(tt, mm, vv, cu(g), 3, lr=2e-3, grad_scale=0.25)
    P = C.unflatten(th.astype(np.float64))
    G = C.unflatten(0.25 * g.astype(np.float64))
    M = C.unflatten(m.astype(np.float64))
    V = C.unflatten(v.astype(np.float64))
    # the kernel's hyperparameters are FP32 numbers (1 - float(0.999) differs
    # from 0.001 by 1.3e-5 relative): give the oracle the same values
    f32 = lambda x: float(np.float32(x))
    newp, (t, newm, newv) = C.adam_step(P, G, (2, M, V), lr=f32(2e-3), beta1=f32(0.9), beta2=f32(0.999),
                                        eps=f32(1e-8))
    assert t == 3
    # FP32 rounding of each update: a few float ulps of the largest term
    # (m and v can cancel to near zero, so the bound is absolute in the terms)
    eps = 2.0 ** -23
    gs = 0.25 * np.abs(g.astype(np.float64))
    tol_m = 4 * eps * (0.9 * np.abs(m) + 0.1 * gs)
    tol_v = 4 * eps * (0.999 * np.abs(v) + 0.001 * gs * gs)
    assert np.all(np.abs(mm.cpu().numpy() - C.flatten(newm)) <= tol_m + 1e-30)
    assert np.all(np.abs(vv.cpu().numpy() - C.flatten(newv)) <= tol_v + 1e-30)
    # the step lr * mhat / (sqrt(vhat) + eps): in FP32 the bias correction
    # 1 - beta2^t (0.003 at t = 3) carries eps / 0.003 = 2e-5 relative error,
    # halved by the square root; plus the rounding of theta itself
    step = np.abs(th - C.flatten(newp))
    assert np.all(np.abs(tt.cpu().numpy() - C.flatten(newp)) <= 4 * eps * np.abs(th) + 3e-5 * step)


def test_invalid_arguments_are_rejected(S):
    d = (4, 4, 4)
    ws = S.cnn_workspace(d)
    t = torch.zeros(I.CNN_PARAMS, dtype=torch.float32, device="cuda")
    x = torch.zeros(128, dtype=torch.float32, device="cuda")
    y = torch.zeros(64, dtype=torch.float32, device="cuda")
    with pytest.raises(S.SmgError):
        S.cnn_forward((0, 4, 4), t, x, y, ws)
    with pytest.raises(S.SmgError):
        S.cnn_forward(d, t, x, y, ws[:16])  # short workspace


# ---------------------------------------------------------------------------
# the post-smoother inside the V-cycle, and training pairs
# ---------------------------------------------------------------------------

def varcoef(d, seed):
    A, g = I.varcoef7(d, seed)
    return A.numpy(), g.numpy()


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


def test_training_pair_matches_oracle(S, C, orc):
    d = (16, 16, 16)
    A, logk = varcoef(d, 1000)
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.FPCG)
    mg = orc.MG(d, I.OFF7, A, smoother=orc.SGS)
    n = A.shape[0]
    e0 = np.random.default_rng(41).normal(size=n)
    in2 = torch.empty(2 * n, dtype=torch.float32, device="cuda")
    tgt = torch.empty(n, dtype=torch.float32, device="cuda")
    h.learned_sample(cu(e0), cu(logk), in2, tgt)
    diag = A[:, I.OFF7.index((0, 0, 0))]
    xr, tr = C.training_pair(lambda v: orc.spmv(d, I.OFF7, A, v), mg.vcycle, e0, logk.reshape(d), diag=diag)
    assert rel_max(in2.cpu().numpy()[:n], xr[0].ravel()) < 1e-6
    assert np.array_equal(in2.cpu().numpy()[n:], logk.astype(np.float32))
    assert rel_max(tgt.cpu().numpy(), tr.ravel()) < 1e-6


def test_residual_loss_and_gradients_match_oracle(S, C, orc):
    """Loss |A y - r'/s|^2 / n on the context's finest matrix and its
    gradient, against the oracle in its BF16-rounding mode (the A products
    amplify the network's rounding differences by the spread of A's
    eigenvalues, hence twice the forward tolerance)."""
    d = (16, 16, 16)
    A, logk = varcoef(d, 7)
    n = A.shape[0]
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.FPCG)
    theta = I.cnn_theta(5)
    theta[880 - 16:880] = 0.03
    x = I.cnn_volume(d, 2, seed=8)
    x[1] = torch.from_numpy(logk.astype(np.float32))
    ws = S.cnn_workspace(d)
    grad = torch.zeros(I.CNN_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    h.learned_loss_grad(cu(theta.numpy()), cu(x.numpy()), None, grad, loss, ws, kind=S.LOSS_RESIDUAL)
    torch.cuda.synchronize()
    params = C.unflatten(theta.numpy())
    xo = x.numpy().astype(np.float64).reshape((2,) + d)
    dinv = 1.0 / A[:, I.OFF7.index((0, 0, 0))]
    lref, gref = C.residual_loss_and_grads(params, xo, lambda v: orc.spmv(d, I.OFF7, A, v), bf=True, dinv=dinv)
    assert abs(loss.item() - lref) <= 2 * TOL_EMU * lref
    g = grad.cpu().numpy().astype(np.float64)
    gflat = C.flatten(gref)
    o = 0
    for l, (W, b) in enumerate(params):
        nw = W.size
        assert rel2(g[o:o + nw], gflat[o:o + nw]) < 4 * TOL_EMU, (l, "W")
        assert rel2(g[o + nw:o + nw + b.size], gflat[o + nw:o + nw + b.size]) < 4 * TOL_EMU, (l, "b")
        o += nw + b.size
    with pytest.raises(S.SmgError):
        h.learned_loss_grad(cu(theta.numpy()), cu(x.numpy()), None, grad, loss, ws, kind=7)


def test_post_smoother_matches_oracle_when_accepted_and_rejected(S, C, orc):
    d = (16, 16, 16)
    A, logk = varcoef(d, 3)
    n = A.shape[0]
    r = I.rhs(n, 4).numpy()
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.FPCG)
    mg = orc.MG(d, I.OFF7, A, smoother=orc.SGS)
    Aop = lambda v: orc.spmv(d, I.OFF7, A, v)
    z_plain = torch.empty(n, dtype=torch.float64, device="cuda")
    h.vcycle(cu(r), z_plain)
    zo = mg.vcycle(r)
    # (1) a damped Jacobi step delta = 0.3 D^-1 r' (the identity network
    #     times 0.3 through the Jacobi scaling): accepted
    dinv = 1.0 / A[:, I.OFF7.index((0, 0, 0))]
    gain = 0.3
    params = C.identity_network(gain)
    theta = cu(C.flatten(params).astype(np.float32))
    lk = cu(logk)
    h.set_learned_smoother(theta, lk)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    h.vcycle(cu(r), z)
    zref, ok = C.post_smooth(Aop, r, zo, logk.reshape(d), C.unflatten(C.flatten(params).astype(np.float32)), bf=True,
                             dinv=dinv)
    assert ok
    assert rel2(z.cpu().numpy(), zref) < 1e-6
    assert rel2(z.cpu().numpy(), z_plain.cpu().numpy()) > 1e-6  # the step changed z
    # (2) the same step with the wrong sign increases the residual: rejected,
    #     and the result is the plain V-cycle's bit for bit
    h.set_learned_smoother(cu(C.flatten(C.identity_network(-gain)).astype(np.float32)), lk)
    h.vcycle(cu(r), z)
    assert torch.equal(z, z_plain)
    # (3) detached: the plain V-cycle again
    h.set_learned_smoother(None, None)
    h.vcycle(cu(r), z)
    assert torch.equal(z, z_plain)


def test_replace_mode_falls_back_to_the_plain_vcycle_and_converges(S, C):
    """SMG_LEARNED_REPLACE: the network stands in for the finest level's
    post-smoothing.  (1) A correction the test rejects (the wrong-sign Jacobi
    step) makes the skipped post-smoothing run: the result is the plain
    V-cycle's bit for bit.  (2) An accepted one (a damped Jacobi step) gives
    another, still contracting, preconditioner.  (3) FPCG with it converges
    to the tolerance, the true residual confirming it."""
    d = (16, 16, 16)
    A, logk = varcoef(d, 3)
    n = A.shape[0]
    r = cu(I.rhs(n, 4).numpy())
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.FPCG)
    z_plain = torch.empty(n, dtype=torch.float64, device="cuda")
    h.vcycle(r, z_plain)
    lk = cu(logk)
    h.set_learned_mode(S.LEARNED_REPLACE)
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    h.set_learned_smoother(cu(C.flatten(C.identity_network(-0.3)).astype(np.float32)), lk)
    h.vcycle(r, z)
    assert torch.equal(z, z_plain)
    h.set_learned_smoother(cu(C.flatten(C.identity_network(0.3)).astype(np.float32)), lk)
    h.vcycle(r, z)
    assert not torch.equal(z, z_plain)
    from oracle import oracle as orc
    res = np.linalg.norm(host_np(r) - orc.spmv(d, I.OFF7, A, host_np(z))) / np.linalg.norm(host_np(r))
    assert res < 1.0
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr, rc = h.solve(r, x, tol=1e-9, maxit=200)
    assert rc == 0 and rr < 1e-9
    res = np.linalg.norm(host_np(r) - orc.spmv(d, I.OFF7, A, host_np(x))) / np.linalg.norm(host_np(r))
    assert res < 1e-9
    with pytest.raises(S.SmgError):
        h.set_learned_mode(7)


def host_np(t):
    return t.detach().cpu().numpy()


def test_learned_smoother_requires_a_flexible_krylov_method(S):
    d = (8, 8, 8)
    A, logk = varcoef(d, 5)
    h = S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.PCG)
    with pytest.raises(S.SmgError):
        h.set_learned_smoother(cu(I.cnn_theta(0).numpy()), cu(logk))


def test_training_lowers_the_loss_and_the_iteration_count(S):
    """Trains on 32^3 problems of the variable-coefficient family (training
    seeds), then solves a problem of another seed with FPCG and the learned
    post-smoother, against FPCG with the plain V-cycle."""
    from paper_2506_21932_gb300.learned import PostSmootherTrainer
    d = (32, 32, 32)
    hs, lks = [], []
    for seed in (1000, 1001, 1002, 1003):
        A, logk = varcoef(d, seed)
        hs.append(S.SMG(d, I.OFF7, cu(A), smoother=S.SGS, krylov=S.FPCG))
        lks.append(cu(logk))
    tr = PostSmootherTrainer(hs, lks, seed=0, lr=2e-3, batch=4)
    before = tr.eval_loss(8)
    tr.train(150)
    after = tr.eval_loss(8)
    print("residual loss %.4g -> %.4g" % (before, after))
    # below 1: on average the correction leaves a smaller residual than r'
    assert after < 0.8 * before and after < 1.0, (before, after)

    A2, logk2 = varcoef(d, 0)
    n = A2.shape[0]
    b = cu(I.rhs(n, 0).numpy())
    plain = S.SMG(d, I.OFF7, cu(A2), smoother=S.SGS, krylov=S.FPCG)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it_plain, rr_plain, _ = plain.solve(b, x, tol=1e-9, maxit=200)
    learned = S.SMG(d, I.OFF7, cu(A2), smoother=S.SGS, krylov=S.FPCG)
    learned.set_learned_smoother(tr.theta, cu(logk2))
    x.zero_()
    it_l, rr_l, _ = learned.solve(b, x, tol=1e-9, maxit=200)
    # what one preconditioner application leaves of a random residual
    ratios = {}
    for name, h in (("plain", plain), ("learned", learned)):
        acc = []
        for seed in range(3):
            r = cu(np.random.default_rng(100 + seed).normal(size=n))
            z = torch.empty_like(r)
            h.vcycle(r, z)
            t = torch.empty_like(r)
            h.level_apply(0, S.OP_RESIDUAL, x=z, b=r, y=t)
            acc.append(float(t.norm() / r.norm()))
        ratios[name] = sum(acc) / len(acc)
    print("loss %.4g -> %.4g; residual left by one application: plain %.4g, learned %.4g; FPCG iterations "
          "plain %d, learned %d" % (before, after, ratios["plain"], ratios["learned"], it_plain, it_l))
    assert rr_l < 1e-9 and rr_plain < 1e-9
    assert ratios["learned"] < 0.8 * ratios["plain"]
    assert it_l <= it_plain
