"""Pins of the FP64 CNN reference (oracle/cnn_oracle.py) against facts it
does not compute itself: scipy's correlate with zero padding, a single-tap
kernel that is a pure shift, central finite differences for every gradient,
and the closed form of Adam's first step."""
import numpy as np
import pytest

scipy_nd = pytest.importorskip("scipy.ndimage")

from oracle import cnn_oracle as C


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6, 7))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    b = rng.normal(size=2)
    got = C.conv3d(x, W, b)
    for o in range(2):
        ref = sum(scipy_nd.correlate(x[c], W[o, c], mode="constant", cval=0.0) for c in range(3)) + b[o]
        assert np.max(np.abs(got[o] - ref)) < 1e-12


def test_single_tap_is_a_shift():
    x = np.random.default_rng(1).normal(size=(1, 4, 5, 6))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 2, 0, 1] = 1.0  # tap (dx,dy,dz) = (+1,-1,0): out[x] = in[x + (1,-1,0)]
    out = C.conv3d(x, W, np.zeros(1))[0]
    ref = np.zeros_like(out)
    ref[:-1, 1:, :] = x[0, 1:, :-1, :]
    assert np.array_equal(out, ref)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    params = C.init_params(seed=3)
    for sample in range(2):
        x = rng.normal(size=(2, 6, 6, 6))
        target = rng.normal(size=(1, 6, 6, 6))
        loss, grads = C.mse_loss_and_grads(params, x, target)
        h = 1e-6
        for l in range(3):
            W, b = params[l]
            for idx in [(0, 0, 1, 1, 1), (W.shape[0] - 1, W.shape[1] - 1, 0, 2, 1), (0, W.shape[1] - 1, 2, 2, 0)]:
                def L(delta):
                    P = [(w.copy(), bb.copy()) for w, bb in params]
                    P[l][0][idx] += delta
                    return C.mse_loss_and_grads(P, x, target)[0]
                fd = (L(h) - L(-h)) / (2 * h)
                assert abs(grads[l][0][idx] - fd) <= 1e-6 * max(1e-3, abs(fd)), (l, idx)
            def Lb(delta):
                P = [(w.copy(), bb.copy()) for w, bb in params]
                P[l][1][0] += delta
                return C.mse_loss_and_grads(P, x, target)[0]
            fd = (Lb(h) - Lb(-h)) / (2 * h)
            assert abs(grads[l][1][0] - fd) <= 1e-6 * max(1e-3, abs(fd))


def test_input_gradient_of_convolution_is_the_adjoint():
    """<conv(x), y> = <x, conv^T(y)> with conv^T from conv3d_backward."""
    rng = np.random.default_rng(4)
    x = rng.normal(size=(3, 5, 4, 6))
    y = rng.normal(size=(2, 5, 4, 6))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    lhs = np.sum(C.conv3d(x, W, np.zeros(2)) * y)
    gx, _, _ = C.conv3d_backward(x, W, y)
    assert abs(lhs - np.sum(x * gx)) < 1e-10 * abs(lhs)


def test_adam_first_step_closed_form():
    """From a zero state, the bias-corrected first moment is g and the second
    g^2, so the first update is -lr * g / (|g| + eps)."""
    params = [(np.array([[[[[1.0]]]]]), np.array([2.0]))]
    grads = [(np.array([[[[[0.5]]]]]), np.array([-3.0]))]
    newp, state = C.adam_step(params, grads, C.adam_init(params), lr=0.1)
    assert abs(newp[0][0].item() - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15
    assert abs(newp[0][1].item() - (2.0 + 0.1 * 3.0 / (3.0 + 1e-8))) < 1e-15
    assert state[0] == 1


def test_network_has_the_stated_size():
    n = sum(W.size + b.size for W, b in C.init_params())
    assert n == 2 * 16 * 27 + 16 + 16 * 16 * 27 + 16 + 16 * 27 + 1 == 8241


def test_bf16_rounding_matches_torch_and_the_c_oracle():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-20, 20, size=4000),
                        # exact ties between two BF16 values (both parities)
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(C.bf16(x), ref)
    from oracle import oracle as O
    for v in x[:50]:
        assert C.bf16(v) == O.bf16_round(float(np.float32(v)))


def test_flat_parameter_layout_round_trips():
    p = C.init_params(seed=7)
    q = C.unflatten(C.flatten(p))
    for (W, b), (W2, b2) in zip(p, q):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)
    assert C.flatten(p)[880 - 16:880].tolist() == [0.0] * 16  # b1 follows W1 (16*2*27 = 864)


def test_identity_network_solves_a_diagonal_system_exactly():
    """With A = c I the exact error is r'/c; the identity network scaled by
    1/c yields it, so the step is accepted and z becomes A^-1 r.  With the
    Jacobi scaling dinv = 1/c the unscaled identity network does the same."""
    rng = np.random.default_rng(6)
    dims = (4, 5, 6)
    c = 3.0
    r = rng.normal(size=np.prod(dims))
    z = rng.normal(size=np.prod(dims))
    logk = rng.normal(size=dims)
    A = lambda v: c * v
    znew, ok = C.post_smooth(A, r, z, logk, C.identity_network(1.0 / c))
    assert ok
    assert np.max(np.abs(znew - r / c)) < 1e-13
    znew, ok = C.post_smooth(A, r, z, logk, C.identity_network(1.0), dinv=np.full(r.size, 1.0 / c))
    assert ok
    assert np.max(np.abs(znew - r / c)) < 1e-13


def test_post_smoother_rejects_a_step_that_does_not_reduce_the_residual():
    rng = np.random.default_rng(7)
    dims = (4, 4, 4)
    r, z = rng.normal(size=64), rng.normal(size=64)
    A = lambda v: 2.0 * v
    zero = [(np.zeros_like(W), np.zeros_like(b)) for W, b in C.init_params()]
    znew, ok = C.post_smooth(A, r, z, rng.normal(size=dims), zero)  # delta = 0
    assert not ok and np.array_equal(znew, z)
    znew, ok = C.post_smooth(A, r, z, rng.normal(size=dims), C.identity_network(-1.0))  # wrong sign
    assert not ok and np.array_equal(znew, z)


def test_training_pair_of_an_exact_solver_is_zero():
    """If the V-cycle were exact, it would leave no error: target 0."""
    rng = np.random.default_rng(8)
    dims = (4, 4, 4)
    e0 = rng.normal(size=64)
    A = lambda v: 2.0 * v
    near_exact = lambda rr: rr / 2.0 + 1e-3 * rng.normal(size=64)
    x, t = C.training_pair(A, near_exact, e0, np.zeros(dims))
    # e1 = -1e-3 noise, r' = 2 e1, s = rms(r'); target = e1 / s has rms 1/2
    assert abs(np.sqrt(np.mean(t ** 2)) - 0.5) < 1e-12
    assert np.allclose(x[0].ravel(), 2.0 * t.ravel())


def test_residual_loss_with_a_scaled_identity_is_a_scaled_mse():
    """A = c I: loss = mean((c y - rhat)^2) = c^2 mean((y - rhat/c)^2), and
    its gradients are c^2 times those of the MSE against rhat / c."""
    rng = np.random.default_rng(9)
    params = C.init_params(seed=10)
    x = rng.normal(size=(2, 5, 4, 6))
    c = 1.7
    lr_, gr = C.residual_loss_and_grads(params, x, lambda v: c * v)
    lm, gm = C.mse_loss_and_grads(params, x, x[:1] / c)
    assert abs(lr_ - c * c * lm) < 1e-12 * lr_
    for (a, b), (e, f) in zip(gr, gm):
        assert np.max(np.abs(a - c * c * e)) < 1e-12 * max(1.0, np.max(np.abs(a)))
        assert np.max(np.abs(b - c * c * f)) < 1e-12 * max(1.0, np.max(np.abs(b)))


def test_residual_loss_gradients_match_central_differences():
    """A = a symmetric positive 7-point operator on the 5x5x5 grid."""
    rng = np.random.default_rng(11)
    dims = (5, 5, 5)
    params = C.init_params(seed=12)
    x = rng.normal(size=(2,) + dims)

    def A(v):
        u = v.reshape(dims)
        out = 8.0 * u
        for ax in range(3):
            for sh in (-1, 1):
                out -= C.shifted(u[None], tuple(sh if a == ax else 0 for a in range(3)))[0]
        return out.reshape(-1)

    loss, grads = C.residual_loss_and_grads(params, x, A)
    h = 1e-6
    for l in range(3):
        W = params[l][0]
        for idx in [(0, 0, 1, 1, 1), (W.shape[0] - 1, W.shape[1] - 1, 2, 0, 1)]:
            def L(delta):
                P = [(w.copy(), bb.copy()) for w, bb in params]
                P[l][0][idx] += delta
                return C.residual_loss_and_grads(P, x, A)[0]
            fd = (L(h) - L(-h)) / (2 * h)
            assert abs(grads[l][0][idx] - fd) <= 1e-6 * max(1e-3, abs(fd)), (l, idx)


def test_residual_loss_with_jacobi_scaling_of_a_diagonal_matrix_is_the_mse():
    """A = diag(d) with dinv = 1/d: A (dinv y) = y, so the residual loss is
    the MSE of y against rhat and the gradients agree with it."""
    rng = np.random.default_rng(13)
    dims = (4, 5, 3)
    params = C.init_params(seed=14)
    x = rng.normal(size=(2,) + dims)
    d = rng.uniform(0.5, 3.0, size=np.prod(dims))
    lr_, gr = C.residual_loss_and_grads(params, x, lambda v: d * v, dinv=1.0 / d)
    lm, gm = C.mse_loss_and_grads(params, x, x[:1])
    assert abs(lr_ - lm) < 1e-12 * lm
    for (a, b), (e, f) in zip(gr, gm):
        assert np.max(np.abs(a - e)) < 1e-12 * max(1.0, np.max(np.abs(a)))
        assert np.max(np.abs(b - f)) < 1e-12 * max(1.0, np.max(np.abs(b)))


def test_training_target_reproduces_the_error_through_the_jacobi_scaling():
    rng = np.random.default_rng(15)
    dims = (3, 4, 5)
    n = int(np.prod(dims))
    diag = rng.uniform(1.0, 4.0, size=n)
    A = lambda v: diag * v + 0.1 * np.roll(v, 1) + 0.1 * np.roll(v, -1)
    e0 = rng.normal(size=n)
    vc = lambda rr: rr / diag
    x, t = C.training_pair(A, vc, e0, np.zeros(dims), diag=diag)
    e1 = e0 - vc(A(e0))
    s = np.sqrt(np.mean(A(e1) ** 2))
    assert np.allclose(s * t.ravel() / diag, e1, rtol=1e-13, atol=1e-15)
