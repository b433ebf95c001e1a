"""Plain FP64 reference of the learned post-smoother's network and training step.

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's baseline
leg, never by the product path).  Not in the paper: this is the optional
learned smoother of the build -- a three-layer 3x3x3 convolutional network
applied on the finest level after the V-cycle -- written from the textbook
definitions with numpy loops over the 27 taps, no blocking or fusion.

Layout: a volume with C channels is an array [C, nx, ny, nz]; a 3x3x3
convolution from Cin to Cout channels has weights W[Cout, Cin, 3, 3, 3] and
bias b[Cout]; taps outside the grid read zero (zero padding):
    out[co, x] = b[co] + sum_{ci, d in {-1,0,1}^3} W[co, ci, d+1] * in[ci, x+d].
Network: conv(2->16) -> ReLU -> conv(16->16) -> ReLU -> conv(16->1).

Precision: by default everything is FP64.  With bf16=True the functions round
at the points of the mixed-precision scheme the network is specified with
(BF16 operands, FP32 accumulation): the input, the weights and every hidden
activation are rounded to BF16 (round to nearest even), the biases and the
output to FP32; backward, the loss gradient and every back-propagated signal
are rounded to BF16.  The accumulation itself stays FP64 here.
"""
import itertools

import numpy as np

TAPS = list(itertools.product((-1, 0, 1), repeat=3))
CHANNELS = (2, 16, 16, 1)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), via FP32; returns FP64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def unflatten(theta):
    """Flat parameter vector (per layer W[cout][cin][3][3][3], then b) -> list of (W, b)."""
    theta = np.asarray(theta, dtype=np.float64)
    params, o = [], 0
    for cin, cout in zip(CHANNELS[:-1], CHANNELS[1:]):
        W = theta[o:o + cout * cin * 27].reshape(cout, cin, 3, 3, 3)
        o += cout * cin * 27
        params.append((W.copy(), theta[o:o + cout].copy()))
        o += cout
    assert o == theta.size
    return params


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def shifted(v, d):
    """v[..., x + d] with zero outside the grid (last three axes are space)."""
    out = np.zeros_like(v)
    src = [slice(max(0, t), v.shape[-3 + a] + min(0, t)) for a, t in enumerate(d)]
    dst = [slice(max(0, -t), v.shape[-3 + a] + min(0, -t)) for a, t in enumerate(d)]
    out[(Ellipsis,) + tuple(dst)] = v[(Ellipsis,) + tuple(src)]
    return out


def conv3d(x, W, b):
    """3x3x3 convolution with zero padding: x [Cin, X, Y, Z] -> [Cout, X, Y, Z]."""
    cout = W.shape[0]
    out = np.zeros((cout,) + x.shape[1:])
    for t, d in enumerate(TAPS):
        xs = shifted(x, d)
        out += np.einsum("oc,cxyz->oxyz", W[:, :, d[0] + 1, d[1] + 1, d[2] + 1], xs)
    return out + b[:, None, None, None]


def conv3d_backward(x, W, gout):
    """Gradients of sum(gout * conv3d(x, W, b)) w.r.t. x, W and b."""
    gW = np.zeros_like(W)
    gx = np.zeros_like(x)
    for d in TAPS:
        xs = shifted(x, d)
        gW[:, :, d[0] + 1, d[1] + 1, d[2] + 1] = np.einsum("oxyz,cxyz->oc", gout, xs)
        # out[x] uses in[x+d]  =>  d in[y] gets gout[y-d]
        gx += np.einsum("oc,oxyz->cxyz", W[:, :, d[0] + 1, d[1] + 1, d[2] + 1], shifted(gout, tuple(-t for t in d)))
    gb = gout.sum(axis=(1, 2, 3))
    return gx, gW, gb


def init_params(seed=0, scale=None):
    """He-style uniform initialisation, seeded."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in zip(CHANNELS[:-1], CHANNELS[1:]):
        lim = np.sqrt(6.0 / (27 * cin)) if scale is None else scale
        params.append((rng.uniform(-lim, lim, size=(cout, cin, 3, 3, 3)), np.zeros(cout)))
    return params


def _cast_params(params, bf):
    return [(bf16(W), fp32(b)) for W, b in params] if bf else params


def forward(params, x, bf=False):
    """Returns the output [1, X, Y, Z] and the activations needed backward."""
    params = _cast_params(params, bf)
    h = bf16(x) if bf else x
    acts = [h]
    for l, (W, b) in enumerate(params):
        z = conv3d(h, W, b)
        if l < len(params) - 1:
            h = np.maximum(z, 0.0)
            h = bf16(h) if bf else h
        else:
            h = fp32(z) if bf else z
        acts.append(h)
    return h, acts


def mse_loss_and_grads(params, x, target, bf=False):
    """Mean squared error over the voxels of one sample and its gradients."""
    y, acts = forward(params, x, bf)
    cp = _cast_params(params, bf)
    n = y.size
    diff = y - target
    loss = float(np.sum(diff * diff) / n)
    g = 2.0 * diff / n
    g = bf16(g) if bf else g
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = cp[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0.0)  # ReLU: derivative 1 where the output is positive
            g = bf16(g) if bf else g
        gx, gW, gb = conv3d_backward(acts[l], W, g)
        grads[l] = (gW, gb)
        g = gx
    return loss, grads


def adam_step(params, grads, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; state = (t, m, v)."""
    t, m, v = state
    t += 1
    newp, newm, newv = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        out = []
        for p_, g_, m_, v_ in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m2 = beta1 * m_ + (1 - beta1) * g_
            v2 = beta2 * v_ + (1 - beta2) * g_ * g_
            mh = m2 / (1 - beta1 ** t)
            vh = v2 / (1 - beta2 ** t)
            out.append((p_ - lr * mh / (np.sqrt(vh) + eps), m2, v2))
        newp.append((out[0][0], out[1][0]))
        newm.append((out[0][1], out[1][1]))
        newv.append((out[0][2], out[1][2]))
    return newp, (t, newm, newv)


def adam_init(params):
    z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    return (0, z, [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])


def post_smooth(apply_A, r, z, logk, params, bf=False, dinv=None):
    """Learned post-smoother step on the finest level.

    r' = r - A z,  s = ||r'||_2 / sqrt(n),  delta = s * dinv * f(r'/s, logk)
    (dinv = 1 / diag(A), the network corrects a Jacobi step; None = 1),
    and z + delta is returned if ||r' - A delta||_2 < ||r'||_2, else z.
    Vectors are flat in grid order (dims from logk's shape, [X, Y, Z]).
    Returns (new z, accepted)."""
    dims = logk.shape
    rp = r - apply_A(z)
    n = rp.size
    s = np.sqrt(np.dot(rp, rp) / n)
    inv_s = 1.0 / s if s > 0 else 0.0
    x = np.stack([(rp * inv_s).reshape(dims), logk])
    y, _ = forward(params, x, bf)
    delta = s * (1.0 if dinv is None else dinv) * y.reshape(-1)
    t = rp - apply_A(delta)
    if np.dot(t, t) < np.dot(rp, rp):
        return z + delta, True
    return z.copy(), False


def training_pair(apply_A, vcycle, e0, logk, diag=None):
    """One training pair from a known error e0: the V-cycle is applied to
    r0 = A e0, e1 = e0 - V(r0) is the error it leaves, r' = A e1 and
    s = ||r'||_2 / sqrt(n).  Returns (input [2, X, Y, Z], target [1, X, Y, Z])
    = ([r'/s, logk], diag * e1 / s): the network output y for which the
    post-smoother's correction s * y / diag equals e1 (diag None = 1)."""
    dims = logk.shape
    e1 = e0 - vcycle(apply_A(e0))
    rp = apply_A(e1)
    s = np.sqrt(np.dot(rp, rp) / rp.size)
    t = e1 / s if diag is None else diag * e1 / s
    return np.stack([(rp / s).reshape(dims), logk]), t.reshape((1,) + dims)


def identity_network(gain=1.0):
    """Parameters with f(x)[p] = gain * x[0, p] exactly (channel 1 ignored):
    layer 1 splits x into relu(x) and relu(-x), layer 2 copies both, layer 3
    recombines them with the centre tap."""
    W1 = np.zeros((16, 2, 3, 3, 3))
    W1[0, 0, 1, 1, 1], W1[1, 0, 1, 1, 1] = 1.0, -1.0
    W2 = np.zeros((16, 16, 3, 3, 3))
    W2[0, 0, 1, 1, 1], W2[1, 1, 1, 1, 1] = 1.0, 1.0
    W3 = np.zeros((1, 16, 3, 3, 3))
    W3[0, 0, 1, 1, 1], W3[0, 1, 1, 1, 1] = gain, -gain
    return [(W1, np.zeros(16)), (W2, np.zeros(16)), (W3, np.zeros(1))]


def residual_loss_and_grads(params, x, apply_A, bf=False, dinv=None):
    """Loss of the correction measured by the residual it leaves: with
    rhat = x[0] (the scaled residual r'/s) and y = f(x), the scaled
    correction is dinv * y and q = A (dinv * y) - rhat, loss = mean(q^2),
    i.e. the squared residual of the corrected iterate relative to n.  A must
    be symmetric (apply_A maps a flat vector to a flat vector), so
    d loss / d y = 2 dinv * (A q) / n.  dinv None = 1.  In bf16 mode y is the
    FP32 network output, q and A q are FP64 and the back-propagated signal is
    rounded to BF16 as in mse_loss_and_grads."""
    y, acts = forward(params, x, bf)
    cp = _cast_params(params, bf)
    n = y.size
    dv = 1.0 if dinv is None else dinv
    q = apply_A(dv * y.reshape(-1)) - x[0].reshape(-1)
    loss = float(np.dot(q, q) / n)
    g = (2.0 * dv * apply_A(q) / n).reshape(y.shape)
    g = bf16(g) if bf else g
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = cp[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0.0)
            g = bf16(g) if bf else g
        gx, gW, gb = conv3d_backward(acts[l], W, g)
        grads[l] = (gW, gb)
        g = gx
    return loss, grads
