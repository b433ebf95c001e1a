"""Training loop of the learned post-smoother (argument marshalling and loop
control only: the training pairs, the forward and backward passes, the loss
and the Adam update all run in the library's kernels).

Each training pair comes from a known error: e0 ~ N(0, 1) iid on the finest
grid, r0 = A e0, e1 = e0 - V(r0) is the error one V-cycle leaves, and the
network learns a correction delta ~ e1 from (r' = A e1, log kappa), both
scaled by s = rms(r').  The default loss measures delta by the residual it
leaves, |r' - A delta|^2 (the quantity the post-smoother's acceptance test
compares); the plain error MSE |delta - e1|^2 is the alternative.  The Gaussian draws are the only random numbers; they come from
a seeded device generator and enter the library as inputs.
"""
import torch

from . import smg as S
from .inputs import CNN_PARAMS, cnn_theta


class PostSmootherTrainer:
    """Trains the network on the finest level of one or more hierarchies.

    `mg` is an smg.SMG with one unknown per point, or a list of them (one
    per coefficient field, all on the same grid); `logk` is log(kappa) on
    that grid (float64 device tensor), or the matching list.  Samples cycle
    through the fields in order."""

    def __init__(self, mg, logk, seed=0, lr=1e-3, batch=4, theta=None, loss_kind=S.LOSS_RESIDUAL, stream=None):
        self.fields = list(zip(mg, logk)) if isinstance(mg, (list, tuple)) else [(mg, logk)]
        self.lr, self.batch, self.loss_kind = lr, int(batch), loss_kind
        mg, logk = self.fields[0]
        assert all(tuple(m.dims) == tuple(mg.dims) for m, _ in self.fields)
        self.nsamples = 0
        self.dims = list(mg.dims)
        n = self.dims[0] * self.dims[1] * self.dims[2]
        dev = logk.device
        self.theta = (cnn_theta(seed) if theta is None else theta.float().cpu()).to(dev).contiguous()
        assert self.theta.numel() == CNN_PARAMS
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.ws = S.cnn_workspace(self.dims)
        self.in2 = torch.empty(2 * n, dtype=torch.float32, device=dev)
        self.target = torch.empty(n, dtype=torch.float32, device=dev)
        self.e0 = torch.empty(n, dtype=torch.float64, device=dev)
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(int(seed) + 7919)
        self.t = 0
        self.stream = stream

    def sample(self):
        """Draws e0 and builds one training pair into (in2, target); returns
        the hierarchy it came from."""
        mg, logk = self.fields[self.nsamples % len(self.fields)]
        self.nsamples += 1
        self.e0.normal_(generator=self.gen)
        mg.learned_sample(self.e0, logk, self.in2, self.target, self.stream)
        return mg

    def _loss_grad(self, mg, grad, loss):
        mg.learned_loss_grad(self.theta, self.in2, self.target, grad, loss, self.ws, self.loss_kind, self.stream)

    def step(self):
        """One Adam step on a fresh batch; returns the batch's mean loss as a
        device tensor (reading it synchronises)."""
        self.grad.zero_()
        self.loss.zero_()
        for _ in range(self.batch):
            self._loss_grad(self.sample(), self.grad, self.loss)
        self.t += 1
        S.cnn_adam(self.theta, self.m, self.v, self.grad, self.t, lr=self.lr, grad_scale=1.0 / self.batch,
                   stream=self.stream)
        return self.loss / self.batch

    def eval_loss(self, samples=4):
        """Mean loss of the current parameters over fresh pairs (no update)."""
        scratch = torch.zeros_like(self.grad)
        loss = torch.zeros(1, dtype=torch.float32, device=self.theta.device)
        for _ in range(samples):
            self._loss_grad(self.sample(), scratch, loss)
        return float(loss.item()) / samples

    def train(self, steps):
        """Runs `steps` Adam steps; returns the per-step losses (host floats)."""
        losses = [self.step() for _ in range(int(steps))]
        return [float(x.item()) for x in losses]
