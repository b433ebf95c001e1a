"""Seeded synthetic inputs: structured matrices and right-hand sides.

This module only DEFINES test problems (discretisations and random fields); it
holds none of the multigrid method's arithmetic, and both the CUDA path and the
CPU oracle consume its output as plain input data.  The paper's own matrices
(Laplace, rhd, oil-4C, ... in Sec. 5.1) are not available, so the problems below
stand in for them with the shapes and structure that section describes.

Layout of every matrix returned here (SG-DIA, Sec. 4.1): a float64 array of
shape [nx*ny*nz, ns] (or [n, ns, B, B] for B unknowns per point), point index
p = (i*ny + j)*nz + k with z fastest, one column per stencil offset listed in
``offsets`` (lexicographic, dx slowest), off-grid coefficients zero.

Random numbers are always drawn on the CPU from ``torch.Generator`` seeded
with ``seed`` so a given seed yields the same draws on every machine; the
deterministic arithmetic that follows runs on ``device``.
"""
import itertools
import math

import torch

OFF7 = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
OFF27 = [o for o in itertools.product((-1, 0, 1), repeat=3)]
OFF19 = [o for o in OFF27 if sum(abs(t) for t in o) <= 2]


def _gen(seed):
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def rhs(n_unknowns, seed, device="cpu"):
    """Right-hand side with iid entries uniform on [-1, 1]."""
    b = torch.rand(int(n_unknowns), generator=_gen(seed), dtype=torch.float64) * 2.0 - 1.0
    return b.to(device)


def _zero_offgrid(A, dims, offsets):
    nx, ny, nz = dims
    i = torch.arange(nx, device=A.device).view(nx, 1, 1)
    j = torch.arange(ny, device=A.device).view(1, ny, 1)
    k = torch.arange(nz, device=A.device).view(1, 1, nz)
    A4 = A.view(nx, ny, nz, len(offsets), *A.shape[2:])
    for e, (dx, dy, dz) in enumerate(offsets):
        ok = ((i + dx >= 0) & (i + dx < nx) & (j + dy >= 0) & (j + dy < ny) & (k + dz >= 0) & (k + dz < nz))
        m = ok
        while m.dim() < A4[:, :, :, e].dim():
            m = m.unsqueeze(-1)
        A4[:, :, :, e] = torch.where(m, A4[:, :, :, e], torch.zeros((), dtype=A.dtype, device=A.device))
    return A


def laplace7(dims, device="cpu"):
    """7-point finite-difference Laplacian (-Delta u) with homogeneous Dirichlet
    boundary, unit spacing: diagonal 6, neighbours -1 (Table 3 'Laplace')."""
    dims = tuple(int(t) for t in dims)
    n = dims[0] * dims[1] * dims[2]
    A = torch.full((n, 7), -1.0, dtype=torch.float64, device=device)
    A[:, 3] = 6.0
    return _zero_offgrid(A, dims, OFF7)


def smoothed_field(shape, seed, sigma=4.0, std=1.5, trunc=3.0, device="cpu"):
    """iid N(0,1) per cell, separable Gaussian smoothing (sigma cells, kernel
    truncated at +-trunc*sigma, reflecting boundary), then shifted and scaled
    to mean 0 and standard deviation ``std``."""
    g = torch.randn(*shape, generator=_gen(seed), dtype=torch.float64).to(device)
    r = int(round(trunc * sigma))
    t = torch.arange(-r, r + 1, dtype=torch.float64, device=device)
    ker = torch.exp(-0.5 * (t / sigma) ** 2)
    ker = ker / ker.sum()
    x = g
    for ax in range(3):
        x = x.movedim(ax, -1).contiguous()
        m = x.shape[-1]
        pad = min(r, m - 1)
        kk = ker[r - pad:r + pad + 1] / ker[r - pad:r + pad + 1].sum()
        if pad > 0:
            # reflecting boundary without repeating the edge value
            xp = torch.cat([x[..., 1:pad + 1].flip(-1), x, x[..., m - 1 - pad:m - 1].flip(-1)], dim=-1)
        else:
            xp = x
        y = torch.zeros_like(x)
        for t in range(2 * pad + 1):
            y += kk[t] * xp[..., t:t + m]
        x = y.movedim(-1, ax)
    x = x - x.mean()
    s = x.std()
    if s > 0:
        x = x / s * std
    return x


def q1_aniso27(dims, seed, sigma=4.0, std=1.5, aniso=(1.0, 1.0, 1e-3), device="cpu"):
    """27-point variable-coefficient anisotropic diffusion: trilinear (Q1) finite
    elements on (nx+1)(ny+1)(nz+1) unit cells around nx*ny*nz interior nodes,
    element matrix kappa_e * (kx K(x)M(x)M + ky M(x)K(x)M + kz M(x)M(x)K) with
    K = [[1,-1],[-1,1]], M = [[2,1],[1,2]]/6, kappa_e = exp(g_e) for a smoothed
    Gaussian field g (std ``std``); Dirichlet zero on the boundary nodes.
    Symmetric positive definite, 27-point pattern."""
    nx, ny, nz = (int(t) for t in dims)
    kap = torch.exp(smoothed_field((nx + 1, ny + 1, nz + 1), seed, sigma, std, device=device))
    K1 = [[1.0, -1.0], [-1.0, 1.0]]
    M1 = [[2.0 / 6.0, 1.0 / 6.0], [1.0 / 6.0, 2.0 / 6.0]]
    kx, ky, kz = aniso
    A = torch.zeros((nx, ny, nz, 27), dtype=torch.float64, device=device)
    for al in itertools.product((0, 1), repeat=3):
        for be in itertools.product((0, 1), repeat=3):
            a, b, c = al
            a2, b2, c2 = be
            coef = (kx * K1[a][a2] * M1[b][b2] * M1[c][c2] + ky * M1[a][a2] * K1[b][b2] * M1[c][c2]
                    + kz * M1[a][a2] * M1[b][b2] * K1[c][c2])
            o = (a2 - a, b2 - b, c2 - c)
            e = (o[0] + 1) * 9 + (o[1] + 1) * 3 + (o[2] + 1)
            # node x (interior index) lies in cell x + 1 - alpha
            A[:, :, :, e] += coef * kap[1 - a:1 - a + nx, 1 - b:1 - b + ny, 1 - c:1 - c + nz]
    A = A.reshape(nx * ny * nz, 27)
    return _zero_offgrid(A, (nx, ny, nz), OFF27)


def _harm(a, b):
    return 2.0 * a * b / (a + b)


def fv7(dims, kappa, device="cpu"):
    """Cell-centred finite-volume 7-point operator for -div(kappa grad u): face
    transmissibility = harmonic mean of the two cells' kappa, a boundary face
    contributes kappa of its cell to the diagonal.  kappa == 1 gives exactly the
    7-point Laplacian of ``laplace7``."""
    nx, ny, nz = (int(t) for t in dims)
    kap = kappa.to(device=device, dtype=torch.float64).reshape(nx, ny, nz)
    A = torch.zeros((nx, ny, nz, 7), dtype=torch.float64, device=device)
    diag = torch.zeros((nx, ny, nz), dtype=torch.float64, device=device)
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        T = _harm(kap[tuple(lo)], kap[tuple(hi)])
        e_minus = OFF7.index(tuple(-1 if t == ax else 0 for t in range(3)))
        e_plus = OFF7.index(tuple(1 if t == ax else 0 for t in range(3)))
        A[tuple(hi) + (e_minus,)] = -T
        A[tuple(lo) + (e_plus,)] = -T
        diag[tuple(lo)] += T
        diag[tuple(hi)] += T
        b0 = [slice(None)] * 3
        b1 = [slice(None)] * 3
        b0[ax] = slice(0, 1)
        b1[ax] = slice(-1, None)
        diag[tuple(b0)] += kap[tuple(b0)]
        diag[tuple(b1)] += kap[tuple(b1)]
    A[..., 3] = diag
    return A.reshape(nx * ny * nz, 7)


def varcoef7(dims, seed, sigma=4.0, std=2.0, device="cpu"):
    """7-point variable-coefficient diffusion with kappa = exp(g), g a smoothed
    Gaussian field of standard deviation ``std``.  Returns (A, log_kappa)."""
    g = smoothed_field(tuple(int(t) for t in dims), seed, sigma, std, device=device)
    return fv7(dims, torch.exp(g), device=device), g.reshape(-1)


# exchange between the three unknowns of a cell: a nonsymmetric M-matrix with
# zero row sums (diagonal = minus the sum of the row's off-diagonal entries)
COUPLING3 = [[0.30, -0.20, -0.10], [-0.15, 0.35, -0.20], [-0.10, -0.15, 0.25]]


def block7_layered(dims, seed, layer=8, lo=1e-3, hi=1e3, device="cpu"):
    """Three unknowns per cell on a 7-point stencil (3x3 block per entry):
    per-component finite volumes with face transmissibility T = harmonic mean
    of the cells' permeability K (boundary face: K of the cell); K constant on
    ``layer``-cell-thick z-layers, log-uniform on [lo, hi].  Diagonal block =
    (sum of face T) * (I + C) with the fixed nonsymmetric exchange matrix C =
    COUPLING3 (zero row sums); off-diagonal blocks = -T * I.  The result is a
    nonsymmetric, weakly block-diagonally dominant M-matrix.  Returns A with
    shape [n, 7, 3, 3]."""
    nx, ny, nz = (int(t) for t in dims)
    nl = (nz + layer - 1) // layer
    u = torch.rand(nl, generator=_gen(seed), dtype=torch.float64)
    Kl = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    kz = Kl[torch.arange(nz) // layer].to(device)
    kap = kz.view(1, 1, nz).expand(nx, ny, nz).contiguous()
    S = fv7((nx, ny, nz), kap, device=device).reshape(nx * ny * nz, 7)
    I3 = torch.eye(3, dtype=torch.float64, device=device)
    C = torch.tensor(COUPLING3, dtype=torch.float64, device=device)
    A = S.view(-1, 7, 1, 1) * I3.view(1, 1, 3, 3)
    A[:, 3] = S[:, 3].view(-1, 1, 1) * (I3 + C).view(1, 3, 3)
    return A.contiguous()


# The learned post-smoother's network: channel counts per layer and the size
# of its parameter vector (per layer W[cout][cin][3][3][3] followed by b[cout]).
CNN_CHANNELS = (2, 16, 16, 1)
CNN_PARAMS = sum(co * ci * 27 + co for ci, co in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]))


def cnn_theta(seed):
    """Seeded initial parameters of the post-smoother network (FP32, flat):
    weights uniform on +-sqrt(6 / (27 cin)) (He-uniform), biases zero."""
    g = _gen(seed)
    parts = []
    for ci, co in zip(CNN_CHANNELS[:-1], CNN_CHANNELS[1:]):
        lim = math.sqrt(6.0 / (27 * ci))
        parts.append((torch.rand(co * ci * 27, generator=g, dtype=torch.float64) * 2.0 - 1.0) * lim)
        parts.append(torch.zeros(co, dtype=torch.float64))
    return torch.cat(parts).to(torch.float32)


def cnn_volume(dims, channels, seed, scale=1.0):
    """Seeded FP32 volume [channels][nx*ny*nz] with iid normal entries."""
    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    return (torch.randn(channels, n, generator=_gen(seed), dtype=torch.float64) * scale).to(torch.float32)
