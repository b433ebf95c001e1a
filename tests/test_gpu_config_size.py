"""Parity with the oracle at the configurations' own sizes, in the launch
configuration the benchmark times (default options):

* one whole ILU(0) V-cycle of the 27-point anisotropic problem at 256^3
  against the oracle's, 1e-12 in the 2-norm;
* the PCG solve of the same family at 128^3: the same iteration count within
  one, the true residual recomputed by the oracle below the tolerance, and
  the FP32 / BF16 hierarchies' FPCG solutions stated against the oracle's
  FP64 solution;
* the FP32 and BF16 cycles against the oracle's same-precision cycle at 96^3;
* the 3-unknown system at its full 128 x 128 x 64 under FGMRES(30), FP64 and
  FP32 hierarchies, iteration counts within one of the oracle's;
* one forward pass of the learned post-smoother at 64^3 (the training size)
  against the oracle's BF16-rounding network.

The oracle's set-up runs its Galerkin products on all host cores (each
coarse point is independent; no sum changes order)."""
import numpy as np
import pytest

from paper_2506_21932_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_VCYCLE = 1e-12
TOL_LOWP = 2e-5
TOL_EMU = 2e-3


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


def q1(d, seed=0):
    A = I.q1_aniso27(d, seed, device="cuda").contiguous()
    return A, A.cpu().numpy()


def test_c2_whole_vcycle_at_256(S, orc):
    """One ILU(0) V-cycle over all seven levels of the 256^3 hierarchy."""
    d = (256, 256, 256)
    A_d, A = q1(d)
    r = I.rhs(256 ** 3, 3).numpy()
    h = S.SMG(d, I.OFF27, A_d, smoother=S.ILU0)
    z = torch.empty(256 ** 3, dtype=torch.float64, device="cuda")
    h.vcycle(cu(r), z)
    h.close()
    del A_d
    torch.cuda.empty_cache()
    zr = orc.MG(d, I.OFF27, A, smoother=orc.ILU0).vcycle(r)
    assert rel2(host(z), zr) < TOL_VCYCLE


@pytest.fixture(scope="module")
def c2_128(S, orc):
    d = (128, 128, 128)
    A_d, A = q1(d)
    b = I.rhs(128 ** 3, 1000).numpy()
    x64, rc, it, rr, _ = orc.MG(d, I.OFF27, A, smoother=orc.ILU0).pcg(b, tol=1e-9, maxit=500)
    assert rc == 0
    return d, A_d, A, b, x64, it


def test_c2_pcg_at_128_matches_oracle(S, orc, c2_128):
    d, A_d, A, b, x64, it_ref = c2_128
    h = S.SMG(d, I.OFF27, A_d, smoother=S.ILU0)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=500)
    assert rc == 0 and rr < 1e-9 and abs(it - it_ref) <= 1
    res = np.linalg.norm(orc.residual(d, I.OFF27, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9
    # the same iterates as the oracle's, up to rounding
    assert rel2(host(x), x64) < 1e-8


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_precision_solutions_at_128_against_fp64(S, orc, c2_128, prec):
    """FPCG with an FP32 / BF16 hierarchy (FP64 outer iteration) reaches the
    same relative residual; its error against the oracle's FP64 solution is
    that of two 1e-9 solves, not of the hierarchy's precision."""
    d, A_d, A, b, x64, it_ref = c2_128
    h = S.SMG(d, I.OFF27, A_d, smoother=S.ILU0, precision=prec, krylov=S.FPCG)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    it, rr, rc = h.solve(cu(b), x, tol=1e-9, maxit=500)
    assert rc == 0 and rr < 1e-9 and it <= it_ref + 3
    res = np.linalg.norm(orc.residual(d, I.OFF27, A, b, host(x))) / np.linalg.norm(b)
    assert res < 1e-9
    # two solves to a relative residual of 1e-9 differ by at most the
    # condition number times that; measured well below it
    assert rel2(host(x), x64) < 1e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_c3_reduced_precision_vcycle_at_96(S, orc, prec):
    d = (96, 96, 96)
    A_d, A = q1(d)
    r = I.rhs(96 ** 3, 4).numpy()
    h = S.SMG(d, I.OFF27, A_d, smoother=S.ILU0, precision=prec, krylov=S.FPCG)
    z = torch.empty(96 ** 3, dtype=torch.float64, device="cuda")
    h.vcycle(cu(r), z)
    zr = orc.MG(d, I.OFF27, A, smoother=orc.ILU0, precision=prec).vcycle(r)
    assert rel2(host(z), zr) < TOL_LOWP


@pytest.mark.parametrize("prec", [0, 1])
def test_c4_full_size_fgmres(S, orc, prec):
    """The 3-unknown system at 128 x 128 x 64 (3.1 M unknowns), FGMRES(30) to
    1e-8: the iteration count of the oracle's run at the same precision within
    one, and the true residual recomputed by the oracle."""
    d = (128, 128, 64)
    A = I.block7_layered(d, 0).numpy()
    n = 3 * 128 * 128 * 64
    b = I.rhs(n, 1000).numpy()
    h = S.SMG(d, I.OFF7, cu(A), block=3, smoother=S.SGS, transfer=S.PC8C, precision=prec, krylov=S.FGMRES,
              restart=30)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    it, rr, rc = h.solve(cu(b), x, tol=1e-8, maxit=300)
    assert rc == 0 and rr < 1e-8
    _, rco, ito, _, _ = orc.MG(d, I.OFF7, A, B=3, transfer=orc.PC8C, precision=prec).fgmres(b, tol=1e-8, restart=30,
                                                                                        maxit=300)
    assert rco == 0 and abs(it - ito) <= 1
    res = np.linalg.norm(orc.residual(d, I.OFF7, A, b, host(x), B=3)) / np.linalg.norm(b)
    assert res < 1e-8


def test_cnn_forward_at_64(S):
    """One forward pass of the post-smoother network over a whole 64^3
    volume (the training size: every brick shape of the launch)."""
    from oracle import cnn_oracle as C
    d = (64, 64, 64)
    theta = I.cnn_theta(21)
    theta[880 - 16:880] = torch.linspace(-0.2, 0.2, 16)
    theta[-1] = 0.05
    x = I.cnn_volume(d, 2, seed=22)
    out = torch.empty(64 ** 3, dtype=torch.float32, device="cuda")
    S.cnn_forward(d, cu(theta.numpy()), cu(x.numpy()), out, S.cnn_workspace(d))
    ref = C.forward(C.unflatten(theta.numpy()), x.numpy().astype(np.float64).reshape((2,) + d), bf=True)[0].ravel()
    assert rel2(host(out).astype(np.float64), ref) < TOL_EMU
