"""GPU adjoint (spod_backward, SpodEigs) against the oracle's analytic gradient,
FP64 finite differences and the invariants of the gradient.

Gates: within 1e-5 (relative 2-norm) of the oracle's analytic gradient and
within 1e-3 of central finite differences."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import diff_like, planted

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


from paper_2309_11808_gb300 import SPOD, SpodError, _lib, spod_eigs  # noqa: E402


def loss_weights(nf, nb, bins, k=2):
    g = np.zeros((nf, nb))
    for f in bins:
        if f < nf:
            g[f, :min(k, nb)] = 1.0
    return g


def gpu_grad(X, sp, g):
    Xd = X.to(DEV).contiguous()
    sp.fit(Xd)
    dX = torch.empty(Xd.shape, dtype=torch.float64 if sp.f64 else torch.float32, device=DEV)
    _lib.spod_backward(sp.handle, torch.from_numpy(g).to(DEV), Xd, dX)
    torch.cuda.synchronize()
    return dX.double().cpu().numpy(), sp.eigs()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@cuda
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-10)])
def test_backward_matches_oracle_gradient(prec, tol):
    # differentiation workload shape, reduced: 32 x 16 grid, 2 variables, nfft 64
    dt = torch.float64 if prec == "fp64" else torch.float32
    wl = diff_like(nx=32, ny=16, nvars=2, nt=1024, nfft=64, seed=1, dtype=dt)
    sp = SPOD(wl.npoints, 2, 1024, 64, 32, dtype=dt, precision=prec, weights=wl.W)
    g = loss_weights(sp.nf, sp.nb, range(5, 21))
    dX, lam = gpu_grad(wl.X, sp, g)
    d = O.Desc(nt=1024, M=wl.M, nfft=64, noverlap=32, weights=wl.W.numpy())
    ref = O.spod_grad(wl.X.double().numpy(), d, g)
    assert rel(dX, ref) <= tol
    # invariants: zero time-sum per point (mean projection), <grad, X> = 2 L
    assert np.abs(dX.sum(axis=0)).max() <= 1e-5 * np.abs(dX).max() * 1024
    L = float((g * lam).sum())
    assert abs(float((dX * wl.X.double().numpy()).sum()) - 2 * L) <= 1e-4 * abs(L)
    sp.close()


@cuda
def test_backward_finite_differences_fp64_small_config():
    # FD check in FP64 on the 64 x 32, nt = 2048, nfft = 256 size
    wl = planted(64 * 32, 1, 2048, 256, 128, noise_std=0.1, seed=2, dtype=torch.float64)
    sp = SPOD(64 * 32, 1, 2048, 256, 128, dtype=torch.float64, precision="fp64")
    g = loss_weights(sp.nf, sp.nb, range(5, 41))
    dX, lam = gpu_grad(wl.X, sp, g)

    def L(Y):
        sp.fit(Y.to(DEV))
        return float((g * sp.eigs()).sum())

    X = wl.X
    r = torch.Generator().manual_seed(3)
    for _ in range(4):
        V = torch.randn(X.shape, generator=r, dtype=torch.float64)
        eps = 1e-5 * float(X.norm() / V.norm())
        fd = (L(X + eps * V) - L(X - eps * V)) / (2 * eps)
        an = float((dX * V.numpy()).sum())
        assert abs(fd - an) <= 1e-3 * abs(an), (fd, an)
    sp.close()


@cuda
def test_backward_chunked_and_ragged():
    g0 = torch.Generator().manual_seed(9)
    npts, nt, nfft, nov = 333, 300, 30, 10          # odd M (no TMA ring), radix 2*3*5, tail samples
    X = torch.randn(nt, npts, generator=g0, dtype=torch.float64) + 2.0
    W = (0.5 + torch.rand(npts, generator=g0, dtype=torch.float64)).numpy()
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nov, weights=W)
    nb = d.nb
    g = np.random.default_rng(4).standard_normal((d.nf, nb))
    ref = O.spod_grad(X.numpy(), d, g)
    for chunk in (0, 64):
        sp = SPOD(npts, 1, nt, nfft, nov, dtype=torch.float64, precision="fp64", weights=W, chunk_points=chunk)
        dX, _ = gpu_grad(X, sp, g)
        assert rel(dX, ref) <= 1e-10, chunk
        sp.close()


@cuda
def test_autograd_function_and_bf16x3():
    wl = diff_like(nx=32, ny=16, nvars=2, nt=1024, nfft=64, seed=5)
    X = wl.X.to(DEV).requires_grad_(True)
    d = O.Desc(nt=1024, M=wl.M, nfft=64, noverlap=32, weights=wl.W.numpy())
    for prec, tol in (("fp32", 1e-5), ("bf16x3", 1e-5)):
        sp = SPOD(wl.npoints, 2, 1024, 64, 32, precision=prec, weights=wl.W)
        lam = spod_eigs(X, sp)
        g = torch.from_numpy(loss_weights(sp.nf, sp.nb, range(5, 21))).to(DEV)
        loss = (lam * g).sum()
        (gx,) = torch.autograd.grad(loss, X)
        ref = O.spod_grad(wl.X.double().numpy(), d, g.cpu().numpy())
        err = rel(gx.double().cpu().numpy(), ref)
        print(prec, "gradient rel err", err)
        assert err <= tol
        sp.close()


@cuda
def test_backward_before_fit():
    sp = SPOD(64, 1, 200, 32, 16)
    g = torch.zeros((sp.nf, sp.nb), dtype=torch.float64, device=DEV)
    X = torch.randn(200, 64, device=DEV)
    with pytest.raises(SpodError) as e:
        _lib.spod_backward(sp.handle, g, X, torch.empty_like(X))
    assert e.value.status == _lib.SPOD_ESTATE
    sp.close()


@cuda
@pytest.mark.slow
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_backward_at_the_differentiation_size_sampled(prec, tol):
    # the differentiation workload at its full size: 256 x 128 grid, 2 variables,
    # nt = 4096, nfft = 256 (nb = 31), cos-latitude weights, loss = sum over
    # bins 5..40 of lambda_1 + lambda_2.  The oracle forms the whole Gram over
    # spatial chunks (numpy FFT step), its eigenvectors, and the gradient of
    # 1024 sampled columns (a column's gradient depends on the data only
    # through that column and the eigenvectors)
    wl = diff_like(seed=2, dtype=torch.float32, device=DEV)
    X = wl.X
    M = X.shape[1]
    sp = SPOD(wl.npoints, 2, wl.nt, wl.nfft, wl.noverlap, dtype=torch.float32, precision=prec, weights=wl.W)
    g = loss_weights(sp.nf, sp.nb, range(5, 41))
    sp.fit(X)
    dX = torch.empty(X.shape, dtype=torch.float32, device=DEV)
    _lib.spod_backward(sp.handle, torch.from_numpy(g).to(DEV), X, dX)
    cols = np.unique(np.linspace(0, M - 1, 1024).round().astype(np.int64))
    tc = torch.from_numpy(cols).to(DEV)
    got = dX[:, tc].double().cpu().numpy()
    lam = sp.eigs()
    sp.close()
    W = wl.W.numpy()
    d = O.Desc(nt=wl.nt, M=M, nfft=wl.nfft, noverlap=wl.noverlap, weights=W)
    G = np.zeros((d.nf, d.nb, d.nb), dtype=np.complex128)
    for m0 in range(0, M, 8192):
        xc = X[:, m0:m0 + 8192].double().cpu().numpy()
        Q = O.block_dft(xc, d.nfft, d.noverlap, d.w(), O.time_mean(xc), method="fft")
        G += O.gram(Q, W[m0:m0 + 8192], d.norm)
    lam_ref, Psi, _, conv = O.jacobi_eigh(G)
    assert np.all(conv)
    ref = O.grad_columns(X[:, tc].double().cpu().numpy(), d, g, Psi, W[cols])
    err = rel(got, ref)
    print(prec, "differentiation size: sampled-gradient rel err %.3e, eigenvalues of the loss bins %.3e"
          % (err, float(np.abs(lam[5:41, :2] - lam_ref[5:41, :2]).max() / lam_ref[5:41, :2].min())))
    assert err <= tol
