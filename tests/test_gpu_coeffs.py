"""Expansion coefficients and reconstruction (Eqs. coeffs and SPODrec) on the
GPU, through the C ABI, against the FP64 oracle's complex formulation.

Gates: FP64 plan 1e-9 relative (coefficients and reconstruction); FP32 plan
1e-4 relative to the largest coefficient / data value.
"""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import planted

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


from paper_2309_11808_gb300 import SPOD, SpodError, _lib  # noqa: E402


def _run(prec, dtype, fsel, nmodes_r, npts=48 * 16, nt=2048, nfft=128, nmodes=4, expect_fold=None):
    W = 0.5 + torch.rand(npts, generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    wl = planted(npts, 1, nt, nfft, nfft // 2, bins=(6, 13, 30), amps=(3.0, 2.0, 1.0), noise_std=0.2,
                 weights=W, seed=5, dtype=dtype, offset=0.4 + 0.1 * torch.rand(npts, dtype=torch.float64))
    sp = SPOD(npts, 1, nt, nfft, nfft // 2, dtype=dtype, precision=prec, weights=W)
    if expect_fold is not None:
        assert sp.mean_in_fft == expect_fold
    X = wl.X.to(DEV).contiguous()
    sp.fit(X)
    Phi = sp.modes(X, nmodes)
    cdt = torch.complex128
    A = torch.empty((len(fsel), nmodes_r, nt), dtype=cdt, device=DEV)
    _lib.spod_coeffs(sp.handle, X, Phi, nmodes, nmodes_r, fsel, A)
    Xr = torch.empty_like(X)
    _lib.spod_reconstruct(sp.handle, Phi, nmodes, nmodes_r, fsel, A, Xr)
    _lib.spod_sync(sp.handle)
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nfft // 2, weights=W.numpy())
    fit = O.spod_fit(wl.X.double().numpy(), d, dft="fft")
    Pref = O.spod_modes(fit, d, nmodes)
    Aref, P, labels = O.expansion_coefficients(wl.X.double().numpy(), d, Pref, fsel, nmodes_r, mu=fit.mu)
    Xref = O.reconstruct(Aref, P, fit.mu)
    # the oracle's A rows are (bin, mode, conjugated); the library returns the
    # coefficient of each (bin, mode) at the positive bin
    Apos = np.stack([Aref[i] for i, (f, k, cj) in enumerate(labels) if not cj]).reshape(len(fsel), nmodes_r, nt)
    sp.close()
    return A.cpu().numpy(), Apos, Xr.cpu().double().numpy(), Xref, wl.X.double().numpy()


@cuda
@pytest.mark.parametrize("prec,dtype,tol", [("fp64", torch.float64, 1e-9), ("fp32", torch.float32, 1e-4)])
def test_coefficients_and_reconstruction_match_the_oracle(prec, dtype, tol):
    fsel = [0, 6, 13, 30, 64]                    # DC, the planted bins, Nyquist
    A, Aref, Xr, Xref, X = _run(prec, dtype, fsel, 2)
    assert np.abs(A - Aref).max() <= tol * np.abs(Aref).max()
    assert np.abs(Xr - Xref).max() <= tol * np.abs(X).max()
    # the planted bins dominate the reconstruction: the residual is mostly noise
    assert np.abs(Xr - X).std() < np.abs(X - X.mean(axis=0)).std()


@cuda
def test_coefficients_and_reconstruction_with_the_mean_in_the_fft():
    # bf16x3 plan at nfft 256 (nb = 15): the time mean is taken inside the FFT
    # pass, and the reconstruction adds it back; modes from the tensor cores
    fsel = [0, 6, 13, 30, 128]
    A, Aref, Xr, Xref, X = _run("bf16x3", torch.float32, fsel, 2, nfft=256, expect_fold=True)
    assert np.abs(A - Aref).max() <= 1e-4 * np.abs(Aref).max()
    assert np.abs(Xr - Xref).max() <= 1e-4 * np.abs(X).max()


@cuda
def test_coefficients_argument_checks():
    npts, nt, nfft = 128, 512, 64
    X = torch.randn(nt, npts, device=DEV, dtype=torch.float32)
    sp = SPOD(npts, 1, nt, nfft, 32)
    Phi = torch.empty((sp.nf, 2, npts), dtype=torch.complex64, device=DEV)
    A = torch.empty((2, 1, nt), dtype=torch.complex128, device=DEV)
    with pytest.raises(SpodError) as e:
        _lib.spod_coeffs(sp.handle, X, Phi, 2, 1, [0, 3], A)
    assert e.value.status == _lib.SPOD_ESTATE
    sp.fit(X)
    sp.modes(X, 2, out=Phi)
    for nm, nr, fs in [(2, 3, [0, 3]), (2, 1, [3, 3]), (2, 1, [0, 99]), (0, 1, [1])]:
        with pytest.raises(SpodError) as e:
            _lib.spod_coeffs(sp.handle, X, Phi, nm, nr, fs, A)
        assert e.value.status == _lib.SPOD_EINVAL
    sp.close()
    spc = SPOD(npts, 1, nt, nfft, 32, dtype=torch.complex64)
    Xc = torch.randn(nt, npts, device=DEV, dtype=torch.complex64)
    spc.fit(Xc)
    with pytest.raises(SpodError) as e:
        _lib.spod_coeffs(spc.handle, Xc, Phi, 2, 1, [0], A)
    assert e.value.status == _lib.SPOD_EUNSUPPORTED
    spc.close()
