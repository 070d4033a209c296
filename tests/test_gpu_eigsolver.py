"""The batched Hermitian eigen-solver (Householder + implicit QL) on matrices
with a prescribed spectrum, fed through spod_fit_from_grams.

Each frequency gets M_f = U diag(lambda) U^H with a seeded random unitary U
and one of four spectra: eigenvalues spread over twelve decades, tight
clusters (equal to the last bit and split by 1e-9), a rank-deficient Gram
(five nonzero eigenvalues, the rest exactly zero) and uniform ones, each
scaled by a power of ten.  The reference is numpy's FP64 eigh of the same
stored matrix.  Gates, relative to lambda_1 of the frequency (a backward
stable solver moves each eigenvalue by at most c u ||M||_2, Weyl):
eigenvalues 1e-13 (FP64 plans, u = 2^-53) and 1e-11 (the other plans, whose
rotation chain runs in double-FP32, u = 2^-47); residuals
||M psi_k - lambda_k psi_k|| and ||Psi^H Psi - I|| the same; eigenvectors of
eigenvalues separated from the rest by >= 1e-3 lambda_1 parallel to the
reference within 1e-9.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
DEV = "cuda:0"
NFFT, NB = 64, 38
NT = NFFT + (NB - 1) * (NFFT // 2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def spectrum(f, n, rng):
    kind = f % 4
    if kind == 0:
        lam = np.logspace(0, -12, n)
    elif kind == 1:
        base = np.logspace(0, -6, n // 3 + 1)
        lam = np.repeat(base, 3)[:n].copy()
        lam[1::3] *= 1.0 + 1e-9
    elif kind == 2:
        lam = np.zeros(n)
        lam[:5] = np.logspace(0, -3, 5)
    else:
        lam = rng.uniform(0.0, 1.0, n)
    return lam * 10.0 ** ((f % 7) - 3)


def hermitian(lam, rng):
    n = lam.size
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    m = (q * lam) @ q.conj().T
    m = 0.5 * (m + m.conj().T)
    m[np.diag_indices(n)] = m[np.diag_indices(n)].real
    return m


@cuda
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-11), ("bf16x3", 1e-11)])
def test_prescribed_spectra(prec, tol):
    from paper_2309_11808_gb300 import SPOD, _lib
    dt = torch.float64 if prec == "fp64" else torch.float32
    sp = SPOD(16, 1, NT, NFFT, NFFT // 2, dtype=dt, precision=prec)
    assert sp.nb == NB
    nf = sp.nf
    st = torch.cuda.current_stream()
    X = torch.randn(NT, 16, dtype=dt, device=DEV)
    part = torch.empty((nf, NB, NB, 2), dtype=torch.float64, device=DEV)
    _lib.spod_fit_partial(sp.handle, X, part, st)
    rng = np.random.default_rng(20260)
    mats = np.stack([hermitian(spectrum(f, NB, rng), rng) for f in range(nf)])
    grams = torch.from_numpy(np.stack([mats.real, mats.imag], axis=-1)[None].copy()).to(DEV)
    _lib.spod_fit_from_grams(sp.handle, grams, 1, st)
    lam, psi = sp.eigs(vectors=True)
    sp.close()
    worst = dict(lam=0.0, res=0.0, orth=0.0, vec=0.0)
    for f in range(nf):
        m = mats[f]
        w, v = np.linalg.eigh(m)
        w, v = w[::-1], v[:, ::-1]
        scale = max(abs(w[0]), 1e-300)
        assert np.all(np.diff(lam[f]) <= 0.0), f
        worst["lam"] = max(worst["lam"], np.max(np.abs(lam[f] - w)) / scale)
        P = psi[f]
        worst["res"] = max(worst["res"], np.max(np.linalg.norm(m @ P - P * lam[f], axis=0)) / scale)
        worst["orth"] = max(worst["orth"], np.max(np.abs(P.conj().T @ P - np.eye(NB))))
        gap = np.full(NB, np.inf)
        gap[:-1] = np.minimum(gap[:-1], w[:-1] - w[1:])
        gap[1:] = np.minimum(gap[1:], w[:-1] - w[1:])
        for k in np.nonzero(gap >= 1e-3 * scale)[0]:
            worst["vec"] = max(worst["vec"], 1.0 - abs(np.vdot(v[:, k], P[:, k])))
    print(prec, {k: f"{x:.2e}" for k, x in worst.items()})
    assert worst["lam"] <= tol
    assert worst["res"] <= tol
    assert worst["orth"] <= tol
    assert worst["vec"] <= 1e-9
