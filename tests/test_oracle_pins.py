"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numbers the
paper prints, closed forms for planted signals, identities (Parseval, trace,
W-orthonormality, reconstruction), independent library routines (numpy FFT,
LAPACK eigvalsh, scipy windows) and brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from workloads import planted, w_orthonormal_modes

HERE = os.path.dirname(os.path.abspath(__file__))


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- sizes
def test_block_counts_printed_in_paper():
    with open(os.path.join(HERE, "golden", "paper_block_counts.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        assert O.n_blocks(c["nt"], c["nfft"], c["noverlap"]) == c["L"], c["cite"]


def test_block_counts_workloads():
    assert O.n_blocks(2048, 256, 128) == 15
    assert O.n_blocks(10000, 512, 256) == 38
    assert O.n_blocks(4096, 256, 128) == 31
    # tail dropped, blocks from t = 0
    assert O.n_blocks(300, 100, 0) == 3 and O.n_blocks(299, 100, 0) == 2
    with pytest.raises(ValueError):
        O.n_blocks(10, 16, 0)
    with pytest.raises(ValueError):
        O.n_blocks(100, 16, 16)


def test_one_sided_count():
    # floor(N/2)+1: for even N this equals the paper's ceil(N/2)+1
    for n in (2, 6, 256, 512, 720):
        assert O.n_freqs(n) == math.ceil(n / 2) + 1
    assert O.n_freqs(15) == 8


# ---------------------------------------------------------------- window
def test_windows_match_scipy():
    sig = pytest.importorskip("scipy.signal")
    for n in (6, 15, 256, 384):
        np.testing.assert_allclose(O.window(O.WIN_HAMMING, n), sig.windows.hamming(n, sym=True), atol=1e-15)
        np.testing.assert_allclose(O.window(O.WIN_HAMMING_PERIODIC, n), sig.windows.hamming(n, sym=False), atol=1e-15)
        np.testing.assert_allclose(O.window(O.WIN_HANN, n), sig.windows.hann(n, sym=True), atol=1e-15)
    assert np.all(O.window(O.WIN_RECT, 7) == 1.0)


# ---------------------------------------------------------------- DFT
@pytest.mark.parametrize("nfft,nov", [(16, 8), (15, 5), (30, 0), (6, 3), (24, 12)])
def test_direct_dft_matches_numpy_fft(nfft, nov):
    r = _rng(nfft)
    nt, M = 3 * nfft + 5, 7
    X = r.standard_normal((nt, M)) + 2.0
    w = O.window(O.WIN_HAMMING, nfft)
    mu = X.mean(axis=0)
    Qd = O.block_dft(X, nfft, nov, w, mu, method="direct")
    # independent: numpy FFT of each windowed block, one-sided part
    step = nfft - nov
    nb = O.n_blocks(nt, nfft, nov)
    for l in range(nb):
        ref = np.fft.fft(w[:, None] * (X[l * step:l * step + nfft] - mu), axis=0)[: nfft // 2 + 1] / w.sum()
        np.testing.assert_allclose(Qd[:, l, :], ref, atol=1e-13)
    Qf = O.block_dft(X, nfft, nov, w, mu, method="fft")
    np.testing.assert_allclose(Qd, Qf, atol=1e-13)


def test_dft_bin_centred_sinusoid_amplitude():
    # a bin-centred sinusoid of amplitude a under the periodic Hamming window gives
    # |q_hat| = a/2 at its bin (c = 1/sum w, Sec. 2.2 DFT reading)
    nfft, k, a = 64, 5, 3.0
    t = np.arange(nfft)
    X = (a * np.sin(2 * np.pi * k * t / nfft + 0.3))[:, None]
    Q = O.block_dft(X, nfft, 0, O.window(O.WIN_HAMMING_PERIODIC, nfft), None)
    assert abs(abs(Q[k, 0, 0]) - a / 2) < 1e-13
    assert abs(abs(Q[k + 1, 0, 0]) - (a / 2) * 0.23 / 0.54) < 1e-13
    assert abs(Q[k + 3, 0, 0]) < 1e-13


# ---------------------------------------------------------------- eig
def _rand_herm(r, B, n, rank=None):
    A = r.standard_normal((B, n, n)) + 1j * r.standard_normal((B, n, n))
    if rank is not None:
        A = A[:, :, :rank] @ np.conj(np.transpose(A[:, :, :rank], (0, 2, 1)))
    else:
        A = A + np.conj(np.transpose(A, (0, 2, 1)))
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 7, 15, 38])
def test_jacobi_matches_lapack(n):
    r = _rng(n)
    A = _rand_herm(r, 5, n)
    lam, V, sweeps, conv = O.jacobi_eigh(A)
    assert conv
    ref = np.linalg.eigvalsh(A)[:, ::-1]
    np.testing.assert_allclose(lam, ref, atol=1e-12 * np.abs(ref).max())
    # residual, unitarity, phase rule
    R = A @ V - V * lam[:, None, :]
    assert np.abs(R).max() < 1e-11 * np.abs(ref).max()
    VV = np.conj(np.transpose(V, (0, 2, 1))) @ V
    np.testing.assert_allclose(VV, np.broadcast_to(np.eye(n), VV.shape), atol=1e-12)
    idx = np.argmax(np.abs(V), axis=1)
    piv = np.take_along_axis(V, idx[:, None, :], axis=1)
    assert np.all(np.abs(piv.imag) < 1e-14) and np.all(piv.real > 0)


def test_jacobi_special_cases():
    D = np.diag([3.0, 1.0, 2.0]).astype(complex)[None]
    lam, V, sweeps, conv = O.jacobi_eigh(D)
    assert conv and sweeps == 0
    np.testing.assert_array_equal(lam[0], [3.0, 2.0, 1.0])
    # ties keep the lower diagonal index first
    I = np.eye(4, dtype=complex)[None] * 2.0
    lam, V, _, _ = O.jacobi_eigh(I)
    np.testing.assert_array_equal(lam[0], [2.0] * 4)
    np.testing.assert_array_equal(np.abs(V[0]), np.eye(4))
    # PSD rank-deficient (the Gram when nb > M)
    r = _rng(3)
    A = _rand_herm(r, 2, 6, rank=2)
    lam, V, _, conv = O.jacobi_eigh(A)
    assert conv
    assert np.all(np.abs(lam[:, 2:]) < 1e-12 * lam[:, :1])
    # zero matrix
    lam, V, sweeps, conv = O.jacobi_eigh(np.zeros((1, 3, 3), complex))
    assert conv and np.all(lam == 0)


# ---------------------------------------------------------------- whole fit
def _small_desc(nt=160, M=24, nfft=32, nov=16, window=O.WIN_HAMMING, seed=0, W=None):
    r = _rng(seed)
    if W is None:
        W = 0.5 + r.random(M)
    return O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, window=window, weights=W)


def test_snapshot_method_equals_direct_csd():
    # Eq. csd-discrete / spod-discrete vs Eq. spod-discrete-snapshots: the M x M
    # problem C_k W phi = lambda phi and the nb x nb Gram share nonzero eigenvalues;
    # the oracle's modes solve the M x M problem.
    d = _small_desc(nt=200, M=12, nfft=32, nov=16)
    X = _rng(1).standard_normal((d.nt, d.M)) * 1.5 + 0.7
    fit = O.spod_fit(X, d)
    nb = d.nb
    Phi = O.spod_modes(fit, d, nb)
    W = d.W()
    for f in (0, 3, d.nf - 1):
        Qk = fit.Qhat[f].T                                   # M x nb
        C = Qk @ np.conj(Qk.T) / nb                          # Eq. csd-discrete with 1/nb
        ev = np.sort(np.linalg.eigvals(C @ np.diag(W)).real)[::-1]
        r = min(nb, d.M)
        np.testing.assert_allclose(fit.lam[f, :r], ev[:r], rtol=1e-9, atol=1e-12 * ev[0])
        for k in range(r):
            phi = Phi[f, k]
            res = C @ (W * phi) - fit.lam[f, k] * phi
            assert np.linalg.norm(res) < 1e-9 * fit.lam[f, 0]


@pytest.mark.parametrize("nfft,nov", [(32, 16), (31, 10), (30, 0)])
def test_parseval_identity(nfft, nov):
    d = _small_desc(nt=7 * nfft + 3, M=10, nfft=nfft, nov=nov, seed=nfft)
    X = _rng(nfft + 1).standard_normal((d.nt, d.M)) + 5.0
    fit = O.spod_fit(X, d)
    g = O.one_sided_multiplicity(nfft)
    lhs = float((g * np.trace(fit.M, axis1=1, axis2=2).real).sum())
    rhs = O.parseval_rhs(X, d)
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_trace_orthonormality_reconstruction():
    d = _small_desc(nt=180, M=40, nfft=24, nov=12, seed=5)
    X = _rng(6).standard_normal((d.nt, d.M))
    fit = O.spod_fit(X, d)
    tr = np.trace(fit.M, axis1=1, axis2=2).real
    np.testing.assert_allclose(fit.lam.sum(axis=1), tr, rtol=1e-12)
    nb = d.nb
    Phi = O.spod_modes(fit, d, nb)
    W = d.W()
    for f in range(d.nf):
        P = Phi[f].T                                         # M x nb
        G = np.conj(P.T) @ (W[:, None] * P)
        np.testing.assert_allclose(G, np.eye(nb), atol=1e-10)  # Sec. 2.2: Phi^* W Phi = I
        # full-rank reconstruction: sqrt(nb) Phi Lambda^{1/2} Psi^H = Qhat_f
        Qr = math.sqrt(nb) * (P * np.sqrt(fit.lam[f])[None, :]) @ np.conj(fit.Psi[f].T)
        np.testing.assert_allclose(Qr, fit.Qhat[f].T, atol=1e-10 * np.abs(fit.Qhat[f]).max())


def test_planted_closed_form_periodic_hamming():
    # Planted W-orthonormal modes x bin-centred sinusoids, periodic Hamming:
    # lambda_1 = a^2/4 at the planted bin, (a^2/4)(0.23/0.54)^2 at its neighbours,
    # and 0 elsewhere.  A per-point offset and a tail outside the last block test
    # the mean subtraction (over all nt) and the block layout.
    npts, nt, nfft = 64 * 32, 2048 + 77, 256
    W = torch.tensor(0.5 + _rng(9).random(npts))
    off = torch.tensor(_rng(10).standard_normal(npts) * 10.0)
    wl = planted(npts, 1, nt, nfft, nfft // 2, noise_std=0.0, weights=W, seed=4, offset=off)
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nfft // 2, window=O.WIN_HAMMING_PERIODIC,
               weights=W.numpy())
    fit = O.spod_fit(wl.X.numpy(), d, dft="fft")
    r = (0.23 / 0.54) ** 2
    expect = np.zeros(d.nf)
    for k, a in zip((10, 25, 60), (3.0, 2.0, 1.0)):
        expect[k] = a * a / 4
        expect[k - 1] = expect[k + 1] = a * a / 4 * r
    # the tail makes the sinusoids' sample mean nonzero: that constant only
    # reaches bins 0 and 1 through the window, so compare from bin 3 on
    np.testing.assert_allclose(fit.lam[3:, 0], expect[3:], atol=1e-12)
    assert np.all(fit.lam[3:, 1] < 1e-12)


def test_planted_closed_form_no_tail_all_bins():
    npts, nt, nfft = 256, 1024, 128
    wl = planted(npts, 1, nt, nfft, nfft // 2, bins=(3, 17, 40), amps=(1.0, 2.0, 0.5),
                 noise_std=0.0, seed=8)
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nfft // 2, window=O.WIN_HAMMING_PERIODIC)
    fit = O.spod_fit(wl.X.numpy(), d)
    r = (0.23 / 0.54) ** 2
    expect = np.zeros(d.nf)
    for k, a in zip((3, 17, 40), (1.0, 2.0, 0.5)):
        expect[k] = a * a / 4
        expect[k - 1] = expect[k + 1] = a * a / 4 * r
    np.testing.assert_allclose(fit.lam[:, 0], expect, atol=1e-12)


def test_planted_closed_form_symmetric_hamming():
    # With the symmetric window the planted part of Qhat_f is
    #   sum_j phi_j c_j^T,  c_j[l] = (a_j c / 2i) (e^{i th_jl} Wh(f-k_j) - e^{-i th_jl} Wh(f+k_j)),
    # th_jl = th_j + 2 pi k_j l step / nfft, Wh the window's DFT; with W-orthonormal
    # phi the nonzero eigenvalues of M_f are those of (1/nb) C C^H (3 x 3).
    npts, nt, nfft, nov = 512, 2048, 256, 128
    W = torch.tensor(0.5 + _rng(2).random(npts))
    wl = planted(npts, 1, nt, nfft, nov, noise_std=0.0, weights=W, seed=3)
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nov, window=O.WIN_HAMMING, weights=W.numpy())
    fit = O.spod_fit(wl.X.numpy(), d, dft="fft")
    w = O.window(O.WIN_HAMMING, nfft)
    c = 1.0 / w.sum()
    n = np.arange(nfft)
    step, nb = nfft - nov, d.nb

    def Wh(k):
        return np.sum(w * np.exp(-2j * np.pi * k * n / nfft))

    th = wl.meta["theta"].numpy()
    for f in (4, 10, 11, 25, 33, 60, 61, 100):
        C = np.zeros((3, nb), complex)
        for j, (k, a) in enumerate(zip(wl.meta["bins"], wl.meta["amps"])):
            for l in range(nb):
                thl = th[j] + 2 * np.pi * k * l * step / nfft
                C[j, l] = a * c / 2j * (np.exp(1j * thl) * Wh(f - k) - np.exp(-1j * thl) * Wh(f + k))
        ev = np.sort(np.linalg.eigvalsh(C @ np.conj(C.T) / nb))[::-1]
        np.testing.assert_allclose(fit.lam[f, :3], ev, atol=1e-13 + 1e-11 * ev[0])


def test_mean_offset_invariance_and_norm_option():
    d = _small_desc(nt=150, M=9, nfft=20, nov=10, seed=2)
    X = _rng(4).standard_normal((d.nt, d.M))
    a = O.spod_fit(X, d)
    b = O.spod_fit(X + 100.0 * _rng(5).standard_normal(d.M)[None, :], d)
    np.testing.assert_allclose(a.lam, b.lam, rtol=1e-9, atol=1e-12 * a.lam.max())
    # without mean subtraction the DC bin changes
    d2 = O.Desc(**{**d.__dict__, "subtract_mean": False})
    c2 = O.spod_fit(X + 100.0, d2)
    assert c2.lam[0, 0] > 1e3 * a.lam[0, 0]
    # Bessel normalisation of Eq. csd-discrete scales eigenvalues by nb/(nb-1)
    d3 = O.Desc(**{**d.__dict__, "norm": O.NORM_NB_MINUS_1})
    e = O.spod_fit(X, d3)
    np.testing.assert_allclose(e.lam, a.lam * d.nb / (d.nb - 1), rtol=1e-12, atol=1e-15)
    P1 = O.spod_modes(a, d, 3)
    P3 = O.spod_modes(e, d3, 3)
    np.testing.assert_allclose(P1, P3, atol=1e-12)


def test_workload_modes_are_w_orthonormal():
    W = torch.tensor(0.5 + _rng(1).random(50))
    phi = w_orthonormal_modes(50, 3, W, 0)
    G = phi.T @ (W[:, None] * phi)
    np.testing.assert_allclose(G.numpy(), np.eye(3), atol=1e-13)


# ---------------------------------------------------------------- gradient
def _grad_case(seed=0, nt=96, M=10, nfft=16, nov=8):
    d = _small_desc(nt=nt, M=M, nfft=nfft, nov=nov, seed=seed)
    X = _rng(seed + 100).standard_normal((d.nt, d.M)) + 1.0
    g = _rng(seed + 200).standard_normal((d.nf, d.nb))
    return d, X, g


def test_gradient_matches_finite_differences():
    d, X, g = _grad_case()
    fit = O.spod_fit(X, d)
    gap = np.min(np.abs(np.diff(fit.lam, axis=1)) / fit.lam[:, :1])
    assert gap > 1e-6        # simple eigenvalues
    G = O.spod_grad(X, d, g, fit)

    def L(Y):
        return O.loss_from_fit(O.spod_fit(Y, d), g)

    r = _rng(7)
    for _ in range(5):
        V = r.standard_normal(X.shape)
        eps = 1e-5 * np.linalg.norm(X) / np.linalg.norm(V)
        fd = (L(X + eps * V) - L(X - eps * V)) / (2 * eps)
        an = float((G * V).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_gradient_of_sampled_columns_equals_the_whole_gradient():
    # the gradient restricted to a few columns (their own Qhat, the whole
    # fit's eigenvectors) equals those columns of the whole-array gradient,
    # which is pinned against finite differences above
    rng = _rng(33)
    nt, M, nfft = 700, 40, 64
    W = 0.5 + rng.random(M)
    X = rng.standard_normal((nt, M)) + 2.0 * rng.standard_normal(M)[None, :]
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=32, weights=W)
    fit = O.spod_fit(X, d)
    g = np.zeros((d.nf, d.nb))
    g[3:20, :2] = 1.0
    g[7, 4] = -0.5
    full = O.spod_grad(X, d, g, fit)
    cols = [0, 7, 8, 39]
    part = O.grad_columns(X[:, cols], d, g, fit.Psi, W[cols])
    np.testing.assert_allclose(part, full[:, cols], rtol=0, atol=1e-12 * np.abs(full).max())


def test_gradient_homogeneity_and_shift():
    d, X, g = _grad_case(seed=1)
    fit = O.spod_fit(X, d)
    G = O.spod_grad(X, d, g, fit)
    L = O.loss_from_fit(fit, g)
    # eigenvalues are quadratic in X: <grad L, X> = 2 L
    assert abs(float((G * X).sum()) - 2 * L) <= 1e-10 * abs(L)
    # mean subtraction: gradient sums to zero over time at every point
    assert np.abs(G.sum(axis=0)).max() < 1e-12 * np.abs(G).max() * d.nt


def test_gradient_identity_weights_is_time_domain_parseval():
    # g[f, k] = multiplicity g_f for all k makes G_f = g_f I (full rank), so
    # L = sum_f g_f tr M_f = parseval_rhs, whose gradient is 2 C w_n^2 W_m xt
    # overlap-added, then mean-projected.
    d, X, _ = _grad_case(seed=2, nt=60, M=30, nfft=12, nov=6)
    assert d.nb <= d.M
    mult = O.one_sided_multiplicity(d.nfft)
    g = np.repeat(mult[:, None], d.nb, axis=1)
    G = O.spod_grad(X, d, g)
    w = d.w()
    C = (1.0 / w.sum()) ** 2 * d.nfft / d.nb
    xt = X - X.mean(axis=0)
    ref = np.zeros_like(X)
    step = d.nfft - d.noverlap
    for l in range(d.nb):
        ref[l * step:l * step + d.nfft] += 2 * C * (w ** 2)[:, None] * d.W()[None, :] * xt[l * step:l * step + d.nfft]
    ref -= ref.mean(axis=0)
    np.testing.assert_allclose(G, ref, atol=1e-12 * np.abs(ref).max())


def test_gram_at_freqs_closed_form_and_full_gram():
    # Selected-bin Gram over spatial chunks: closed-form planted eigenvalues
    # (periodic Hamming, with a per-point offset removed by each chunk's own
    # mean) and the full-transform Gram on a noisy case
    npts, nt, nfft = 40 * 24, 1024, 128
    W = torch.tensor(0.5 + _rng(21).random(npts))
    off = torch.tensor(_rng(22).standard_normal(npts) * 5.0)
    wl = planted(npts, 1, nt, nfft, nfft // 2, bins=(3, 17, 40), amps=(1.0, 2.0, 0.5), noise_std=0.0,
                 weights=W, seed=23, offset=off)
    d = O.Desc(nt=nt, M=npts, nfft=nfft, noverlap=nfft // 2, window=O.WIN_HAMMING_PERIODIC, weights=W.numpy())
    X = wl.X.numpy()
    fsel = [3, 4, 17, 40, 41, 55]
    G = O.gram_at_freqs(d, fsel, lambda a, b: X[:, a:b], chunk=100)
    lam = np.sort(np.linalg.eigvalsh(G), axis=1)[:, ::-1]
    r = (0.23 / 0.54) ** 2
    expect = {3: 0.25, 4: 0.25 * r, 17: 1.0, 40: 0.0625, 41: 0.0625 * r, 55: 0.0}
    for i, f in enumerate(fsel):
        assert abs(lam[i, 0] - expect[f]) < 1e-12, f
        assert lam[i, 1] < 1e-12
    rng = _rng(24)
    Xn = X + 0.1 * rng.standard_normal(X.shape)
    Gn = O.gram_at_freqs(d, fsel, lambda a, b: Xn[:, a:b], chunk=77)
    full = O.gram(O.block_dft(Xn, nfft, nfft // 2, d.w(), O.time_mean(Xn)), d.W())
    np.testing.assert_allclose(Gn, full[fsel], rtol=0, atol=1e-13 * np.abs(full).max())


def test_qhat_at_freqs_matches_the_fft_transform():
    # Selected-bin, selected-column Qhat from DFT rows (with each column's own
    # mean) against numpy's FFT of the whole array (with the array's mean)
    rng = _rng(31)
    nt, M, nfft, nov = 700, 37, 96, 40
    X = rng.standard_normal((nt, M)) + 3.0 * rng.standard_normal(M)[None, :]
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, window=O.WIN_HANN)
    full = O.block_dft(X, nfft, nov, d.w(), X.mean(axis=0), method="fft")
    fsel, cols = [0, 1, 7, 33, 48], [0, 5, 6, 36]
    Q = O.qhat_at_freqs(X[:, cols], d, fsel)
    np.testing.assert_allclose(Q, full[fsel][:, :, cols], rtol=0, atol=1e-12 * np.abs(full).max())
    # without the mean, and with the means given
    d0 = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, window=O.WIN_HANN, subtract_mean=False)
    raw = O.block_dft(X, nfft, nov, d.w(), None, method="fft")
    np.testing.assert_allclose(O.qhat_at_freqs(X[:, cols], d0, fsel), raw[fsel][:, :, cols], rtol=0,
                               atol=1e-12 * np.abs(raw).max())
    mu = X[:, cols].mean(axis=0)
    np.testing.assert_allclose(O.qhat_at_freqs(X[:, cols], d, fsel, mu=mu), Q, rtol=0, atol=1e-13 * np.abs(Q).max())


def test_modes_at_sampled_columns_equal_the_full_modes():
    # Modes restricted to a few columns and bins equal those columns of the
    # whole-grid modes (which are pinned by W-orthonormality above)
    rng = _rng(32)
    nt, M, nfft = 900, 60, 64
    W = 0.5 + rng.random(M)
    X = rng.standard_normal((nt, M))
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=32, weights=W, norm=O.NORM_NB_MINUS_1)
    fit = O.spod_fit(X, d)
    Phi = O.spod_modes(fit, d, 6)
    fsel, cols = [0, 3, 20, 32], [1, 2, 30, 59]
    Q = O.qhat_at_freqs(X[:, cols], d, fsel)
    Pm = O.modes_at(Q, fit.lam[fsel], fit.Psi[fsel], 6, d.norm, d.nb)
    np.testing.assert_allclose(Pm, Phi[fsel][:, :, cols], rtol=0, atol=1e-12 * np.abs(Phi).max())


# ---------------------------------------------------------------- complex data
# Complex Q (allowed by Eq. data-matrix): all nfft bins, no conjugate symmetry.
def test_complex_direct_dft_matches_fft_and_two_sided_parseval():
    rs = np.random.RandomState(21)
    nt, M, nfft, nov = 300, 7, 30, 10
    X = rs.randn(nt, M) + 1j * rs.randn(nt, M) + (0.5 - 0.3j)
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, weights=0.5 + rs.rand(M), complex_input=True)
    q1 = O.block_dft(X, nfft, nov, d.w(), O.time_mean(X), method="direct")
    q2 = O.block_dft(X, nfft, nov, d.w(), O.time_mean(X), method="fft")
    assert q1.shape == (nfft, d.nb, M)
    np.testing.assert_allclose(q1, q2, rtol=0, atol=1e-13 * np.abs(q1).max())
    fit = O.spod_fit(X, d)
    tr = np.real(np.trace(fit.M, axis1=1, axis2=2)).sum()        # every bin once
    np.testing.assert_allclose(tr, O.parseval_rhs(X, d), rtol=1e-12)
    # the mean of the complex data is removed from both parts
    np.testing.assert_allclose(O.time_mean(X), X.mean(axis=0), rtol=1e-14)


def test_real_data_as_complex_reproduces_the_one_sided_fit():
    rs = np.random.RandomState(22)
    nt, M, nfft, nov = 400, 9, 32, 16
    X = rs.randn(nt, M) + 2.0
    W = 0.5 + rs.rand(M)
    dr = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, weights=W)
    dc = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, weights=W, complex_input=True)
    fr = O.spod_fit(X, dr)
    fc = O.spod_fit(X.astype(np.complex128), dc)
    nf1 = nfft // 2 + 1
    np.testing.assert_allclose(fc.lam[:nf1], fr.lam, rtol=1e-11, atol=1e-13 * fr.lam.max())
    # conjugate symmetry of real data: bin nfft - f carries the conjugate spectrum
    for f in range(1, nfft // 2):
        np.testing.assert_allclose(fc.lam[nfft - f], fc.lam[f], rtol=1e-11, atol=1e-13 * fr.lam.max())
        np.testing.assert_allclose(fc.Qhat[nfft - f], np.conj(fc.Qhat[f]), rtol=0, atol=1e-13)
    assert np.allclose(O.freqs(nfft, 0.1, True)[nfft - 1], -1.0 / (nfft * 0.1))


def test_planted_complex_exponential_sits_in_one_bin():
    # x[t, m] = a phi_m exp(+2 pi i k t / nfft), phi W-orthonormal, periodic
    # Hamming (its DFT lives on bins 0, +-1): lambda_1 = a^2 at bin k, a^2
    # (0.23/0.54)^2 at bins k +- 1, and nothing at the mirrored bin nfft - k
    rs = np.random.RandomState(23)
    nt, M, nfft, nov, k, a = 2048, 12, 64, 32, 9, 1.7
    W = 0.5 + rs.rand(M)
    phi = rs.randn(M) + 1j * rs.randn(M)
    phi /= np.sqrt(np.sum(W * np.abs(phi) ** 2))
    t = np.arange(nt)[:, None]
    X = a * phi[None, :] * np.exp(2j * np.pi * k * t / nfft)
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, window=O.WIN_HAMMING_PERIODIC, weights=W,
               subtract_mean=False, complex_input=True)
    fit = O.spod_fit(X, d, dft="fft")
    np.testing.assert_allclose(fit.lam[k, 0], a * a, rtol=1e-12)
    for kk in (k - 1, k + 1):
        np.testing.assert_allclose(fit.lam[kk, 0], a * a * (0.23 / 0.54) ** 2, rtol=1e-12)
    assert fit.lam[nfft - k].max() <= 1e-24 * a * a
    assert fit.lam[k, 1:].max() <= 1e-12 * a * a                  # rank one


# ---------------------------------------------------------------- expansion coefficients
def _coeff_case(M=6, nt=256, nfft=8, nov=4, seed=41):
    rs = np.random.RandomState(seed)
    X = rs.randn(nt, M) + 0.5
    W = 0.5 + rs.rand(M)
    d = O.Desc(nt=nt, M=M, nfft=nfft, noverlap=nov, weights=W)
    fit = O.spod_fit(X, d)
    return X, d, fit


def test_expansion_full_span_reconstructs_the_data():
    # 6 points, nfft = 8: the leading mode of bins 0 and 4 (DC, Nyquist: real)
    # and of bins 1, 2 with their conjugates give six columns spanning C^6, so
    # the oblique projection is the identity
    X, d, fit = _coeff_case()
    Phi = O.spod_modes(fit, d, 1)
    A, P, labels = O.expansion_coefficients(X, d, Phi, [0, 1, 2, 4], 1)
    assert P.shape == (6, 6) and np.linalg.cond(P) < 1e6
    Xr = O.reconstruct(A, P, fit.mu)
    np.testing.assert_allclose(Xr, X, rtol=0, atol=1e-10 * np.abs(X).max())
    assert np.abs((P @ A).imag).max() <= 1e-10 * np.abs(X).max()


def test_expansion_residual_is_w_orthogonal_and_projection_idempotent():
    X, d, fit = _coeff_case(M=20, nt=400, nfft=16, nov=8, seed=42)
    Phi = O.spod_modes(fit, d, 2)
    A, P, labels = O.expansion_coefficients(X, d, Phi, [0, 2, 5], 2)
    Xr = O.reconstruct(A, P, fit.mu)
    R = (X - Xr).T                                               # M x nt residual
    res = np.conj(P).T @ (d.W()[:, None] * R)
    assert np.abs(res).max() <= 1e-10 * np.abs(X).max()
    # projecting the reconstruction again leaves it unchanged
    A2, _, _ = O.expansion_coefficients(Xr, d, Phi, [0, 2, 5], 2, mu=fit.mu)
    np.testing.assert_allclose(A2, A, rtol=0, atol=1e-10 * np.abs(A).max())
    assert len(labels) == 2 * (1 + 2 + 2)


def test_expansion_dc_modes_are_w_orthonormal_so_coefficients_are_projections():
    # DC modes are real and W-orthonormal, and carry no conjugate: G = I and
    # A = Phi^T W (X - mu)^T
    X, d, fit = _coeff_case(M=20, nt=400, nfft=16, nov=8, seed=43)
    Phi = O.spod_modes(fit, d, 3)
    A, P, _ = O.expansion_coefficients(X, d, Phi, [0], 3)
    assert np.abs(P.imag).max() <= 1e-12
    direct = (P.real.T * d.W()[None, :]) @ (X - fit.mu[None, :]).T
    np.testing.assert_allclose(A.real, direct, rtol=0, atol=1e-10 * np.abs(direct).max())
