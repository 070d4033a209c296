"""FP64 CPU oracle of the SPOD hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline and reference legs) may import this module.  The
CUDA library never calls it, and this module never imports the CUDA path.

It is a plain, slow, obviously-correct restatement of the method of
Rogowski et al., "Unlocking massively parallel spectral proper orthogonal
decompositions in the PySPOD package" (arXiv 2309.11808), Sec. 2.2
("Practical implementation"):

* data matrix Q, real, M = M_space * M_vars rows               (Eq. data-matrix)
* temporal mean subtracted                                      (Sec. 2.2, first paragraph)
* Welch segmentation into L blocks of N_f snapshots            (Eq. blocks)
* DFT of every block in time                                   (Eq. blocks-ft)
* regrouping per frequency, Q_k in C^{M x L}                    (Eq. blocks-k)
* method-of-snapshots eigenproblem Q_k^* W Q_k Psi = Psi Lambda (Eq. spod-discrete-snapshots)
* modes Phi_k = Q_k Psi_k Lambda_k^{-1/2} (scaled, see below)   (Eq. spod-discrete-snapshots)
* one-sided spectrum for real data                              (Eq. discrete_modes)
* complex data (the paper allows complex Q, Eq. data-matrix): every bin
  f = 0 .. N_f - 1 is kept, since there is no conjugate symmetry

Readings where the paper is silent or at odds with itself:

* Gram normalisation: 1/L by default; 1/(L-1), the "Bessel" factor of
  Eq. csd-discrete, as an option.
* Mode scaling: Phi_k[:, j] = Q_k psi_j / sqrt(L * lambda_j) (or (L-1)), the
  scaling for which Phi_k^* W Phi_k = I holds, as Sec. 2.2 states after
  Eq. spod-discrete-snapshots.
* DFT: q_hat[f] = c * sum_n w_n x_n exp(-2 pi i f n / N_f), c = 1 / sum_n w_n.
* Window: symmetric Hamming by default (the paper names none).
* Number of one-sided frequencies: floor(N_f / 2) + 1 (the paper's
  ceil(N_f/2)+1 after Eq. discrete_modes is one too many for odd N_f).
* Mean over all N_t snapshots, tail samples included; blocks start at t = 0.

Eigen-decomposition: cyclic complex Jacobi, written out here (no LAPACK).
Frequencies are processed as a batch: every plane rotation (p, q) is applied
to all frequencies at once, each with its own angle.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WIN_HAMMING = "hamming"                   # symmetric
WIN_HAMMING_PERIODIC = "hamming_periodic"
WIN_HANN = "hann"                         # symmetric
WIN_RECT = "rect"

NORM_NB = "nb"
NORM_NB_MINUS_1 = "nb-1"

JACOBI_TOL = 1e-15      # stop when off(A) <= tol * ||A||_F
JACOBI_MAX_SWEEPS = 50
MODE_RANK_TOL = 1e-12   # modes with lambda_j <= tol * lambda_1 are returned as zero


# --------------------------------------------------------------------------
# Sizes (Eq. blocks; one-sided spectrum after Eq. discrete_modes)
# --------------------------------------------------------------------------
def n_blocks(nt: int, nfft: int, noverlap: int) -> int:
    """Number of Welch blocks L (Eq. blocks).

    Block l covers snapshots [l*step, l*step + nfft), step = nfft - noverlap;
    blocks start at t = 0 and a tail that does not fill a block is dropped.
    Reproduces L = 155 for 20 000 snapshots, N_f = 256, 50 % overlap (Sec. 4.1)
    and L = 8 for 727 584 snapshots, N_f = 87 600, no overlap (Sec. 4.2).
    """
    if not (0 <= noverlap < nfft <= nt):
        raise ValueError("need 0 <= noverlap < nfft <= nt")
    step = nfft - noverlap
    return (nt - noverlap) // step


def n_freqs(nfft: int, two_sided: bool = False) -> int:
    """Frequency count: floor(nfft/2) + 1 for real data (one-sided, Sec. 2.2),
    nfft for complex data (all bins; the paper allows complex Q, Eq. data-matrix)."""
    return nfft if two_sided else nfft // 2 + 1


def freqs(nfft: int, dt: float, two_sided: bool = False) -> np.ndarray:
    """Frequency of bin f of the block DFT (Eq. blocks-ft): f / (nfft * dt);
    two-sided bins f >= nfft/2 rounded up are the negative frequencies
    (f - nfft) / (nfft * dt)."""
    f = np.arange(n_freqs(nfft, two_sided))
    if two_sided:
        f = np.where(f < (nfft + 1) // 2, f, f - nfft)
    return f / (nfft * dt)


# --------------------------------------------------------------------------
# Window (not specified by the paper; reading: symmetric Hamming)
# --------------------------------------------------------------------------
def window(kind: str, nfft: int, user: np.ndarray | None = None) -> np.ndarray:
    """Window w_n of the windowed block DFT (Eq. blocks-ft).  The paper leaves
    the window open; the symmetric Hamming table is the default reading, the
    others are options."""
    n = np.arange(nfft, dtype=np.float64)
    if kind == "user":
        w = np.asarray(user, dtype=np.float64)
        if w.shape != (nfft,):
            raise ValueError("user window must have nfft entries")
        return w.copy()
    if kind == WIN_RECT or nfft == 1:
        return np.ones(nfft)
    if kind == WIN_HAMMING:
        return 0.54 - 0.46 * np.cos(2.0 * np.pi * n / (nfft - 1))
    if kind == WIN_HAMMING_PERIODIC:
        return 0.54 - 0.46 * np.cos(2.0 * np.pi * n / nfft)
    if kind == WIN_HANN:
        return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / (nfft - 1))
    raise ValueError(f"unknown window {kind!r}")


# --------------------------------------------------------------------------
# Steps of Sec. 2.2
# --------------------------------------------------------------------------
def _as_data(X: np.ndarray) -> np.ndarray:
    """X in FP64, complex128 when it is complex (Eq. data-matrix admits both)."""
    return np.asarray(X, dtype=np.complex128 if np.iscomplexobj(X) else np.float64)


def time_mean(X: np.ndarray) -> np.ndarray:
    """Temporal mean of every row of Q over all nt snapshots (Sec. 2.2).

    X is laid out [nt][M] (time-major).  FP64 pairwise summation (complex data:
    of the real and imaginary parts).
    """
    return _as_data(X).mean(axis=0)


def dft_matrix(nfft: int, two_sided: bool = False) -> np.ndarray:
    """E[f, n] = exp(-2 pi i ((f*n) mod nfft) / nfft) of Eq. blocks-ft, f one-sided
    (or all bins).

    The angle is reduced exactly in integers before the cos/sin calls.
    """
    f = np.arange(n_freqs(nfft, two_sided), dtype=np.int64)[:, None]
    n = np.arange(nfft, dtype=np.int64)[None, :]
    ang = 2.0 * np.pi * ((f * n) % nfft).astype(np.float64) / nfft
    return np.cos(ang) - 1j * np.sin(ang)


def block_dft(X: np.ndarray, nfft: int, noverlap: int, w: np.ndarray,
              mu: np.ndarray | None, method: str = "direct") -> np.ndarray:
    """Windowed DFT of every Welch block (Eqs. blocks, blocks-ft, blocks-k).

    Returns Qhat[f][l][m] = c * sum_n w_n (X[l*step+n, m] - mu_m) e^{-2 pi i f n/nfft}
    with c = 1 / sum_n w_n, for the one-sided f = 0 .. nfft//2 of real data, or
    for every bin f = 0 .. nfft-1 of complex data (no conjugate symmetry).

    method="direct": multiplication by the explicit DFT matrix (the definition).
    method="fft": numpy.fft.rfft (complex data: numpy.fft.fft) as a library
    step (used for large inputs; it is checked against "direct" by the tests).
    """
    X = _as_data(X)
    two = np.iscomplexobj(X)
    nt, M = X.shape
    nb = n_blocks(nt, nfft, noverlap)
    step = nfft - noverlap
    nf = n_freqs(nfft, two)
    c = 1.0 / w.sum()
    E = dft_matrix(nfft, two) if method == "direct" else None
    out = np.empty((nf, nb, M), dtype=np.complex128)
    for l in range(nb):
        xb = X[l * step: l * step + nfft]
        if mu is not None:
            xb = xb - mu[None, :]
        xw = w[:, None] * xb
        if method == "direct":
            out[:, l, :] = c * (E @ xw)
        elif method == "fft":
            out[:, l, :] = c * (np.fft.fft(xw, axis=0) if two else np.fft.rfft(xw, axis=0))
        else:
            raise ValueError(method)
    return out


def gram(Qhat: np.ndarray, W: np.ndarray, norm: str = NORM_NB) -> np.ndarray:
    """M_f = kappa * Qhat_f^* W Qhat_f  (Eq. spod-discrete-snapshots).

    Qhat is [nf][nb][M]; the result is [nf][nb][nb] with
    M_f[l, l'] = kappa * sum_m W_m conj(Qhat[f,l,m]) Qhat[f,l',m],
    kappa = 1/nb (default) or 1/(nb-1) (the factor of Eq. csd-discrete).
    """
    nb = Qhat.shape[1]
    kappa = 1.0 / gram_denominator(nb, norm)
    Qw = np.conj(Qhat) * W[None, None, :]
    return kappa * np.matmul(Qw, np.transpose(Qhat, (0, 2, 1)))


def gram_denominator(nb: int, norm: str) -> float:
    """1 / kappa of the cross-spectral density: nb (the default reading) or
    nb - 1 (the factor printed in Eq. csd-discrete)."""
    if norm == NORM_NB:
        return float(nb)
    if norm == NORM_NB_MINUS_1:
        if nb < 2:
            raise ValueError("nb-1 normalisation needs nb >= 2")
        return float(nb - 1)
    raise ValueError(norm)


def jacobi_eigh(A: np.ndarray, tol: float = JACOBI_TOL,
                max_sweeps: int = JACOBI_MAX_SWEEPS):
    """Cyclic complex Jacobi for a batch of Hermitian matrices A[b][n][n]: the
    eigen-decomposition of M_f in Eq. spod-discrete-snapshots.

    Row-cyclic order (p < q).  Each rotation first turns a_pq real with a
    diagonal phase, then applies the real symmetric Jacobi rotation that
    annihilates it.  Stops when every matrix has off(A) <= tol * ||A||_F.

    Returns (lam[b][n] descending, V[b][n][n] with eigenvectors in columns,
    sweeps used, converged flag).  Ties are ordered by the lower original
    diagonal index; each eigenvector has unit 2-norm and its largest-modulus
    entry (lowest index on ties) made real positive.
    """
    A = np.array(A, dtype=np.complex128, copy=True)
    B, n, _ = A.shape
    V = np.broadcast_to(np.eye(n, dtype=np.complex128), (B, n, n)).copy()
    fro = np.sqrt((np.abs(A) ** 2).sum(axis=(1, 2)))
    offmask = ~np.eye(n, dtype=bool)
    sweeps = 0
    converged = False
    for sweeps in range(1, max_sweeps + 1):
        off = _off_norm(A, offmask)
        if np.all(off <= tol * fro):
            converged = True
            sweeps -= 1
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[:, p, q]
                mag = np.abs(apq)
                app = A[:, p, p].real
                aqq = A[:, q, q].real
                # entries below 2^-60 of the diagonal scale (or subnormal) are
                # left alone: zeroing them moves no eigenvalue by a rounding unit
                act = (mag > 1e-290) & (mag > 2.0 ** -60 * (np.abs(app) + np.abs(aqq)))
                if not np.any(act):
                    continue
                safe = np.where(act, mag, 1.0)
                # phase that makes the (p, q) entry real and non-negative
                ph = np.where(act, (apq.real / safe) - 1j * (apq.imag / safe), 1.0)
                zeta = (aqq - app) / (2.0 * safe)
                t = np.where(zeta >= 0.0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                t = np.where(act, t, 0.0)
                cs = 1.0 / np.sqrt(1.0 + t * t)
                sn = t * cs
                # G = diag(1, ph) @ [[c, s], [-s, c]]
                g00 = cs.astype(np.complex128)
                g01 = sn.astype(np.complex128)
                g10 = -sn * ph
                g11 = cs * ph
                # A <- A G  (columns p, q)
                cp = A[:, :, p].copy()
                cq = A[:, :, q].copy()
                A[:, :, p] = cp * g00[:, None] + cq * g10[:, None]
                A[:, :, q] = cp * g01[:, None] + cq * g11[:, None]
                # A <- G^H A  (rows p, q)
                rp = A[:, p, :].copy()
                rq = A[:, q, :].copy()
                A[:, p, :] = np.conj(g00)[:, None] * rp + np.conj(g10)[:, None] * rq
                A[:, q, :] = np.conj(g01)[:, None] * rp + np.conj(g11)[:, None] * rq
                A[:, p, q] = np.where(act, 0.0, A[:, p, q])
                A[:, q, p] = np.where(act, 0.0, A[:, q, p])
                A[:, p, p] = A[:, p, p].real
                A[:, q, q] = A[:, q, q].real
                vp = V[:, :, p].copy()
                vq = V[:, :, q].copy()
                V[:, :, p] = vp * g00[:, None] + vq * g10[:, None]
                V[:, :, q] = vp * g01[:, None] + vq * g11[:, None]
    else:
        converged = bool(np.all(_off_norm(A, offmask) <= tol * fro))
    lam = np.diagonal(A, axis1=1, axis2=2).real.copy()
    order = np.argsort(-lam, axis=1, kind="stable")
    lam = np.take_along_axis(lam, order, axis=1)
    V = np.take_along_axis(V, order[:, None, :], axis=2)
    V = fix_phase(V)
    return lam, V, sweeps, converged


def _off_norm(A: np.ndarray, offmask: np.ndarray) -> np.ndarray:
    """Frobenius norm of the off-diagonal part, summed entry by entry (the
    stopping test of the eigen-decomposition, Eq. spod-discrete-snapshots)."""
    return np.sqrt((np.abs(A[:, offmask]) ** 2).sum(axis=1))


def fix_phase(V: np.ndarray) -> np.ndarray:
    """Unit 2-norm columns (the eigenvectors of Eq. spod-discrete-snapshots);
    the largest-|.| entry of each (lowest index on ties) made real and
    positive, a phase the paper leaves free."""
    V = V / np.sqrt((np.abs(V) ** 2).sum(axis=-2, keepdims=True))
    idx = np.argmax(np.abs(V), axis=-2)                       # [b][k]
    piv = np.take_along_axis(V, idx[..., None, :], axis=-2)    # [b][1][k]
    return V * (np.conj(piv) / np.abs(piv))


def modes(Qhat: np.ndarray, lam: np.ndarray, Psi: np.ndarray, nmodes: int,
          norm: str = NORM_NB) -> np.ndarray:
    """Phi_f[:, k] = Qhat_f psi_k / sqrt(den * lambda_k)   (Eq. spod-discrete-snapshots).

    den = nb (or nb-1), the scaling that makes Phi_f^* W Phi_f = I.  Modes whose
    eigenvalue is <= MODE_RANK_TOL * lambda_1 (or not positive) are returned as
    zero.  Output layout [nf][nmodes][M].
    """
    nf, nb, M = Qhat.shape
    den = gram_denominator(nb, norm)
    # Qhat_f (M x nb) = Qhat[f].T ; Q psi: [nf][M][k]
    QP = np.matmul(np.transpose(Qhat, (0, 2, 1)), Psi[:, :, :nmodes])
    lk = lam[:, :nmodes]
    keep = (lk > MODE_RANK_TOL * lam[:, :1]) & (lk > 0.0)
    scale = np.where(keep, 1.0 / np.sqrt(den * np.where(keep, lk, 1.0)), 0.0)
    Phi = QP * scale[:, None, :]
    return np.transpose(Phi, (0, 2, 1)).copy()


# --------------------------------------------------------------------------
# Whole fit
# --------------------------------------------------------------------------
@dataclass
class Desc:
    """Sizes and options of one SPOD (Sec. 2.2): nt snapshots of M points,
    Welch blocks of Eq. blocks, window, weights W, normalisation."""
    nt: int
    M: int
    nfft: int
    noverlap: int
    window: str = WIN_HAMMING
    user_window: np.ndarray | None = None
    weights: np.ndarray | None = None      # [M], > 0
    norm: str = NORM_NB
    subtract_mean: bool = True
    complex_input: bool = False            # two-sided spectrum, nf = nfft

    @property
    def nb(self) -> int:
        return n_blocks(self.nt, self.nfft, self.noverlap)

    @property
    def nf(self) -> int:
        return n_freqs(self.nfft, self.complex_input)

    def w(self) -> np.ndarray:
        return window(self.window, self.nfft, self.user_window)

    def W(self) -> np.ndarray:
        if self.weights is None:
            return np.ones(self.M)
        return np.asarray(self.weights, dtype=np.float64)


@dataclass
class Fit:
    """One fit: the mean, Qhat (Eq. blocks-k), M_f, eigenvalues and
    eigenvectors (Eq. spod-discrete-snapshots), Jacobi sweeps and convergence."""
    mu: np.ndarray
    Qhat: np.ndarray
    M: np.ndarray
    lam: np.ndarray
    Psi: np.ndarray
    sweeps: int
    converged: bool
    extra: dict = field(default_factory=dict)


def spod_fit(X: np.ndarray, d: Desc, dft: str = "direct") -> Fit:
    """Mean, blocks, window, DFT, Gram and eigen-decomposition (Sec. 2.2)."""
    X = _as_data(X)
    if X.shape != (d.nt, d.M):
        raise ValueError("X must be [nt][M]")
    if np.iscomplexobj(X) != d.complex_input:
        raise ValueError("complex X needs Desc(complex_input=True), real X the default")
    mu = time_mean(X) if d.subtract_mean else None
    Qhat = block_dft(X, d.nfft, d.noverlap, d.w(), mu, method=dft)
    Mf = gram(Qhat, d.W(), d.norm)
    lam, Psi, sweeps, conv = jacobi_eigh(Mf)
    return Fit(mu if mu is not None else np.zeros(d.M), Qhat, Mf, lam, Psi, sweeps, conv)


def spod_modes(fit: Fit, d: Desc, nmodes: int) -> np.ndarray:
    """The leading nmodes modes of a fit (Eq. spod-discrete-snapshots)."""
    return modes(fit.Qhat, fit.lam, fit.Psi, nmodes, d.norm)


def spod_grad(X: np.ndarray, d: Desc, dLdlam: np.ndarray, fit: Fit | None = None,
              dft: str = "direct") -> np.ndarray:
    """Gradient of L = sum_{f,k} g[f,k] lambda_{k,f} with respect to X (not in
    the paper: the adjoint of Eqs. blocks to spod-discrete-snapshots).

    For simple eigenvalues d lambda_k = psi_k^H dM_f psi_k.  With
    G_f = sum_k g[f,k] psi_k psi_k^H and R_f = 2 kappa W Qhat_f G_f (M x nb):
      dL/dxt[l*step+n, m] += c w_n Re( sum_f R_f[m, l] e^{+2 pi i f n / nfft} )
    summed over the blocks that hold snapshot t (overlap-add), over the
    one-sided f only; then the mean projection
      dL/dX[t, m] = dL/dxt[t, m] - (1/nt) sum_t' dL/dxt[t', m].
    """
    X = np.asarray(X, dtype=np.float64)
    if d.complex_input:
        raise ValueError("the gradient is defined for real data only")
    if fit is None:
        fit = spod_fit(X, d, dft=dft)
    nf, nb, M = fit.Qhat.shape
    kappa = 1.0 / gram_denominator(nb, d.norm)
    w = d.w()
    c = 1.0 / w.sum()
    step = d.nfft - d.noverlap
    g = np.asarray(dLdlam, dtype=np.float64)
    G = np.matmul(fit.Psi * g[:, None, :], np.conj(np.transpose(fit.Psi, (0, 2, 1))))
    # R_f[m, l] = 2 kappa W_m sum_l' Qhat[f,l',m] G_f[l', l]
    Qm = np.transpose(fit.Qhat, (0, 2, 1))                    # [nf][M][nb]
    R = 2.0 * kappa * d.W()[None, :, None] * np.matmul(Qm, G)  # [nf][M][nb]
    f = np.arange(nf, dtype=np.int64)[None, :]
    n = np.arange(d.nfft, dtype=np.int64)[:, None]
    ang = 2.0 * np.pi * ((f * n) % d.nfft).astype(np.float64) / d.nfft
    Einv = np.cos(ang) + 1j * np.sin(ang)                      # [nfft][nf]
    dxt = np.zeros((d.nt, M))
    for l in range(nb):
        contrib = (Einv @ R[:, :, l]).real                    # [nfft][M]
        dxt[l * step: l * step + d.nfft] += c * w[:, None] * contrib
    if d.subtract_mean:
        dxt = dxt - dxt.mean(axis=0, keepdims=True)
    return dxt


def grad_columns(xcols: np.ndarray, d: Desc, dLdlam: np.ndarray, Psi: np.ndarray, Wcols: np.ndarray,
                 mu: np.ndarray | None = None) -> np.ndarray:
    """The gradient of ``spod_grad`` restricted to a few spatial columns.

    Column m of dL/dX depends on the data only through column m itself and
    the eigenvectors Psi of the whole fit (through G_f): R_f[m, :] =
    2 kappa W_m Qhat_f[:, m]^T G_f, then the inverse one-sided DFT, window,
    overlap-add and the mean projection of that column.  ``xcols`` is X[:, cols]
    (promoted exactly to FP64), ``Wcols`` their weights, ``Psi`` [nf][nb][nb]
    the whole fit's eigenvectors; ``mu`` the columns' means (computed when
    None).  Returns dL/dX[:, cols]."""
    xc = np.asarray(xcols, dtype=np.float64)
    nf = n_freqs(d.nfft)
    Q = qhat_at_freqs(xc, d, np.arange(nf), mu)          # [nf][nb][ncols]
    nb = Q.shape[1]
    kappa = 1.0 / gram_denominator(nb, d.norm)
    w = d.w()
    c = 1.0 / w.sum()
    step = d.nfft - d.noverlap
    g = np.asarray(dLdlam, dtype=np.float64)
    G = np.matmul(Psi * g[:, None, :], np.conj(np.transpose(Psi, (0, 2, 1))))
    R = 2.0 * kappa * np.asarray(Wcols, dtype=np.float64)[None, :, None] * np.matmul(
        np.transpose(Q, (0, 2, 1)), G)                     # [nf][ncols][nb]
    f = np.arange(nf, dtype=np.int64)[None, :]
    n = np.arange(d.nfft, dtype=np.int64)[:, None]
    ang = 2.0 * np.pi * ((f * n) % d.nfft).astype(np.float64) / d.nfft
    Einv = np.cos(ang) + 1j * np.sin(ang)
    dxt = np.zeros((d.nt, xc.shape[1]))
    for l in range(nb):
        dxt[l * step: l * step + d.nfft] += c * w[:, None] * (Einv @ R[:, :, l]).real
    if d.subtract_mean:
        dxt = dxt - dxt.mean(axis=0, keepdims=True)
    return dxt


def loss_from_fit(fit: Fit, dLdlam: np.ndarray) -> float:
    """L = sum g lambda, the eigenvalue loss whose gradient spod_grad gives
    (not in the paper)."""
    return float((np.asarray(dLdlam) * fit.lam).sum())


def parseval_rhs(X: np.ndarray, d: Desc) -> float:
    """Parseval's theorem for the block DFT of Eq. blocks-ft summed as in Eq.
    csd-discrete (a pin, not a step of the method):
    (c^2 nfft / den) sum_l sum_n w_n^2 sum_m W_m |xt[l*step+n, m]|^2.

    Equals sum_f g_f tr(M_f) with g_f = 1 for f = 0 and f = nfft/2 (even nfft)
    and 2 otherwise (Parseval for each block's DFT of a real sequence); for
    complex data every g_f = 1 over all nfft bins."""
    X = _as_data(X)
    w = d.w()
    c = 1.0 / w.sum()
    step = d.nfft - d.noverlap
    xt = X - X.mean(axis=0, keepdims=True) if d.subtract_mean else X
    W = d.W()
    tot = 0.0
    for l in range(d.nb):
        blk = xt[l * step: l * step + d.nfft]
        tot += float(((w ** 2)[:, None] * np.abs(blk) ** 2 * W[None, :]).sum())
    return c * c * d.nfft / gram_denominator(d.nb, d.norm) * tot


def one_sided_multiplicity(nfft: int) -> np.ndarray:
    """How often each one-sided bin (after Eq. discrete_modes) stands for itself
    in the full spectrum of real data: 1 for DC and Nyquist, 2 otherwise."""
    g = np.full(n_freqs(nfft), 2.0)
    g[0] = 1.0
    if nfft % 2 == 0:
        g[-1] = 1.0
    return g


def qhat_at_freqs(xcols: np.ndarray, d: Desc, fsel, mu: np.ndarray | None = None) -> np.ndarray:
    """Qhat[f][l][j] (Eqs. blocks-ft, blocks-k) of a few spatial columns at the
    selected one-sided bins only, from the rows of the DFT matrix for those
    bins (the plain definition of Eq. blocks-ft restricted to f in ``fsel``).

    ``xcols`` is X[:, cols] (promoted exactly to FP64); ``mu`` their temporal
    means over all nt snapshots (computed here when None and the descriptor
    subtracts the mean).  Returns [len(fsel)][nb][ncols] complex."""
    fsel = np.asarray(fsel, dtype=np.int64)
    xc = np.asarray(xcols, dtype=np.float64)
    if xc.ndim == 1:
        xc = xc[:, None]
    if d.subtract_mean:
        xc = xc - (time_mean(xc) if mu is None else np.asarray(mu, dtype=np.float64))[None, :]
    w = d.w()
    c = 1.0 / w.sum()
    E = dft_matrix(d.nfft)[fsel]                      # [F][nfft]
    step = d.nfft - d.noverlap
    Q = np.empty((len(fsel), d.nb, xc.shape[1]), dtype=np.complex128)
    for l in range(d.nb):
        Q[:, l, :] = c * (E @ (w[:, None] * xc[l * step: l * step + d.nfft]))
    return Q


def modes_at(Q: np.ndarray, lam: np.ndarray, Psi: np.ndarray, nmodes: int, norm: str, nb: int) -> np.ndarray:
    """Modes of Eq. spod-discrete-snapshots restricted to the columns whose
    Qhat is given: Phi[f][k][j] = sum_l Q[f][l][j] Psi[f][l][k] / sqrt(den * lambda_k)
    with den the Gram denominator (the scaling for which Phi^* W Phi = I over
    the whole grid), zero where lambda_k <= MODE_RANK_TOL * lambda_1.  Q, lam and
    Psi are those of the same selected bins."""
    den = gram_denominator(nb, norm)
    out = np.zeros((Q.shape[0], nmodes, Q.shape[2]), dtype=np.complex128)
    for i in range(Q.shape[0]):
        for k in range(nmodes):
            if lam[i, k] > MODE_RANK_TOL * lam[i, 0] and lam[i, k] > 0:
                out[i, k] = (Q[i].T @ Psi[i][:, k]) / np.sqrt(den * lam[i, k])
    return out


def gram_at_freqs(d: Desc, fsel, get_chunk, chunk: int) -> np.ndarray:
    """M_f (Eq. spod-discrete-snapshots) at the selected one-sided bins only.

    For grids too large for a full FP64 transform: X is visited in spatial
    chunks (``get_chunk(m0, m1)`` returns X[:, m0:m1], promoted exactly to
    FP64); each chunk's columns get their own temporal mean over all nt
    snapshots (a column's mean depends on that column alone), and Qhat is
    formed from the rows of the DFT matrix for the bins in ``fsel`` (the plain
    definition of Eq. blocks-ft restricted to those f).  Returns [len(fsel)][nb][nb].
    """
    fsel = np.asarray(fsel, dtype=np.int64)
    W = d.W()
    w = d.w()
    c = 1.0 / w.sum()
    E = dft_matrix(d.nfft)[fsel]                      # [F][nfft]
    Er, Ei = np.ascontiguousarray(E.real), np.ascontiguousarray(E.imag)
    step = d.nfft - d.noverlap
    acc = np.zeros((len(fsel), d.nb, d.nb), dtype=np.complex128)
    for m0 in range(0, d.M, chunk):
        m1 = min(d.M, m0 + chunk)
        xc = np.asarray(get_chunk(m0, m1), dtype=np.float64)
        if d.subtract_mean:
            xc = xc - time_mean(xc)[None, :]
        Q = np.empty((len(fsel), d.nb, m1 - m0), dtype=np.complex128)
        for l in range(d.nb):
            xw = w[:, None] * xc[l * step: l * step + d.nfft]
            Q[:, l, :] = c * (Er @ xw + 1j * (Ei @ xw))
        Qw = np.conj(Q) * W[None, None, m0:m1]
        acc += np.matmul(Qw, np.transpose(Q, (0, 2, 1)))
    return acc / gram_denominator(d.nb, d.norm)


# --------------------------------------------------------------------------
# Expansion coefficients and reconstruction (SPOD for data compression,
# Eqs. coeffs and SPODrec)
# --------------------------------------------------------------------------
def is_self_conjugate_bin(f: int, nfft: int) -> bool:
    """DC and (even nfft) Nyquist: the one-sided bins of real data whose DFT is
    real, which have no separate conjugate bin in Eq. coeffs."""
    return f == 0 or (nfft % 2 == 0 and f == nfft // 2)


def coeff_basis(Phi: np.ndarray, fsel, nmodes_r: int, nfft: int) -> tuple[np.ndarray, list]:
    """Columns of Phi_r of Eq. coeffs for real data: the leading nmodes_r modes of every
    selected one-sided bin and, for the bins other than DC and Nyquist, their
    complex conjugates (the modes of the negative frequency -f, so that the
    two-sided set is closed under conjugation and the reconstruction of real
    data is real).  Returns P [M][K] and the (bin, mode, conjugated) labels."""
    cols, labels = [], []
    for f in fsel:
        for k in range(nmodes_r):
            cols.append(Phi[f, k])
            labels.append((f, k, False))
            if not is_self_conjugate_bin(f, nfft):
                cols.append(np.conj(Phi[f, k]))
                labels.append((f, k, True))
    return np.stack(cols, axis=1), labels


def expansion_coefficients(X: np.ndarray, d: Desc, Phi: np.ndarray, fsel, nmodes_r: int,
                           mu: np.ndarray | None = None):
    """A = (Phi_r^* W Phi_r)^{-1} Phi_r^* W Q  (Eq. coeffs), Q = X^T - mu (M x nt).

    Returns (A [K][nt] complex, P [M][K], labels).  The solve is a plain dense
    one of the Hermitian positive definite K x K system."""
    X = np.asarray(X, dtype=np.float64)
    if mu is None:
        mu = time_mean(X) if d.subtract_mean else np.zeros(d.M)
    P, labels = coeff_basis(Phi, fsel, nmodes_r, d.nfft)
    W = d.W()
    PW = np.conj(P).T * W[None, :]                  # Phi_r^* W  [K][M]
    G = PW @ P
    A = np.linalg.solve(G, PW @ (X - mu[None, :]).T)
    return A, P, labels


def reconstruct(A: np.ndarray, P: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Q~ = Phi_r A_r  (Eq. SPODrec), as data [nt][M]: Re(P A)^T + mu (the
    imaginary part vanishes for a conjugation-closed set of modes)."""
    return (P @ A).real.T + mu[None, :]
