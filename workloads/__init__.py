"""Seeded synthetic snapshot generators shared by the tests and ``bench.py``.

This module holds no SPOD arithmetic: it only builds input matrices X[nt][M]
(time-major, M = nvars * npoints, variable-major within a snapshot) and
positive quadrature weights W[M].  The structures stand in for the paper's two
workloads (Sec. 4): a twin-jet LES field (travelling wave packets on an (x, r)
grid, red noise) and ERA5-like lat-lon fields (AR(1) red noise with planted
low-frequency and diurnal patterns, cos(latitude) weights).

Everything is generated with torch on the requested device from explicit seeds,
so the same call gives the same values on every run of the same machine type.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

__all__ = ["Workload", "planted", "jet_like", "diff_like", "geo_like", "geo_datasets",
           "ar1_", "w_orthonormal_modes"]


@dataclass
class Workload:
    """Generated input: X [nt][M], W [M] (float64, CPU) and what was planted."""
    X: torch.Tensor
    W: torch.Tensor
    npoints: int
    nvars: int
    nt: int
    nfft: int
    noverlap: int
    meta: dict

    @property
    def M(self) -> int:
        return self.npoints * self.nvars


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def w_orthonormal_modes(M: int, J: int, W: torch.Tensor, seed: int) -> torch.Tensor:
    """J columns phi_j with phi^T diag(W) phi = I (float64, CPU).

    QR of a seeded Gaussian M x J matrix gives orthonormal columns Q; then
    phi = W^{-1/2} Q.
    """
    g = _gen(seed, "cpu")
    G = torch.randn(M, J, generator=g, dtype=torch.float64)
    Q, _ = torch.linalg.qr(G)
    return Q / torch.sqrt(W.to(torch.float64))[:, None]


def ar1_(X: torch.Tensor, phi: float, sigma: float, seed: int, chunk: int = 256) -> torch.Tensor:
    """Add AR(1) red noise in place: e_t = phi e_{t-1} + sigma n_t, n_t ~ N(0, 1),
    started from the stationary distribution N(0, sigma^2 / (1 - phi^2)).
    Independent per column of X[nt][M]."""
    nt, M = X.shape
    g = _gen(seed, X.device)
    prev = torch.randn(M, generator=g, device=X.device, dtype=torch.float32)
    prev.mul_(sigma / math.sqrt(1.0 - phi * phi))
    for t0 in range(0, nt, chunk):
        t1 = min(nt, t0 + chunk)
        eps = torch.randn(t1 - t0, M, generator=g, device=X.device, dtype=torch.float32)
        eps.mul_(sigma)
        for i in range(t1 - t0):
            prev.mul_(phi).add_(eps[i])
            X[t0 + i].add_(prev.to(X.dtype))
    return X


def planted(npoints: int, nvars: int, nt: int, nfft: int, noverlap: int,
            bins=(10, 25, 60), amps=(3.0, 2.0, 1.0), noise_std: float = 0.1,
            weights: torch.Tensor | None = None, seed: int = 0,
            dtype=torch.float64, device="cpu", offset: torch.Tensor | None = None) -> Workload:
    """Orthonormal spatial modes times bin-centred sinusoids plus white noise.

    X[t, m] = sum_j a_j phi_j[m] sin(2 pi k_j t / nfft + theta_j) + noise + offset[m],
    with phi W-orthonormal, theta_j seeded.  (The small FP64 correctness
    workload: a 64 x 32 grid, one variable, nt = 2048, nfft = 256.)
    """
    M = npoints * nvars
    W = torch.ones(M, dtype=torch.float64) if weights is None else weights.to(torch.float64).cpu()
    J = len(bins)
    phi = w_orthonormal_modes(M, J, W, seed + 1)
    g = _gen(seed + 2, "cpu")
    theta = torch.rand(J, generator=g, dtype=torch.float64) * 2 * math.pi
    t = torch.arange(nt, dtype=torch.float64)
    T = torch.stack([amps[j] * torch.sin(2 * math.pi * bins[j] * t / nfft + theta[j])
                     for j in range(J)], dim=1)                     # [nt][J]
    X = (T @ phi.T)                                                 # [nt][M] float64
    if noise_std > 0:
        gn = _gen(seed + 3, "cpu")
        X += noise_std * torch.randn(nt, M, generator=gn, dtype=torch.float64)
    if offset is not None:
        X += offset.to(torch.float64)[None, :]
    X = X.to(dtype).to(device)
    return Workload(X, W, npoints, nvars, nt, nfft, noverlap,
                    dict(phi=phi, theta=theta, bins=tuple(bins), amps=tuple(amps)))


def _rank_update_(X: torch.Tensor, T: torch.Tensor, S: torch.Tensor, chunk: int = 512) -> None:
    """X += T @ S in row chunks (T [nt][K], S [K][M] on X's device, float32 math)."""
    nt = X.shape[0]
    for t0 in range(0, nt, chunk):
        t1 = min(nt, t0 + chunk)
        X[t0:t1] += (T[t0:t1] @ S).to(X.dtype)


def jet_like(nx: int = 512, nr: int = 256, nvars: int = 3, nt: int = 10000, nfft: int = 512,
             noverlap: int | None = None, seed: int = 0, dtype=torch.float32, device="cpu",
             ar_phi: float = 0.9, ar_sigma: float = 0.2) -> Workload:
    """Twin-jet-shaped field on an (x, r) grid (stand-in for the LES data of Sec. 4.1).

    Four travelling Gaussian wave packets
      A_j exp(-(x-x_j)^2/2sx^2 - (r-r_j)^2/2sr^2) cos(kappa_j x - 2 pi k_j t/nfft + theta_j)
    at bins k = 12, 40, 90, 150 (scaled for other nfft), amplitudes 2, 1.5, 1, 0.5,
    per-variable factors (1, 0.5, 0.3), plus AR(1) red noise (phi 0.9, sigma 0.2)
    independent per (variable, point).  Weights W ~ r (cell volume of an
    axisymmetric grid) times a seeded factor in [0.9, 1.1].
    Layout: m = v * (nx*nr) + ix * nr + ir.
    """
    if noverlap is None:
        noverlap = nfft // 2
    npts = nx * nr
    M = npts * nvars
    g = _gen(seed, "cpu")
    x = (torch.arange(nx, dtype=torch.float64) + 0.5) / nx * 20.0      # x in (0, 20)
    r = (torch.arange(nr, dtype=torch.float64) + 0.5) / nr              # r in (0, 1)
    dx, dr = 20.0 / nx, 1.0 / nr
    wpt = (r[None, :] * dx * dr).expand(nx, nr).reshape(-1)
    wpt = wpt * (1.0 + 0.1 * (2 * torch.rand(npts, generator=g, dtype=torch.float64) - 1))
    W = wpt.repeat(nvars)
    scale = nfft / 512.0
    bins = [max(1, min(nfft // 2 - 1, int(round(k * scale)))) for k in (12, 40, 90, 150)]
    amps = [2.0, 1.5, 1.0, 0.5]
    xc = [4.0, 8.0, 12.0, 16.0]
    rc = [0.25, 0.5, 0.35, 0.6]
    sx, sr = 2.0, 0.12
    vfac = [1.0, 0.5, 0.3] + [0.2] * max(0, nvars - 3)
    kap = [1.5, 2.5, 4.0, 6.0]
    theta = torch.rand(4, generator=g, dtype=torch.float64) * 2 * math.pi
    t = torch.arange(nt, dtype=torch.float64)
    Tcols, Srows = [], []
    for j in range(4):
        env = amps[j] * torch.exp(-(x[:, None] - xc[j]) ** 2 / (2 * sx * sx)
                                  - (r[None, :] - rc[j]) ** 2 / (2 * sr * sr))
        ph = kap[j] * x[:, None] + theta[j]
        a = (env * torch.cos(ph)).reshape(-1)
        b = (env * torch.sin(ph)).reshape(-1)
        om = 2 * math.pi * bins[j] * t / nfft
        # cos(ph - om) = cos(ph) cos(om) + sin(ph) sin(om)
        Tcols += [torch.cos(om), torch.sin(om)]
        Srows += [torch.cat([vfac[v] * a for v in range(nvars)]),
                  torch.cat([vfac[v] * b for v in range(nvars)])]
    T = torch.stack(Tcols, 1).to(torch.float32).to(device)
    S = torch.stack(Srows, 0).to(torch.float32).to(device)
    X = torch.zeros(nt, M, dtype=torch.float32, device=device)
    _rank_update_(X, T, S)
    ar1_(X, ar_phi, ar_sigma, seed + 7)
    X = X.to(dtype)
    return Workload(X, W, npts, nvars, nt, nfft, noverlap,
                    dict(bins=bins, amps=amps, kind="jet"))


def diff_like(nx: int = 256, ny: int = 128, nvars: int = 2, nt: int = 4096, nfft: int = 256,
              noverlap: int | None = None, seed: int = 0, dtype=torch.float32, device="cpu",
              noise_std: float = 0.05) -> Workload:
    """Planted spectra for the differentiation workload (256 x 128 grid, 2 variables).

    At every bin k in 5..40 two W-orthonormal spatial patterns are planted with
    independent sinusoids whose amplitudes differ by 25 %, so that the leading
    eigenvalues there are separated by well over 5 %; plus white noise.
    W = cos(latitude) with the 128 rows mapped to (-80, 80) degrees.
    """
    if noverlap is None:
        noverlap = nfft // 2
    npts = nx * ny
    M = npts * nvars
    lat = torch.linspace(-80.0, 80.0, ny, dtype=torch.float64) * math.pi / 180.0
    W = torch.cos(lat)[None, :].expand(nx, ny).reshape(-1).repeat(nvars)
    bins = list(range(5, 41))
    J = 2 * len(bins)
    phi = w_orthonormal_modes(M, J, W, seed + 11)
    g = _gen(seed + 12, "cpu")
    theta = torch.rand(J, generator=g, dtype=torch.float64) * 2 * math.pi
    t = torch.arange(nt, dtype=torch.float64)
    cols = []
    for i, k in enumerate(bins):
        a1 = 1.0 + 0.5 * math.cos(0.3 * i)
        for s, a in enumerate((a1, 0.75 * a1)):
            # a slightly detuned second tone so the two patterns are not coherent
            kk = k + (0.0 if s == 0 else 0.37)
            cols.append(a * torch.sin(2 * math.pi * kk * t / nfft + theta[2 * i + s]))
    T = torch.stack(cols, 1).to(device, torch.float32)
    S = phi.T.contiguous().to(device, torch.float32)
    X = torch.zeros(nt, M, dtype=torch.float32, device=device)
    _rank_update_(X, T, S)
    if noise_std > 0:
        gn = _gen(seed + 13, device)
        for t0 in range(0, nt, 512):
            t1 = min(nt, t0 + 512)
            X[t0:t1] += noise_std * torch.randn(t1 - t0, M, generator=gn, device=device)
    X = X.to(dtype)
    return Workload(X, W, npts, nvars, nt, nfft, noverlap, dict(bins=bins, kind="diff"))


def geo_like(nlat: int, nlon: int, nt: int, nfft: int, nvars: int = 2, noverlap: int | None = None,
             seed: int = 0, dtype=torch.float32, device="cpu",
             ar_phi: float = 0.95, ar_sigma: float = 0.1) -> Workload:
    """ERA5-shaped lat-lon field (stand-in for the reanalysis data of Sec. 4.2).

    AR(1) red noise (phi 0.95, sigma 0.1) plus a planted low-frequency pattern at
    bin 1 and a "diurnal" pattern at the bin nearest nfft * dt / 24 h, where a
    one-year record gives dt = 8760 h / nt.  W = cos(latitude).
    Layout: m = v * (nlat*nlon) + ilat * nlon + ilon.
    """
    if noverlap is None:
        noverlap = nfft // 2
    npts = nlat * nlon
    M = npts * nvars
    lat = torch.linspace(-90.0, 90.0, nlat, dtype=torch.float64) * math.pi / 180.0
    lon = torch.linspace(0.0, 2 * math.pi, nlon + 1, dtype=torch.float64)[:-1]
    wlat = torch.cos(lat).clamp_min(1e-3)
    W = wlat[:, None].expand(nlat, nlon).reshape(-1).repeat(nvars)
    dt_h = 8760.0 / nt
    kd = max(1, min(nfft // 2 - 1, int(round(nfft * dt_h / 24.0))))
    g = _gen(seed, "cpu")
    theta = torch.rand(2, generator=g, dtype=torch.float64) * 2 * math.pi
    pat1 = (torch.exp(-(lat[:, None] / 0.35) ** 2) * torch.ones_like(lon)[None, :]).reshape(-1)
    pat2 = (torch.cos(lat[:, None]) * torch.cos(lon[None, :])).reshape(-1)
    pat2b = (torch.cos(lat[:, None]) * torch.sin(lon[None, :])).reshape(-1)
    t = torch.arange(nt, dtype=torch.float64)
    o1 = 2 * math.pi * 1 * t / nfft + theta[0]
    o2 = 2 * math.pi * kd * t / nfft + theta[1]
    T = torch.stack([0.5 * torch.sin(o1), 0.3 * torch.cos(o2), 0.3 * torch.sin(o2)], 1)
    S = torch.stack([pat1.repeat(nvars), pat2.repeat(nvars), pat2b.repeat(nvars)], 0)
    X = torch.zeros(nt, M, dtype=torch.float32, device=device)
    _rank_update_(X, T.to(device, torch.float32), S.to(device, torch.float32))
    ar1_(X, ar_phi, ar_sigma, seed + 5)
    X = X.to(dtype)
    return Workload(X, W, npts, nvars, nt, nfft, noverlap, dict(diurnal_bin=kd, kind="geo"))


def geo_datasets():
    """The six (grid, nt, nfft) combinations of the batched ERA5-like workload:
    one-year records on 1, 0.5 and 0.25 degree grids."""
    return [((181, 360), 2920, 256), ((361, 720), 4380, 384), ((361, 720), 8760, 512),
            ((721, 1440), 2920, 720), ((721, 1440), 4380, 256), ((721, 1440), 8760, 720)]
