"""Out-of-core run (spod_run_host_ooc): X and Phi in pinned host memory,
gathered and scattered in column tiles; compared with the device-resident
fit + modes of the same plan (same spatial chunks, hence the same arithmetic)
and with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import jet_like

pytestmark = pytest.mark.gpu

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


from paper_2309_11808_gb300 import SPOD, SpodError, _lib  # noqa: E402

DEV = "cuda:0"


def _pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype, pin_memory=True)


def _ooc_vs_device(X, npts, nvars, nfft, prec, nmodes, tile, W=None):
    nt, M = X.shape
    sp = SPOD(npts, nvars, nt, nfft, nfft // 2, dtype=X.dtype, precision=prec, weights=W, chunk_points=tile)
    Xd = X.to(DEV).contiguous()
    sp.fit(Xd)
    lam = sp.eigs()
    Phi = sp.modes(Xd, nmodes).cpu() if nmodes else None
    torch.cuda.synchronize()
    hX = _pinned(X.shape, X.dtype)
    hX.copy_(X)
    cdt = torch.complex128 if prec == "fp64" else torch.complex64
    hPhi = _pinned((sp.nf, nmodes, M), cdt) if nmodes else None
    hlam = np.empty_like(lam)
    _lib.spod_run_host_ooc(sp.handle, hX, nmodes, hPhi, hlam, tile)
    sp.close()
    return lam, Phi, hlam, hPhi


@cuda
@pytest.mark.parametrize("prec,nfft", [("fp32", 64), ("fp64", 64), ("bf16x3", 64), ("bf16x3", 256), ("fp32", 256)])
def test_ooc_equals_device_path(prec, nfft):
    wl = jet_like(nx=20, nr=10, nvars=2, nt=4 * nfft, nfft=nfft, seed=41,
                  dtype=torch.float64 if prec == "fp64" else torch.float32)
    # 400 points in tiles of 128: three full tiles and a ragged one of 16
    lam, Phi, hlam, hPhi = _ooc_vs_device(wl.X, wl.npoints, 2, nfft, prec, 3, 128, W=wl.W.numpy())
    assert np.array_equal(hlam, lam)
    assert torch.equal(hPhi, Phi)


@cuda
def test_ooc_against_oracle_and_without_modes():
    wl = jet_like(nx=24, nr=12, nvars=3, nt=700, nfft=64, seed=42, dtype=torch.float32)
    nt, M = wl.X.shape
    d = O.Desc(nt=nt, M=M, nfft=64, noverlap=32, window=O.WIN_HAMMING, weights=wl.W.numpy().astype(np.float64))
    ref = O.spod_fit(wl.X.double().numpy(), d)
    sp = SPOD(wl.npoints, 3, nt, 64, 32, weights=wl.W, precision="fp32")
    hX = _pinned(wl.X.shape, torch.float32)
    hX.copy_(wl.X)
    hlam = np.empty((sp.nf, sp.nb))
    for tile in (0, 64, 320, M):     # automatic, many tiles, ragged, a single tile
        hlam[:] = np.nan
        _lib.spod_run_host_ooc(sp.handle, hX, 0, None, hlam, tile)
        rel = np.abs(hlam[:, :5] - ref.lam[:, :5]) / ref.lam[:, :5]
        assert rel.max() <= 1e-4, (tile, rel.max())
    sp.close()


@cuda
def test_ooc_complex_input():
    g = torch.Generator().manual_seed(43)
    nt, M, nfft = 512, 300, 64
    X = torch.complex(torch.randn(nt, M, generator=g), torch.randn(nt, M, generator=g))
    lam, Phi, hlam, hPhi = _ooc_vs_device(X, M, 1, nfft, "fp32", 2, 128)
    assert np.array_equal(hlam, lam)
    assert torch.equal(hPhi, Phi)


@cuda
def test_ooc_argument_checks():
    sp = SPOD(128, 1, 256, 32, 16)
    g = torch.Generator().manual_seed(44)
    hX = _pinned((256, 128), torch.float32)
    hX.copy_(torch.randn(256, 128, generator=g))
    Phi = _pinned((sp.nf, 2, 128), torch.complex64)
    lam = np.empty((sp.nf, sp.nb))
    _lib.spod_run_host_ooc(sp.handle, hX, 2, Phi, lam, 64)
    # pageable memory: refused, unless the device reads pageable memory
    # through the host's page tables -- then the results are the same
    X = hX.numpy().copy()
    P2 = np.zeros((sp.nf, 2, 128), dtype=np.complex64)
    l2 = np.empty_like(lam)
    try:
        _lib.spod_run_host_ooc(sp.handle, X, 2, P2, l2, 64)
    except SpodError as e:
        assert e.status == _lib.SPOD_EINVAL
    else:
        assert np.array_equal(l2, lam) and np.array_equal(P2, Phi.numpy())
    with pytest.raises(SpodError) as e:
        _lib.spod_run_host_ooc(sp.handle, hX, 2, Phi, None, -1)
    assert e.value.status == _lib.SPOD_EINVAL
    with pytest.raises(SpodError) as e:
        _lib.spod_run_host_ooc(sp.handle, hX, sp.nb + 1, Phi, None, 0)
    assert e.value.status == _lib.SPOD_EINVAL
    sp.close()
