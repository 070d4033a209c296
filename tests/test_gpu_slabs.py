"""The paper's spatial decomposition (Sec. 3.1) through the library, on one GPU.

Two plans over two column slabs of one grid each run spod_fit_partial; their
slab Grams, stacked in slab order, go to spod_fit_from_grams on both plans
(the one reduction of the decomposition and the redundant eigen-solve).  The
eigenvalues must be bit-identical on both plans and equal to the whole-grid
fit, and each slab's modes and gradient must be the whole-grid modes and
gradient restricted to its columns.
"""
import numpy as np
import pytest
import torch

from workloads import jet_like

pytestmark = pytest.mark.gpu

cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _whole_and_slabs(prec, nfft, bounds, nmodes=4):
    from paper_2309_11808_gb300 import SPOD, _lib
    dt = torch.float64 if prec == "fp64" else torch.float32
    nt = 4 * nfft
    wl = jet_like(nx=24, nr=16, nvars=2, nt=nt, nfft=nfft, seed=41, dtype=dt)
    X = wl.X.to(DEV)
    W = wl.W.numpy()
    M = X.shape[1]
    st = torch.cuda.current_stream()
    sp = SPOD(M, 1, nt, nfft, nfft // 2, dtype=dt, precision=prec, weights=W)
    sp.fit(X)
    lam, psi = sp.eigs(vectors=True)
    Phi = sp.modes(X, nmodes)
    gl = torch.zeros((sp.nf, sp.nb), dtype=torch.float64, device=DEV)
    gl[:, :2] = 1.0
    dX = torch.empty(X.shape, dtype=dt, device=DEV)
    _lib.spod_backward(sp.handle, gl, X, dX, st)
    whole = dict(lam=lam, Phi=Phi.cpu().numpy(), dX=dX.cpu().numpy(), nf=sp.nf, nb=sp.nb)
    sp.close()
    plans, parts, xs = [], [], []
    for a, b in zip(bounds[:-1], bounds[1:]):
        xr = X[:, a:b].contiguous()
        pr = SPOD(b - a, 1, nt, nfft, nfft // 2, dtype=dt, precision=prec, weights=W[a:b])
        g = torch.empty((pr.nf, pr.nb, pr.nb, 2), dtype=torch.float64, device=DEV)
        _lib.spod_fit_partial(pr.handle, xr, g, st)
        plans.append(pr)
        parts.append(g)
        xs.append(xr)
    grams = torch.stack(parts).contiguous()
    out = []
    for pr, xr in zip(plans, xs):
        _lib.spod_fit_from_grams(pr.handle, grams, len(parts), st)
        lam_r = pr.eigs()
        Phi_r = pr.modes(xr, nmodes).cpu().numpy()
        dX_r = torch.empty(xr.shape, dtype=dt, device=DEV)
        _lib.spod_backward(pr.handle, gl, xr, dX_r, st)
        out.append(dict(lam=lam_r, Phi=Phi_r, dX=dX_r.cpu().numpy()))
        pr.close()
    return whole, out


@cuda
@pytest.mark.parametrize("prec,nfft,tol_lam,tol_vec", [("fp64", 64, 1e-11, 1e-9), ("fp32", 256, 1e-5, 1e-4),
                                                        ("bf16x3", 256, 1e-5, 1e-4)])
def test_two_slab_plans_reproduce_the_whole_grid(prec, nfft, tol_lam, tol_vec):
    bounds = [0, 320, 768]                       # uneven slabs of the 768 columns
    whole, slabs = _whole_and_slabs(prec, nfft, bounds)
    # the same parts summed in the same order: bit-identical on every slab
    for r in slabs[1:]:
        assert np.array_equal(r["lam"], slabs[0]["lam"])
    lam, lr = whole["lam"], slabs[0]["lam"]
    keep = lam > 1e-10 * lam[:, :1]
    assert (np.abs(lr - lam)[keep] / lam[keep]).max() <= tol_lam
    # modes and gradient of each slab are the whole grid's, restricted to its columns
    Phi = np.concatenate([r["Phi"] for r in slabs], axis=2)
    dX = np.concatenate([r["dX"] for r in slabs], axis=1)
    gap = np.abs(lam[:, :4] - lam[:, 1:5]) / lam[:, :4]
    gap = np.minimum(gap, np.concatenate([np.full((lam.shape[0], 1), np.inf),
                                          np.abs(lam[:, 1:4] - lam[:, :3]) / lam[:, 1:4]], axis=1))
    ok = (gap >= 1e-2) & (lam[:, :4] > 1e-8 * lam[:, :1])
    err = np.linalg.norm(Phi - whole["Phi"], axis=2) / np.linalg.norm(whole["Phi"], axis=2)
    assert err[ok].max() <= tol_vec
    gerr = np.linalg.norm(dX - whole["dX"]) / np.linalg.norm(whole["dX"])
    assert gerr <= tol_vec


@cuda
def test_slab_entries_check_call_order_and_arguments():
    from paper_2309_11808_gb300 import SPOD, SpodError, _lib
    sp = SPOD(256, 1, 512, 64, 32, precision="fp32")
    g = torch.zeros((sp.nf, sp.nb, sp.nb, 2), dtype=torch.float64, device=DEV)
    with pytest.raises(SpodError) as e:
        _lib.spod_fit_from_grams(sp.handle, g, 1)
    assert e.value.status == _lib.SPOD_ESTATE
    X = torch.randn(512, 256, device=DEV)
    _lib.spod_fit_partial(sp.handle, X, g)
    with pytest.raises(SpodError) as e:
        _lib.spod_fit_from_grams(sp.handle, g, 0)
    assert e.value.status == _lib.SPOD_EINVAL
    with pytest.raises(SpodError) as e:           # a partial fit is not a fit
        sp.eigs()
    assert e.value.status == _lib.SPOD_ESTATE
    _lib.spod_fit_from_grams(sp.handle, g, 1)
    assert np.all(np.isfinite(sp.eigs()))
    sp.close()
