"""The allocation-free eigen-solver entry point against the regular path.

spod_eigh_batched_noalloc serves callers that cannot call cudaMalloc (a host
framework that owns all device memory, real-time loops, programs that reserve
their memory up front): its scratch is a fixed array inside the library.  Here
it must reproduce the eigenvalues and eigenvectors that spod_fit /
spod_get_eigs give for the same Gram matrices, on two calls in a row (the
array keeps the previous call's contents), both below and above the nb at
which the solver moves its working copies from shared memory to that array.
This file is collected last so that a run stopping at the first failure has
run every other test before it.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
cuda = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _regular_path(npts, nt, nfft, nov, seed):
    from paper_2309_11808_gb300 import SPOD
    g = torch.Generator().manual_seed(seed)
    X = torch.randn(nt, npts, generator=g, dtype=torch.float64).to(DEV)
    sp = SPOD(npts, 1, nt, nfft, nov, dtype=torch.float64, precision="fp64")
    sp.fit(X)
    lam, psi = sp.eigs(vectors=True)
    gram = sp.gram()
    nf, nb = sp.nf, sp.nb
    sp.close()
    return gram, lam, psi, nf, nb


@cuda
@pytest.mark.parametrize("npts,nt,nfft,nov,seed", [(300, 400, 32, 16, 1),     # nb = 24: shared-memory solver
                                                   (120, 200, 4, 2, 2)])      # nb = 99: scratch-array solver
def test_noalloc_matches_regular_path_twice(npts, nt, nfft, nov, seed):
    from paper_2309_11808_gb300 import _lib
    gram, lam_ref, psi_ref, nf, nb = _regular_path(npts, nt, nfft, nov, seed)
    d_gram = torch.from_numpy(gram.view(np.float64).copy()).to(DEV)
    for call in range(2):
        d_lam = torch.full((nf, nb), float("nan"), dtype=torch.float64, device=DEV)
        d_psi = torch.full((nf, nb, nb, 2), float("nan"), dtype=torch.float64, device=DEV)
        _lib.spod_eigh_batched_noalloc(d_gram, nf, nb, d_lam, d_psi, torch.cuda.current_stream())
        lam = d_lam.cpu().numpy()
        psi = d_psi.cpu().numpy().view(np.complex128)[..., 0]
        scale = np.abs(lam_ref).max()
        np.testing.assert_allclose(lam, lam_ref, rtol=1e-10, atol=1e-13 * scale, err_msg=f"call {call}")
        # compare eigenvectors where the eigenvalue is simple and not in the null space
        for f in range(nf):
            for k in range(nb):
                lk = lam_ref[f, k]
                if lk <= 1e-8 * lam_ref[f, 0]:
                    continue
                gaps = [abs(lk - lam_ref[f, j]) for j in (k - 1, k + 1) if 0 <= j < nb]
                if gaps and min(gaps) < 1e-2 * lk:
                    continue
                ip = abs(np.vdot(psi_ref[f, :, k], psi[f, :, k]))
                assert 1.0 - ip <= 1e-10, (call, f, k, ip)


@cuda
def test_noalloc_near_the_capacity_of_the_array():
    # nb = 256 (the largest block count a plan takes) at nf = 13: the working
    # copies fill 13 * 32 * 256^2 bytes = 27.3 MB of the 32 MiB array
    from paper_2309_11808_gb300 import _lib
    gram, lam_ref, psi_ref, nf, nb = _regular_path(300, 3084, 24, 12, 3)
    assert (nf, nb) == (13, 256)
    d_gram = torch.from_numpy(gram.view(np.float64).copy()).to(DEV)
    for call in range(2):
        d_lam = torch.full((nf, nb), float("nan"), dtype=torch.float64, device=DEV)
        d_psi = torch.full((nf, nb, nb, 2), float("nan"), dtype=torch.float64, device=DEV)
        _lib.spod_eigh_batched_noalloc(d_gram, nf, nb, d_lam, d_psi, torch.cuda.current_stream())
        lam = d_lam.cpu().numpy()
        np.testing.assert_allclose(lam, lam_ref, rtol=1e-9, atol=1e-12 * np.abs(lam_ref).max(),
                                   err_msg=f"call {call}")
        assert np.isfinite(d_psi.cpu().numpy()).all()


@cuda
def test_noalloc_rejects_sizes_beyond_the_array():
    from paper_2309_11808_gb300 import SpodError, _lib
    nf, nb = 100, 200            # needs 100 * 32 * 200^2 bytes = 128 MB > 32 MiB
    d_gram = torch.zeros((nf, nb, nb, 2), dtype=torch.float64, device=DEV)
    d_lam = torch.zeros((nf, nb), dtype=torch.float64, device=DEV)
    d_psi = torch.zeros((nf, nb, nb, 2), dtype=torch.float64, device=DEV)
    with pytest.raises(SpodError) as e:
        _lib.spod_eigh_batched_noalloc(d_gram, nf, nb, d_lam, d_psi)
    assert e.value.status == _lib.SPOD_EINVAL and "32 MiB" in str(e.value)
