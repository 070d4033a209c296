"""Failure statuses of the library, raised without faulting the GPU.

* SPOD_ETIMEOUT: every device wait of the library is bounded (TMA copies,
  tensor-core MMAs, pipeline stages).  With the self-test switch the
  tensor-core Gram leaves its first pipeline stage unfilled (a barrier that
  nothing completes); with the wait bound set to 1 ms the waits on it run out,
  the kernel stops early (copies and MMAs already in flight land first,
  tensor memory is freed), and spod_sync reports SPOD_ETIMEOUT.  The plan
  then fits normally, with the same result as before, once both are reset.
* SPOD_ENOTCONVERGED: the eigen-solver given one implicit QL iteration per
  eigenvalue cannot deflate a dense Gram; the next synchronising call reports
  it, and the default cap gives the ordinary result again.
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


@cuda
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_wait_bound_runs_out_then_the_plan_recovers(prec):
    from paper_2309_11808_gb300 import SPOD, SpodError, _lib
    wl = jet_like(nx=32, nr=16, nvars=2, nt=2048, nfft=256, seed=5, dtype=torch.float32)
    X = wl.X.to(DEV)
    sp = SPOD(wl.npoints, 2, 2048, 256, 128, precision=prec, weights=wl.W)
    sp.fit(X)
    lam0 = sp.eigs()
    _lib.spod_plan_set_tuning(sp.handle, wait_timeout_us=1000, wait_selftest=1)
    t = _lib.spod_plan_get_tuning(sp.handle)
    assert t.wait_timeout_us == 1000 and t.wait_selftest == 1
    sp.fit(X)
    with pytest.raises(SpodError) as e:
        sp.sync()
    assert e.value.status == _lib.SPOD_ETIMEOUT
    _lib.spod_plan_set_tuning(sp.handle, wait_timeout_us=0, wait_selftest=0)
    sp.fit(X)
    lam1 = sp.eigs()                      # no status raised: the flags were cleared by the fit
    np.testing.assert_array_equal(lam1, lam0)
    sp.close()


@cuda
@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_iteration_cap_reports_not_converged(prec):
    from paper_2309_11808_gb300 import SPOD, SpodError, _lib
    wl = jet_like(nx=16, nr=16, nvars=1, nt=1500, nfft=64, seed=6,
                  dtype=torch.float64 if prec == "fp64" else torch.float32)
    X = wl.X.to(DEV)
    sp = SPOD(wl.npoints, 1, 1500, 64, 32, dtype=X.dtype, precision=prec, weights=wl.W)
    sp.fit(X)
    lam0 = sp.eigs()
    _lib.spod_plan_set_tuning(sp.handle, eig_max_iter=1)
    sp.fit(X)
    with pytest.raises(SpodError) as e:
        sp.eigs()
    assert e.value.status == _lib.SPOD_ENOTCONVERGED
    _lib.spod_plan_set_tuning(sp.handle, eig_max_iter=0)
    sp.fit(X)
    np.testing.assert_array_equal(sp.eigs(), lam0)
    sp.close()


@cuda
def test_tuning_ranges_are_checked():
    from paper_2309_11808_gb300 import SPOD, SpodError, _lib
    sp = SPOD(256, 1, 512, 64, 32, precision="fp32")
    for kw in ({"eig_max_iter": 1001}, {"eig_max_iter": -1}, {"wait_timeout_us": 4000001}, {"wait_timeout_us": -2},
               {"wait_selftest": 2}):
        with pytest.raises(SpodError) as e:
            _lib.spod_plan_set_tuning(sp.handle, **kw)
        assert e.value.status == _lib.SPOD_EINVAL
    sp.close()
