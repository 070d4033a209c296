"""ctypes binding of libspod.so: the entry points of include/spod.h under the
same names.  Argument marshalling only -- every step of the SPOD path runs in
the library's CUDA kernels.  Importing this module does not load the library;
the first call does, and raises if libspod.so has not been built."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libspod.so")

# enums (values as in include/spod.h)
SPOD_OK, SPOD_EINVAL, SPOD_ENOMEM, SPOD_ECUDA, SPOD_ESTATE = 0, 1, 2, 3, 4
SPOD_ENANINPUT, SPOD_ENOTCONVERGED, SPOD_ETIMEOUT, SPOD_EUNSUPPORTED = 5, 6, 7, 8
SPOD_F64, SPOD_F32, SPOD_BF16, SPOD_C64, SPOD_C128 = 0, 1, 2, 3, 4
SPOD_PREC_FP64, SPOD_PREC_FP32, SPOD_PREC_BF16, SPOD_PREC_BF16X3 = 0, 1, 2, 3
SPOD_WIN_HAMMING, SPOD_WIN_HAMMING_PERIODIC, SPOD_WIN_HANN, SPOD_WIN_RECT, SPOD_WIN_USER = 0, 1, 2, 3, 4
SPOD_NORM_NB, SPOD_NORM_NB_MINUS_1 = 0, 1

STATUS_NAMES = {0: "SPOD_OK", 1: "SPOD_EINVAL", 2: "SPOD_ENOMEM", 3: "SPOD_ECUDA", 4: "SPOD_ESTATE",
                5: "SPOD_ENANINPUT", 6: "SPOD_ENOTCONVERGED", 7: "SPOD_ETIMEOUT", 8: "SPOD_EUNSUPPORTED"}

# every symbol include/spod.h declares
EXPORTED = ["spod_desc_init", "spod_plan_create", "spod_plan_destroy", "spod_plan_get_info", "spod_fit",
            "spod_get_eigs", "spod_get_gram", "spod_get_freqs", "spod_modes", "spod_backward",
            "spod_run_host", "spod_run_host_many", "spod_sync", "spod_fit_batch", "spod_profile_enable",
            "spod_profile_read", "spod_eigh_batched_noalloc", "spod_plan_get_tuning", "spod_plan_set_tuning",
            "spod_plan_autotune", "spod_coeffs", "spod_reconstruct", "spod_run_host_ooc", "spod_fit_partial",
            "spod_fit_from_grams", "spod_last_error", "spod_version"]

PHASES = ["mean", "fft", "gram", "reduce", "eig", "modes", "backward"]


class spod_plan_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("dims", C.c_int64 * 3), ("nvars", C.c_int), ("nt", C.c_int64),
                ("nfft", C.c_int), ("noverlap", C.c_int), ("window", C.c_int),
                ("user_window", C.POINTER(C.c_double)), ("weights", C.POINTER(C.c_double)),
                ("dt", C.c_double), ("in_dtype", C.c_int), ("precision", C.c_int), ("norm", C.c_int),
                ("subtract_mean", C.c_int), ("chunk_points", C.c_int64), ("mean_in_fft", C.c_int)]


class spod_plan_info(C.Structure):
    _fields_ = [("M", C.c_int64), ("nt", C.c_int64), ("nfft", C.c_int), ("noverlap", C.c_int),
                ("step", C.c_int), ("nb", C.c_int), ("nf", C.c_int), ("device", C.c_int),
                ("workspace_bytes", C.c_size_t), ("chunk_points", C.c_int64), ("mean_in_fft", C.c_int)]


class spod_tuning(C.Structure):
    _fields_ = [("gram_splits", C.c_int), ("gram_splits_max", C.c_int), ("gram_flush_blocks", C.c_int),
                ("modes_ctas", C.c_int), ("eig_max_iter", C.c_int), ("wait_timeout_us", C.c_int),
                ("wait_selftest", C.c_int), ("fft_tile_points", C.c_int)]


class SpodError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_lib = None


def lib() -> C.CDLL:
    """Load libspod.so (raises if it was not built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.spod_desc_init.argtypes = [C.POINTER(spod_plan_desc)]
        L.spod_plan_create.argtypes = [C.POINTER(spod_plan_desc), C.POINTER(P)]
        L.spod_plan_destroy.argtypes = [P]
        L.spod_plan_get_info.argtypes = [P, C.POINTER(spod_plan_info)]
        L.spod_fit.argtypes = [P, P, P]
        L.spod_get_eigs.argtypes = [P, P, P, C.c_int]
        L.spod_get_gram.argtypes = [P, P]
        L.spod_get_freqs.argtypes = [P, P]
        L.spod_modes.argtypes = [P, P, C.c_int, P, P]
        L.spod_backward.argtypes = [P, P, P, P, P]
        L.spod_run_host.argtypes = [P, P, C.c_int, P, P, P]
        L.spod_run_host_many.argtypes = [P, C.c_int, C.POINTER(P), C.c_int, C.POINTER(P), C.POINTER(P), P]
        L.spod_sync.argtypes = [P, P]
        L.spod_fit_batch.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int, P]
        L.spod_profile_enable.argtypes = [P, C.c_int]
        L.spod_profile_read.argtypes = [P, P, P]
        L.spod_eigh_batched_noalloc.argtypes = [P, C.c_int, C.c_int, P, P, P]
        L.spod_plan_get_tuning.argtypes = [P, C.POINTER(spod_tuning)]
        L.spod_plan_set_tuning.argtypes = [P, C.POINTER(spod_tuning)]
        L.spod_plan_autotune.argtypes = [P, P, P, C.POINTER(spod_tuning)]
        L.spod_coeffs.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), P, P]
        L.spod_run_host_ooc.argtypes = [P, P, C.c_int, P, P, C.c_int64, P]
        L.spod_reconstruct.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), P, P, P]
        L.spod_fit_partial.argtypes = [P, P, P, P]
        L.spod_fit_from_grams.argtypes = [P, P, C.c_int, P]
        L.spod_last_error.restype = C.c_char_p
        L.spod_version.restype = C.c_char_p
        for name in EXPORTED[:-2]:
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != SPOD_OK:
        raise SpodError(status, where, lib().spod_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    """Device or host address of a tensor / array / int (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------- entry points
def spod_desc_init() -> spod_plan_desc:
    d = spod_plan_desc()
    check(lib().spod_desc_init(C.byref(d)), "spod_desc_init")
    return d


def spod_plan_create(desc: spod_plan_desc) -> int:
    h = C.c_void_p()
    check(lib().spod_plan_create(C.byref(desc), C.byref(h)), "spod_plan_create")
    return h.value


def spod_plan_destroy(plan: int) -> None:
    check(lib().spod_plan_destroy(plan), "spod_plan_destroy")


def spod_plan_get_info(plan: int) -> spod_plan_info:
    info = spod_plan_info()
    check(lib().spod_plan_get_info(plan, C.byref(info)), "spod_plan_get_info")
    return info


def spod_fit(plan: int, X, stream=None) -> None:
    check(lib().spod_fit(plan, _ptr(X), _stream(stream)), "spod_fit")


def spod_fit_partial(plan: int, X, gram, stream=None) -> None:
    check(lib().spod_fit_partial(plan, _ptr(X), _ptr(gram), _stream(stream)), "spod_fit_partial")


def spod_fit_from_grams(plan: int, grams, nparts: int, stream=None) -> None:
    check(lib().spod_fit_from_grams(plan, _ptr(grams), int(nparts), _stream(stream)), "spod_fit_from_grams")


def spod_get_eigs(plan: int, lam, psi=None, on_device: bool = False) -> None:
    check(lib().spod_get_eigs(plan, _ptr(lam), _ptr(psi), int(on_device)), "spod_get_eigs")


def spod_get_gram(plan: int, gram) -> None:
    check(lib().spod_get_gram(plan, _ptr(gram)), "spod_get_gram")


def spod_get_freqs(plan: int, freqs) -> None:
    check(lib().spod_get_freqs(plan, _ptr(freqs)), "spod_get_freqs")


def spod_modes(plan: int, X, nmodes: int, Phi, stream=None) -> None:
    check(lib().spod_modes(plan, _ptr(X), int(nmodes), _ptr(Phi), _stream(stream)), "spod_modes")


def spod_backward(plan: int, dLdlam, X, dX, stream=None) -> None:
    check(lib().spod_backward(plan, _ptr(dLdlam), _ptr(X), _ptr(dX), _stream(stream)), "spod_backward")


def spod_run_host(plan: int, hX, nmodes: int, hPhi, hlam, stream=None) -> None:
    check(lib().spod_run_host(plan, _ptr(hX), int(nmodes), _ptr(hPhi), _ptr(hlam), _stream(stream)),
          "spod_run_host")


def spod_run_host_many(plan: int, hXs, nmodes: int, hPhis, hlams=None, stream=None) -> None:
    n = len(hXs)
    arr_x = (C.c_void_p * n)(*[_ptr(x) for x in hXs])
    arr_p = (C.c_void_p * n)(*[_ptr(x) for x in hPhis]) if hPhis is not None else None
    arr_l = (C.c_void_p * n)(*[_ptr(x) for x in hlams]) if hlams is not None else None
    check(lib().spod_run_host_many(plan, n, arr_x, int(nmodes), arr_p, arr_l, _stream(stream)),
          "spod_run_host_many")


def spod_run_host_ooc(plan: int, hX, nmodes: int, hPhi, hlam, tile_points: int = 0, stream=None) -> None:
    check(lib().spod_run_host_ooc(plan, _ptr(hX), int(nmodes), _ptr(hPhi), _ptr(hlam), int(tile_points),
                                  _stream(stream)), "spod_run_host_ooc")


def spod_coeffs(plan: int, X, Phi, nmodes: int, nmodes_r: int, freqs, A, stream=None) -> None:
    fr = (C.c_int * len(freqs))(*[int(f) for f in freqs])
    check(lib().spod_coeffs(plan, _ptr(X), _ptr(Phi), int(nmodes), int(nmodes_r), len(freqs), fr, _ptr(A),
                            _stream(stream)), "spod_coeffs")


def spod_reconstruct(plan: int, Phi, nmodes: int, nmodes_r: int, freqs, A, Xrec, stream=None) -> None:
    fr = (C.c_int * len(freqs))(*[int(f) for f in freqs])
    check(lib().spod_reconstruct(plan, _ptr(Phi), int(nmodes), int(nmodes_r), len(freqs), fr, _ptr(A), _ptr(Xrec),
                                 _stream(stream)), "spod_reconstruct")


def spod_sync(plan: int, stream=None) -> None:
    check(lib().spod_sync(plan, _stream(stream)), "spod_sync")


def spod_fit_batch(plans, Xs, stream=None) -> None:
    n = len(plans)
    arr_p = (C.c_void_p * n)(*plans)
    arr_x = (C.c_void_p * n)(*[_ptr(x) for x in Xs])
    check(lib().spod_fit_batch(arr_p, arr_x, n, _stream(stream)), "spod_fit_batch")


def spod_profile_enable(plan: int, enable: bool = True) -> None:
    check(lib().spod_profile_enable(plan, int(enable)), "spod_profile_enable")


def spod_profile_read(plan: int):
    """Returns ({phase: ms}, {phase: kernel launches}) since the previous read."""
    import numpy as np
    ms = np.zeros(len(PHASES), dtype=np.float64)
    ln = np.zeros(len(PHASES), dtype=np.int64)
    check(lib().spod_profile_read(plan, ms.ctypes.data, ln.ctypes.data), "spod_profile_read")
    return dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, ln.tolist()))


def spod_eigh_batched_noalloc(gram, nf: int, nb: int, lam, psi, stream=None) -> None:
    check(lib().spod_eigh_batched_noalloc(_ptr(gram), int(nf), int(nb), _ptr(lam), _ptr(psi), _stream(stream)),
          "spod_eigh_batched_noalloc")


def spod_plan_get_tuning(plan: int) -> spod_tuning:
    t = spod_tuning()
    check(lib().spod_plan_get_tuning(plan, C.byref(t)), "spod_plan_get_tuning")
    return t


def spod_plan_set_tuning(plan: int, gram_splits: int = 0, gram_flush_blocks: int = 0, modes_ctas: int = 0,
                         eig_max_iter: int = 0, wait_timeout_us: int = 0, wait_selftest: int = 0,
                         fft_tile_points: int = 0) -> None:
    t = spod_tuning(int(gram_splits), 0, int(gram_flush_blocks), int(modes_ctas), int(eig_max_iter),
                    int(wait_timeout_us), int(wait_selftest), int(fft_tile_points))
    check(lib().spod_plan_set_tuning(plan, C.byref(t)), "spod_plan_set_tuning")


def spod_plan_autotune(plan: int, X, stream=None) -> spod_tuning:
    t = spod_tuning()
    check(lib().spod_plan_autotune(plan, _ptr(X), _stream(stream), C.byref(t)), "spod_plan_autotune")
    return t


def spod_last_error() -> str:
    return lib().spod_last_error().decode(errors="replace")


def spod_version() -> str:
    return lib().spod_version().decode()
