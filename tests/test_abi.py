"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/spod.h declares, the ctypes structs match the C
layout, and argument validation fails cleanly."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2309_11808_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spod.h")


@pytest.fixture(scope="module")
def L():
    _build.build()
    return _lib.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(spod_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_expected_entry_points():
    names = declared_functions()
    for must in ("spod_plan_create", "spod_fit", "spod_modes", "spod_backward", "spod_get_eigs"):
        assert must in names
    assert sorted(_lib.EXPORTED) == names


def test_every_declaration_cites_its_passage():
    # each entry point's comment names the passage that defines it (Sec. / Eq.)
    # or says that the paper has no counterpart
    src = open(HEADER).read()
    decl = re.compile(r"^\s*(?:const\s+)?\w+\s*\*?\s*(spod_\w+)\s*\(", flags=re.M)
    cite = re.compile(r"Sec\.|Eq\.|Algorithm|[Nn]o counterpart|not in the paper|paper has no counterpart")
    shared = {"spod_profile_read": "spod_profile_enable"}     # one comment for the pair
    found = {}
    for m in decl.finditer(src):
        c0, c1 = src.rfind("/*", 0, m.start()), src.rfind("*/", 0, m.start())
        text = src[c0:c1] if c1 > c0 >= 0 and ";" not in src[c1 + 2:m.start()] else ""
        found[m.group(1)] = bool(cite.search(text))
    for name, ok in found.items():
        assert ok or found.get(shared.get(name, ""), False), name


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    assert _lib.spod_version().startswith("spod-gb300")


def test_struct_layout_matches_c(tmp_path):
    fields_desc = [f for f, _ in _lib.spod_plan_desc._fields_]
    fields_info = [f for f, _ in _lib.spod_plan_info._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    prog.append('printf("desc %zu\\n", sizeof(spod_plan_desc));')
    prog.append('printf("info %zu\\n", sizeof(spod_plan_info));')
    prog.append('printf("tun %zu\\n", sizeof(spod_tuning));')
    for f, _ in _lib.spod_tuning._fields_:
        prog.append(f'printf("t.{f} %zu\\n", offsetof(spod_tuning, {f}));')
    for f in fields_desc:
        prog.append(f'printf("d.{f} %zu\\n", offsetof(spod_plan_desc, {f}));')
    for f in fields_info:
        prog.append(f'printf("i.{f} %zu\\n", offsetof(spod_plan_info, {f}));')
    prog.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(c), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    assert int(out["desc"]) == ctypes.sizeof(_lib.spod_plan_desc)
    assert int(out["info"]) == ctypes.sizeof(_lib.spod_plan_info)
    for f in fields_desc:
        assert int(out[f"d.{f}"]) == getattr(_lib.spod_plan_desc, f).offset, f
    for f in fields_info:
        assert int(out[f"i.{f}"]) == getattr(_lib.spod_plan_info, f).offset, f
    assert int(out["tun"]) == ctypes.sizeof(_lib.spod_tuning)
    for f, _ in _lib.spod_tuning._fields_:
        assert int(out[f"t.{f}"]) == getattr(_lib.spod_tuning, f).offset, f


def test_argument_validation_on_host(L):
    d = _lib.spod_desc_init()
    assert d.window == _lib.SPOD_WIN_HAMMING and d.subtract_mean == 1 and d.dt == 1.0
    h = ctypes.c_void_p()
    # NULL desc / out
    assert L.spod_plan_create(None, ctypes.byref(h)) == _lib.SPOD_EINVAL
    assert L.spod_plan_create(ctypes.byref(d), None) == _lib.SPOD_EINVAL
    # invalid sizes are rejected before any device call
    d.dims[0] = 10
    d.nt, d.nfft, d.noverlap = 100, 16, 16
    assert L.spod_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.SPOD_EINVAL
    assert "noverlap" in _lib.spod_last_error()
    d.noverlap, d.nfft = 8, 200
    assert L.spod_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.SPOD_EINVAL
    d.nfft, d.ndim = 16, 0
    assert L.spod_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.SPOD_EINVAL
    d.ndim, d.nvars = 1, 0
    assert L.spod_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.SPOD_EINVAL
    d.nvars, d.dt = 1, 0.0
    assert L.spod_plan_create(ctypes.byref(d), ctypes.byref(h)) == _lib.SPOD_EINVAL
    assert h.value is None
    # NULL plan handles
    assert L.spod_fit(None, None, None) == _lib.SPOD_EINVAL
    assert L.spod_plan_destroy(None) == _lib.SPOD_OK
    E = _lib.SPOD_EINVAL
    info = _lib.spod_plan_info()
    tun = _lib.spod_tuning()
    assert L.spod_plan_get_info(None, ctypes.byref(info)) == E
    assert L.spod_get_eigs(None, None, None, 0) == E
    assert L.spod_get_gram(None, None) == E
    assert L.spod_get_freqs(None, None) == E
    assert L.spod_modes(None, None, 1, None, None) == E
    assert L.spod_backward(None, None, None, None, None) == E
    assert L.spod_sync(None, None) == E
    assert L.spod_run_host(None, None, 0, None, None, None) == E
    assert L.spod_run_host_many(None, 1, None, 0, None, None, None) == E
    assert L.spod_run_host_ooc(None, None, 0, None, None, 0, None) == E
    assert L.spod_coeffs(None, None, None, 1, 1, 0, None, None, None) == E
    assert L.spod_reconstruct(None, None, 1, 1, 0, None, None, None, None) == E
    assert L.spod_plan_get_tuning(None, ctypes.byref(tun)) == E
    assert L.spod_plan_set_tuning(None, ctypes.byref(tun)) == E
    assert L.spod_plan_autotune(None, None, None, ctypes.byref(tun)) == E
    assert L.spod_profile_enable(None, 1) == E
    assert L.spod_profile_read(None, None, None) == E
    assert L.spod_fit_batch(None, None, 1, None) == E
    assert L.spod_fit_partial(None, None, None, None) == E
    assert L.spod_fit_from_grams(None, None, 1, None) == E
