"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every entry point include/tomo.h declares, the binding's
structures have the C layout, and argument validation answers TOMO_EINVAL
before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2404_02844_gb300 as tomo
from paper_2404_02844_gb300 import build as tomo_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tomo.h")


@pytest.fixture(scope="module")
def L():
    tomo_build.build()
    return tomo.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tomo_[A-Za-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "tomo_plan" in names and "tomo_fit" in names and "tomo_objective" in names
    out = subprocess.run(["nm", "-D", "--defined-only", tomo_build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tomo_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the binding knows all of them
    assert set(names) == {n for n, _, _ in tomo.EXPORTS}


def test_struct_layouts_match_c(tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "tomo.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(tomo_desc),"
        " sizeof(tomo_fit_opts), sizeof(tomo_fit_report), offsetof(tomo_desc, stream),"
        " offsetof(tomo_fit_opts, max_newton), offsetof(tomo_fit_report, iters_s1));return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(tomo.tomo_desc), ctypes.sizeof(tomo.tomo_fit_opts),
            ctypes.sizeof(tomo.tomo_fit_report), tomo.tomo_desc.stream.offset,
            tomo.tomo_fit_opts.max_newton.offset, tomo.tomo_fit_report.iters_s1.offset]
    assert got == want


def test_default_options_follow_the_paper(L):
    o = tomo.tomo_fit_opts_default()
    assert (o.beta, o.c, o.switch_tol) == (0.75, 0.1, 1e-4)
    assert o.start_stage == 1 and o.warm_start == 0


def _desc(M=10, N=3, lam=None, gamma=0.0, prec=0, band_k=10.0, flags=0):
    lam = np.linspace(0, 5, 7) if lam is None else np.asarray(lam, dtype=np.float64)
    d = tomo.tomo_desc(M, N, len(lam), lam.ctypes.data, band_k, gamma, prec, 0, None, flags)
    return d, lam


@pytest.mark.parametrize("kw", [dict(M=0), dict(N=1), dict(N=2000), dict(gamma=-1.0),
                                dict(gamma=float("nan")), dict(prec=7), dict(flags=2),
                                dict(lam=[0.0, 2.0, 1.0]), dict(lam=[0.0, float("inf")]),
                                dict(lam=[-1.0, 2.0]), dict(band_k=float("nan"))])
def test_invalid_descriptors_are_rejected_before_cuda(L, kw):
    d, lam = _desc(**kw)
    h = ctypes.c_void_p(123)
    st = L.tomo_plan(ctypes.byref(h), ctypes.byref(d))
    assert st == 1, tomo.STATUS.get(st)
    assert h.value is None
    assert L.tomo_last_error()


def test_null_arguments(L):
    assert L.tomo_plan(None, None) == 1
    assert L.tomo_objective(None, None, None, None, None) == 1
    assert L.tomo_fit(None, None, None, None, None) == 1
    L.tomo_plan_destroy(None)


def test_library_has_no_cpu_fallback_symbols():
    """The product library links no oracle code."""
    out = subprocess.run(["nm", "-D", tomo_build.LIB], capture_output=True, text=True).stdout
    assert "orc_" not in out
