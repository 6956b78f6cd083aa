"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every entry point declared in include/fredec.h, and
rejects bad arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from helpers import ROOT, ensure_built


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    import paper_1309_0100_b300 as F
    return F


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fredec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fredec_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "fredec_periodogram" in names and "fredec_tuple_grad" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(fredec_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    raw = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        getattr(raw, n)


def test_built_for_sm103a(lib):
    from paper_1309_0100_b300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_opts(lib):
    assert "sm_103a" in lib.version()
    o = lib._opts()
    assert o.precision == 0 and o.topk == 0 and o.flag_tau == 0.0


@pytest.mark.parametrize("case", ["small_N", "nbase", "sigma", "nan_t", "nan_f", "topk", "prec", "nfneg"])
def test_validation_errors(lib, case):
    N = 20
    t = np.linspace(0, 10, N)
    y = np.sin(t)
    s = np.ones(N)
    f = np.linspace(0.01, 1, 10)
    base = []
    kw = {}
    if case == "small_N":
        t, y, s = t[:4], y[:4], s[:4]
        base = [0.1]
    elif case == "nbase":
        base = list(np.linspace(0.1, 1, 13))
    elif case == "sigma":
        s = s.copy(); s[3] = 0.0
    elif case == "nan_t":
        t = t.copy(); t[2] = np.nan
    elif case == "nan_f":
        f = f.copy(); f[5] = np.inf
    elif case == "topk":
        kw["topk"] = 65
    elif case == "prec":
        kw["precision"] = 7
    if case == "nfneg":
        r = lib.lib().fredec_periodogram(lib._p(t), lib._p(y), lib._p(s), N, None, 0, lib._p(f), -1, lib._p(f))
        assert r == 1
        return
    with pytest.raises(lib.FredecError) as ei:
        lib.periodogram(t, y, s, base, f, **kw)
    assert ei.value.code == 1
    assert lib.lib().fredec_last_error().decode()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1309_0100_b300 as F
    monkeypatch.setattr(F, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(F, "_lib_handle", None)
    with pytest.raises(F.FredecError):
        F.periodogram([0, 1, 2, 3], [1, 2, 3, 4], [1, 1, 1, 1], [], [0.1])
