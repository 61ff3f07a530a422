"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/tabi.h declares; parameter defaults match the paper.
No compute calls (no GPU here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "tabi.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tabi_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_07782_gb300 import build, tabi
    build.build()
    return tabi.load()


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 9
    for s in syms:
        assert hasattr(lib, s), s


def test_param_defaults_follow_the_paper(lib):
    from paper_2602_07782_gb300 import tabi
    p = tabi.params_default()
    assert (p.gutter, p.knee_abs_pct, p.knee_rel_pct, p.lr_sig_pct) == (1, 10, 20, 10)
    assert p.flags == tabi.F_ALL and p.scale_fanout == 0  # 0: tuned / default launch shape
    assert p.laabb_count == 10  # local AABBs per axis (App. A)
    assert (p.topt_permille, p.hybrid_min_charts) == (10, 10000)  # Sec. 4.4: 1 % above 10,000 charts
    assert ctypes.sizeof(tabi.Params) == 44 and p.version == 2
    assert tabi.status_str(tabi.TABI_ERR_NO_FIT) == "no candidate scale fits"


def test_binding_refuses_a_missing_library(tmp_path):
    from paper_2602_07782_gb300 import tabi
    saved = tabi._lib
    tabi._lib = None
    try:
        with pytest.raises(RuntimeError):
            tabi.load(str(tmp_path / "missing.so"))
    finally:
        tabi._lib = saved


def test_arena_sizing_is_monotone(lib):
    from paper_2602_07782_gb300 import tabi
    import synth
    a = tabi.arena_bytes(synth.plain64())
    b = tabi.arena_bytes(synth.stars(3, 2000, 2048))
    assert 0 < a < b
