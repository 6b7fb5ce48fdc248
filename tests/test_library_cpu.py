"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every symbol include/ftk.h declares, sizes workspaces and rejects bad
arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from ftk_inputs import named

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ftk():
    from paper_1802_02854_gb300 import build
    build.build()
    import paper_1802_02854_gb300 as m
    return m


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "ftk.h")).read()
    return sorted(set(re.findall(r"\b(ftk_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(ftk):
    declared = _header_symbols()
    assert set(declared) == set(ftk.EXPORTS)
    lib = C.CDLL(ftk.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def test_footprint_layout(ftk):
    f64 = ftk.ftk_footprint(12, 4, 2, ftk.FTK_FP64)
    f32 = ftk.ftk_footprint(12, 4, 2, ftk.FTK_FP32)
    d = 1 << 12
    # 2 TPQ (always FP64) + 4 shells + 2 probes + 3*2 Krylov vectors
    assert f64 >= 14 * d * 16 and f32 >= 2 * d * 16 + 12 * d * 8
    assert f64 - f32 >= 12 * d * 8 - 14 * 256
    assert ftk.ftk_footprint(31, 1, 1, 0) == 0
    assert ftk.ftk_footprint(12, 0, 1, 0) == 0
    assert ftk.ftk_footprint(12, 1, 33, 0) == 0
    assert ftk.ftk_footprint(12, 1, 1, 7) == 0


@pytest.mark.parametrize("bad", ["site", "self", "gamma", "prec", "rhs"])
def test_create_rejects_bad_arguments(ftk, bad):
    from ftk_inputs import named
    cl = named(8)
    bonds = cl.bonds.copy()
    kw = dict(precision=ftk.FTK_FP64, max_rhs=1, n_saved=1)
    if bad == "site":
        bonds[0, 1] = 8
    elif bad == "self":
        bonds[0, 1] = bonds[0, 0]
    elif bad == "gamma":
        bonds[0, 2] = 3
    elif bad == "prec":
        kw["precision"] = 5
    elif bad == "rhs":
        kw["max_rhs"] = 64
    with pytest.raises(ftk.FtkError) as e:
        ftk.ftk_create(cl.n_sites, cl.pos, bonds, -1.0, 0.1, **kw)
    assert e.value.status == ftk.FTK_EINVAL


@pytest.mark.parametrize("n,prec,passes", [
    (12, "fp64", 1), (12, "fp32", 1), (12, "df", 1),     # N <= tile sites: one pass, the optimum
    (16, "fp64", 2), (16, "fp32", 2), (16, "df", 2),     # N > tile sites and every site has bonds: >= 2
    (24, "fp32", 3), (24, "fp64", 3), (24, "df", 3),     # the 24-site plans the measurements use
])
def test_suggest_order_plans(ftk, n, prec, passes):
    """Host planner (no GPU): a permutation of the sites and the number of H.v
    passes of the relabelled cluster; deterministic (seeded restarts)."""
    from ftk_inputs import named
    cl = named(n)
    perm, npass = ftk.ftk_suggest_order(n, cl.bonds, ftk.PRECISIONS[prec], 1)
    assert sorted(perm.tolist()) == list(range(n))
    assert npass == passes
    perm2, npass2 = ftk.ftk_suggest_order(n, cl.bonds, ftk.PRECISIONS[prec], 1)
    assert (perm2 == perm).all() and npass2 == npass


def test_suggest_order_rejects_bad_arguments(ftk):
    from ftk_inputs import named
    cl = named(12)
    with pytest.raises(Exception):
        ftk.ftk_suggest_order(12, cl.bonds, ftk.FTK_FP64, 3)            # n_rhs not a power of two
    with pytest.raises(Exception):
        ftk.ftk_suggest_order(12, [(0, 0, 2)], ftk.FTK_FP64, 1)         # i == j
    with pytest.raises(Exception):
        ftk.ftk_suggest_order(12, [(0, 12, 2)], ftk.FTK_FP64, 1)        # site out of range
    with pytest.raises(Exception):
        ftk.ftk_suggest_order(31, cl.bonds, ftk.FTK_FP64, 1)            # more sites than supported


def test_no_fallback_without_the_library(ftk, monkeypatch):
    """Without libftk.so every call raises (there is no CPU path)."""
    monkeypatch.setattr(ftk, "_lib", None)
    monkeypatch.setattr(ftk, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libftk.so"))
    with pytest.raises(ftk.FtkError):
        ftk.ftk_footprint(12, 1, 1, ftk.FTK_FP64)
    with pytest.raises(ftk.FtkError):
        ftk.ftk_suggest_order(12, named(12).bonds, ftk.FTK_FP64, 1)


def test_product_and_oracle_are_independent():
    """The product package (Python and CUDA sources) never imports or links the
    oracle, and the oracle never imports the product; they share only the
    seeded input generators (ftk_inputs)."""
    pkg = os.path.join(ROOT, "paper_1802_02854_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                src = open(os.path.join(dirpath, f), encoding="utf-8").read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f
                assert "liboracle" not in src and "orc_" not in src, f
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(odir, f), encoding="utf-8").read()
            assert "paper_1802_02854_gb300" not in src and "ftk_" not in src.replace("ftk_inputs", ""), f
