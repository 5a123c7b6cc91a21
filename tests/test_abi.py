"""The C-ABI library builds, loads and exports every symbol include/kt.h declares.

No compute call is made here (no GPU needed); host-only entry points that touch no
device (option defaults, network parsing and validation) are exercised.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"\b(kt_[a-z0-9_]+)\s*\(", text):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def kt():
    from paper_2504_04941_gb300 import build, kt as ktm
    build.build()
    return ktm


def test_exports_every_declared_symbol(kt):
    L = kt.lib()
    names = _declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_options_default_and_network_parse(kt, tmp_path):
    from paper_2504_04941_gb300 import inputs as I
    o = kt.options()
    assert o.rtol == 1e-6 and o.max_newton == 8 and o.form == kt.KT_FORM_FP64
    net = kt.Network(I.network(2))
    assert (net.ns, net.ne, net.nr, net.energy) == (10, 2, 60, 1)
    bad = I.robertson_network()
    import numpy as np
    bad.counts = np.array([[1], [1], [2]])
    p = str(tmp_path / "bad.net")
    bad.write(p)
    with pytest.raises(kt.KtError) as ei:
        kt.Network(p)
    assert ei.value.code == -5
    (tmp_path / "junk.net").write_text("not a network\n")
    with pytest.raises(kt.KtError) as ei:
        kt.Network(str(tmp_path / "junk.net"))
    assert ei.value.code == -4


def test_options_lane_variant_default_and_range(kt):
    """lane_variant defaults to automatic and an out-of-range value is refused by the
    option check before any device work (a NULL-buffer call on zero cells)."""
    import ctypes as C
    from paper_2504_04941_gb300 import inputs as I
    o = kt.options()
    # 9 doubles and 16 ints: lane_variant took one of the reserved ints, the size is unchanged
    assert o.lane_variant == kt.KT_LANE_AUTO and C.sizeof(kt.Options) == 9 * 8 + 16 * 4
    net = kt.Network(I.network(2))
    L = kt.lib()
    for bad in (-1, 3):
        o = kt.options(lane_variant=bad)
        rc = L.kt_integrate_ptrs(net.ptr, 0, None, None, None, 1e-6, C.byref(o), None, None, None, None,
                                 None, None, None)
        assert rc == -1 and b"out of range" in L.kt_last_error()
    for good in (kt.KT_LANE_AUTO, kt.KT_LANE_JCACHE, kt.KT_LANE_LEAN):
        o = kt.options(lane_variant=good)
        rc = L.kt_integrate_ptrs(net.ptr, 0, None, None, None, 1e-6, C.byref(o), None, None, None, None,
                                 None, None, None)
        assert rc == 0, L.kt_last_error()


def test_no_oracle_in_product_path():
    """The CUDA package never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2504_04941_gb300")
    pat = re.compile(r"(^\s*(from|import)\s+oracle\b|kt_oracle|libkt_oracle|\bko_[a-z]+\()", re.M)
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not pat.search(text), fn
