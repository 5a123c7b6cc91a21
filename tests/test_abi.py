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


def test_no_oracle_in_product_path():
    """The CUDA package never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2504_04941_gb300")
    pat = re.compile(r"(^\s*(from|import)\s+oracle\b|kt_oracle|libkt_oracle|\bko_[a-z]+\()", re.M)
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not pat.search(text), fn
