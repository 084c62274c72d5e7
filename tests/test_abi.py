"""The C-ABI library loads and exports every function include/extrass.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["init_grid", "load_atomic_data", "run_transport", "get_photoexcitation_rates",
                 "get_spectrum", "xt_create", "xt_destroy", "xt_last_error"]:
        assert need in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    import paper_2511_07539_gb300 as xt
    L = ctypes.CDLL(xt.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_has_same_names():
    import paper_2511_07539_gb300 as xt
    for n in declared_functions():
        assert hasattr(xt, n), n
