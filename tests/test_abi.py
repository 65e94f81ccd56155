"""The C-ABI library loads and exports every entry point include/ declares
(host-only checks: no GPU compute call)."""
import ctypes as C
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(kfac_pinn_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2405_15603_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(kfac_pinn_\w+)\b", out))
    assert declared <= exported, declared - exported
    from paper_2405_15603_gb300 import _lib
    assert set(_lib.EXPORTS) == declared


def test_param_count_host_only(lib):
    from paper_2405_15603_gb300.api import make_config
    with open(os.path.join(ROOT, "tests", "golden", "param_counts.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        cfg = make_config(c["d"], c["widths"])
        assert lib.kfac_pinn_param_count(C.byref(cfg)) == c["D"]
    bad = make_config(2, (4, 2))          # last width must be 1
    assert lib.kfac_pinn_param_count(C.byref(bad)) == -1


def test_status_strings(lib):
    assert lib.kfac_pinn_status_string(0) == b"KFAC_OK"
    assert lib.kfac_pinn_status_string(2) == b"KFAC_NOT_PD"


def test_null_handle_is_bad_arg(lib):
    assert lib.kfac_pinn_invert(None, None) == 1
    assert lib.kfac_pinn_destroy(None) == 1
    assert lib.kfac_pinn_create(None, None) == 1


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2405_15603_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in txt.replace("oracle_", ""), fn
