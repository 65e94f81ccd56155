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
    n = C.c_int()
    assert lib.kfac_pinn_set_autotune(None, 1) == 1
    assert lib.kfac_pinn_get_tuning(None, None, 0, C.byref(n)) == 1
    assert lib.kfac_pinn_set_tuning(None, None, 0) == 1
    assert lib.kfac_pinn_set_graph(None, 1) == 1
    assert lib.kfac_pinn_set_cta_pairs(None, 1) == 1


_LAYOUT_PROBE = r"""
#include <stddef.h>
#include <stdio.h>
#include "kfac_pinn.h"
#define F(T, f) printf("%s.%s %zu %zu\n", #T, #f, offsetof(T, f), sizeof(((T*)0)->f))
#define V(x) printf("%s %d\n", #x, (int)(x))
int main(void) {
    printf("kfac_config_t %zu\n", sizeof(kfac_config_t));
    F(kfac_config_t, d); F(kfac_config_t, L); F(kfac_config_t, widths); F(kfac_config_t, op);
    F(kfac_config_t, kappa); F(kfac_config_t, precision); F(kfac_config_t, variant);
    F(kfac_config_t, beta); F(kfac_config_t, lambda); F(kfac_config_t, damping_sqrt);
    F(kfac_config_t, factor_init_identity); F(kfac_config_t, lr); F(kfac_config_t, momentum);
    F(kfac_config_t, max_n_int); F(kfac_config_t, max_n_bdy); F(kfac_config_t, update);
    F(kfac_config_t, eig_sm_budget); F(kfac_config_t, op_coef); F(kfac_config_t, residual);
    printf("kfac_residual_t %zu\n", sizeof(kfac_residual_t));
    F(kfac_residual_t, M); F(kfac_residual_t, b); F(kfac_residual_t, Q); F(kfac_residual_t, W);
    printf("kfac_tune_entry_t %zu\n", sizeof(kfac_tune_entry_t));
    F(kfac_tune_entry_t, kind); F(kfac_tune_entry_t, P); F(kfac_tune_entry_t, Q); F(kfac_tune_entry_t, K);
    F(kfac_tune_entry_t, tiles); F(kfac_tune_entry_t, sym); F(kfac_tune_entry_t, split);
    F(kfac_tune_entry_t, chunk); F(kfac_tune_entry_t, model_chunk); F(kfac_tune_entry_t, us);
    F(kfac_tune_entry_t, model_us);
    V(KFAC_MAX_LAYERS); V(KFAC_TUNE_CAP); V(KFAC_MAX_RESIDUALS);
    V(KFAC_OK); V(KFAC_BAD_ARG); V(KFAC_NOT_PD); V(KFAC_NONFINITE); V(KFAC_TIMEOUT); V(KFAC_OOM);
    V(KFAC_CUDA_ERROR); V(KFAC_NOT_READY);
    V(KFAC_FP64); V(KFAC_MIXED_BF16); V(KFAC_MIXED_SPLIT); V(KFAC_FP32); V(KFAC_EXPAND); V(KFAC_REDUCE);
    V(KFAC_OP_LAPLACE); V(KFAC_OP_HEAT); V(KFAC_OP_GENERAL);
    V(KFAC_UPDATE_FIXED); V(KFAC_UPDATE_LINE_SEARCH); V(KFAC_UPDATE_AUTO);
    V(KFAC_A_INT); V(KFAC_B_INT); V(KFAC_A_BDY); V(KFAC_B_BDY);
    V(KFAC_KC_LAYER_GEMM); V(KFAC_KC_ADJOINT_GEMM); V(KFAC_KC_GRAM); V(KFAC_KC_ELEMENTWISE);
    V(KFAC_KC_EIG); V(KFAC_KC_PRECOND); V(KFAC_KC_COUNT);
    V(KFAC_TUNE_GRAM); V(KFAC_TUNE_FWD_TAN); V(KFAC_TUNE_BWD_TAN);
    return 0;
}
"""


def test_ctypes_mirrors_match_the_header(tmp_path):
    # the binding's structures and constants against the C compiler's view
    # of include/kfac_pinn.h (host gcc, no CUDA)
    from paper_2405_15603_gb300 import _lib, api
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_PROBE)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = {}
    for line in filter(None, out):
        key, *vals = line.split()
        c[key] = tuple(int(v) for v in vals)
    for T, S in (("kfac_config_t", _lib.KfacConfig), ("kfac_tune_entry_t", _lib.KfacTuneEntry),
                 ("kfac_residual_t", _lib.KfacResidual)):
        assert c[T] == (C.sizeof(S),), T
        assert [f for f, _ in S._fields_] == [k.split(".")[1].replace("lambda", "lambda_")
                                               for k in c if k.startswith(T + ".")], T
        for f, _ in S._fields_:
            desc = getattr(S, f)
            assert c[f"{T}.{f.rstrip('_')}"] == (desc.offset, desc.size), (T, f)
    assert c["KFAC_MAX_LAYERS"] == (_lib.KFAC_MAX_LAYERS,)
    assert c["KFAC_TUNE_CAP"] == (_lib.KFAC_TUNE_CAP,)
    assert c["KFAC_MAX_RESIDUALS"] == (_lib.KFAC_MAX_RESIDUALS,)
    for code, name in _lib.STATUS.items():
        assert c[name] == (code,), name
    for name, v in api.PRECISIONS.items():
        assert c[{"fp64": "KFAC_FP64", "mixed_bf16": "KFAC_MIXED_BF16", "mixed_split": "KFAC_MIXED_SPLIT",
                  "fp32": "KFAC_FP32"}[name]] == (v,)
    for name, v in api.VARIANTS.items():
        assert c["KFAC_" + name.upper()] == (v,)
    for name, v in api.OPS.items():
        assert c["KFAC_OP_" + name.upper()] == (v,)
    for name, v in api.UPDATES.items():
        assert c["KFAC_UPDATE_" + {"fixed": "FIXED", "line_search": "LINE_SEARCH", "kfac_star": "AUTO"}[name]] == (v,)
    for name, v in api.FACTORS.items():
        assert c["KFAC_" + name.upper()] == (v,)
    for v, name in _lib.KERNEL_CLASSES.items():
        assert c["KFAC_KC_" + name.upper()] == (v,)
    assert c["KFAC_KC_COUNT"] == (len(_lib.KERNEL_CLASSES),)
    for v, name in _lib.TUNE_KINDS.items():
        assert c["KFAC_TUNE_" + name.upper()] == (v,)


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2405_15603_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "oracle" not in txt.replace("oracle_", ""), fn


def test_failure_hooks_validate_arguments_without_a_gpu():
    # argument errors are returned before anything touches the device
    from paper_2405_15603_gb300 import _lib
    lib = _lib.load()
    assert lib.kfac_pinn_inject_alloc_failure(-2) == 1      # KFAC_BAD_ARG
    assert lib.kfac_pinn_inject_alloc_failure(3) == 0
    assert lib.kfac_pinn_inject_alloc_failure(-1) == 0
    assert lib.kfac_pinn_check_wait_timeout(None, None, 0, 50) == 1
