"""The C-ABI library loads and exports every symbol include/tgv.h declares;
host-only entry points validate arguments (no CUDA call is made here)."""
import ctypes as C
import math
import os
import re
import subprocess
import sys
import textwrap

import pytest

import paper_2505_20911_b300 as tgv
from paper_2505_20911_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tgv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(_abi.LIB_PATH)
    declared = _declared_functions()
    assert len(declared) >= 15, declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(_abi.SIGNATURES), set(declared) - set(_abi.SIGNATURES)


def test_abi_version_and_strerror():
    assert _abi.lib().tgv_abi_version() == _abi.TGV_ABI_VERSION
    for s in range(0, -8, -1):
        assert _abi.strerror(s) != "unknown status"
    assert _abi.strerror(42) == "unknown status"


@pytest.mark.parametrize("mode", sorted(tgv.MODES))
def test_all_named_modes_are_built(mode):
    assert tgv.tgv_check_config(tgv.Config(n=32, mode=mode)) == 0


def test_invalid_configs_are_rejected_on_host():
    bad = [tgv.Config(n=4), tgv.Config(n=2048), tgv.Config(n=33), tgv.Config(n=32, mach=0.0),
           tgv.Config(n=32, re=-1.0), tgv.Config(n=32, mu=-1.0), tgv.Config(n=32, tile=9),
           tgv.Config(n=32, zchunk=64)]
    for c in bad:
        assert tgv.tgv_check_config(c) == _abi.TGV_ERR_ARG, c
    cfg = tgv.Config(n=32).c()
    cfg.q_storage, cfg.qt_storage, cfg.compute, cfg.accumulate = 3, 0, 0, 3
    assert _abi.lib().tgv_check_config(C.byref(cfg)) == _abi.TGV_ERR_UNSUPPORTED
    assert _abi.lib().tgv_check_config(None) == _abi.TGV_ERR_ARG


@pytest.mark.parametrize("split", ["blaisdell", "divergence", "feiereisen", "kgp", "keep"])
def test_every_split_form_is_a_valid_config(split):
    assert tgv.tgv_check_config(tgv.Config(n=32, split=split)) == 0


def test_unknown_split_form_is_rejected():
    cfg = tgv.Config(n=32).c()
    cfg.split_form = 5
    assert _abi.lib().tgv_check_config(C.byref(cfg)) == _abi.TGV_ERR_ARG


def _run_without_devices(body: str) -> None:
    """Run `body` in a child process that sees no CUDA device: the entry
    points below get fabricated device addresses, so if a validation were ever
    reordered or a mode became supported, the launch fails with "no device"
    instead of touching address 256 on a GPU."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    code = ("import ctypes as C\nimport paper_2505_20911_b300 as tgv\n"
            "from paper_2505_20911_b300 import _abi\nlib = _abi.lib()\n"
            "fake = C.c_void_p(256)\n" + textwrap.dedent(body))
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr


def test_null_pointers_fail_before_any_cuda_call():
    _run_without_devices("""
        cfg = tgv.Config(n=32).c()
        assert lib.tgv_init(C.byref(cfg), None, None) == _abi.TGV_ERR_ARG
        assert lib.rhs_eval(C.byref(cfg), None, None, None) == _abi.TGV_ERR_ARG
        assert lib.rk_substep(C.byref(cfg), None, None, None, 0, 0.001, None) == _abi.TGV_ERR_ARG
        assert lib.rk_step(C.byref(cfg), None, None, None, 0.001, 1, 0, None, None, 0, None,
                           None) == _abi.TGV_ERR_ARG
        assert lib.rk_substep(C.byref(cfg), fake, fake, fake, 0, 0.001, None) == _abi.TGV_ERR_ARG
        assert lib.rk_substep(C.byref(cfg), fake, C.c_void_p(512), fake, 3, 0.001,
                              None) == _abi.TGV_ERR_ARG
        assert lib.diagnostics_reduce(C.byref(cfg), fake, fake, None, 0,
                                      None) == _abi.TGV_ERR_WORKSPACE
        # unstable dt is refused before any launch
        assert lib.rk_step(C.byref(cfg), fake, C.c_void_p(512), C.c_void_p(1024), 1.0, 1, 0,
                           None, None, 0, None, None) == _abi.TGV_ERR_UNSTABLE_DT
    """)


def test_sizes_and_stability_limit():
    c = tgv.Config(n=32, mode="fp16_fp32")
    assert tgv.tgv_state_bytes(c) == 5 * 32 ** 3 * 2
    assert tgv.tgv_qt_bytes(tgv.Config(n=32, mode="hpsp")) == 5 * 32 ** 3 * 2
    assert tgv.tgv_state_bytes(tgv.Config(n=32, mode="spdp")) == 5 * 32 ** 3 * 8
    # dt_max = sqrt(3) / (1.3722/h * (sqrt(3)/M + 1))
    for n, m in ((32, 0.1), (256, 0.1), (512, 0.1), (96, 0.2)):
        h = 2 * math.pi / n
        ref = math.sqrt(3) / (1.3722 / h * (math.sqrt(3) / m + 1))
        assert abs(tgv.tgv_dt_max(tgv.Config(n=n, mach=m)) - ref) < 1e-15
    # the TGV settings used by the tests and the benchmark
    assert tgv.tgv_dt_max(tgv.Config(n=32)) > 0.004
    assert tgv.tgv_dt_max(tgv.Config(n=256)) > 0.00125
    assert tgv.tgv_dt_max(tgv.Config(n=512)) > 0.000625
    assert tgv.tgv_dt_max(tgv.Config(n=256)) < 0.004      # the 256^3 dt of 0.004 is unstable
    assert tgv.tgv_dt_max(tgv.Config(n=512)) < 0.001      # and so is 0.001 at 512^3


def test_tile_shapes_and_workspace():
    assert tgv.tgv_tile_shapes() == [(32, 16), (16, 16), (16, 8)]
    assert tgv.tgv_workspace_bytes(tgv.Config(n=64)) > 0
    assert tgv.tgv_run_host_workspace_bytes(tgv.Config(n=32), 10, 5) >= \
        2 * tgv.tgv_state_bytes(tgv.Config(n=32))


def test_adjoint_entry_points_validate_on_host():
    assert tgv.tgv_adjoint_workspace_bytes(tgv.Config(n=32)) == 16 * 32 ** 3 * 8
    assert tgv.tgv_adjoint_workspace_bytes(tgv.Config(n=32, mode="fp16_fp32")) == 0
    assert tgv.tgv_grad_workspace_bytes(tgv.Config(n=32), 200, 20) > 10 * 5 * 32 ** 3 * 8
    _run_without_devices("""
        c64, c16 = tgv.Config(n=32).c(), tgv.Config(n=32, mode="fp16_fp32").c()
        assert lib.rhs_vjp(C.byref(c16), fake, fake, fake, fake, 1 << 30, None) == \\
            _abi.TGV_ERR_UNSUPPORTED
        assert lib.rhs_vjp(C.byref(c64), fake, fake, fake, None, 0, None) == \\
            _abi.TGV_ERR_WORKSPACE
        assert lib.rk_step_adjoint(C.byref(c64), None, fake, 0.004, fake, 1 << 30, None) == \\
            _abi.TGV_ERR_ARG
        assert lib.tgv_grad_final_ke(C.byref(c64), fake, 0.004, 0, 20, fake, fake, fake,
                                     1 << 40, None) == _abi.TGV_ERR_ARG
        assert lib.tgv_grad_final_ke(C.byref(c64), fake, 1.0, 10, 5, fake, fake, fake,
                                     1 << 40, None) == _abi.TGV_ERR_UNSTABLE_DT
    """)


def test_missing_library_fails_loudly(monkeypatch):
    """No fallback: without libtgv.so the binding raises instead of computing."""
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libtgv.so"))
    with pytest.raises(ImportError):
        _abi.lib()
