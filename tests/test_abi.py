"""The C ABI library builds, loads without a GPU and exports every function
that include/swccl.h declares; host-side logic that needs no device.

No call here launches a kernel: only argument validation and the threshold
arithmetic, which return before any CUDA call.
"""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swccl.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def lib():
    from paper_1105_5804_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_documented_entry_points():
    names = _declared_functions()
    for required in ("sw_create", "sw_create_ex", "sw_create_threshold", "sw_sweep", "sw_observables",
                     "sw_get_spins", "sw_set_spins", "sw_debug_dump", "sw_destroy", "ccl_label",
                     "ccl_bonds_from_pixels", "ccl_perc_mask", "sw_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_has_the_same_names():
    import paper_1105_5804_gb300 as sw
    missing = [n for n in _declared_functions() if not hasattr(sw, n)]
    assert not missing, missing


def test_threshold_matches_oracle_and_self_dual_point():
    import oracle
    import paper_1105_5804_gb300 as sw
    cases = [(2, 0.5 * math.log(1 + math.sqrt(2)), sw.SW_CONV_AUTO), (2, 0.3, sw.SW_CONV_POTTS),
             (3, math.log(1 + math.sqrt(3)), sw.SW_CONV_AUTO), (4, math.log(3.0), sw.SW_CONV_POTTS),
             (2, 0.0, sw.SW_CONV_ISING), (5, 900.0, sw.SW_CONV_POTTS)]
    for q, beta, conv in cases:
        T = sw.sw_threshold_for(q, beta, 1.0, conv)
        assert T == oracle.threshold(oracle.coupling_K(q, beta, 1.0, conv))
    assert sw.sw_threshold_for(2, 400.0) == 1 << 32


@pytest.mark.parametrize("L,q", [(0, 2), (6, 2), (3, 2), (46344, 2), (64, 1), (64, 128)])
def test_create_rejects_bad_arguments_before_touching_the_device(L, q):
    import paper_1105_5804_gb300 as sw
    with pytest.raises(sw.SwcclError) as ei:
        sw.sw_create(L, q, 0.4, 1)
    assert ei.value.code == sw.SW_ERR_ARG
    assert sw.sw_last_error()


def test_create_rejects_bad_beta_and_threshold(lib):
    import paper_1105_5804_gb300 as sw
    with pytest.raises(sw.SwcclError):
        sw.sw_create_ex(64, 2, -1.0, 1.0, 0, 1, False)
    with pytest.raises(sw.SwcclError):
        sw.sw_create_ex(64, 2, float("nan"), 1.0, 0, 1, False)
    with pytest.raises(sw.SwcclError):
        sw.sw_create_threshold(64, 2, (1 << 32) + 1, 1, False)


def test_workspace_size_validation():
    import paper_1105_5804_gb300 as sw
    assert sw.ccl_workspace_bytes(0, 5) == -1
    assert sw.ccl_workspace_bytes(1 << 16, 1 << 16) == -1
    assert sw.ccl_workspace_bytes(1, 1) > 0
    # two int32 per site (pair lists / root lists, hook logs) plus small seam records
    b = sw.ccl_workspace_bytes(4096, 4096)
    assert 8 * 4096 * 4096 <= b < 8.5 * 4096 * 4096


def _header_define(name):
    """Integer value of a `#define NAME <expr>` of include/swccl.h (C integer
    suffixes dropped)."""
    src = open(HEADER).read()
    m = re.search(r"^#define\s+%s\s+(.+?)\s*$" % name, src, flags=re.M)
    assert m, name
    expr = m.group(1).split("/*", 1)[0].strip()
    expr = re.sub(r"(?<=\d)(LL|ULL|L|U)\b", "", expr)
    return int(eval(expr, {"__builtins__": {}}))


def test_binding_constants_equal_the_header():
    import paper_1105_5804_gb300 as sw
    assert sw.CCL_NOALLOC_SCRATCH_BYTES == _header_define("CCL_NOALLOC_SCRATCH_BYTES")
    for name in ("SW_OK", "SW_ERR_ARG", "SW_ERR_OOM", "SW_ERR_CUDA", "SW_ERR_TIMEOUT", "SW_ERR_STATE",
                 "SW_CONV_AUTO", "SW_CONV_POTTS", "SW_CONV_ISING", "SW_MODE_STAGED", "SW_MODE_FUSED",
                 "SW_BATCH_PHASES", "SW_BATCH_PERSISTENT", "SW_UPDATE_SW", "SW_UPDATE_FEW", "SW_N_PHASES"):
        assert getattr(sw, name) == _header_define(name), name


def test_batch_barrier_limit_refuses_bad_arguments(lib):
    lib.sw_batch_set_barrier_limit.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    lib.sw_batch_set_barrier_limit.restype = ctypes.c_int
    assert lib.sw_batch_set_barrier_limit(None, 0) == 1          # SW_ERR_ARG


def test_sweep_io_refuses_bad_arguments_on_the_host():
    """sw_sweep_io checks its handle and sweep count before touching the
    device (this runs without a GPU)."""
    from paper_1105_5804_gb300 import _lib
    L = _lib.lib()
    assert L.sw_sweep_io(None, None, 1, None, None) == _lib.SW_ERR_ARG
    assert "sw_sweep_io" in L.sw_last_error().decode()
