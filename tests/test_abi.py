"""Host-side checks of the C ABI (no GPU needed): the library builds, loads
and exports every function declared in include/dsrg.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dsrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dsrg_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_00561_gb300._buildlib import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["dsrg_df_plan", "dsrg_mrpt2_energy", "dsrg_mrpt2_energy_grad", "dsrg_plan_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_python_binding_lists_every_symbol():
    from paper_1603_00561_gb300 import _native
    assert sorted(_native.EXPORTS) == _declared_functions()


def test_status_strings_without_gpu(lib):
    from paper_1603_00561_gb300 import _native
    L = _native.load()
    for st in range(7):
        assert L.dsrg_status_string(st)


def test_argument_errors_without_gpu(lib):
    """Size and pointer checks happen on the host before any device call."""
    from paper_1603_00561_gb300 import _native
    L = _native.load()
    h = ctypes.c_void_p()
    assert L.dsrg_df_plan(None, None, 0, None, 0) == _native.ERR_INVALID_ARG
    bad = [(0, 2, 10, 20), (2, -1, 10, 20), (2, 2, 0, 20), (2, 2, 10, 0)]
    for s in bad:
        sz = _native.Sizes(*s)
        assert L.dsrg_df_plan(ctypes.byref(h), ctypes.byref(sz), 0, None, 0) == \
            _native.ERR_INVALID_ARG
    sz = _native.Sizes(2, 9, 10, 20)   # nactive above the built maximum
    assert L.dsrg_df_plan(ctypes.byref(h), ctypes.byref(sz), 0, None, 0) == _native.ERR_UNSUPPORTED
    sz = _native.Sizes(2, 2, 10, 20)
    assert L.dsrg_df_plan(ctypes.byref(h), ctypes.byref(sz), 7, None, 0) == _native.ERR_INVALID_ARG
    assert L.dsrg_mrpt2_energy(None, None, None, None, None, 0.5, None) == _native.ERR_INVALID_ARG
    assert L.dsrg_plan_destroy(None) == _native.OK


def test_missing_library_raises(monkeypatch):
    """No fallback: without the compiled library the binding raises."""
    from paper_1603_00561_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError):
        _native.load(os.path.join(ROOT, "no-such-dir", "libdsrg.so"))


def test_no_cpu_path_without_gpu():
    """On a machine without a GPU the plan refuses to exist (there is no CPU path)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1603_00561_gb300 as pk
    with pytest.raises(RuntimeError):
        pk.Plan(2, 1, 10, 8)
    with pytest.raises(RuntimeError):
        pk.Batch([(2, 1, 10, 8)])
