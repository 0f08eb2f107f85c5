"""The C-ABI library loads, exports every entry point include/accr.h declares,
and rejects invalid regions on the host before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1412_1127_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"ACCR_API[^;(]*?\b(accr_\w+)\s*\(", txt, flags=re.S))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    import __graft_entry__ as g
    g.build()
    return _native.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "accr_reduce" in names and "accr_rowreduce" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in _native.SIGNATURES, "binding lacks " + n


def test_only_accr_symbols_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True).stdout
    funcs = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert funcs and all(f.startswith("accr_") for f in funcs), funcs


def _clause(op, acc, out=1):
    c = _native.Clause()
    c.op, c.acc_type, c.init, c.out = op, acc, None, out
    return (_native.Clause * 1)(c)


def test_version(L):
    assert L.accr_version() == 100


@pytest.mark.parametrize("in_type,op,acc,code", [
    (2, 4, 2, _native.ACCR_ETYPE),   # & on float
    (3, 7, 3, _native.ACCR_ETYPE),   # && on double
    (1, 0, 0, _native.ACCR_ETYPE),   # int64 into int32 (narrowing)
    (0, 0, 3, _native.ACCR_ETYPE),   # int into double
    (2, 0, 0, _native.ACCR_ETYPE),   # float into int
    (0, 9, 0, _native.ACCR_EINVAL),  # not an operator
    (0, 0, 7, _native.ACCR_EINVAL),  # not a type
    (5, 0, 0, _native.ACCR_EINVAL),  # not an element type
])
def test_reduce_rejects_bad_clause_on_host(L, in_type, op, acc, code):
    rc = L.accr_reduce(None, 0, in_type, _clause(op, acc), 1, 0, None)
    assert rc == code
    assert L.accr_last_error()


def test_reduce_rejects_bad_arguments_on_host(L):
    assert L.accr_reduce(None, -1, 0, _clause(0, 0), 1, 0, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 0, 0, _clause(0, 0), 0, 0, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 0, 0, _clause(0, 0), 5, 0, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 0, 0, None, 1, 0, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 0, 0, _clause(0, 0, out=None), 1, 0, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 0, 0, _clause(0, 0), 1, 0x100, None) == _native.ACCR_EINVAL
    assert L.accr_reduce(None, 10, 0, _clause(0, 0), 1, 0, None) == _native.ACCR_EINVAL   # NULL in
    assert L.accr_reduce(ctypes.c_void_p(2), 10, 0, _clause(0, 0), 1, 0, None) == _native.ACCR_EINVAL
    assert "aligned" in L.accr_last_error().decode()


def test_rowreduce_rejects_bad_arguments_on_host(L):
    assert L.accr_rowreduce(None, 4, 8, 7, 0, _clause(0, 0), 1, 0, None) == _native.ACCR_EINVAL
    assert L.accr_rowreduce(None, -1, 8, 8, 0, _clause(0, 0), 1, 0, None) == _native.ACCR_EINVAL
    assert L.accr_rowreduce(None, 4, 8, 8, 2, _clause(5, 2), 1, 0, None) == _native.ACCR_ETYPE
    assert L.accr_rowreduce(None, 4, 8, 8, 0, _clause(0, 0), 1, 0x4, None) == _native.ACCR_EINVAL


def test_fault_inject_rejects_bad_kind(L):
    assert L.accr_fault_inject(0, 1) == _native.ACCR_EINVAL
    assert L.accr_fault_inject(4, 1) == _native.ACCR_EINVAL
    assert L.accr_fault_inject(1, -1) == _native.ACCR_EINVAL
    assert L.accr_fault_inject(2, 0) == _native.ACCR_OK


def test_submit_and_server_reject_bad_arguments_on_host(L):
    h = ctypes.c_void_p()
    assert L.accr_server_create(0, 1, 1, ctypes.byref(h)) == _native.ACCR_EINVAL
    assert L.accr_server_create(1 << 20, 0, 1, ctypes.byref(h)) == _native.ACCR_EINVAL
    assert L.accr_submit(None, None, None) == _native.ACCR_EINVAL
    assert L.accr_batch_create(None, 0, 0, None) == _native.ACCR_EINVAL
    assert L.accr_batch_tiling(17, 0, None, None) == _native.ACCR_EINVAL
    assert L.accr_matmul_nest(None, None, None, 4, 9, 0, None) == _native.ACCR_EINVAL


def _run_bad_call(env_level):
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1412_1127_gb300 import _native\n"
            "print(_native.lib().accr_reduce(None, -1, 0, None, 1, 0, None))\n") % ROOT
    env = dict(os.environ)
    env.pop("ACCR_LOG", None)
    if env_level is not None:
        env["ACCR_LOG"] = str(env_level)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=120)


def test_log_level_reports_errors_on_stderr(L):
    """ACCR_LOG=1 prints each recorded error to stderr; by default the library
    is silent.  (The failing call is rejected on the host: no GPU needed.)"""
    quiet = _run_bad_call(None)
    loud = _run_bad_call(1)
    assert quiet.returncode == 0 and loud.returncode == 0
    assert quiet.stdout.strip() == loud.stdout.strip() == str(_native.ACCR_EINVAL)
    assert "accr:" not in quiet.stderr
    assert "accr: error %d: accr_reduce: n = -1 < 0" % _native.ACCR_EINVAL in loud.stderr


def test_release_build_reports_no_bounds_checks(L):
    """accr_debug_report on the release library: no checks compiled in, nothing
    counted, and no CUDA call made (so it runs without a GPU)."""
    if os.path.basename(_native.LIB_PATH) != "libaccr.so":
        pytest.skip("another library was selected with ACCR_LIBRARY")
    from paper_1412_1127_gb300 import api
    assert api.accr_debug_report(clear=True) == (0, 0, False)
    assert api.accr_debug_report(clear=False) == (0, 0, False)
