"""The C-ABI library builds, loads and exports every entry point that
include/gh.h declares; host-side argument checks and fault injection work
without a GPU."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\s*(?:gh_status|long long|int|const char\s*\*)\s+(gh_\w+)\s*\(", text, re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09101_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_core_entry_points():
    names = set(_declared())
    for n in ["gh_create_domain", "gh_destroy_domain", "gh_set_analytic_kerr_schild", "gh_rhs",
              "gh_rk4_step", "gh_constraints", "gh_derivatives", "gh_apply_filters", "gh_sync"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def _run_create(env_extra, shells_expr):
    code = r"""
import ctypes, sys
sys.path.insert(0, %r)
from paper_1804_09101_gb300 import gh
P = gh.gh_params(1.0, -1.0, 1.0, 36.0, 32, 0, -1)
shells = %s
arr = (gh.gh_shell * len(shells))(*[gh.gh_shell(*s) for s in shells])
h = ctypes.c_void_p()
st = gh.library().gh_create_domain(arr, len(shells), ctypes.byref(P), None, ctypes.byref(h))
print(st, gh.library().gh_last_error(None).decode())
""" % (ROOT, shells_expr)
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    st, _, msg = r.stdout.strip().partition(" ")
    return int(st), msg


def test_invalid_shells_are_rejected_before_any_device_call(lib):
    st, msg = _run_create({}, "[(2.0, 1.0, 11, 7)]")
    assert st == 1 and "r_in" in msg                      # GH_EINVAL
    st, msg = _run_create({}, "[(1.0, 2.0, 11, 7), (2.5, 3.0, 11, 7)]")
    assert st == 1 and "does not start" in msg
    st, msg = _run_create({}, "[(1.0, 2.0, 2, 7)]")
    assert st == 1


def test_injected_allocation_fault_returns_enomem_without_touching_the_gpu(lib):
    st, msg = _run_create({"GH_FAULT": "alloc"}, "[(1.0, 2.0, 11, 7)]")
    assert st == 2 and "GH_FAULT" in msg                  # GH_ENOMEM


def test_schedule_entry_points_reject_bad_arguments_on_the_host(lib):
    v = (ctypes.c_int * 9)(2, 1, 2, 1, 128, 49152, 128, 49152, 0)
    lib.gh_get_schedule.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.gh_set_schedule.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.gh_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.gh_get_schedule(None, v, 9) == 1          # GH_EINVAL: no domain
    assert lib.gh_set_schedule(None, v, 9) == 1
    assert lib.gh_autotune(None, 3) == 1


def test_overlap_switch_rejects_bad_arguments_on_the_host(lib):
    lib.gh_set_overlap.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.gh_set_overlap(None, 1) == 1              # GH_EINVAL: no domain


def test_binding_fails_loudly_without_the_library(tmp_path):
    """A copy of the package without libgh.so: importing the binding raises
    instead of falling back to anything."""
    import shutil
    src = os.path.join(ROOT, "paper_1804_09101_gb300")
    shutil.copytree(src, str(tmp_path / "paper_1804_09101_gb300"),
                    ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_1804_09101_gb300.gh"], cwd=str(tmp_path),
                       capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0 and "libgh.so not built" in r.stderr, r.stderr[-500:]


def test_host_step_rejects_bad_arguments_on_the_host(lib):
    lib.gh_rk4_step_host.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    buf = (ctypes.c_double * 4)()
    assert lib.gh_rk4_step_host(None, 0.1, 1, buf, buf, None) == 1     # GH_EINVAL: no domain
