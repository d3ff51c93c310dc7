"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/qcpd.h declares; the ctypes structs match the
header's layout.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(qcp_[a-z0-9_]+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_17522_gb300.buildlib import build
    build()
    from paper_2508_17522_gb300 import _native
    return _native.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(lib, n), f"{n} missing from libqcpd.so"


def test_options_defaults_without_gpu(lib):
    from paper_2508_17522_gb300 import _native as N
    o = N.qcp_options()
    lib.qcp_default_options(ctypes.byref(o))
    assert o.solver == 0 and o.rtol == 1e-10 and o.maxiter == 100000 and o.check_every == 32
    assert lib.qcp_version() >= 100
    assert lib.qcp_plan_destroy(None) == 0


def test_struct_layout():
    from paper_2508_17522_gb300 import _native as N
    assert ctypes.sizeof(N.qcp_csr) == 48
    assert ctypes.sizeof(N.qcp_cone) == 32
    assert ctypes.sizeof(N.qcp_problem) == 16 + 3 * 48 + 24 + 32
    assert ctypes.sizeof(N.qcp_options) == 72
    assert ctypes.sizeof(N.qcp_info) == 40


def test_built_for_sm103a_only():
    from paper_2508_17522_gb300 import buildlib
    assert buildlib.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_argument_errors_without_gpu(lib):
    """Calls the header documents as QCP_ERR_ARG on bad arguments return it
    before any device work, with a message in qcp_last_error."""
    from paper_2508_17522_gb300 import _native as N
    QCP_ERR_ARG = 1
    o = N.qcp_options()
    lib.qcp_default_options(ctypes.byref(o))
    info = (N.qcp_info * 2)()
    assert lib.qcp_derivative_jvp(None, ctypes.byref(o), *([None] * 7), info) == QCP_ERR_ARG
    assert lib.qcp_derivative_vjp(None, ctypes.byref(o), *([None] * 7), info) == QCP_ERR_ARG
    assert lib.qcp_derivative_jvp_vjp_multi(None, ctypes.byref(o), 1, *([None] * 7), 1, *([None] * 7),
                                            info) == QCP_ERR_ARG
    assert lib.qcp_plan_set_cluster(None, 4) == QCP_ERR_ARG
    assert lib.qcp_plan_set_equilibration(None, 3) == QCP_ERR_ARG
    assert lib.qcp_plan_set_schedule(None, 4096, 512, 1 << 20) == QCP_ERR_ARG
    assert lib.qcp_plan_set_barrier_wait(None, 16, 0) == QCP_ERR_ARG
    assert lib.qcp_plan_set_stream_pairing(None, 1) == QCP_ERR_ARG
    shared = ctypes.c_int64()
    assert lib.qcp_plan_last_shared_passes(None, ctypes.byref(shared)) == QCP_ERR_ARG
    cnt = ctypes.c_int32()
    assert lib.qcp_plan_autotune(None, ctypes.byref(o), 0, 1, 16, None, 0, ctypes.byref(cnt), None) == QCP_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.qcp_plan_create(None, None, 0, 1, None, ctypes.byref(out)) == QCP_ERR_ARG
    assert lib.qcp_plan_last_engine(None) == -1
    assert lib.qcp_plan_last_launches(None) == 0
    assert b"" != N.lib().qcp_last_error()


def test_header_is_plain_c():
    """include/qcpd.h compiles as strict C99 (no C++ or torch types leak
    into the boundary) and as C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    tmp = os.path.join(ROOT, ".tmp", f"hdr_{os.getpid()}")
    os.makedirs(tmp, exist_ok=True)
    try:
        src = os.path.join(tmp, "use_header.c")
        with open(src, "w") as f:
            f.write('#include "qcpd.h"\n'
                    "int main(void) { qcp_options o; qcp_default_options(&o); return (int)o.maxiter; }\n")
        env = dict(os.environ, TMPDIR=tmp)
        for cmd in ([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror"],
                    [gcc, "-x", "c++", "-std=c++17", "-Wall", "-Werror"]):
            out = subprocess.run(cmd + ["-I", os.path.join(ROOT, "include"), "-c", src, "-o",
                                        os.path.join(tmp, "use_header.o")], capture_output=True, text=True, env=env)
            assert out.returncode == 0, out.stderr
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
