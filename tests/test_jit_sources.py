"""CPU checks of the run-time specialised sweeps: the embedded device headers
compile under NVRTC for sm_103a with the three class thresholds as constants,
for every sweep variant that names a specialised form and for the
checkerboard kernel, and the host-side controls behave (no GPU needed:
compiling emits a cubin, nothing is launched).
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_1908_07341_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1908_07341_gb300", "csrc")


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC not loadable")


def _name_expressions():
    """The specialised kernel names of the sweep variant tables."""
    with open(os.path.join(CSRC, "kernels.cu")) as f:
        text = f.read()
    out = []
    for kernel, args in re.findall(r'SHK_JIT_NAMES\((\w+),\s*"([^"]+)"\)', text):
        if kernel == "kernel":
            continue   # the macro's own definition
        out += [f"shk::{kernel}<0, {args}>", f"shk::{kernel}<1, {args}>"]
    # launch shapes that differ only in grid size share their kernels
    return list(dict.fromkeys(out))


def _compile(nv, names, U):
    from paper_1908_07341_gb300 import build
    headers = build.JIT_SOURCES
    texts = []
    for h in headers:
        with open(os.path.join(CSRC, h), "rb") as f:
            texts.append(f.read())
    prog = ctypes.c_void_p()
    hn = (ctypes.c_char_p * len(headers))(*[h.encode() for h in headers])
    ht = (ctypes.c_char_p * len(headers))(*texts)
    assert nv.nvrtcCreateProgram(ctypes.byref(prog), b'#include "sweep_kernels.cuh"\n#include "checkerboard.cuh"\n',
                                 b"shk_jit.cu", len(headers), ht, hn) == 0
    for n in names:
        assert nv.nvrtcAddNameExpression(prog, n.encode()) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17"] + [f"-DSHK_JIT_U{i}={u}u".encode()
                                                             for i, u in enumerate(U)]
    rc = nv.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    sz = ctypes.c_size_t()
    nv.nvrtcGetProgramLogSize(prog, ctypes.byref(sz))
    log = ctypes.create_string_buffer(sz.value + 1)
    nv.nvrtcGetProgramLog(prog, log)
    lowered = []
    cubin = 0
    if rc == 0:
        for n in names:
            p = ctypes.c_char_p()
            assert nv.nvrtcGetLoweredName(prog, n.encode(), ctypes.byref(p)) == 0
            lowered.append(p.value.decode())
        c = ctypes.c_size_t()
        assert nv.nvrtcGetCUBINSize(prog, ctypes.byref(c)) == 0
        cubin = c.value
    nv.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace"), lowered, cubin


def test_variant_tables_name_specialised_forms():
    names = _name_expressions()
    # distinct kernels; bit-packed: queue-v4 (one, two or four waves), queue x3, queue-v2,
    # queue-v4 x2, strip-async, strip, queue-128, queue x4; int8: strip-async (one or two waves), strip-bulk,
    # strip, queue x2
    assert len(names) == 2 * 13
    assert "shk::k_sweep_strip_bulk<0, 256, 3, 4>" in names
    assert "shk::k_sweep_qv<1, 4, 256, 2>" in names
    assert "shk::k_sweep_q<0, 1, 256, 3>" in names
    assert "shk::k_sweep_strip_async<1, 2, 256, 3, 2>" in names


def test_embedded_sources_compile_under_nvrtc():
    nv = _nvrtc()
    # thresholds of q = J = 0.5 from the library's own table: the s = +1 half (T[3], T[4], T[5])
    T = (ctypes.c_uint32 * 6)()
    assert _lib.lib().shk_thresholds(0.5, 0.5, T) == _lib.OK
    U = [T[3], T[4], T[5]]
    names = _name_expressions() + ["shk::k_checkerboard<0>", "shk::k_checkerboard<1>"]
    rc, log, lowered, cubin = _compile(nv, names, U)
    assert rc == 0, log
    assert cubin > 0
    assert len(set(lowered)) == len(names)
    assert all(n.startswith("_ZN3shk") for n in lowered)


def test_extreme_thresholds_compile():
    # all-zero and all-one thresholds (q, J at the edges of the table) fold to
    # constant masks too
    nv = _nvrtc()
    names = _name_expressions()[:2]
    for U in ([0, 0, 0], [0xFFFFFFFF] * 3, [0, 0x80000000, 0xFFFFFFFF]):
        rc, log, _, cubin = _compile(nv, names, U)
        assert rc == 0 and cubin > 0, log


def test_specialize_controls_host_only():
    so = _lib.lib()
    c, f, qd = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1)
    buf = ctypes.create_string_buffer(64)
    assert so.shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(qd), None, buf, 64) == _lib.OK
    assert c.value >= 0 and f.value >= 0 and qd.value >= 0
    assert so.shk_specialize_status(None, None, None, None, None, 0) == _lib.OK
    for mode in (0, 2, 1):
        assert so.shk_set_specialize(mode) == _lib.OK
    assert so.shk_set_specialize(3) == _lib.EINVAL
    assert so.shk_set_specialize(-1) == _lib.EINVAL


def test_prepare_compiles_without_a_gpu():
    _nvrtc()
    so = _lib.lib()
    assert so.shk_specialize_prepare(_lib.BITPACK, 0, 0.9, 0.41, 1) == _lib.OK
    c, f, qd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    secs = ctypes.c_double()
    assert so.shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(qd), ctypes.byref(secs),
                                    None, 0) == _lib.OK
    assert c.value >= 1 and f.value == 0 and secs.value > 0
    # the same table again is already there
    assert so.shk_specialize_prepare(_lib.BITPACK, 0, 0.9, 0.41, 1) == _lib.OK
    c2 = ctypes.c_int()
    so.shk_specialize_status(ctypes.byref(c2), None, None, None, None, 0)
    assert c2.value == c.value
    n_bp = so.shk_sweep_variant_count(_lib.BITPACK)
    assert so.shk_specialize_prepare(_lib.BITPACK, n_bp - 1, 0.9, 0.41, 1) == _lib.EINVAL   # plain: none
    assert b"no specialised form" in so.shk_last_error(None)
    assert so.shk_specialize_prepare(_lib.BITPACK, n_bp, 0.9, 0.41, 1) == _lib.EINVAL
    assert so.shk_specialize_prepare(_lib.INT8, 0, float("nan"), 0.41, 1) == _lib.EINVAL
    assert so.shk_set_specialize(0) == _lib.OK
    try:
        assert so.shk_specialize_prepare(_lib.BITPACK, 0, 0.9, 0.41, 1) == _lib.ESTATE
    finally:
        so.shk_set_specialize(1)


_EXIT_CHILD = r"""
import ctypes, sys, time
so = ctypes.CDLL(sys.argv[1])
so.shk_specialize_prepare.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
for k in range(3):
    assert so.shk_specialize_prepare(1, 0, 0.5 + 0.01 * k, 0.3, 0) == 0
time.sleep(float(sys.argv[2]))
print("exiting", flush=True)
"""


_EXIT_CHILD_BINDING = r"""
import sys, time
from paper_1908_07341_gb300 import _lib
so = _lib.lib()
for k in range(3):
    assert so.shk_specialize_prepare(_lib.BITPACK, 0, 0.7 + 0.01 * k, 0.3, 0) == 0
time.sleep(float(sys.argv[1]))
print("exiting", flush=True)
"""


@pytest.mark.parametrize("delay", [0.0, 0.15, 0.4, 0.8])
def test_exit_during_a_background_compile_is_clean(delay):
    """A process that exits while compiles are queued or running waits for
    the one in flight and exits normally (no crash or hang in NVRTC's exit
    handlers): through the C exit handler (plain ctypes), and through the
    binding's interpreter-exit hook."""
    _nvrtc()
    r = subprocess.run([sys.executable, "-c", _EXIT_CHILD, _lib.LIB_PATH, str(delay)], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    assert "exiting" in r.stdout
    r = subprocess.run([sys.executable, "-c", _EXIT_CHILD_BINDING, str(delay)], capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
    assert "exiting" in r.stdout


def test_shutdown_stops_background_compiles():
    _nvrtc()
    child = r"""
import ctypes, sys
so = ctypes.CDLL(sys.argv[1])
so.shk_specialize_prepare.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
assert so.shk_specialize_prepare(1, 0, 0.61, 0.3, 0) == 0      # first compile: on this thread
assert so.shk_specialize_prepare(1, 0, 0.62, 0.3, 0) == 0      # background
assert so.shk_specialize_shutdown() == 0                        # waits for it
assert so.shk_specialize_shutdown() == 0                        # idempotent
c, f, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
so.shk_specialize_status(ctypes.byref(c), ctypes.byref(f), ctypes.byref(q), None, None, 0)
assert q.value <= 1 and f.value == 0, (c.value, f.value, q.value)
assert so.shk_specialize_prepare(1, 0, 0.63, 0.3, 0) != 0      # nothing new after shutdown
print("ok", c.value, q.value)
"""
    r = subprocess.run([sys.executable, "-c", child, _lib.LIB_PATH], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, (r.returncode, r.stdout, r.stderr[-2000:])


def test_forked_child_does_not_wait_for_compiles():
    """A child forked after the compile thread started has no such thread: its
    blocking requests return at once instead of waiting for ever."""
    _nvrtc()
    child = r"""
import ctypes, os, sys
so = ctypes.CDLL(sys.argv[1])
so.shk_specialize_prepare.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int]
assert so.shk_specialize_prepare(1, 0, 0.71, 0.3, 1) == 0      # first compile, starts the thread
assert so.shk_specialize_prepare(1, 0, 0.72, 0.3, 0) == 0      # queued in the background
pid = os.fork()
if pid == 0:
    rc = so.shk_specialize_prepare(1, 0, 0.73, 0.3, 1)         # must not block
    os._exit(0 if rc != 0 else 3)
_, status = os.waitpid(pid, 0)
assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0, status
assert so.shk_specialize_prepare(1, 0, 0.74, 0.3, 1) == 0      # the parent still compiles
print("ok")
"""
    r = subprocess.run([sys.executable, "-W", "ignore", "-c", child, _lib.LIB_PATH], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, (r.returncode, r.stdout, r.stderr[-2000:])
