"""C-ABI library: loads without a GPU, exports every symbol the header
declares, and rejects malformed codes on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_03567_gb300 import build, binding
    build.build_library()
    return binding


def header_functions():
    txt = open(os.path.join(ROOT, "include", "nbldpc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nbldpc_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_binding_names(lib):
    assert header_functions() == sorted(lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    for name in header_functions():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_status_strings(lib):
    for st in range(0, -8, -1):
        s = lib.nbldpc_status_string(st)
        assert s and s != "unknown status"
    assert lib.nbldpc_status_string(5) == "unknown status"


def _create(lib, q, poly, n, m, rp, ci, cf):
    with pytest.raises(lib.NbldpcError) as ei:
        lib.nbldpc_code_create(q, poly, n, m, rp, ci, cf)
    return ei.value.status


def test_rejects_bad_field(lib):
    rp, ci, cf = [0, 2], [0, 1], [1, 1]
    assert _create(lib, 6, 0x7, 2, 1, rp, ci, cf) == lib.NBLDPC_ERR_POLY      # not a power of two
    assert _create(lib, 512, 0x211, 2, 1, rp, ci, cf) == lib.NBLDPC_ERR_POLY  # too big
    assert _create(lib, 16, 0x1F, 2, 1, rp, ci, cf) == lib.NBLDPC_ERR_POLY    # x has order 5
    assert _create(lib, 4, 0x5, 2, 1, rp, ci, cf) == lib.NBLDPC_ERR_POLY      # reducible
    assert _create(lib, 8, 0x13, 2, 1, rp, ci, cf) == lib.NBLDPC_ERR_POLY     # wrong degree


def test_rejects_bad_matrix(lib):
    E = lib.NBLDPC_ERR_H
    assert _create(lib, 4, 0x7, 3, 1, [0, 1], [0], [1]) == E                   # row degree 1
    assert _create(lib, 4, 0x7, 3, 1, [0, 2], [0, 0], [1, 2]) == E             # column twice in a row
    assert _create(lib, 4, 0x7, 3, 1, [0, 2], [0, 3], [1, 2]) == E             # column out of range
    assert _create(lib, 4, 0x7, 3, 1, [0, 2], [0, 1], [1, 4]) == E             # coefficient >= q
    assert _create(lib, 4, 0x7, 3, 1, [0, 2], [0, 1], [0, 1]) == E             # zero coefficient
    assert _create(lib, 4, 0x7, 3, 1, [0, 2], [0, 1], [1, 1]) == E             # column 2 unused
    assert _create(lib, 4, 0x7, 3, 1, [1, 3], [0, 1, 2], [1, 1, 1]) == E       # row_ptr[0] != 0


def test_rejects_oversized_code(lib):
    d = 65
    assert _create(lib, 4, 0x7, d, 1, [0, d], list(range(d)), [1] * d) == lib.NBLDPC_ERR_UNSUPPORTED


def test_rejects_null_arguments(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    assert L.nbldpc_code_create(4, 7, 2, 1, None, None, None, ctypes.byref(h)) == lib.NBLDPC_ERR_ARG
    assert L.nbldpc_code_create(4, 7, 2, 1, None, None, None, None) == lib.NBLDPC_ERR_ARG
    assert L.nbldpc_code_info(None, None, None, None, None) == lib.NBLDPC_ERR_ARG
    sz = ctypes.c_size_t()
    assert L.nbldpc_decode_workspace_size(None, 1, ctypes.byref(sz)) == lib.NBLDPC_ERR_ARG
    assert L.nbldpc_decode(None, None, 1, 1, 1, None, None, None, None, 0, None) == lib.NBLDPC_ERR_ARG


def test_message_width_arguments_are_checked(lib):
    L = lib.lib()
    assert L.nbldpc_code_set_message_bits(None, 8) == lib.NBLDPC_ERR_ARG
    b = ctypes.c_int()
    assert L.nbldpc_code_get_message_bits(None, ctypes.byref(b)) == lib.NBLDPC_ERR_ARG


def test_fftspa_arguments_are_checked_without_a_device(lib):
    L = lib.lib()
    b = ctypes.c_size_t()
    assert L.nbldpc_fftspa_workspace_size(None, 4, ctypes.byref(b)) == lib.NBLDPC_ERR_ARG
    assert L.nbldpc_fftspa_decode(None, None, 4, 5, 1, None, None, None, None, None, 0, None) == lib.NBLDPC_ERR_ARG


def test_cnp_schedule_arguments_are_checked(lib):
    L = lib.lib()
    assert L.nbldpc_code_set_cnp_schedule(None, lib.NBLDPC_CNP_MINIMAL) == lib.NBLDPC_ERR_ARG
    s = ctypes.c_int()
    assert L.nbldpc_code_get_cnp_schedule(None, ctypes.byref(s)) == lib.NBLDPC_ERR_ARG


def test_server_arguments_are_checked(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    assert L.nbldpc_server_create_custom(None, 1 << 20, 2, 4, 0, ctypes.byref(h)) == lib.NBLDPC_ERR_ARG
    ex = lib.nbldpc_server_executor()          # no callbacks
    assert L.nbldpc_server_create_custom(ctypes.byref(ex), 1 << 20, 2, 4, 0, ctypes.byref(h)) == lib.NBLDPC_ERR_ARG
    assert not h.value
    n = ctypes.c_int()
    assert L.nbldpc_server_poll(None, None, 0, ctypes.byref(n)) == lib.NBLDPC_ERR_ARG
    st = lib.nbldpc_server_stats()
    assert L.nbldpc_server_stats_get(None, ctypes.byref(st)) == lib.NBLDPC_ERR_ARG
    L.nbldpc_server_destroy(None)


def test_header_and_library_from_plain_c(lib, tmp_path):
    """tests/c/abi_c99.c: the header compiles as C99 with warnings as errors, the program links
    against the library and its argument checks pass (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    libdir = os.path.dirname(lib.LIB_PATH)
    exe = str(tmp_path / "abi_c99")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                           os.path.join(here, "c", "abi_c99.c"), "-L", libdir, "-lnbldpc",
                           f"-Wl,-rpath,{libdir}", "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert "c99 abi ok" in out.stdout


def _function_body(src: str, name: str) -> str:
    m = re.search(r"\b" + name + r"\([^;{]*\)\s*\{", src)
    assert m, name
    depth, i = 1, m.end()
    while depth:
        depth += {"{": 1, "}": -1}.get(src[i], 0)
        i += 1
    return src[m.end():i]


def test_every_launching_entry_point_checks_the_device():
    """A handle's code description lives in the memory of the device it was created on: every entry
    point that queues GPU work on a handle compares the current device with it (check_device, which
    returns NBLDPC_ERR_ARG otherwise) before it queues anything.  One GPU per box here, so this is a
    check of the source: the check precedes the first launch or copy in each body."""
    csrc = os.path.join(ROOT, "paper_2508_03567_gb300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in ("nbldpc.cu", "fftspa_host.cu"))
    for name in ("nbldpc_decode", "nbldpc_decode_noalloc", "nbldpc_decode_host", "nbldpc_code_autotune",
                 "nbldpc_code_set_tuning", "nbldpc_code_set_message_bits", "nbldpc_code_set_cnp_schedule",
                 "nbldpc_fftspa_decode", "nbldpc_fftspa_decode_host", "batch_plan"):
        body = _function_body(src, name)
        assert "check_device(c)" in body, name
        first_work = min([body.find(w) for w in ("launch(", "launch_plan(", "fft_launch(", "host_chunks(",
                                                 "configure(", "cudaMemsetAsync(") if w in body] or [len(body)])
        assert body.find("check_device(c)") < first_work, name
    assert "batch_plan(jobs, n_jobs" in _function_body(src, "nbldpc_decode_batch")
