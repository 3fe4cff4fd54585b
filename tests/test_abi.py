"""C ABI checks that need no GPU: the library builds, loads, exports every
symbol include/gbbfs.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1604_02844_gb300 as gb
from paper_1604_02844_gb300 import build as lib_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbbfs.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return sorted(set(re.findall(r"\b(bfs_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return gb.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("bfs_graph_create", "bfs_graph_destroy", "bfs_run", "bfs_run_batch",
                     "bfs_submit", "bfs_poll", "bfs_server_create", "bfs_graph_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", gb.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(gb.SIGNATURES) == set(header_functions())


def test_abi_version(lib):
    assert gb.bfs_abi_version() == 1


def test_host_side_argument_errors(lib):
    ro = np.array([0, 1, 2], np.int32)
    col = np.array([1, 0], np.int32)
    # n out of range, missing col_idx: rejected before any CUDA call
    assert not lib.bfs_graph_create(ro.ctypes.data, col.ctypes.data, 0, 2)
    assert lib.bfs_last_status() == gb.BFS_ERR_INVALID_ARG
    assert "n" in gb.last_error()
    assert not lib.bfs_graph_create(ro.ctypes.data, None, 2, 2)
    assert lib.bfs_last_status() == gb.BFS_ERR_INVALID_ARG
    assert not lib.bfs_graph_create(None, col.ctypes.data, 2, 2)
    # sizes past the 32-bit index headroom (2^31 - 2^24), also before any access
    top = (1 << 31) - (1 << 24)
    assert not lib.bfs_graph_create(ro.ctypes.data, col.ctypes.data, top + 1, 2)
    assert lib.bfs_last_status() == gb.BFS_ERR_INVALID_ARG
    assert not lib.bfs_graph_create(ro.ctypes.data, col.ctypes.data, 2, top + 1)
    assert lib.bfs_last_status() == gb.BFS_ERR_INVALID_ARG
    assert lib.bfs_run(None, 0, None, None, None) == gb.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_status(None) == gb.BFS_ERR_INVALID_ARG
    assert lib.bfs_run_batch(None, None, 0, None) == gb.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_set_option(None, gb.BFS_OPT_BLOCK, 512) == gb.BFS_ERR_INVALID_ARG
    assert lib.bfs_graph_destroy(None) == gb.BFS_OK
    with pytest.raises(gb.BfsError):
        gb.bfs_graph_create(ro, col, 0, 2)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(gb, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gb.load(str(tmp_path / "nope.so"))


def test_every_declaration_states_its_provenance():
    """Each entry point's comment (the nearest one above it) cites the passage
    of the paper that defines the operation, or says that it is not in the
    paper."""
    import re
    src = open(HEADER).read()
    cites = ("Sec.", "Alg.", "Table", "Listing", "not in the paper")
    missing = []
    for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(bfs_\w+)\s*\(", src, re.M):
        head = src[:m.start()]
        last = head.rfind("*/")
        comment = head[head.rfind("/*", 0, last):last] if last >= 0 else ""
        if not any(c in comment for c in cites):
            missing.append(m.group(1))
    assert not missing, f"declarations without a cited passage: {missing}"


def test_server_wait_timeout_and_failure(monkeypatch):
    """Server.wait on a stand-in poll: returns when done, raises TimeoutError
    past its limit, and passes a failed query's error on."""
    s = gb.Server.__new__(gb.Server)  # no native server: poll is replaced below
    s.handle, s._keep = None, {}
    calls = {"n": 0}

    def done_after_three(handle, ticket):
        calls["n"] += 1
        return gb.BFS_OK if calls["n"] >= 3 else gb.BFS_NOT_READY

    monkeypatch.setattr(gb, "bfs_poll", done_after_three)
    s.wait(1)
    assert calls["n"] == 3
    monkeypatch.setattr(gb, "bfs_poll", lambda h, t: gb.BFS_NOT_READY)
    with pytest.raises(TimeoutError):
        s.wait(2, sleep_s=0.001, timeout_s=0.05)

    def failed(handle, ticket):
        raise gb.BfsError(gb.BFS_ERR_TIMEOUT, "a device-side wait ran out")

    monkeypatch.setattr(gb, "bfs_poll", failed)
    with pytest.raises(gb.BfsError):
        s.wait(3)


def test_ticket_info_layout_matches_the_header(tmp_path):
    """The binding's bfs_ticket_record structure has the C layout (size and
    field offsets printed by a program compiled against the header)."""
    import ctypes
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "gbbfs.h"\n'
                   "int main(void) { printf(\"%zu\", sizeof(bfs_ticket_record));\n"
                   + "".join(f'  printf(" %zu", offsetof(bfs_ticket_record, {f}));\n'
                             for f, _ in gb.TicketInfo._fields_)
                   + "  return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(gb.TicketInfo)
    assert got[1:] == [getattr(gb.TicketInfo, f).offset for f, _ in gb.TicketInfo._fields_]


def test_binding_sets_one_hardware_queue_per_stream_by_default():
    """Importing the binding first gives the process 32 CUDA hardware work
    queues (unless the caller chose a value), so that the serving loop's
    per-graph streams do not queue behind each other; an explicit setting is
    left alone."""
    code = ("import os, sys; sys.path.insert(0, {root!r}); "
            "import paper_1604_02844_gb300; print(os.environ.get('CUDA_DEVICE_MAX_CONNECTIONS'))")
    env = {k: v for k, v in os.environ.items() if k != "CUDA_DEVICE_MAX_CONNECTIONS"}
    out = subprocess.run(["python", "-c", code.format(root=ROOT)], env=env, capture_output=True, text=True,
                         check=True).stdout.strip()
    assert out == "32"
    env["CUDA_DEVICE_MAX_CONNECTIONS"] = "4"
    out = subprocess.run(["python", "-c", code.format(root=ROOT)], env=env, capture_output=True, text=True,
                         check=True).stdout.strip()
    assert out == "4"


def test_bounds_checking_build_exports_every_declared_symbol():
    """The bounds-checking build (-DBFS_BOUNDS_CHECK) compiles from the same
    sources and exports the same C ABI, so any caller can load it instead
    (GBBFS_LIB for the Python binding)."""
    path = lib_build.build_checked()
    assert path != gb.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing
