"""Host-side checks of the C-ABI library (no GPU work): it builds, loads and exports every
entry point include/dfs.h declares; the binding refuses to run without it."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dfs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfs_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2310_17556_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dfs_solve", "dfs_solve_batched", "dfs_gram", "dfs_cholesky", "dfs_trsm", "dfs_fisher_pass",
                     "dfs_solve_host", "dfs_create", "dfs_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dfs_[a-z_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_ctypes_loads_and_binds(libpath):
    from paper_2310_17556_gb300 import _lib

    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name)
    assert set(_lib.EXPORTS) == set(declared_functions())
    assert lib.dfs_status_string(2) == b"DFS_ERR_NOT_SPD"
    assert lib.dfs_status_string(0) == b"DFS_OK"


def test_every_nvcc_command_targets_sm103a_only(monkeypatch, tmp_path):
    """The build compiles and links each source for sm_103a alone: the nvcc command lines it
    issues (captured, not run) carry one -gencode, arch=compute_103a,code=sm_103a."""
    from paper_2310_17556_gb300 import build

    cmds = []

    class Done:
        returncode, stdout, stderr = 0, "", ""

    def fake_run(cmd, **kw):
        cmds.append(list(cmd))
        open(cmd[cmd.index("-o") + 1], "w").close()
        return Done()

    monkeypatch.setattr(build.subprocess, "run", fake_run)
    monkeypatch.setattr(build, "BUILD", str(tmp_path))
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libdfs.so"))
    build.build(force=True)
    assert len(cmds) == len(build._sources()) + 1  # each source, then the link
    for cmd in cmds:
        targets = [a for a in cmd if a.startswith(("arch=", "-arch", "--gpu-architecture", "-code", "--gpu-code"))]
        assert targets == ["arch=compute_103a,code=sm_103a"] and cmd.count("-gencode") == 1, cmd


def test_debug_build_has_its_own_flag_objects_and_library(monkeypatch, tmp_path):
    """--debug-bounds compiles every source with -DDFS_DEBUG_BOUNDS into its own object folder and
    links libdfs_debug.so; the release build carries no such define (commands captured, not run)."""
    from paper_2310_17556_gb300 import build

    cmds = []

    class Done:
        returncode, stdout, stderr = 0, "", ""

    def fake_run(cmd, **kw):
        cmds.append(list(cmd))
        open(cmd[cmd.index("-o") + 1], "w").close()
        return Done()

    monkeypatch.setattr(build.subprocess, "run", fake_run)
    monkeypatch.setattr(build, "BUILD", str(tmp_path / "rel"))
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libdfs.so"))
    monkeypatch.setattr(build, "BUILD_DEBUG", str(tmp_path / "dbg"))
    monkeypatch.setattr(build, "LIB_DEBUG", str(tmp_path / "libdfs_debug.so"))
    assert build.build(force=True, debug_bounds=True) == str(tmp_path / "libdfs_debug.so")
    compiles, link = cmds[:-1], cmds[-1]
    assert len(compiles) == len(build._sources())
    for cmd in compiles:
        assert "-DDFS_DEBUG_BOUNDS" in cmd and cmd[cmd.index("-o") + 1].startswith(str(tmp_path / "dbg")), cmd
    assert link[link.index("-o") + 1].startswith(str(tmp_path / "libdfs_debug.so"))
    cmds.clear()
    build.build(force=True)
    assert all("-DDFS_DEBUG_BOUNDS" not in cmd for cmd in cmds)


def test_debug_checks_guard_the_hot_kernels():
    """Each kernel source the debug build instruments holds index checks, under its own source id."""
    csrc = os.path.join(ROOT, "paper_2310_17556_gb300", "csrc")
    total = 0
    for name, sid in (("pass_cluster.cu", 1), ("pass.cu", 2), ("gram_tc.cu", 3), ("gram_fused.cu", 4),
                      ("cholesky.cu", 5), ("nspace.cu", 6)):
        text = open(os.path.join(csrc, name)).read()
        assert f"#define DFS_SRC_ID {sid}\n" in text, name
        assert text.count("DFS_IN_BOUNDS(") >= 1, name
        total += text.count("DFS_IN_BOUNDS(")
    assert total >= 15


def test_debug_library_is_selected_by_the_environment(monkeypatch, tmp_path):
    from paper_2310_17556_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_DEBUG_PATH", str(tmp_path / "libdfs_debug.so"))
    monkeypatch.setenv("DFS_DEBUG_BOUNDS", "1")
    assert _lib.lib_path() == str(tmp_path / "libdfs_debug.so")
    with pytest.raises(RuntimeError, match="--debug-bounds"):
        _lib.load()
    monkeypatch.setenv("DFS_DEBUG_BOUNDS", "0")
    assert _lib.lib_path() == _lib.LIB_PATH


def test_null_handle_is_rejected(libpath):
    from paper_2310_17556_gb300 import _lib

    lib = _lib.load()
    assert lib.dfs_destroy(None) == _lib.DFS_ERR_INVALID_ARG
    assert lib.dfs_solve(None, None, 1, 1, 1, 4, None, 1, 1, 1.0, None, 1, None, None, None) == _lib.DFS_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2310_17556_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libdfs.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()


def test_errors_print_only_with_dfs_log(libpath):
    """The library prints nothing unless DFS_LOG is set; then each recorded error goes to stderr.
    A handle for device 999 fails on any machine, before any GPU work."""
    code = ("import ctypes as C, sys\n"
            "from paper_2310_17556_gb300 import _lib\n"
            "h = C.c_void_p()\n"
            "sys.exit(0 if _lib.load().dfs_create(C.byref(h), 999) == _lib.DFS_ERR_CUDA else 1)\n")
    runs = {}
    for log in (None, "0", "1"):
        env = {k: v for k, v in os.environ.items() if k != "DFS_LOG"}
        if log is not None:
            env["DFS_LOG"] = log
        r = subprocess.run(["python", "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr
        runs[log] = r.stderr
    assert "dfs:" not in runs[None] and "dfs:" not in runs["0"]
    assert "dfs: DFS_ERR_CUDA: no CUDA device 999" in runs["1"]
