"""The C-ABI library builds, loads and exports what include/*.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from conftest import ROOT

HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(gvm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    return g


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ["gvm_init", "gvm_attach", "gvm_submit", "gvm_sync", "gvm_shutdown", "gvm_vadd_f32", "gvm_sgemm_f32"]:
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = built.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gvm_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported
    # Nothing beyond the declared C ABI leaks out of the library.
    assert exported <= set(declared_functions())


def test_python_binding_covers_the_abi(built):
    from paper_1511_07658_gb300 import _abi

    assert set(_abi.PROTOTYPES) == set(declared_functions())


def test_struct_layouts_match_c(built, tmp_path):
    from paper_1511_07658_gb300 import GvmConfig, GvmStats, GvmTask
    from paper_1511_07658_gb300._abi import GvmIpcTask

    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "gvm.h"\n#include "gvm_ipc.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(gvm_config), sizeof(gvm_task),"
        " sizeof(gvm_stats), offsetof(gvm_config, copy_streams), offsetof(gvm_config, ingest_quantum),"
        " offsetof(gvm_task, c_off), offsetof(gvm_stats, device_where), sizeof(gvm_ipc_task),"
        " offsetof(gvm_ipc_task, c_off)); return 0;}\n"
    )
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [
        ctypes.sizeof(GvmConfig),
        ctypes.sizeof(GvmTask),
        ctypes.sizeof(GvmStats),
        GvmConfig.copy_streams.offset,
        GvmConfig.ingest_quantum.offset,
        GvmTask.c_off.offset,
        GvmStats.device_where.offset,
        ctypes.sizeof(GvmIpcTask),
        GvmIpcTask.c_off.offset,
    ]
    assert vals == want


def test_host_only_calls_without_gpu(built):
    from ctypes import byref, c_void_p

    from paper_1511_07658_gb300 import GVM_EINVAL, GvmConfig, lib

    L = lib()
    assert L.gvm_strerror(0) == b"ok"
    assert L.gvm_strerror(-3).startswith(b"ring slot")
    cfg = GvmConfig()
    cfg.max_ranks, cfg.ring_depth, cfg.mode, cfg.sgemm_path = 16, 64, 0, 1
    assert L.gvm_ctrl_bytes(byref(cfg)) > 16 * 64 * 512
    for mode in (1, 2, 3):  # continuous, PS-1, PS-2
        cfg.mode = mode
        assert L.gvm_ctrl_bytes(byref(cfg)) > 0
    cfg.mode = 4
    assert L.gvm_ctrl_bytes(byref(cfg)) == 0
    cfg.mode = 0
    cfg.ring_depth = 63  # not a power of two
    assert L.gvm_ctrl_bytes(byref(cfg)) == 0
    h = c_void_p()
    assert L.gvm_init(byref(cfg), byref(h)) == GVM_EINVAL
    assert L.gvm_sgemm_scratch_bytes(512, 512, 512, 1) == 4 * (512 + 512) * 512
    assert L.gvm_sgemm_scratch_bytes(512, 512, 512, 0) == 0
    assert L.gvm_sgemm_scratch_bytes(0, 5, 5, 1) == 0
    assert L.gvm_vadd_f32(None, None, None, -1, None) == GVM_EINVAL
    assert L.gvm_vadd_f32(None, None, None, 0, None) == 0
    assert L.gvm_vmul_f32(None, None, None, 0, 15, None) == 0
    assert L.gvm_vmul_f32(None, None, None, 0, 0, None) == GVM_EINVAL
    assert L.gvm_vmul_f32(None, None, None, 16, 1025, None) == GVM_EINVAL
    assert L.gvm_sgemm_f32(None, None, None, 0, 4, 4, 0, None, 0, None) == GVM_EINVAL
    assert L.gvm_attach(None, 0, byref(h)) == GVM_EINVAL
    assert L.gvm_submit(None, None, None) == GVM_EINVAL


def test_no_oracle_on_product_path():
    """The product package neither imports nor loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1511_07658_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library every entry point raises; nothing falls back."""
    code = (
        "import paper_1511_07658_gb300 as g\n"
        "import torch\n"
        "for call in (lambda: g._abi.lib(), lambda: g.vadd_f32(torch.ones(4), torch.ones(4), torch.ones(4), 0)):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'libgvm.so not found' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('no error')\n"
        "print('ok')\n"
    )
    env = dict(os.environ, GVM_LIB=str(tmp_path / "absent" / "libgvm.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr[-2000:]
