"""The C ABI from plain C (tests/c_client/gvm_c_client.c): the client builds
against include/gvm.h and libgvm.so with gcc (CPU test), and on a GPU its
results match the CPU oracle (vector add bit-exact, SGEMM within the split
bound)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

SRC = os.path.join(ROOT, "tests", "c_client", "gvm_c_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    import __graft_entry__

    __graft_entry__.build()
    from paper_1511_07658_gb300 import lib_path

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    libdir = os.path.dirname(lib_path())
    exe = str(tmp_path_factory.mktemp("cclient") / "gvm_c_client")
    cmd = [gcc, "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-I",
           os.path.join(CUDA, "include"), SRC, "-o", exe, "-L", libdir, "-lgvm", "-Wl,-rpath," + libdir,
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    assert os.path.exists(os.path.join(libdir, "libgvm.so"))
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_client_builds(client):
    assert os.access(client, os.X_OK)


@pytest.mark.gpu
def test_c_client_runs_and_matches_the_oracle(client, tmp_path):
    import oracle
    import synth
    from sgemm_bounds import check_sgemm

    n, m, k, nn = 100003, 130, 257, 200
    a, b = synth.vadd_inputs(synth.task_seed(0, 77), n)
    A, B = synth.sgemm_inputs(synth.task_seed(1, 77), m, nn, k)
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(np.int64(n).tobytes() + np.array([m, k, nn], np.int32).tobytes())
        for x in (a, b, A, B):
            f.write(np.ascontiguousarray(x, np.float32).tobytes())
    r = subprocess.run([client, str(fin), str(fout)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(fout, dtype=np.float32)
    c, C = out[:n], out[n:].reshape(m, nn)
    assert np.array_equal(c.view(np.uint32), oracle.vadd(a, b).view(np.uint32))
    check_sgemm(C, A, B)
