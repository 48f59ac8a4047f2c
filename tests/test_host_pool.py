"""The host worker pool of the batched solves (csrc/host_pool.cpp), compiled
for the host by g++ (tests/host_pool_shim.cpp): every task of a job runs
exactly once, jobs follow one another without mixing, n = 0 and n = 1 work,
and with SBCI_HOST_THREADS=0 everything runs on the calling thread."""
import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so_path(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ is missing")
    out = str(tmp_path_factory.mktemp("pool") / "libpoolhost.so")
    csrc = os.path.join(ROOT, "paper_2603_06101_gb300", "csrc")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I" + csrc,
                    os.path.join(ROOT, "tests", "host_pool_shim.cpp"), os.path.join(csrc, "host_pool.cpp"),
                    "-o", out], check=True)
    return out


def _run(lib, jobs, n):
    counts = np.zeros(jobs * n, dtype=np.int32)
    threads = np.full(jobs * n, -1, dtype=np.int32)
    nt = lib.host_pool_run(jobs, n, counts.ctypes.data, threads.ctypes.data)
    return nt, counts, threads


def test_every_task_once(so_path):
    lib = ctypes.CDLL(so_path)
    lib.host_pool_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    for jobs, n in [(1, 0), (3, 1), (5, 16), (50, 7), (4, 200)]:
        nt, counts, threads = _run(lib, jobs, n)
        assert np.all(counts == 1), (jobs, n)
        if n:
            assert threads.min() >= 0
    if (os.cpu_count() or 1) > 2:
        nt, _, _ = _run(lib, 2, 64)
        assert nt > 1  # the workers take part


def test_single_thread_when_disabled(so_path):
    code = ("import ctypes, numpy as np; L = ctypes.CDLL(%r); "
            "L.host_pool_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]; "
            "c = np.zeros(64, dtype=np.int32); t = np.zeros(64, dtype=np.int32); "
            "nt = L.host_pool_run(2, 32, c.ctypes.data, t.ctypes.data); "
            "assert nt == 1 and (c == 1).all(), (nt, c)") % so_path
    env = dict(os.environ, SBCI_HOST_THREADS="0")
    subprocess.run([sys.executable, "-c", code], check=True, env=env)
