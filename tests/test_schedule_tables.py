"""Host-side checks of the plan's gridding tables (gather lists of the FP32
kernel, round schedule of the tensor kernels): a small C++ program linked
against the library builds the tables for seeded layouts and checks that every
footprint contribution is listed exactly once, every cell of a touched row is
written exactly once per sample, and the schedules keep their bank and cell
rules.  No GPU needed."""
import os
import shutil
import subprocess

import pytest

from paper_2301_09662_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = build_lib.build()
    libdir = os.path.dirname(so)
    exe = str(tmp_path_factory.mktemp("tables") / "schedule_tables_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2301_09662_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "schedule_tables_check.cu"),
                    "-o", exe, "-L", libdir, "-lepic", "-Xlinker", "-rpath=" + libdir],
                   check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("A,K,N,C,P", [
    (256, 5, 128, 3, 2),    # LWA-like
    (256, 5, 96, 2, 2),     # folded side 48
    (256, 1, 128, 2, 2),    # point kernel (taper)
    (101, 3, 64, 2, 1),     # single polarisation: 16-lane bank groups
    (2048, 7, 512, 1, 2),   # dense: long lists
    (4096, 15, 128, 1, 1),  # limits: n_ant * n_pol = 4096, K = 15
    (64, 3, 96, 2, 1),      # folded side 48, single polarisation
    (500, 15, 96, 1, 2),    # folded side 48, footprints wider than a bank group
    (37, 1, 64, 2, 1),      # point kernel, few antennas (fewer batches than warps)
])
def test_tables(checker, A, K, N, C, P):
    r = subprocess.run([checker, str(A), str(K), str(N), str(C), str(P)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
