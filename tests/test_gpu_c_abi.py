"""The C ABI used from plain C: tests/c_abi/abi_client.c is compiled against
include/ir_filter.h and linked with libirfnr.so, the CUDA runtime and the C
oracle (test infrastructure), then run; it checks run2, run and a batch bit
for bit against the oracle and exits non-zero on any difference."""
import os
import subprocess

import pytest

from paper_1201_3972_gb300 import _build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_client_bit_exact(tmp_path):
    _build.build()
    exe = str(tmp_path / "abi_client")
    lib_dir = os.path.dirname(_build.LIB_PATH)
    cmd = [_build.nvcc(), "-O2", "-o", exe, os.path.join(HERE, "c_abi", "abi_client.c"),
           os.path.join(ROOT, "oracle", "fnr_oracle.c"), "-I", os.path.join(ROOT, "include"),
           "-L", lib_dir, "-lirfnr", "-Xlinker", f"-rpath={lib_dir}", "-lcudart", "-Xcompiler", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "bit-exact" in run.stdout
