"""The debug-check build, a stand-in for a memory sanitizer: kernels compiled
with FNR_DEBUG_CHECKS check their list indices, TMA coordinates and launch
layout and record a failure as IR_ECHECK instead of faulting. A parity sweep runs against that build in a separate
process, so this process keeps the release library."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
def test_debug_check_build_sweep():
    from paper_1201_3972_gb300 import _build
    path = _build.build_debug()
    env = dict(os.environ, IRFNR_LIBRARY=path)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_sweep.py")], env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "no kernel check failed" in r.stdout


def test_debug_check_build_compiles():
    """One kernel unit of the library compiles with the debug checks (nvcc only, no GPU)."""
    from paper_1201_3972_gb300 import _build
    root = os.path.dirname(HERE)
    src = os.path.join(root, "paper_1201_3972_gb300", "csrc", "fnr_inst_k5_7.cu")
    out = os.path.join(root, "_build", "debug_check_probe.o")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    try:
        nvcc = _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    r = subprocess.run([nvcc] + _build.NVCC_FLAGS + ["-DFNR_DEBUG_CHECKS", "-c", src, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
