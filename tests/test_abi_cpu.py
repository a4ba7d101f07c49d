"""CPU-only checks of the C-ABI library and of the generated selection networks.

No compute call runs here (there is no GPU): the library must build, load,
export every entry point that include/ir_filter.h declares, and fail cleanly.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1201_3972_gb300 import _build, _lib
from paper_1201_3972_gb300.csrc import gen_networks as gn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ir_filter.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ir_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ir_filter_create", "ir_filter_run", "ir_filter_destroy", "ir_filter_run2",
                 "ir_filter_run_batch"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(_lib.EXPORTED)


def test_status_strings_and_version(lib):
    assert lib.ir_filter_version() == b"0.1.0"
    for s in range(8):
        assert lib.ir_status_string(s)
    assert lib.ir_status_string(0) == b"ok"


def test_create_without_device_fails_cleanly(lib):
    h = ctypes.c_void_p()
    st = lib.ir_filter_create(ctypes.byref(h), 0 if not _has_gpu() else 10_000)
    assert st == _lib.IR_EINVAL
    assert not h.value
    assert lib.ir_filter_last_error(None)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.ir_filter_run(None, None, 1, 1, 1, 0, 3, None) == _lib.IR_EINVAL
    assert lib.ir_filter_run2(None, None, 1, None, 1, 1, 1, 0, 3, None, None) == _lib.IR_EINVAL
    assert lib.ir_filter_run_batch(None, None, 0, None) == _lib.IR_EINVAL
    assert lib.ir_filter_run_host(None, None, 0, 0, None) == _lib.IR_EINVAL
    assert lib.ir_filter_sync_status(None) == _lib.IR_EINVAL
    assert lib.ir_filter_launch_count(None) == 0
    assert lib.ir_filter_set_border(None, 0) == _lib.IR_EINVAL
    assert lib.ir_filter_set_detector(None, 0) == _lib.IR_EINVAL
    assert lib.ir_filter_set_strict_alignment(None, 1) == _lib.IR_EINVAL
    assert lib.ir_filter_get_detector(None) == _lib.IR_DETECT_EXTREME
    lib.ir_filter_destroy(None)
    lib.ir_batch_plan_destroy(None)


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError):
        _lib.load(str(tmp_path / "missing.so"))


# ---------------------------------------------------------------------------
# selection networks (0-1 principle)
# ---------------------------------------------------------------------------
def _zero_one_check(net, out, n, m, chunk_bits=20):
    """Evaluate the network on all 2^n 0-1 inputs (in chunks, vectorised).
    For a 0-1 input the rank-m element is 0 exactly when more than m inputs
    are 0, so wire `out` must equal (number of zeros <= m)."""
    total = 1 << n
    step = 1 << min(chunk_bits, n)
    for start in range(0, total, step):
        idx = np.arange(start, start + step, dtype=np.uint64)
        wires = [((idx >> np.uint64(i)) & np.uint64(1)).astype(bool) for i in range(n)]
        ones = np.bitwise_count(idx).astype(np.int64)
        for a, b, _, _ in net:
            wires[a], wires[b] = wires[a] & wires[b], wires[a] | wires[b]
        if not np.array_equal(wires[out], (n - ones) <= m):
            return False
    return True


@pytest.mark.parametrize("k", [3, 5])
def test_median_network_zero_one_principle(k):
    net, out = gn.median_network(k)
    n = k * k
    assert _zero_one_check(net, out, n, (n - 1) // 2)


@pytest.mark.parametrize("k", [7, 9])
def test_median_network_random(k):
    net, out = gn.median_network(k)
    n = k * k
    rng = np.random.default_rng(k)
    for _ in range(3000):
        v = rng.integers(0, 6, n).tolist()
        assert gn.apply(net, v)[out] == sorted(v)[(n - 1) // 2]


@pytest.mark.parametrize("k", [7, 9])
def test_median_network_zero_one_near_median(k):
    """0-1 inputs whose count of ones is within 3 of the median boundary, where
    a wrong selection network fails first (random positions, 20000 each)."""
    net, out = gn.median_network(k)
    n = k * k
    m = (n - 1) // 2
    rng = np.random.default_rng(100 + k)
    for ones in range(n - m - 3, n - m + 4):
        X = np.zeros((20000, n), dtype=bool)
        for row in X:
            row[rng.choice(n, ones, replace=False)] = True
        wires = [X[:, i].copy() for i in range(n)]
        for a, b, _, _ in net:
            wires[a], wires[b] = wires[a] & wires[b], wires[a] | wires[b]
        assert np.all(wires[out] == ((n - ones) <= m))


def test_pairwise_network_sorts():
    """Parberry's pairwise network sorts: every 0-1 input on 16 wires, and
    random inputs on the padded 49- and 81-wire forms (all wires checked)."""
    N = 16
    idx = np.arange(1 << N, dtype=np.uint32)
    wires = [((idx >> i) & 1).astype(bool) for i in range(N)]
    for a, b in gn.pairwise(N):
        wires[a], wires[b] = wires[a] & wires[b], wires[a] | wires[b]
    ones = np.bitwise_count(idx).astype(np.int64)
    for i in range(N):
        assert np.array_equal(wires[i], i >= N - ones)
    rng = np.random.default_rng(7)
    for n in (25, 49, 81):
        ces = gn.pairwise_padded(n)
        for _ in range(300):
            v = rng.integers(0, 1000, n).tolist()
            for a, b in ces:
                if v[a] > v[b]:
                    v[a], v[b] = v[b], v[a]
            assert v == sorted(v)


def test_generated_header_is_current():
    with open(gn.HEADER) as fh:
        assert fh.read() == gn.emit()


def test_dense3_identity_zero_one():
    """The DENSE3 kernel takes g_m = med3(max(lo), med3(mid), min(hi)) of the
    three vertically sorted columns; check that identity on all 2^9 0-1
    windows (0-1 principle for the min/max circuit it forms)."""
    for bits in range(1 << 9):
        w = [(bits >> i) & 1 for i in range(9)]
        cols = [sorted(w[j::3]) for j in range(3)]
        lo = [c[0] for c in cols]
        md = [c[1] for c in cols]
        hi = [c[2] for c in cols]
        med = sorted([max(lo), sorted(md)[1], min(hi)])[1]
        assert med == sorted(w)[4]
        assert min(lo) == min(w) and max(hi) == max(w)


def test_shared_memory_layout_regions_are_disjoint():
    """Every region of the kernel's shared-memory layout (stages, output tiles,
    per-warp blocks, barriers, tile records, frame directory) lies inside the
    total and overlaps no other, for every strategy, window and tile shape the
    library accepts; the layout function is compiled from the kernel header."""
    import subprocess
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = r'''
#include <cstdio>
#include "fnr_params.h"
using namespace fnr;
static bool overlap(long a0, long a1, long b0, long b1) { return a0 < b1 && b0 < a1; }
int main() {
  int bad = 0, n = 0;
  for (int es = 1; es <= 2; ++es)
    for (int k = 3; k <= kMaxK; k += 2)
      for (int algo = ALGO_DENSE3; algo <= ALGO_DENSE; ++algo) {
        if (algo == ALGO_DENSE3 && k != 3) continue;
        if (algo == ALGO_DENSE && k != 5 && k != 7) continue;
        if (algo == ALGO_NETWORK && k > 9) continue;
        for (int tw = 8; tw <= 256; tw += 8)
          for (int th = 8; th <= 256; th += 8) {
            if ((tw * es) % 16 || th % tile_h_multiple(k, algo)) continue;
            const Layout L = make_layout(es, k, algo, th, tw);
            if (L.bw > 256 || L.bh > 256) continue;
            ++n;
            long r[20][2]; int m = 0;
            const long stage = L.off_stage[1] - L.off_stage[0];
            for (int s = 0; s < num_stages(algo); ++s) { r[m][0] = L.off_stage[0] + s * stage; r[m][1] = r[m][0] + (long)L.bw * L.bh * es; ++m; }
            const long outb = dense_algo(algo) ? 0 : (long)tw * th * es;
            for (int o = 0; o < out_buffers(algo); ++o) { r[m][0] = L.off_out[o]; r[m][1] = r[m][0] + outb; ++m; }
            if (out_buffers(algo) == 1 && L.off_out[1] != L.off_out[0]) ++bad;
            r[m][0] = L.off_warp; r[m][1] = L.off_warp + (long)kConsumerWarps * L.warp_bytes; ++m;
            r[m][0] = L.off_bar; r[m][1] = L.off_bar + 16 * kMaxStages; ++m;
            r[m][0] = L.off_info; r[m][1] = L.off_info + 32 * kMaxStages; ++m;
            r[m][0] = L.off_dir; r[m][1] = L.off_dir + kDirMax * 4; ++m;
            r[m][0] = L.off_sync; r[m][1] = L.off_sync + 16 * kMaxStages + 4 * kConsumerWarps * kMaxStages; ++m;
            for (int i = 0; i < m; ++i) {
              if (r[i][0] < 0 || r[i][1] > L.total) ++bad;
              for (int j = i + 1; j < m; ++j)
                if (r[i][1] > r[i][0] && r[j][1] > r[j][0] && overlap(r[i][0], r[i][1], r[j][0], r[j][1])) ++bad;
            }
            if (!dense_algo(algo)) {  // inside a warp block: list, then extremes (planes overlay them)
              const long list1 = L.w_list + (long)L.list_bytes * (pool_medians(algo, k) ? 2 : 1);
              const long v0 = L.w_vmin, v1 = L.w_vmax + (long)L.sr * L.nps * 4;
              if (L.list_bytes < (long)L.sr * tw * 2) ++bad;
              if (overlap(L.w_list, list1, v0, v1) || v1 > L.warp_bytes) ++bad;
              if (algo == ALGO_BITPLANE) {
                const long p1 = L.w_planes + (long)L.nbmax * L.plane_rows * L.pw * 4;
                if (overlap(L.w_list, list1, L.w_planes, p1) || p1 > L.warp_bytes) ++bad;
              }
            }
          }
      }
  printf("%d %d\n", n, bad);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "lay.cpp")
        exe = os.path.join(d, "lay")
        with open(c, "w") as fh:
            fh.write(src)
        cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
        r = subprocess.run(["g++", "-std=c++17", "-D__host__=", "-D__device__=", "-I",
                            os.path.join(root, "paper_1201_3972_gb300", "csrc"), "-I", os.path.join(root, "include"),
                            "-I", cuda_inc, "-o", exe, c], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no host compiler for the layout check: " + r.stderr[-300:])
        n, bad = map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split())
    assert n > 100 and bad == 0


def test_descriptors_from_cpu_tensors():
    """The binding's descriptors for host frames (run_host) take the host
    address, geometry, pitch and pixel type of CPU tensors."""
    import torch
    a = torch.zeros((7, 40), dtype=torch.int16)
    b = torch.zeros((7, 48), dtype=torch.int16)[:, :40]        # a row pitch wider than the row
    c = torch.zeros((3, 5), dtype=torch.uint8)
    d = _lib.Filter.make_descs([{"in": a, "out": b, "k": 5, "u14": True}, {"in": c, "out": c.clone(), "k": 3}])
    assert d[0].in_ == a.data_ptr() and d[0].out == b.data_ptr()
    assert (d[0].H, d[0].W, d[0].in_pitch, d[0].out_pitch, d[0].k) == (7, 40, 80, 96, 5)
    assert d[0].dtype == _lib.IR_U14 and d[1].dtype == _lib.IR_U8
    assert (d[1].H, d[1].W, d[1].in_pitch) == (3, 5, 5)
    assert not d[0].flagged_count
