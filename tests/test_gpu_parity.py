"""GPU parity: the CUDA library against the CPU oracle, bit for bit.

Every test calls the library through its C ABI (ctypes binding) on device
buffers and compares every output pixel, and the flagged count, with the
oracle on the same seeded input. Sizes span several tiles plus ragged tails;
the workload tests run the full frame sizes the benchmark times.
"""
import contextlib

import numpy as np
import pytest

import oracle
from _dev import download, empty_like_frame, guard_bytes_intact, upload
from _golden import all_fixtures
from paper_1201_3972_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

ALL_K = tuple(range(3, 22, 2))


@pytest.fixture(scope="module")
def flt():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1201_3972_gb300 import _build
    _build.build()
    f = _lib.Filter(0)
    yield f
    f.sync_status()
    f.close()


def algos_for(k):
    out = [_lib.IR_ALGO_BITPLANE]
    if k <= 9:
        out.append(_lib.IR_ALGO_NETWORK)
    if k == 3:
        out.append(_lib.IR_ALGO_DENSE3)
    if k in (5, 7):
        out.append(_lib.IR_ALGO_DENSE)
    return out


DENSE_ALGOS = (_lib.IR_ALGO_DENSE3, _lib.IR_ALGO_DENSE)


def row_group(k):
    return 8 if k >= 8 else (4 if k >= 4 else 2)


def tiles_for(es, k, algo):
    """Tile shapes the kernels accept: tile_w * bytes a multiple of 16, tile
    plus halo within the 256-pixel TMA box, tile_h split into 8 warp strips
    of whole row groups (row pairs for the dense paths)."""
    r = (k - 1) // 2
    xoff = -(-r // (16 // es)) * (16 // es)
    mult = 8 * (2 if algo in DENSE_ALGOS else row_group(k))
    out = []
    for tw, th in ((64, 64), (128, 32), (32, 16), (16, 16), (8, 16), (128, 64), (192, 32), (64, 128), (128, 128),
                   (128, 48), (64, 96)):
        if tw + 2 * xoff <= 256 and th + 2 * r <= 256 and (tw * es) % 16 == 0 and th % mult == 0:
            out.append((tw, th))
    return out


def dtype_code(frame, u14=False):
    return _lib.IR_U8 if frame.dtype == np.uint8 else (_lib.IR_U14 if u14 else _lib.IR_U16)


def gpu_fnr(flt, frame, k, u14=False, in_pitch=None, out_pitch=None, in_off=0, out_off=0, count=True):
    """Run ir_filter_run2 on a copy of `frame`; returns (output, flagged)."""
    import torch
    H, W = frame.shape
    ib, ia, ip = upload(frame, in_pitch, in_off)
    ob, oa, op = empty_like_frame(frame, out_pitch, out_off)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda") if count else None
    flt.ir_filter_run2(ia, ip, oa, op, H, W, dtype_code(frame, u14), k, None, ctr)
    out = download(ob, oa, op, H, W, frame.dtype)
    assert guard_bytes_intact(ob, oa, op, H, W, frame.itemsize), "write outside the frame"
    flagged = int(ctr.item()) if count else None
    return out, flagged


def check(flt, frame, k, **kw):
    want, wf = oracle.fnr(frame, k)
    got, gf = gpu_fnr(flt, frame, k, **kw)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        y, x = bad[0]
        raise AssertionError(f"k={k} {frame.shape} {frame.dtype}: {len(bad)} pixels differ; first at "
                             f"({y},{x}) got {got[y, x]} want {want[y, x]}")
    if gf is not None:
        assert gf == wf, f"flagged {gf} != oracle {wf}"


def with_config(flt, dtype, k, algo, tw, th):
    flt.set_config(dtype, k, tw, th, algo)


@contextlib.contextmanager
def exact_tiles(flt):
    """Launches use the configured tile as it is (no shrinking of launches
    with fewer tiles than SMs), so that a sweep tests exactly its shapes."""
    flt.set_tile_fit(False)
    try:
        yield
    finally:
        flt.set_tile_fit(True)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("fx", all_fixtures(), ids=lambda f: f["name"])
def test_golden_fixtures_every_algo(flt, fx):
    k = fx["k"]
    es = fx["input"].itemsize
    for algo in algos_for(k):
        for dt in ((_lib.IR_U8,) if es == 1 else (_lib.IR_U16, _lib.IR_U14)):
            with_config(flt, dt, k, algo, 64, 64)
        flt.set_detector(fx["detector"])
        try:
            got, gf = gpu_fnr(flt, fx["input"], k, u14=(fx["dtype"] == _lib.IR_U14))
        finally:
            flt.set_detector("extreme")
        np.testing.assert_array_equal(got, fx["output"])
        assert gf == fx["flagged"]
    flt.set_config(_lib.IR_U8, k, 0, 0, _lib.IR_ALGO_AUTO)
    flt.set_config(_lib.IR_U16, k, 0, 0, _lib.IR_ALGO_AUTO)


@pytest.mark.parametrize("k", ALL_K)
@pytest.mark.parametrize("es", [1, 2])
def test_every_algo_and_tile_random(flt, k, es):
    """Uniform random and tie-heavy frames, every (algo, tile) built for k,
    ragged sizes that are not multiples of any tile side."""
    rng = np.random.default_rng(1000 * k + es)
    dt = _lib.IR_U8 if es == 1 else _lib.IR_U16
    npdt = np.uint8 if es == 1 else np.uint16
    maxv = 255 if es == 1 else 65535
    shapes = [(67, 150), (33, 29)]
    with exact_tiles(flt):
        _sweep_random(flt, k, es, dt, npdt, maxv, rng, shapes)
    flt.set_config(dt, k, 0, 0, _lib.IR_ALGO_AUTO)


def _sweep_random(flt, k, es, dt, npdt, maxv, rng, shapes):
    for algo in algos_for(k):
        for tw, th in tiles_for(es, k, algo):
            try:
                flt.set_config(dt, k, tw, th, algo)
            except _lib.IrError as e:     # a shape that needs more shared memory than a CTA has
                assert e.status == _lib.IR_EINVAL
                continue
            for H, W in shapes:
                a = rng.integers(0, maxv + 1, (H, W)).astype(npdt)
                check(flt, a, k)
                b = rng.choice([0, 1, maxv // 2, maxv], (H, W)).astype(npdt)
                check(flt, b, k)


@pytest.mark.parametrize("k", ALL_K)
@pytest.mark.parametrize("es", [1, 2])
def test_every_algo_and_tile_on_the_tma_path(flt, k, es):
    """The same (algo, tile) sweep with 16-byte aligned bases and pitches, so
    that tiles are staged and strips stored by TMA (strips smaller than 128
    bytes store with plain stores, since a TMA copy needs its shared-memory
    side 128-byte aligned)."""
    rng = np.random.default_rng(2000 * k + es)
    dt = _lib.IR_U8 if es == 1 else _lib.IR_U16
    npdt = np.uint8 if es == 1 else np.uint16
    maxv = 255 if es == 1 else 65535
    with exact_tiles(flt):
        for algo in algos_for(k):
            for tw, th in tiles_for(es, k, algo):
                try:
                    flt.set_config(dt, k, tw, th, algo)
                except _lib.IrError as e:
                    assert e.status == _lib.IR_EINVAL
                    continue
                for H, W in ((67, 150), (33, 29)):
                    pitch = -(-W * es // 16) * 16 // es
                    check(flt, rng.integers(0, maxv + 1, (H, W)).astype(npdt), k, in_pitch=pitch, out_pitch=pitch)
    flt.set_config(dt, k, 0, 0, _lib.IR_ALGO_AUTO)
    flt.sync_status()


@pytest.mark.parametrize("k", [11, 15, 21])
@pytest.mark.parametrize("es", [1, 2])
def test_bitplane_sparse_and_dense_strips(flt, k, es):
    """The bit-plane strategy selects per pixel across the warp in strips with
    few flagged pixels and through bit planes otherwise: a smooth plateaued
    field with rare impulses (few flagged per strip, many tied values in each
    window), the same with dense impulses, and the two mixed in one frame."""
    rng = np.random.default_rng(77 * k + es)
    dt = _lib.IR_U8 if es == 1 else _lib.IR_U14
    npdt = np.uint8 if es == 1 else np.uint16
    maxv = 255 if es == 1 else 16383
    H, W = 150, 203
    y, x = np.mgrid[0:H, 0:W]
    base = ((x + 2 * y) // 7 * (maxv // 90)) % (maxv // 2) + maxv // 8
    flt.set_config(dt, k, 64, 64, _lib.IR_ALGO_BITPLANE)
    for p in (0.002, 0.3):
        a = base.copy()
        m = rng.random((H, W)) < p
        a[m] = rng.integers(0, maxv + 1, int(m.sum()))
        check(flt, a.astype(npdt), k, u14=(es == 2))
    a = base.copy()
    m = (rng.random((H, W)) < 0.3) & (x < W // 2)
    a[m] = rng.choice([0, maxv], int(m.sum()))
    check(flt, a.astype(npdt), k, u14=(es == 2))
    flt.set_config(dt, k, 0, 0, _lib.IR_ALGO_AUTO)


@pytest.mark.parametrize("k", [3, 5, 7, 9, 15, 21])
def test_edge_shapes(flt, k):
    """1x1, single rows and columns, frames smaller than the window, odd
    widths, for both pixel types and every algo."""
    rng = np.random.default_rng(k)
    for es, dt in ((1, _lib.IR_U8), (2, _lib.IR_U16)):
        npdt = np.uint8 if es == 1 else np.uint16
        for algo in algos_for(k):
            flt.set_config(dt, k, 64, 64, algo)
            for H, W in ((1, 1), (1, 7), (7, 1), (1, 300), (300, 1), (2, 3), (k - 1, k + 2), (5, 17), (9, 130)):
                a = rng.integers(0, 256 if es == 1 else 65536, (H, W)).astype(npdt)
                check(flt, a, k)
        flt.set_config(dt, k, 0, 0, _lib.IR_ALGO_AUTO)


@pytest.mark.parametrize("k", [3, 5, 9, 21])
def test_unaligned_pitch_and_base(flt, k):
    """Odd pitches and misaligned bases take the plain-load / plain-store path;
    aligned-in/unaligned-out and the reverse mix TMA and plain paths."""
    rng = np.random.default_rng(7 + k)
    for npdt in (np.uint8, np.uint16):
        maxv = np.iinfo(npdt).max
        a = rng.integers(0, maxv + 1, (70, 133)).astype(npdt)
        check(flt, a, k, in_pitch=137, out_pitch=141)
        check(flt, a, k, in_off=1, out_off=3, in_pitch=160, out_pitch=160)
        check(flt, a, k, in_pitch=144, out_pitch=139)
        check(flt, a, k, in_pitch=139, out_pitch=144)
        # 16-byte aligned pitch, row of W*e bytes not a multiple of 16: the
        # bytes between W and the pitch belong to the caller
        check(flt, a, k, in_pitch=144, out_pitch=144)
        check(flt, a[:, :129].copy(), k, in_pitch=256, out_pitch=256)


def test_in_place_run_matches_oracle(flt):
    import torch
    for s in (synth.workload_single_u8()[0], synth.workload_sweep_u14()[4]):
        f = s.make()
        want, _ = oracle.fnr(f, s.k)
        buf, addr, pitch = upload(f)
        flt.ir_filter_run(addr, f.shape[0], f.shape[1], pitch, s.dtype, s.k)
        torch.cuda.synchronize()
        got = download(buf, addr, pitch, f.shape[0], f.shape[1], f.dtype)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("spec", synth.workload_single_u8() + synth.workload_sweep_u14(), ids=lambda s: s.tag)
def test_workload_small_k_full_size(flt, spec):
    """320x240 u8 (3x3) and the 640x512 14-bit sweep (5-40% impulses, 3/5/7),
    full frames, every algo."""
    f = spec.make()
    want, wf = oracle.fnr(f, spec.k)
    with exact_tiles(flt):
        for algo in algos_for(spec.k):
            flt.set_config(spec.dtype, spec.k, 128 if algo in DENSE_ALGOS else 64, 64, algo)
            got, gf = gpu_fnr(flt, f, spec.k, u14=spec.dtype == _lib.IR_U14)
            np.testing.assert_array_equal(got, want)
            assert gf == wf
    flt.set_config(spec.dtype, spec.k, 0, 0, _lib.IR_ALGO_AUTO)
    # the default configuration with tile fitting (a single frame shrinks its tile)
    got, gf = gpu_fnr(flt, f, spec.k, u14=spec.dtype == _lib.IR_U14)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


@pytest.mark.parametrize("spec", synth.workload_large_k(), ids=lambda s: s.tag)
def test_workload_large_k_full_size(flt, spec):
    """1280x1024 14-bit, 20% random-valued impulses, windows 9-21."""
    f = spec.make()
    want, wf = oracle.fnr_mt(f, spec.k, 16)
    got, gf = gpu_fnr(flt, f, spec.k, u14=True)
    np.testing.assert_array_equal(got, want)
    assert gf == wf


def test_errors_are_reported(flt):
    import torch
    a = torch.zeros(64, dtype=torch.uint8, device="cuda")
    addr = int(a.data_ptr())
    for k in (2, 1, 23, 0, -3):
        with pytest.raises(_lib.IrError) as e:
            flt.ir_filter_run2(addr, 8, addr + 32, 8, 2, 8, _lib.IR_U8, k)
        assert e.value.status == _lib.IR_EINVAL
    with pytest.raises(_lib.IrError):
        flt.ir_filter_run2(addr, 8, addr + 4, 8, 2, 8, _lib.IR_U8, 3)      # overlap
    with pytest.raises(_lib.IrError):
        flt.ir_filter_run2(addr, 4, addr + 32, 8, 2, 8, _lib.IR_U8, 3)      # pitch < W
    with pytest.raises(_lib.IrError):
        flt.ir_filter_run2(0, 8, addr + 32, 8, 2, 8, _lib.IR_U8, 3)         # null
    with pytest.raises(_lib.IrError):
        flt.ir_filter_run2(addr, 8, addr + 32, 8, 0, 8, _lib.IR_U8, 3)      # H = 0
    with pytest.raises(_lib.IrError):
        flt.set_config(_lib.IR_U8, 5, 64, 32, _lib.IR_ALGO_DENSE3)          # dense3 is k=3 only
    with pytest.raises(_lib.IrError):
        flt.set_config(_lib.IR_U8, 3, 250, 32, _lib.IR_ALGO_DENSE3)         # box > 256
    with pytest.raises(_lib.IrError):
        flt.set_config(_lib.IR_U16, 9, 64, 32, _lib.IR_ALGO_BITPLANE)       # 32 rows: not 8 strips of 8
    flt.sync_status()


def test_strict_alignment_refuses_misaligned_frames(flt):
    """With strict alignment a misaligned base or pitch (input or output,
    single frames, in place and batches) is IR_EALIGN and nothing is written;
    aligned frames still run, and turning it off restores the plain path."""
    import torch
    rng = np.random.default_rng(11)
    a = rng.integers(0, 256, (40, 70)).astype(np.uint8)
    flt.set_strict_alignment(True)
    try:
        for kw in (dict(in_pitch=73), dict(out_pitch=75), dict(in_off=1, in_pitch=80), dict(out_off=2, out_pitch=80)):
            ib, ia, ip = upload(a, kw.get("in_pitch"), kw.get("in_off", 0))
            ob, oa, op = empty_like_frame(a, kw.get("out_pitch"), kw.get("out_off", 0))
            before = ob.clone()
            with pytest.raises(_lib.IrError) as e:
                flt.ir_filter_run2(ia, ip, oa, op, 40, 70, _lib.IR_U8, 3)
            assert e.value.status == _lib.IR_EALIGN
            torch.cuda.synchronize()
            assert torch.equal(ob, before)
        ib, ia, ip = upload(a, 75)
        with pytest.raises(_lib.IrError) as e:
            flt.ir_filter_run(ia, 40, 70, ip, _lib.IR_U8, 3)
        assert e.value.status == _lib.IR_EALIGN
        arr = (_lib.ir_frame_desc * 1)()
        ob, oa, op = empty_like_frame(a, 80)
        arr[0].in_, arr[0].out, arr[0].H, arr[0].W = ia, oa, 40, 70
        arr[0].in_pitch, arr[0].out_pitch, arr[0].dtype, arr[0].k = ip, op, _lib.IR_U8, 5
        with pytest.raises(_lib.IrError) as e:
            flt.ir_filter_run_batch(arr, 1)
        assert e.value.status == _lib.IR_EALIGN
        check(flt, a, 3, in_pitch=80, out_pitch=96)   # aligned: runs
    finally:
        flt.set_strict_alignment(False)
    check(flt, a, 3, in_pitch=73, out_pitch=75)       # off again: the plain path
    flt.sync_status()


def test_autotune_keeps_results_exact(flt):
    f = synth.workload_sweep_u14()[1].make()
    for k in (3, 5, 9):
        flt.autotune(_lib.IR_U14, k, 512, 640)
        cfg = flt.get_config(_lib.IR_U14, k)
        assert cfg["algo"] in algos_for(k)
        check(flt, f, k, u14=True)
        flt.set_config(_lib.IR_U14, k, 0, 0, _lib.IR_ALGO_AUTO)


def test_autotune_batch_on_the_callers_frames(flt):
    """ir_filter_autotune_batch tunes each class on the given frames: every
    class is reported with its candidates timed, the choice is no slower than
    the default in the tuner's own timing (the default is one of the
    candidates), the tuned plan's results equal the oracle's, and a fresh
    timing of the tuned plan is not slower than the default plan's."""
    import statistics
    import torch
    specs = synth.workload_sweep_u14()
    frames = [s.make() for s in specs]
    reps = 4
    ins = [torch.from_numpy(f.view(np.int16)).cuda() for f in frames * reps]
    outs = [torch.empty_like(t) for t in ins]
    descs = flt.make_descs([{"in": a, "out": b, "k": specs[i % len(specs)].k, "u14": True}
                            for i, (a, b) in enumerate(zip(ins, outs))])
    try:
        res = flt.autotune_batch(descs, reps=20)
        assert sorted(r["k"] for r in res) == [3, 5, 7]
        for r in res:
            assert r["dtype"] == _lib.IR_U16 and r["frames"] == reps * 4 and r["candidates"] >= 2
            assert 0 < r["chosen_ms"] <= r["default_ms"] * (1 + 1e-6)
            assert flt.get_config(_lib.IR_U14, r["k"]) == r["chosen"]
        plan = _lib.BatchPlan(flt, descs)
        plan.launch()
        torch.cuda.synchronize()
        for i, o in enumerate(outs[:len(specs)]):
            want, _ = oracle.fnr(frames[i], specs[i].k)
            np.testing.assert_array_equal(o.cpu().numpy().view(np.uint16), want)

        def timed(p):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(30)]
            for a, b in ev:
                a.record()
                p.launch()
                b.record()
            torch.cuda.synchronize()
            return statistics.median(a.elapsed_time(b) for a, b in ev)
        t_tuned = timed(plan)
        plan.close()
        for r in res:
            flt.set_config(_lib.IR_U14, r["k"], 0, 0, _lib.IR_ALGO_AUTO)
        dplan = _lib.BatchPlan(flt, descs)
        t_default = timed(dplan)
        dplan.close()
        assert t_tuned <= 1.10 * t_default, (t_tuned, t_default)
    finally:
        for k in (3, 5, 7):
            flt.set_config(_lib.IR_U14, k, 0, 0, _lib.IR_ALGO_AUTO)


def test_launch_counter_counts_kernels(flt):
    before = flt.launch_count()
    f = synth.workload_single_u8()[0].make()
    for _ in range(3):
        gpu_fnr(flt, f, 3, count=False)
    assert flt.launch_count() - before == 3


def test_tuning_table_round_trip(flt, tmp_path):
    """A tuned table saved under a device name and loaded into a fresh handle
    gives the same configurations, and results stay exact with it."""
    import torch
    name = torch.cuda.get_device_name(0)
    flt.set_config(_lib.IR_U16, 7, 128, 32, _lib.IR_ALGO_NETWORK)
    path = str(tmp_path / "tuning.json")
    flt.save_configs(path, name)
    other = _lib.Filter(0)
    try:
        assert other.configs() != flt.configs()
        assert other.load_configs(path, name)
        assert other.configs() == flt.configs()
        assert not other.load_configs(path, name + " (another model)")
        a = np.random.default_rng(3).integers(0, 65536, (70, 150)).astype(np.uint16)
        check(other, a, 7)
    finally:
        other.close()
        flt.set_config(_lib.IR_U16, 7, 0, 0, _lib.IR_ALGO_AUTO)
