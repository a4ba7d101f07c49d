"""GPU parity of the batched form: many frames of mixed sizes, pixel types
and windows in one graph launch, each output compared with the CPU oracle."""
import numpy as np
import pytest

import oracle
from _dev import download, empty_like_frame, upload
from paper_1201_3972_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flt():
    import torch
    assert torch.cuda.is_available()
    from paper_1201_3972_gb300 import _build
    _build.build()
    f = _lib.Filter(0)
    yield f
    f.sync_status()
    f.close()


def _stage(frames):
    """Upload (frame, k, u14) triples; returns descriptor dicts plus buffers."""
    import torch
    items = []
    for f, k, u14 in frames:
        ib, ia, ip = upload(f)
        ob, oa, op = empty_like_frame(f)
        ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
        items.append(dict(frame=f, k=k, u14=u14, ib=ib, ia=ia, ip=ip, ob=ob, oa=oa, op=op, ctr=ctr))
    return items


def _descs(items):
    arr = (_lib.ir_frame_desc * len(items))()
    for i, it in enumerate(items):
        f = it["frame"]
        arr[i].in_ = it["ia"]
        arr[i].out = it["oa"]
        arr[i].H, arr[i].W = f.shape
        arr[i].in_pitch, arr[i].out_pitch = it["ip"], it["op"]
        arr[i].dtype = _lib.IR_U8 if f.dtype == np.uint8 else (_lib.IR_U14 if it["u14"] else _lib.IR_U16)
        arr[i].k = it["k"]
        arr[i].flagged_count = int(it["ctr"].data_ptr())
    return arr


def _verify(items, threads=16):
    for it in items:
        f = it["frame"]
        want, wf = oracle.fnr_mt(f, it["k"], threads)
        got = download(it["ob"], it["oa"], it["op"], f.shape[0], f.shape[1], f.dtype)
        np.testing.assert_array_equal(got, want)
        assert int(it["ctr"].item()) == wf


def test_small_mixed_batch(flt):
    rng = np.random.default_rng(3)
    frames = []
    for i in range(24):
        H, W = int(rng.integers(1, 90)), int(rng.integers(1, 200))
        u8 = bool(rng.integers(0, 2))
        k = int(rng.choice([3, 5, 7, 9, 11, 15, 21]))
        maxv = 255 if u8 else 16383
        a = rng.integers(0, maxv + 1, (H, W)).astype(np.uint8 if u8 else np.uint16)
        frames.append((a, k, not u8))
    items = _stage(frames)
    flt.ir_filter_run_batch(_descs(items), len(items))
    _verify(items)


def test_plan_replays_read_current_inputs(flt):
    import torch
    rng = np.random.default_rng(5)
    frames = [(rng.integers(0, 256, (50, 70)).astype(np.uint8), 3, False),
              (rng.integers(0, 16384, (40, 90)).astype(np.uint16), 5, True),
              (rng.integers(0, 16384, (33, 65)).astype(np.uint16), 9, True)]
    items = _stage(frames)
    descs = _descs(items)
    plan = _lib.BatchPlan(flt, descs)
    assert plan.kernel_count == 3
    plan.launch()
    _verify(items)
    # new contents, same buffers: the replay must see them
    for it in items:
        f = it["frame"]
        nf = rng.integers(0, 200, f.shape).astype(f.dtype)
        it["frame"] = nf
        host = torch.from_numpy(nf.view(np.uint8).reshape(-1).copy())
        it["ib"][: host.numel()].copy_(host)
    plan.launch()
    plan.launch()
    _verify(items)
    plan.close()


def test_batch_cache_reuses_graph(flt):
    rng = np.random.default_rng(9)
    frames = [(rng.integers(0, 256, (64, 64)).astype(np.uint8), k, False) for k in (3, 5, 7)]
    items = _stage(frames)
    descs = _descs(items)
    before = flt.launch_count()
    for _ in range(4):
        flt.ir_filter_run_batch(descs, len(items))
    assert flt.launch_count() - before == 4 * 3
    _verify(items)


def test_full_mixed_batch_256_frames(flt):
    """The mixed batch at full size: 256 frames, 5 frame sizes up to
    1920x1080, u8 and 14-bit, windows 3/5/7/9/15, 5-30% salt-and-pepper."""
    specs = synth.workload_batch()
    frames = [(s.make(), s.k, s.dtype == synth.U14) for s in specs]
    items = _stage(frames)
    flt.ir_filter_run_batch(_descs(items), len(items))
    _verify(items)


def test_batch_beyond_the_shared_directory(flt):
    """More frames in one class than the kernel's shared-memory frame
    directory holds (512): tiles are then located by a search of the frame
    table in global memory."""
    rng = np.random.default_rng(17)
    frames = [(rng.integers(0, 256, (int(rng.integers(1, 40)), int(rng.integers(1, 70)))).astype(np.uint8), 3, False)
              for _ in range(600)]
    items = _stage(frames)
    flt.ir_filter_run_batch(_descs(items), len(items))
    _verify(items, threads=4)


def _host_descs(items):
    """items: (host_in_addr, host_out_addr, H, W, pitch_bytes, dtype, k, counter or None)."""
    arr = (_lib.ir_frame_desc * len(items))()
    for i, (ia, oa, H, W, p, dt, k, ctr) in enumerate(items):
        arr[i].in_, arr[i].out, arr[i].H, arr[i].W = ia, oa, H, W
        arr[i].in_pitch = arr[i].out_pitch = p
        arr[i].dtype, arr[i].k = dt, k
        arr[i].flagged_count = int(ctr.data_ptr()) if ctr is not None else None
    return arr


def test_host_frames_pinned_pageable_and_in_place(flt):
    """ir_filter_run_host: frames in pinned and in pageable host memory,
    separate and back to back (one copy per run of frames), several chunk
    counts, in place on the host, per-frame counts; every output against
    the oracle."""
    import torch
    rng = np.random.default_rng(41)
    frames = []
    for i in range(13):
        H, W = int(rng.integers(1, 200)), int(rng.integers(1, 330))
        u8 = bool(i % 3 == 0)
        k = int(rng.choice([3, 5, 7, 9, 15]))
        frames.append((synth.make_frame(H, W, synth.U8 if u8 else synth.U14, 700 + i, 2.0 if u8 else 8.0, 0.2), k))
    want = [oracle.fnr(f, k) for f, k in frames]
    dts = [(_lib.IR_U8 if f.dtype == np.uint8 else _lib.IR_U14) for f, _ in frames]
    for chunks in (0, 1, 3, 50):
        # pinned, one tensor per frame
        ins = [torch.from_numpy(np.ascontiguousarray(f)).pin_memory() for f, _ in frames]
        outs = [torch.empty_like(t).pin_memory() for t in ins]
        ctrs = [torch.zeros(1, dtype=torch.int64, device="cuda") for _ in frames]
        items = [(int(a.data_ptr()), int(b.data_ptr()), f.shape[0], f.shape[1], f.shape[1] * f.itemsize, dt, k, c)
                 for a, b, (f, k), dt, c in zip(ins, outs, frames, dts, ctrs)]
        flt.ir_filter_run_host(_host_descs(items), len(items), chunks)
        torch.cuda.synchronize()
        for o, c, (w, wf) in zip(outs, ctrs, want):
            np.testing.assert_array_equal(o.numpy(), w)
            assert int(c.item()) == wf
    # back to back in one pinned buffer, rows padded to 16 bytes (runs of frames move as one copy), in place
    pads = [-(-f.shape[1] * f.itemsize // 16) * 16 for f, _ in frames]
    sizes = [f.shape[0] * p for (f, _), p in zip(frames, pads)]
    buf = torch.zeros(sum(sizes), dtype=torch.uint8).pin_memory()
    hb = buf.numpy()
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(int)
    for (f, _), o, p in zip(frames, offs, pads):
        view = np.lib.stride_tricks.as_strided(hb[o:].view(f.dtype), shape=f.shape, strides=(p, f.itemsize))
        view[...] = f
    base = int(buf.data_ptr())
    items = [(base + int(o), base + int(o), f.shape[0], f.shape[1], p, dt, k, None)
             for (f, k), o, p, dt in zip(frames, offs, pads, dts)]
    flt.ir_filter_run_host(_host_descs(items), len(items), 4)
    torch.cuda.synchronize()
    for (f, _), o, p, (w, _) in zip(frames, offs, pads, want):
        got = np.lib.stride_tricks.as_strided(hb[o:].view(f.dtype), shape=f.shape, strides=(p, f.itemsize))
        np.testing.assert_array_equal(got, w)
    # pageable numpy frames
    outs = [np.zeros_like(f) for f, _ in frames]
    ins = [np.ascontiguousarray(f) for f, _ in frames]
    items = [(a.ctypes.data, b.ctypes.data, a.shape[0], a.shape[1], a.strides[0], dt, k, None)
             for a, b, (_, k), dt in zip(ins, outs, frames, dts)]
    flt.ir_filter_run_host(_host_descs(items), len(items), 3)
    torch.cuda.synchronize()
    for o, (w, _) in zip(outs, want):
        np.testing.assert_array_equal(o, w)
    flt.sync_status()


def test_host_frames_restage_and_errors(flt):
    """A larger set after a small one regrows the staging; bad descriptors are
    refused before anything runs."""
    import torch
    small = synth.make_frame(30, 40, synth.U8, 90, 2.0, 0.1)
    big = synth.make_frame(700, 900, synth.U14, 91, 8.0, 0.1)
    for f, k in ((small, 3), (big, 7), (small, 5)):
        src = torch.from_numpy(f).pin_memory()
        dst = torch.empty_like(src).pin_memory()
        dt = _lib.IR_U8 if f.dtype == np.uint8 else _lib.IR_U14
        items = [(int(src.data_ptr()), int(dst.data_ptr()), f.shape[0], f.shape[1], f.shape[1] * f.itemsize, dt, k,
                  None)]
        flt.ir_filter_run_host(_host_descs(items), 1)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dst.numpy(), oracle.fnr(f, k)[0])
    src = torch.zeros(64, dtype=torch.uint8).pin_memory()
    a = int(src.data_ptr())
    for bad in ((a, a + 4, 2, 8, 8, _lib.IR_U8, 3, None),     # overlap (not the same frame)
                (a, a + 32, 2, 8, 8, _lib.IR_U8, 4, None),    # even k
                (0, a + 32, 2, 8, 8, _lib.IR_U8, 3, None)):   # null
        with pytest.raises(_lib.IrError) as e:
            flt.ir_filter_run_host(_host_descs([bad]), 1)
        assert e.value.status == _lib.IR_EINVAL
    with pytest.raises(_lib.IrError):
        flt.ir_filter_run_host(_host_descs([]), 0)
    flt.sync_status()
