"""Serving many video streams with the continuous-batching server.

``Server`` is the ctypes binding of the ``ir_server_*`` entry points (the
scheduling, admission, batching and completion tracking all run in the
library's C++ threads). ``simulate`` drives it with simulated IR cameras:
every stream produces frames at Poisson arrival times, frames are submitted
from pinned host memory as they arrive, results are hashed and compared
with the same frames filtered one at a time by the plain entry point, and
per-frame latency (arrival -> completion observed) is recorded.
"""
from __future__ import annotations

import ctypes
import hashlib
import queue
import threading
import time
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib, synth


class Server:
    """One ``ir_server``: device-resident stream buffers + batcher + poller."""

    def __init__(self, device: int = 0, max_streams: int = 256, ring_depth: int = 8, max_batch: int = 256,
                 exec_streams: int = 3, hbm_reserve_bytes: int = 1 << 30, poll_us: int = 20):
        self.lib = _lib.load()
        cfg = _lib.ir_server_config(max_streams, ring_depth, max_batch, exec_streams, hbm_reserve_bytes, poll_us)
        p = ctypes.c_void_p()
        st = self.lib.ir_server_create(int(device), ctypes.byref(cfg), ctypes.byref(p))
        if st != _lib.IR_OK:
            raise _lib.IrError(st, (self.lib.ir_filter_last_error(None) or b"").decode() or "ir_server_create failed")
        self.p = p
        self._buf = (_lib.ir_completion * 4096)()

    def close(self) -> None:
        if getattr(self, "p", None):
            self.lib.ir_server_destroy(self.p)
            self.p = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _err(self, st: int) -> None:
        if st != _lib.IR_OK:
            h = self.lib.ir_server_filter(self.p)
            raise _lib.IrError(st, (self.lib.ir_filter_last_error(h) or b"").decode() or "server call failed")

    def set_config(self, dtype: int, k: int, tile_w: int, tile_h: int, algo: int) -> None:
        """Kernel configuration for a class, before opening streams of it."""
        c = _lib.ir_kernel_config(tile_w, tile_h, algo, 0)
        self._err(self.lib.ir_filter_set_config(self.lib.ir_server_filter(self.p), dtype, k, ctypes.byref(c)))

    def open_stream(self, H: int, W: int, dtype: int, k: int) -> int:
        sid = ctypes.c_int(-1)
        self._err(self.lib.ir_server_open_stream(self.p, H, W, dtype, k, ctypes.byref(sid)))
        return sid.value

    def close_stream(self, sid: int) -> None:
        self._err(self.lib.ir_server_close_stream(self.p, sid))

    def submit(self, sid: int, host_addr: int, host_pitch: int, tag: int) -> Optional[int]:
        """Queue a frame; returns its slot, or None when the stream is full (busy)."""
        slot = ctypes.c_int(-1)
        st = self.lib.ir_server_submit(self.p, sid, ctypes.c_void_p(host_addr), host_pitch, tag, ctypes.byref(slot))
        if st == _lib.IR_EBUSY:
            return None
        self._err(st)
        return slot.value

    def poll(self) -> List[_lib.ir_completion]:
        n = self.lib.ir_server_poll(self.p, self._buf, len(self._buf))
        return [_lib.ir_completion.from_buffer_copy(self._buf[i]) for i in range(n)]

    def wait_idle(self, timeout_s: float = 30.0) -> bool:
        return self.lib.ir_server_wait_idle(self.p, timeout_s) == _lib.IR_OK

    def read(self, sid: int, slot: int, out: np.ndarray) -> None:
        self._err(self.lib.ir_server_read(self.p, sid, slot, ctypes.c_void_p(out.ctypes.data), out.strides[0]))

    def release(self, sid: int, slot: int) -> None:
        self._err(self.lib.ir_server_release(self.p, sid, slot))

    def stats(self) -> Dict[str, int]:
        s = _lib.ir_server_stats()
        self._err(self.lib.ir_server_get_stats(self.p, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def clock(self) -> float:
        return self.lib.ir_server_clock()


def frame_hash(a: np.ndarray) -> bytes:
    return hashlib.blake2b(np.ascontiguousarray(a).tobytes(), digest_size=8).digest()


@dataclass
class Pools:
    """Pinned host copies of the shared frame pools, one per resolution."""
    frames: Dict[int, List[np.ndarray]]
    pinned: Dict[int, list]          # torch tensors keeping the pinned memory alive
    addrs: Dict[int, List[int]]


def make_pools(streams: Sequence[synth.StreamSpec]) -> Pools:
    import torch
    frames, pinned, addrs = {}, {}, {}
    for si in sorted({s.size_index for s in streams}):
        pool = streams[[s.size_index for s in streams].index(si)].pool
        fs = [spec.make() for spec in synth.serve_pool(si, pool)]
        ts = [torch.from_numpy(f.view(np.int16)).pin_memory() for f in fs]
        frames[si] = fs
        pinned[si] = ts
        addrs[si] = [int(t.data_ptr()) for t in ts]
    return Pools(frames, pinned, addrs)


def reference_hashes(pools: Pools, streams: Sequence[synth.StreamSpec], device: int = 0) -> Dict[Tuple[int, int, int], bytes]:
    """Hash of every (resolution, pool frame, k) the streams use, filtered one
    frame at a time by the plain entry point (ir_filter_run2)."""
    import torch
    flt = _lib.Filter(device)
    out = {}
    try:
        for si, k in sorted({(s.size_index, s.k) for s in streams}):
            for j, f in enumerate(pools.frames[si]):
                src = torch.from_numpy(f.view(np.int16)).cuda(device)
                dst = torch.empty_like(src)
                flt.run2(src, dst, k, u14=True)
                out[(si, j, k)] = frame_hash(dst.cpu().numpy().view(np.uint16))
        torch.cuda.synchronize()
    finally:
        flt.close()
    return out


def simulate(streams: Sequence[synth.StreamSpec], duration_s: float, pools: Pools,
             ref: Optional[Dict[Tuple[int, int, int], bytes]] = None, verify_every: int = 1,
             device: int = 0, seed: int = 4, closed_loop: bool = False, server_kwargs: Optional[dict] = None,
             keep_outputs: bool = False) -> dict:
    """Run the streams against a fresh server for ``duration_s`` seconds.

    Open loop (default): every stream submits at its Poisson arrival times;
    latency is measured from the scheduled arrival to the completion the
    server observed. Closed loop: each stream resubmits as soon as it gets a
    slot back (saturation throughput). Every ``verify_every``-th completion is
    read back and its hash compared with ``ref`` by a pool of verifier
    threads, which release the slot afterwards; the latency of a frame is
    taken by the server when its completion event fires, so the verification
    does not enter it.
    """
    srv = Server(device, **(server_kwargs or {}))
    try:
        sids = [srv.open_stream(s.H, s.W, synth.U14, s.k) for s in streams]
        rng = np.random.Generator(np.random.PCG64(synth.seed_for(4, 9999 + seed)))
        if closed_loop:
            schedule = []
        else:
            events = []
            for s in streams:
                t = synth.poisson_arrivals(rng, s.fps, duration_s)
                events += [(float(ti), s.stream_id, j) for j, ti in enumerate(t)]
            events.sort()
            schedule = events
        arrivals: Dict[int, Tuple[float, int, int]] = {}
        lat, done_px = [], 0
        dropped = 0
        mismatches, verified = 0, 0
        outputs = {}
        lock = threading.Lock()
        producer_done = threading.Event()
        t0 = srv.clock() + 0.05
        next_j = {s.stream_id: 0 for s in streams}

        def submit(s, j, t_arr, tag):
            nonlocal dropped
            si = s.size_index
            pi = s.pool_index(j)
            with lock:
                arrivals[tag] = (t_arr, s.stream_id, j)
            slot = srv.submit(sids[s.stream_id], pools.addrs[si][pi], s.W * 2, tag)
            if slot is None:
                with lock:
                    arrivals.pop(tag, None)
                    dropped += 1
                return False
            return True

        def producer():
            tag = 0
            for t_arr, sid, j in schedule:
                wake = t0 + t_arr
                while True:
                    d = wake - srv.clock()
                    if d <= 0:
                        break
                    time.sleep(min(d, 0.002))
                submit(streams[sid], j, wake, tag)
                tag += 1
            producer_done.set()

        tag_counter = [0]
        vq: "queue.Queue" = queue.Queue()
        vlock = threading.Lock()

        def verifier():
            # pinned read-back buffers: the copies then neither stage through
            # driver buffers nor hold the host thread longer than the transfer
            import torch
            scratch = {si: torch.empty(pools.frames[si][0].shape, dtype=torch.int16, pin_memory=True).numpy()
                       .view(np.uint16) for si in pools.frames}
            nonlocal verified, mismatches
            while True:
                item = vq.get()
                if item is None:
                    vq.task_done()
                    return
                sid, slot, j = item
                s = streams[sid]
                buf = scratch[s.size_index]
                srv.read(sids[sid], slot, buf)
                ok = frame_hash(buf) == ref[(s.size_index, s.pool_index(j), s.k)]
                with vlock:
                    verified += 1
                    mismatches += 0 if ok else 1
                    if keep_outputs:
                        outputs[(sid, j)] = buf.copy()
                srv.release(sids[sid], slot)
                if closed_loop and srv.clock() < deadline:
                    closed_submit(s)  # the stream's next frame, once its slot is back
                vq.task_done()

        deadline = t0 + duration_s
        verifiers = [threading.Thread(target=verifier, daemon=True) for _ in range(3)] if ref is not None else []
        for v in verifiers:
            v.start()

        def closed_submit(s):
            with lock:
                tag = tag_counter[0]
                tag_counter[0] += 1
                j = next_j[s.stream_id]
                next_j[s.stream_id] = j + 1
            return submit(s, j, srv.clock(), tag)

        if closed_loop:
            for s in streams:
                for _ in range(2):
                    closed_submit(s)
            th = None
        else:
            th = threading.Thread(target=producer, daemon=True)
            th.start()
        t_start = srv.clock()
        n_done = 0
        while True:
            comps = srv.poll()
            for c in comps:
                with lock:
                    t_arr, sid, j = arrivals.pop(c.tag)
                s = streams[sid]
                lat.append(c.t_done - t_arr)
                done_px += s.H * s.W
                n_done += 1
                if ref is not None and verify_every and n_done % verify_every == 0:
                    vq.put((sid, c.slot, j))  # the verifier releases the slot (and resubmits in closed loop)
                else:
                    srv.release(sids[sid], c.slot)
                    if closed_loop and srv.clock() < deadline:
                        closed_submit(s)
            if closed_loop:
                # a verifier marks its item done only after resubmitting, so
                # an empty queue and no arrivals mean nothing more will come
                if srv.clock() >= deadline and not arrivals and vq.unfinished_tasks == 0:
                    break
            elif producer_done.is_set() and not arrivals:
                break
            if srv.clock() > deadline + 30.0:
                raise RuntimeError(f"serving simulation did not drain: {len(arrivals)} frames outstanding")
            if not comps:
                time.sleep(0.0002)
        t_end = srv.clock()
        if th is not None:
            th.join()
        for _ in verifiers:
            vq.put(None)
        vq.join()
        for v in verifiers:
            v.join()
        st = srv.stats()
    finally:
        srv.close()
    lat_ms = np.array(lat) * 1e3
    span = max(t_end - t_start, 1e-9)
    res = {
        "streams": len(streams), "duration_s": round(span, 3), "closed_loop": closed_loop,
        "frames_completed": len(lat), "frames_dropped_busy": dropped,
        "mpx_s": round(done_px / span / 1e6, 1),
        "latency_ms": {"p50": round(float(np.percentile(lat_ms, 50)), 3) if len(lat) else None,
                       "p99": round(float(np.percentile(lat_ms, 99)), 3) if len(lat) else None,
                       "max": round(float(lat_ms.max()), 3) if len(lat) else None},
        "batches": st["batches"], "mean_batch_frames": round(st["frames_in_batches"] / max(1, st["batches"]), 2),
        "max_inflight_batches": st["max_inflight"], "device_bytes": st["device_bytes"],
        "verified": verified, "mismatches": mismatches,
    }
    if keep_outputs:
        res["outputs"] = outputs
    return res


def drive(streams: Sequence[synth.StreamSpec], pools: Pools, seconds: float, inflight: int = 2, plain: bool = False,
          device: int = 0) -> dict:
    """Closed-loop saturation through the library's native driver
    (``ir_server_drive``): served (batched) or plain (one launch per frame)."""
    srv = Server(device)
    try:
        sids = [srv.open_stream(s.H, s.W, synth.U14, s.k) for s in streams]
        n = len(streams)
        ids = (ctypes.c_int * n)(*sids)
        fr = (ctypes.c_void_p * n)(*[pools.addrs[s.size_index][s.pool_index(0)] for s in streams])
        pt = (ctypes.c_size_t * n)(*[s.W * 2 for s in streams])
        res = _lib.ir_drive_result()
        srv._err(srv.lib.ir_server_drive(srv.p, ids, fr, pt, n, seconds, inflight, 1 if plain else 0,
                                         ctypes.byref(res)))
        st = srv.stats()
    finally:
        srv.close()
    out = {"frames": res.frames, "mpx_s": round(res.megapixels / res.seconds, 1), "seconds": round(res.seconds, 3)}
    if not plain:
        out.update({"p50_ms": round(res.p50_ms, 3), "p99_ms": round(res.p99_ms, 3), "max_ms": round(res.max_ms, 3),
                    "mean_batch_frames": round(st["frames_in_batches"] / max(1, st["batches"]), 2),
                    "max_inflight_batches": st["max_inflight"]})
    return out


def plain_throughput(pools: Pools, streams: Sequence[synth.StreamSpec], frames: int, device: int = 0) -> float:
    """Mpx/s of the plain path on the same kind of traffic: one frame at a
    time, host->device copy from pinned memory, ir_filter_run2, stream order."""
    import torch
    flt = _lib.Filter(device)
    try:
        bufs = {}
        for si, fs in pools.frames.items():
            H, W = fs[0].shape
            bufs[si] = (torch.empty((H, W), dtype=torch.int16, device="cuda"),
                        torch.empty((H, W), dtype=torch.int16, device="cuda"))
        order = [(streams[i % len(streams)], i // len(streams)) for i in range(frames)]
        px = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s, j in order:
            d_in, d_out = bufs[s.size_index]
            d_in.copy_(pools.pinned[s.size_index][s.pool_index(j)], non_blocking=True)
            flt.run2(d_in, d_out, s.k, u14=True)
            px += s.H * s.W
        torch.cuda.synchronize()
        return px / (time.perf_counter() - t0) / 1e6
    finally:
        flt.close()
