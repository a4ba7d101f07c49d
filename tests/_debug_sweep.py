"""Parity sweep for the debug-check build of the library.

Run by tests/test_gpu_debug_checks.py in a process of its own whose
IRFNR_LIBRARY names libirfnr_debug.so (kernels built with FNR_DEBUG_CHECKS:
list indices, TMA coordinates and the launch layout are checked inside the
kernels, and a failed check is recorded as IR_ECHECK instead of faulting).
Covers every strategy, several tile shapes, every window, both pixel types,
all border readings, both detectors, odd shapes and pitches and a mixed
batch. Exit status 0 iff every output is bit-exact, no write leaves its frame
and no kernel check failed; the last line says what ran.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from _dev import download, empty_like_frame, guard_bytes_intact, upload  # noqa: E402
from paper_1201_3972_gb300 import _lib, synth  # noqa: E402


def algos_for(k):
    return [_lib.IR_ALGO_BITPLANE] + ([_lib.IR_ALGO_NETWORK] if k <= 9 else []) + \
        ([_lib.IR_ALGO_DENSE3] if k == 3 else []) + ([_lib.IR_ALGO_DENSE] if k in (5, 7) else [])


def tiles_for(es, k, algo):
    r = (k - 1) // 2
    xoff = -(-r // (16 // es)) * (16 // es)
    rg = 8 if k >= 8 else (4 if k >= 4 else 2)
    mult = 8 * (2 if algo in (_lib.IR_ALGO_DENSE3, _lib.IR_ALGO_DENSE) else rg)
    return [(tw, th) for tw, th in ((64, 64), (32, 16), (128, 32), (32, 128))
            if tw + 2 * xoff <= 256 and th + 2 * r <= 256 and (tw * es) % 16 == 0 and th % mult == 0]


def main() -> int:
    assert os.path.basename(_lib.library_path()) == "libirfnr_debug.so", _lib.library_path()
    flt = _lib.Filter(0)
    flt.set_tile_fit(False)   # every tile shape exactly as configured
    rng = np.random.default_rng(2026)
    runs = 0
    for k in (3, 5, 7, 9, 11, 15, 21):
        for es, dt in ((1, _lib.IR_U8), (2, _lib.IR_U16)):
            npdt = np.uint8 if es == 1 else np.uint16
            for algo in algos_for(k):
                for tw, th in tiles_for(es, k, algo):
                    flt.set_config(dt, k, tw, th, algo)
                    for border, detector in (("replicate", "extreme"), ("mirror", "directional"), ("zero", "extreme")):
                        flt.set_border(border)
                        flt.set_detector(detector)
                        for H, W, pitch in ((57, 133, 144), (57, 133, 139), (3, 5, 16), (130, 70, 80)):
                            a = rng.integers(0, 256 if es == 1 else 65536, (H, W)).astype(npdt)
                            if detector == "directional":
                                want, wf = oracle.fnr_directional(a, k, border)
                            else:
                                want, wf = oracle.fnr_border(a, k, border)
                            ib, ia, ip = upload(a, pitch)
                            ob, oa, op = empty_like_frame(a, pitch)
                            ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
                            flt.ir_filter_run2(ia, ip, oa, op, H, W, dt, k, None, ctr)
                            got = download(ob, oa, op, H, W, npdt)
                            tag = f"k{k} es{es} algo{algo} {tw}x{th} {border} {detector} {H}x{W} p{pitch}"
                            if not np.array_equal(got, want) or int(ctr.item()) != wf:
                                print("MISMATCH", tag)
                                return 1
                            if not guard_bytes_intact(ob, oa, op, H, W, es):
                                print("WRITE OUTSIDE THE FRAME", tag)
                                return 1
                            runs += 1
                    flt.sync_status()  # raises IrError(IR_ECHECK) if a kernel check failed
                flt.set_config(dt, k, 0, 0, _lib.IR_ALGO_AUTO)
    flt.set_border("replicate")
    flt.set_detector("extreme")
    # a mixed batch through the default configurations, with per-frame counts
    frames = []
    for i in range(20):
        H, W = int(rng.integers(1, 140)), int(rng.integers(1, 300))
        k = int(rng.choice([3, 5, 7, 9, 13, 21]))
        u8 = bool(i % 2)
        a = synth.make_frame(H, W, synth.U8 if u8 else synth.U14, 500 + i, 2.0 if u8 else 8.0, 0.2)
        frames.append((a, k, u8))
    staged = []
    arr = (_lib.ir_frame_desc * len(frames))()
    for i, (a, k, u8) in enumerate(frames):
        ib, ia, ip = upload(a)
        ob, oa, op = empty_like_frame(a)
        ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
        staged.append((ib, ob, oa, op, ctr))
        arr[i].in_, arr[i].out, arr[i].H, arr[i].W = ia, oa, a.shape[0], a.shape[1]
        arr[i].in_pitch, arr[i].out_pitch, arr[i].k = ip, op, k
        arr[i].dtype = _lib.IR_U8 if u8 else _lib.IR_U14
        arr[i].flagged_count = int(ctr.data_ptr())
    flt.ir_filter_run_batch(arr, len(frames))
    for (a, k, u8), (ib, ob, oa, op, ctr) in zip(frames, staged):
        want, wf = oracle.fnr(a, k)
        if not np.array_equal(download(ob, oa, op, a.shape[0], a.shape[1], a.dtype), want) or int(ctr.item()) != wf:
            print("BATCH MISMATCH", a.shape, k)
            return 1
        runs += 1
    flt.sync_status()
    flt.close()
    print(f"debug-check build: {runs} runs bit-exact, no kernel check failed")
    return 0


if __name__ == "__main__":
    sys.exit(main())
