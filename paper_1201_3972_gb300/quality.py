"""Noise-reduction quality of FNR against the standard median filter (MF).

The paper's Table 1 compares MF and FNR on one 364x244 8-bit IR image with
20% and 30% impulse noise: the number of sorts (medians taken), the time,
and PSNR (Eq. 5: 10 log10(MAX^2 / MSE) against the noise-free image). That
image is not available, so ``table1`` runs the same comparison on seeded
synthetic frames of the same size (and a 14-bit variant) whose noise-free
version is known, through the library's CUDA entry points.
"""
from __future__ import annotations

import time
from typing import Dict

import numpy as np

from . import _lib, synth


def psnr(img: np.ndarray, ref: np.ndarray, maxv: int) -> float:
    """Eq. 5: 10 log10(MAX^2 / MSE); infinite for identical images."""
    mse = np.mean((img.astype(np.float64) - ref.astype(np.float64)) ** 2)
    return float("inf") if mse == 0 else float(10.0 * np.log10(maxv * maxv / mse))


def clean_and_noisy(H: int, W: int, dtype: int, p: float, seed: int):
    """A noise-free synthetic IR frame (T^4 field + sensor noise) and the same
    frame with salt-and-pepper impulses of density p."""
    maxv = synth.MAXV[dtype]
    rng = np.random.Generator(np.random.PCG64(seed))
    g = synth.emittance_to_gray(synth.thermal_field(rng, H, W), maxv) + rng.normal(0, synth.sigma_for(dtype), (H, W))
    clean = np.clip(np.rint(g), 0, maxv).astype(synth.NP_DTYPE[dtype])
    return clean, synth.add_impulses(rng, clean, p, maxv, "sp")


def table1(flt: _lib.Filter, k: int = 3, H: int = 244, W: int = 364) -> Dict[str, dict]:
    """PSNR, sort counts and GPU time of MF and FNR (one and two passes) at
    20% and 30% impulses, u8 and 14-bit."""
    import torch
    out = {}
    for dtype, name in ((synth.U8, "u8"), (synth.U14, "u14")):
        maxv = synth.MAXV[dtype]
        for p in (0.20, 0.30):
            clean, noisy = clean_and_noisy(H, W, dtype, p, synth.seed_for(5, int(p * 100) + 10 * dtype))
            t = torch.from_numpy(noisy.view(np.int16) if noisy.dtype == np.uint16 else noisy).cuda()
            res = {"noisy_psnr": round(psnr(noisy, clean, maxv), 2)}
            for label, call in (("mf", "median"), ("fnr", "fnr")):
                for passes in (1, 2):
                    dst = torch.empty_like(t)
                    ctr = torch.zeros(passes, dtype=torch.int64, device="cuda")
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    if call == "median":
                        src = t
                        for q in range(passes):
                            nxt = torch.empty_like(t)
                            flt.median_filter(src, nxt, k, u14=dtype == synth.U14, median_count=ctr[q:q + 1])
                            src = nxt
                        dst = src
                    else:
                        flt.run_passes(t, dst, k, passes, u14=dtype == synth.U14, flagged_per_pass=ctr)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                    img = dst.cpu().numpy().view(noisy.dtype)
                    res[f"{label}{passes}_psnr"] = round(psnr(img, clean, maxv), 2)
                    res[f"{label}{passes}_sorts"] = [int(v) for v in ctr.cpu().tolist()]
                    res[f"{label}{passes}_ms"] = round(dt * 1e3, 3)
            out[f"{name}_{int(p * 100)}pct"] = res
    return out


def retention(out: np.ndarray, pre: np.ndarray, noisy: np.ndarray, mask: np.ndarray, maxv: int) -> dict:
    """Detail retention on thin structures: over the structure pixels that no
    impulse hit (mask & noisy == pre), the fraction the filter left at their
    value before impulses, and the PSNR there against that value."""
    sel = mask & (noisy == pre)
    n = int(sel.sum())
    if n == 0:
        return {"pixels": 0, "kept": None, "psnr": None}
    return {"pixels": n, "kept": round(float(np.mean(out[sel] == pre[sel])), 4),
            "psnr": round(psnr(out[sel], pre[sel], maxv), 2)}


def detail_retention(flt: _lib.Filter, ks=(3, 5, 7), p: float = 0.10) -> Dict[str, dict]:
    """How FNR and the median filter treat 1-pixel hot lines and 2x2 hot
    targets (the detail the paper says FNR keeps, Sec. 4): a 640x512 14-bit
    frame with the sweep's thin structures, sensor noise and 10%
    salt-and-pepper, filtered once by each; reported, not asserted (under the
    literal flag rule a line pixel that is its window's maximum is replaced)."""
    import torch
    dtype = synth.U14
    maxv = synth.MAXV[dtype]
    noisy, pre, mask = synth.make_frame_parts(512, 640, dtype, synth.seed_for(6, 1), synth.sigma_for(dtype), p,
                                              "sp", True)
    src = torch.from_numpy(noisy.view(np.int16)).cuda()
    out = {"frame": "640x512 14-bit, thin structures, sigma 8 DN, 10% salt-and-pepper",
           "noisy_frame_psnr": round(psnr(noisy, pre, maxv), 2)}
    for k in ks:
        res = {}
        for label in ("fnr", "mf"):
            dst = torch.empty_like(src)
            if label == "fnr":
                flt.run2(src, dst, k, u14=True)
            else:
                flt.median_filter(src, dst, k, u14=True)
            img = dst.cpu().numpy().view(np.uint16)
            r = retention(img, pre, noisy, mask, maxv)
            res[label] = {"structure": r, "frame_psnr": round(psnr(img, pre, maxv), 2)}
        out[f"k{k}"] = res
    return out
