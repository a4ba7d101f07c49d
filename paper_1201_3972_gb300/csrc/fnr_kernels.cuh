// Device code of the FNR impulse filter (arXiv 1201.3972, Sec. 3.3-3.4).
//
// One persistent kernel per (pixel type, window k, selection strategy). A CTA
// walks a strided list of output tiles; for each tile it
//   1. stages the tile plus a k-1 pixel halo in shared memory with a 2-D TMA
//      load (double-buffered: the next tile's load is in flight while this one
//      is computed), or with plain clamped loads when the frame is not 16-byte
//      aligned, and replicates the frame border into the zero-filled part;
//   2. computes g_min and g_max of every window (Eq. 3a/3b) and flags the
//      pixels equal to one of them (Sec. 3.3, step 2);
//   3. replaces flagged pixels by the window median g_m (Sec. 3.4);
//   4. writes the output tile with a TMA store (or plain stores).
// All arithmetic is integer min/max/compare, so results are bit-exact.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "fnr_networks.cuh"
#include "fnr_params.h"

namespace fnr {

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA (cp.async.bulk.tensor), proxy fences.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for phase `parity` of `bar`, giving up after `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_addr(src)), "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) accesses of the same bytes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Packed 2 x u16 min / max (one instruction each on sm_90 and later).
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

struct ScalarOp {
  __device__ __forceinline__ uint32_t mn(uint32_t a, uint32_t b) const { return a < b ? a : b; }
  __device__ __forceinline__ uint32_t mx(uint32_t a, uint32_t b) const { return a < b ? b : a; }
};

constexpr long long kWaitCycles = 2000000000LL;  // about one second at GB300 clocks

// ---------------------------------------------------------------------------
// Tile bookkeeping.
// ---------------------------------------------------------------------------
// Where the tiles of one launch come from. Frames are contiguous ranges of
// the launch's tile index space (tile_begin); a tile is (frame, tile in frame).
struct TileInfo {
  int valid, f, tl, W, H, tiles_x, flags, pad;
};

__device__ __forceinline__ const FrameDev *frame_ptr(const FnrParams &p, int f) {
  return p.table == nullptr ? &p.single : p.table + f;
}

// Thread 0 resolves tile t; `dir` is the shared-memory copy of every frame's
// tile_begin when the launch has at most kDirMax frames (else the table is
// searched in global memory).
__device__ __forceinline__ TileInfo locate_tile(const FnrParams &p, const int *dir, int t) {
  TileInfo ti{};
  if (t >= p.total_tiles) return ti;
  int f = 0;
  if (p.table != nullptr) {
    int lo = 0, hi = p.nframes - 1;
    const bool in_smem = p.nframes <= kDirMax;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      const int tb = in_smem ? dir[mid] : p.table[mid].tile_begin;
      if (tb <= t) lo = mid;
      else hi = mid - 1;
    }
    f = lo;
  }
  const FrameDev *fd = frame_ptr(p, f);
  ti.valid = 1;
  ti.f = f;
  ti.tl = t - fd->tile_begin;
  ti.W = fd->W;
  ti.H = fd->H;
  ti.tiles_x = fd->tiles_x;
  ti.flags = fd->flags;
  return ti;
}

template <typename T>
__device__ __forceinline__ T load_global(const unsigned char *base, long long pitch, int y, int x) {
  return __ldg(reinterpret_cast<const T *>(base + (long long)y * pitch) + x);
}

// Plain staging for frames TMA cannot address: clamped coordinates give the
// replicated border directly.
template <typename T>
__device__ void plain_tile_load(const FrameDev *f, int xs, int ys, T *S, int BW, int BH) {
  const int H = f->H, W = f->W;
  for (int i = threadIdx.x; i < BW * BH; i += kThreads) {
    const int row = i / BW, col = i - row * BW;
    int gy = ys + row, gx = xs + col;
    gy = gy < 0 ? 0 : (gy >= H ? H - 1 : gy);
    gx = gx < 0 ? 0 : (gx >= W ? W - 1 : gx);
    S[i] = load_global<T>(f->in, f->in_pitch, gy, gx);
  }
}

// TMA fills out-of-frame cells with zero; overwrite them with the nearest
// in-frame row, then column (replicate border). Only out-of-frame cells are
// touched: whole rows move as 16-byte chunks, columns one thread per row.
template <typename T>
__device__ void fixup_border(T *S, int xs, int ys, int BW, int BH, int W, int H) {
  const int top = -ys;         // rows [0, top) lie above the frame
  const int bot = H - 1 - ys;  // rows (bot, BH) lie below it
  const int ntop = top > 0 ? top : 0;
  const int nbot = bot < BH - 1 ? BH - 1 - bot : 0;
  if (ntop + nbot > 0) {
    const int chunks = BW * static_cast<int>(sizeof(T)) / 16;
    const int items = (ntop + nbot) * chunks;
    for (int i = threadIdx.x; i < items; i += kThreads) {
      const int rr = i / chunks, c = i - rr * chunks;
      const int row = rr < ntop ? rr : bot + 1 + (rr - ntop);
      const int src = rr < ntop ? top : bot;
      reinterpret_cast<uint4 *>(S + row * BW)[c] = reinterpret_cast<const uint4 *>(S + src * BW)[c];
    }
    __syncthreads();
  }
  const int lft = -xs;         // columns [0, lft) lie left of the frame
  const int rgt = W - 1 - xs;  // columns (rgt, BW) lie right of it
  if (lft > 0 || rgt < BW - 1) {
    for (int row = threadIdx.x; row < BH; row += kThreads) {
      T *R = S + row * BW;
      if (lft > 0) {
        const T v = R[lft];
        for (int j = 0; j < lft; ++j) R[j] = v;
      }
      if (rgt < BW - 1) {
        const T v = R[rgt];
        for (int j = rgt + 1; j < BW; ++j) R[j] = v;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__device__ void plain_tile_store(const FrameDev *f, const T *O, int x0, int y0, int TW, int TH) {
  const int H = f->H, W = f->W;
  for (int i = threadIdx.x; i < TW * TH; i += kThreads) {
    const int row = i / TW, col = i - row * TW;
    const int gy = y0 + row, gx = x0 + col;
    if (gy < H && gx < W) reinterpret_cast<T *>(f->out + (long long)gy * f->out_pitch)[gx] = O[i];
  }
}

// ---------------------------------------------------------------------------
// DENSE3: k = 3, median for every pixel.
//
// A thread owns 8 consecutive outputs in 2 consecutive rows. Pixels are held
// as packed pairs (x, x+1) of 16-bit lanes. Each of the 4 input rows gives 6
// even-aligned pair words E_-1..E_4 covering columns x-2..x+9. Columns are
// sorted vertically once (sort of the shared middle two rows, then one
// insertion per output row), and the odd-aligned pairs (x-1,x), (x+1,x+2)...
// are byte-permutes of the sorted even words (sorting is per lane). For the 3
// sorted columns L, M, R of a window:
//   g_min = min(lo), g_max = max(hi),
//   g_m   = med3(max(lo), med3(mid), min(hi))  (the median of a 3x3 set whose
//           columns are sorted; pinned by the 0-1 principle in the tests).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void load_row8(const T *p, uint32_t (&e)[6]);

template <>
__device__ __forceinline__ void load_row8<uint16_t>(const uint16_t *p, uint32_t (&e)[6]) {
  const uint4 c = *reinterpret_cast<const uint4 *>(p);
  e[0] = *reinterpret_cast<const uint32_t *>(p - 2);
  e[1] = c.x; e[2] = c.y; e[3] = c.z; e[4] = c.w;
  e[5] = *reinterpret_cast<const uint32_t *>(p + 8);
}

template <>
__device__ __forceinline__ void load_row8<uint8_t>(const uint8_t *p, uint32_t (&e)[6]) {
  const uint2 c = *reinterpret_cast<const uint2 *>(p);
  const uint32_t l = *reinterpret_cast<const uint32_t *>(p - 4);
  const uint32_t r = *reinterpret_cast<const uint32_t *>(p + 8);
  e[0] = __byte_perm(l, 0, 0x4342);
  e[1] = __byte_perm(c.x, 0, 0x4140);
  e[2] = __byte_perm(c.x, 0, 0x4342);
  e[3] = __byte_perm(c.y, 0, 0x4140);
  e[4] = __byte_perm(c.y, 0, 0x4342);
  e[5] = __byte_perm(r, 0, 0x4140);
}

template <typename T>
__device__ __forceinline__ void store_row8(T *q, const uint32_t (&v)[4]);

template <>
__device__ __forceinline__ void store_row8<uint16_t>(uint16_t *q, const uint32_t (&v)[4]) {
  *reinterpret_cast<uint4 *>(q) = make_uint4(v[0], v[1], v[2], v[3]);
}

template <>
__device__ __forceinline__ void store_row8<uint8_t>(uint8_t *q, const uint32_t (&v)[4]) {
  *reinterpret_cast<uint2 *>(q) = make_uint2(__byte_perm(v[0], v[1], 0x6420), __byte_perm(v[2], v[3], 0x6420));
}

__device__ __forceinline__ uint32_t med3v(uint32_t a, uint32_t b, uint32_t c) {
  return vmax2(vmin2(a, b), vmin2(vmax2(a, b), c));
}

// (hi lane of a, lo lane of b): the odd-aligned pair between two even pairs.
__device__ __forceinline__ uint32_t odd_pair(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5432); }

// Per 16-bit lane: 1 where g_min < c < g_max (signal pixel), 0 where c equals
// g_min or g_max (noisy). c - g_min and g_max - c never borrow across lanes
// because every lane satisfies g_min <= c <= g_max.
__device__ __forceinline__ uint32_t signal_bits(uint32_t c, uint32_t gmin, uint32_t gmax) {
  return vmin2(vmin2(c - gmin, gmax - c), 0x00010001u);
}

// tw_valid, th_valid: the part of the tile inside the frame (only those
// pixels are counted as flagged; the rest is never stored).
template <typename T, bool COUNT>
__device__ void dense3_tile(const T *S, T *O, int TW, int TH, int BW, int tw_valid, int th_valid, int &flagged) {
  constexpr int XOFF = xoff_for(1, sizeof(T));
  const int segs = TW >> 3;
  const int items = (TH >> 1) * segs;
  for (int it = threadIdx.x; it < items; it += kThreads) {
    const int sx = it % segs, ry = it / segs;
    const int tx = sx << 3, ty = ry << 1;
    uint32_t e[4][6];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) load_row8<T>(S + (ty + rr) * BW + XOFF + tx, e[rr]);
    uint32_t lo[2][6], md[2][6], hi[2][6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const uint32_t bl = vmin2(e[1][q], e[2][q]);
      const uint32_t bh = vmax2(e[1][q], e[2][q]);
      lo[0][q] = vmin2(e[0][q], bl);
      hi[0][q] = vmax2(e[0][q], bh);
      md[0][q] = vmax2(bl, vmin2(e[0][q], bh));
      lo[1][q] = vmin2(e[3][q], bl);
      hi[1][q] = vmax2(e[3][q], bh);
      md[1][q] = vmax2(bl, vmin2(e[3][q], bh));
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      uint32_t olo[5], omd[5], ohi[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        olo[q] = odd_pair(lo[o][q], lo[o][q + 1]);
        omd[q] = odd_pair(md[o][q], md[o][q + 1]);
        ohi[q] = odd_pair(hi[o][q], hi[o][q + 1]);
      }
      uint32_t res[4];
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) {
        const uint32_t mlo = lo[o][pp + 1], mmd = md[o][pp + 1], mhi = hi[o][pp + 1];
        const uint32_t maxlo = vmax2(vmax2(olo[pp], mlo), olo[pp + 1]);
        const uint32_t gmin = vmin2(vmin2(olo[pp], mlo), olo[pp + 1]);
        const uint32_t medmd = med3v(omd[pp], mmd, omd[pp + 1]);
        const uint32_t minhi = vmin2(vmin2(ohi[pp], mhi), ohi[pp + 1]);
        const uint32_t gmax = vmax2(vmax2(ohi[pp], mhi), ohi[pp + 1]);
        const uint32_t gm = med3v(maxlo, medmd, minhi);
        const uint32_t c = e[1 + o][pp + 1];
        const uint32_t sig = signal_bits(c, gmin, gmax);
        const uint32_t keep = sig * 0xffffu;
        res[pp] = (c & keep) | (gm & ~keep);
        if constexpr (COUNT) {
          const int col = tx + 2 * pp;
          const uint32_t valid =
              (ty + o < th_valid) ? ((col < tw_valid ? 1u : 0u) | (col + 1 < tw_valid ? 0x10000u : 0u)) : 0u;
          flagged += __popc((sig ^ 0x00010001u) & valid);
        }
      }
      store_row8<T>(O + (ty + o) * TW + tx, res);
    }
  }
}

// ---------------------------------------------------------------------------
// Compacted strategies (any k): separable g_min/g_max, flag, list of flagged
// pixels, then one median per flagged pixel.
// ---------------------------------------------------------------------------

// Sliding extreme over windows [q, q+K-1], q = 0..RG-1, of RG+K-1 values,
// sharing the core [RG-1, K-1] common to all windows (RG <= K).
template <int K, int RG, bool MAX>
__device__ __forceinline__ void sliding_extreme(const uint32_t (&v)[RG + K - 1], uint32_t (&out)[RG]) {
  auto op = [](uint32_t a, uint32_t b) { return MAX ? (a < b ? b : a) : (a < b ? a : b); };
  uint32_t core = v[RG - 1];
#pragma unroll
  for (int i = RG; i <= K - 1; ++i) core = op(core, v[i]);
  uint32_t suf[RG], pre[RG];
  if constexpr (RG >= 2) {
    suf[RG - 2] = v[RG - 2];
#pragma unroll
    for (int q = RG - 3; q >= 0; --q) suf[q] = op(v[q], suf[q + 1]);
    pre[1] = v[K];
#pragma unroll
    for (int q = 2; q < RG; ++q) pre[q] = op(pre[q - 1], v[K - 1 + q]);
  }
#pragma unroll
  for (int q = 0; q < RG; ++q) {
    uint32_t a = core;
    if (q <= RG - 2) a = op(a, suf[q]);
    if (q >= 1) a = op(a, pre[q]);
    out[q] = a;
  }
}

template <int K>
struct RowGroup {
  static constexpr int value = K >= 8 ? 8 : (K >= 4 ? 4 : 2);
};

// Vertical pass: vmin/vmax[ty][j] = min/max of stage column (XOFF-R+j) over
// rows ty..ty+K-1, for ty < TH and j < TW + K - 1.
template <typename T, int K>
__device__ void vertical_pass(const T *S, uint16_t *vmin, uint16_t *vmax, int TW, int TH, int BW, int VW) {
  constexpr int R = (K - 1) / 2, RG = RowGroup<K>::value;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  const int items = VW * (TH / RG);
  for (int it = threadIdx.x; it < items; it += kThreads) {
    const int j = it % VW, g = it / VW;
    const T *col = S + g * RG * BW + (XOFF - R) + j;
    uint32_t v[RG + K - 1];
#pragma unroll
    for (int i = 0; i < RG + K - 1; ++i) v[i] = col[i * BW];
    uint32_t mn[RG], mx[RG];
    sliding_extreme<K, RG, false>(v, mn);
    sliding_extreme<K, RG, true>(v, mx);
#pragma unroll
    for (int q = 0; q < RG; ++q) {
      vmin[(g * RG + q) * VW + j] = static_cast<uint16_t>(mn[q]);
      vmax[(g * RG + q) * VW + j] = static_cast<uint16_t>(mx[q]);
    }
  }
}

// Horizontal pass + flag: writes every centre value to the output tile and
// appends flagged pixels (ty << 8 | tx) to the list. Returns nothing; the
// list length accumulates in *count.
template <typename T, int K>
__device__ void horizontal_flag_pass(const T *S, const uint16_t *vmin, const uint16_t *vmax, T *O,
                                     uint16_t *list, unsigned *count, int TW, int TH, int BW, int VW, int tw_valid,
                                     int th_valid) {
  constexpr int R = (K - 1) / 2, RG = RowGroup<K>::value;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  const int per_row = TW / RG;
  const int items = TH * per_row;
  const int lane = threadIdx.x & 31;
  for (int it0 = 0; it0 < items; it0 += kThreads) {
    const int it = it0 + threadIdx.x;
    uint32_t fm = 0;
    int ty = 0, tx0 = 0;
    if (it < items) {
      ty = it / per_row;
      tx0 = (it - ty * per_row) * RG;
      uint32_t hmn[RG + K - 1], hmx[RG + K - 1];
#pragma unroll
      for (int i = 0; i < RG + K - 1; ++i) {
        hmn[i] = vmin[ty * VW + tx0 + i];
        hmx[i] = vmax[ty * VW + tx0 + i];
      }
      uint32_t gmin[RG], gmax[RG];
      sliding_extreme<K, RG, false>(hmn, gmin);
      sliding_extreme<K, RG, true>(hmx, gmax);
      const T *crow = S + (ty + R) * BW + XOFF + tx0;
#pragma unroll
      for (int q = 0; q < RG; ++q) {
        const uint32_t c = crow[q];
        O[ty * TW + tx0 + q] = static_cast<T>(c);
        const bool inside = ty < th_valid && tx0 + q < tw_valid;
        fm |= static_cast<uint32_t>(inside && (c == gmin[q] || c == gmax[q])) << q;
      }
    }
    // warp-aggregated append
    const int cnt = __popc(fm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int base = 0;
    if (lane == 31 && total) base = static_cast<int>(atomicAdd(count, static_cast<unsigned>(total)));
    base = __shfl_sync(0xffffffffu, base, 31);
    int pos = base + incl - cnt;
#pragma unroll
    for (int q = 0; q < RG; ++q)
      if ((fm >> q) & 1u) list[pos++] = static_cast<uint16_t>((ty << 8) | (tx0 + q));
  }
}

struct PackedOp {
  __device__ __forceinline__ uint32_t mn(uint32_t a, uint32_t b) const { return vmin2(a, b); }
  __device__ __forceinline__ uint32_t mx(uint32_t a, uint32_t b) const { return vmax2(a, b); }
};

// Flagged pixels, two per thread: the two k x k windows are gathered into the
// low and high 16-bit lanes of the same registers and one packed selection
// network serves both (an odd tail pixel is paired with itself).
template <typename T, int K>
__device__ void network_medians(const T *S, T *O, const uint16_t *list, int F, int TW, int BW) {
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  const int pairs = (F + 1) >> 1;
  for (int i = threadIdx.x; i < pairs; i += kThreads) {
    const int ea = list[2 * i];
    const int eb = 2 * i + 1 < F ? list[2 * i + 1] : ea;
    const T *ba = S + (ea >> 8) * BW + (XOFF - R) + (ea & 255);
    const T *bb = S + (eb >> 8) * BW + (XOFF - R) + (eb & 255);
    uint32_t v[K * K];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = 0; b < K; ++b)
        v[a * K + b] = static_cast<uint32_t>(ba[a * BW + b]) | (static_cast<uint32_t>(bb[a * BW + b]) << 16);
    const uint32_t m = MedianNet<K>::run(v, PackedOp{});
    O[(ea >> 8) * TW + (ea & 255)] = static_cast<T>(m & 0xffffu);
    O[(eb >> 8) * TW + (eb & 255)] = static_cast<T>(m >> 16);
  }
}

// Bit planes of the staged tile: plane b, row i, word w holds bit b of the
// 32 pixels of row i starting at column 32w. One ballot per (row, word, bit).
template <typename T>
__device__ void build_planes(const T *S, uint32_t *planes, unsigned *tile_or, int BW, int BH, int PW, int NBMAX) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wpr = PW - 1;
  const int items = BH * wpr;
  uint32_t orv = 0;
  for (int it = warp; it < items; it += kThreads / 32) {
    const int row = it / wpr, w = it - row * wpr;
    const int col = (w << 5) + lane;
    const uint32_t v = col < BW ? static_cast<uint32_t>(S[row * BW + col]) : 0u;
    orv |= v;
    uint32_t mine = 0;
    for (int b = 0; b < NBMAX; ++b) {
      const uint32_t bits = __ballot_sync(0xffffffffu, (v >> b) & 1u);
      if (lane == b) mine = bits;
    }
    if (lane < NBMAX) planes[(lane * BH + row) * PW + w] = mine;
  }
  for (int it = threadIdx.x; it < NBMAX * BH; it += kThreads) planes[it * PW + wpr] = 0u;
  orv = __reduce_or_sync(0xffffffffu, orv);
  if (lane == 0 && orv) atomicOr(tile_or, orv);
}

// Flagged pixels: radix select on the window, most significant bit first.
// alive[a] marks the window pixels of row a whose bits above the current bit
// match the answer so far; each round counts the live pixels with a 0 bit.
template <int K>
__device__ void bitplane_medians(const uint32_t *planes, uint16_t *O16, uint8_t *O8, bool is16,
                                 const uint16_t *list, int F, int TW, int BH, int PW, int NB, int XOFF) {
  constexpr int R = (K - 1) / 2;
  constexpr uint32_t kMask = (1u << K) - 1u;
  for (int i = threadIdx.x; i < F; i += kThreads) {
    const int e = list[i];
    const int ty = e >> 8, tx = e & 255;
    const int c0 = XOFF - R + tx;
    const int wi = c0 >> 5, sh = c0 & 31;
    uint32_t alive[K];
#pragma unroll
    for (int a = 0; a < K; ++a) alive[a] = kMask;
    uint32_t rank = (K * K - 1) / 2, res = 0;
    for (int b = NB - 1; b >= 0; --b) {
      const uint32_t *P = planes + (b * BH + ty) * PW + wi;
      uint32_t seg[K];
      uint32_t cnt = 0;
#pragma unroll
      for (int a = 0; a < K; ++a) {
        seg[a] = __funnelshift_r(P[a * PW], P[a * PW + 1], sh);
        cnt += __popc(alive[a] & ~seg[a]);
      }
      if (rank < cnt) {
#pragma unroll
        for (int a = 0; a < K; ++a) alive[a] &= ~seg[a];
      } else {
        rank -= cnt;
        res |= 1u << b;
#pragma unroll
        for (int a = 0; a < K; ++a) alive[a] &= seg[a];
      }
    }
    if (is16) O16[ty * TW + tx] = static_cast<uint16_t>(res);
    else O8[ty * TW + tx] = static_cast<uint8_t>(res);
  }
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <typename T, int K, int ALGO>
__global__ void __launch_bounds__(kThreads, (ALGO == ALGO_NETWORK ? 3 : 2)) fnr_kernel(const __grid_constant__ FnrParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int E = sizeof(T);
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, E);
  static_assert(ALGO != ALGO_DENSE3 || K == 3, "DENSE3 is the 3x3 window only");

  const int TW = p.tile_w, TH = p.tile_h;
  const Layout L = make_layout(E, K, ALGO, TH, TW);
  const int BW = L.bw, BH = L.bh;
  const uint32_t box_bytes = static_cast<uint32_t>(BW * BH * E);
  T *const stage0 = reinterpret_cast<T *>(smem + L.off_stage[0]);
  T *const stage1 = reinterpret_cast<T *>(smem + L.off_stage[1]);
  T *const out0 = reinterpret_cast<T *>(smem + L.off_out[0]);
  T *const out1 = reinterpret_cast<T *>(smem + L.off_out[1]);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L.off_bar);
  unsigned *misc = reinterpret_cast<unsigned *>(smem + L.off_misc);  // [0] flagged count, [1] tile OR
  TileInfo *info = reinterpret_cast<TileInfo *>(smem + L.off_info);  // [stage]: tile staged there
  int *dir = reinterpret_cast<int *>(smem + L.off_dir);
  const int tid = threadIdx.x;

  if (p.table != nullptr && p.nframes <= kDirMax)
    for (int f = tid; f < p.nframes; f += kThreads) dir[f] = p.table[f].tile_begin;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if (blockIdx.x == 0 && p.launches != nullptr) atomicAdd(p.launches, 1ull);
  }
  __syncthreads();

  auto issue = [&](const TileInfo &ti, T *dst, uint64_t *b) {
    const int gx = (ti.tl % ti.tiles_x) * TW - XOFF;
    const int gy = (ti.tl / ti.tiles_x) * TH - R;
    mbar_arrive_expect_tx(b, box_bytes);
    tma_load_2d(dst, &frame_ptr(p, ti.f)->tin, b, gx, gy);
  };

  if (tid == 0) {
    const TileInfo first = locate_tile(p, dir, blockIdx.x);
    info[0] = first;
    if (first.valid && (first.flags & kFrameTmaIn)) issue(first, stage0, &bar[0]);
  }
  __syncthreads();

  uint32_t phase = 0;
  int t = blockIdx.x;
  for (int i = 0;; ++i, t += static_cast<int>(gridDim.x)) {
    const int s = i & 1;
    const TileInfo cur = info[s];
    if (!cur.valid) break;
    const FrameDev *cf = frame_ptr(p, cur.f);
    if (tid == 0) {
      // resolve and prefetch the next tile into the other stage (its previous
      // tile finished with the barrier that ended the last iteration)
      const TileInfo nx = locate_tile(p, dir, t + static_cast<int>(gridDim.x));
      info[s ^ 1] = nx;
      if (nx.valid && (nx.flags & kFrameTmaIn)) {
        fence_proxy_async_smem();
        issue(nx, s ? stage0 : stage1, &bar[s ^ 1]);
      }
      misc[0] = 0;
      misc[1] = 0;
      bulk_wait_read<1>();  // the store that last read this output buffer (two tiles ago) is done
    }

    const int x0 = (cur.tl % cur.tiles_x) * TW, y0 = (cur.tl / cur.tiles_x) * TH;
    const int xs = x0 - XOFF, ys = y0 - R;
    const bool tma_in = (cur.flags & kFrameTmaIn) != 0;
    // A TMA store clips the box at the frame edge in whole 16-byte units, so a
    // right-edge tile of a frame whose row is not a multiple of 16 bytes would
    // touch the bytes between W and the pitch: such tiles use plain stores.
    const bool ragged_right = x0 + TW > cur.W && ((cur.W * E) & 15) != 0;
    const bool tma_out = (cur.flags & kFrameTmaOut) != 0 && !ragged_right;
    T *const S = s ? stage1 : stage0;
    T *const O = s ? out1 : out0;

    bool ok = true;
    if (tma_in) {
      ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u, kWaitCycles);
      phase ^= 1u << s;
    } else {
      plain_tile_load<T>(cf, xs, ys, S, BW, BH);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(p.status, kStatusTimeout);
        const TileInfo nx = info[s ^ 1];
        if (nx.valid && (nx.flags & kFrameTmaIn))
          mbar_wait_bounded(&bar[s ^ 1], (phase >> (s ^ 1)) & 1u, kWaitCycles);
      }
      break;
    }
    if (tma_in && (xs < 0 || ys < 0 || xs + BW > cur.W || ys + BH > cur.H))
      fixup_border<T>(S, xs, ys, BW, BH, cur.W, cur.H);

    if constexpr (ALGO == ALGO_DENSE3) {
      int flagged = 0;
      if (cf->flagged != nullptr) {
        dense3_tile<T, true>(S, O, TW, TH, BW, cur.W - x0, cur.H - y0, flagged);
        flagged = __reduce_add_sync(0xffffffffu, flagged);
        if ((tid & 31) == 0 && flagged) atomicAdd(&misc[0], static_cast<unsigned>(flagged));
      } else {
        dense3_tile<T, false>(S, O, TW, TH, BW, cur.W - x0, cur.H - y0, flagged);
      }
    } else {
      uint16_t *list = reinterpret_cast<uint16_t *>(smem + L.off_list);
      uint16_t *vmin = reinterpret_cast<uint16_t *>(smem + L.off_vmin);
      uint16_t *vmax = reinterpret_cast<uint16_t *>(smem + L.off_vmax);
      if constexpr (ALGO == ALGO_BITPLANE) {
        build_planes<T>(S, reinterpret_cast<uint32_t *>(smem + L.off_planes), &misc[1], BW, BH, L.pw, L.nbmax);
      }
      vertical_pass<T, K>(S, vmin, vmax, TW, TH, BW, L.vw);
      __syncthreads();
      horizontal_flag_pass<T, K>(S, vmin, vmax, O, list, &misc[0], TW, TH, BW, L.vw, cur.W - x0, cur.H - y0);
      __syncthreads();
      const int F = static_cast<int>(misc[0]);
      if constexpr (ALGO == ALGO_NETWORK) {
        network_medians<T, K>(S, O, list, F, TW, BW);
      } else {
        const int NB = 32 - __clz(static_cast<int>(misc[1]));
        bitplane_medians<K>(reinterpret_cast<const uint32_t *>(smem + L.off_planes),
                            reinterpret_cast<uint16_t *>(O), reinterpret_cast<uint8_t *>(O), E == 2, list, F, TW,
                            BH, L.pw, NB, XOFF);
      }
    }

    if (tma_out) {
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) tma_store_2d(&cf->tout, O, x0, y0);
    } else {
      __syncthreads();
      plain_tile_store<T>(cf, O, x0, y0, TW, TH);
    }
    if (tid == 0) {
      bulk_commit();
      if (misc[0] != 0) {
        unsigned long long *ctr = cf->flagged;
        if (ctr != nullptr) atomicAdd(ctr, static_cast<unsigned long long>(misc[0]));
      }
    }
    fence_proxy_async_smem();  // generic writes to this stage precede the TMA that will refill it
    __syncthreads();
  }
  if (tid == 0) bulk_wait_all<0>();
}

template <typename T, int K>
inline const void *kernel_for(int algo) {
  switch (algo) {
    case ALGO_DENSE3:
      if constexpr (K == 3) return reinterpret_cast<const void *>(&fnr_kernel<T, 3, ALGO_DENSE3>);
      return nullptr;
    case ALGO_NETWORK:
      if constexpr (K <= 7) return reinterpret_cast<const void *>(&fnr_kernel<T, K, ALGO_NETWORK>);
      return nullptr;
    case ALGO_BITPLANE:
      return reinterpret_cast<const void *>(&fnr_kernel<T, K, ALGO_BITPLANE>);
    default:
      return nullptr;
  }
}

}  // namespace fnr
