// Device code of the FNR impulse filter (arXiv 1201.3972, Sec. 3.3-3.4).
//
// One persistent kernel per (pixel type, window k, selection strategy). A CTA
// walks a strided list of output tiles with one producer warp and eight
// consumer warps and no block-wide barrier in the loop:
//   * the producer resolves each tile, waits until every consumer released
//     the staging buffer, and stages the tile plus a k-1 pixel halo with one
//     2-D TMA load (or clamped plain loads when the frame is not 16-byte
//     aligned); two buffers (three for the dense strategies), so the next
//     tiles load while this one computes;
//   * each consumer warp owns a horizontal strip of tile_h/8 output rows: it
//     replicates the frame border into the zero-filled cells it reads,
//     computes g_min and g_max of every window (Eq. 3a/3b), flags the pixels
//     equal to one of them (Sec. 3.3, step 2), replaces flagged pixels by the
//     window median g_m (Sec. 3.4) and releases the buffer. The dense
//     strategies (k = 3, 5, 7) take every pixel's median with networks shared
//     by neighbouring windows and store straight from registers; the
//     compacted ones (network, bit planes) list the flagged pixels, select
//     their medians and write the strip with a TMA store (or plain stores).
// All arithmetic is integer min/max/compare, so results are bit-exact.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "fnr_networks.cuh"
#include "fnr_params.h"
#include "fnr_separable.cuh"

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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
// Frames are contiguous ranges of the launch's tile index space (tile_begin);
// a tile is (frame, tile in frame).
struct TileInfo {
  int valid, f, x0, y0, W, H, flags, counted;  // counted: the frame has a flagged-pixel counter
};

__device__ __forceinline__ const FrameDev *frame_ptr(const FnrParams &p, int f) {
  return p.table == nullptr ? &p.single : p.table + f;
}

// `dir` is the shared-memory copy of every frame's tile_begin when the launch
// has at most kDirMax frames (else the table is searched in global memory).
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
  const int tl = t - fd->tile_begin;
  const int tiles_x = fd->tiles_x;
  ti.valid = 1;
  ti.f = f;
  ti.x0 = (tl % tiles_x) * p.tile_w;
  ti.y0 = (tl / tiles_x) * p.tile_h;
  ti.W = fd->W;
  ti.H = fd->H;
  ti.flags = fd->flags;
  ti.counted = fd->flagged != nullptr;
  return ti;
}

template <typename T>
__device__ __forceinline__ T load_global(const unsigned char *base, long long pitch, int y, int x) {
  return __ldg(reinterpret_cast<const T *>(base + (long long)y * pitch) + x);
}

// In-frame index that frame coordinate i (frame size n) reads under a border
// reading, or -1 when it reads 0 (zero border). Mirror reflects about the
// edge pixel and repeats with period 2(n-1) for offsets wider than the frame.
__device__ __forceinline__ int border_src(int i, int n, int border) {
  if (i >= 0 && i < n) return i;
  if (border == kBorderZero) return -1;
  if (border == kBorderMirror) {
    if (n == 1) return 0;
    const int period = 2 * (n - 1);
    int j = i % period;
    j = j < 0 ? j + period : j;
    return j < n ? j : period - j;
  }
  return i < 0 ? 0 : n - 1;
}

// Plain staging by one warp for frames TMA cannot address: the border
// mapping gives the out-of-frame cells directly.
template <typename T>
__device__ void plain_tile_load(const FrameDev *f, int xs, int ys, T *S, int BW, int BH, int border, int lane) {
  const int H = f->H, W = f->W;
  for (int row = 0; row < BH; ++row) {
    const int gy = border_src(ys + row, H, border);
    for (int col = lane; col < BW; col += 32) {
      const int gx = border_src(xs + col, W, border);
      S[row * BW + col] = (gy < 0 || gx < 0) ? T(0) : load_global<T>(f->in, f->in_pitch, gy, gx);
    }
  }
}

// TMA fills out-of-frame cells with zero (already right for the zero
// border). For replicate and mirror a warp rewrites, in the stage rows
// [row0, row1) it is about to read, every out-of-frame cell that a window of
// an in-frame pixel reads (columns [cmin, cmax], frame rows and columns
// within R of the frame) with the in-frame pixel the border reading maps it
// to: first the in-frame columns of out-of-frame rows (copied from the mapped
// row), then the out-of-frame columns of every row (from the mapped column of
// the same row). Several warps may patch the same cell; every write stores
// that cell's final value, so the overlap is harmless.
template <typename T>
__device__ void fixup_rows_warp(T *S, int xs, int ys, int BW, int W, int H, int row0, int row1, int cmin, int cmax,
                                int R, int border, int lane) {
  const int lft = -xs, rgt = W - 1 - xs;     // stage columns of frame columns 0 and W-1
  const int c0 = lft > cmin ? lft : cmin;
  const int c1 = rgt < cmax ? rgt : cmax;
  for (int row = row0; row < row1; ++row) {
    const int gy = ys + row;
    if (gy >= 0 && gy < H) continue;
    if (gy < -R || gy > H - 1 + R) continue;  // no in-frame window reaches it
    const int src = border_src(gy, H, border) - ys;
    for (int c = c0 + lane; c <= c1; c += 32) S[row * BW + c] = S[src * BW + c];
  }
  __syncwarp();
  const int jlo = cmin > -R - xs ? cmin : -R - xs;          // columns with frame x >= -R
  const int jhi = cmax < W - 1 + R - xs ? cmax : W - 1 + R - xs;
  if (lft > jlo || rgt < jhi) {
    for (int row = row0 + lane; row < row1; row += 32) {
      T *Rw = S + row * BW;
      for (int j = jlo; j < lft; ++j) Rw[j] = Rw[border_src(xs + j, W, border) - xs];
      for (int j = rgt + 1; j <= jhi; ++j) Rw[j] = Rw[border_src(xs + j, W, border) - xs];
    }
  }
  __syncwarp();
  (void)BW;
}

// Plain store of output rows [r0, r0+rows) of the tile (frame-clipped).
template <typename T>
__device__ void plain_strip_store(const FrameDev *f, const T *O, int x0, int y0, int TW, int r0, int rows, int lane) {
  const int H = f->H, W = f->W;
  for (int row = r0; row < r0 + rows; ++row) {
    const int gy = y0 + row;
    if (gy >= H) break;
    T *dst = reinterpret_cast<T *>(f->out + (long long)gy * f->out_pitch);
    for (int col = lane; col < TW; col += 32) {
      const int gx = x0 + col;
      if (gx < W) dst[gx] = O[row * TW + col];
    }
  }
}

// ---------------------------------------------------------------------------
// DENSE3: k = 3, median for every pixel.
//
// A lane owns 8 consecutive outputs in 2 consecutive rows. Pixels are held as
// packed pairs (x, x+1) of 16-bit lanes. Each of the 4 input rows gives 6
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

// Integer multiply-add on the FMA pipe: a * b + c (mod 2^32).
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Operations of the selection networks on two pixels per 32-bit word.
// A full compare-exchange needs min and max of the same two words; the
// packed min/max both run on the integer ALU pipe, which bounds the median
// stage. For 16-bit halves max = a + b - min holds per half, and the 32-bit
// sum a + b - min is exact modulo 2^32 (the carries of the low half cancel),
// so part of the exchanges take their max as two multiply-adds on the
// otherwise idle FMA pipe (the flag tests take their lane-wise differences
// there too). `unit` is 1 and `neg` is 0xffffffff, read from
// the launch parameters so that the compiler keeps them as multiplies.
struct PackedOp {
  // of every kCxPeriod full exchanges, kCxAlu take the ALU max (measured best
  // split for the k=5/7 networks on GB300)
  static constexpr int kCxPeriod = 5, kCxAlu = 2;
  uint32_t unit, neg;
  __device__ __forceinline__ uint32_t mn(uint32_t a, uint32_t b) const { return vmin2(a, b); }
  __device__ __forceinline__ uint32_t mx(uint32_t a, uint32_t b) const { return vmax2(a, b); }
  // a - b per 16-bit lane, for lanes where a >= b (no borrow between lanes)
  __device__ __forceinline__ uint32_t sub(uint32_t a, uint32_t b) const { return imad(b, neg, a); }
  template <int J>
  __device__ __forceinline__ void cx(uint32_t &a, uint32_t &b) const {
    const uint32_t lo = vmin2(a, b);
    if (J % kCxPeriod < kCxAlu)
      b = vmax2(a, b);
    else
      b = imad(lo, neg, imad(a, unit, b));
    a = lo;
  }
  // max(a, b) of an exchange whose min `lo` is computed anyway
  template <int J>
  __device__ __forceinline__ uint32_t cmax(uint32_t a, uint32_t b, uint32_t lo) const {
    if (J % kCxPeriod < kCxAlu) return vmax2(a, b);
    return imad(lo, neg, imad(a, unit, b));
  }
};

// The separable networks of the dense 5x5 / 7x7 strategy issue little but
// min/max, so the ALU pipe bounds them: of every kPeriod exchanges, kAlu take
// the ALU max and the others the FMA-pipe form. Measured on GB300 (640x512
// sweep, 128 frames per class): k = 5 with 1 of 8 on the ALU 0.0968 ms
// against 0.1029 with 2 of 5 (eight consumer warps per SM at two CTAs); k = 7
// (sliding items, one CTA per SM) 0.1685 ms with 1 of 3 against 0.1704 with
// 2 of 5, 0.1688 with 3 of 10, 0.1706 with 2 of 7, 0.1746 with 1 of 5 and
// 0.1725 with 1 of 2.
template <int K>
struct DenseOp : PackedOp {
  static constexpr int kPeriod = K == 5 ? 8 : 3, kAlu = K == 5 ? 1 : 1;
  template <int J>
  __device__ __forceinline__ uint32_t cmax(uint32_t a, uint32_t b, uint32_t lo) const {
    if (J % kPeriod < kAlu) return vmax2(a, b);
    return imad(lo, neg, imad(a, unit, b));
  }
};

__device__ __forceinline__ uint32_t med3v(uint32_t a, uint32_t b, uint32_t c) {
  return vmax2(vmin2(a, b), vmin2(vmax2(a, b), c));
}

// (hi lane of a, lo lane of b): the odd-aligned pair between two even pairs.
__device__ __forceinline__ uint32_t odd_pair(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5432); }

// The directional detector (Fig. 1) on the two pixels of word j + 1 of row b,
// where a, b, c are three consecutive rows of pixel pairs as load_row8 gives
// them (word q: the pixels 2q - 2 and 2q - 1 from the first centre column).
// Per 16-bit lane: 1 where the pixel lies strictly between its two
// neighbours along at least one of the four lines through it (a signal
// pixel: its gray level varies monotonically there, Sec. 3), 0 where along
// none (noisy).
__device__ __forceinline__ uint32_t strictly_between(uint32_t g, uint32_t u, uint32_t v, const PackedOp op) {
  const uint32_t lo = vmin2(u, v), hi = vmax2(u, v);
  // max(g, lo) - lo is nonzero iff g > lo, hi - min(g, hi) iff g < hi; both
  // differences are lane-wise non-negative, so no borrow crosses lanes
  return vmin2(vmin2(op.sub(vmax2(g, lo), lo), op.sub(hi, vmin2(g, hi))), 0x00010001u);
}

__device__ __forceinline__ uint32_t directional_sig(const uint32_t (&a)[6], const uint32_t (&b)[6],
                                                    const uint32_t (&c)[6], int j, const PackedOp op) {
  const uint32_t g = b[j + 1];
  uint32_t sig = strictly_between(g, odd_pair(b[j], b[j + 1]), odd_pair(b[j + 1], b[j + 2]), op);  // west, east
  sig |= strictly_between(g, a[j + 1], c[j + 1], op);                                            // north, south
  sig |= strictly_between(g, odd_pair(a[j], a[j + 1]), odd_pair(c[j + 1], c[j + 2]), op);        // north-west, south-east
  sig |= strictly_between(g, odd_pair(a[j + 1], a[j + 2]), odd_pair(c[j], c[j + 1]), op);        // north-east, south-west
  return sig;
}

// Output rows [r0, r0+SR) of the tile, written straight to the frame: 16-byte
// (u16) or 8-byte (u8) stores when the 8 pixels are inside the frame and the
// frame is 16-byte aligned, else per-pixel stores clipped to the frame.
// tw_valid, th_valid: the part of the tile inside the frame. tile_w / 8 is a
// power of two (seg_shift = log2 of it).
template <typename T, bool COUNT, int MODE>
__device__ void dense3_strip(const T *S, const FrameDev *f, int x0, int y0, int TW, int BW, int r0, int SR,
                             int seg_shift, int tw_valid, int th_valid, bool vec_ok, int lane, int &flagged,
                             const PackedOp op) {
  constexpr int XOFF = xoff_for(1, sizeof(T));
  const int items = (SR >> 1) << seg_shift;
  const int seg_mask = (1 << seg_shift) - 1;
  unsigned char *const out = f->out;
  const long long pitch = f->out_pitch;
  for (int it = lane; it < items; it += 32) {
    const int sx = it & seg_mask, ry = it >> seg_shift;
    const int tx = sx << 3, ty = r0 + (ry << 1);
    uint32_t e[4][6];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) load_row8<T>(S + (ty + rr) * BW + XOFF + tx, e[rr]);
    // directional detector: the flags of both output rows first, as bit
    // 4 o + pp of each 16-bit lane, so that the rows need not stay live
    uint32_t dsig = 0;
    if constexpr (MODE == kModeDirectional) {
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int pp = 0; pp < 4; ++pp) dsig |= directional_sig(e[o], e[o + 1], e[o + 2], pp, op) << (4 * o + pp);
    }
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
        // per 16-bit lane: 1 where g_min < c < g_max (signal pixel), 0 where c
        // equals g_min or g_max (noisy); c - g_min and g_max - c never borrow
        // across lanes since g_min <= c <= g_max. The standard median filter
        // treats every pixel as noisy; the directional detector tests lines.
        uint32_t sig;
        if constexpr (MODE == kModeMedian)
          sig = 0u;
        else if constexpr (MODE == kModeDirectional)
          sig = (dsig >> (4 * o + pp)) & 0x00010001u;
        else
          sig = vmin2(vmin2(op.sub(c, gmin), op.sub(gmax, c)), 0x00010001u);
        const uint32_t keep = sig * 0xffffu;
        res[pp] = (c & keep) | (gm & ~keep);
        if constexpr (COUNT && MODE != kModeDirectional) {
          const int col = tx + 2 * pp;
          const uint32_t valid =
              (ty + o < th_valid) ? ((col < tw_valid ? 1u : 0u) | (col + 1 < tw_valid ? 0x10000u : 0u)) : 0u;
          flagged += __popc((sig ^ 0x00010001u) & valid);
        }
      }
      if (ty + o < th_valid) {
        T *dst = reinterpret_cast<T *>(out + (long long)(y0 + ty + o) * pitch) + x0 + tx;
        if (vec_ok && tx + 8 <= tw_valid) {
          store_row8<T>(dst, res);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (tx + q < tw_valid) dst[q] = static_cast<T>((res[q >> 1] >> (16 * (q & 1))) & 0xffffu);
        }
      }
    }
    if constexpr (COUNT && MODE == kModeDirectional) {
      // in-frame pixels, in the bit order of dsig
      const int nlo = min(max((tw_valid - tx + 1) >> 1, 0), 4), nhi = min(max((tw_valid - tx) >> 1, 0), 4);
      const uint32_t row = ((1u << nlo) - 1u) | (((1u << nhi) - 1u) << 16);
      const uint32_t valid = (ty < th_valid ? row : 0u) | (ty + 1 < th_valid ? row << 4 : 0u);
      flagged += __popc(~dsig & valid);
    }
  }
}

// ---------------------------------------------------------------------------
// DENSE (k = 5, 7): the median of every pixel from the separable networks of
// fnr_separable.cuh (columns sorted once for two output rows, sorted columns
// merged into blocks that neighbouring windows share), kept where the
// detector flags the pixel.
//
// A lane item is a pair of output rows times eight output columns. The
// item's k+1 stage rows are loaded as x-packed words (two neighbouring
// pixels per word, columns x0 + kFirstCol ..); the network hands back, per
// output column, row-packed words (low half row y, high half row y+1) of
// g_m, g_min and g_max; the flag test and the blend run on those, and byte
// permutes turn the results back into rows for 16-byte (u16) or 8-byte (u8)
// stores straight to the frame (no output tile).
// ---------------------------------------------------------------------------
// x-packed word `WORD` (columns x0 + kFirstCol + 2 WORD and the next) of the
// item's stage row `ROW`, read where the network first needs it.
template <typename T, int K>
struct DenseLoad {
  const T *base;  // stage row of the item's first row, column x0 + kFirstCol
  int BW;
  template <int ROW, int WORD>
  __device__ __forceinline__ uint32_t get() const {
    if constexpr (sizeof(T) == 2) {
      return *reinterpret_cast<const uint32_t *>(base + ROW * BW + 2 * WORD);
    } else {
      const uint32_t h = *reinterpret_cast<const uint16_t *>(base + ROW * BW + 2 * WORD);
      return __byte_perm(h, 0, 0x4140);  // two bytes into two 16-bit halves
    }
  }
  // words WORD and WORD + 1 by one read: the sliding network asks for pairs
  // that start on an 8-byte (u16) or 4-byte (u8) boundary of the stage
  template <int ROW, int WORD>
  __device__ __forceinline__ void get2(uint32_t &a, uint32_t &b) const {
    if constexpr (sizeof(T) == 2) {
      const uint2 t = *reinterpret_cast<const uint2 *>(base + ROW * BW + 2 * WORD);
      a = t.x;
      b = t.y;
    } else {
      const uint32_t t = *reinterpret_cast<const uint32_t *>(base + ROW * BW + 2 * WORD);
      a = __byte_perm(t, 0, 0x4140);
      b = __byte_perm(t, 0, 0x4342);
    }
  }
};

template <typename T, int K, bool COUNT, int MODE>
struct DenseEmit {
  using Net = SepNet<K>;
  static constexpr int R = (K - 1) / 2;
  const T *centre;                // stage row of output row y, column x0
  int BW;
  const uint32_t (&dsig)[2][Net::kOut / 2];  // directional detector: x-packed signal bits of rows y, y+1
  uint32_t (&res)[Net::kOut];
  const PackedOp op;
  const int tx, ty, tw_valid, th_valid;
  int &flagged;
  template <int J>
  __device__ __forceinline__ void put(uint32_t gm, uint32_t gmin, uint32_t gmax) {
    // the centre pixels of output column x0 + J in rows y and y + 1 (row-packed)
    uint32_t c;
    if constexpr (sizeof(T) == 2) {
      const uint32_t a = *reinterpret_cast<const uint32_t *>(centre + (J & ~1));
      const uint32_t b = *reinterpret_cast<const uint32_t *>(centre + BW + (J & ~1));
      c = (J & 1) ? __byte_perm(a, b, 0x7632) : __byte_perm(a, b, 0x5410);
    } else {
      c = __byte_perm(static_cast<uint32_t>(centre[J]), static_cast<uint32_t>(centre[BW + J]), 0x5410);
    }
    finish<J>(gm, gmin, gmax, c);
  }
  // the same, with the centre pixels taken from the network's input words a
  // (row y) and b (row y + 1), x-packed with 16-bit lanes for both pixel types
  template <int J>
  __device__ __forceinline__ void put(uint32_t gm, uint32_t gmin, uint32_t gmax, uint32_t a, uint32_t b) {
    finish<J>(gm, gmin, gmax, (J & 1) ? __byte_perm(a, b, 0x7632) : __byte_perm(a, b, 0x5410));
  }
  template <int J>
  __device__ __forceinline__ void finish(uint32_t gm, uint32_t gmin, uint32_t gmax, uint32_t c) {
    // per 16-bit lane: 1 where the pixel is a signal pixel, 0 where noisy
    uint32_t sig;
    if constexpr (MODE == kModeMedian)
      sig = 0u;
    else if constexpr (MODE == kModeDirectional)
      sig = (J & 1) ? __byte_perm(dsig[0][J >> 1], dsig[1][J >> 1], 0x7632)
                    : __byte_perm(dsig[0][J >> 1], dsig[1][J >> 1], 0x5410);
    else
      sig = vmin2(vmin2(op.sub(c, gmin), op.sub(gmax, c)), 0x00010001u);  // g_min <= c <= g_max lane-wise
    const uint32_t keep = sig * 0xffffu;
    res[J] = (c & keep) | (gm & ~keep);
    if constexpr (COUNT) {
      const uint32_t valid =
          tx + J < tw_valid ? ((ty < th_valid ? 1u : 0u) | (ty + 1 < th_valid ? 0x10000u : 0u)) : 0u;
      flagged += __popc((sig ^ 0x00010001u) & valid);
    }
  }
};

// The item's results, turned back into rows (byte permutes) and stored
// straight to the frame: 16-byte (u16) or 8-byte (u8) stores where the whole
// eight columns are in the frame and the frame allows vector stores.
template <typename T, int NO>
__device__ __forceinline__ void dense_store_item(unsigned char *out, long long pitch, int x0, int y0, int tx, int ty,
                                                 const uint32_t (&res)[NO], int tw_valid, int th_valid, bool vec_ok) {
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    if (ty + o < th_valid) {
#pragma unroll
      for (int g = 0; g < NO / 8; ++g) {
        uint32_t rw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          rw[q] = __byte_perm(res[8 * g + 2 * q], res[8 * g + 2 * q + 1], o ? 0x7632 : 0x5410);
        const int cx = tx + 8 * g;
        T *dst = reinterpret_cast<T *>(out + (long long)(y0 + ty + o) * pitch) + x0 + cx;
        if (vec_ok && cx + 8 <= tw_valid) {
          store_row8<T>(dst, rw);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (cx + q < tw_valid) dst[q] = static_cast<T>((rw[q >> 1] >> (16 * (q & 1))) & 0xffffu);
        }
      }
    }
  }
}

// The directional detector's signal bits of an item's two rows (stage rows
// ty + R and ty + R + 1), eight columns at a time.
template <typename T, int K, int NO>
__device__ __forceinline__ void dense_item_dsig(const T *item, int BW, uint32_t (&dsig)[2][NO / 2],
                                                const PackedOp op) {
  constexpr int R = (K - 1) / 2;
#pragma unroll
  for (int g = 0; g < NO / 8; ++g) {
    uint32_t e[4][6];
#pragma unroll
    for (int q = 0; q < 4; ++q) load_row8<T>(item + (R - 1 + q) * BW + 8 * g, e[q]);
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int pp = 0; pp < 4; ++pp) dsig[o][4 * g + pp] = directional_sig(e[o], e[o + 1], e[o + 2], pp, op);
  }
}

template <typename T, int K, bool COUNT, int MODE>
__device__ void dense_sep_strip(const T *S, const FrameDev *f, int x0, int y0, int BW, int r0, int SR, int seg_shift,
                                int tw_valid, int th_valid, bool vec_ok, int lane, int &flagged, const PackedOp op) {
  using Net = SepNet<K>;
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  constexpr int NO = Net::kOut;  // output columns per item (a multiple of 8)
  static_assert(Net::kRows == K + 1 && NO % 8 == 0 && NO == dense_item_cols(ALGO_DENSE, K), "network shape");
  static_assert(Net::kSliding == dense_sliding(K), "network form");
  unsigned char *const out = f->out;
  const long long pitch = f->out_pitch;
  if constexpr (Net::kSliding) {
    // A lane takes a span of 2^span_shift neighbouring items of one row
    // pair, as many as spread the strip's items over the 32 lanes: the
    // span's first item starts from its carry (Net::pre), and every item
    // hands its carry (sorted columns and merged blocks that the next item's
    // windows share) on. Neighbouring lanes take neighbouring row pairs of
    // the same span column: the stage row pitch is an odd number of 16-byte
    // units, so their reads spread over the banks (lanes of one row pair
    // would be a span apart, in a few banks).
    const int pairs = SR >> 1;
    const int span_shift = min(seg_shift, max(0, seg_shift + (31 - __clz(pairs)) - 5));
    const int units = pairs << (seg_shift - span_shift);
    for (int u = lane; u < units; u += 32) {
      const int ry = u % pairs, sp = u / pairs;
      const int ty = r0 + (ry << 1);
      const T *const row = S + ty * BW + XOFF;  // stage row ty, output column x0
      int tx = sp * (NO << span_shift);
      uint32_t carry[Net::kCarry];
      Net::pre(DenseOp<K>{op}, DenseLoad<T, K>{row + tx + Net::kFirstCol, BW}, carry);
#pragma unroll 1
      for (int s = 0; s < (1 << span_shift); ++s, tx += NO) {
        const T *const item = row + tx;
        uint32_t dsig[2][NO / 2] = {};
        if constexpr (MODE == kModeDirectional) dense_item_dsig<T, K, NO>(item, BW, dsig, op);
        uint32_t res[NO];
        Net::body(DenseOp<K>{op}, DenseLoad<T, K>{item + Net::kFirstCol, BW},
                  DenseEmit<T, K, COUNT, MODE>{item + R * BW, BW, dsig, res, op, tx, ty, tw_valid, th_valid, flagged},
                  carry);
        dense_store_item<T, NO>(out, pitch, x0, y0, tx, ty, res, tw_valid, th_valid, vec_ok);
      }
    }
  } else {
    // items: (row pair, NO-column segment), one at a time; seg_shift = log2(tile_w / NO)
    const int items = (SR >> 1) << seg_shift;
    const int seg_mask = (1 << seg_shift) - 1;
    for (int it = lane; it < items; it += 32) {
      const int sx = it & seg_mask, ry = it >> seg_shift;
      const int tx = sx * NO, ty = r0 + (ry << 1);
      const T *const item = S + ty * BW + XOFF + tx;  // stage row ty, output column x0
      uint32_t dsig[2][NO / 2] = {};
      if constexpr (MODE == kModeDirectional) dense_item_dsig<T, K, NO>(item, BW, dsig, op);
      uint32_t res[NO];
      Net::run(DenseOp<K>{op}, DenseLoad<T, K>{item + Net::kFirstCol, BW},
               DenseEmit<T, K, COUNT, MODE>{item + R * BW, BW, dsig, res, op, tx, ty, tw_valid, th_valid, flagged});
      dense_store_item<T, NO>(out, pitch, x0, y0, tx, ty, res, tw_valid, th_valid, vec_ok);
    }
  }
}

#ifndef FNR_SPARSE_LIMIT
#define FNR_SPARSE_LIMIT 16
#endif

// ---------------------------------------------------------------------------
// Compacted strategies (any k): separable g_min/g_max over the warp's strip,
// flag, warp-local list of flagged pixels, then one median per flagged pixel.
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

// Fast exact division by a runtime divisor d >= 1 for dividends below 2^16:
// q = umulhi(n, ceil(2^32 / d)); d = 1 (whose multiplier 2^32 does not fit in
// 32 bits) returns n itself.
struct FastDiv {
  uint32_t m;
  bool one;
  __device__ explicit FastDiv(uint32_t d)
      : m(d > 1 ? static_cast<uint32_t>((0xffffffffull + d) / d) : 0u), one(d <= 1) {}
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return one ? n : __umulhi(n, m); }
};

// Pair word of stage row `row` at even stage column `col`: pixels (col, col+1)
// in the low and high 16-bit lanes.
template <typename T>
__device__ __forceinline__ uint32_t pair_word(const T *S, int row, int BW, int col);

template <>
__device__ __forceinline__ uint32_t pair_word<uint16_t>(const uint16_t *S, int row, int BW, int col) {
  return *reinterpret_cast<const uint32_t *>(S + row * BW + col);
}

template <>
__device__ __forceinline__ uint32_t pair_word<uint8_t>(const uint8_t *S, int row, int BW, int col) {
  return __byte_perm(static_cast<uint32_t>(*reinterpret_cast<const uint16_t *>(S + row * BW + col)), 0, 0x4140);
}

// Sliding packed extreme (min.u16x2 / max.u16x2) over windows [q, q+K-1] of
// RG+K-1 words, sharing the core [RG-1, K-1] common to all windows (RG <= K).
template <int K, int RG, bool MAX>
__device__ __forceinline__ void sliding_extreme2(const uint32_t (&v)[RG + K - 1], uint32_t (&out)[RG]) {
  auto op = [](uint32_t a, uint32_t b) { return MAX ? vmax2(a, b) : vmin2(a, b); };
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

// Vertical pass over the strip on column pairs: vminP/vmaxP[q * NPS + p] =
// packed min/max of stage columns (cb + 2p, cb + 2p + 1) over stage rows
// r0+q .. r0+q+K-1, q < SR, p < NP.
template <typename T, int K>
__device__ void vertical_pairs(const T *S, uint32_t *vminP, uint32_t *vmaxP, int BW, int NP, int NPS, int cb, int r0,
                               int SR, const FastDiv &divNP, int lane) {
  constexpr int RG = row_group(K);
  const int items = NP * (SR / RG);
  for (int it = lane; it < items; it += 32) {
    const int g = static_cast<int>(divNP.div(static_cast<uint32_t>(it))), p = it - g * NP;
    const int col = cb + 2 * p, row0 = r0 + g * RG;
    uint32_t v[RG + K - 1];
#pragma unroll
    for (int i = 0; i < RG + K - 1; ++i) v[i] = pair_word<T>(S, row0 + i, BW, col);
    uint32_t mn[RG], mx[RG];
    sliding_extreme2<K, RG, false>(v, mn);
    sliding_extreme2<K, RG, true>(v, mx);
#pragma unroll
    for (int q = 0; q < RG; ++q) {
      vminP[(g * RG + q) * NPS + p] = mn[q];
      vmaxP[(g * RG + q) * NPS + p] = mx[q];
    }
  }
}

// Horizontal pass + flag over the strip, PPI = 4 output pairs (8 pixels) per
// lane item: every centre value goes to the output tile; flagged in-frame
// pixels (all in-frame pixels when `all`) are appended to the warp's list as
// (row in strip << 8 | column). The window of output column x spans stage
// columns XOFF+x-R .. XOFF+x+R; for a pair (x, x+1) the packed window term at
// offset d is the pair word at stage column XOFF+x+d, which is a byte permute
// of two stored words when that column is odd relative to cb (compile time).
// The item's extreme words, centre pixels and output pixels are each moved
// as 16-byte (8-byte for u8 pixels) vectors. Returns the list length
// (warp-uniform).
template <typename T>
__device__ __forceinline__ void load_centre8(const T *p, uint32_t (&c)[4]);

template <>
__device__ __forceinline__ void load_centre8<uint16_t>(const uint16_t *p, uint32_t (&c)[4]) {
  const uint4 v = *reinterpret_cast<const uint4 *>(p);
  c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
}

template <>
__device__ __forceinline__ void load_centre8<uint8_t>(const uint8_t *p, uint32_t (&c)[4]) {
  const uint2 v = *reinterpret_cast<const uint2 *>(p);
  c[0] = __byte_perm(v.x, 0, 0x4140);
  c[1] = __byte_perm(v.x, 0, 0x4342);
  c[2] = __byte_perm(v.y, 0, 0x4140);
  c[3] = __byte_perm(v.y, 0, 0x4342);
}

template <typename T>
__device__ __forceinline__ void store_centre8(T *p, const uint32_t (&c)[4]);

template <>
__device__ __forceinline__ void store_centre8<uint16_t>(uint16_t *p, const uint32_t (&c)[4]) {
  *reinterpret_cast<uint4 *>(p) = make_uint4(c[0], c[1], c[2], c[3]);
}

template <>
__device__ __forceinline__ void store_centre8<uint8_t>(uint8_t *p, const uint32_t (&c)[4]) {
  *reinterpret_cast<uint2 *>(p) = make_uint2(__byte_perm(c[0], c[1], 0x6420), __byte_perm(c[2], c[3], 0x6420));
}

template <typename T, int K>
__device__ int horizontal_pairs(const T *S, const uint32_t *vminP, const uint32_t *vmaxP, T *O, uint16_t *list, int TW,
                                int BW, int NPS, int r0, int SR, int tw_valid, int th_valid, int mode,
                                const FastDiv &divG, const PackedOp op, int lane) {
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  constexpr int CB = (XOFF - R) & ~1;
  constexpr int OFF0 = XOFF - CB;          // stage column XOFF relative to CB (R or R + 1)
  constexpr int PPI = 4;                   // output pairs per item
  constexpr int NW = ((OFF0 + 2 * PPI - 1 + R) >> 1) + 1;  // words an item reads, from word x0p / 2
  constexpr int NV = (NW + 3) / 4;         // 16-byte vectors covering them
  static_assert(OFF0 - R == 0 || OFF0 - R == 1, "first word of an item is x0p / 2");
  const int gpr = TW / (2 * PPI);          // items per row
  const int items = SR * gpr;
  int base = 0;
  for (int it0 = 0; it0 < items; it0 += 32) {
    const int it = it0 + lane;
    uint32_t fm = 0;                       // bit j: pixel 2j flagged; bit 4 + j: pixel 2j + 1
    int q = 0, x0p = 0;
    if (it < items) {
      q = static_cast<int>(divG.div(static_cast<uint32_t>(it)));
      const int grp = it - q * gpr;
      x0p = grp * 2 * PPI;                 // first output column of the item (tile coordinates)
      const int ty = r0 + q;
      uint32_t c[PPI];
      load_centre8<T>(S + (ty + R) * BW + XOFF + x0p, c);
      store_centre8<T>(O + ty * TW + x0p, c);
      uint32_t sig = 0;                    // per 16-bit lane, bit j: pair j is a signal pixel
      if (mode == kModeDirectional) {
        // the rows above, through and below the centres
        uint32_t ra[6], rb[6], rc[6];
        const T *sp = S + (ty + R - 1) * BW + XOFF + x0p;
        load_row8<T>(sp, ra);
        load_row8<T>(sp + BW, rb);
        load_row8<T>(sp + 2 * BW, rc);
#pragma unroll
        for (int j = 0; j < PPI; ++j) sig = imad(directional_sig(ra, rb, rc, j, op), op.unit << j, sig);
      } else {
        uint32_t mnw[4 * NV], mxw[4 * NV];
        const uint4 *vn = reinterpret_cast<const uint4 *>(vminP + q * NPS + (x0p >> 1));
        const uint4 *vx = reinterpret_cast<const uint4 *>(vmaxP + q * NPS + (x0p >> 1));
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const uint4 a = vn[i], b = vx[i];
          mnw[4 * i] = a.x; mnw[4 * i + 1] = a.y; mnw[4 * i + 2] = a.z; mnw[4 * i + 3] = a.w;
          mxw[4 * i] = b.x; mxw[4 * i + 1] = b.y; mxw[4 * i + 2] = b.z; mxw[4 * i + 3] = b.w;
        }
#pragma unroll
        for (int j = 0; j < PPI; ++j) {
          uint32_t gmin = 0xffffffffu, gmax = 0u;
#pragma unroll
          for (int d = -R; d <= R; ++d) {
            const int col = OFF0 + 2 * j + d;  // relative to x0p, plus OFF0 (compile time)
            const int w = col >> 1;
            uint32_t a, b;
            if (col & 1) {
              a = __byte_perm(mnw[w], mnw[w + 1], 0x5432);
              b = __byte_perm(mxw[w], mxw[w + 1], 0x5432);
            } else {
              a = mnw[w];
              b = mxw[w];
            }
            gmin = d == -R ? a : vmin2(gmin, a);
            gmax = d == -R ? b : vmax2(gmax, b);
          }
          // 1 per 16-bit lane where g_min < c < g_max, 0 where c is an extreme
          // (no borrow between lanes: g_min <= c <= g_max lane-wise)
          const uint32_t z = vmin2(vmin2(op.sub(c[j], gmin), op.sub(gmax, c[j])), 0x00010001u);
          sig = imad(z, op.unit << j, sig);
        }
      }
      // in-frame pixels of the item, in the bit order of fm
      const int n = ty < th_valid ? min(max(tw_valid - x0p, 0), 2 * PPI) : 0;
      const uint32_t valid = ((1u << ((n + 1) >> 1)) - 1u) | (((1u << (n >> 1)) - 1u) << 4);
      const uint32_t noisy = ~sig & 0x000f000fu;
      fm = (mode == kModeMedian ? 0xffu : ((noisy & 0xfu) | (noisy >> 12))) & valid;
    }
    const int cnt = __popc(fm);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int pos = base + incl - cnt;
    while (fm) {
      const int bit = __ffs(fm) - 1;
      fm &= fm - 1;
      list[pos++] = static_cast<uint16_t>((q << 8) | (x0p + ((bit & 3) << 1) + (bit >> 2)));
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncwarp();
  return base;
}

// The medians of two flagged pixels, at stage-window rows ya / yb (tile row
// of the output pixel; the window spans stage rows ya .. ya + K - 1) and tile
// columns xa / xb, gathered into the low and high 16-bit lanes of the same
// registers so that one packed selection network serves both; the results go
// to the output tile.
//
// 16-bit pixels are gathered as 32-bit words: a window row of K = 2R+1
// pixels always lies in R+1 aligned words, whose 2R+2 halves hold the row
// plus one unused half, the first (pixel at an odd element) or the last (at
// an even one). The halves 1..2R are pixels of the row whatever the parity,
// so they pair up between the two pixels with fixed selectors; the one
// remaining pixel of each row (half 0 or half 2R+1) is picked with a
// per-pixel selector. The network does not care in which order a window's
// values arrive, only that each register holds one value of each pixel.
template <typename T, int K>
__device__ __forceinline__ void median_pair(const T *S, T *O, int TW, int BW, int ya, int xa, int yb, int xb,
                                            PackedOp op) {
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  // only the two output offsets stay live across the network
  const int oa = ya * TW + xa, ob = yb * TW + xb;
  uint32_t v[K * K];
  if constexpr (sizeof(T) == 2) {
    const uint32_t *W32 = reinterpret_cast<const uint32_t *>(S);
    const int BWW = BW >> 1;  // BW is even: rows start on a word
    const int sa = ya * BW + (XOFF - R) + xa, sb = yb * BW + (XOFF - R) + xb;
    const uint32_t *wa = W32 + (sa >> 1), *wb = W32 + (sb >> 1);
    // leftover pixel: low half of word 0 (even start) or high half of word R (odd start)
    const uint32_t sel_a = (sa & 1) ? 0x0076u : 0x0010u;
    const uint32_t sel_b = (sb & 1) ? 0x7600u : 0x1000u;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      uint32_t ua[R + 1], ub[R + 1];
#pragma unroll
      for (int t = 0; t <= R; ++t) {
        ua[t] = wa[a * BWW + t];
        ub[t] = wb[a * BWW + t];
      }
#pragma unroll
      for (int h = 1; h <= 2 * R; ++h)
        v[a * K + h - 1] = __byte_perm(ua[h >> 1], ub[h >> 1], (h & 1) ? 0x7632u : 0x5410u);
      v[a * K + 2 * R] = __byte_perm(__byte_perm(ua[0], ua[R], sel_a), __byte_perm(ub[0], ub[R], sel_b), 0x7610u);
    }
  } else {
    // 8-bit pixels: a window row lies in NWL aligned words; a funnel shift by
    // the pixel's byte offset realigns them so that window pixel j is byte j,
    // and one byte permute then puts 257 * a_j and 257 * b_j into the two
    // 16-bit lanes (v -> 257 v keeps the order, and the low byte of the
    // selected lane is the 8-bit median)
    constexpr int NWL = (K + 2) / 4 + 1;  // words covering byte offset (0..3) + K pixels
    constexpr int NWA = (K + 3) / 4;      // realigned words holding the K pixels
    const uint32_t *W32 = reinterpret_cast<const uint32_t *>(S);
    const int BWW = BW >> 2;  // BW is a multiple of 16: rows start on a word
    const int sa = ya * BW + (XOFF - R) + xa, sb = yb * BW + (XOFF - R) + xb;
    const uint32_t *wa = W32 + (sa >> 2), *wb = W32 + (sb >> 2);
    const uint32_t sha = static_cast<uint32_t>(sa & 3) * 8u, shb = static_cast<uint32_t>(sb & 3) * 8u;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      uint32_t la[NWL + 1], lb[NWL + 1];
#pragma unroll
      for (int t = 0; t < NWL; ++t) {
        la[t] = wa[a * BWW + t];
        lb[t] = wb[a * BWW + t];
      }
      la[NWL] = lb[NWL] = 0u;
      uint32_t ua[NWA], ub[NWA];
#pragma unroll
      for (int t = 0; t < NWA; ++t) {
        ua[t] = __funnelshift_r(la[t], la[t + 1], sha);
        ub[t] = __funnelshift_r(lb[t], lb[t + 1], shb);
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const uint32_t q = static_cast<uint32_t>(j & 3);
        v[a * K + j] = __byte_perm(ua[j >> 2], ub[j >> 2], q | (q << 4) | ((4u + q) << 8) | ((4u + q) << 12));
      }
    }
  }
  const uint32_t m = MedianNet<K>::run(v, op);
  O[oa] = static_cast<T>(m & 0xffffu);
  O[ob] = static_cast<T>(m >> 16);
}

// The flagged pixels of the warp's strip, two per lane.
template <typename T, int K>
__device__ void network_strip(const T *S, T *O, const uint16_t *list, int F, int TW, int BW, int r0, int lane,
                              PackedOp op) {
  const int pairs = (F + 1) >> 1;
  for (int i = lane; i < pairs; i += 32) {
    const int ea = list[2 * i];
    const int eb = 2 * i + 1 < F ? list[2 * i + 1] : ea;
    median_pair<T, K>(S, O, TW, BW, r0 + (ea >> 8), ea & 255, r0 + (eb >> 8), eb & 255, op);
  }
}

// Whether the network strategy pools the flagged pixels of a tile across its
// strips (network_pooled). Pooling saves the partial round each strip would
// run on its own but synchronises the tile's warps twice; measured on GB300
// it pays for the 81-input network of k = 9 (67 against 80 us per eight
// 1280x1024 frames with 3.5% flagged pixels), is even for k = 7 and loses
// for k = 5 (273 against 297 Gpx/s), where a round is cheap.
template <int K>
struct PoolMedians {
  static constexpr bool value = pool_medians(ALGO_NETWORK, K);
};

// The flagged pixels of the whole tile, pooled: the warps' lists, in warp
// order, form one sequence; pair p takes its entries 2p and 2p + 1 (an odd
// last entry pairs with itself) and round r of 32 pairs goes to warp
// r mod 8. A strip alone would run a partial round of its own; pooled, the
// tile runs ceil(pairs / 32) rounds in all. counts[w] is the length of warp
// w's list, total their sum; list entries are (row in strip << 8 | column).
template <typename T, int K>
__device__ void network_pooled(const T *S, T *O, const unsigned char *warp_blocks, int warp_bytes, int w_list,
                               const int *counts, int total, int TW, int BW, int SR, int warp, int lane,
                               PackedOp op) {
  const int pairs = (total + 1) >> 1;
  for (int pi = warp * 32 + lane; pi - lane < pairs; pi += 32 * kConsumerWarps) {
    if (pi >= pairs) continue;
    const int ga = 2 * pi, gb = 2 * pi + 1 < total ? 2 * pi + 1 : ga;
    // the list each entry lives in, from the counts in shared memory (kept
    // out of registers: they would be live across the network)
    int wa = 0, wb = 0, base_a = 0, base_b = 0, pre = 0;
#pragma unroll
    for (int j = 1; j < kConsumerWarps; ++j) {
      pre += counts[j - 1];
      if (ga >= pre) { wa = j; base_a = pre; }
      if (gb >= pre) { wb = j; base_b = pre; }
    }
    const int ea = reinterpret_cast<const uint16_t *>(warp_blocks + wa * warp_bytes + w_list)[ga - base_a];
    const int eb = reinterpret_cast<const uint16_t *>(warp_blocks + wb * warp_bytes + w_list)[gb - base_b];
    median_pair<T, K>(S, O, TW, BW, wa * SR + (ea >> 8), ea & 255, wb * SR + (eb >> 8), eb & 255, op);
  }
}

// Transpose of the 32x32 bit matrix whose row l is lane l's word: afterwards
// lane j holds the word whose bit l is bit j of lane l's word. Five rounds
// of one shuffle each swap the off-diagonal blocks of halving size (16, 8,
// 4, 2, 1) between lane pairs l, l ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  constexpr uint32_t kMask[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int s = 16 >> i;
    const uint32_t m = kMask[i];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
  }
  return x;
}

// Bit planes of the stage rows [r0, r0 + rows): word (bit b, row i, word w)
// at planes[(b * rows + i) * PW + w] holds bit b of the 32 pixels of row
// r0 + i from stage column c0 + 32w, where c0 is the first column a window of
// the tile reads (bits beyond the stage are zero). This order keeps the
// selection's reads, where each lane reads its own pixel's rows at one bit,
// in distinct banks. Lane l packs the pixels of its column of 32 / NB
// consecutive rows (2 of 16 bits, 4 of 8 bits) into one word; one warp
// transpose turns the 32 words into the 32 plane words of those rows (lane
// q * NB + b: bit b of the group's row q), each stored by its lane. Returns
// the OR of the pixels.
template <typename T>
__device__ uint32_t build_planes_warp(const T *S, uint32_t *planes, int BW, int c0, int r0, int rows, int PW,
                                      int lane) {
  constexpr int NB = 8 * sizeof(T);
  constexpr int P = 32 / NB;  // rows per transpose
  const int groups = (rows + P - 1) / P;
  const int b = lane & (NB - 1), q = lane / NB;  // the plane word this lane holds after a transpose
  uint32_t orv = 0;
  for (int it = 0; it < groups * PW; ++it) {
    const int g = it / PW, w = it - g * PW;
    const int col = c0 + (w << 5) + lane;
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const int row = g * P + j;
      const uint32_t px = (col < BW && row < rows) ? static_cast<uint32_t>(S[(r0 + row) * BW + col]) : 0u;
      x |= px << (NB * j);
    }
    orv |= x;
    x = warp_transpose32(x, lane);
    const int row = g * P + q;
    if (row < rows) planes[(b * rows + row) * PW + w] = x;
  }
  __syncwarp();
#pragma unroll
  for (int j = 1; j < P; ++j) orv |= orv >> (NB * j);
  return __reduce_or_sync(0xffffffffu, orv & ((1u << NB) - 1u));
}

// Flagged pixels of the strip: radix select on the window, most significant
// bit first. alive marks the window pixels whose bits above the current bit
// match the answer so far; each round counts the live pixels with a 0 bit.
// Plane rows are relative to the strip's first stage row. Windows up to 16
// wide keep two rows per register (segments of rows 2j and 2j+1 in the low
// and high halves), so one popcount serves both.
template <typename T, int K, bool kTwoWords>
__device__ __forceinline__ void bitplane_select(const uint32_t *planes, T *O, const uint16_t *list, int F, int TW,
                                                int rows, int PW, int NB, int r0, int lane) {
  constexpr uint32_t kMask = (1u << K) - 1u;
  constexpr bool kPack = K <= 16;
  constexpr int NA = kPack ? (K + 1) / 2 : K;  // alive words
  for (int i = lane; i < F; i += 32) {
    const int e = list[i];
    const int q = e >> 8, tx = e & 255;
    const int wi = kTwoWords ? 0 : tx >> 5, sh = tx & 31;
    uint32_t alive[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a)
      alive[a] = kPack ? (2 * a + 1 < K ? kMask | (kMask << 16) : kMask) : kMask;
    uint32_t rank = (K * K - 1) / 2, res = 0;
    for (int b = NB - 1; b >= 0; --b) {
      const uint32_t *P = planes + (b * rows + q) * PW + wi;
      // the window's bits of plane row r: bits sh .. sh + K - 1 of words wi, wi + 1
      auto row_bits = [&](int r) {
        if constexpr (kTwoWords) {  // a row is two words: one aligned 8-byte read
          const uint2 w = *reinterpret_cast<const uint2 *>(P + 2 * r);
          return __funnelshift_r(w.x, w.y, sh);
        } else {
          return __funnelshift_r(P[r * PW], P[r * PW + 1], sh);
        }
      };
      uint32_t seg[NA];
      uint32_t cnt = 0;
#pragma unroll
      for (int a = 0; a < NA; ++a) {
        if constexpr (kPack) {
          const int ra = 2 * a, rb = 2 * a + 1 < K ? 2 * a + 1 : 2 * a;
          seg[a] = __byte_perm(row_bits(ra), row_bits(rb), 0x5410);  // bits beyond K in each half meet no live bit
        } else {
          seg[a] = row_bits(a);
        }
        cnt += __popc(alive[a] & ~seg[a]);
      }
      // keep the 0-bit pixels when the rank falls among them, else the 1-bit ones
      const bool one = rank >= cnt;
      const uint32_t flip = one ? 0u : 0xffffffffu;
      rank -= one ? cnt : 0u;
      res |= (one ? 1u : 0u) << b;
#pragma unroll
      for (int a = 0; a < NA; ++a) alive[a] &= seg[a] ^ flip;
    }
    O[(r0 + q) * TW + tx] = static_cast<T>(res);
  }
}

// Flagged pixels of the strip (see bitplane_select). A tile of at most 32
// columns keeps two plane words per row (PW == 2, set by the layout only for
// such tiles), read as one aligned 8-byte word.
template <typename T, int K>
__device__ void bitplane_strip(const uint32_t *planes, T *O, const uint16_t *list, int F, int TW, int rows, int PW,
                               int NB, int r0, int lane) {
  if (PW == 2)
    bitplane_select<T, K, true>(planes, O, list, F, TW, rows, PW, NB, r0, lane);
  else
    bitplane_select<T, K, false>(planes, O, list, F, TW, rows, PW, NB, r0, lane);
}

// Sparse strips (few flagged pixels): building the strip's bit planes costs
// the same however few pixels need a median, so below a threshold the whole
// warp selects the medians of two flagged pixels at a time instead, packed in
// the two 16-bit halves of each register. Lane l holds the window cells
// l, l + 32, ... (n = K*K of them) of both pixels; a median is fixed MSB
// first: with the bits above b already those of the answer, the cells whose
// bits from b up equal that prefix followed by a 0 are counted over the warp
// (one reduction per bit for both pixels); the answer takes a 0 bit when the
// remaining rank falls among them, else a 1 bit and the rank drops by their
// count.
template <typename T, int K>
__device__ void radix_sparse_strip(const T *S, T *O, const uint16_t *list, int F, int TW, int BW, int r0, int lane) {
  constexpr int R = (K - 1) / 2;
  constexpr int N = K * K;
  constexpr int NV = (N + 31) / 32;
  constexpr int XOFF = xoff_for(R, sizeof(T));
  int off[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    const int i = lane + 32 * j;
    off[j] = i < N ? (i / K) * BW + (i % K) : 0;
  }
  const bool last_valid = lane + 32 * (NV - 1) < N;  // the other slots are always window cells
  for (int e = 0; e < F; e += 2) {
    const int ea = list[e];
    const int eb = e + 1 < F ? list[e + 1] : ea;
    const T *ba = S + (r0 + (ea >> 8)) * BW + (XOFF - R) + (ea & 255);
    const T *bb = S + (r0 + (eb >> 8)) * BW + (XOFF - R) + (eb & 255);
    uint32_t w[NV];
    uint32_t orv = 0;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      w[j] = static_cast<uint32_t>(ba[off[j]]) | (static_cast<uint32_t>(bb[off[j]]) << 16);
      if (j < NV - 1 || last_valid) orv |= w[j];
    }
    orv = __reduce_or_sync(0xffffffffu, orv);
    const int nb = 32 - __clz(static_cast<int>((orv | (orv >> 16)) & 0xffffu));
    uint32_t rank_a = (N - 1) / 2, rank_b = (N - 1) / 2, res = 0;  // res: answer of a (low) and b (high)
    for (int bit = nb - 1; bit >= 0; --bit) {
      const uint32_t keep = (0xffffu >> bit) * 0x00010001u;  // the bits from `bit` up, per half
      const uint32_t want = (res >> bit) & keep;             // both answers' prefixes, then a 0
      uint32_t t[NV];  // per half: 1 where the cell does not match
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        t[j] = vmin2(((w[j] >> bit) & keep) ^ want, 0x00010001u);
        if (j == NV - 1 && !last_valid) t[j] = 0x00010001u;
      }
      // balanced sum: the bit loop is a serial chain, keep its depth short
#pragma unroll
      for (int st = 1; st < NV; st <<= 1)
#pragma unroll
        for (int j = 0; j + st < NV; j += 2 * st) t[j] += t[j + st];
      const uint32_t miss = t[0];
      // matches of both pixels in one reduction (each count <= 441 fits a half)
      const uint32_t c = static_cast<uint32_t>(NV * 32) * 0x00010001u - __reduce_add_sync(0xffffffffu, miss);
      const uint32_t ca = c & 0xffffu, cb = c >> 16;
      if (rank_a >= ca) {  // warp-uniform
        rank_a -= ca;
        res |= 1u << bit;
      }
      if (rank_b >= cb) {
        rank_b -= cb;
        res |= 0x10000u << bit;
      }
    }
    if (lane == 0) O[(r0 + (ea >> 8)) * TW + (ea & 255)] = static_cast<T>(res & 0xffffu);
    if (lane == 1 && e + 1 < F) O[(r0 + (eb >> 8)) * TW + (eb & 255)] = static_cast<T>(res >> 16);
  }
}

// Flagged pixels per strip up to which the bit-plane strategy selects per
// pixel across the warp (radix_sparse_strip) rather than building planes.
template <int K>
struct SparseLimit {
  static constexpr int value = FNR_SPARSE_LIMIT;
};

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
#ifdef FNR_DEBUG_CHECKS
// Debug builds: a strip's flagged list must fit its capacity and every entry
// must name a pixel of the strip (row < SR, column < TW), since the median
// stages index the stage, the output tile and the bit planes with it. On a
// violation the status word records it and the strip takes no medians.
__device__ __forceinline__ int debug_check_list(const uint16_t *list, int F, int SR, int TW, unsigned *status, int lane) {
  bool bad = F < 0 || F > SR * TW;
  for (int j = lane; !bad && j < F; j += 32) {
    const int e = list[j];
    bad = (e >> 8) >= SR || (e & 255) >= TW;
  }
  bad = __any_sync(0xffffffffu, bad);
  if (bad && lane == 0) atomicOr(status, kStatusCheck);
  return bad ? 0 : F;
}

// Debug builds: a TMA box copy must start on a 16-byte boundary in x and at
// a 128-byte aligned shared-memory address (the hardware faults otherwise),
// and a store must not start above the frame.
__device__ __forceinline__ bool debug_tma_ok(int x, int y, int esize, bool store, const void *smem_side,
                                             unsigned *status) {
  const bool ok = ((x * esize) & 15) == 0 && (!store || y >= 0) && (smem_addr(smem_side) & 127u) == 0;
  if (!ok) atomicOr(status, kStatusCheck);
  return ok;
}
#endif

template <int ALGO, int K>
struct MinBlocks {
  // the 81-input network of k = 9 needs about 96 registers, as does the dense
  // 5x5 item; the dense 7x7 item about 150
  static constexpr int value = ALGO == ALGO_DENSE ? (K >= 7 ? 1 : 2) : ((ALGO == ALGO_BITPLANE || K >= 9) ? 2 : 3);
};

template <bool B>
struct Bool {
  static constexpr bool value = B;
};
template <int I>
struct Int {
  static constexpr int value = I;
};

template <typename T, int K, int ALGO>
__global__ void __launch_bounds__(kThreads, MinBlocks<ALGO, K>::value) fnr_kernel(const __grid_constant__ FnrParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int E = sizeof(T);
  constexpr int R = (K - 1) / 2;
  constexpr int XOFF = xoff_for(R, E);
  static_assert(ALGO != ALGO_DENSE3 || K == 3, "DENSE3 is the 3x3 window only");
  static_assert(ALGO != ALGO_DENSE || K == 5 || K == 7, "DENSE is built for the 5x5 and 7x7 windows");

  const int TW = p.tile_w, TH = p.tile_h;
  const Layout L = make_layout(E, K, ALGO, TH, TW);
  const int BW = L.bw, BH = L.bh, SR = L.sr;
  constexpr int NS = num_stages(ALGO);
  const uint32_t box_bytes = static_cast<uint32_t>(BW * BH * E);
  const int stage_stride = L.off_stage[1] - L.off_stage[0];
  auto stage_ptr = [&](int s) { return reinterpret_cast<T *>(smem + L.off_stage[0] + s * stage_stride); };
  T *const out0 = reinterpret_cast<T *>(smem + L.off_out[0]);
  T *const out1 = reinterpret_cast<T *>(smem + L.off_out[1]);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.off_bar);  // [NS]: tile staged
  uint64_t *empty = full + NS;                                       // [NS]: all consumers done with it
  uint64_t *pooled = reinterpret_cast<uint64_t *>(smem + L.off_sync);  // [NS]: network: lists complete
  int *counts = reinterpret_cast<int *>(smem + L.off_sync + 16 * kMaxStages);  // [NS][warps]: list lengths
  TileInfo *info = reinterpret_cast<TileInfo *>(smem + L.off_info);  // [stage]: tile staged there
  int *dir = reinterpret_cast<int *>(smem + L.off_dir);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (p.table != nullptr && p.nframes <= kDirMax)
    for (int f = tid; f < p.nframes; f += kThreads) dir[f] = p.table[f].tile_begin;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
      mbar_init(&pooled[s], kConsumerWarps * 32);  // every consumer lane arrives (releasing its own writes)
    }
    fence_mbar_init();
    if (blockIdx.x == 0 && p.launches != nullptr) atomicAdd(p.launches, 1ull);
#ifdef FNR_DEBUG_CHECKS
    // the launch provides the layout's shared memory, and the tile splits
    // into the consumer warps' strips
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (dyn < static_cast<uint32_t>(L.total) || SR * kConsumerWarps != TH || TW % 8 != 0)
      atomicOr(p.status, kStatusCheck);
#endif
  }
  __syncthreads();  // the only block-wide barrier

  if (warp == kConsumerWarps) {
    // ------------------------------------------------------------- producer
    // Tiles are handed out by an atomic counter when the launch has one and
    // more tiles than CTAs (tiles differ in cost: a strip's median work grows
    // with its flagged pixels), else in static round robin. A CTA's first tile
    // is its own index either way, so no atomic precedes the first load; the
    // counter hands out the tiles after the grid's first ones.
    const bool dynamic = p.sched != nullptr && static_cast<int>(gridDim.x) < p.total_tiles;
    for (int i = 0;; ++i) {
      const int s = i % NS, use = i / NS;
      // the stage's previous tile (i - NS) must be released by every consumer warp
      if (use >= 1 && !mbar_wait_bounded(&empty[s], (use - 1) & 1u, kWaitCycles)) {
        if (lane == 0) atomicOr(p.status, kStatusTimeout);
        break;
      }
      int tile = blockIdx.x + i * static_cast<int>(gridDim.x);
      if (dynamic && i > 0) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&p.sched[0], 1u);
        tile = static_cast<int>(min(__shfl_sync(0xffffffffu, t, 0) + gridDim.x, 0x7fffffffu));
      }
      const TileInfo ti = locate_tile(p, dir, tile);
      T *const S = stage_ptr(s);
      if (lane == 0) info[s] = ti;
      if (!ti.valid) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
        break;
      }
      const int xs = ti.x0 - XOFF;
      const int ys = ti.y0 - R;
      bool tma_load = (ti.flags & kFrameTmaIn) != 0;
#ifdef FNR_DEBUG_CHECKS
      if (tma_load)
        tma_load = __shfl_sync(0xffffffffu, lane == 0 ? debug_tma_ok(xs, ys, E, false, S, p.status) : true, 0);
#endif
      if (tma_load) {
        if (lane == 0) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&full[s], box_bytes);
          tma_load_2d(S, &frame_ptr(p, ti.f)->tin, &full[s], xs, ys);
        }
      } else {
        plain_tile_load<T>(frame_ptr(p, ti.f), xs, ys, S, BW, BH, p.border, lane);
        fence_proxy_async_smem();  // these generic writes precede a later TMA refill of the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
      }
    }
    if (dynamic && lane == 0) {
      // this CTA takes no more tiles; the last CTA to get here resets the slot
      __threadfence();
      if (atomicAdd(&p.sched[1], 1u) == gridDim.x - 1) {
        __threadfence();
        p.sched[0] = 0u;
        p.sched[1] = 0u;
      }
    }
    return;
  }

  // --------------------------------------------------------------- consumers
  const int r0 = warp * SR;  // this warp's output rows [r0, r0 + SR)
  // dense strategies: items of 8 (3x3) or SepNet<K>::kOut output columns, tile_w / that a power of two
  const int seg_shift = 31 - __clz(TW / dense_item_cols(ALGO, K));
  const FastDiv divNP(static_cast<uint32_t>(L.np));     // compacted: vertical items per row group
  const FastDiv divG(static_cast<uint32_t>(TW / 8));    // compacted: horizontal items per row
  unsigned char *const wbase = smem + L.off_warp + warp * L.warp_bytes;
  // pooled network strategy: this warp's strip of the previous tile, stored
  // after the next pooling point (one bulk group per call)
  struct PrevStrip {
    const FrameDev *cf;
    int x0, y0;
    bool live, tma_out;
    T *O;
  } prev{nullptr, 0, 0, false, false, nullptr};
  auto store_prev = [&]() {
    if (prev.live) {
      if (prev.tma_out) {
        if (lane == 0) tma_store_2d(&prev.cf->tout, prev.O + r0 * TW, prev.x0, prev.y0 + r0);
      } else {
        plain_strip_store<T>(prev.cf, prev.O, prev.x0, prev.y0, TW, r0, SR, lane);
      }
    }
    if (lane == 0) bulk_commit();
    prev.live = false;
  };
  for (int i = 0;; ++i) {
    const int s = i % NS;
    if (!mbar_wait_bounded(&full[s], (i / NS) & 1u, kWaitCycles)) {
      if (lane == 0) atomicOr(p.status, kStatusTimeout);
      break;
    }
    const TileInfo cur = info[s];
    if (!cur.valid) {
      if constexpr (ALGO == ALGO_NETWORK && PoolMedians<K>::value) {
        // the end: once every warp is here, the last tile's medians are all written
        mbar_arrive(&pooled[s]);
        if (mbar_wait_bounded(&pooled[s], (i / NS) & 1u, kWaitCycles)) store_prev();
        else if (lane == 0) atomicOr(p.status, kStatusTimeout);
      }
      break;
    }
    const FrameDev *cf = frame_ptr(p, cur.f);
    const int x0 = cur.x0, y0 = cur.y0;
    const int xs = x0 - XOFF, ys = y0 - R;
    const bool tma_in = (cur.flags & kFrameTmaIn) != 0;
    // A TMA store clips the box at the frame edge in whole 16-byte units, so a
    // right-edge tile of a frame whose row is not a multiple of 16 bytes would
    // touch the bytes between W and the pitch: such tiles use plain stores. A
    // TMA copy also needs its shared-memory side 128-byte aligned, so each
    // warp's strip of the output tile (SR rows of TW pixels) must be a
    // multiple of 128 bytes; smaller tiles store their strips with plain stores.
    const bool ragged_right = x0 + TW > cur.W && ((cur.W * E) & 15) != 0;
    bool tma_out = (cur.flags & kFrameTmaOut) != 0 && !ragged_right && ((SR * TW * E) & 127) == 0;
    T *const S = stage_ptr(s);
    T *const O = (i & 1) ? out1 : out0;  // output tiles alternate independently of the stage ring
#ifdef FNR_DEBUG_CHECKS
    if (ALGO != ALGO_DENSE3 && ALGO != ALGO_DENSE && tma_out)
      tma_out = __shfl_sync(0xffffffffu, lane == 0 ? debug_tma_ok(x0, y0 + r0, E, true, O + r0 * TW, p.status) : true,
                            0);
#endif
    const bool live = y0 + r0 < cur.H;  // any of this strip's rows inside the frame

    if (live && (ALGO == ALGO_DENSE3 || ALGO == ALGO_DENSE)) {
      const PackedOp d3op{p.unit, 0u - p.unit};
      // the dense 5x5 / 7x7 items read whole words: for odd R one more column
      // on each side, whose values feed no output
      if (tma_in && p.border != kBorderZero && (x0 < R || ys < 0 || x0 + TW + R > cur.W || ys + BH > cur.H))
        fixup_rows_warp<T>(S, xs, ys, BW, cur.W, cur.H, r0, r0 + SR + K - 1, XOFF - R, XOFF + TW + R - 1, R,
                           p.border, lane);
      // results go straight from registers to the frame (no output tile)
      const bool vec_ok = (cur.flags & kFrameTmaOut) != 0;
      int flagged = 0;
      auto strip = [&](auto count, auto mode) {
        if constexpr (ALGO == ALGO_DENSE3)
          dense3_strip<T, decltype(count)::value, decltype(mode)::value>(S, cf, x0, y0, TW, BW, r0, SR, seg_shift,
                                                                         cur.W - x0, cur.H - y0, vec_ok, lane,
                                                                         flagged, d3op);
        else if constexpr (ALGO == ALGO_DENSE && (K == 5 || K == 7))
          dense_sep_strip<T, K, decltype(count)::value, decltype(mode)::value>(
              S, cf, x0, y0, BW, r0, SR, seg_shift, cur.W - x0, cur.H - y0, vec_ok, lane, flagged, d3op);
      };
      if (p.mode == kModeMedian) {
        strip(Bool<false>{}, Int<kModeMedian>{});
        if (cur.counted && lane == 0) {  // every in-frame pixel of the strip takes a median
          const int rows = min(SR, cur.H - y0 - r0), cols = min(TW, cur.W - x0);
          atomicAdd(cf->flagged, static_cast<unsigned long long>(rows) * static_cast<unsigned long long>(cols));
        }
      } else if (p.mode == kModeDirectional) {
        strip(Bool<true>{}, Int<kModeDirectional>{});
        flagged = __reduce_add_sync(0xffffffffu, flagged);
        if (cur.counted && lane == 0 && flagged != 0) atomicAdd(cf->flagged, static_cast<unsigned long long>(flagged));
      } else if (cur.counted) {
        strip(Bool<true>{}, Int<kModeFnr>{});
        flagged = __reduce_add_sync(0xffffffffu, flagged);
        if (lane == 0 && flagged != 0) atomicAdd(cf->flagged, static_cast<unsigned long long>(flagged));
      } else {
        strip(Bool<false>{}, Int<kModeFnr>{});
      }
    } else if constexpr (ALGO == ALGO_NETWORK && PoolMedians<K>::value) {
      // Every consumer warp takes part, live strip or not: the strips' flagged
      // pixels are pooled across the tile (network_pooled) after one CTA-level
      // point per tile, an mbarrier with a bounded wait (`pooled`): every list
      // of this tile and its fix-up rows are complete, and every median of the
      // previous tile is written and fenced, so the strips of the previous
      // tile are stored right after it (its output tile is the other one).
      const int w_list = L.w_list + (i & 1) * L.list_bytes;  // this tile's list (see pool_medians)
      uint16_t *list = reinterpret_cast<uint16_t *>(wbase + w_list);
      int flagged = 0;
      if (live && tma_in && p.border != kBorderZero &&
          (x0 < R || ys < 0 || x0 + TW + R > cur.W || ys + BH > cur.H))
        fixup_rows_warp<T>(S, xs, ys, BW, cur.W, cur.H, r0, r0 + SR + K - 1, XOFF - R, XOFF + TW + R - 1, R,
                           p.border, lane);
      // the store issued during the previous tile (of the tile before it, from
      // this output tile) has read its strip
      if (lane == 0) bulk_wait_read<0>();
      __syncwarp();
      if (live) {
        uint32_t *vmin = reinterpret_cast<uint32_t *>(wbase + L.w_vmin);
        uint32_t *vmax = reinterpret_cast<uint32_t *>(wbase + L.w_vmax);
        // the window extremes (the directional detector needs none)
        if (p.mode != kModeDirectional) vertical_pairs<T, K>(S, vmin, vmax, BW, L.np, L.nps, L.cb, r0, SR, divNP, lane);
        __syncwarp();
        flagged = horizontal_pairs<T, K>(S, vmin, vmax, O, list, TW, BW, L.nps, r0, SR, cur.W - x0, cur.H - y0,
                                         p.mode, divG, PackedOp{p.unit, 0u - p.unit}, lane);
#ifdef FNR_DEBUG_CHECKS
        flagged = debug_check_list(list, flagged, SR, TW, p.status, lane);
#endif
      }
      if (lane == 0) {
        counts[s * kConsumerWarps + warp] = flagged;
        if (flagged != 0 && cur.counted) atomicAdd(cf->flagged, static_cast<unsigned long long>(flagged));
      }
      __syncwarp();
      mbar_arrive(&pooled[s]);
      if (!mbar_wait_bounded(&pooled[s], (i / NS) & 1u, kWaitCycles)) {
        if (lane == 0) atomicOr(p.status, kStatusTimeout);
        break;
      }
      store_prev();
      int total = 0;
#pragma unroll
      for (int j = 0; j < kConsumerWarps; ++j) total += counts[s * kConsumerWarps + j];
      network_pooled<T, K>(S, O, smem + L.off_warp, L.warp_bytes, w_list, counts + s * kConsumerWarps, total, TW, BW,
                           SR, warp, lane, PackedOp{p.unit, 0u - p.unit});
      fence_proxy_async_smem();  // these medians precede the TMA stores issued after the next pooling point
      prev = PrevStrip{cf, x0, y0, live, tma_out, O};
    } else if (live) {
      if (tma_in && p.border != kBorderZero && (x0 < R || ys < 0 || x0 + TW + R > cur.W || ys + BH > cur.H))
        fixup_rows_warp<T>(S, xs, ys, BW, cur.W, cur.H, r0, r0 + SR + K - 1, XOFF - R, XOFF + TW + R - 1, R,
                           p.border, lane);
      // this warp's store from the same output tile (two tiles ago, or the
      // previous tile when there is one output tile) has read its strip
      if (lane == 0) {
        if constexpr (out_buffers(ALGO) == 2) bulk_wait_read<1>();
        else bulk_wait_read<0>();
      }
      __syncwarp();
      int flagged = 0;
      {
        uint16_t *list = reinterpret_cast<uint16_t *>(wbase + L.w_list);
        uint32_t *vmin = reinterpret_cast<uint32_t *>(wbase + L.w_vmin);
        uint32_t *vmax = reinterpret_cast<uint32_t *>(wbase + L.w_vmax);
        // the window extremes (the directional detector needs none)
        if (p.mode != kModeDirectional) vertical_pairs<T, K>(S, vmin, vmax, BW, L.np, L.nps, L.cb, r0, SR, divNP, lane);
        __syncwarp();
        flagged = horizontal_pairs<T, K>(S, vmin, vmax, O, list, TW, BW, L.nps, r0, SR, cur.W - x0, cur.H - y0,
                                         p.mode, divG, PackedOp{p.unit, 0u - p.unit}, lane);
#ifdef FNR_DEBUG_CHECKS
        flagged = debug_check_list(list, flagged, SR, TW, p.status, lane);
#endif
        if constexpr (ALGO == ALGO_NETWORK) {
          network_strip<T, K>(S, O, list, flagged, TW, BW, r0, lane, PackedOp{p.unit, 0u - p.unit});
        } else if (flagged <= SparseLimit<K>::value) {
          radix_sparse_strip<T, K>(S, O, list, flagged, TW, BW, r0, lane);
        } else {
          uint32_t *planes = reinterpret_cast<uint32_t *>(wbase + L.w_planes);
          const uint32_t orv = build_planes_warp<T>(S, planes, BW, XOFF - R, r0, L.plane_rows, L.pw, lane);
          bitplane_strip<T, K>(planes, O, list, flagged, TW, L.plane_rows, L.pw, 32 - __clz(static_cast<int>(orv)),
                               r0, lane);
        }
      }
      __syncwarp();
      if (tma_out) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tma_store_2d(&cf->tout, O + r0 * TW, x0, y0 + r0);
      } else {
        plain_strip_store<T>(cf, O, x0, y0, TW, r0, SR, lane);
      }
      if (lane == 0) {
        bulk_commit();
        if (flagged != 0 && cur.counted) atomicAdd(cf->flagged, static_cast<unsigned long long>(flagged));
      }
    } else if (ALGO != ALGO_DENSE3 && ALGO != ALGO_DENSE && lane == 0) {
      bulk_commit();  // keep one bulk group per tile so the wait above stays exact
    }
    fence_proxy_async_smem();  // this warp's generic writes to the stage precede its refill by TMA
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (lane == 0) bulk_wait_all<0>();
}

template <typename T, int K>
inline const void *kernel_for(int algo) {
  switch (algo) {
    case ALGO_DENSE3:
      if constexpr (K == 3) return reinterpret_cast<const void *>(&fnr_kernel<T, 3, ALGO_DENSE3>);
      return nullptr;
    case ALGO_NETWORK:
      if constexpr (K <= 9) return reinterpret_cast<const void *>(&fnr_kernel<T, K, ALGO_NETWORK>);
      return nullptr;
    case ALGO_DENSE:
      if constexpr (K == 5 || K == 7) return reinterpret_cast<const void *>(&fnr_kernel<T, K, ALGO_DENSE>);
      return nullptr;
    case ALGO_BITPLANE:
      return reinterpret_cast<const void *>(&fnr_kernel<T, K, ALGO_BITPLANE>);
    default:
      return nullptr;
  }
}

}  // namespace fnr
