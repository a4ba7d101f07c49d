// Kernel parameter blocks and shared-memory layout, shared by the host code
// and the kernels of the FNR filter library.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace fnr {

constexpr int kConsumerWarps = 8;      // warps that filter; each owns a strip of tile_h / 8 rows
constexpr int kThreads = (kConsumerWarps + 1) * 32;  // + one producer warp (tile loads)
constexpr int kMaxK = 21;              // largest window built
constexpr int kNumK = (kMaxK - 3) / 2 + 1;
constexpr int kDirMax = 512;           // frames whose tile ranges a CTA keeps in shared memory

enum Algo : int { ALGO_AUTO = 0, ALGO_DENSE3 = 1, ALGO_NETWORK = 2, ALGO_BITPLANE = 3, ALGO_DENSE = 4 };

// The dense strategies take a median for every pixel and write results
// straight from registers: no output tile, no per-warp lists.
__host__ __device__ constexpr bool dense_algo(int algo) { return algo == ALGO_DENSE3 || algo == ALGO_DENSE; }

// Output columns of one lane item of the dense strategies (a row pair times
// this many columns): 8 for the 3x3 path; for the separable networks the
// generator's choice (fnr_separable.cuh, SepNet<K>::kOut), repeated here for
// the host's tile checks.
// Whether a lane of the dense strategy filters a span of neighbouring items,
// handing the sorted columns and merged blocks they share from item to item
// (the 7x7 network), rather than each item on its own (5x5).
__host__ __device__ constexpr bool dense_sliding(int k) { return k == 7; }
__host__ __device__ constexpr int dense_item_cols(int algo, int k) {
  return algo == ALGO_DENSE && k == 7 ? 8 : 8;
}

// Frame flags
constexpr int kFrameTmaIn = 1;     // load tiles with TMA (16 B aligned base and pitch)
constexpr int kFrameTmaOut = 2;    // store tiles with TMA

// One frame as the kernel sees it. The tensor maps come first: they need
// 128-byte alignment.
struct alignas(128) FrameDev {
  CUtensorMap tin;                 // box = (tile_w + 2*xoff) x (tile_h + 2r), u8/u16
  CUtensorMap tout;                // box = tile_w x (tile_h / kConsumerWarps): one warp's strip
  const unsigned char *in;
  unsigned char *out;
  long long in_pitch;
  long long out_pitch;
  int H, W;
  int tiles_x, tiles_y;
  int tile_begin;                  // first global tile index of this frame in its class
  int flags;
  unsigned long long *flagged;     // nullable, device
};

struct alignas(128) FnrParams {
  FrameDev single;                 // used when table == nullptr
  const FrameDev *table;           // device array of nframes frames (batch)
  int nframes;
  int total_tiles;
  int tile_w, tile_h;
  unsigned int *status;            // device status word (bit 0: bounded wait timed out)
  unsigned long long *launches;    // device launch counter (nullable)
  // dynamic tile order (nullable: static round robin): each CTA's first tile
  // is its block index; when there are more tiles than CTAs, sched[0] hands
  // out the rest (tile gridDim.x + counter), sched[1] counts CTAs that are
  // done, and the last CTA zeroes both, so a slot is ready for the next
  // launch ordered after this one (a launch with no more tiles than CTAs
  // leaves the slot untouched)
  unsigned int *sched;
  int mode;                        // kModeFnr, kModeMedian or kModeDirectional: which pixels are noisy
  int border;                      // kBorderReplicate / kBorderMirror / kBorderZero
  unsigned int unit = 1u;          // always 1: multiplier of the median networks' multiply-add form
};

constexpr int kBorderReplicate = 0;  // clamp to the nearest edge pixel (default)
constexpr int kBorderMirror = 1;     // reflect about the edge pixel: d c b | a b c d | c b a
constexpr int kBorderZero = 2;       // outside pixels read 0

constexpr int kModeFnr = 0;        // replace only pixels equal to a window extreme (Sec. 3.3-3.4)
constexpr int kModeMedian = 1;     // standard median filter: replace every pixel (the paper's MF, Sec. 2)
// directional detector (Fig. 1): a pixel is noisy iff along none of the four
// lines through it (horizontal, vertical, two diagonals) it lies strictly
// between its two neighbours; noisy pixels take the k x k median as in FNR
constexpr int kModeDirectional = 2;

constexpr unsigned int kStatusTimeout = 1u;
// builds with FNR_DEBUG_CHECKS: an internal index or alignment check failed
// in a kernel, which skipped the access (or took the plain path) instead
constexpr unsigned int kStatusCheck = 2u;

__host__ __device__ constexpr int align_up(int v, int a) { return (v + a - 1) / a * a; }

// Left halo (in pixels) rounded up so that every TMA box starts on a 16-byte
// boundary: x0 - xoff is a multiple of 16 / esize when x0 is.
__host__ __device__ constexpr int xoff_for(int r, int esize) {
  return align_up(r, 16 / esize);
}

// Staging buffers per CTA (a ring: the producer loads up to this many tiles
// ahead of the slowest consumer warp).
__host__ __device__ constexpr int num_stages(int algo) { return dense_algo(algo) ? 3 : 2; }
__host__ __device__ constexpr int out_buffers(int algo) { return algo == ALGO_BITPLANE ? 1 : 2; }
// Whether the network strategy pools the flagged pixels of a tile across its
// strips; a pooling warp keeps two flagged lists, alternating by tile, since
// the other warps may still read its previous list while it builds the next.
__host__ __device__ constexpr bool pool_medians(int algo, int k) { return algo == ALGO_NETWORK && k >= 9; }
constexpr int kMaxStages = 3;

// Default strategy and output tile per (pixel size, k), used by handles until
// tuned and by the allocation-free entry point. Measured on GB300 (tile
// sweeps of all strategies): the 640x512 14-bit sweep for k <= 7 (k = 5:
// dense 128x64 0.097 ms per 128 frames against 0.144 for the network
// strategy; k = 7: dense 128x128 0.197 against 0.234); for the bit-plane
// windows, 1280x1024 frames with sparse random-valued impulses and the mixed
// batch's dense k = 15 frames, where a taller strip (16 rows per warp) builds
// fewer halo rows of planes per output row.
struct DefaultTile {
  int algo, tile_w, tile_h;
};
__host__ __device__ constexpr DefaultTile default_tile(int /*esize: the same for both pixel sizes*/, int k) {
  return k == 3   ? DefaultTile{ALGO_DENSE3, 128, 64}
         : k == 5 ? DefaultTile{ALGO_DENSE, 128, 64}
         : k == 7 ? DefaultTile{ALGO_DENSE, 128, 128}
         : k <= 9 ? DefaultTile{ALGO_NETWORK, 64, 64}
                  : DefaultTile{ALGO_BITPLANE, 32, 128};
}

// Rows per vertical/horizontal extreme group of the compacted strategies.
__host__ __device__ constexpr int row_group(int k) { return k >= 8 ? 8 : (k >= 4 ? 4 : 2); }

// tile_h must split into kConsumerWarps strips, each a whole number of row
// groups (compacted strategies) or of row pairs (dense 3x3).
__host__ __device__ constexpr int tile_h_multiple(int k, int algo) {
  return kConsumerWarps * (dense_algo(algo) ? 2 : row_group(k));
}

// Shared-memory layout of one CTA (byte offsets). Identical on host and device.
// Per CTA: two staging buffers and two output tiles; per consumer warp: its
// flagged list, vertical extremes and (bit-plane strategy) bit planes.
struct Layout {
  int r, bw, bh, vw, pw, nbmax, sr;
  int cb, np;          // packed column pairs: first stage column (even) and words per row
  int nps;             // row stride of the per-warp extreme words (np padded for 16-byte reads)
  int off_stage[kMaxStages];
  int off_out[2];
  int off_warp;        // first per-warp block
  int warp_bytes;      // size of one per-warp block
  int w_list, w_vmin, w_vmax, w_planes;  // offsets inside a per-warp block
  int list_bytes;                        // one flagged list (two when pooling, alternating by tile)
  int plane_rows;      // rows of bit planes a warp builds (its strip + halo)
  int off_bar;         // full[stages], empty[stages]
  int off_sync;        // network strategy: pooled[stages] barriers (and a spare row), then list counts [stages][warps]
  int off_info;
  int off_dir;
  int total;
};

__host__ __device__ inline Layout make_layout(int esize, int k, int algo, int tile_h, int tile_w) {
  Layout L{};
  L.r = (k - 1) / 2;
  const int xoff = xoff_for(L.r, esize);
  L.bw = tile_w + 2 * xoff;
  // the sliding dense items: a row pitch of an odd number of 16-byte units
  // (the box reads a few more columns), so that lanes reading the same column
  // of neighbouring row pairs fall in different banks
  if (algo == ALGO_DENSE && dense_sliding(k) && ((L.bw * esize / 16) & 1) == 0) L.bw += 16 / esize;
  L.bh = tile_h + 2 * L.r;
  L.vw = tile_w + 2 * L.r;
  // pair words cover stage columns [cb, cb + 2 np): every column a window reads
  L.cb = (xoff - L.r) & ~1;
  L.np = (xoff + tile_w + L.r - 1 - L.cb) / 2 + 1;
  {
    // the horizontal pass reads the words of 8 output columns as 16-byte
    // vectors: nw words from word x0/2, rounded up to whole vectors
    const int par = (xoff - L.r) & 1;
    const int nw = ((2 * L.r + par + 7) >> 1) + 1;
    const int nwr = (nw + 3) & ~3;
    const int need = tile_w / 2 - 4 + nwr;
    L.nps = align_up(L.np > need ? L.np : need, 4);
  }
  // bit-plane words per row, from stage column xoff - r (the first column a
  // window of the tile reads): a window starting at tile column tx reads bits
  // tx .. tx + 2r of words tx / 32 and tx / 32 + 1. Tiles up to 32 columns
  // whose windows fit in 64 bits keep exactly two words (read as one 8-byte
  // word); wider ones keep the words the windows reach plus one more.
  L.pw = (tile_w <= 32 && tile_w + 2 * L.r <= 64) ? 2 : (tile_w + 2 * L.r + 31) / 32 + 1;
  L.nbmax = 8 * esize;
  L.sr = tile_h / kConsumerWarps;
  L.plane_rows = L.sr + k - 1;
  int off = 0;
  // +16: a pair word may read one pixel past the last staged column (never used)
  const int stage = align_up(L.bw * L.bh * esize + 16, 128);
  // the dense strategies write results straight from registers: no output tile
  const int outb = dense_algo(algo) ? 0 : align_up(tile_w * tile_h * esize, 128);
  for (int i = 0; i < kMaxStages; ++i) {
    L.off_stage[i] = off;
    if (i < num_stages(algo)) off += stage;
  }
  // output tiles: two, alternating by tile, except for the bit-plane strategy,
  // whose shared memory is the tightest (its warps wait for their previous
  // store instead)
  L.off_out[0] = off; off += outb;
  L.off_out[1] = L.off_out[0];
  if (out_buffers(algo) == 2) {
    L.off_out[1] = off;
    off += outb;
  }
  L.w_list = L.w_vmin = L.w_vmax = L.w_planes = -1;
  int w = 0;
  if (!dense_algo(algo)) {
    L.list_bytes = align_up(L.sr * tile_w * 2, 16);
    L.w_list = w; w += L.list_bytes * (pool_medians(algo, k) ? 2 : 1);
    L.w_vmin = w; w += align_up(L.sr * L.nps * 4, 16);
    L.w_vmax = w; w += align_up(L.sr * L.nps * 4, 16);
  }
  if (algo == ALGO_BITPLANE) {
    // the planes are built after the horizontal pass has consumed the extreme
    // words, so they overlay them
    const int planes = align_up(L.nbmax * L.plane_rows * L.pw * 4, 16);
    L.w_planes = L.w_vmin;
    if (L.w_planes + planes > w) w = L.w_planes + planes;
  }
  L.warp_bytes = align_up(w, 128);
  L.off_warp = off; off += kConsumerWarps * L.warp_bytes;
  L.off_bar = off; off += 16 * kMaxStages;
  L.off_sync = off; off += 16 * kMaxStages + 4 * kConsumerWarps * kMaxStages;
  L.off_info = off; off += 32 * kMaxStages;
  L.off_dir = off; off += kDirMax * 4;
  L.total = align_up(off, 128);
  return L;
}

}  // namespace fnr
