// Host side of the C ABI declared in include/ir_filter.h: argument checks,
// tensor-map encoding, per-(dtype, k) kernel configuration and tuning,
// launches, batch plans (explicit CUDA graphs) and error reporting.
#include "ir_filter.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fnr_host.h"
#include "fnr_params.h"

namespace fnr {
const void *get_kernel_k3(int esize, int k, int algo);
const void *get_kernel_k5_7(int esize, int k, int algo);
const void *get_kernel_k9_11(int esize, int k, int algo);
const void *get_kernel_k13_15(int esize, int k, int algo);
const void *get_kernel_k17_21(int esize, int k, int algo);

static const void *get_kernel(int esize, int k, int algo) {
  if (k == 3) return get_kernel_k3(esize, k, algo);
  if (k <= 7) return get_kernel_k5_7(esize, k, algo);
  if (k <= 11) return get_kernel_k9_11(esize, k, algo);
  if (k <= 15) return get_kernel_k13_15(esize, k, algo);
  return get_kernel_k17_21(esize, k, algo);
}
}  // namespace fnr

using namespace fnr;

namespace {

thread_local std::string g_last_error;

int esize_of(ir_dtype d) { return d == IR_U8 ? 1 : 2; }
int kslot(int k) { return (k - 3) / 2; }

bool valid_dtype(int d) { return d == IR_U8 || d == IR_U16 || d == IR_U14; }
bool valid_k(int k) { return k >= 3 && k <= kMaxK && (k & 1); }

}  // namespace

// ir_filter_run_host pipelines its chunks over three streams: host-to-device
// copies, filtering, device-to-host copies
constexpr int kHostStreams = 3;
constexpr int kHostChunks = 16;  // its default number of pipeline chunks

struct PlanKey {
  std::vector<unsigned char> bytes;
  bool operator<(const PlanKey &o) const { return bytes < o.bytes; }
  bool operator==(const PlanKey &o) const { return bytes == o.bytes; }
};

struct ir_filter {
  int device = 0;
  int sm_count = 0;
  int max_smem = 0;
  unsigned *d_status = nullptr;
  unsigned long long *d_launches = nullptr;
  unsigned *d_sched = nullptr;  // kSchedSlots tile-order slots (2 words each) for one-off launches
  std::atomic<unsigned> sched_next{0};  // also taken by a server's batcher thread
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  ir_kernel_config cfg[2][kNumK];
  int border = kBorderReplicate;
  int detector = kModeFnr;  // kModeFnr (Eq. 3a/3b) or kModeDirectional
  bool strict_align = false;  // misaligned frames are refused (IR_EALIGN) instead of staged with plain loads
  bool tile_fit = true;       // launches with fewer tiles than SMs shrink their tile (fit_tile)
  std::string last_error;
  std::map<std::pair<const void *, int>, int> occupancy;  // (kernel, smem) -> CTAs per SM
  std::map<const void *, int> smem_attr;                  // kernel -> dynamic smem attribute set
  std::map<PlanKey, ir_batch_plan *> plans;               // ir_filter_run_batch cache
  std::vector<PlanKey> plan_order;                        // LRU, oldest first
  // ir_filter_run_host: copy streams, device staging and one plan per chunk
  cudaStream_t host_streams[kHostStreams] = {};
  cudaEvent_t host_start = nullptr, host_done = nullptr;
  std::vector<cudaEvent_t> host_events;  // per chunk: copied in, filtered
  unsigned char *host_stage = nullptr;
  size_t host_stage_bytes = 0;
  std::vector<PlanKey> host_keys;
  std::vector<ir_batch_plan *> host_plans;
};

struct ir_batch_plan {
  ir_filter *h = nullptr;
  FrameDev *d_table = nullptr;
  unsigned *d_sched = nullptr;  // one tile-order slot per class kernel
  std::vector<ClassLaunch> classes;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
ir_status fnr::host_fail(ir_filter *h, ir_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  if (h) h->last_error = buf;
  return s;
}

static ir_status fail(ir_filter *h, ir_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
static ir_status fail(ir_filter *h, ir_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return fnr::host_fail(h, s, "%s", buf);
}

#define IR_CUDA(h, call)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((h), IR_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (prev_ >= 0 && prev_ != dev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1, dev_ = 0;
};

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------
static ir_kernel_config default_config(int esize, int k) {
  const DefaultTile d = default_tile(esize, k);
  ir_kernel_config c{};
  c.ctas_per_sm = 0;
  c.algo = d.algo;
  c.tile_w = d.tile_w;
  c.tile_h = d.tile_h;
  return c;
}

static bool config_ok(const ir_filter *h, int esize, int k, const ir_kernel_config &c, std::string *why) {
  auto no = [&](const char *m) {
    if (why) *why = m;
    return false;
  };
  if (c.tile_w < 8 || c.tile_h < 8 || (c.tile_w % 8) || (c.tile_h % 8)) return no("tile sides must be multiples of 8");
  // every TMA x coordinate (a multiple of tile_w, minus a 16-byte aligned
  // halo) and every box row must be a whole number of 16-byte units
  if ((c.tile_w * esize) % 16) return no("tile_w * bytes per pixel must be a multiple of 16");
  if (c.algo == IR_ALGO_DENSE3 && k != 3) return no("DENSE3 is the 3x3 window only");
  if (c.algo == IR_ALGO_DENSE && k != 5 && k != 7) return no("DENSE is built for k = 5 and 7");
  if (c.algo == IR_ALGO_NETWORK && k > 9) return no("NETWORK is built for k <= 9");
  if (c.algo != IR_ALGO_DENSE3 && c.algo != IR_ALGO_NETWORK && c.algo != IR_ALGO_BITPLANE && c.algo != IR_ALGO_DENSE)
    return no("unknown algo");
  if (c.ctas_per_sm < 0) return no("ctas_per_sm < 0");
  if (c.tile_h % tile_h_multiple(k, c.algo)) return no("tile_h must split into 8 warp strips of whole row groups");
  if (c.algo == IR_ALGO_DENSE3 || c.algo == IR_ALGO_DENSE) {
    const int cols = dense_item_cols(c.algo, k);
    if (c.tile_w % cols || ((c.tile_w / cols) & (c.tile_w / cols - 1)))
      return no("the dense strategies need tile_w a power-of-two multiple of their item width");
  }
  const Layout L = make_layout(esize, k, c.algo, c.tile_h, c.tile_w);
  if (L.bw > 256 || L.bh > 256) return no("tile plus halo exceeds the 256-pixel TMA box");
  if (c.tile_w > 256 || c.tile_h > 256) return no("tile side > 256");
  if (h && L.total > h->max_smem) return no("tile needs more shared memory than a CTA can have");
  return true;
}

// A class whose frames give fewer tiles than the GPU has SMs would leave SMs
// idle: its tile shrinks (height first, then width, keeping the strategy and
// at least 4096 pixels per tile, so that every consumer warp still has a lane
// item per lane) until the tiles cover the SMs or it cannot shrink further.
static ir_kernel_config fit_tile(const ir_filter *h, int es, int k, ir_kernel_config c, const int *Hs, const int *Ws,
                                 int n) {
  auto tiles = [&](const ir_kernel_config &x) {
    long long t = 0;
    for (int i = 0; i < n; ++i)
      t += static_cast<long long>((Ws[i] + x.tile_w - 1) / x.tile_w) * ((Hs[i] + x.tile_h - 1) / x.tile_h);
    return t;
  };
  while (h->tile_fit && tiles(c) < h->sm_count) {
    ir_kernel_config a = c, b = c;
    a.tile_h /= 2;
    b.tile_w /= 2;
    if (a.tile_h * a.tile_w >= 4096 && config_ok(h, es, k, a, nullptr)) c = a;
    else if (b.tile_h * b.tile_w >= 4096 && config_ok(h, es, k, b, nullptr)) c = b;
    else break;
  }
  return c;
}

// ---------------------------------------------------------------------------
// frames
// ---------------------------------------------------------------------------
static bool ranges_overlap(const void *a, size_t a_len, const void *b, size_t b_len) {
  const auto pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
  return pa < pb + b_len && pb < pa + a_len;
}

static bool tma_addressable(const void *p, size_t pitch);

static ir_status check_frame(ir_filter *h, const void *in, size_t in_pitch, const void *out, size_t out_pitch, int H,
                             int W, int dtype, int k, bool host_frame = false) {
  if (!in || !out) return fail(h, IR_EINVAL, "null frame pointer");
  if (H < 1 || W < 1) return fail(h, IR_EINVAL, "H and W must be >= 1 (got %d x %d)", H, W);
  if (!valid_dtype(dtype)) return fail(h, IR_EINVAL, "unknown dtype %d", dtype);
  if (!valid_k(k)) return fail(h, IR_EINVAL, "k must be odd and in [3, %d] (got %d)", kMaxK, k);
  const size_t row = static_cast<size_t>(W) * esize_of(static_cast<ir_dtype>(dtype));
  if (in_pitch < row || out_pitch < row) return fail(h, IR_EINVAL, "pitch smaller than W * bytes per pixel");
  if (static_cast<long long>(H) * W > (1LL << 40)) return fail(h, IR_EINVAL, "frame too large");
  const size_t in_len = (H - 1) * in_pitch + row, out_len = (H - 1) * out_pitch + row;
  // host frames are staged through separate device buffers, so one may be filtered in place
  const bool same = host_frame && in == out && in_pitch == out_pitch;
  if (!same && ranges_overlap(in, in_len, out, out_len)) return fail(h, IR_EINVAL, "input and output overlap");
  if (!host_frame && h && h->strict_align && (!tma_addressable(in, in_pitch) || !tma_addressable(out, out_pitch)))
    return fail(h, IR_EALIGN, "strict alignment: frame base or pitch is not a multiple of 16 bytes");
  return IR_OK;
}

static bool tma_addressable(const void *p, size_t pitch) {
  return (reinterpret_cast<uintptr_t>(p) % 16) == 0 && (pitch % 16) == 0 && pitch < (1ull << 40);
}

static bool encode_map(ir_filter *h, CUtensorMap *map, int esize, const void *base, int H, int W, size_t pitch, int box_w,
                       int box_h) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_w), static_cast<cuuint32_t>(box_h)};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = h->encode(map, esize == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                               const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void fnr::host_make_frame_dev(ir_filter *h, FrameDev &f, const void *in, size_t in_pitch, void *out, size_t out_pitch,
                           int H, int W, int esize, int k, const ir_kernel_config &c, unsigned long long *flagged) {
  std::memset(&f, 0, sizeof f);
  const int r = (k - 1) / 2;
  const Layout L = make_layout(esize, k, c.algo, c.tile_h, c.tile_w);
  f.in = static_cast<const unsigned char *>(in);
  f.out = static_cast<unsigned char *>(out);
  f.in_pitch = static_cast<long long>(in_pitch);
  f.out_pitch = static_cast<long long>(out_pitch);
  f.H = H;
  f.W = W;
  f.tiles_x = (W + c.tile_w - 1) / c.tile_w;
  f.tiles_y = (H + c.tile_h - 1) / c.tile_h;
  f.flagged = flagged;
  f.flags = 0;
  (void)r;
  const bool box_ok = (c.tile_w * esize) % 16 == 0 && (L.bw * esize) % 16 == 0;
  if (box_ok && tma_addressable(in, in_pitch) && encode_map(h, &f.tin, esize, in, H, W, in_pitch, L.bw, L.bh))
    f.flags |= kFrameTmaIn;
  if (box_ok && tma_addressable(out, out_pitch) &&
      encode_map(h, &f.tout, esize, out, H, W, out_pitch, c.tile_w, c.tile_h / kConsumerWarps))
    f.flags |= kFrameTmaOut;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
ir_kernel_config fnr::host_config(const ir_filter *h, int esize, int k) { return h->cfg[esize - 1][kslot(k)]; }
int fnr::host_device(const ir_filter *h) { return h->device; }
int fnr::host_sm_count(const ir_filter *h) { return h->sm_count; }
unsigned *fnr::host_status_word(const ir_filter *h) { return h->d_status; }
unsigned long long *fnr::host_launch_counter(const ir_filter *h) { return h->d_launches; }

// Launches that are not part of a plan take the handle's slots in turn: each
// kernel resets its slot when it ends, and a slot is only reused kSchedSlots
// launches later, so launches in flight together on several streams get
// different slots unless more than kSchedSlots of them overlap.
unsigned *fnr::host_sched_slot(ir_filter *h) { return h->d_sched + 2 * (h->sched_next.fetch_add(1) % kSchedSlots); }

ir_status fnr::host_prepare_class(ir_filter *h, ClassLaunch &cl) {
  cl.fn = get_kernel(cl.esize, cl.k, cl.cfg.algo);
  if (!cl.fn) return fail(h, IR_EUNSUPPORTED, "no kernel built for esize=%d k=%d algo=%d", cl.esize, cl.k, cl.cfg.algo);
  const Layout L = make_layout(cl.esize, cl.k, cl.cfg.algo, cl.cfg.tile_h, cl.cfg.tile_w);
  cl.smem = L.total;
  int &attr = h->smem_attr[cl.fn];
  if (attr < cl.smem) {
    IR_CUDA(h, cudaFuncSetAttribute(cl.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, h->max_smem));
    attr = h->max_smem;
  }
  auto key = std::make_pair(cl.fn, cl.smem);
  auto it = h->occupancy.find(key);
  int per_sm = 0;
  if (it == h->occupancy.end()) {
    IR_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cl.fn, kThreads, cl.smem));
    h->occupancy[key] = per_sm;
  } else {
    per_sm = it->second;
  }
  if (per_sm < 1) return fail(h, IR_EUNSUPPORTED, "kernel does not fit on an SM with %d bytes of shared memory", cl.smem);
  if (cl.cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, cl.cfg.ctas_per_sm);
  cl.grid = std::max(1, std::min(cl.prm.total_tiles, per_sm * h->sm_count));
  return IR_OK;
}

ir_status fnr::host_launch_class(ir_filter *h, ClassLaunch &cl, cudaStream_t st) {
  if (cl.prm.sched == nullptr) cl.prm.sched = host_sched_slot(h);
  void *args[] = {&cl.prm};
  IR_CUDA(h, cudaLaunchKernel(cl.fn, dim3(cl.grid), dim3(kThreads), args, cl.smem, st));
  return IR_OK;
}

static ir_status ensure_scratch(ir_filter *h, size_t bytes) {
  if (h->scratch_bytes >= bytes) return IR_OK;
  if (h->scratch) {
    cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_bytes = 0;
  }
  const size_t want = std::max(bytes, static_cast<size_t>(1) << 20);
  if (cudaMalloc(&h->scratch, want) != cudaSuccess) {
    cudaGetLastError();
    h->scratch = nullptr;
    return fail(h, IR_ENOMEM, "cannot allocate %zu bytes of scratch", want);
  }
  h->scratch_bytes = want;
  return IR_OK;
}

static ir_status run_one(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch, int H, int W,
                         ir_dtype dtype, int k, cudaStream_t st, unsigned long long *flagged, int mode = kModeFnr) {
  ClassLaunch cl;
  cl.esize = esize_of(dtype);
  cl.k = k;
  cl.cfg = fit_tile(h, cl.esize, k, h->cfg[cl.esize - 1][kslot(k)], &H, &W, 1);
  cl.prm = FnrParams{};
  host_make_frame_dev(h, cl.prm.single, in, in_pitch, out, out_pitch, H, W, cl.esize, k, cl.cfg, flagged);
  cl.prm.table = nullptr;
  cl.prm.nframes = 1;
  cl.prm.total_tiles = cl.prm.single.tiles_x * cl.prm.single.tiles_y;
  cl.prm.tile_w = cl.cfg.tile_w;
  cl.prm.tile_h = cl.cfg.tile_h;
  cl.prm.status = h->d_status;
  cl.prm.launches = h->d_launches;
  cl.prm.mode = mode == kModeFnr ? h->detector : mode;
  cl.prm.border = h->border;
  ir_status s = host_prepare_class(h, cl);
  if (s != IR_OK) return s;
  if (flagged) IR_CUDA(h, cudaMemsetAsync(flagged, 0, sizeof(unsigned long long), st));
  return host_launch_class(h, cl, st);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *ir_filter_version(void) { return "0.1.0"; }

const char *ir_status_string(ir_status s) {
  switch (s) {
    case IR_OK: return "ok";
    case IR_EINVAL: return "invalid argument";
    case IR_EALIGN: return "misaligned frame";
    case IR_ENOMEM: return "out of device memory";
    case IR_ECUDA: return "CUDA error";
    case IR_ETIMEOUT: return "device-side wait timed out";
    case IR_EBUSY: return "busy";
    case IR_EUNSUPPORTED: return "unsupported configuration";
    case IR_ECHECK: return "internal check failed in a kernel (debug build)";
  }
  return "unknown status";
}

const char *ir_filter_last_error(const ir_filter *h) { return h ? h->last_error.c_str() : g_last_error.c_str(); }

ir_status ir_filter_create(ir_filter **out, int device) {
  if (!out) return fail(nullptr, IR_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, IR_EINVAL, "no CUDA device %d", device);
  }
  DeviceGuard g(device);
  std::unique_ptr<ir_filter> h(new ir_filter());
  h->device = device;
  IR_CUDA(nullptr, cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device));
  IR_CUDA(nullptr, cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return fail(nullptr, IR_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  }
  h->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  IR_CUDA(nullptr, cudaMalloc(&h->d_status, sizeof(unsigned)));
  IR_CUDA(nullptr, cudaMalloc(&h->d_launches, sizeof(unsigned long long)));
  IR_CUDA(nullptr, cudaMemset(h->d_status, 0, sizeof(unsigned)));
  IR_CUDA(nullptr, cudaMemset(h->d_launches, 0, sizeof(unsigned long long)));
  IR_CUDA(nullptr, cudaMalloc(&h->d_sched, 2 * sizeof(unsigned) * kSchedSlots));
  IR_CUDA(nullptr, cudaMemset(h->d_sched, 0, 2 * sizeof(unsigned) * kSchedSlots));
  for (int e = 1; e <= 2; ++e)
    for (int k = 3; k <= kMaxK; k += 2) h->cfg[e - 1][kslot(k)] = default_config(e, k);
  *out = h.release();
  return IR_OK;
}

void ir_batch_plan_destroy(ir_batch_plan *plan);

void ir_filter_destroy(ir_filter *h) {
  if (!h) return;
  DeviceGuard g(h->device);
  for (int i = 0; i < kHostStreams; ++i)
    if (h->host_streams[i]) cudaStreamSynchronize(h->host_streams[i]);
  for (ir_batch_plan *p : h->host_plans) ir_batch_plan_destroy(p);
  for (int i = 0; i < kHostStreams; ++i)
    if (h->host_streams[i]) cudaStreamDestroy(h->host_streams[i]);
  for (cudaEvent_t e : h->host_events) cudaEventDestroy(e);
  if (h->host_start) cudaEventDestroy(h->host_start);
  if (h->host_done) cudaEventDestroy(h->host_done);
  if (h->host_stage) cudaFree(h->host_stage);
  for (auto &kv : h->plans) ir_batch_plan_destroy(kv.second);
  h->plans.clear();
  if (h->scratch) cudaFree(h->scratch);
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_launches) cudaFree(h->d_launches);
  if (h->d_sched) cudaFree(h->d_sched);
  delete h;
}

ir_status ir_filter_run2(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch, int H, int W,
                         ir_dtype dtype, int k, void *cuda_stream, unsigned long long *flagged_count) {
  fnr::NvtxRange nvtx_range("ir_filter_run2");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  ir_status s = check_frame(h, in, in_pitch, out, out_pitch, H, W, dtype, k);
  if (s != IR_OK) return s;
  DeviceGuard g(h->device);
  return run_one(h, in, in_pitch, out, out_pitch, H, W, dtype, k, static_cast<cudaStream_t>(cuda_stream),
                 flagged_count);
}

ir_status ir_filter_run(ir_filter *h, void *frame, int H, int W, size_t pitch_bytes, ir_dtype dtype, int k,
                        void *cuda_stream) {
  fnr::NvtxRange nvtx_range("ir_filter_run");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (!frame) return fail(h, IR_EINVAL, "null frame pointer");
  if (H < 1 || W < 1 || !valid_dtype(dtype)) return check_frame(h, frame, pitch_bytes, frame, pitch_bytes, H, W, dtype, k);
  DeviceGuard g(h->device);
  const int es = esize_of(dtype);
  const size_t row = static_cast<size_t>(W) * es;
  const size_t spitch = (row + 255) / 256 * 256;
  ir_status s = ensure_scratch(h, spitch * static_cast<size_t>(H));
  if (s != IR_OK) return s;
  s = check_frame(h, h->scratch, spitch, frame, pitch_bytes, H, W, dtype, k);
  if (s != IR_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  IR_CUDA(h, cudaMemcpy2DAsync(h->scratch, spitch, frame, pitch_bytes, row, H, cudaMemcpyDeviceToDevice, st));
  return run_one(h, h->scratch, spitch, frame, pitch_bytes, H, W, dtype, k, st, nullptr);
}

ir_status ir_filter_median_filter(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch, int H,
                                  int W, ir_dtype dtype, int k, void *cuda_stream, unsigned long long *median_count) {
  fnr::NvtxRange nvtx_range("ir_filter_median_filter");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  ir_status s = check_frame(h, in, in_pitch, out, out_pitch, H, W, dtype, k);
  if (s != IR_OK) return s;
  DeviceGuard g(h->device);
  return run_one(h, in, in_pitch, out, out_pitch, H, W, dtype, k, static_cast<cudaStream_t>(cuda_stream),
                 median_count, kModeMedian);
}

ir_status ir_filter_run_passes(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch, int H,
                               int W, ir_dtype dtype, int k, int passes, void *cuda_stream,
                               unsigned long long *flagged_per_pass) {
  fnr::NvtxRange nvtx_range("ir_filter_run_passes");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (passes < 1 || passes > 64) return fail(h, IR_EINVAL, "passes must be in [1, 64] (got %d)", passes);
  ir_status s = check_frame(h, in, in_pitch, out, out_pitch, H, W, dtype, k);
  if (s != IR_OK) return s;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (passes == 1) return run_one(h, in, in_pitch, out, out_pitch, H, W, dtype, k, st, flagged_per_pass);
  // ping-pong between `out` and handle scratch, arranged so the last pass writes `out`
  const size_t row = static_cast<size_t>(W) * esize_of(dtype);
  const size_t spitch = (row + 255) / 256 * 256;
  s = ensure_scratch(h, spitch * static_cast<size_t>(H));
  if (s != IR_OK) return s;
  const void *src = in;
  size_t src_pitch = in_pitch;
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    void *dst = to_out ? out : h->scratch;
    const size_t dst_pitch = to_out ? out_pitch : spitch;
    s = run_one(h, src, src_pitch, dst, dst_pitch, H, W, dtype, k, st,
                flagged_per_pass ? flagged_per_pass + p : nullptr);
    if (s != IR_OK) return s;
    src = dst;
    src_pitch = dst_pitch;
  }
  return IR_OK;
}

ir_status ir_filter_sync_status(ir_filter *h) {
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  DeviceGuard g(h->device);
  IR_CUDA(h, cudaDeviceSynchronize());
  unsigned st = 0;
  IR_CUDA(h, cudaMemcpy(&st, h->d_status, sizeof st, cudaMemcpyDeviceToHost));
  IR_CUDA(h, cudaMemset(h->d_status, 0, sizeof st));
  if (st & kStatusTimeout) {
    // a kernel that gave up may not have reset its tile-order slot
    IR_CUDA(h, cudaMemset(h->d_sched, 0, 2 * sizeof(unsigned) * kSchedSlots));
    return fail(h, IR_ETIMEOUT, "a bounded device-side wait gave up");
  }
  if (st & kStatusCheck) return fail(h, IR_ECHECK, "an index or alignment check inside a kernel failed");
  return IR_OK;
}

unsigned long long ir_filter_launch_count(const ir_filter *h) {
  if (!h) return 0;
  DeviceGuard g(h->device);
  unsigned long long n = 0;
  if (cudaMemcpy(&n, h->d_launches, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

ir_status ir_filter_set_border(ir_filter *h, ir_border mode) {
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (mode != IR_BORDER_REPLICATE && mode != IR_BORDER_MIRROR && mode != IR_BORDER_ZERO)
    return fail(h, IR_EINVAL, "unknown border mode %d", static_cast<int>(mode));
  h->border = static_cast<int>(mode);
  return IR_OK;
}

ir_border ir_filter_get_border(const ir_filter *h) {
  return h ? static_cast<ir_border>(h->border) : IR_BORDER_REPLICATE;
}

ir_status ir_filter_set_strict_alignment(ir_filter *h, int on) {
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  h->strict_align = on != 0;
  return IR_OK;
}

ir_status ir_filter_set_tile_fit(ir_filter *h, int on) {
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  h->tile_fit = on != 0;
  return IR_OK;
}

ir_status ir_filter_set_detector(ir_filter *h, ir_detector detector) {
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (detector != IR_DETECT_EXTREME && detector != IR_DETECT_DIRECTIONAL)
    return fail(h, IR_EINVAL, "unknown detector %d", static_cast<int>(detector));
  h->detector = detector == IR_DETECT_DIRECTIONAL ? kModeDirectional : kModeFnr;
  return IR_OK;
}

ir_detector ir_filter_get_detector(const ir_filter *h) {
  return h && h->detector == kModeDirectional ? IR_DETECT_DIRECTIONAL : IR_DETECT_EXTREME;
}

ir_status ir_filter_get_config(ir_filter *h, ir_dtype dtype, int k, ir_kernel_config *out) {
  if (!h || !out) return fail(h, IR_EINVAL, "null argument");
  if (!valid_dtype(dtype) || !valid_k(k)) return fail(h, IR_EINVAL, "bad dtype or k");
  *out = h->cfg[esize_of(dtype) - 1][kslot(k)];
  return IR_OK;
}

ir_status ir_filter_set_config(ir_filter *h, ir_dtype dtype, int k, const ir_kernel_config *cfg) {
  if (!h || !cfg) return fail(h, IR_EINVAL, "null argument");
  if (!valid_dtype(dtype) || !valid_k(k)) return fail(h, IR_EINVAL, "bad dtype or k");
  ir_kernel_config c = *cfg;
  const int es = esize_of(dtype);
  if (c.algo == IR_ALGO_AUTO) c = default_config(es, k);
  std::string why;
  if (!config_ok(h, es, k, c, &why)) return fail(h, IR_EINVAL, "config rejected: %s", why.c_str());
  if (!get_kernel(es, k, c.algo)) return fail(h, IR_EUNSUPPORTED, "algo %d not built for k=%d", c.algo, k);
  h->cfg[es - 1][kslot(k)] = c;
  return IR_OK;
}

// ---------------------------------------------------------------------------
// batch plans
// ---------------------------------------------------------------------------
ir_status ir_batch_plan_create(ir_filter *h, const ir_frame_desc *descs, int n, ir_batch_plan **out) {
  fnr::NvtxRange nvtx_range("ir_batch_plan_create");
  if (!h || !out) return fail(h, IR_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1 || !descs) return fail(h, IR_EINVAL, "empty batch");
  for (int i = 0; i < n; ++i) {
    const ir_frame_desc &d = descs[i];
    ir_status s = check_frame(h, d.in, d.in_pitch, d.out, d.out_pitch, d.H, d.W, d.dtype, d.k);
    if (s != IR_OK) return fail(h, s, "frame %d: %s", i, h->last_error.c_str());
  }
  // outputs must not overlap any input of the batch (frames run concurrently)
  for (int i = 0; i < n; ++i) {
    const size_t orow = static_cast<size_t>(descs[i].W) * esize_of(descs[i].dtype);
    const size_t olen = (descs[i].H - 1) * descs[i].out_pitch + orow;
    for (int j = 0; j < n; ++j) {
      const size_t irow = static_cast<size_t>(descs[j].W) * esize_of(descs[j].dtype);
      const size_t ilen = (descs[j].H - 1) * descs[j].in_pitch + irow;
      if (ranges_overlap(descs[i].out, olen, descs[j].in, ilen))
        return fail(h, IR_EINVAL, "output of frame %d overlaps input of frame %d", i, j);
    }
  }
  DeviceGuard g(h->device);
  std::unique_ptr<ir_batch_plan> plan(new ir_batch_plan());
  plan->h = h;
  // group by (esize, k): one persistent launch per class
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) groups[{esize_of(descs[i].dtype), descs[i].k}].push_back(i);
  std::vector<FrameDev> host(n);
  int slot = 0;
  std::vector<std::pair<int, int>> ranges;  // (first slot, count) per class
  for (auto &kv : groups) {
    ClassLaunch cl;
    cl.esize = kv.first.first;
    cl.k = kv.first.second;
    {
      std::vector<int> Hs, Ws;
      for (int i : kv.second) {
        Hs.push_back(descs[i].H);
        Ws.push_back(descs[i].W);
      }
      cl.cfg = fit_tile(h, cl.esize, cl.k, h->cfg[cl.esize - 1][kslot(cl.k)], Hs.data(), Ws.data(),
                        static_cast<int>(Hs.size()));
    }
    int tiles = 0;
    const int first = slot;
    for (int i : kv.second) {
      const ir_frame_desc &d = descs[i];
      host_make_frame_dev(h, host[slot], d.in, d.in_pitch, d.out, d.out_pitch, d.H, d.W, cl.esize, cl.k, cl.cfg,
                     d.flagged_count);
      host[slot].tile_begin = tiles;
      tiles += host[slot].tiles_x * host[slot].tiles_y;
      ++slot;
    }
    cl.prm = FnrParams{};
    cl.prm.nframes = static_cast<int>(kv.second.size());
    cl.prm.total_tiles = tiles;
    cl.prm.tile_w = cl.cfg.tile_w;
    cl.prm.tile_h = cl.cfg.tile_h;
    cl.prm.status = h->d_status;
    cl.prm.launches = h->d_launches;
    cl.prm.mode = h->detector;
    cl.prm.border = h->border;
    ir_status s = host_prepare_class(h, cl);
    if (s != IR_OK) return s;
    plan->classes.push_back(cl);
    ranges.emplace_back(first, cl.prm.nframes);
  }
  IR_CUDA(h, cudaMalloc(&plan->d_table, sizeof(FrameDev) * n));
  IR_CUDA(h, cudaMemcpy(plan->d_table, host.data(), sizeof(FrameDev) * n, cudaMemcpyHostToDevice));
  IR_CUDA(h, cudaMalloc(&plan->d_sched, 2 * sizeof(unsigned) * plan->classes.size()));
  IR_CUDA(h, cudaMemset(plan->d_sched, 0, 2 * sizeof(unsigned) * plan->classes.size()));
  for (size_t c = 0; c < plan->classes.size(); ++c) {
    plan->classes[c].prm.table = plan->d_table + ranges[c].first;
    plan->classes[c].prm.sched = plan->d_sched + 2 * c;
  }

  // explicit graph: counter memsets first, then one kernel node per class
  IR_CUDA(h, cudaGraphCreate(&plan->graph, 0));
  std::vector<cudaGraphNode_t> memsets;
  std::vector<unsigned long long *> counters;
  for (int i = 0; i < n; ++i)
    if (descs[i].flagged_count &&
        std::find(counters.begin(), counters.end(), descs[i].flagged_count) == counters.end())
      counters.push_back(descs[i].flagged_count);
  {
    // the tile-order slots start every replay at zero (a kernel also resets
    // its slot when it ends; this covers a replay after one that gave up)
    cudaMemsetParams mp{};
    mp.dst = plan->d_sched;
    mp.elementSize = 4;
    mp.width = 2 * plan->classes.size();
    mp.height = 1;
    mp.pitch = 0;
    mp.value = 0;
    cudaGraphNode_t node;
    IR_CUDA(h, cudaGraphAddMemsetNode(&node, plan->graph, nullptr, 0, &mp));
    memsets.push_back(node);
  }
  for (unsigned long long *ctr : counters) {
    cudaMemsetParams mp{};
    mp.dst = ctr;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    mp.pitch = 0;
    mp.value = 0;
    cudaGraphNode_t node;
    IR_CUDA(h, cudaGraphAddMemsetNode(&node, plan->graph, nullptr, 0, &mp));
    memsets.push_back(node);
  }
  for (ClassLaunch &cl : plan->classes) {
    void *args[] = {&cl.prm};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(cl.fn);
    kp.gridDim = dim3(cl.grid);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = static_cast<unsigned>(cl.smem);
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaGraphNode_t node;
    IR_CUDA(h, cudaGraphAddKernelNode(&node, plan->graph, memsets.empty() ? nullptr : memsets.data(), memsets.size(),
                                      &kp));
  }
  IR_CUDA(h, cudaGraphInstantiate(&plan->exec, plan->graph, 0));
  *out = plan.release();
  return IR_OK;
}

ir_status ir_batch_plan_launch(ir_batch_plan *plan, void *cuda_stream) {
  fnr::NvtxRange nvtx_range("ir_batch_plan_launch");
  if (!plan) return fail(nullptr, IR_EINVAL, "null plan");
  DeviceGuard g(plan->h->device);
  IR_CUDA(plan->h, cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(cuda_stream)));
  return IR_OK;
}

int ir_batch_plan_kernel_count(const ir_batch_plan *plan) {
  return plan ? static_cast<int>(plan->classes.size()) : 0;
}

void ir_batch_plan_destroy(ir_batch_plan *plan) {
  if (!plan) return;
  DeviceGuard g(plan->h->device);
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->d_table) cudaFree(plan->d_table);
  if (plan->d_sched) cudaFree(plan->d_sched);
  delete plan;
}

// A plan is reused for the same descriptors under the same handle settings.
static PlanKey plan_key(const ir_filter *h, const ir_frame_desc *descs, int n) {
  PlanKey key;
  auto put = [&](const void *p, size_t len) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    key.bytes.insert(key.bytes.end(), b, b + len);
  };
  put(descs, sizeof(ir_frame_desc) * n);
  put(h->cfg, sizeof(h->cfg));
  put(&h->border, sizeof(h->border));
  put(&h->detector, sizeof(h->detector));
  put(&h->tile_fit, sizeof(h->tile_fit));
  return key;
}

ir_status ir_filter_run_batch(ir_filter *h, const ir_frame_desc *descs, int n, void *cuda_stream) {
  fnr::NvtxRange nvtx_range("ir_filter_run_batch");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (n < 1 || !descs) return fail(h, IR_EINVAL, "empty batch");
  const PlanKey key = plan_key(h, descs, n);
  auto it = h->plans.find(key);
  ir_batch_plan *plan = nullptr;
  if (it != h->plans.end()) {
    plan = it->second;
    auto pos = std::find(h->plan_order.begin(), h->plan_order.end(), key);
    if (pos != h->plan_order.end()) h->plan_order.erase(pos);
    h->plan_order.push_back(key);
  } else {
    ir_status s = ir_batch_plan_create(h, descs, n, &plan);
    if (s != IR_OK) return s;
    constexpr size_t kMaxPlans = 8;
    if (h->plans.size() >= kMaxPlans) {
      // the oldest plan may still be in flight on some stream: wait before freeing it
      DeviceGuard g(h->device);
      cudaDeviceSynchronize();
      ir_batch_plan_destroy(h->plans[h->plan_order.front()]);
      h->plans.erase(h->plan_order.front());
      h->plan_order.erase(h->plan_order.begin());
    }
    h->plans[key] = plan;
    h->plan_order.push_back(key);
  }
  return ir_batch_plan_launch(plan, cuda_stream);
}

// Copies of one chunk between host frames and their device staging: runs of
// frames that are contiguous on the host with a row pitch equal to the
// staging pitch go as one copy, the others one 2-D copy each.
static ir_status host_copies(ir_filter *h, const ir_frame_desc *d, const size_t *off, const size_t *dp, int a, int b,
                             bool to_device, cudaStream_t st) {
  int i = a;
  while (i < b) {
    const unsigned char *hp = static_cast<const unsigned char *>(to_device ? d[i].in : d[i].out);
    const size_t hpitch = to_device ? d[i].in_pitch : d[i].out_pitch;
    const size_t row = static_cast<size_t>(d[i].W) * esize_of(d[i].dtype);
    if (hpitch != dp[i]) {
      void *dev = h->host_stage + off[i];
      IR_CUDA(h, to_device ? cudaMemcpy2DAsync(dev, dp[i], hp, hpitch, row, d[i].H, cudaMemcpyHostToDevice, st)
                           : cudaMemcpy2DAsync(const_cast<unsigned char *>(hp), hpitch, dev, dp[i], row, d[i].H,
                                               cudaMemcpyDeviceToHost, st));
      ++i;
      continue;
    }
    size_t bytes = static_cast<size_t>(d[i].H) * dp[i];
    int j = i + 1;
    while (j < b) {
      const unsigned char *hq = static_cast<const unsigned char *>(to_device ? d[j].in : d[j].out);
      const size_t qpitch = to_device ? d[j].in_pitch : d[j].out_pitch;
      if (qpitch != dp[j] || hq != hp + bytes || off[j] != off[i] + bytes) break;
      bytes += static_cast<size_t>(d[j].H) * dp[j];
      ++j;
    }
    void *dev = h->host_stage + off[i];
    IR_CUDA(h, to_device ? cudaMemcpyAsync(dev, hp, bytes, cudaMemcpyHostToDevice, st)
                         : cudaMemcpyAsync(const_cast<unsigned char *>(hp), dev, bytes, cudaMemcpyDeviceToHost, st));
    i = j;
  }
  return IR_OK;
}

static ir_status host_chunk(ir_filter *h, const ir_frame_desc *descs, const ir_frame_desc *dd, const size_t *in_off,
                            const size_t *out_off, const size_t *dp, int a, int b, int c, cudaStream_t s_in,
                            cudaStream_t s_filter, cudaStream_t s_out);

ir_status ir_filter_run_host(ir_filter *h, const ir_frame_desc *descs, int n, int chunks, void *cuda_stream) {
  fnr::NvtxRange nvtx_range("ir_filter_run_host");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (n < 1 || !descs) return fail(h, IR_EINVAL, "empty batch");
  for (int i = 0; i < n; ++i) {
    const ir_frame_desc &d = descs[i];
    ir_status s = check_frame(h, d.in, d.in_pitch, d.out, d.out_pitch, d.H, d.W, d.dtype, d.k, true);
    if (s != IR_OK) return s;
  }
  DeviceGuard g(h->device);
  // staging: every input, then every output, back to back with rows padded to
  // 16 bytes (so every frame starts 16-byte aligned, as TMA needs, and frames
  // that lie back to back on the host do so here too)
  std::vector<size_t> dp(n), in_off(n), out_off(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    dp[i] = (static_cast<size_t>(descs[i].W) * esize_of(descs[i].dtype) + 15) / 16 * 16;
    in_off[i] = total;
    total += static_cast<size_t>(descs[i].H) * dp[i];
  }
  for (int i = 0; i < n; ++i) out_off[i] = in_off[i] + total;
  const size_t need = 2 * total;
  if (!h->host_start) {
    IR_CUDA(h, cudaEventCreateWithFlags(&h->host_start, cudaEventDisableTiming));
    IR_CUDA(h, cudaEventCreateWithFlags(&h->host_done, cudaEventDisableTiming));
    for (int i = 0; i < kHostStreams; ++i)
      IR_CUDA(h, cudaStreamCreateWithFlags(&h->host_streams[i], cudaStreamNonBlocking));
  }
  if (h->host_stage_bytes < need) {
    // nothing of the previous calls may still use the old staging or its plans
    for (int i = 0; i < kHostStreams; ++i) IR_CUDA(h, cudaStreamSynchronize(h->host_streams[i]));
    for (ir_batch_plan *p : h->host_plans) ir_batch_plan_destroy(p);
    h->host_plans.clear();
    h->host_keys.clear();
    if (h->host_stage) cudaFree(h->host_stage);
    h->host_stage = nullptr;
    h->host_stage_bytes = 0;
    if (cudaMalloc(&h->host_stage, need) != cudaSuccess) {
      cudaGetLastError();
      h->host_stage = nullptr;
      return fail(h, IR_ENOMEM, "cannot allocate %zu bytes of host-frame staging", need);
    }
    h->host_stage_bytes = need;
  }
  // chunks of whole frames; with four or more, the first two and the last
  // two are a quarter and a half of the others, so that the pipeline fills
  // and drains quickly (the copy-in of the first chunk and the filtering and
  // copy-out of the last are not overlapped with anything)
  const int C = std::max(1, std::min(chunks > 0 ? chunks : kHostChunks, n));
  std::vector<double> cum(C);
  {
    double sum = 0;
    for (int c = 0; c < C; ++c) {
      const int edge = std::min(c, C - 1 - c);
      sum += C < 4 ? 1.0 : (edge == 0 ? 1.0 : (edge == 1 ? 2.0 : 4.0));
      cum[c] = sum;
    }
    for (double &x : cum) x /= sum;
  }
  std::vector<int> bounds{0};
  {
    size_t acc = 0;
    for (int i = 0; i + 1 < n && static_cast<int>(bounds.size()) < C; ++i) {
      acc += static_cast<size_t>(descs[i].H) * dp[i];
      if (static_cast<double>(acc) >= cum[bounds.size() - 1] * static_cast<double>(total)) bounds.push_back(i + 1);
    }
    bounds.push_back(n);
  }
  const int used = static_cast<int>(bounds.size()) - 1;
  if (static_cast<int>(h->host_plans.size()) < used) {
    h->host_plans.resize(used, nullptr);
    h->host_keys.resize(used);
  }
  while (static_cast<int>(h->host_events.size()) < 2 * used) {
    cudaEvent_t e;
    IR_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->host_events.push_back(e);
  }
  cudaStream_t caller = static_cast<cudaStream_t>(cuda_stream);
  cudaStream_t s_in = h->host_streams[0], s_filter = h->host_streams[1], s_out = h->host_streams[2];
  // the chunks start after the caller's queued work and after this handle's
  // previous host-frame call (whose end host_done marks; waiting on it is a
  // no-op before the first call), whatever stream that call was on, since
  // they reuse its staging
  for (int i = 0; i < kHostStreams; ++i) IR_CUDA(h, cudaStreamWaitEvent(h->host_streams[i], h->host_done, 0));
  IR_CUDA(h, cudaEventRecord(h->host_start, caller));
  for (int i = 0; i < kHostStreams; ++i) IR_CUDA(h, cudaStreamWaitEvent(h->host_streams[i], h->host_start, 0));
  std::vector<ir_frame_desc> dd(n);
  for (int i = 0; i < n; ++i) {
    dd[i] = descs[i];
    dd[i].in = h->host_stage + in_off[i];
    dd[i].out = h->host_stage + out_off[i];
    dd[i].in_pitch = dd[i].out_pitch = dp[i];
  }
  // chunk c: copied in on s_in, filtered on s_filter once in, copied out on
  // s_out once filtered; each stream runs the chunks in order, so the copies
  // of chunk c + 1 overlap the filtering of chunk c and the copy-out of c - 1
  // chunks queued before an error still run; the caller's stream is joined
  // with them either way
  ir_status err = IR_OK;
  for (int c = 0; c < used && err == IR_OK; ++c) {
    err = host_chunk(h, descs, dd.data(), in_off.data(), out_off.data(), dp.data(), bounds[c], bounds[c + 1], c,
                     s_in, s_filter, s_out);
  }
  // the last copy-out follows every other step of the call
  IR_CUDA(h, cudaEventRecord(h->host_done, s_out));
  IR_CUDA(h, cudaStreamWaitEvent(caller, h->host_done, 0));
  return err;
}

// One chunk of ir_filter_run_host: copy in on s_in, filter on s_filter once
// in, copy out on s_out once filtered.
static ir_status host_chunk(ir_filter *h, const ir_frame_desc *descs, const ir_frame_desc *dd, const size_t *in_off,
                            const size_t *out_off, const size_t *dp, int a, int b, int c, cudaStream_t s_in,
                            cudaStream_t s_filter, cudaStream_t s_out) {
  cudaEvent_t ev_in = h->host_events[2 * c], ev_filtered = h->host_events[2 * c + 1];
  ir_status s = host_copies(h, descs, in_off, dp, a, b, true, s_in);
  if (s != IR_OK) return s;
  IR_CUDA(h, cudaEventRecord(ev_in, s_in));
  IR_CUDA(h, cudaStreamWaitEvent(s_filter, ev_in, 0));
  // the chunk's plan, rebuilt when its frames or the handle's settings change
  const PlanKey key = plan_key(h, dd + a, b - a);
  if (!h->host_plans[c] || !(h->host_keys[c] == key)) {
    if (h->host_plans[c]) {
      // the old plan may still run on one of the copy streams
      for (int i = 0; i < kHostStreams; ++i) IR_CUDA(h, cudaStreamSynchronize(h->host_streams[i]));
      ir_batch_plan_destroy(h->host_plans[c]);
      h->host_plans[c] = nullptr;
    }
    s = ir_batch_plan_create(h, dd + a, b - a, &h->host_plans[c]);
    if (s != IR_OK) return s;
    h->host_keys[c] = key;
  }
  s = ir_batch_plan_launch(h->host_plans[c], s_filter);
  if (s != IR_OK) return s;
  IR_CUDA(h, cudaEventRecord(ev_filtered, s_filter));
  IR_CUDA(h, cudaStreamWaitEvent(s_out, ev_filtered, 0));
  return host_copies(h, descs, out_off, dp, a, b, false, s_out);
}

// ---------------------------------------------------------------------------
// tuning
// ---------------------------------------------------------------------------
static std::vector<ir_kernel_config> candidates(int esize, int k) {
  std::vector<ir_kernel_config> out;
  auto add = [&](int algo, int tw, int th) { out.push_back(ir_kernel_config{tw, th, algo, 0}); };
  if (k == 3) {
    for (int tw : {32, 64, 128})
      for (int th : {32, 64, 128}) add(IR_ALGO_DENSE3, tw, th);
    add(IR_ALGO_NETWORK, 64, 64);
    add(IR_ALGO_BITPLANE, 64, 64);
  } else if (k <= 7) {
    for (int tw : {32, 64, 128})
      for (int th : {32, 64, 128}) add(IR_ALGO_NETWORK, tw, th);
    for (int tw : {64, 128})
      for (int th : {32, 64, 128}) add(IR_ALGO_DENSE, tw, th);
    add(IR_ALGO_BITPLANE, 64, 64);
  } else {
    for (int tw : {32, 64, 128})
      for (int th : {64, 128}) add(IR_ALGO_BITPLANE, tw, th);
    if (k <= 9)
      for (int tw : {32, 64})
        for (int th : {64, 128}) add(IR_ALGO_NETWORK, tw, th);
  }
  (void)esize;
  return out;
}

// Host-side synthetic tuning frame: smooth ramp plus 10% salt-and-pepper
// (a small LCG; only the timing depends on it).
static void tuning_frame(std::vector<unsigned char> &buf, int H, int W, int esize, size_t pitch) {
  buf.assign(pitch * H, 0);
  uint64_t s = 0x9e3779b97f4a7c15ull;
  auto next = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return static_cast<uint32_t>(s >> 33);
  };
  const uint32_t maxv = esize == 1 ? 255u : 16383u;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      uint32_t v = (static_cast<uint32_t>(x + y) * (maxv / 4)) / static_cast<uint32_t>(W + H) + maxv / 4 + (next() % 9);
      const uint32_t u = next() % 100;
      if (u < 5) v = 0;
      else if (u < 10) v = maxv;
      if (esize == 1) buf[y * pitch + x] = static_cast<unsigned char>(v);
      else std::memcpy(&buf[y * pitch + 2 * x], &v, 2);
    }
}

// Median time (ms) of `reps` launches of a batch plan of descs[0..n) under
// configuration c for its (single) class, each launch preceded by a memset of
// `flush` (flush_bytes, nullable) outside the timed events.
static ir_status time_config(ir_filter *h, const ir_frame_desc *descs, int n, int es, int k, const ir_kernel_config &c,
                             int reps, cudaStream_t st, void *flush, size_t flush_bytes, cudaEvent_t e0,
                             cudaEvent_t e1, float *ms_out) {
  const ir_kernel_config saved = h->cfg[es - 1][kslot(k)];
  h->cfg[es - 1][kslot(k)] = c;
  ir_batch_plan *plan = nullptr;
  ir_status s = ir_batch_plan_create(h, descs, n, &plan);
  h->cfg[es - 1][kslot(k)] = saved;
  if (s != IR_OK) return s;
  std::vector<float> t;
  for (int w = 0; w < 2 && s == IR_OK; ++w) s = ir_batch_plan_launch(plan, st);
  for (int r = 0; r < reps && s == IR_OK; ++r) {
    if (flush && cudaMemsetAsync(flush, r & 0xff, flush_bytes, st) != cudaSuccess) {
      s = fail(h, IR_ECUDA, "L2 flush failed");
      break;
    }
    if (cudaEventRecord(e0, st) != cudaSuccess) s = fail(h, IR_ECUDA, "cudaEventRecord failed");
    if (s == IR_OK) s = ir_batch_plan_launch(plan, st);
    if (s == IR_OK && cudaEventRecord(e1, st) != cudaSuccess) s = fail(h, IR_ECUDA, "cudaEventRecord failed");
    float ms = 0;
    if (s == IR_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      s = fail(h, IR_ECUDA, "timing a tuning launch failed");
    t.push_back(ms);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && s == IR_OK) s = fail(h, IR_ECUDA, "tuning launch failed");
  ir_batch_plan_destroy(plan);
  if (s != IR_OK) return s;
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return IR_OK;
}

// Tunes (es, k) on descs[0..n) (frames of that class only); fills *res.
static ir_status tune_class(ir_filter *h, const ir_frame_desc *descs, int n, int es, int k, int reps, cudaStream_t st,
                            ir_tune_result *res) {
  size_t bytes = 0;
  for (int i = 0; i < n; ++i) bytes += 2 * static_cast<size_t>(descs[i].H) * descs[i].W * es;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) l2 = 128 << 20;
  const size_t flush_bytes = 2 * static_cast<size_t>(l2);
  void *flush = nullptr;
  if (bytes < flush_bytes && cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, IR_ENOMEM, "cannot allocate the %zu-byte L2 flush buffer for tuning", flush_bytes);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ir_status s = IR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    s = fail(h, IR_ECUDA, "cudaEventCreate failed");
  const ir_kernel_config def = default_config(es, k);
  std::vector<ir_kernel_config> cands = candidates(es, k);
  bool has_def = false;
  for (const ir_kernel_config &c : cands)
    has_def |= c.algo == def.algo && c.tile_w == def.tile_w && c.tile_h == def.tile_h && c.ctas_per_sm == def.ctas_per_sm;
  if (!has_def) cands.insert(cands.begin(), def);
  ir_kernel_config best = def;
  float best_ms = 1e30f, def_ms = 0.f;
  int timed = 0;
  for (const ir_kernel_config &c : cands) {
    if (s != IR_OK) break;
    if (!config_ok(h, es, k, c, nullptr) || !get_kernel(es, k, c.algo)) continue;
    float ms = 0.f;
    s = time_config(h, descs, n, es, k, c, reps, st, flush, flush_bytes, e0, e1, &ms);
    if (s == IR_EUNSUPPORTED) {  // a shape that does not fit an SM: skip it
      s = IR_OK;
      continue;
    }
    if (s != IR_OK) break;
    ++timed;
    const bool is_def = c.algo == def.algo && c.tile_w == def.tile_w && c.tile_h == def.tile_h &&
                        c.ctas_per_sm == def.ctas_per_sm;
    if (is_def) def_ms = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (flush) cudaFree(flush);
  if (s != IR_OK) return s;
  if (timed == 0) return fail(h, IR_EUNSUPPORTED, "no configuration could be timed for esize=%d k=%d", es, k);
  h->cfg[es - 1][kslot(k)] = best;
  if (res) {
    res->dtype = es == 1 ? IR_U8 : IR_U16;
    res->k = k;
    res->frames = n;
    res->candidates = timed;
    res->chosen = best;
    res->chosen_ms = best_ms;
    res->defaults = def;
    res->default_ms = def_ms;
  }
  return IR_OK;
}

ir_status ir_filter_autotune_batch(ir_filter *h, const ir_frame_desc *descs, int n, int reps, void *cuda_stream,
                                   ir_tune_result *results, int max_results, int *n_results) {
  fnr::NvtxRange nvtx_range("ir_filter_autotune_batch");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (n < 1 || !descs) return fail(h, IR_EINVAL, "empty batch");
  if (reps < 0 || reps > 100000) return fail(h, IR_EINVAL, "reps must be in [0, 100000]");
  if (max_results < 0 || (max_results > 0 && !results)) return fail(h, IR_EINVAL, "bad results buffer");
  if (n_results) *n_results = 0;
  reps = std::max(reps, 20);
  for (int i = 0; i < n; ++i) {
    const ir_frame_desc &d = descs[i];
    ir_status s = check_frame(h, d.in, d.in_pitch, d.out, d.out_pitch, d.H, d.W, d.dtype, d.k);
    if (s != IR_OK) return fail(h, s, "frame %d: %s", i, h->last_error.c_str());
  }
  DeviceGuard g(h->device);
  std::map<std::pair<int, int>, std::vector<ir_frame_desc>> groups;
  for (int i = 0; i < n; ++i) {
    ir_frame_desc d = descs[i];
    d.flagged_count = nullptr;  // tuning leaves the caller's counters alone
    groups[{esize_of(d.dtype), d.k}].push_back(d);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int c = 0;
  for (auto &kv : groups) {
    ir_tune_result r{};
    ir_status s = tune_class(h, kv.second.data(), static_cast<int>(kv.second.size()), kv.first.first, kv.first.second,
                             reps, st, &r);
    if (s != IR_OK) return s;
    if (c < max_results) results[c] = r;
    ++c;
  }
  if (n_results) *n_results = c;
  return IR_OK;
}

ir_status ir_filter_autotune(ir_filter *h, ir_dtype dtype, int k, int H, int W, void *cuda_stream) {
  fnr::NvtxRange nvtx_range("ir_filter_autotune");
  if (!h) return fail(nullptr, IR_EINVAL, "null handle");
  if (!valid_dtype(dtype) || !valid_k(k) || H < 1 || W < 1) return fail(h, IR_EINVAL, "bad tuning arguments");
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int es = esize_of(dtype);
  const size_t pitch = (static_cast<size_t>(W) * es + 255) / 256 * 256;
  std::vector<unsigned char> hbuf;
  tuning_frame(hbuf, H, W, es, pitch);
  void *din = nullptr, *dout = nullptr;
  if (cudaMalloc(&din, pitch * H) != cudaSuccess || cudaMalloc(&dout, pitch * H) != cudaSuccess) {
    cudaGetLastError();
    if (din) cudaFree(din);
    return fail(h, IR_ENOMEM, "cannot allocate tuning frames");
  }
  ir_status s = IR_OK;
  if (cudaMemcpy(din, hbuf.data(), pitch * H, cudaMemcpyHostToDevice) != cudaSuccess)
    s = fail(h, IR_ECUDA, "tuning setup failed");
  if (s == IR_OK) {
    ir_frame_desc d{};
    d.in = din;
    d.out = dout;
    d.H = H;
    d.W = W;
    d.in_pitch = d.out_pitch = pitch;
    d.dtype = dtype;
    d.k = k;
    d.flagged_count = nullptr;
    s = tune_class(h, &d, 1, es, k, 20, st, nullptr);
  }
  cudaFree(din);
  cudaFree(dout);
  return s;
}

}  // extern "C"
