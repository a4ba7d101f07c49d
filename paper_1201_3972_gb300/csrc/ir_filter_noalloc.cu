// ir_filter_run_noalloc: in-place FNR filtering for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA-graph
// capture or a real-time frame loop where an allocation would stall or is
// forbidden, plug-ins whose host application owns every device allocation,
// and embedded pipelines with a fixed memory budget set at start-up. The
// regular in-place entry point (ir_filter_run) needs a handle, and both the
// handle and its scratch buffer are allocated with cudaMalloc. This entry
// point needs neither: it stages the input copy in a file-scope device array
// that is part of the loaded library image.
//
// Limits and behaviour:
//   * the staged copy of one frame (H rows of W * bytes-per-pixel, each row
//     rounded up to 16 bytes) must fit in kStaticScratchBytes (8 MiB: e.g.
//     2048 x 2048 u16, 4096 x 2048 u8); larger frames are rejected with
//     IR_EINVAL and nothing is launched;
//   * every GPU that loads the library holds the 8 MiB array until the
//     process exits;
//   * all calls share the one array per device, which keeps the last call's
//     contents: calls that overlap on the GPU (different streams, or host
//     threads, without ordering between them) race and give wrong results;
//   * the first call on each device does a one-time set-up (looks up the
//     array's device address, sets kernel attributes); make that first call
//     before any stream capture;
//   * nothing here calls cudaMalloc, cudaFree or any allocating library
//     routine; the window configuration is the library's default per (pixel
//     type, k) (default_tile in fnr_params.h, the table a handle starts
//     from), not a tuned one;
//   * a kernel whose bounded wait gave up ORs a flag into a second static
//     word, which ir_filter_noalloc_status reads and clears.
#include "ir_filter.h"

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "fnr_params.h"

namespace fnr {
const void *get_kernel_k3(int esize, int k, int algo);
const void *get_kernel_k5_7(int esize, int k, int algo);
const void *get_kernel_k9_11(int esize, int k, int algo);
const void *get_kernel_k13_15(int esize, int k, int algo);
const void *get_kernel_k17_21(int esize, int k, int algo);
}  // namespace fnr

namespace {

using namespace fnr;

constexpr size_t kStaticScratchBytes = 8u << 20;
constexpr int kMaxDevices = 64;

// The staging copy of the input frame, and a status word the kernels report
// bounded-wait timeouts into. In host code these names are host-side stand-ins
// for the device symbols: only the addresses from cudaGetSymbolAddress below
// may be handed to a kernel.
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];
static __device__ __align__(256) unsigned int g_status;

struct DeviceState {
  bool ready = false;
  unsigned char *scratch = nullptr;
  unsigned int *status = nullptr;
  int sm_count = 0;
  int max_smem = 0;
};

std::mutex g_mu;
DeviceState g_dev[kMaxDevices];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
char g_err[256];

ir_status err(ir_status s, const char *msg, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess) snprintf(g_err, sizeof g_err, "%s: %s", msg, cudaGetErrorString(e));
  else snprintf(g_err, sizeof g_err, "%s", msg);
  fprintf(stderr, "ir_filter_run_noalloc: %s\n", g_err);
  return s;
}

const void *kernel_for_k(int esize, int k, int algo) {
  if (k == 3) return get_kernel_k3(esize, k, algo);
  if (k <= 7) return get_kernel_k5_7(esize, k, algo);
  if (k <= 11) return get_kernel_k9_11(esize, k, algo);
  if (k <= 15) return get_kernel_k13_15(esize, k, algo);
  return get_kernel_k17_21(esize, k, algo);
}

// The library's default strategy and tile (the table handles start from).
void static_config(int esize, int k, int &algo, int &tw, int &th) {
  const DefaultTile d = default_tile(esize, k);
  algo = d.algo;
  tw = d.tile_w;
  th = d.tile_h;
}

// One-time set-up of `dev` (the current device). Called under g_mu.
ir_status setup_device(int dev, DeviceState &st) {
  if (st.ready) return IR_OK;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&st.scratch), g_scratch);
  if (e != cudaSuccess || st.scratch == nullptr) return err(IR_ECUDA, "cudaGetSymbolAddress(scratch) failed", e);
  e = cudaGetSymbolAddress(reinterpret_cast<void **>(&st.status), g_status);
  if (e != cudaSuccess || st.status == nullptr) return err(IR_ECUDA, "cudaGetSymbolAddress(status) failed", e);
  if ((e = cudaDeviceGetAttribute(&st.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return err(IR_ECUDA, "cudaDeviceGetAttribute failed", e);
  if ((e = cudaDeviceGetAttribute(&st.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return err(IR_ECUDA, "cudaDeviceGetAttribute failed", e);
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return err(IR_ECUDA, "cuTensorMapEncodeTiled is not available", e);
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  for (int k = 3; k <= kMaxK; k += 2) {
    for (int es = 1; es <= 2; ++es) {
      int algo, tw, th;
      static_config(es, k, algo, tw, th);
      const void *fn = kernel_for_k(es, k, algo);
      if (!fn) continue;
      if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, st.max_smem)) != cudaSuccess)
        return err(IR_ECUDA, "cudaFuncSetAttribute failed", e);
    }
  }
  st.ready = true;
  return IR_OK;
}

bool encode(CUtensorMap *map, int esize, const void *base, int H, int W, size_t pitch, int bw, int bh) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(bw), static_cast<cuuint32_t>(bh)};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(map, esize == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" ir_status ir_filter_run_noalloc(void *frame, int H, int W, size_t pitch_bytes, ir_dtype dtype, int k,
                                           void *cuda_stream) {
  if (!frame) return err(IR_EINVAL, "null frame pointer");
  if (H < 1 || W < 1) return err(IR_EINVAL, "H and W must be >= 1");
  if (dtype != IR_U8 && dtype != IR_U16 && dtype != IR_U14) return err(IR_EINVAL, "unknown dtype");
  if (k < 3 || k > kMaxK || !(k & 1)) return err(IR_EINVAL, "k must be odd and in [3, 21]");
  const int esize = dtype == IR_U8 ? 1 : 2;
  const size_t row = static_cast<size_t>(W) * esize;
  if (pitch_bytes < row) return err(IR_EINVAL, "pitch smaller than W * bytes per pixel");
  const size_t spitch = (row + 15) / 16 * 16;
  if (static_cast<unsigned long long>(H) * spitch > kStaticScratchBytes)
    return err(IR_EINVAL, "frame does not fit the 8 MiB static scratch of ir_filter_run_noalloc");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(IR_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= kMaxDevices) return err(IR_EUNSUPPORTED, "device index out of range");
  DeviceState st;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    ir_status s = setup_device(dev, g_dev[dev]);
    if (s != IR_OK) return s;
    st = g_dev[dev];
  }

  int algo, tw, th;
  static_config(esize, k, algo, tw, th);
  const void *fn = kernel_for_k(esize, k, algo);
  if (!fn) return err(IR_EUNSUPPORTED, "no kernel built for this window");
  const Layout L = make_layout(esize, k, algo, th, tw);

  FnrParams prm{};
  FrameDev &f = prm.single;
  f.in = st.scratch;
  f.out = static_cast<unsigned char *>(frame);
  f.in_pitch = static_cast<long long>(spitch);
  f.out_pitch = static_cast<long long>(pitch_bytes);
  f.H = H;
  f.W = W;
  f.tiles_x = (W + tw - 1) / tw;
  f.tiles_y = (H + th - 1) / th;
  f.tile_begin = 0;
  f.flagged = nullptr;
  f.flags = 0;
  if (encode(&f.tin, esize, st.scratch, H, W, spitch, L.bw, L.bh)) f.flags |= kFrameTmaIn;
  const bool out_ok = (reinterpret_cast<uintptr_t>(frame) % 16) == 0 && pitch_bytes % 16 == 0;
  if (out_ok && encode(&f.tout, esize, frame, H, W, pitch_bytes, tw, th / kConsumerWarps)) f.flags |= kFrameTmaOut;
  prm.table = nullptr;
  prm.nframes = 1;
  prm.total_tiles = f.tiles_x * f.tiles_y;
  prm.tile_w = tw;
  prm.tile_h = th;
  prm.status = st.status;
  prm.launches = nullptr;

  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, L.total);
  if (e != cudaSuccess || per_sm < 1) return err(IR_ECUDA, "occupancy query failed", e);
  int grid = per_sm * st.sm_count;
  if (grid > prm.total_tiles) grid = prm.total_tiles;

  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  e = cudaMemcpy2DAsync(st.scratch, spitch, frame, pitch_bytes, row, H, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return err(IR_ECUDA, "staging copy failed", e);
  void *args[] = {&prm};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, L.total, s);
  if (e != cudaSuccess) return err(IR_ECUDA, "kernel launch failed", e);
  return IR_OK;
}

// The status word of the allocation-free path on the current device: its
// kernels OR a flag into it when a bounded wait gives up (they then leave part
// of the frame unfiltered). This waits for the device, reads the word into a
// host variable and clears it; like the entry point it allocates nothing. A
// device on which ir_filter_run_noalloc never ran has nothing to report.
extern "C" ir_status ir_filter_noalloc_status(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(IR_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= kMaxDevices) return err(IR_EUNSUPPORTED, "device index out of range");
  unsigned int *status = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[dev].ready) return IR_OK;
    status = g_dev[dev].status;
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return err(IR_ECUDA, "cudaDeviceSynchronize failed", e);
  unsigned int word = 0;
  if ((e = cudaMemcpy(&word, status, sizeof word, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return err(IR_ECUDA, "reading the status word failed", e);
  if ((e = cudaMemset(status, 0, sizeof word)) != cudaSuccess) return err(IR_ECUDA, "clearing the status word failed", e);
  if (word & kStatusTimeout) return err(IR_ETIMEOUT, "a bounded device-side wait gave up");
  if (word & kStatusCheck) return err(IR_ECHECK, "an index or alignment check inside a kernel failed");
  return IR_OK;
}
