// Host-side helpers shared by the library's translation units (not part of
// the C ABI): one launch of a (pixel type, k) class and the frame
// descriptors it reads.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "fnr_params.h"
#include "ir_filter.h"

namespace fnr {

// An NVTX range for the lifetime of the object: the library's calls show up
// by name on a profiler's timeline (a no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct ClassLaunch {
  int esize = 0, k = 0;
  ir_kernel_config cfg{};
  const void *fn = nullptr;
  int grid = 0, smem = 0;
  FnrParams prm{};
};

// Record an error on the handle (and the thread's last error); returns s.
ir_status host_fail(ir_filter *h, ir_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
// Fill a frame descriptor: geometry, tensor maps when the frame is TMA-addressable.
void host_make_frame_dev(ir_filter *h, FrameDev &f, const void *in, size_t in_pitch, void *out, size_t out_pitch,
                         int H, int W, int esize, int k, const ir_kernel_config &c, unsigned long long *flagged);
// Resolve the kernel, set its shared-memory attribute, size the persistent grid
// (cl.prm.total_tiles must be set).
ir_status host_prepare_class(ir_filter *h, ClassLaunch &cl);
// Launch on st; a launch without a tile-order slot takes the handle's next one.
ir_status host_launch_class(ir_filter *h, ClassLaunch &cl, cudaStream_t st);
// Tile-order slots of the handle for launches outside a batch plan.
constexpr unsigned kSchedSlots = 256;
unsigned *host_sched_slot(ir_filter *h);
ir_kernel_config host_config(const ir_filter *h, int esize, int k);
int host_device(const ir_filter *h);
int host_sm_count(const ir_filter *h);
unsigned *host_status_word(const ir_filter *h);
unsigned long long *host_launch_counter(const ir_filter *h);

}  // namespace fnr
