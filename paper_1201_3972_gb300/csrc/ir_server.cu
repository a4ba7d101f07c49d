// Continuous-batching server for many video streams (ir_server_* in
// include/ir_filter.h).
//
// Request life cycle, per stream slot:
//   FREE --submit--> QUEUED --batcher--> RUNNING --poller--> DONE --release--> FREE
// The batcher thread waits until requests are queued and an execution lane
// (a CUDA stream with its own pinned/device descriptor table) is free, takes
// every queued request up to max_batch, copies the frames host->device on
// that lane, uploads the batch's frame table and launches one persistent
// kernel per (pixel type, k) class. Requests that arrive meanwhile queue for
// the next lane, so consecutive batches overlap on the device. The poller
// thread watches each lane's completion event and publishes completions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fnr_host.h"
#include "fnr_params.h"
#include "ir_filter.h"

using namespace fnr;

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

enum SlotState { SLOT_FREE = 0, SLOT_QUEUED = 1, SLOT_RUNNING = 2, SLOT_DONE = 3 };

struct Slot {
  unsigned char *d_in = nullptr;
  unsigned char *d_out = nullptr;
  FrameDev proto{};              // descriptor of this slot (tensor maps of d_in/d_out)
  SlotState state = SLOT_FREE;
  const void *host = nullptr;
  size_t host_pitch = 0;
  unsigned long long tag = 0;
  double t_submit = 0;
};

struct Stream {
  bool open = false;
  int H = 0, W = 0, k = 0, esize = 0;
  ir_dtype dtype = IR_U8;
  size_t pitch = 0;
  std::vector<Slot> slots;
};

struct Req {
  int stream, slot;
};

// Everything the batcher needs about one request, copied under the lock so
// the launch itself touches no shared state.
struct Job {
  Req req;
  int esize, k, H, W;
  size_t pitch;
  unsigned char *d_in;
  const void *host;
  size_t host_pitch;
  FrameDev proto;
};

// A prepared (pixel type, k) class: kernel, shared memory, largest grid.
struct ClassInfo {
  const void *fn = nullptr;
  int smem = 0;
  int max_grid = 0;
  FnrParams prm{};  // tile size, status word, launch counter
};

struct Lane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  FrameDev *h_table = nullptr;   // pinned
  FrameDev *d_table = nullptr;
  bool busy = false;      // owns a batch (set by the batcher, cleared by the poller)
  bool launched = false;  // its completion event is recorded for that batch
  std::vector<Req> reqs;
  std::vector<Job> jobs;
  std::map<std::pair<int, int>, ClassInfo> classes;  // snapshot for this batch
  double t_launch = 0;
  ir_status status = IR_OK;
};

}  // namespace

struct ir_server {
  ir_filter *h = nullptr;
  ir_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work;   // batcher: work queued or a lane freed
  std::condition_variable cv_idle;   // waiters: something completed
  std::vector<Stream> streams;
  std::deque<Req> queue;
  std::vector<Lane> lanes;
  std::deque<ir_completion> completions;
  std::map<std::pair<int, int>, ClassInfo> classes;  // prepared per (esize, k) at stream open
  ir_server_stats stats{};
  unsigned long long outstanding = 0;  // submitted and not yet completed
  bool stop = false;
  std::thread batcher, poller;
};

namespace {

ir_status make_lane(ir_server *s, Lane &L) {
  if (cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&L.h_table), sizeof(FrameDev) * s->cfg.max_batch) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void **>(&L.d_table), sizeof(FrameDev) * s->cfg.max_batch) != cudaSuccess) {
    cudaGetLastError();
    return host_fail(s->h, IR_ECUDA, "server lane set-up failed");
  }
  return IR_OK;
}

// Launch one batch on lane L (batcher thread, no lock held): reads only the
// lane's own snapshot.
ir_status launch_batch(ir_server *s, Lane &L) {
  NvtxRange nvtx_range("ir_server batch");
  ir_filter *h = s->h;
  const int n = static_cast<int>(L.jobs.size());
  for (const Job &j : L.jobs) {
    if (cudaMemcpy2DAsync(j.d_in, j.pitch, j.host, j.host_pitch, static_cast<size_t>(j.W) * j.esize, j.H,
                          cudaMemcpyHostToDevice, L.stream) != cudaSuccess) {
      cudaGetLastError();
      return host_fail(h, IR_ECUDA, "server: frame upload failed");
    }
  }
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) groups[{L.jobs[i].esize, L.jobs[i].k}].push_back(i);
  struct Launch {
    const ClassInfo *ci;
    int first, count, tiles;
  };
  std::vector<Launch> launches;
  int slot = 0;
  for (auto &kv : groups) {
    int tiles = 0;
    const int first = slot;
    for (int i : kv.second) {
      FrameDev &f = L.h_table[slot++];
      f = L.jobs[i].proto;
      f.tile_begin = tiles;
      tiles += f.tiles_x * f.tiles_y;
    }
    launches.push_back(Launch{&L.classes.at(kv.first), first, static_cast<int>(kv.second.size()), tiles});
  }
  if (cudaMemcpyAsync(L.d_table, L.h_table, sizeof(FrameDev) * n, cudaMemcpyHostToDevice, L.stream) != cudaSuccess) {
    cudaGetLastError();
    return host_fail(h, IR_ECUDA, "server: table upload failed");
  }
  for (const Launch &lc : launches) {
    FnrParams prm = lc.ci->prm;
    prm.table = L.d_table + lc.first;
    prm.nframes = lc.count;
    prm.total_tiles = lc.tiles;
    prm.sched = host_sched_slot(h);
    const int grid = std::max(1, std::min(lc.tiles, lc.ci->max_grid));
    void *args[] = {&prm};
    if (cudaLaunchKernel(lc.ci->fn, dim3(grid), dim3(kThreads), args, lc.ci->smem, L.stream) != cudaSuccess) {
      cudaGetLastError();
      return host_fail(h, IR_ECUDA, "server: kernel launch failed");
    }
  }
  if (cudaEventRecord(L.done, L.stream) != cudaSuccess) {
    cudaGetLastError();
    return host_fail(h, IR_ECUDA, "server: event record failed");
  }
  return IR_OK;
}

void batcher_main(ir_server *s) {
  cudaSetDevice(host_device(s->h));
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    Lane *lane = nullptr;
    s->cv_work.wait(lk, [&] {
      if (s->stop) return true;
      if (s->queue.empty()) return false;
      for (Lane &L : s->lanes)
        if (!L.busy) return true;
      return false;
    });
    if (s->stop && s->queue.empty()) break;
    for (Lane &L : s->lanes)
      if (!L.busy) {
        lane = &L;
        break;
      }
    if (!lane) continue;
    lane->reqs.clear();
    lane->jobs.clear();
    lane->classes.clear();
    while (!s->queue.empty() && static_cast<int>(lane->reqs.size()) < s->cfg.max_batch) {
      Req r = s->queue.front();
      s->queue.pop_front();
      Stream &st = s->streams[r.stream];
      Slot &sl = st.slots[r.slot];
      sl.state = SLOT_RUNNING;
      lane->reqs.push_back(r);
      lane->jobs.push_back(Job{r, st.esize, st.k, st.H, st.W, st.pitch, sl.d_in, sl.host, sl.host_pitch, sl.proto});
      const auto key = std::make_pair(st.esize, st.k);
      if (!lane->classes.count(key)) lane->classes[key] = s->classes.at(key);
    }
    lane->busy = true;
    lane->launched = false;
    int inflight = 0;
    for (Lane &L : s->lanes) inflight += L.busy ? 1 : 0;
    s->stats.max_inflight = std::max(s->stats.max_inflight, inflight);
    s->stats.batches++;
    s->stats.frames_in_batches += lane->reqs.size();
    lk.unlock();
    lane->t_launch = now_s();
    lane->status = launch_batch(s, *lane);
    if (lane->status != IR_OK) cudaEventRecord(lane->done, lane->stream);  // report the batch as finished
    lk.lock();
    lane->launched = true;
  }
}

void poller_main(ir_server *s) {
  cudaSetDevice(host_device(s->h));
  for (;;) {
    bool any = false, busy = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (Lane &L : s->lanes) {
        if (!L.busy) continue;
        busy = true;
        if (!L.launched) continue;  // the batcher is still issuing it
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        const double t = now_s();
        ir_status st = L.status;
        if (q != cudaSuccess) {
          cudaGetLastError();
          st = IR_ECUDA;
        }
        for (const Req &r : L.reqs) {
          Slot &sl = s->streams[r.stream].slots[r.slot];
          sl.state = SLOT_DONE;
          ir_completion c{};
          c.stream_id = r.stream;
          c.slot = r.slot;
          c.tag = sl.tag;
          c.t_submit = sl.t_submit;
          c.t_launch = L.t_launch;
          c.t_done = t;
          c.batch_frames = static_cast<int>(L.reqs.size());
          c.status = st;
          s->completions.push_back(c);
          s->stats.completed++;
          s->outstanding--;
        }
        L.reqs.clear();
        L.busy = false;
        any = true;
      }
      if (any) {
        s->cv_work.notify_all();
        s->cv_idle.notify_all();
      }
      if (s->stop && !busy && s->queue.empty()) break;
    }
    if (!any) std::this_thread::sleep_for(std::chrono::microseconds(std::max(1, s->cfg.poll_us)));
  }
}

ir_status stream_ok(ir_server *s, int id) {
  if (id < 0 || id >= static_cast<int>(s->streams.size()) || !s->streams[id].open)
    return host_fail(s->h, IR_EINVAL, "no open stream %d", id);
  return IR_OK;
}

}  // namespace

extern "C" {

double ir_server_clock(void) { return now_s(); }

ir_status ir_server_create(int device, const ir_server_config *cfg, ir_server **out) {
  if (!out) return IR_EINVAL;
  *out = nullptr;
  ir_server_config c{};
  c.max_streams = 256;
  c.ring_depth = 8;
  c.max_batch = 256;
  c.exec_streams = 3;
  c.hbm_reserve_bytes = static_cast<size_t>(1) << 30;
  c.poll_us = 20;
  if (cfg) {
    if (cfg->max_streams > 0) c.max_streams = cfg->max_streams;
    if (cfg->ring_depth > 0) c.ring_depth = cfg->ring_depth;
    if (cfg->max_batch > 0) c.max_batch = cfg->max_batch;
    if (cfg->exec_streams > 0) c.exec_streams = cfg->exec_streams;
    c.hbm_reserve_bytes = cfg->hbm_reserve_bytes;
    if (cfg->poll_us > 0) c.poll_us = cfg->poll_us;
  }
  ir_filter *h = nullptr;
  ir_status st = ir_filter_create(&h, device);
  if (st != IR_OK) return st;
  ir_server *s = new ir_server();
  s->h = h;
  s->cfg = c;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  s->lanes.resize(c.exec_streams);
  for (Lane &L : s->lanes) {
    st = make_lane(s, L);
    if (st != IR_OK) break;
  }
  cudaSetDevice(prev);
  if (st != IR_OK) {
    ir_server_destroy(s);
    return st;
  }
  s->batcher = std::thread(batcher_main, s);
  s->poller = std::thread(poller_main, s);
  *out = s;
  return IR_OK;
}

void ir_server_destroy(ir_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->batcher.joinable()) s->batcher.join();
  if (s->poller.joinable()) s->poller.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(host_device(s->h));
  for (Lane &L : s->lanes) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.done) cudaEventDestroy(L.done);
    if (L.stream) cudaStreamDestroy(L.stream);
    if (L.h_table) cudaFreeHost(L.h_table);
    if (L.d_table) cudaFree(L.d_table);
  }
  for (Stream &st : s->streams)
    for (Slot &sl : st.slots) {
      if (sl.d_in) cudaFree(sl.d_in);
      if (sl.d_out) cudaFree(sl.d_out);
    }
  cudaSetDevice(prev);
  ir_filter_destroy(s->h);
  delete s;
}

ir_filter *ir_server_filter(ir_server *s) { return s ? s->h : nullptr; }

ir_status ir_server_open_stream(ir_server *s, int H, int W, ir_dtype dtype, int k, int *stream_id) {
  if (!s || !stream_id) return IR_EINVAL;
  *stream_id = -1;
  if (H < 1 || W < 1 || (dtype != IR_U8 && dtype != IR_U16 && dtype != IR_U14) || k < 3 || k > kMaxK || !(k & 1))
    return host_fail(s->h, IR_EINVAL, "bad stream geometry or window");
  std::lock_guard<std::mutex> lk(s->mu);
  int open = 0;
  for (const Stream &st : s->streams) open += st.open ? 1 : 0;
  if (open >= s->cfg.max_streams) return host_fail(s->h, IR_EBUSY, "max_streams (%d) are open", s->cfg.max_streams);
  const int esize = dtype == IR_U8 ? 1 : 2;
  const size_t pitch = (static_cast<size_t>(W) * esize + 255) / 256 * 256;
  const size_t need = static_cast<size_t>(s->cfg.ring_depth) * 2 * pitch * H;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(host_device(s->h));
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    cudaSetDevice(prev);
    return host_fail(s->h, IR_ECUDA, "cudaMemGetInfo failed");
  }
  if (free_b < need || free_b - need < s->cfg.hbm_reserve_bytes) {
    cudaSetDevice(prev);
    return host_fail(s->h, IR_ENOMEM, "admission refused: %zu bytes needed, %zu free, %zu reserved", need, free_b,
                     s->cfg.hbm_reserve_bytes);
  }
  Stream st;
  st.open = true;
  st.H = H;
  st.W = W;
  st.k = k;
  st.esize = esize;
  st.dtype = dtype;
  st.pitch = pitch;
  st.slots.resize(s->cfg.ring_depth);
  const ir_kernel_config cfg = host_config(s->h, esize, k);
  ir_status result = IR_OK;
  for (Slot &sl : st.slots) {
    if (cudaMalloc(reinterpret_cast<void **>(&sl.d_in), pitch * H) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&sl.d_out), pitch * H) != cudaSuccess) {
      cudaGetLastError();
      result = host_fail(s->h, IR_ENOMEM, "stream buffer allocation failed");
      break;
    }
    host_make_frame_dev(s->h, sl.proto, sl.d_in, pitch, sl.d_out, pitch, H, W, esize, k, cfg, nullptr);
  }
  auto key = std::make_pair(esize, k);
  if (result == IR_OK && !s->classes.count(key)) {
    // resolve the kernel, its shared-memory attribute and occupancy once,
    // here under the lock; batches then launch it directly
    ClassLaunch cl;
    cl.esize = esize;
    cl.k = k;
    cl.cfg = cfg;
    cl.prm = FnrParams{};
    cl.prm.tile_w = cfg.tile_w;
    cl.prm.tile_h = cfg.tile_h;
    cl.prm.status = host_status_word(s->h);
    cl.prm.launches = host_launch_counter(s->h);
    cl.prm.total_tiles = 1 << 30;
    result = host_prepare_class(s->h, cl);
    if (result == IR_OK) {
      ClassInfo ci;
      ci.fn = cl.fn;
      ci.smem = cl.smem;
      ci.max_grid = cl.grid;
      ci.prm = cl.prm;
      s->classes[key] = ci;
    }
  }
  if (result != IR_OK) {
    for (Slot &sl : st.slots) {
      if (sl.d_in) cudaFree(sl.d_in);
      if (sl.d_out) cudaFree(sl.d_out);
    }
    cudaSetDevice(prev);
    return result;
  }
  cudaSetDevice(prev);
  int id = -1;
  for (size_t i = 0; i < s->streams.size(); ++i)
    if (!s->streams[i].open) {
      id = static_cast<int>(i);
      break;
    }
  if (id < 0) {
    id = static_cast<int>(s->streams.size());
    s->streams.push_back(Stream());
  }
  s->streams[id] = std::move(st);
  s->stats.open_streams = open + 1;
  s->stats.device_bytes += need;
  *stream_id = id;
  return IR_OK;
}

ir_status ir_server_close_stream(ir_server *s, int id) {
  if (!s) return IR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  ir_status st = stream_ok(s, id);
  if (st != IR_OK) return st;
  Stream &S = s->streams[id];
  for (const Slot &sl : S.slots)
    if (sl.state == SLOT_QUEUED || sl.state == SLOT_RUNNING)
      return host_fail(s->h, IR_EBUSY, "stream %d has frames in flight", id);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(host_device(s->h));
  for (Slot &sl : S.slots) {
    cudaFree(sl.d_in);
    cudaFree(sl.d_out);
  }
  cudaSetDevice(prev);
  s->stats.device_bytes -= static_cast<size_t>(S.slots.size()) * 2 * S.pitch * S.H;
  s->stats.open_streams--;
  S = Stream();
  return IR_OK;
}

ir_status ir_server_submit(ir_server *s, int id, const void *host_frame, size_t host_pitch, unsigned long long tag,
                           int *slot) {
  if (!s || !host_frame) return IR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  ir_status st = stream_ok(s, id);
  if (st != IR_OK) return st;
  Stream &S = s->streams[id];
  if (host_pitch < static_cast<size_t>(S.W) * S.esize) return host_fail(s->h, IR_EINVAL, "host pitch too small");
  int free_slot = -1;
  for (size_t i = 0; i < S.slots.size(); ++i)
    if (S.slots[i].state == SLOT_FREE) {
      free_slot = static_cast<int>(i);
      break;
    }
  if (free_slot < 0) {
    s->stats.rejected_busy++;
    return IR_EBUSY;
  }
  Slot &sl = S.slots[free_slot];
  sl.state = SLOT_QUEUED;
  sl.host = host_frame;
  sl.host_pitch = host_pitch;
  sl.tag = tag;
  sl.t_submit = now_s();
  s->queue.push_back(Req{id, free_slot});
  s->stats.submitted++;
  s->outstanding++;
  if (slot) *slot = free_slot;
  lk.unlock();
  s->cv_work.notify_one();
  return IR_OK;
}

int ir_server_poll(ir_server *s, ir_completion *out, int max) {
  if (!s || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int n = 0;
  while (n < max && !s->completions.empty()) {
    out[n++] = s->completions.front();
    s->completions.pop_front();
  }
  return n;
}

ir_status ir_server_wait_idle(ir_server *s, double timeout_s) {
  if (!s) return IR_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_idle.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&] { return s->outstanding == 0; });
  return ok ? IR_OK : IR_ETIMEOUT;
}

ir_status ir_server_output(ir_server *s, int id, int slot, const void **dev_out, size_t *pitch) {
  if (!s || !dev_out || !pitch) return IR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  ir_status st = stream_ok(s, id);
  if (st != IR_OK) return st;
  Stream &S = s->streams[id];
  if (slot < 0 || slot >= static_cast<int>(S.slots.size()) || S.slots[slot].state != SLOT_DONE)
    return host_fail(s->h, IR_EINVAL, "slot %d of stream %d holds no completed frame", slot, id);
  *dev_out = S.slots[slot].d_out;
  *pitch = S.pitch;
  return IR_OK;
}

ir_status ir_server_read(ir_server *s, int id, int slot, void *host_dst, size_t host_pitch) {
  if (!s) return IR_EINVAL;
  const void *d = nullptr;
  size_t pitch = 0, row = 0;
  int H = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ir_status st = stream_ok(s, id);
    if (st != IR_OK) return st;
    const Stream &S = s->streams[id];
    if (slot < 0 || slot >= static_cast<int>(S.slots.size()) || S.slots[slot].state != SLOT_DONE)
      return host_fail(s->h, IR_EINVAL, "slot %d of stream %d holds no completed frame", slot, id);
    d = S.slots[slot].d_out;
    pitch = S.pitch;
    row = static_cast<size_t>(S.W) * S.esize;
    H = S.H;
  }
  if (!host_dst || host_pitch < row) return host_fail(s->h, IR_EINVAL, "bad host buffer");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(host_device(s->h));
  const cudaError_t e = cudaMemcpy2D(host_dst, host_pitch, d, pitch, row, H, cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return host_fail(s->h, IR_ECUDA, "read failed: %s", cudaGetErrorString(e));
  return IR_OK;
}

ir_status ir_server_release(ir_server *s, int id, int slot) {
  if (!s) return IR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  ir_status st = stream_ok(s, id);
  if (st != IR_OK) return st;
  Stream &S = s->streams[id];
  if (slot < 0 || slot >= static_cast<int>(S.slots.size()) || S.slots[slot].state != SLOT_DONE)
    return host_fail(s->h, IR_EINVAL, "slot %d of stream %d is not completed", slot, id);
  S.slots[slot].state = SLOT_FREE;
  S.slots[slot].host = nullptr;
  return IR_OK;
}

ir_status ir_server_get_stats(ir_server *s, ir_server_stats *out) {
  if (!s || !out) return IR_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return IR_OK;
}

ir_status ir_server_drive(ir_server *s, const int *ids, const void *const *frames, const size_t *pitches, int n,
                          double seconds, int inflight, int plain, ir_drive_result *out) {
  if (!s || !ids || !frames || !pitches || n < 1 || !out || inflight < 1 || seconds <= 0) return IR_EINVAL;
  std::memset(out, 0, sizeof *out);
  std::vector<int> H(n), W(n), es(n), k(n);
  std::vector<ir_dtype> dt(n);
  std::vector<unsigned char *> d_in(n), d_out(n);
  std::vector<size_t> dpitch(n);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < n; ++i) {
      ir_status st = stream_ok(s, ids[i]);
      if (st != IR_OK) return st;
      const Stream &S = s->streams[ids[i]];
      H[i] = S.H;
      W[i] = S.W;
      es[i] = S.esize;
      k[i] = S.k;
      dt[i] = S.dtype;
      d_in[i] = S.slots[0].d_in;
      d_out[i] = S.slots[0].d_out;
      dpitch[i] = S.pitch;
    }
  }
  double px = 0;
  std::vector<double> lat;
  const double t0 = now_s();
  if (plain) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(host_device(s->h));
    cudaStream_t st = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      cudaSetDevice(prev);
      return host_fail(s->h, IR_ECUDA, "drive: stream set-up failed");
    }
    ir_status result = IR_OK;
    // rounds of one frame per stream; at most two rounds queued on the GPU
    for (int round = 0; now_s() - t0 < seconds && result == IR_OK; ++round) {
      cudaEvent_t e = ev[round & 1];
      if (round >= 2) cudaEventSynchronize(e);
      for (int i = 0; i < n && result == IR_OK; ++i) {
        if (cudaMemcpy2DAsync(d_in[i], dpitch[i], frames[i], pitches[i], static_cast<size_t>(W[i]) * es[i], H[i],
                              cudaMemcpyHostToDevice, st) != cudaSuccess) {
          cudaGetLastError();
          result = host_fail(s->h, IR_ECUDA, "drive: copy failed");
          break;
        }
        result = ir_filter_run2(s->h, d_in[i], dpitch[i], d_out[i], dpitch[i], H[i], W[i], dt[i], k[i], st, nullptr);
        px += static_cast<double>(H[i]) * W[i];
        out->frames++;
      }
      cudaEventRecord(e, st);
    }
    cudaStreamSynchronize(st);
    out->seconds = now_s() - t0;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaStreamDestroy(st);
    cudaSetDevice(prev);
    out->megapixels = px / 1e6;
    return result;
  }
  std::vector<int> pending(n, inflight);  // submissions owed per stream
  std::vector<ir_completion> buf(1024);
  unsigned long long outstanding = 0;
  for (;;) {
    const bool running = now_s() - t0 < seconds;
    if (running)
      for (int i = 0; i < n; ++i)
        while (pending[i] > 0) {
          int slot = -1;
          const ir_status st = ir_server_submit(s, ids[i], frames[i], pitches[i], static_cast<unsigned long long>(i), &slot);
          if (st == IR_EBUSY) break;
          if (st != IR_OK) return st;
          pending[i]--;
          outstanding++;
        }
    const int m = ir_server_poll(s, buf.data(), static_cast<int>(buf.size()));
    for (int c = 0; c < m; ++c) {
      const ir_completion &cp = buf[c];
      const int i = static_cast<int>(cp.tag);
      lat.push_back((cp.t_done - cp.t_submit) * 1e3);
      px += static_cast<double>(H[i]) * W[i];
      out->frames++;
      outstanding--;
      ir_server_release(s, cp.stream_id, cp.slot);
      pending[i]++;
    }
    if (!running && outstanding == 0) break;
    if (m == 0) std::this_thread::sleep_for(std::chrono::microseconds(10));
    if (now_s() - t0 > seconds + 30.0) return host_fail(s->h, IR_ETIMEOUT, "drive: frames did not complete");
  }
  out->seconds = now_s() - t0;
  out->megapixels = px / 1e6;
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) { return lat[std::min(lat.size() - 1, static_cast<size_t>(q * (lat.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = lat.back();
  }
  return IR_OK;
}

}  // extern "C"
