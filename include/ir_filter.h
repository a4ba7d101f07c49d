/*
 * ir_filter.h - C ABI of the GB300 FNR impulse filter for infrared frames.
 *
 * The filter is the "fast noise reduction" (FNR) method of arXiv 1201.3972:
 *   - S_xy is the k x k window around pixel p(x, y), centre included (Sec. 3.3);
 *   - g_max = max S_xy, g_min = min S_xy (Eq. 3a, 3b);
 *   - p(x, y) is noisy iff g(x, y) == g_min or g(x, y) == g_max (Sec. 3.3,
 *     step 2) - there is no threshold or other preset parameter;
 *   - a noisy pixel is replaced by the median g_m of S_xy and every other
 *     pixel is left unchanged (Sec. 3.4).
 * Readings this library fixes where the paper is silent: the border is
 * replicated by default (every pixel gets a full k x k window; mirror and
 * zero are options), every window reads the unfiltered input (one
 * non-recursive pass), ties with g_min/g_max flag, and k is odd so g_m is the
 * element of rank (k*k-1)/2 of the sorted window. A second detector after
 * Fig. 1 (the line test of ir_filter_set_detector) is an option.
 * Results are integer-exact: every entry point returns the same bytes as a
 * plain CPU evaluation of the rules above.
 *
 * Memory: every frame pointer is a CUDA DEVICE pointer to a row-pitched
 * image (pitch in bytes, rows contiguous), except for ir_filter_run_host and
 * ir_server_submit/read, which take host memory. The caller owns all frame
 * memory.
 * A handle owns its scratch memory (grown on demand), cached tensor maps,
 * its tuning table and a device status word. Handles are not thread-safe:
 * use one per host thread (several may share a device).
 *
 * Streams: `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream). Calls are asynchronous: argument errors are returned at
 * once, launch errors are returned by the call, and results (and device-side
 * errors) are valid after the stream is synchronised.
 *
 * Errors never abort the process: every entry point returns an ir_status and
 * ir_filter_last_error() gives a one-line description of the last failure.
 */
#ifndef IR_FILTER_H
#define IR_FILTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IR_OK = 0,
  IR_EINVAL = 1,        /* bad argument (k even/out of range, H or W < 1, NULL, pitch too small, overlap) */
  IR_EALIGN = 2,        /* strict alignment only (ir_filter_set_strict_alignment): a frame's base or pitch is not
                           16-byte aligned; otherwise such frames take a plain-load path and are no error */
  IR_ENOMEM = 3,        /* device scratch could not be grown / admission refused for lack of memory */
  IR_ECUDA = 4,         /* a CUDA runtime call failed (see ir_filter_last_error) */
  IR_ETIMEOUT = 5,      /* a bounded device-side wait gave up (reported by ir_filter_sync_status) */
  IR_EBUSY = 6,         /* no free slot right now (server admission) */
  IR_EUNSUPPORTED = 7,  /* configuration not built into this library */
  IR_ECHECK = 8         /* debug builds (FNR_DEBUG_CHECKS) only: an index or alignment check inside a kernel
                           failed and the access was skipped (reported by ir_filter_sync_status) */
} ir_status;

/* Pixel types. IR_U14 is 16-bit storage whose values the caller promises are
 * <= 16383 (14-bit sensors); the result is exact for any 16-bit value anyway. */
typedef enum { IR_U8 = 0, IR_U16 = 1, IR_U14 = 2 } ir_dtype;

/* Median-selection strategies (all give identical results; they differ in speed). */
typedef enum {
  IR_ALGO_AUTO = 0,          /* tuned choice for (dtype, k) */
  IR_ALGO_DENSE3 = 1,        /* k = 3 only: median for every pixel with shared column sorts, packed 16x2 */
  IR_ALGO_NETWORK = 2,       /* k <= 9: flagged pixels compacted, register selection network each */
  IR_ALGO_BITPLANE = 3,      /* any k: flagged pixels compacted, bit-plane radix select (MSB first) */
  IR_ALGO_DENSE = 4          /* k = 5 and 7: median for every pixel from separable networks (columns sorted
                                once for two rows, merges shared by neighbouring windows), packed 16x2 */
} ir_algo;

/* How windows read pixels outside the frame. The paper does not say; every
 * pixel, border included, gets a full k x k window (Table 1 evaluates all
 * 364 x 244 pixels), so the default replicates the nearest edge pixel. */
typedef enum {
  IR_BORDER_REPLICATE = 0,   /* clamp to the nearest edge pixel (default) */
  IR_BORDER_MIRROR = 1,      /* reflect about the edge pixel: d c b | a b c d | c b a */
  IR_BORDER_ZERO = 2         /* outside pixels read as 0 */
} ir_border;

/* Which pixels are noisy (Sec. 3.3). Both replace a noisy pixel by the median
 * of its k x k window (Sec. 3.4) and leave every other pixel bit-identical. */
typedef enum {
  IR_DETECT_EXTREME = 0,     /* Eq. 3a/3b: g(x, y) equals the window's min or max (default) */
  IR_DETECT_DIRECTIONAL = 1  /* Fig. 1: along none of the four lines through p(x, y) (horizontal,
                                vertical, two diagonals) does g(x, y) lie strictly between its two
                                neighbours at distance one; the lines read the border like the window */
} ir_detector;

/* Kernel configuration for one (dtype, k) class. tile_w, tile_h: output tile
 * in pixels (multiples of 8; tile_w + halo <= 256 pixels). ctas_per_sm: 0 = as
 * many as fit. A launch whose frames give fewer tiles than the GPU has SMs
 * (a small single frame, a small batch class) runs the same strategy with
 * its tile halved, height first, while the tiles do not cover the SMs and the
 * tile keeps at least 4096 pixels (unless ir_filter_set_tile_fit turns this
 * off). */
typedef struct {
  int tile_w;
  int tile_h;
  int algo;          /* ir_algo */
  int ctas_per_sm;
} ir_kernel_config;

typedef struct ir_filter ir_filter;

/* Create a handle on CUDA device `device` (made current for the call; the
 * calling thread's current device is restored afterwards). *out is NULL on
 * failure. Largest supported window: 21. */
ir_status ir_filter_create(ir_filter **out, int device);

/* Destroy a handle and free everything it owns (NULL-safe). Pending work on
 * streams that used it must be complete. */
void ir_filter_destroy(ir_filter *h);

/* Filter one frame IN PLACE (the input is first copied into handle scratch,
 * then filtered back into `frame`). H, W >= 1; pitch >= W * bytes per pixel;
 * k odd in [3, 21] (k may exceed H or W: the border is replicated).
 * Uses scratch memory of H * W * bytes-per-pixel. */
ir_status ir_filter_run(ir_filter *h, void *frame, int H, int W, size_t pitch_bytes,
                        ir_dtype dtype, int k, void *cuda_stream);

/* Filter one frame out of place. `in` and `out` must not overlap. If
 * `flagged_count` is not NULL it must be a DEVICE pointer; it is set to the
 * number of noisy pixels (the number of medians taken, Table 1's "sort
 * times"). No scratch memory is used. */
ir_status ir_filter_run2(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch,
                         int H, int W, ir_dtype dtype, int k, void *cuda_stream,
                         unsigned long long *flagged_count);

/* The standard median filter the paper compares FNR against (Sec. 2, Table 1:
 * "MF"): every pixel is replaced by the median of its k x k window (replicate
 * border), no detection step. Arguments as ir_filter_run2; `median_count`
 * (nullable device pointer) is set to H * W, the number of medians taken. */
ir_status ir_filter_median_filter(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch,
                                  int H, int W, ir_dtype dtype, int k, void *cuda_stream,
                                  unsigned long long *median_count);

/* Iterative FNR (Figs. 3-6 apply FNR twice): `passes` non-recursive passes,
 * each reading the previous pass's output, the last one written to `out`.
 * passes in [1, 64]; more than one pass uses handle scratch of H rows of
 * W * bytes per pixel. `flagged_per_pass` (nullable) is a DEVICE array of
 * `passes` counters, entry p set to the number of noisy pixels of pass p. */
ir_status ir_filter_run_passes(ir_filter *h, const void *in, size_t in_pitch, void *out, size_t out_pitch,
                               int H, int W, ir_dtype dtype, int k, int passes, void *cuda_stream,
                               unsigned long long *flagged_per_pass);

/* One frame of a batch: same meaning as the arguments of ir_filter_run2. */
typedef struct {
  const void *in;
  void *out;
  int H, W;
  size_t in_pitch, out_pitch;
  ir_dtype dtype;
  int k;
  unsigned long long *flagged_count;  /* nullable, device pointer */
} ir_frame_desc;

/* Filter n frames of mixed sizes, dtypes and windows in one CUDA-graph launch:
 * one persistent kernel per (dtype, k) class present, the classes running
 * concurrently as branches of the graph. The graph is built on first use of
 * a descriptor set and replayed while the same set (same pointers, shapes,
 * windows) is submitted again. Outputs must not overlap any input. */
ir_status ir_filter_run_batch(ir_filter *h, const ir_frame_desc *descs, int n, void *cuda_stream);

/* Frames in host memory: descs[i].in and descs[i].out are HOST addresses (the
 * same descriptors as ir_filter_run_batch otherwise; flagged_count, if set, is
 * a DEVICE address). Every frame is copied to device staging memory owned by
 * the handle (rows padded to 16 bytes), the frames are filtered as batches,
 * and the results are copied back. The frames go in `chunks` groups of whole
 * frames (0 = 16; at most n; with four or more the two first and two last
 * are a quarter and a half the size of the others, so the pipeline fills and
 * drains quickly) through the handle's three
 * streams (copies in, filtering, copies out), so that one chunk's copies
 * overlap another's filtering and the two copy directions overlap each other; frames that lie back to back in host
 * memory with rows of the padded size move as one copy. In place (in == out,
 * same pitch) is allowed here; other overlaps are IR_EINVAL. Asynchronous on
 * cuda_stream: the chunks start after the work already queued there, and the
 * outputs are valid once cuda_stream is synchronised. Host memory should be
 * pinned (cudaHostAlloc / cudaHostRegister) for full speed and asynchrony;
 * pageable memory works, but its copies are staged by the driver and partly
 * synchronous. The staging grows on demand (the handle then waits for its own
 * earlier host-frame work): IR_ENOMEM if it cannot. Other errors as
 * ir_filter_run_batch; strict alignment does not apply (the staging is
 * aligned). Descriptors are checked before anything is queued; after a later
 * error (a failed copy or plan), the chunks already queued still run and
 * cuda_stream is joined with them. Calls on one handle must not overlap from
 * several host threads. */
ir_status ir_filter_run_host(ir_filter *h, const ir_frame_desc *descs, int n, int chunks, void *cuda_stream);

/* Explicit batch plans: validate and upload a descriptor set once, capture
 * its graph, then launch it any number of times. */
typedef struct ir_batch_plan ir_batch_plan;
ir_status ir_batch_plan_create(ir_filter *h, const ir_frame_desc *descs, int n, ir_batch_plan **out);
ir_status ir_batch_plan_launch(ir_batch_plan *plan, void *cuda_stream);
/* Number of kernel launches one replay of the plan performs. */
int ir_batch_plan_kernel_count(const ir_batch_plan *plan);
void ir_batch_plan_destroy(ir_batch_plan *plan);

/* In-place filtering that allocates nothing (no handle, no cudaMalloc, no
 * cudaFree, no allocating library call). The paper has no counterpart: this
 * is a deployment entry point for callers that cannot allocate device memory,
 * e.g. code inside a graph capture or a real-time frame loop, plug-ins whose
 * host application owns all device memory, or pipelines with a fixed memory
 * budget. Same arguments and result as ir_filter_run, with the library's
 * default (untuned) strategy and tile per (dtype, k), the table a new handle
 * starts from. The input copy is staged in a fixed 8 MiB
 * device array inside the library (every GPU that loads the library holds it
 * until exit): a frame needing more than 8 MiB (H rows of W * bytes per pixel,
 * each row rounded up to 16 bytes) is rejected with IR_EINVAL. All calls
 * share that array, so calls that overlap on the GPU race; order them on one
 * stream. The first call on each device does a one-time set-up and should be
 * made before any stream capture. Errors: IR_EINVAL (arguments, size);
 * IR_EUNSUPPORTED (the current device's index is 64 or more, or no kernel is
 * built for the window); IR_ECUDA (the one-time set-up or a launch failed).
 * A bounded device-side wait that gives up is not reported by this call: it
 * sets a status word that ir_filter_noalloc_status reads. */
ir_status ir_filter_run_noalloc(void *frame, int H, int W, size_t pitch_bytes, ir_dtype dtype, int k,
                                void *cuda_stream);

/* Read and clear the status word of ir_filter_run_noalloc on the current
 * device, allocating nothing: waits for the device, then IR_ETIMEOUT if a
 * bounded wait inside one of its kernels gave up since the last read (that
 * call's frame is then partly unfiltered), IR_ECHECK in a debug build if an
 * internal check failed, IR_OK otherwise (also when ir_filter_run_noalloc
 * never ran on this device). IR_ECUDA if the synchronisation or the read
 * fails. The paper has no counterpart. */
ir_status ir_filter_noalloc_status(void);

/* Read and clear the handle's device status word (synchronises the device).
 * IR_ETIMEOUT if a bounded wait inside a kernel gave up since the last call;
 * the handle's tile-order counters are then zeroed as well, since a kernel
 * that gave up may have left its counter mid-count. In a debug build,
 * IR_ECHECK if a kernel's internal index or alignment check failed. */
ir_status ir_filter_sync_status(ir_filter *h);

/* Border reading for the handle's later calls (single frames, passes, median
 * filter, batch plans created afterwards). IR_EINVAL for an unknown mode.
 * ir_filter_run_noalloc and the server always replicate. */
ir_status ir_filter_set_border(ir_filter *h, ir_border mode);
ir_border ir_filter_get_border(const ir_filter *h);

/* Strict alignment for the handle's later calls (on != 0): every frame's base
 * address and row pitch, input and output, must be multiples of 16 bytes,
 * which the TMA tile copies need, or the call returns IR_EALIGN and launches
 * nothing (a batch plan is refused when any frame fails). Off (the default),
 * such frames are staged and written with plain loads and stores instead.
 * Frames whose row (W * bytes per pixel) is not a multiple of 16 bytes are
 * accepted either way (their right-edge tiles use plain stores). */
ir_status ir_filter_set_strict_alignment(ir_filter *h, int on);

/* Tile fitting for the handle's later calls and plans (on != 0, the
 * default): a launch whose frames give fewer tiles than the GPU has SMs
 * shrinks its tile as described at ir_kernel_config. Off, every launch uses
 * the table's tile as it is (e.g. to time or test one exact shape). */
ir_status ir_filter_set_tile_fit(ir_filter *h, int on);

/* Noise detector for the handle's later calls, like ir_filter_set_border
 * (single frames, in place, passes, batch plans created afterwards; tuning
 * times the detector in use). flagged_count counts the pixels the detector
 * flags. The median filter flags every pixel whatever the detector.
 * IR_EINVAL for an unknown detector. ir_filter_run_noalloc and the server
 * always use IR_DETECT_EXTREME. */
ir_status ir_filter_set_detector(ir_filter *h, ir_detector detector);
ir_detector ir_filter_get_detector(const ir_filter *h);

/* Tuning. ir_filter_autotune times every built candidate for (dtype, k) on a
 * synthetic H x W frame (smooth ramp, 10% salt-and-pepper) on `cuda_stream`,
 * 20 launches each with L2 flushed before every launch, and keeps the fastest
 * by median time; synchronous. The table is per handle. get/set read or
 * override one entry. ir_filter_autotune_batch below tunes on real frames. */
ir_status ir_filter_autotune(ir_filter *h, ir_dtype dtype, int k, int H, int W, void *cuda_stream);
ir_status ir_filter_get_config(ir_filter *h, ir_dtype dtype, int k, ir_kernel_config *out);

/* One (pixel size, k) class tuned by ir_filter_autotune_batch. */
typedef struct {
  int dtype;                  /* IR_U8 or IR_U16 (the pixel size; IR_U14 shares IR_U16's entry) */
  int k;
  int frames;                 /* frames of the batch in this class */
  int candidates;             /* configurations timed */
  ir_kernel_config chosen;    /* the fastest, now the handle's entry for the class */
  float chosen_ms;            /* median time of one launch of the class's frames with it */
  ir_kernel_config defaults;  /* the library's default configuration for the class */
  float default_ms;           /* its median time, measured the same way */
} ir_tune_result;

/* Tune the handle's table on the caller's own frames: for every (pixel size,
 * k) class present in descs (the same descriptors as ir_filter_run_batch),
 * time every built (strategy, tile) candidate, default included, on a batch
 * plan of exactly that class's frames: `reps` timed launches each (at least
 * 20; 0 = 20) after two warm-up launches, CUDA events on cuda_stream, with L2
 * flushed before every timed launch (a device memset over twice the L2 size,
 * in memory allocated for the call and freed before it returns) unless the
 * class's frames are larger than that already; the fastest by median time
 * becomes the handle's entry. The frames are filtered as a side effect (the
 * outputs hold the filtered frames afterwards; flagged counters are not
 * touched). Synchronous: returns when tuning is done. results (nullable):
 * up to max_results entries, one per class, *n_results (nullable) set to the
 * number of classes. Errors: as ir_batch_plan_create; IR_ENOMEM if the flush
 * buffer cannot be allocated. The table can then be saved and reused by
 * later handles on the same GPU model (ir_filter_get_config / set_config). */
ir_status ir_filter_autotune_batch(ir_filter *h, const ir_frame_desc *descs, int n, int reps, void *cuda_stream,
                                   ir_tune_result *results, int max_results, int *n_results);
ir_status ir_filter_set_config(ir_filter *h, ir_dtype dtype, int k, const ir_kernel_config *cfg);

/* Number of FNR kernel launches this handle has issued (graph replays count
 * each kernel node). */
unsigned long long ir_filter_launch_count(const ir_filter *h);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of frames from many video streams.
 *
 * A server owns its own handle on `device`, device-resident buffers per open
 * stream (a ring of `ring_depth` input/output slots, admitted against free
 * HBM), and two host threads: a batcher that takes every queued request
 * (up to max_batch) as soon as one of `exec_streams` execution lanes is free,
 * copies the frames host->device and launches one persistent kernel per
 * (pixel type, k) class on that lane; and a completion poller that
 * timestamps finished batches. Requests that arrive while earlier batches
 * run join the next batch on another lane, so their work overlaps on the
 * device. Results stay in the stream's device slot until released.
 * The paper's claim this serves: real-time video processing (Sec. 5).
 * ---------------------------------------------------------------------- */
typedef struct ir_server ir_server;

typedef struct {
  int max_streams;           /* default 256 */
  int ring_depth;            /* slots per stream, default 8 */
  int max_batch;             /* frames per batch launch, default 256 */
  int exec_streams;          /* batches in flight at once, default 3 */
  size_t hbm_reserve_bytes;  /* free device memory admission leaves untouched, default 1 GiB */
  int poll_us;               /* completion poll period in microseconds, default 20 */
} ir_server_config;

typedef struct {
  int stream_id;
  int slot;
  unsigned long long tag;
  double t_submit;           /* ir_server_clock() seconds at ir_server_submit */
  double t_launch;           /* when its batch was launched */
  double t_done;             /* when the batch's completion was observed */
  int batch_frames;          /* frames in the batch it ran in */
  int status;                /* ir_status of the batch */
} ir_completion;

typedef struct {
  unsigned long long submitted, completed, rejected_busy, batches, frames_in_batches;
  int open_streams;
  int max_inflight;          /* most batches seen in flight at once */
  size_t device_bytes;       /* device memory held for stream buffers */
} ir_server_stats;

/* cfg may be NULL (defaults). */
ir_status ir_server_create(int device, const ir_server_config *cfg, ir_server **out);
/* Waits for in-flight batches, stops the threads, frees everything (NULL-safe). */
void ir_server_destroy(ir_server *srv);
/* The server's handle, for ir_filter_set_config / ir_filter_autotune before
 * the first stream is opened. Do not call it concurrently with the server. */
ir_filter *ir_server_filter(ir_server *srv);
/* Admit a stream of H x W frames: allocates ring_depth input and output
 * slots; IR_ENOMEM if free device memory minus hbm_reserve_bytes cannot hold
 * them, IR_EBUSY if max_streams are open. */
ir_status ir_server_open_stream(ir_server *srv, int H, int W, ir_dtype dtype, int k, int *stream_id);
/* IR_EBUSY while any of its slots is queued or running. */
ir_status ir_server_close_stream(ir_server *srv, int stream_id);
/* Queue one frame (host memory, row pitch host_pitch bytes; pinned memory
 * gives an asynchronous copy). The frame is read when its batch launches and
 * must stay valid until its completion is reported. *slot receives the slot
 * index. IR_EBUSY when every slot of the stream is queued, running or holds
 * an unreleased result. */
ir_status ir_server_submit(ir_server *srv, int stream_id, const void *host_frame, size_t host_pitch,
                           unsigned long long tag, int *slot);
/* Copy up to max completions reported since the last poll; returns the count. */
int ir_server_poll(ir_server *srv, ir_completion *out, int max);
/* Block until every submitted frame has completed or timeout_s passes (IR_ETIMEOUT). */
ir_status ir_server_wait_idle(ir_server *srv, double timeout_s);
/* Device address and pitch of a completed slot's output. */
ir_status ir_server_output(ir_server *srv, int stream_id, int slot, const void **dev_out, size_t *pitch);
/* Copy a completed slot's output to host memory (synchronous). */
ir_status ir_server_read(ir_server *srv, int stream_id, int slot, void *host_dst, size_t host_pitch);
/* Return a completed slot to the stream's free pool. */
ir_status ir_server_release(ir_server *srv, int stream_id, int slot);
ir_status ir_server_get_stats(ir_server *srv, ir_server_stats *out);
/* Seconds on the monotonic clock the server stamps requests with. */
double ir_server_clock(void);

/* Closed-loop load driver (benchmarking). For `seconds`, stream
 * stream_ids[i] keeps `inflight` copies of host_frames[i] (pitch
 * host_pitches[i]) queued or running: every completion is released and the
 * frame resubmitted at once, all from the calling thread. plain = 0 drives the
 * server (batched, overlapped lanes); plain = 1 sends the same traffic
 * round-robin through the plain path instead (per frame: one host->device copy
 * and one ir_filter_run2 launch on one CUDA stream, into the stream's first
 * slot), with no batching. The server must have no other traffic meanwhile. */
typedef struct {
  unsigned long long frames;
  double megapixels;
  double seconds;
  double p50_ms, p99_ms, max_ms;   /* submit -> completion (served mode only) */
} ir_drive_result;
ir_status ir_server_drive(ir_server *srv, const int *stream_ids, const void *const *host_frames,
                          const size_t *host_pitches, int n, double seconds, int inflight, int plain,
                          ir_drive_result *out);

const char *ir_status_string(ir_status s);
/* Last error message of this handle ("" if none). NULL handle: last global error. */
const char *ir_filter_last_error(const ir_filter *h);

/* Library version, e.g. "0.1.0". */
const char *ir_filter_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IR_FILTER_H */
