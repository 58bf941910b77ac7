/*
 * mb.h -- C ABI of the GB300 escape-time (Mandelbrot) renderer.
 *
 * The library computes, for every pixel (i, j) of an m x n image, the Boolean
 * escape-time count of Sec. I of "Efficient Generation of Mandelbrot Set using
 * Message Passing Interface" (Eq. 1: f(z) = z^2 + c iterated from z = 0;
 * Eq. 2: I_{i,j} = Iteration_{i,j}): the number of z-updates made before the
 * first iterate with |z|^2 > R^2, or iterMax if there is none.  Every count is
 * bit-identical to a plain IEEE binary64 evaluation in this order:
 *     zr2 = zr*zr; zi2 = zi*zi; if (zr2 + zi2 > R2) stop;
 *     zi = (2*zr)*zi + ci; zr = (zr2 - zi2) + cr;
 * with the pixel map (the Cx / Cy arrays of Sec. III-A)
 *     c_re(j) = xmin + (j*(xmax - xmin))/n,  c_im(i) = ymax - (i*(ymax - ymin))/m,
 * each operation rounded to nearest-even on its own (no fused multiply-add).
 *
 * Conventions shared by every entry point:
 *  - Return value: MB_OK (0) or one of the MB_E* codes below; mb_strerror()
 *    names them.  Arguments are validated before anything is launched; an
 *    invalid call changes no memory.
 *  - Pointers documented as "device" must point to memory of the current CUDA
 *    device; "host" pointers to ordinary (or pinned) host memory.  The library
 *    never frees memory it did not allocate.
 *  - Launches are asynchronous on the stream given in mb_opts (NULL = the
 *    legacy default stream); results are valid once that stream is synchronised.
 *  - Temporary device memory the library needs (the Cx/Cy arrays, work
 *    counters) comes from opts->workspace when given, else from
 *    cudaMallocAsync/cudaFreeAsync on the same stream.
 *  - Counts are uint32, row-major, out[i*n + j]; row 0 is the top (c_im = ymax).
 */
#ifndef MB_H
#define MB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MB_OK 0
#define MB_EINVAL 1      /* bad argument: zero size, non-finite or empty window, R2 <= 0, NULL output */
#define MB_ENOMEM 2      /* device or host allocation failed, or a memory budget would be exceeded */
#define MB_ECUDA 3       /* a CUDA runtime call failed */
#define MB_ETIMEDOUT 4   /* a bounded wait ran out */
#define MB_EBUSY 5       /* a server queue is full */
#define MB_ENOTFOUND 6   /* unknown request id */
#define MB_EDEVICE 7     /* a kernel reported an internal error in its status word */
#define MB_ECANCELED 8   /* a queued server request was cancelled by mb_serve_destroy */

/* Complex window: c_re spans [xmin, xmax), c_im spans (ymin, ymax]. */
typedef struct {
  double xmin, xmax, ymin, ymax;
} mb_window;

/* Row / tile schedulers: the paper's three partition schemes (Sec. III) run as
 * on-device schedulers.  A "worker" is one CTA; its warps share the worker's
 * pixels and refill a lane as soon as that lane's pixel finishes. */
typedef enum {
  MB_SCHED_NAIVE = 0,        /* Sec. III-A: CTA b of G owns rows [b*(m/G), (b+1)*(m/G)), the last CTA also the m mod G rest */
  MB_SCHED_ALTERNATING = 1,  /* Sec. III-C: CTA b owns rows b, b+G, b+2G, ... */
  MB_SCHED_FCFS_ROWS = 2,    /* Sec. III-B: persistent CTAs take the next row from a global atomic counter */
  MB_SCHED_FCFS_TILES = 3,   /* as FCFS_ROWS, with tile x tile blocks in raster order as work items */
  MB_SCHED_FCFS_ITEMS = 4    /* as FCFS_TILES, over a caller-given device list of mb_item (e.g. longest-first) */
} mb_sched;

/* Arithmetic of the escape step (mb_opts.precision).  Only MB_PREC_FP64 is the
 * paper's method and bit-identical to the binary64 evaluation above.  The other
 * two trade count accuracy for throughput; each is defined by its exact
 * operation sequence, with the same per-iteration order:
 *  - MB_PREC_FP32: c_re, c_im and R2 are the binary64 values rounded once to
 *    binary32 (nearest-even); every operation is then one binary32 operation.
 *  - MB_PREC_DFLOAT: double-float.  A value is an unevaluated sum h + l of two
 *    binary32 numbers; a binary64 x becomes h = RN32(x), l = RN32(x - h).
 *    Sums use the accurate double-word sum and products the double-word product
 *    with three fused multiply-adds (Joldes, Muller, Popescu, ACM TOMS 44(2),
 *    2017: relative errors below 3u^2 and 4u^2, u = 2^-24).  2*x doubles both
 *    parts, and the escape test compares (h, l) pairs lexicographically.
 * Their counts differ from binary64 on some pixels near the set's boundary
 * (binary32 on a few per mille of a full view at iterMax 1000, double-float on a
 * few per hundred thousand).  The difference grows with zoom depth and
 * iterMax, and binary32 stops resolving pixels once the pixel spacing nears
 * 2^-24 |c|.  The paper has no counterpart: it computes in double precision. */
typedef enum {
  MB_PREC_FP64 = 0,
  MB_PREC_FP32 = 1,
  MB_PREC_DFLOAT = 2
} mb_precision;

/* One work item of MB_SCHED_FCFS_ITEMS: rows [row0, row0+rows) of tile `tile`
 * (tiles numbered row-major, tile x tile pixels, cut at the image edge). */
typedef struct {
  uint32_t tile;
  uint16_t row0;
  uint16_t rows;
} mb_item;

/* Per-CTA trace record written when opts->trace is given (globaltimer ns). */
typedef struct {
  uint64_t start_ns;
  uint64_t end_ns;
  uint32_t smid;
  uint32_t items;    /* work items (rows / tiles / list entries) this CTA took */
} mb_cta_trace;

typedef struct {
  int sched;                 /* mb_sched; default MB_SCHED_FCFS_TILES */
  uint32_t tile;             /* tile side, a power of two in [8, 256]; 0 = 64 */
  uint32_t grid;             /* CTAs; 0 = SM count x resident CTAs per SM */
  uint32_t block;            /* threads per CTA, multiple of 32 in [32, 512]; 0 = 256 */
  uint32_t unroll;           /* escape steps between lane refills: 4, 8 or 16; 0 = 4.  The cycle-detection and
                                reduced-precision kernels use 16 when 16 is asked, else 8; a binary32 step is
                                four iterations */
  void* stream;              /* cudaStream_t; NULL = legacy default stream */
  const mb_item* items;      /* device; required for MB_SCHED_FCFS_ITEMS */
  uint32_t n_items;
  uint64_t* tile_totals;     /* device, optional: += sum of counts per tile (row-major tiles); caller zeroes it */
  mb_cta_trace* trace;       /* device, optional: one record per CTA, for CTAs below trace_len */
  uint32_t trace_len;        /* records available at `trace` */
  uint32_t* status;          /* device, optional: kernels OR error bits into it (0 = fine; 1 = a bounded wait
                                ran out, 2 = an item outside its tile, 4 = max_seconds reached) */
  void* workspace;           /* device, optional: temporary memory, >= mb_render_workspace_size() bytes, 256-byte aligned */
  size_t workspace_bytes;
  uint32_t split;            /* mb_render_learned: split divisor S of the order-and-split rule; 0 = 4 */
  uint32_t round_tiles;      /* mb_serve_create: tiles per round; 0 = 16 x grid */
  uint32_t max_seconds;      /* 0 = no limit; else each CTA of the main render stops after running this long
                                and ORs 4 into *status (a guard for interactive use; the image is then incomplete) */
  uint32_t fp64_products;    /* 1 = form the three products of a step on the FP64 pipe (MB_SCHED_FCFS_TILES
                                only; a measured baseline), 0 = exactly on the integer pipes (default) */
  void* ev_start;            /* cudaEvent_t, optional: recorded on the stream right before the main render kernel */
  void* ev_stop;             /* cudaEvent_t, optional: recorded right after it (to time that kernel alone) */
  uint32_t precision;        /* mb_precision; 0 = MB_PREC_FP64.  Other values are accepted by mb_render (any
                                scheduler; not with fp64_products), mb_render_batch, mb_batch_plan_create and
                                mb_serve_create; every other entry point returns MB_EINVAL for them */
  uint32_t cycle_check;      /* 1 = stop a pixel as soon as its binary64 state (zr, zi) at the start of a block of
                                steps equals, bit for bit, its state at an earlier block start (kept at blocks
                                1, 2, 4, 8, ...): the orbit is then periodic and never escapes, so the count is
                                iterMax.  Counts are identical to cycle_check = 0; fewer steps run.  Not in the
                                paper.  Honoured by mb_render, mb_render_batch, mb_batch_plan_create and
                                mb_serve_create (binary64 only, not with fp64_products); the other entry points
                                return MB_EINVAL for it; 0 = off */
  uint32_t learned_order;    /* mb_render_batch / mb_batch_plan_create (mb_serve_create: see there): 1 = queue the (view, tile) items of all
                                views longest-first by predicted cost, with heavy tiles split into row strips (the
                                order-and-split rule of mb_order_split over the batch's tiles, split divisor
                                `split`, on the costs after the neighbourhood guard of mb_guard_costs within
                                each view), instead of decreasing iterMax then raster order; the costs come from a
                                probe of every view (8 x 8 samples per tile, tile >= 16) run once when the plan is
                                built, and from `model` (or, when model is NULL, the probe-sum estimate).
                                Scheduling only: the counts are unchanged.  0 = off */
  const float* model;        /* device, MB_MLP_PARAMS floats: the tile-cost network for learned_order; may be NULL */
  uint32_t min_strips;       /* mb_render_learned and learned batch queues: cut every tile into at least this many
                                row strips (a power of two <= 16 and <= tile; 0 = 1), so that the queue's items
                                are small even where the prediction says cheap -- the order is made per tile
                                (the probe takes 64 of each tile's pixels) while the items, and with them the
                                tail of the render, are as fine as smaller tiles; MB_EINVAL otherwise */
} mb_opts;

/* Library version string (not in the paper). */
const char* mb_version(void);

/* Human-readable name of a return code (not in the paper). */
const char* mb_strerror(int code);

/* Render one image (Eq. 2 for all i < m, j < n).
 *   w        host; the complex window (finite, xmin < xmax, ymin < ymax)
 *   m, n     rows and columns, each in [1, 2^20]; fewer than 2^32 - 1 tiles
 *   iter_max iteration budget per pixel (0 allowed: every count is 0)
 *   escape_r2  squared escape radius R^2, finite and > 0
 *   out      m*n uint32, written in full, in memory the current device can write: its own device
 *            memory, managed memory, pinned / registered host memory (the kernels then store
 *            the counts straight into host memory -- over NVLink-C2C on GB300 -- with no copy
 *            step), or ordinary host memory where the device reports pageable memory access;
 *            anything else is MB_EINVAL.  The same holds for mb_render_learned and for the
 *            `out` of each mb_view.
 *   opt      host, may be NULL (all defaults); opt->precision selects binary64 (default,
 *            the paper's method, bit-exact) or a reduced-precision variant (mb_precision)
 * Errors: MB_EINVAL for bad arguments; MB_ENOMEM / MB_ECUDA from the launch. */
int mb_render(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
              uint32_t* out, const mb_opts* opt);

/* Largest m and n that mb_render_noalloc accepts. */
#define MB_NOALLOC_MAX_SIDE 16384

/* Not in the paper: there is no counterpart of this entry point there.  It exists
 * for callers that must not allocate device memory -- code running where the
 * allocator may not be entered (host callbacks, real-time loops), or processes
 * whose device memory another framework has reserved up front.  Its counts are
 * those of mb_render for the same arguments, but it calls no cudaMalloc /
 * cudaMallocAsync / cudaFree: the temporary memory it needs sits in one fixed
 * array inside the library's device image (262,656 bytes, resident on every GPU
 * that loads the library until exit).
 *   m, n   each in [1, MB_NOALLOC_MAX_SIDE]; larger sizes return MB_EINVAL.
 *   out    as mb_render (checked the same way before any launch).
 *   opt    as mb_render: sched, tile, block, grid, unroll, items / n_items,
 *          tile_totals, trace, status, max_seconds, ev_start / ev_stop and stream
 *          are honoured.  Rejected with MB_EINVAL: workspace (the fixed array is
 *          the workspace), precision other than MB_PREC_FP64, cycle_check and
 *          fp64_products (their kernels come with mb_render only).
 * Nothing is recorded for mb_last_stats.  All calls on a device share the
 * array and it keeps the last call's contents; every part a render reads is
 * rewritten (the work counter zeroed) on the stream before the render kernel
 * runs.  Calls whose kernels overlap on the GPU race on the array: issue them
 * on one stream.  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress); make it before any stream capture starts. */
int mb_render_noalloc(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                      uint32_t* out, const mb_opts* opt);

/* Bytes of temporary device memory mb_render needs for this size and options
 * (the Cx/Cy arrays of Sec. III-A and the work counters of the Sec. III-B
 * scheduler), so that a caller can pass opts->workspace. */
size_t mb_render_workspace_size(uint32_t m, uint32_t n, const mb_opts* opt);

/* Sum of `count` uint32 values (device) into *total (device uint64, overwritten),
 * i.e. the number of z-updates of a rendered image: the sum of its Eq. 2 counts,
 * the work unit of every throughput figure (not an operation of the paper). */
int mb_sum_counts(const uint32_t* counts, uint64_t count, uint64_t* total, void* stream);

/* Statistics of one render launch (the per-worker accounting behind the paper's
 * load-balance comparison of Sec. III-IV and Table II). */
typedef struct {
  uint64_t makespan_ns;   /* first CTA start to last CTA end of the main render launch (globaltimer) */
  uint64_t iterations;    /* sum of the counts in the output buffer, i.e. z-updates of the image */
  uint32_t ctas;          /* CTAs that wrote a record */
  uint32_t sms;           /* SMs that ran at least one of them */
  double idle_tail;       /* sum over the GPU's SMs of (makespan - that SM's last CTA end), over SMs x makespan */
  double sm_busy_min;     /* per SM: (its last CTA end - its first CTA start) / makespan; min, mean, max */
  double sm_busy_mean;
  double sm_busy_max;
} mb_run_stats;

/* Statistics of the calling host thread's most recent mb_render or
 * mb_render_learned call that launched its main render (mb_render_noalloc,
 * batches and the server are not recorded; a call rejected with an error leaves
 * the previous record).  Waits for that call's stream, then reads the per-CTA
 * records -- the caller's opts->trace when given, else a small device buffer the
 * library keeps per thread and device until the process exits -- and sums the
 * counts of that call's output buffer, which must still hold them.  The stream of
 * that call must still exist.  Renders one thread keeps in flight at once on
 * several streams share that thread's buffer: pass opts->trace to each of them
 * to keep their records apart.
 *   st   host, filled in
 * Errors: MB_EINVAL (st NULL), MB_ENOTFOUND (no render recorded on this thread, or
 * its launch failed), MB_ECUDA. */
int mb_last_stats(mb_run_stats* st);

/* ---- batched mode: many viewports in one persistent launch ----
 * Not in the paper: one first-come-first-served worker pool (Sec. III-B) over
 * the tiles of many images at once; every image's counts are those of Eq. 2.
 * A view: window, size, iteration budget, R^2 and its own output buffer
 * (device, m*n uint32).  Each view is rendered exactly as mb_render would. */
typedef struct {
  mb_window w;
  uint32_t m, n, iter_max;
  double escape_r2;
  uint32_t* out;
} mb_view;

/* One-shot batch: pixel maps of all views in one launch, then one FCFS render
 * over (view, tile) items -- views queued by decreasing iter_max, tiles in
 * raster order.  1 <= count <= 65535; opts as for mb_render (sched ignored).
 * Synchronises opts->stream before returning. */
int mb_render_batch(const mb_view* views, uint32_t count, const mb_opts* opt);

/* A reusable batch: device tables built once, the two launches captured into
 * a CUDA graph.  mb_batch_plan_launch replays the graph on `stream`
 * (asynchronous); destroy synchronises the device and frees the plan. */
typedef struct mb_batch_plan mb_batch_plan;
int mb_batch_plan_create(const mb_view* views, uint32_t count, const mb_opts* opt, mb_batch_plan** plan);
int mb_batch_plan_launch(mb_batch_plan* plan, void* stream);
int mb_batch_plan_info(const mb_batch_plan* plan, uint32_t* n_items, uint32_t* grid, uint64_t* pixels);
int mb_batch_plan_destroy(mb_batch_plan* plan);

/* Autotuner: times graph replays of the batch (every sample_stride-th view) for
 * tile in {16, 32, 64} x block in {256, 512} x unroll in {8, 16} and writes the
 * fastest into *best (other fields copied from base, may be NULL) and its time
 * into *best_ms.  cache_path (may be NULL): a text file of
 * "key tile block unroll ms" lines; a hit skips the search. */
int mb_batch_autotune(const mb_view* views, uint32_t count, const mb_opts* base, uint32_t sample_stride,
                      const char* cache_path, mb_opts* best, float* best_ms);

/* ---- serving: continuous batching under a device-memory budget ----
 * Not in the paper: requests share first-come-first-served rounds (Sec. III-B);
 * every request's counts are those of Eq. 2.  A request is one view; the server allocates its counts (m*n uint32) and Cx/Cy
 * arrays on the device, charging align256(m*n*4) + align256((m+n)*8) bytes to
 * the budget until the request is released.  Requests that do not fit yet wait
 * in a FIFO of at most queue_limit entries.  A worker thread keeps four rounds
 * in flight on four streams; each round is one FCFS render over the next tiles
 * of every admitted request (oldest first, at most round_tiles tiles), so requests
 * that arrive while others run join the next round and share the GPU.  Counts
 * are exactly those of mb_render.  Timestamps are host steady-clock ns. */
typedef struct {
  mb_window w;
  uint32_t m, n, iter_max;
  double escape_r2;
} mb_request;

typedef struct {
  uint64_t submit_ns, admit_ns, start_ns, done_ns;
  uint64_t bytes;
  int status;
} mb_req_stats;

typedef struct {
  uint64_t submitted, admitted, completed, rejected, rounds;
  uint64_t bytes_in_use, peak_bytes;
  uint32_t queued;
} mb_serve_counters;

typedef struct mb_server mb_server;

/* opts: tile (default 32), block (512), unroll (4), grid, round_tiles, precision and
 * cycle_check (as for mb_render, applied to every request), learned_order and
 * model (not in the paper: each admitted request is probed once, 8 x 8 samples
 * per tile written into its counts, its tiles' costs predicted by `model` or the
 * probe-sum estimate and guarded as in mb_guard_costs, and its tiles handed to
 * the rounds longest-first instead of in raster order; tile >= 16; the probe
 * counts, features and ranking are charged to the budget with the request; the
 * model must stay valid until mb_serve_destroy); other fields ignored.
 * queue_limit 0 = 1024.  The budget is a charge, not a reservation: if the device
 * cannot allocate an admitted request's memory (a budget above the free device
 * memory), every pending request fails with MB_ECUDA and later calls return it. */
int mb_serve_create(size_t mem_budget_bytes, uint32_t queue_limit, const mb_opts* opt, mb_server** s);
/* MB_ENOMEM if the request alone exceeds the budget, MB_EBUSY if the queue is full. */
int mb_serve_submit(mb_server* s, const mb_request* rq, uint64_t* id);
/* Waits up to timeout_ms for completion: MB_OK, MB_ETIMEDOUT, MB_ENOTFOUND, or
 * the request's failure code (MB_ECANCELED, MB_ECUDA, ...). */
int mb_serve_wait(mb_server* s, uint64_t id, uint32_t timeout_ms, mb_req_stats* st);
/* Device pointer to a completed request's counts, valid until mb_serve_release. */
int mb_serve_result(mb_server* s, uint64_t id, uint32_t** dev_out);
/* Copies the first `count` counts of a completed request into dst (device or
 * host memory; unified addressing picks the direction) on `stream`, and waits
 * for the copy.  Must not overlap with mb_serve_release of the same id. */
int mb_serve_read(mb_server* s, uint64_t id, uint32_t* dst, uint64_t count, void* stream);
/* Frees a completed or failed request's device memory and budget (MB_EBUSY while it runs). */
int mb_serve_release(mb_server* s, uint64_t id);
int mb_serve_counters_get(mb_server* s, mb_serve_counters* c);
/* Marks the server failed with `code` (fault injection for tests, or an
 * application's own abort): pending requests fail with it, new submits return it. */
int mb_serve_fail(mb_server* s, int code);
/* Cancels queued requests (MB_ECANCELED), lets admitted ones finish, joins the
 * worker, returns every thread blocked in mb_serve_wait, then frees all device
 * memory.  No other call on `s` may start once destroy has begun. */
int mb_serve_destroy(mb_server* s);

/* ---- learned tile-cost model (not in the paper: it orders the FCFS queue of
 * Sec. III-B longest-first and splits heavy tiles; the counts do not change) ----
 *
 * Probe: PROBE 8 x 8 samples per tile x tile block; sample (a, b) of tile
 * (ty, tx) is pixel (ty*T + a*s + s/2, tx*T + b*s + s/2), s = T/8, clamped to
 * the last row / column.  Features (70 floats per tile, FP32):
 *   f[8a+b] = log2(1 + probe[a][b]) / log2(1 + iterMax); f[64] = (tx+0.5)/tiles_x;
 *   f[65] = (ty+0.5)/tiles_y; f[66] = log2(1 + iterMax)/17;
 *   f[67] = -log10((xmax - xmin)/n)/16; f[68] = log2(1 + (T*T/64) * sum of the probe)/32;
 *   f[69] = (samples at iterMax)/64.
 * Network: 70 -> 64 -> 64 -> 1, ReLU, FP32, residual on the probe-sum feature:
 *   y = f[68] + W3 . relu(W2 relu(W1 f + b1) + b2) + b3; flat parameters
 *   (MB_MLP_PARAMS) W1[64][70], b1[64], W2[64][64], b2[64], W3[64], b3 (row-major W[out][in]).
 * Target: log2(1 + tile total)/32; loss: mean squared error over the batch.
 * Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   p -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps).
 * Order and split (integers after one FP32 rounding): q = 0 if y <= 0 else
 *   min(trunc(fp32(y*128)), 191); tiles sorted by q descending, ties by tile
 *   index; c(q) = (2^(q>>2) * {65536,77936,92682,110218}[q&3]) >> 16 (uint64);
 *   target = max(1, (saturating sum of c) / (S G)), G = CTAs of the render,
 *   S = the split divisor (default 4; larger S cuts heavy tiles into more strips);
 *   s = smallest power of two >= ceil(c/target), at most min(16, T/4); the
 *   tile yields items (tile, k*T/s, T/s), k < s, in sorted order. */
#define MB_MLP_PARAMS 8769
#define MB_MLP_FEATURES 70

/* Probe counts (device, tiles*64 uint32) of a view with tile side opts->tile
 * (>= 16); when image_out (device, m*n) is given the samples are also stored
 * at their pixels there.  Exact counts, as mb_render. */
int mb_probe(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
             uint32_t* probe_out, uint32_t* image_out, const mb_opts* opt);

/* Features (device, tiles x 70 floats) from probe counts (device). */
int mb_tile_features(const uint32_t* probe, const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max,
                     uint32_t tile, float* feat, void* stream);

/* Training labels y[t] = log2(1 + totals[t]) / 32 (device arrays), from the
 * per-tile sums of counts that mb_render records in opts->tile_totals. */
int mb_tile_targets(const uint64_t* totals, uint32_t ntiles, float* y, void* stream);

/* Predictions y[count] (device) of the network for `count` feature rows (device). */
int mb_mlp_forward(const float* params, const float* x, uint32_t count, float* y, void* stream);

/* Loss (device float, may be NULL) and gradient (device, MB_MLP_PARAMS floats,
 * overwritten) of the mean squared error over the rows idx[0..batch) of x
 * (idx may be NULL: rows 0..batch-1); target is indexed like the rows of x. */
int mb_mlp_grad(const float* params, const float* x, const uint32_t* idx, uint32_t batch, const float* target,
                float* grad, float* loss, void* stream);

/* One Adam step, t >= 1 (device arrays of `count` floats). */
int mb_adam_step(float* params, const float* grad, float* m, float* v, uint32_t count, uint32_t t, float lr,
                 float beta1, float beta2, float eps, void* stream);

/* Train on the device: `epochs` passes, each over order[e*count .. e*count+count)
 * (device sample indices, e.g. a seeded shuffle per epoch) in minibatches of
 * `batch` (the last count % batch samples of an epoch are skipped); Adam with
 * lr, beta1 0.9, beta2 0.999, eps 1e-8, state in adam_m / adam_v (device,
 * zeroed by the caller for a fresh start).  epoch_loss (device, may be NULL)
 * receives the mean minibatch loss of each epoch. */
int mb_model_train(float* params, float* adam_m, float* adam_v, const float* x, const float* target, uint32_t count,
                   const uint32_t* order, uint32_t epochs, uint32_t batch, float lr, float* epoch_loss, void* stream);

/* Work list from predicted tile costs (device, ntiles floats), split divisor
 * S = split (0 = 4, at most 4096): items (device,
 * capacity entries) and their number (device uint32), per the rule above.
 * capacity >= 16 * ntiles always suffices; if it is exceeded, *n_items = 0 and
 * bit 2 is ORed into *status (device, may be NULL). */
int mb_order_split(const float* cost_pred, uint32_t ntiles, uint32_t tile, uint32_t grid, uint32_t split,
                   mb_item* items, uint32_t capacity, uint32_t* n_items, uint32_t* status, void* stream);

/* The learned pipeline for one view: probe (its samples go straight into
 * `out`), features, network, neighbourhood guard (mb_guard_costs), order and
 * split, then the FCFS render of the other pixels over that list.  Same counts as mb_render.  opts->tile >= 16 (default
 * 64); opts->sched is ignored; opts->trace records the final render's CTAs.
 * params == NULL is the ablation without the network: each tile's cost is
 * taken as log2(1 + (T*T/64) * sum of its probe counts) / 32. */
int mb_render_learned(const mb_window* w, uint32_t m, uint32_t n, uint32_t iter_max, double escape_r2,
                      uint32_t* out, const float* params, const mb_opts* opt);

/* Neighbourhood guard of predicted tile costs (device, tiles_x * tiles_y floats,
 * row-major tiles of one view): guarded[t] = the largest cost_pred over the 3 x 3
 * tiles around t that lie in the grid (NaN values are ignored; NaN only where all
 * of them are NaN).  The learned render and learned batch queues order and split
 * by the guarded costs: the set's interior regions are connected, so a tile whose
 * probe missed them almost always borders tiles whose probe saw them, and the
 * guard keeps it out of the cheap end of the queue, where one mispredicted heavy
 * tile would set the makespan.  Not in the paper (scheduling only).  Asynchronous
 * on `stream`; guarded must not overlap cost_pred.  Errors: MB_EINVAL, MB_ECUDA. */
int mb_guard_costs(const float* cost_pred, uint32_t tiles_x, uint32_t tiles_y, float* guarded, void* stream);

/* Save / load the network parameters (device, MB_MLP_PARAMS floats) as a small
 * binary file: 8-byte tag "MBMLP701", uint32 count, float32 values. */
int mb_model_save(const float* params, const char* path);
int mb_model_load(const char* path, float* params);

/* ---- output: iteration -> colour (Sec. I) and the image file (Sec. IV) ----
 * Palette (the paper names none): k == iter_max -> black; otherwise
 * r = tri(7k mod 512), g = tri(5k mod 512), b = tri(3k mod 512),
 * tri(x) = x < 256 ? x : 511 - x.  rgb: 3 bytes per pixel, row-major. */

/* Colours (device, 3*count bytes) of counts (device). */
int mb_colorize(const uint32_t* counts, uint64_t count, uint32_t iter_max, uint8_t* rgb, void* stream);

/* Writes a binary PPM (P6, maxval 255) of m rows x n columns from rgb (host). */
int mb_write_ppm(const char* path, const uint8_t* rgb, uint32_t m, uint32_t n);

/* ---- the master gather of one image rendered by several workers (Sec. III-A/B) ----
 * Each worker renders the items it was dealt (first come, first served across
 * GPUs) into its own image; only those pixels are sent to the master, which
 * writes them into its image.  Layout of `packed`: one slot of tile*tile counts
 * per item, item k at offset k*tile*tile, its rows row0..row0+rows-1 at their
 * row offset within the slot, tile counts per row.  Pixels outside the image
 * and slot rows outside the item are not written (pack) or not read (unpack).
 *   img     device, m*n counts, row-major (read by pack, written by unpack)
 *   items   device, n_items entries (tile < tiles of the image, row0+rows <= tile;
 *           an entry that is not sets bit 2 of *status, when given, and is skipped)
 *   packed  device, n_items*tile*tile counts
 *   tile    power of two in [8, 256]; m, n in [1, 2^20]
 * Asynchronous on `stream`; nothing is allocated.  Errors: MB_EINVAL (null
 * pointers, bad sizes), MB_ECUDA. */
int mb_pack_items(const uint32_t* img, uint32_t m, uint32_t n, uint32_t tile, const mb_item* items,
                  uint32_t n_items, uint32_t* packed, uint32_t* status, void* stream);
int mb_unpack_items(const uint32_t* packed, uint32_t m, uint32_t n, uint32_t tile, const mb_item* items,
                    uint32_t n_items, uint32_t* img, uint32_t* status, void* stream);

/* FP64 issue-rate microbenchmark (not in the paper; the measurement's
 * denominator): runs independent chains of one binary64
 * operation (op: 0 = add, 1 = mul, 2 = fma) on every SM and returns the
 * measured rate in operations per second (a fused multiply-add counts as one
 * operation) and the elapsed kernel time.  Synchronous.  This rate is the
 * denominator of "% of FP64 peak". */
int mb_fp64_peak(int op, double* ops_per_s, double* seconds);

/* Self-test of the integer-pipe products used by every render (not in the
 * paper): for i < n, sq[i] = RN(a[i]*a[i]), pr[i] = RN((2*a[i])*b[i]) as the
 * kernels form them, and ok[i] = 1 when both operands are in the range where
 * those results are exact (exponents in [2^-510, 2^511)); outside it the
 * kernels replay the step on the FP64 pipe instead.  Device arrays. */
int mb_selftest_products(const double* a, const double* b, uint64_t n, double* sq, double* pr, uint8_t* ok,
                         void* stream);

/* Self-test of the integer-pipe subtraction used by every other binary64 escape
 * step (not in the paper): for i < n, d[i] = RN(a[i] - b[i]) as the kernels form
 * it, for positive normal a[i], b[i] (the squares of a step), and ok[i] = 1 when
 * that result is exact; ok[i] = 0 (the kernels then replay the step on the FP64
 * pipe) when the exponents differ by more than 31 or the leading 32 bits of
 * the aligned mantissas cancel.  Device arrays. */
int mb_selftest_psub(const double* a, const double* b, uint64_t n, double* d, uint8_t* ok, void* stream);

/* Self-test of the bounded wait in the work-claiming protocol (not in the
 * paper; the failure-detection test of the render kernels).  Launches `ctas`
 * CTAs of 4 warps in which the worker that should publish the next work item
 * never does (its CTA's work word stays past the end of an item): every warp
 * waits in the render kernels' own claim loop, gives up after its bounded spin
 * (a fraction of a second), ORs 1 into *status and reports no work in
 * got[ctas * 4] (device, uint32; 0 expected).  Asynchronous on `stream`; the
 * context stays usable.  MB_EINVAL for NULL pointers or ctas outside [1, 1024]. */
int mb_selftest_wait(uint32_t ctas, uint32_t* status, uint32_t* got, void* stream);

/* Number of SMs and resident CTAs per SM the render kernel gets at `block`
 * threads: the worker count G of the Sec. III schedulers at the default grid. */
int mb_device_info(uint32_t block, uint32_t* sms, uint32_t* ctas_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* MB_H */
