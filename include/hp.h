/*
 * hp.h -- fused image-pipeline library for GB300 (sm_103a), C ABI.
 *
 * The library runs multi-stage image pipelines (DAGs of pointwise, 2-D stencil,
 * pyramid down/upsample and histogram stages over 2-D images) on one GPU.  It
 * keeps the algorithm -- which stages compute what -- separate from the
 * schedule -- how stages are grouped into kernels and tiled -- as the paper
 * sets out (Sec. 1; the compute-location and tiling decisions of Sec. 2 and
 * Sec. 4).  Any valid schedule gives bit-identical results: the per-stage float
 * expression is part of the algorithm and every kernel evaluates it the same
 * way.
 *
 * Conventions
 *   - Images are planar [C][H][W], row-major; x is the column (fastest), y the row.
 *   - hp_buffer strides are in bytes and must be multiples of 16; data pointers
 *     must be 16-byte aligned.
 *   - Every stencil, downsample and upsample reads its own producer with a
 *     clamp-to-edge boundary on that producer's domain:
 *     P(min(max(x,0),W-1), min(max(y,0),H-1)).
 *   - Stage ids are dense, assigned in hp_add_stage order; a stage may only read
 *     pipeline inputs and earlier stages, so id order is a topological order.
 *   - All functions return an hp_status; on failure hp_last_error() returns a
 *     message (thread-local, valid until the next call on that thread).  No
 *     function aborts the process.
 *
 * Ownership
 *   - hp_pipeline objects are created and owned by the library; free them with
 *     hp_pipeline_destroy.
 *   - hp_buffer memory is owned by the caller (device memory for hp_realize,
 *     host memory for hp_realize_host) and must stay valid until the work
 *     enqueued on the stream has completed.
 *   - Intermediate images of materialised stages, histogram scratch and TMA
 *     descriptors are owned by the pipeline; they are allocated on the first
 *     hp_realize for a given input size and freed by hp_pipeline_destroy.
 */
#ifndef HP_H
#define HP_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hp_pipeline hp_pipeline;

typedef enum {
  HP_OK = 0,
  HP_ERR_INVALID_ARG = 1,   /* null pointer, bad id, dtype/channel/size mismatch, misalignment */
  HP_ERR_UNSUPPORTED = 2,   /* a stage or group the kernels cannot run */
  HP_ERR_SCHEDULE = 3,      /* schedule violates a rule (group shape, shared-memory or thread limit) */
  HP_ERR_OOM = 4,           /* device allocation of library-owned scratch failed */
  HP_ERR_CUDA = 5,          /* a CUDA runtime call failed; the message names it */
  HP_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up (serving loop) */
  HP_ERR_STATE = 7          /* call out of order (e.g. realize before set_output) */
} hp_status;

typedef enum { HP_U8 = 0, HP_U16 = 1, HP_F16 = 2, HP_BF16 = 3, HP_F32 = 4, HP_U32 = 5 } hp_dtype;

/* Stage kinds: the operations of the imaging apps of Sec. 6. */
typedef enum {
  HP_STENCIL = 0,      /* separable 2-D stencil, per channel:
                          h(x,y') = sum_i wx[i] * in(clamp(x+i-rx), y'),
                          out(x,y) = sum_j wy[j] * h(x, clamp(y+j-ry));
                          rx, ry <= HP_MAX_RADIUS (Sec. 2, Fig. 1 stencil chain) */
  HP_POINTWISE = 1,    /* hp_op on same-size inputs at the same (x, y) (inlined producers, Sec. 4) */
  HP_DOWNSAMPLE2 = 2,  /* binomial [1,4,6,4,1]/16 per axis at (2x+i, 2y+j); size ceil(W/2) x ceil(H/2) */
  HP_UPSAMPLE2 = 3,    /* zero-stuff + [1,4,6,4,1]/8 per axis, coarse index clamped; inputs[1] is a
                          size reference whose domain the output takes (it is not read) */
  HP_HISTOGRAM = 4,    /* 256-bin counts of a 1-channel u8 image; output 256 x 1 u32; images of
                          more than 2^32 - 1 pixels are refused (HP_ERR_UNSUPPORTED) */
  HP_CDF_LUT = 5,      /* equalization LUT (256 x 1 u8) from a histogram stage */
  HP_LUT_APPLY = 6,    /* out = lut[in] for a 1-channel u8 image */
  HP_MAX_STENCIL = 7,  /* per channel, the maximum over the (2rx+1) x (2ry+1) window at clamped
                          coordinates (the max filter app of Sec. 6; exact in any order);
                          rx, ry <= HP_MAX_RADIUS, no taps */
  HP_GRID_SPLAT = 8,   /* bilateral grid (the bilateral grid app of Sec. 6): a 1-channel image
                          v -> a grid of (ceil(W/s)+1) x (ceil(H/s)+1) cells x 2 GZ channels,
                          GZ = floor(1/r + 1/2) + 1; cell (gx, gy) takes the s x s pixels
                          (clamp(gx s + i - s/2), clamp(gy s + j - s/2)) and adds (v, 1),
                          v = clamp(I, 0, 1), to channels 2z and 2z+1, z = floor(v (1/r) + 1/2)
                          in f32, clamped; params = {s, r} */
  HP_GRID_SLICE = 9    /* (grid, 1-channel image) -> 1 channel at the image's size: trilinear
                          interpolation of the grid's value and weight at (x/s, y/s, v/r),
                          indices clamped; out = value / weight (v where the weight is 0);
                          params = {s, r} */
} hp_kind;

/* Point-wise operations (HP_POINTWISE).  The float expression of each is fixed
 * and shared by every kernel that evaluates it. */
typedef enum {
  HP_OP_GRAY = 0,      /* 1 input, 3 ch -> 1 ch: 0.299 R + 0.587 G + 0.114 B, each channel first
                          multiplied by params[0] (1 for float inputs, 1/65535 for u16) */
  HP_OP_MUL = 1,       /* a * b, per channel */
  HP_OP_ADD = 2,       /* a + b */
  HP_OP_SUB = 3,       /* a - b */
  HP_OP_HARRIS = 4,    /* (Sxx, Syy, Sxy) -> Sxx*Syy - Sxy^2 - params[0] * (Sxx + Syy)^2 */
  HP_OP_UNSHARP = 5,   /* (in, blur) -> in + params[0] * (in - blur), per channel */
  HP_OP_LL_REMAP = 6,  /* 1 ch gray -> K+1 ch: channel k < K is the remap r_k(gray) around
                          g_k = k/(K-1); channel K is gray itself.
                          params = {sigma_r, alpha, beta, K} */
  HP_OP_LL_INTERP = 7, /* (G stack K+1 ch, L stack >= K ch) -> 1 ch: t = G[K]*(K-1),
                          k0 = min(floor(t), K-2), f = t - k0, (1-f) L[k0] + f L[k0+1].
                          params = {K} */
  HP_OP_LL_COLOUR = 8, /* (in 3 ch, gray, out_gray) -> 3 ch: v = in*params[0];
                          (gray > 0 ? v * out_gray / gray : out_gray) * params[1] */
  HP_OP_SELECT = 9,    /* 1 input -> 1 ch: channel params[0] */
  HP_OP_SCALE = 10,    /* a * params[0] + params[1], per channel (also dtype conversion) */
  HP_OP_PREMUL = 11,   /* 1 input, 4 ch (RGBA) -> 4 ch: (R a, G a, B a, a) (the interpolate app) */
  HP_OP_OVER = 12,     /* (front 4 ch, back 4 ch) -> 4 ch, premultiplied: front + (1 - front.a) back */
  HP_OP_UNPREMUL = 13, /* 1 input, 4 ch -> 3 ch: a > 0 ? c / a : 0 */
  HP_OP_ZBLUR = 14     /* bilateral grid, 2 GZ ch -> 2 GZ ch: [1,4,6,4,1]/16 along the range
                          levels (channel 2z + k from channels 2 clamp(z + j) + k), params = {GZ} */
} hp_op;

#define HP_MAX_RADIUS 4
#define HP_MAX_INPUTS 4
#define HP_MAX_PARAMS 8
#define HP_INLINE (-1)

typedef struct {
  int kind;              /* hp_kind */
  int op;                /* hp_op for HP_POINTWISE, else ignored */
  int n_inputs;
  const int* inputs;     /* stage id >= 0, or -1-k for pipeline input k */
  int rx, ry;            /* stencil radii */
  const float* wx;       /* 2*rx+1 taps along x (HP_STENCIL) */
  const float* wy;       /* 2*ry+1 taps along y (HP_STENCIL) */
  const float* params;   /* op parameters (see hp_op) */
  int n_params;
  int storage;           /* hp_dtype the stage's values are rounded to wherever they are kept */
  int channels;          /* output channels; must agree with the op's rule */
  int boundary;          /* 0 = clamp-to-edge (the only boundary supported) */
} hp_stage_desc;

/* Schedule: the compute location and tiling decisions of Sec. 4.  Every stage
 * belongs to a fusion group (one kernel per group), or is inlined (HP_INLINE,
 * point-wise stages only: recomputed inside each consumer group).  A group
 * computes every member over the tile its output needs, keeping members in
 * shared memory or registers; only the group's output stage (the one stage read
 * outside the group, or the pipeline output) is written to memory.  Singleton
 * groups everywhere is the stage-per-kernel schedule ("compute root", Sec. 2). */
enum {
  HP_IMPL_AUTO = 0,    /* the kernel the group's shape selects */
  HP_IMPL_GENERIC = 1, /* the generic interpreter */
  HP_IMPL_WAVE = 2,    /* streaming kernels: a warp walks down a strip of columns, rows arrive
                          through a per-warp TMA ring.  Stencil chains of 2 or 4 stages: every stage
                          in registers; strips of 120 columns (2 stages, 4-byte input) or 112 (4
                          stages, or a 2-byte input), tile_h rows per run, threads <= 256.
                          Harris: one warp per column strip of exactly 120 columns (4-byte input) or
                          112 (2-byte input), tile_h rows per run (>= 4), threads <= 256.  Under
                          HP_IMPL_AUTO a Harris group whose tile_w is that strip width (the default)
                          also takes the streaming kernel; other widths take the tiled one.
                          A single 5x5 stencil, alone or with the unsharp combine: the same strips
                          (120 / 112 columns), tile_h rows per run, threads <= 256; again the default
                          under HP_IMPL_AUTO when tile_w is the strip width.
                          A pyramid downsample of f32 planes, and the first local-Laplacian
                          downsample with gray and the remap inlined (K = 8, u16 or f32 input, sigma
                          below the level spacing 1/7): strips of 30 coarse columns, tile_h coarse rows
                          per run, threads <= 256; the default under HP_IMPL_AUTO when tile_w is 30.
                          A local-Laplacian level (K = 8, f32 stages; level 0 from u16 RGB): the same
                          30-column strips (of the coarser level), tile_h coarse rows per run.  Other
                          groups ignore HP_IMPL_WAVE's request when they have no streaming kernel. */
  HP_IMPL_LINES = 3     /* line-buffer stencil chain: a chain of an even number of 5x5 stencils (2..8)
                          whose input, stages and output share one type (f32, f16 or bf16; 16-bit
                          chains of 4 or 8 stages) runs as one thread block per tile_w x tile_h output
                          tile (tile_w a multiple of 8, tile_w + 4 depth <= 256 columns, tile_h >=
                          2 depth + 2 rows); every stage computes 8-column blocks on threads of its
                          own and passes its rows to the next stage through a shared-memory ring
                          (threads and serial_y do not apply).  Other groups, and chains outside these
                          limits, ignore the request and take their default kernel. */
};

typedef struct {
  int n_stages;                /* must equal the pipeline's stage count */
  const int* group_of_stage;   /* per stage: group id in [0, n_groups) or HP_INLINE */
  int n_groups;
  const int* tile_w;           /* per group: output tile width  (NULL: defaults) */
  const int* tile_h;           /* per group: output tile height (NULL: defaults) */
  const int* threads;          /* per group: threads per block  (NULL: defaults) */
  const int* serial_y;         /* per group: rows per thread segment (NULL: defaults) */
  const int* impl;             /* per group: HP_IMPL_* (NULL: auto) */
} hp_schedule;

typedef struct {
  void* data;                  /* device (hp_realize) or host (hp_realize_host) pointer */
  int dtype;                   /* hp_dtype */
  int channels, width, height;
  long long row_stride_bytes;  /* multiple of 16 */
  long long plane_stride_bytes;/* multiple of 16 */
} hp_buffer;

/* Per-group facts after lowering, for tests and the tuner. */
typedef struct {
  int kernel;                  /* hp_kernel_id below */
  int output_stage;
  int n_members;               /* stages computed in the group (inlined ones included) */
  int tile_w, tile_h, threads;
  int grid_x, grid_y, grid_z;
  int smem_bytes;
} hp_group_info;

enum {
  HP_KERNEL_STENCIL_CHAIN = 0, /* fused chain of 5x5 stencils (TMA tile + halo, register sweeps) */
  HP_KERNEL_UNSHARP = 1,       /* 5x5 stencil + unsharp combine, fused */
  HP_KERNEL_HARRIS = 2,        /* whole Harris DAG in one kernel */
  HP_KERNEL_GENERIC = 3,       /* interpreter over any group of stencil/point-wise/pyramid stages */
  HP_KERNEL_POINTWISE = 4,
  HP_KERNEL_DOWNSAMPLE = 5,    /* every channel of a level; also from an inlined LL remap of gray */
  HP_KERNEL_UPSAMPLE = 6,
  HP_KERNEL_HISTOGRAM = 7,
  HP_KERNEL_CDF_LUT = 8,
  HP_KERNEL_LUT_APPLY = 9,
  HP_KERNEL_LL_LEVEL = 10,     /* local-Laplacian level: two-level blend + collapse step (+ colour) */
  HP_KERNEL_STENCIL_WAVE = 11, /* streaming stencil chain of 2 or 4 stages, all in registers */
  HP_KERNEL_HARRIS_ROWS = 12,  /* whole Harris DAG, streaming: one warp per column strip, rows
                                  through a per-warp TMA ring, intermediates in registers */
  HP_KERNEL_STENCIL_ROWS = 13, /* one 5x5 stencil (+ unsharp combine), streaming: one warp per
                                  column strip of one plane, rows through a per-warp TMA ring */
  HP_KERNEL_HISTEQ = 14,       /* histogram + CDF/table + lookup in one group: one cooperative
                                  kernel, a grid-wide barrier between counting and lookup */
  HP_KERNEL_LL_REMAP_ROWS = 15, /* level 1 of the local-Laplacian remap pyramid from the input
                                  (gray, K = 8 remaps, downsample), streaming: one warp per strip
                                  of 30 coarse columns, everything in registers */
  HP_KERNEL_LL_DOWN_ROWS = 16,  /* one pyramid level down of a stack of f32 planes, streaming: one
                                  warp per strip of 30 coarse columns and 3 (or 1) planes */
  HP_KERNEL_LL_LEVEL_ROWS = 17, /* local-Laplacian level (K = 8, f32 stages), streaming: one warp per
                                  strip of 30 coarse (60 fine) columns, upsample window in shared memory */
  HP_KERNEL_MAX_ROWS = 18,      /* max filter (one square window-maximum stage of radius 1..4, or a
                                  horizontal and a vertical one), streaming: one warp per strip of 120
                                  columns of one plane, a ring of row maxima in registers */
  HP_KERNEL_INTERP_ROWS = 19,   /* interpolate level (upsample, composite, optional division by
                                  coverage; f32 RGBA), streaming: one warp per strip of 30 coarse
                                  columns, upsample window in registers */
  HP_KERNEL_PW_ROWS = 20,       /* one point-wise stage over f32 images (add, sub, mul, scale,
                                  unsharp combine, premultiply, over, unpremultiply): 4 pixels per
                                  thread, 128-bit loads and stores */
  HP_KERNEL_GRID_SPLAT = 21,    /* bilateral grid splat: one thread per cell (four, two pixel rows
                                  each, for 8 x 8 cells), accumulators in shared memory */
  HP_KERNEL_GRID_SLICE = 22,    /* bilateral grid slice: four pixels of a row per thread, trilinear */
  HP_KERNEL_GRID_BLUR = 23,     /* bilateral grid blur (range levels, x, y; binomial/16), streaming:
                                  one warp per 28 grid columns x 4 range levels, y taps in order */
  HP_KERNEL_STENCIL_LINES = 24  /* fused chain of 5x5 stencils, line-buffered: every stage on threads of
                                  its own, rows passed through shared-memory rings (HP_IMPL_LINES) */
};

/* Create an empty pipeline with n_inputs inputs of the given dtypes and channel
 * counts.  *out receives the handle. */
hp_status hp_pipeline_create(hp_pipeline** out, int n_inputs, const int* in_dtypes,
                             const int* in_channels);

/* Append a stage; *out_stage_id receives its id.  Validates kinds, ops, input
 * ids, radii, channel rules and parameter counts. */
hp_status hp_add_stage(hp_pipeline* p, const hp_stage_desc* desc, int* out_stage_id);

/* Mark the pipeline's output stage (exactly one). */
hp_status hp_set_output(hp_pipeline* p, int stage_id);

/* Set the schedule (copied).  Host-only validation of group structure; shared
 * memory and thread limits are checked again at realize once sizes are known.
 * Without a call, every stage is its own group. */
hp_status hp_schedule_set(hp_pipeline* p, const hp_schedule* s);

/* Enqueue the pipeline on a CUDA stream (cudaStream_t passed as void*, NULL =
 * legacy default stream).  Inputs and the output are device buffers.  Never
 * synchronises, except that the first call for a new input size allocates the
 * pipeline's scratch (cudaMalloc). */
hp_status hp_realize(hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                     const hp_buffer* output, void* stream);

/* Lowers p for inputs of the given sizes and allocates its buffers and kernel
 * state (on `stream`), without running anything: the first hp_realize for
 * those sizes then starts at once.  Optional; hp_realize does the same on
 * first use. */
hp_status hp_prepare(hp_pipeline* p, const int* widths, const int* heights, int n_inputs, void* stream);
/* Same as hp_realize with HOST buffers: copies the inputs to device staging
 * owned by the pipeline, runs, copies the output back and synchronises the
 * stream before returning.  Pinned host memory gives asynchronous copies. */
hp_status hp_realize_host(hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                          const hp_buffer* output, void* stream);

/* hp_realize_host without waiting, for a stream of images from host memory:
 * enqueues the copies of the inputs to device staging (on a copy stream the
 * pipeline owns), the realize on `stream`, and the copy of the output back
 * (on a second copy stream the pipeline owns), and returns.  The pipeline
 * alternates between two staging sets, so consecutive calls overlap: the
 * copy in of one image with the realize of the previous one and the copy out
 * of the one before.  Every call's input and output host buffers (pinned
 * memory: pageable copies are synchronous) must stay valid and unchanged
 * until hp_realize_host_wait returns; consecutive calls on one pipeline must
 * pass the same `stream` (the realizes share the pipeline's intermediate
 * buffers and are ordered by it).  Errors of the enqueueing calls are
 * returned at once; the device error word is read by hp_check_device_error. */
hp_status hp_realize_host_async(hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                                const hp_buffer* output, void* stream);
/* Waits until every hp_realize_host_async call on p so far has written its
 * output to host memory (a no-op when there was none). */
hp_status hp_realize_host_wait(hp_pipeline* p);

/* Lowering facts of group g for inputs of the given sizes (width/height per
 * input).  Host only: needs no GPU. */
hp_status hp_group_info_get(hp_pipeline* p, const int* in_widths, const int* in_heights,
                            int group, hp_group_info* info);

/* Number of groups of the current schedule. */
hp_status hp_group_count(hp_pipeline* p, int* n_groups);

/* Bounds inference (host only, needs no GPU): for group g and an output tile
 * [x0, x0+w) x [y0, y0+h) of the group's output, the rectangle of every stage
 * the group computes, in that stage's own coordinates, clamped to its domain.
 * rects receives 4 ints per stage id (x0, y0, x1, y1; x1 == x0 for stages the
 * group does not compute). */
hp_status hp_infer_bounds(hp_pipeline* p, const int* in_widths, const int* in_heights,
                          int group, int x0, int y0, int w, int h, int* rects, int n_rects);

/* Pipeline options.
 * HP_OPT_CUDA_GRAPH (0/1, default 0): replay each realize as a CUDA graph.  The
 *   launch sequence is captured per set of buffer addresses (input and output
 *   pointers and strides): the first realize with new addresses runs
 *   uncaptured, the second captures and instantiates a graph, later ones launch
 *   it with one cudaGraphLaunch on the caller's stream.  Up to 16 graphs are
 *   kept per input size (least recently used evicted).  Capture happens on a
 *   private stream, so the caller's stream may be the legacy default stream.
 * HP_OPT_OVERLAP (0/1, default 1): launch the kernels of a realize with
 *   programmatic dependent launch, so that a kernel's blocks may be scheduled
 *   while its predecessor's last blocks drain.  Every kernel waits for its
 *   predecessor to complete before it touches memory, so results are the same
 *   either way.
 * HP_OPT_PROBE_ATTRS (0/1, default 0): while on, every realize that launches
 *   kernels (not a graph replay) records the register count and local-memory
 *   (spill) bytes per thread of each kernel it launches; hp_kernel_attrs_get
 *   returns them.  For the benchmark-driven search, which prunes schedules
 *   whose kernels spill (Sec. 4.6 prunes on hardware limits). */
enum { HP_OPT_CUDA_GRAPH = 1, HP_OPT_OVERLAP = 2, HP_OPT_PROBE_ATTRS = 3 };
hp_status hp_set_option(hp_pipeline* p, int option, long long value);

/* Kernels launched by the last realize that ran with HP_OPT_PROBE_ATTRS on,
 * the largest register count per thread among them, and the largest
 * local-memory size per thread (non-zero: the kernel spills or keeps a stack
 * array).  HP_ERR_INVALID_ARG for null arguments. */
hp_status hp_kernel_attrs_get(hp_pipeline* p, int* n_kernels, int* max_registers, long long* max_local_bytes);

/* ---- Serving loop ---------------------------------------------------------
 * Continuous batching of pipeline requests on one GPU (north of the paper's
 * benchmark loop, Sec. 6).  Requests (a pipeline, input buffers, an output
 * buffer) are admitted in arrival order as soon as one of `slots` CUDA streams
 * and enough of an HBM arena reserved at creation (`hbm_budget_bytes`) are
 * free; admitted requests run concurrently (copy in, realize, copy out).  Up to
 * `max_batch` queued requests for the same pipeline, image size and buffer
 * kind, with at most 32 MB of inputs and outputs in all, are served by one
 * realize: their images are stacked as planes, so each
 * kernel launches once, as one persistent grid, for the batch, and every
 * result equals the request's solo result.  Batching covers pipelines whose
 * stages act on each channel separately (stencils, resampling, per-channel
 * point-wise ops) and the fused Harris and histogram-equalization kernels.
 * Each slot keeps the staging region of a request shape resident in the
 * arena after the request (least recently used regions of idle slots are
 * given back when the arena is full), so its realize of that shape replays as
 * a CUDA graph from the second request on.  Buffers must stay valid until the
 * request completes; pinned host memory gives asynchronous copies.  The
 * pipeline must outlive the server.  Latency = submit to the completion the
 * server's worker thread observes. */
typedef struct hp_server hp_server;
typedef struct {
  unsigned long long submitted, completed, failed;
  unsigned long long batched_launches;  /* realizes that served more than one request */
  unsigned long long peak_bytes;        /* peak arena bytes admitted */
  double p50_us, p99_us, mean_us, max_us;
  double mpix;                          /* output megapixels completed */
  double busy_s;                        /* first submit to last completion */
  unsigned long long graph_replays;     /* slot realizes served by an instantiated CUDA graph */
  unsigned long long resident_bytes;    /* arena bytes held by resident staging regions now */
  unsigned long long device_requests;   /* requests submitted with device buffers */
  unsigned long long evictions;         /* staging regions given back to admit other shapes */
} hp_server_stats;

/* Reserves the arena (cudaMalloc of hbm_budget_bytes, at least 1 MiB), creates
 * `slots` streams (1..64) and the worker thread; max_batch is 1..64.
 * HP_ERR_INVALID_ARG for arguments out of range, HP_ERR_OOM if the arena
 * cannot be reserved. */
hp_status hp_server_create(hp_server** out, long long hbm_budget_bytes, int slots, int max_batch);
/* Enqueues a request with HOST buffers; *ticket identifies it.  Never blocks
 * on the GPU. */
hp_status hp_server_submit(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                           const hp_buffer* output, unsigned long long* ticket);
/* The same with DEVICE buffers (no host copies): served alone, the realize
 * runs on the buffers themselves; in a batch they are gathered into and
 * scattered from the slot's staging region by device-to-device copies. */
hp_status hp_server_submit_device(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs,
                                  const hp_buffer* output, unsigned long long* ticket);
/* Waits up to timeout_ms for a request; HP_ERR_TIMEOUT if it is not complete
 * by then (it stays queued or running), else the request's status. */
hp_status hp_server_wait(hp_server* s, unsigned long long ticket, int timeout_ms, double* latency_us);
hp_status hp_server_stats_get(hp_server* s, hp_server_stats* stats);
/* Makes every slot's copy of pipeline p ready for requests whose inputs have
 * the sizes of `inputs` (only width, height, dtype and channels are read):
 * lowering, scratch and kernel state, a resident staging region and the
 * captured graph of the realize, so the first such request does no
 * allocation, lowering or capture on the worker thread.  When the server
 * batches requests of this shape (max_batch > 1, a batchable pipeline) the
 * same is done for every batch it may form: 2 .. max_batch requests of at most
 * 32 MB of inputs and outputs in all, with host and with device buffers.
 * Call before traffic. */
hp_status hp_server_prepare(hp_server* s, hp_pipeline* p, const hp_buffer* inputs, int n_inputs);
/* Finishes queued and running requests, then frees the server. */
hp_status hp_server_destroy(hp_server* s);

/* Reads and clears the pipeline's device error word (synchronises the device).
 * *code: 0 = no error; 1 = a bounded TMA/mbarrier wait gave up; 2 = a fused
 * kernel's read fell outside the tile bounds inference gave it (the read was
 * skipped); 3 = the fused histogram equalization's grid-wide barrier gave up.
 * A non-zero code means the last outputs are not valid. */
hp_status hp_check_device_error(hp_pipeline* p, int* code);

hp_status hp_pipeline_destroy(hp_pipeline* p);

/* Histogram equalization of one 1-channel u8 image that allocates nothing.
 *
 * For callers that cannot allocate device memory when they run a pipeline: a
 * host framework that owns all device memory through its own pool and forbids
 * cudaMalloc from plugins, a real-time or serving loop that must not block
 * (cudaMalloc can synchronise the device) or fail under memory pressure, or a
 * deployment that reserves all memory once at start-up.  The paper has no
 * counterpart; it is a property of this library.
 *
 * Computes exactly what the HP_HISTOGRAM -> HP_CDF_LUT -> HP_LUT_APPLY pipeline
 * computes, with the same kernels.  The caller passes the device input and
 * output (1-channel u8, equal sizes, 16-byte aligned data and row strides;
 * input == output is allowed, since every thread reads its bytes before it
 * writes them and the table is built only after the whole image is counted); the
 * 256 histogram counters and the 256-entry table live in a fixed 1280-byte
 * array inside the library's device image, which every GPU that loads the
 * library holds until the process exits.  Images of more than
 * HP_NOALLOC_MAX_PIXELS pixels (the counters are 32-bit) are rejected with
 * HP_ERR_INVALID_ARG.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array per device and
 * clears the counters on its stream before counting, so calls run in order on
 * one stream are independent, but calls that overlap on the GPU (different
 * streams, or concurrent host threads) race on the array.  Enqueues work on the
 * stream and returns without synchronising; no cudaMalloc, cudaFree or
 * allocating library routine is called. */
#define HP_NOALLOC_MAX_PIXELS 4294967295ULL
hp_status hp_histeq_u8_noalloc(const hp_buffer* input, const hp_buffer* output, void* stream);

/* FP32 throughput of this GPU, measured: the denominator of the ALU roofline
 * that the benchmark reports (the paper has no counterpart; it measures no
 * roofline).  Runs `launches` launches of a kernel whose threads each execute
 * `iters` x 128 independent FP32 fmas (8 chains), on every SM at the kernel's
 * maximum occupancy, after one untimed launch, on `stream`; times them with
 * CUDA events and SYNCHRONISES on the last event.  paired = 0 issues scalar
 * fma instructions, paired = 1 the paired form (fma.rn.f32x2, two fmas per
 * instruction).  Results: *flops_per_s (2 flops per fma), and when not null
 * *ms_per_launch and *sm_count (the device's multiprocessor count).
 * HP_ERR_INVALID_ARG for a null result pointer or counts below 1,
 * HP_ERR_CUDA if a query or launch fails. */
hp_status hp_measure_fp32_peak(int paired, int iters, int launches, void* stream, double* flops_per_s,
                               double* ms_per_launch, int* sm_count);

/* Message of the last failure on this thread ("" if none). */
const char* hp_last_error(void);

/* Kernel launches this library has issued since the process started. */
unsigned long long hp_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* HP_H */
