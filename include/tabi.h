/*
 * tabi.h -- C ABI of the GB300 atlas packer.
 *
 * Implements the data-parallel hot path of TABI (Gu, Vining, Sheffer,
 * "TABI: Tight and Balanced Interactive Atlas Packing", arXiv 2602.07782).
 * Problem statement (Sec. 4): a set of 2D charts (polygons in texel units)
 * and a fixed atlas size in; one common scale and a rigid transform per
 * chart (translation, 90-degree rotation, reflections) out, such that no two
 * charts or their gutters overlap.
 *
 * Integer conventions.  Vertices are int32 in 1/256 texel ("Q.8"); every
 * coordinate must lie in (-2^20, 2^20).  Candidate scales are k/1024 with
 * k = 16*j, j = 1..64 -- the paper's 64 scales 1/64 .. 64/64 (Sec. 5).  All
 * arithmetic on the path is integer and results are bit-exact with the CPU
 * oracle that ships with the tests.
 *
 * Placement semantics.  For chart c with vertex v (Q.8, input coordinates),
 * its position in the atlas (texels, y down, 0 = atlas top) is obtained by
 *   1. p = v - (min_x, min_y) of the chart's input AABB;
 *   2. if rot90:  p = (p.y, W0 - p.x)      (W0 = input AABB width, Q.8);
 *   3. if flip_y: p.y = Hq - p.y;  if flip_x: p.x = Wq - p.x
 *      (Wq, Hq = AABB size after step 2, Q.8);
 *   4. t = p * k / 2^18  (texels);  w = ceil(Wq * k / 2^18), with k the
 *      placement's own scale (tabi_placement.k);
 *   5. if mirror: t.x = w - t.x;
 *   6. atlas point = (x, y) + t.
 * Every texel whose open square meets a placed chart lies in
 * [x, x + w) x [y, y + h) inside the atlas, and the texels of two charts
 * are at least 2*gutter texels apart (1-px gutters, Sec. 5).
 *
 * Ownership and streams.  The caller owns every input and output buffer.
 * Calls are enqueued on the given CUDA stream (NULL = the legacy default
 * stream) and return after the result is known (one stream synchronisation
 * per call).  A context owns one device arena and must not be used by two
 * host threads at once (TABI_ERR_BUSY otherwise).  No device memory is
 * allocated per call: everything lives in the arena.
 *
 * Errors are returned as tabi_status codes; nothing is thrown across the
 * ABI.  tabi_last_error() gives a one-line description of the last failure
 * on a context.
 */
#ifndef TABI_H
#define TABI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tabi_status {
  TABI_OK = 0,
  TABI_ERR_INVALID_ARG = 1, /* n < 1 or > TABI_MAX_CHARTS, a chart with < 3
                               vertices, an AABB side
                               below one texel, a coordinate outside
                               (-2^20, 2^20), atlas side outside [1, 8192],
                               bad params, or an atlas too wide for the
                               gutter (gutter 0 supports widths up to about
                               3,600 texels, gutter >= 1 every width)       */
  TABI_ERR_NO_FIT = 2,      /* no candidate scale packs every chart          */
  TABI_ERR_OOM = 3,         /* the context arena is too small for this input */
  TABI_ERR_CUDA = 4,        /* a CUDA call failed (see tabi_last_error)      */
  TABI_ERR_TIMEOUT = 5,     /* a bounded wait ran out (serving)              */
  TABI_ERR_BUSY = 6,        /* the context is in use by another call; or a
                               server is shutting down                       */
  TABI_PENDING = 7          /* not an error: the request is still in flight
                               (tabi_poll)                                    */
} tabi_status;

#define TABI_PARAMS_VERSION 2

/* Feature flags (all on = the paper's method; the others are the ablations
 * of Tab. 3 and the boxes-only Chameleon baseline). */
#define TABI_F_HC      1u /* horizontal compacting configurations, Sec. 4.1.2 */
#define TABI_F_BALANCE 2u /* direction choice and knees, Sec. 4.2; off =
                             static left/right alternation                   */
#define TABI_F_OBB     4u /* OBB proxy in the envelopes, Sec. 4.1.1         */
#define TABI_F_LAABB   8u /* local-AABB proxy in the envelopes, Sec. 4.1.1;
                             OBB and LAABB both off = bounding boxes only    */
#define TABI_F_ALL     15u
/* Inspection aid, not part of the method: every candidate is evaluated and
 * its row loop runs to its end.  Without it, candidates above the area
 * bound are skipped (the charts' covers dilated by the gutter never overlap
 * and stay inside the padded atlas, and a simple polygon of area A and
 * larger side E dilated by g covers at least A + 2gE + 4g^2, so a candidate
 * at which these areas exceed (W + 2g)(H + 2g) cannot succeed; charts must
 * be simple polygons), and a candidate is skipped or abandoned between rows
 * once a larger one of the same atlas has succeeded.  The scale and placements are the same
 * either way; only the per-candidate summaries of TABI_INSPECT_SCALE become
 * complete. */
#define TABI_F_EVAL_ALL 16u

/* Largest chart count of one atlas, largest batch. */
#define TABI_MAX_CHARTS 131072
#define TABI_MAX_BATCH 65536

typedef struct tabi_params {
  int32_t version;      /* TABI_PARAMS_VERSION                                */
  int32_t gutter;       /* gutter g in texels, 0..8 (Sec. 5 uses 1)           */
  int32_t knee_abs_pct; /* knee: drop >= this % of the atlas height (10)     */
  int32_t knee_rel_pct; /* knee: drop >= this % of the taller chart (20)     */
  int32_t lr_sig_pct;   /* reflect left/right if areas differ by more than
                           this % of the AABB area (10), App. A              */
  int32_t knee_margin;  /* knee fold wins iff its max frontline is smaller
                           by at least this many texels (1), Sec. 4.2        */
  uint32_t flags;       /* TABI_F_*                                          */
  int32_t scale_fanout; /* candidate scales evaluated per wave of the
                           descending search, 1..64 (64 = all at once), or
                           0 = the autotuned value for this kind of batch
                           (tabi_autotune), else 64 for one atlas and 8 for
                           several.  The result is the same for every
                           value.  Waves share the envelope pools, so a
                           smaller fan-out also needs a smaller arena       */
  int32_t laabb_count;  /* local AABBs per axis K: 10 (App. A), or 2 or 5 (the
                           Tab. 13 ablation: fewer slices, looser envelopes,
                           usually a smaller scale); other values return
                           TABI_ERR_INVALID_ARG.  Slice s of an extent E is
                           [floor(s E / K), floor((s + 1) E / K)]; the ten
                           slots per axis of tabi_chart_info hold slice
                           floor(t K / 10) in slot t                        */
  int32_t topt_permille;     /* t_opt of Sec. 4.4 in permille of the atlas
                                height (10 = the paper's 1 %; 0 = rows are
                                always folded one by one, Tab. 4's t_opt = 0):
                                once no knee is live and a row's tallest
                                chart is shorter than t_opt H at the
                                candidate scale k, the remaining charts are
                                folded by the prefix sum of their offsets
                                (padded width minus the compacting distance
                                to the next chart; chart s+1 never left of
                                chart s-1's right edge) with rows cut
                                modulo W + 2g, so a row's last chart may
                                overflow; then drawn at one intermediate
                                scale k': the largest of k-14 .. k at which
                                every such row, laid from its near end, fits
                                (if none does, the remaining charts are
                                folded row by row as before the switch),
                                laid left-to-right, right-to-left,
                                right-to-left in turn and dropped onto the
                                skyline.  The
                                pack's scale is then the successful
                                candidate with the largest area-weighted
                                mean scale of its charts (ties: the larger
                                candidate); each placement carries its
                                chart's scale; 0..1000                      */
  int32_t hybrid_min_charts; /* the prefix folding applies to atlases of more
                                than this many charts (the paper: 10,000)   */
} tabi_params;

/* One placed chart; see "Placement semantics" above.  k is the chart's
 * scale k/1024: the pack's scale, or for the charts laid out by the
 * prefix-sum tail (Sec. 4.4, topt_permille) the tail's intermediate scale,
 * which is at most the pack's. */
typedef struct tabi_placement {
  int32_t x, y;
  uint8_t rot90, flip_x, flip_y, mirror;
  int32_t k;
} tabi_placement;

typedef struct tabi_ctx tabi_ctx;

/* Fill *p with the paper's defaults: gutter 1, knee 10 % / 20 %, left/right
 * significance 10 %, knee margin 1, all features on, 10 local AABBs per
 * axis, prefix-sum folding past t_opt = 1 % for atlases of more than 10,000
 * charts; fan-out 0 (tuned). */
void tabi_params_default(tabi_params *p);

/* Create a context on CUDA device `device`.  If `arena` is non-NULL it is a
 * caller-owned device buffer of `arena_bytes` (256-byte aligned) that the
 * context uses for all intermediate data and that must outlive the context;
 * if NULL the context allocates `arena_bytes` itself (cudaMalloc) and frees
 * it in tabi_ctx_destroy.  Returns TABI_ERR_INVALID_ARG for a bad device or
 * alignment, TABI_ERR_CUDA if allocation fails. */
tabi_status tabi_ctx_create(tabi_ctx **out, int device, void *arena, size_t arena_bytes);
void tabi_ctx_destroy(tabi_ctx *ctx);
const char *tabi_last_error(const tabi_ctx *ctx);
const char *tabi_status_str(tabi_status s);

/* Arena bytes a pack of this size needs (upper bound, host arithmetic only).
 * `sum_extent_texels` = sum over charts of (input AABB width + height) in
 * whole texels, rounded up. */
size_t tabi_arena_bytes(int32_t n_charts, int32_t n_verts, int32_t atlas_w, int32_t atlas_h,
                        int64_t sum_extent_texels, int32_t gutter);

/* Pack one atlas (Sec. 4.3 Algorithm Summary; Algorithm 5 per candidate
 * scale; largest successful scale, Sec. 3.1 / Sec. 5, or with the
 * prefix-sum tail the largest area-weighted one, Sec. 4.4).  HOST buffers:
 *   offsets[n_charts + 1]  vertex offsets (CSR), offsets[0] = 0,
 *                          offsets[n_charts] = n_verts;
 *   verts[2 * n_verts]     x0, y0, x1, y1, ... (Q.8), one closed loop per
 *                          chart;
 *   out[n_charts]          placements, input order (written on TABI_OK);
 *   out_k                  the chosen candidate k (scale k/1024); 0 on
 *                          NO_FIT (each placement's k is its chart's
 *                          scale: out_k, or the tail's smaller k');
 * The inputs are copied to the device on `stream`, the result back:
 * buffers in pinned (cudaHostAlloc / cudaHostRegister) memory, 4-byte
 * aligned, are read and written by a copy kernel over the host link (one
 * launch each way for the whole batch); other host buffers take one
 * cudaMemcpyAsync each.  Either way the buffers are only touched before the
 * call returns.
 * Returns TABI_OK, TABI_ERR_NO_FIT, TABI_ERR_INVALID_ARG, TABI_ERR_OOM,
 * TABI_ERR_CUDA or TABI_ERR_BUSY. */
tabi_status tabi_pack(tabi_ctx *ctx, const tabi_params *params, int32_t atlas_w, int32_t atlas_h,
                      int32_t n_charts, const uint32_t *offsets, const int32_t *verts,
                      int32_t n_verts, tabi_placement *out, int32_t *out_k, void *stream);

/* Same as tabi_pack with DEVICE pointers for offsets, verts and out; out_k
 * is a host pointer. */
tabi_status tabi_pack_device(tabi_ctx *ctx, const tabi_params *params, int32_t atlas_w,
                             int32_t atlas_h, int32_t n_charts, const uint32_t *offsets,
                             const int32_t *verts, int32_t n_verts, tabi_placement *out,
                             int32_t *out_k, void *stream);

/* One atlas of a batch (tabi_pack_batch, tabi_pack_batch_device): the
 * arguments of tabi_pack in one record.  atlas_w .. out are inputs (out is
 * the caller's placement buffer); scale_k and status are written by the
 * call: status is this atlas's tabi_status (TABI_OK, TABI_ERR_NO_FIT,
 * TABI_ERR_INVALID_ARG or TABI_ERR_OOM) and scale_k its k (0 unless OK). */
typedef struct tabi_request {
  int32_t atlas_w, atlas_h;
  int32_t n_charts, n_verts;
  const uint32_t *offsets; /* [n_charts + 1], offsets[0] = 0, last = n_verts */
  const int32_t *verts;    /* [2 * n_verts] (Q.8)                            */
  tabi_placement *out;     /* [n_charts], input order                        */
  int32_t scale_k;         /* out                                           */
  int32_t status;          /* out                                           */
} tabi_request;

/* Pack many independent atlases of uneven size together (the batched form:
 * every stage runs once over all atlases, each wave of candidate scales
 * over the atlases still searching).  Each atlas gets exactly the result
 * tabi_pack would give it alone.  HOST pointers in the requests; the
 * inputs are copied to the device on `stream`, the results back (pinned
 * buffers by the copy kernel, as for tabi_pack).
 * 1 <= n_reqs <= TABI_MAX_BATCH.  The launch sequence is captured once per
 * launch shape (fan-out, chunks, shared-memory class) into a CUDA graph
 * owned by the context and replayed for every later batch; its waves run
 * in a device-side loop (a conditional WHILE node) that stops as soon as
 * no atlas has a candidate left to try, so later waves cost nothing.  A request that fails
 * the host checks gets TABI_ERR_INVALID_ARG and takes no device work.
 * Returns TABI_OK when every request has its status (which may itself be
 * an error), else TABI_ERR_INVALID_ARG (bad params, n_reqs or pointers),
 * TABI_ERR_OOM (the per-chart arrays do not fit the arena), TABI_ERR_CUDA
 * or TABI_ERR_BUSY, and then no request status is meaningful.  The arena
 * a batch needs is at most the sum of tabi_arena_bytes of its atlases. */
tabi_status tabi_pack_batch(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs,
                            int32_t n_reqs, void *stream);

/* Same with DEVICE pointers for offsets, verts and out (reqs itself is host
 * memory). */
tabi_status tabi_pack_batch_device(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs,
                                   int32_t n_reqs, void *stream);

/* Launch shape of a batch, chosen by tabi_autotune.  None of the knobs
 * changes a result. */
typedef struct tabi_tuning {
  int32_t scale_fanout;      /* candidates per wave                          */
  int32_t raster_warp_items; /* warp-items of a raster wave (sets how many
                                consecutive candidates one warp walks)       */
  int32_t rowloop_threads;   /* threads per row-loop CTA: 1024 or 512        */
  int32_t rowloop_ctas;      /* row-loop CTAs per multiprocessor: 1 or 2     */
  int32_t chunks;            /* chart chunks per wave: 4, 6 or 8 (lazy: a
                                candidate that fails gets no envelopes for
                                the charts after its failing row's chunk; 4
                                is the default for a batch) or 1 (the
                                default for one atlas)                       */
  int32_t progressive_bound; /* 1: a candidate stops as soon as the charts
                                not yet placed cannot fit under its
                                frontline by area (an exact test; the
                                default for a batch), 0: only when its rows
                                overflow (the default for one atlas)         */
  float ms;                  /* device time of one batch with this shape     */
} tabi_tuning;

/* Autotuner: packs the batch (DEVICE pointers, as tabi_pack_batch_device)
 * repeatedly under candidate launch shapes, starting from the default --
 * fan-out 64/16/8/4/2/1, then raster warp-items 16K/64K, then 512-thread
 * row-loop CTAs two per multiprocessor, then the other chunkings (one,
 * four, six or eight chart chunks per wave), then the progressive area bound
 * switched the other way -- times each (CUDA events, second
 * run of each), drops any shape under which some atlas ends with another
 * status (an arena too small for a wide wave), and keeps the fastest for
 * this kind of batch (atlas count, mean chart count and widest atlas in
 * powers of two, gutter, flags): later batches of the kind use it when
 * params->scale_fanout is 0.  The requests end with the results of the
 * chosen shape, the same as one tabi_pack_batch_device call.  *out (may be
 * NULL) receives the choice.  Returns as tabi_pack_batch_device. */
tabi_status tabi_autotune(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs, int32_t n_reqs,
                          void *stream, tabi_tuning *out);

/* tabi_pack_batch (device_pointers = 0) or tabi_pack_batch_device
 * (device_pointers = 1) under an explicit launch shape instead of the
 * tuned or default one (params->scale_fanout is ignored; shape->ms too):
 * for reproducible timing and for tests, since no shape changes a result.
 * scale_fanout 1..64, raster_warp_items >= 1, rowloop_threads 512 or 1024,
 * rowloop_ctas 1 or 2 (2 only with 512 threads and only if two CTAs fit a
 * multiprocessor; else 1), chunks 1..8, progressive_bound 0 or 1; anything
 * else is TABI_ERR_INVALID_ARG.  Returns as tabi_pack_batch. */
tabi_status tabi_pack_batch_shaped(tabi_ctx *ctx, const tabi_params *params, tabi_request *reqs,
                                   int32_t n_reqs, void *stream, int32_t device_pointers,
                                   const tabi_tuning *shape);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of requests as they arrive.
 *
 * A server owns a device-memory budget (arena_bytes, one allocation) split
 * evenly into `lanes`; each lane is a packing context with its own stream.
 * Submitted requests queue in arrival order; whenever a lane is idle a
 * worker thread takes requests from the head of the queue -- as many as the
 * lane's arena admits (the request's arena estimate at the server's
 * fan-out), at most max_batch -- stages them in pinned memory and launches
 * them as one batch.  Batches of different lanes overlap on the GPU, so
 * requests arriving while others run start as soon as a lane frees up.
 * Every request gets exactly the result tabi_pack would give it alone.
 * A request whose estimate exceeds a lane's arena fails with TABI_ERR_OOM.
 * -------------------------------------------------------------------- */
typedef struct tabi_server tabi_server;

typedef struct tabi_server_config {
  int32_t device;      /* CUDA device                                        */
  int32_t lanes;       /* batches in flight at once, 1..64 (4)               */
  int32_t max_batch;   /* requests per batch, 1..TABI_MAX_BATCH (64)         */
  int32_t check;       /* 1: count overlaps and gutter violations of every
                          result on the device behind its batch
                          (tabi_result.*_texels; the default), 0: not      */
  size_t arena_bytes;  /* device memory budget, split over the lanes (8 GiB) */
  tabi_params params;  /* for every request; scale_fanout 1..64 (8)          */
} tabi_server_config;

/* Completion record of one request; times in ns on the host's steady
 * clock, from the server's creation: submitted, batch launched, result
 * handed over. */
typedef struct tabi_result {
  int32_t status;  /* tabi_status of the request (as in tabi_request)        */
  int32_t scale_k;
  int64_t t_submit_ns, t_start_ns, t_done_ns;
  /* with tabi_server_config.check: the result's tabi_quality counts (all 0
     for a correct packing); -1 when unchecked (check off, an error status,
     or no room for the counter's planes) */
  int64_t overlap_texels, gutter_texels, outside_texels;
} tabi_result;

typedef struct tabi_server_stats {
  int64_t submitted, launched, completed; /* requests                        */
  int64_t batches, max_batch;             /* batches launched, largest       */
  int64_t queued, busy_lanes;             /* now                             */
  int64_t checked, check_violations;      /* results counted by the overlap
                                             check, those with a nonzero
                                             count                          */
  int64_t check_ns;                       /* device time of the checks       */
} tabi_server_stats;

void tabi_server_config_default(tabi_server_config *cfg);
/* TABI_ERR_INVALID_ARG (bad config), TABI_ERR_CUDA (allocation). */
tabi_status tabi_server_create(tabi_server **out, const tabi_server_config *cfg);
/* Stops taking batches, fails queued requests with TABI_ERR_BUSY, waits
 * for the batches in flight (bounded: polled, at most about 60 s in all;
 * requests still running then complete with TABI_ERR_TIMEOUT), and frees
 * everything -- except, if a batch is still running after that bound, the
 * device memory and pinned staging it may still touch, which stay
 * allocated. */
void tabi_server_destroy(tabi_server *srv);
/* Queue a request (HOST pointers; offsets, verts and out must stay valid
 * until the request completes; out is written when it completes with
 * TABI_OK).  *ticket identifies it.  The host checks the request before
 * reading its vertices: chart count in [1, TABI_MAX_CHARTS], non-NULL
 * buffers, offsets from 0 to n_verts with at least three vertices per
 * chart; a request that fails them completes at once with
 * TABI_ERR_INVALID_ARG, one whose arena estimate exceeds a lane with
 * TABI_ERR_OOM.  Returns TABI_OK (also for such a request: the ticket
 * carries its status), TABI_ERR_INVALID_ARG for NULL arguments,
 * TABI_ERR_BUSY while shutting down.  Thread-safe. */
tabi_status tabi_submit(tabi_server *srv, const tabi_request *req, uint64_t *ticket);
/* TABI_OK and *res filled (the ticket is released) if the request has
 * completed, TABI_PENDING if not, TABI_ERR_INVALID_ARG for an unknown
 * ticket.  Never blocks on the device. */
tabi_status tabi_poll(tabi_server *srv, uint64_t ticket, tabi_result *res);
/* As tabi_poll, waiting at most timeout_ms: TABI_ERR_TIMEOUT if the request
 * has not completed by then (the ticket stays valid). */
tabi_status tabi_wait(tabi_server *srv, uint64_t ticket, int32_t timeout_ms, tabi_result *res);
tabi_status tabi_server_get_stats(tabi_server *srv, tabi_server_stats *out);

/* Intermediate results of the last pack on this context, copied to host
 * memory for inspection and step-by-step testing; tabi_inspect_atlas
 * selects request `atlas` of the last batch (tabi_inspect = atlas 0).
 * n = that atlas's chart count; `what` selects:
 *   TABI_INSPECT_CHARTS  tabi_chart_info[n], input order (prep, Sec. 3.1,
 *                        Sec. 4.1.1, App. A);
 *   TABI_INSPECT_PERM    int32[n]: input index of each sorted position;
 *   TABI_INSPECT_ENV     for candidate index `scale` (k = 16*(scale+1);
 *                        at most the top candidate of REGIONS, else
 *                        TABI_ERR_INVALID_ARG):
 *                        int64[2] (words of the atlas's column and row
 *                        regions), int32[4n] meta per sorted chart (padded
 *                        width w', padded height h', column start, max
 *                        bottom), int32[n] row start per sorted chart, the
 *                        column region (uint32, Top' | Bot' << 16 per
 *                        padded column, chart s from its column start) and
 *                        the row region (uint32, L' | R' << 16 per padded
 *                        row, chart s from its row start);
 *   TABI_INSPECT_REGIONS int64[64][2] region starts in the column and row
 *                        pools, then int64[64][2] region words, per
 *                        candidate, then int64 top candidate index (the
 *                        largest the area bound allows, -1 if none; regions
 *                        exist for the candidates up to it), then int64
 *                        waves the last pack ran, int64 prep lanes per
 *                        chart it used, int64 padded scanline words
 *                        (columns + rows over every chart and candidate)
 *                        its raster evaluated and int64 the column words
 *                        among them (all four batch-wide);
 *   TABI_INSPECT_PAIRS   int32[n] compacting distance d(s, s+1) then
 *                        uint8[n] flags (bit0 CannotMoveAbove(s, s+1),
 *                        bit1 CannotMoveAbove(s+1, s)) for `scale`;
 *   TABI_INSPECT_SCALE   int32[12]: success, rows, knee-folded rows,
 *                        knees found, final max frontline, charts placed,
 *                        evaluated (0 not run: above the area bound or
 *                        moot; 1 ran to its end; 2 abandoned once it could
 *                        no longer win), rows pushed by the prefix-sum
 *                        tail (topt_permille), the tail's scale k' (0:
 *                        none), its first sorted chart (n: none), two
 *                        unused; then uint64[2] (low, high) the sum over
 *                        the charts of twice their area (Q.8^2) times
 *                        their scale (set on success: the quantity the
 *                        search maximises, Sec. 4.4)
 *                        -- then int32[4n] per sorted chart: x, y, row,
 *                        bits (bit0 mirror, bit1 compacting on, bit2
 *                        knee-folded, bit3 folded by the prefix sum) for
 *                        `scale` (the tail's charts at k': their envelopes
 *                        in TABI_INSPECT_ENV and pairs in
 *                        TABI_INSPECT_PAIRS are those at k' too).
 * Only candidates the last pack ran to their end are meaningful (all of
 * them with TABI_F_EVAL_ALL and scale_fanout 64; with a smaller fan-out a
 * later wave reuses the envelope regions).  *needed receives the byte
 * count; nothing is copied if cap is too small (TABI_ERR_INVALID_ARG). */
enum {
  TABI_INSPECT_CHARTS = 1,
  TABI_INSPECT_PERM = 2,
  TABI_INSPECT_ENV = 3,
  TABI_INSPECT_REGIONS = 4,
  TABI_INSPECT_PAIRS = 5,
  TABI_INSPECT_SCALE = 6
};
tabi_status tabi_inspect(tabi_ctx *ctx, int32_t what, int32_t scale, void *host_dst, size_t cap,
                         size_t *needed);
tabi_status tabi_inspect_atlas(tabi_ctx *ctx, int32_t atlas, int32_t what, int32_t scale,
                               void *host_dst, size_t cap, size_t *needed);

/* Per-stage device time of the packs run on this context (CUDA events
 * recorded on each pack's stream around every stage).  enable = 1 starts
 * collection (and clears the totals), 0 stops it; with a non-NULL stage_ms
 * the accumulated milliseconds are copied out before the state changes:
 *   stage_ms[0..7] = prep, sort, layout (with the waves' plans), raster,
 *                    hcompact, rowloop, select, whole pack;
 *   launches[0..7] = event-timed launches of each;
 *   *packs = packs timed.
 * Timing adds event records between kernels; leave it off otherwise. */
tabi_status tabi_stage_times(tabi_ctx *ctx, int32_t enable, double *stage_ms, int64_t *launches,
                             int64_t *packs);

/* Quality check of a packing: the paper's overlap metric (App. B: texels
 * covered by two or more charts, with and without the gutter dilation),
 * counted on the device.  A texel (c, r) is covered by a placed chart iff
 * its open square (c, c+1) x (r, r+1) meets the chart (see "Placement
 * semantics"; each chart drawn at its placement's k); the dilated cover
 * adds every texel within g (Chebyshev) of one and lies in the padded atlas
 * (W + 2g) x (H + 2g), as the packer's gutters do.  A correct packing has
 * all three counts 0. */
typedef struct tabi_quality {
  int64_t overlap_texels; /* atlas texels covered by two or more charts      */
  int64_t gutter_texels;  /* padded texels covered by two or more dilated
                             covers (gutter violations)                     */
  int64_t outside_texels; /* cover texels outside [0, W) x [0, H)            */
} tabi_quality;

/* Count them for one atlas: DEVICE pointers offsets[n + 1], verts[2 nv]
 * (as for tabi_pack_device) and place[n] (input order, e.g. the output of
 * a pack); *out is host memory.  Uses the context's arena for its bit
 * planes (4 bits per padded texel) and 48 bytes per chart (TABI_ERR_OOM if
 * they do not fit) and so
 * ends the inspectability of the last pack (tabi_inspect returns
 * TABI_ERR_INVALID_ARG until the next one).  Synchronous on `stream`.
 * Returns TABI_OK, TABI_ERR_INVALID_ARG, TABI_ERR_OOM, TABI_ERR_CUDA or
 * TABI_ERR_BUSY. */
tabi_status tabi_check_packing_device(tabi_ctx *ctx, int32_t atlas_w, int32_t atlas_h, int32_t gutter,
                                      int32_t n_charts, const uint32_t *offsets, const int32_t *verts,
                                      int32_t n_verts, const tabi_placement *place, tabi_quality *out,
                                      void *stream);

/* Measurement aid (no counterpart in the paper): the device's rate of the
 * 32-bit integer operation mix the envelope rasterizer is made of (add,
 * min, max, multiply-high, exclusive or, compare-select, subtract), in
 * operations per second over all multiprocessors, best of five timed runs
 * (CUDA events) of a kernel with eight independent chains per thread.  It
 * is the peak the rasterizer's integer-issue roofline is taken against.
 * Allocates 4 bytes of device memory for the run.  Returns TABI_OK,
 * TABI_ERR_INVALID_ARG or TABI_ERR_CUDA. */
tabi_status tabi_measure_int_rate(int32_t device, double *ops_per_second);

/* Height sort with no device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- engines
 * and interactive tools that own a fixed, pre-budgeted device memory pool
 * and forbid allocations outside it, or frame loops where an allocation
 * (which may synchronise the device) would stall the frame.
 *
 * Sorts chart indices 0..n-1 by decreasing height, ties in index order --
 * the same order the pack uses.  DEVICE buffers, owned by the caller:
 *   heights[n]  chart heights (Q.8), expected in [0, 2^21); values outside
 *               are clamped into that range;
 *   perm[n]     output: perm[s] = index of the chart at sorted position s.
 * The sort's scratch is a fixed device array inside the library (1 MiB,
 * kept on every GPU that loads the library until the process exits), so
 * n is limited to 65,536: larger n returns TABI_ERR_INVALID_ARG, as does a
 * NULL pointer or n < 1.  The call allocates nothing and is asynchronous on
 * `stream` (NULL = legacy default stream); synchronise before reading perm.
 * The first call on each device looks up the scratch array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call shares the one scratch array,
 * so calls that overlap on the GPU (concurrent streams) race: serialise
 * them.  Returns TABI_OK, TABI_ERR_INVALID_ARG or TABI_ERR_CUDA (launch or
 * address lookup failed).  CUDA errors are read with cudaPeekAtLastError,
 * never cleared on another's behalf: if an error from earlier work is
 * already pending on the calling thread the call launches nothing and
 * returns TABI_ERR_CUDA, leaving that error in place for its owner; an
 * error raised by this call's own launch is cleared and returned as
 * TABI_ERR_CUDA. */
tabi_status tabi_sort_heights_noalloc(const int32_t *heights, int32_t n, int32_t *perm, void *stream);

/* Per-chart record of the prep step (TABI_INSPECT_CHARTS). */
typedef struct tabi_chart_info {
  int32_t orig, Wq, Hq, rot90, flip_y, flip_x, obb_m, valid;
  int64_t u0, u1, v0, v1;                      /* OBB strips at angle obb_m */
  int32_t ylo[10], yhi[10], xlo[10], xhi[10]; /* final local AABBs: y
                                                 extremes of the x-slices,
                                                 x extremes of the y-slices
                                                 (merged per scanline,
                                                 Sec. 4.1.1)              */
  int64_t area_top, area_bot, area_left, area_right, area_bl2, area_br2;
} tabi_chart_info;

#ifdef __cplusplus
}
#endif
#endif /* TABI_H */
