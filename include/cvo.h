/*
 * cvo.h -- C ABI of the GB300 (sm_103a) implementation of Continuous Visual
 * Odometry (Ghaffari, Clark, Bloch, Eustice, Grizzle, "Continuous Direct
 * Sparse Visual Odometry from RGB-D Images", arXiv 1904.02266).
 *
 * Two coloured point clouds become functions in an RKHS and the relative pose
 * is found by gradient ascent on their inner product (Problem 1, Eq. max):
 *
 *   F(P) = sum_ij c_ij k(x_i, R z_j + T),   k(x,y) = sigma^2 exp(-|x-y|^2 / 2 ell^2)
 *
 * X = {x_i} is the TARGET (fixed) cloud and Z = {z_j} the SOURCE (moving)
 * cloud. A pose P is a row-major 4x4 double matrix [R T; 0 1] that maps source
 * coordinates into the target frame; it is the paper's h^{-1} (Sec. 3, where
 * z~_j = h^{-1} z_j). The solver updates P <- exp(t xi) P (the paper's
 * h <- h exp(t xi) with xi negated, Eq. newstep), so gradients returned here
 * are ascent directions for that left update.
 *
 * All entry points return an int status: CVO_OK (0) or a negative CVO_ERR_*
 * code; cvo_strerror() names it and cvo_last_error() gives the context's
 * detail message. Nothing throws across this boundary. Calls on one context
 * are serialised by an internal lock; use one context per host thread for
 * concurrency.
 *
 * Memory: every host array is read during the call and stays owned by the
 * caller. With CVO_DEVICE_PTR the arrays are device pointers on the context's
 * device; they are read on the given stream (or the context stream when NULL)
 * before the call returns and are never freed by the library. Clouds are
 * copied into library-owned device memory, accounted against the context's
 * HBM budget, and live until cvo_release_cloud or cvo_destroy.
 */
#ifndef CVO_H
#define CVO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CVO_OK 0
#define CVO_ERR_INVALID_ARG (-1)   /* bad size, pointer, handle or non-finite input */
#define CVO_ERR_OUT_OF_BUDGET (-2) /* the HBM budget given to cvo_create is exhausted */
#define CVO_ERR_CUDA (-3)          /* a CUDA runtime call failed (see cvo_last_error) */
#define CVO_ERR_TIMEOUT (-4)       /* a bounded wait expired */
#define CVO_ERR_BUSY (-5)          /* no free request slot */
#define CVO_ERR_NOT_FOUND (-6)     /* unknown cloud handle or ticket */
#define CVO_ERR_INTERNAL (-7)      /* broken internal invariant */

/* ---- label inner product c_ij (Sec. 2 remark defining c_ij) ------------- */
#define CVO_COLOR_NONE 0   /* c_ij = 1 */
#define CVO_COLOR_KERNEL 1 /* c_ij = exp(-|f_i - g_j|^2 / 2 ell_color^2) (appearance kernel) */
#define CVO_COLOR_DOT 2    /* c_ij = color_scale <f_i, g_j>, the paper's choice (Sec. 5 remark) */

/* ---- lengthscale schedule ---------------------------------------------- */
#define CVO_SCHEDULE_DECAY 0  /* ell_{k+1} = max(ell_k * ell_decay, ell_min) */
#define CVO_SCHEDULE_TABLE1 1 /* Table 1: 0.15, then 0.10 after iteration 3, 0.06 after 10, 0.03 after 20 */

/* ---- cvo_set_cloud flags ----------------------------------------------- */
#define CVO_DEVICE_PTR 1u /* xyz / feat are device pointers */

#define CVO_MAX_FEAT 8    /* largest feature (label) dimension */

typedef struct cvo_ctx cvo_ctx;

/* Solver parameters. cvo_params_default() fills the defaults given here. */
typedef struct {
    double ell0;        /* initial spatial lengthscale [m]; 0.15 (Table 1) */
    double ell_decay;   /* per-iteration factor for CVO_SCHEDULE_DECAY; 0.9 */
    double ell_min;     /* floor of the decay schedule; 0.02 */
    int schedule;       /* CVO_SCHEDULE_*; DECAY */
    double sigma;       /* kernel signal std: k = sigma^2 exp(...); 1.0 */
    double kcut;        /* sparsification (Sec. 5): pairs with exp(-d^2/2ell^2) < kcut
                           are dropped, i.e. d > ell sqrt(2 ln(1/kcut)); 1e-3. Must be
                           in (0, 1): the cell list needs a finite radius. */
    int color_mode;     /* CVO_COLOR_*; KERNEL */
    double ell_color;   /* appearance lengthscale for CVO_COLOR_KERNEL; 0.1 */
    double color_scale; /* scale s for CVO_COLOR_DOT; 1e-5 (Sec. 5 remark) */
    double a2, b2;      /* metric weights of Eq. metric (n = 3): a^2 |omega|^2 + b^2 |v|^2; 1, 1 */
    int max_iters;      /* iteration cap; 200 */
    double eps_pose;    /* stop when |t xi| < eps_pose at the lengthscale floor; 1e-5 (Table 1) */
    double eps_grad;    /* ... or when |xi| < eps_grad there; 5e-5 (Table 1) */
    int step_order;     /* 4: first maximiser of the quartic Taylor model (Eq. fourth); 2: quadratic */
    int feat_dim;       /* feature dimension D in [0, CVO_MAX_FEAT]; 5. 0 forces COLOR_NONE */
    int feat_bf16;      /* 1: store the (pre-scaled) features as BF16, rounded to nearest even,
                           and widen them to FP32 in the pair arithmetic (half the feature bytes;
                           the label product then carries BF16 rounding); 0: FP32. Not used by
                           cvo_eval_gradient_static. 0 */
    int reduce_fp32;    /* precision study only: 1 sums the block partials and the cross-block
                           reduction in FP32 instead of FP64 (pair arithmetic and tail unchanged);
                           0 */
    double cell_factor; /* cell edge of the target grid as a multiple of the cutoff radius, in
                           [0.5, 8]; 0.7. Performance only: the cutoff test is exact. */
    /* performance tuning (results do not depend on these): */
    double cluster_factor; /* source cluster (octree node) edge as a multiple of the cell edge,
                              capped so a cluster spans at most 8 x 8 cell rows; 2.0 */
    int cost_chunk;        /* work split: per-chunk overhead in pair-test units; 48 */
    int cost_cluster;      /* work split: cost of staging one cluster in pair-test units; 32 */
    double cost_kept;      /* work split of a reused plan: cost of a kept pair in pair-test
                              units, from the kept pairs counted by the plan's first gradient
                              pass (the split is redone once, at the plan's second iteration);
                              0 disables the rebalance; 0 */
    double team_factor;    /* batches and served requests: a pair's team gets about
                              team_factor * (its share of the estimated pair work) of the
                              blocks, at least one; 4.0 */
    /* failure bounds of the device-side waits (Sec. 4's solve runs as one
       persistent launch whose blocks wait on each other; every wait is
       bounded so that a lost block ends the solve with CVO_ERR_TIMEOUT
       instead of hanging the GPU): */
    int wait_polls;        /* polls of a team barrier before a block gives up, in [1, 2^30]
                              (each poll sleeps about 0.5 us); 4194304 (about 2 s) */
    double join_limit_ms;  /* how long a queued pair's first block waits for the rest of its
                              team to start, in (0, 1e7] ms; 60000 */
} cvo_params;

/* One evaluation at a fixed pose (cvo_eval). */
typedef struct {
    double F;          /* F = sum_ij c_ij k_ij over kept pairs (Eq. scalar) */
    double grad6[6];   /* metric gradient xi = (omega, v): dF/domega / a^2, dF/dv / b^2
                          (Eq. 3_gradient under the left update) */
    double S[5];       /* S0..S4: G(t) = F(exp(t xi) P) ~ S0 + S1 t + ... + S4 t^4 along
                          xi = grad6 (Eq. fourth) */
    int64_t nnz;       /* pairs kept (d <= r_c) in the gradient pass */
    int64_t candidates;/* candidate pairs visited by the cell-list traversal */
} cvo_eval_result;

/* Statistics of one solve (cvo_align, cvo_poll). */
typedef struct {
    int iters;            /* iterations run */
    int converged;        /* 1 if the Table 1 test fired before max_iters */
    int fallback_steps;   /* iterations whose quartic had no maximiser on t > 0 */
    int no_ascent_steps;  /* iterations with S1 <= 0 (no step taken) */
    double final_ell;     /* lengthscale of the last iteration */
    double F_last;        /* F at the last evaluated pose */
    double t_last;        /* last step length */
    int64_t pair_evals;   /* kept pairs summed over every gradient and step pass */
    int64_t candidates;   /* candidate pairs visited over every pass */
    int status;           /* CVO_OK or the error that ended the solve */
    double device_ms;     /* device time of the solve (global timer, from the moment all
                             blocks of its team had started to the published result) */
} cvo_stats;

/* Fill *p with the defaults listed in cvo_params. */
void cvo_params_default(cvo_params* p);

/* Create a context on CUDA device `device` with its own stream. Device memory
 * the context allocates for clouds, grids and solves is limited to
 * hbm_budget_bytes (0 = no limit). Returns CVO_ERR_INVALID_ARG for bad
 * parameters, CVO_ERR_CUDA if the device cannot be used. */
int cvo_create(const cvo_params* params, int device, size_t hbm_budget_bytes, cvo_ctx** out);

/* Free every resource of the context (clouds, grids, graphs, stream). */
int cvo_destroy(cvo_ctx* ctx);

/* Upload a cloud: xyz is n x 3 float32 (row-major), feat is n x feat_dim
 * float32 (ignored, may be NULL, when feat_dim == 0 or color_mode is NONE).
 * The library centres the cloud on its FP64 centroid, packs it
 * structure-of-arrays, orders it along a Morton curve for use as a source, and
 * builds the target cell lists lazily. It returns once xyz and feat have been
 * read (the caller may reuse them); the packing and ordering finish in order
 * on the context's stream, before any later call uses the cloud, so a fault
 * there would be reported by that later call. Errors: CVO_ERR_INVALID_ARG for n <= 0,
 * n > 2^22, NULL pointers or any non-finite value (checked on the device);
 * CVO_ERR_OUT_OF_BUDGET if the copy would exceed the budget. */
int cvo_set_cloud(cvo_ctx* ctx, const float* xyz, const float* feat, int64_t n, uint32_t flags,
                  void* stream, int32_t* handle_out);

/* Release a cloud and every cached grid and plan that uses it. */
int cvo_release_cloud(cvo_ctx* ctx, int32_t handle);

/* One gradient pass and one step pass at pose P and lengthscale ell
 * (Eqs. scalar, 3_gradient, metric, fourth). Synchronous: results are in
 * *out when it returns. */
int cvo_eval(cvo_ctx* ctx, int32_t target, int32_t source, const double P[16], double ell,
             cvo_eval_result* out);

/* Set the failure bounds of the device-side waits (cvo_params.wait_polls and
 * join_limit_ms) of the context and of every plan and batch it already holds;
 * later solves, evaluations and batch runs use them. The paper has no
 * counterpart: the solve of Problem 1 runs as one persistent launch whose
 * blocks wait on each other, and these bounds turn a lost block into
 * CVO_ERR_TIMEOUT instead of a hung GPU. Synchronous. Errors:
 * CVO_ERR_INVALID_ARG for values outside the ranges in cvo_params,
 * CVO_ERR_BUSY while the request loop runs. */
int cvo_set_wait_limits(cvo_ctx* ctx, int wait_polls, double join_limit_ms);

/* Full solve from P0 (Problem 1; Eqs. flow, fourth, newstep, step): gradient,
 * step sums, quartic step and exponential-map update per iteration, with the
 * lengthscale schedule of the context. The whole loop runs on the device in
 * one persistent cooperative kernel launch. Synchronous. P_out receives the
 * final pose; stats (may be NULL) the solve statistics. Returns
 * CVO_ERR_TIMEOUT if a bounded device-side barrier wait expired. */
int cvo_align(cvo_ctx* ctx, int32_t target, int32_t source, const double P0[16],
              double P_out[16], cvo_stats* stats);

/* Per-iteration record of cvo_align_profile. */
typedef struct {
    double ell;               /* lengthscale of the iteration */
    float plan_ms;            /* time spent rebuilding the traversal plan (0 when it was reused) */
    float grad_ms;            /* gradient pass, including its FP64 reduction and tail */
    float step_ms;            /* step pass, including the step length and pose update */
    float grad_pass_ms;       /* part of grad_ms before the barrier that ends the pass (first block) */
    float grad_sync_ms;       /* part of grad_ms up to the end of that barrier */
    float step_pass_ms;       /* the same two points for the step pass */
    float step_sync_ms;
    int replanned;            /* 1 if the traversal plan was rebuilt in this iteration */
    int64_t grad_pairs;       /* pairs kept in the gradient pass */
    int64_t step_pairs;       /* pairs kept in the step pass */
    int64_t grad_candidates;  /* candidates visited in the gradient pass */
    int64_t step_candidates;  /* candidates visited in the step pass */
} cvo_iter_profile;

/* The same solve as cvo_align (same kernel and results) with per-iteration
 * phase timings, taken on the device from the global nanosecond timer by the
 * first block of the solve kernel. Writes min(iters, max_records) records and
 * the count to *n_records (may be NULL). */
int cvo_align_profile(cvo_ctx* ctx, int32_t target, int32_t source, const double P0[16],
                      double P_out[16], cvo_stats* stats, cvo_iter_profile* records,
                      int max_records, int* n_records);

/* The context's CUDA stream (cudaStream_t), on which every kernel of the
 * context runs; NULL for a NULL context. */
void* cvo_stream(cvo_ctx* ctx);

/* ---- batches: many uneven pairs in one persistent launch ---------------- */

typedef struct cvo_batch cvo_batch;

/* Describe a batch of n independent solves, pair i aligning source[i] to
 * target[i] (resident cloud handles; a handle may appear in several pairs).
 * ell0 (may be NULL) gives each pair its own initial lengthscale for the
 * context's schedule. team_sizes (may be NULL) fixes how many blocks solve
 * each pair; otherwise the library estimates each pair's kept-pair work from
 * the point counts, the target's extent and the schedule, and gives it
 * max(1, ceil(team_factor * share * blocks)) blocks. Pairs are queued largest
 * first; blocks of one persistent cooperative kernel claim them as they come
 * free, so small pairs fill in around large ones. The call builds every cell
 * list, cluster set and per-pair plan the solves need and captures the launch
 * (pose upload, kernel, result download) in a CUDA graph. The clouds of a
 * batch cannot be released (CVO_ERR_BUSY) until the batch is destroyed.
 * Errors: CVO_ERR_INVALID_ARG (n < 1, NULL arrays, team size outside
 * [1, blocks], ell0 <= 0), CVO_ERR_NOT_FOUND (unknown handle),
 * CVO_ERR_OUT_OF_BUDGET. */
int cvo_batch_create(cvo_ctx* ctx, int n, const int32_t* targets, const int32_t* sources,
                     const double* ell0, const int32_t* team_sizes, cvo_batch** out);

/* Run every solve of the batch from the poses P0 (n row-major 4x4 doubles).
 * Synchronous. P_out receives n final poses, stats (may be NULL) n records
 * whose status field is that pair's own outcome. Each pair runs the same
 * iteration as cvo_align (same schedule, step rule and stopping test); only
 * the order of the FP64 sums over blocks differs with the team size.
 * Returns the first failing pair's status, else CVO_OK. */
int cvo_batch_run(cvo_ctx* ctx, cvo_batch* batch, const double* P0, double* P_out,
                  cvo_stats* stats);

typedef struct {
    int pairs;          /* pairs in the batch */
    int blocks;         /* blocks of the persistent launch */
    int graph;          /* 1 if the launch is replayed from a captured CUDA graph */
    int max_team;       /* largest team */
    int64_t bytes;      /* device memory held by the batch (plans, states, queue) */
} cvo_batch_info;

/* Shape of a batch; team_sizes (may be NULL) receives the n team sizes in
 * the caller's pair order. */
int cvo_batch_get_info(cvo_ctx* ctx, const cvo_batch* batch, cvo_batch_info* info,
                       int32_t* team_sizes);

/* Free the batch's plans, states and graph. */
int cvo_batch_destroy(cvo_ctx* ctx, cvo_batch* batch);

/* ---- request loop: continuous batching of frame-pair solves -------------- */

/* One request: align a new frame (the source) to a resident keyframe (the
 * target). The frame arrays are copied before cvo_submit returns. */
typedef struct {
    int32_t target;        /* keyframe handle (cvo_set_cloud); kept resident with its cell lists */
    const float* xyz;      /* frame points, n x 3 host float32 */
    const float* feat;     /* frame features, n x feat_dim host float32 (may be NULL when
                              feat_dim == 0 or color_mode is NONE) */
    int64_t n;             /* 1 <= n <= 2^22 */
    double P0[16];         /* initial pose, row-major, mapping the frame into the keyframe */
    double ell0;           /* initial lengthscale; 0 = the context's */
} cvo_request;

/* Outcome of one request (cvo_poll). */
typedef struct {
    double P[16];          /* final pose */
    cvo_stats stats;       /* solve statistics; stats.status is the request's status */
    double queue_ms;       /* cvo_submit until the request was admitted (memory reserved) */
    double latency_ms;     /* cvo_submit until the result was ready */
} cvo_result;

typedef struct {
    int reserve_blocks;    /* block slots of the solve kernel's full occupancy that the
                              serving kernel leaves free, so that the kernels preparing new
                              frames can run while solves do (a block slot is one SM);
                              >= 1; 4 */
    int max_inflight;      /* requests admitted to the device at once, in [1, 65536]; 1024 */
    double linger_ms;      /* the serving kernel stays resident this long without work; 0.5 */
    double idle_limit_ms;  /* device-side bound on the serving kernel's wait for new requests:
                              past it the kernel exits by itself (counted in idle_exits) even if
                              the host never told it to; > 0; 10000 */
    double team_factor;    /* a request's team gets about team_factor * (its share of the
                              estimated work in the system) of the serving kernel's blocks, at
                              least one; in (0, 1024]; 6.0 (cvo_params.team_factor sizes the
                              teams of batches) */
} cvo_serve_params;

typedef struct {
    int64_t submitted;        /* requests accepted by cvo_submit */
    int64_t completed;        /* requests finished (successfully or not) */
    int64_t failed;           /* requests finished with a status other than CVO_OK */
    int64_t kernels_launched; /* serving kernels started (one per busy period) */
    int64_t idle_exits;       /* serving kernels that left on their own idle bound */
} cvo_serve_stats;

/* Fill *p with the defaults listed in cvo_serve_params. */
void cvo_serve_params_default(cvo_serve_params* p);

/* Start the context's request loop (cvo_submit starts it with the defaults
 * when it is not running). A host thread admits queued requests in arrival
 * order while the context's HBM budget allows (a request that could never
 * fit fails with CVO_ERR_OUT_OF_BUDGET; one that fits only after others
 * finish waits), uploads and prepares each frame on the context stream, and
 * hands it to one persistent cooperative kernel that stays resident while
 * there is work: its blocks claim each request's team of slots as they come
 * free, so requests that arrive while others are on the GPU start as soon as
 * blocks and memory allow, and their solves overlap. A request's team size is
 * about team_factor * (its share of the estimated work in the system) of the
 * kernel's blocks. Each solve runs the same iteration as cvo_align. While the
 * loop runs, cvo_align, cvo_align_profile, cvo_eval and cvo_batch_run return
 * CVO_ERR_BUSY (their kernels need the whole GPU resident). Errors:
 * CVO_ERR_BUSY if the loop already runs, CVO_ERR_INVALID_ARG for bad params. */
int cvo_serve_start(cvo_ctx* ctx, const cvo_serve_params* params);

/* Queue a request; *ticket identifies it for cvo_poll. The keyframe cannot be
 * released (CVO_ERR_BUSY) until every request naming it has been polled
 * complete. Errors: CVO_ERR_INVALID_ARG (NULL or bad fields, non-finite
 * pose), CVO_ERR_NOT_FOUND (unknown keyframe). */
int cvo_submit(cvo_ctx* ctx, const cvo_request* req, uint64_t* ticket);

/* Non-blocking: *done = 1 and *out filled (and the ticket retired) when the
 * request has finished, *done = 0 otherwise. The request's own outcome is
 * out->stats.status (CVO_OK, CVO_ERR_OUT_OF_BUDGET, CVO_ERR_TIMEOUT, ...).
 * CVO_ERR_NOT_FOUND for an unknown or already retired ticket. */
int cvo_poll(cvo_ctx* ctx, uint64_t ticket, cvo_result* out, int* done);

/* Finish every queued and running request, then stop the loop and free its
 * device resources. Results stay available to cvo_poll. */
int cvo_serve_stop(cvo_ctx* ctx);

/* Counters of the context's request loop since the context was created
 * (zeros if it never ran). */
int cvo_serve_get_stats(cvo_ctx* ctx, cvo_serve_stats* out);

/* ---- autotuner of the performance parameters ------------------------------ */

typedef struct {
    int n_cell, n_cluster, n_chunk, n_cluster_cost;  /* candidates per dimension (0: built-in set) */
    double cell_factor[8];
    double cluster_factor[8];
    int cost_chunk[8];
    int cost_cluster[8];
    int reps;               /* timed solves per candidate (the fastest counts); 3 */
} cvo_tune_space;

typedef struct {
    double start_ms;        /* solve time with the parameters the context had */
    double best_ms;         /* solve time with the chosen parameters */
    int candidates;         /* settings timed */
    double cell_factor, cluster_factor;   /* the chosen setting (also left in the context) */
    int cost_chunk, cost_cluster;
} cvo_tune_report;

/* Pick the cell size, the source cluster size and the work-split costs for
 * the context by timing whole solves of (target, source) from the identity on
 * the device (CUDA events on the context stream): coordinate descent over
 * cell_factor, cluster_factor, cost_chunk and cost_cluster, one dimension at a
 * time, keeping the fastest. Results do not depend on these parameters (the
 * cutoff test is exact); only the speed does. The context keeps the chosen
 * values; its cached plans, cell lists and clusters of the two clouds are
 * dropped and rebuilt on next use. space may be NULL (built-in candidates).
 * Errors: CVO_ERR_NOT_FOUND, CVO_ERR_BUSY (the request loop runs, or a batch
 * uses one of the clouds), CVO_ERR_INVALID_ARG (a candidate outside the
 * parameter ranges of cvo_params). */
int cvo_autotune(cvo_ctx* ctx, int32_t target, int32_t source, const cvo_tune_space* space,
                 cvo_tune_report* report);

/* ---- semi-dense front end (Sec. 5: high intensity-gradient pixels) -------- */

typedef struct {
    double fx, fy, cx, cy;        /* pinhole intrinsics [pixels]; 525, 525, 319.5, 239.5 */
    double depth_min, depth_max;  /* a pixel is valid if its depth [m] lies in this range; 0.5, 5 */
    double percentile;            /* keep the valid pixels whose intensity-gradient magnitude is
                                     above this percentile of the valid pixels' magnitudes
                                     (linear interpolation between order statistics); 80 */
    double grad_scale;            /* gradient features are clip(g / grad_scale, -1, 1); 0.05 */
    int64_t max_points;           /* when more pixels are kept, keep the ranks
                                     floor(k m / max_points) of the m kept pixels (raster order);
                                     0 = keep all */
} cvo_frontend_params;

/* Fill *p with the defaults listed in cvo_frontend_params. */
void cvo_frontend_params_default(cvo_frontend_params* p);

/* Select, back-project and describe the points of one RGB-D frame on the GPU.
 * depth is H x W float32 [m] (row-major), hsv H x W x 3 float32 (H, S, V;
 * the intensity is V); host arrays, or device arrays with CVO_DEVICE_PTR
 * (read on `stream`, NULL = the context stream). The intensity gradient is
 * taken by central differences (one-sided at the image border) in FP32, its
 * magnitude compared with the percentile threshold in FP64, and the kept
 * pixels, in raster order, are written as points x = ((u - cx) / fx) z,
 * y = ((v - cy) / fy) z, z = depth into out_xyz (n x 3) with features H, S,
 * V, clip(gx / grad_scale), clip(gy / grad_scale) into out_feat (n x 5, may be
 * NULL) and their pixel indices y W + x into out_pixel (may be NULL); all
 * three are device arrays with room for `capacity` points. *n_out receives n.
 * Errors: CVO_ERR_INVALID_ARG (image smaller than 2 x 2 or above 2^20 pixels,
 * bad parameters, no valid pixel, more points than capacity). */
int cvo_frontend_select(cvo_ctx* ctx, const float* depth, const float* hsv, int width, int height,
                        const cvo_frontend_params* params, uint32_t flags, void* stream,
                        float* out_xyz, float* out_feat, int32_t* out_pixel, int64_t capacity,
                        int64_t* n_out);

/* The same selection, uploaded as a resident cloud (as cvo_set_cloud does)
 * without leaving the device. The context's feat_dim must be 5 (or features
 * unused). *handle_out receives the cloud, *n_out (may be NULL) its size. */
int cvo_frontend_cloud(cvo_ctx* ctx, const float* depth, const float* hsv, int width, int height,
                       const cvo_frontend_params* params, uint32_t flags, void* stream,
                       int32_t* handle_out, int64_t* n_out);

/* Gradient pass for callers that must not allocate device memory during the
 * call: a program whose device memory is all owned by its own pool or fixed
 * at start-up (a real-time loop with a frozen footprint, an embedding host
 * that forbids allocation in its hot path) cannot use cvo_set_cloud, which
 * copies clouds into library-allocated buffers. This entry point allocates
 * nothing and needs no context. The paper has no counterpart: it is the
 * all-pairs form of the gradient pass (every target point against every
 * source point, with the same cutoff, label product and FP32 pair
 * arithmetic as cvo_eval), so its cost grows with n * m.
 *
 * Inputs are device pointers on the current device: d_x (n x 3 float32) and
 * d_fx (n x feat_dim) the target, d_z (m x 3) and d_fz (m x feat_dim) the
 * source (features may be NULL when feat_dim is 0 or color_mode is NONE).
 * params supplies sigma, kcut, color_mode, ell_color, color_scale, a2, b2 and
 * feat_dim; P (host, row-major 4x4) the pose; ell the lengthscale. The result
 * is written to d_out, a device array of 8 doubles: F, the metric gradient
 * (omega, v) as in cvo_eval_result.grad6, and the number of kept pairs. The
 * kernels run on `stream` (NULL: the default stream) and the call returns
 * without waiting for them.
 *
 * Scratch: block partials live in a fixed 32 KB array in the library's
 * device memory (512 slots), which every GPU that loads the library holds
 * until the process exits. Each call writes every slot it reads, so nothing
 * carries over between calls, but all calls on one device share the array:
 * calls whose kernels overlap on the GPU (different streams, or different
 * host threads) race and must be serialised by the caller. The first call on
 * each device looks up the array's device address and keeps it for the life
 * of the process; make that first call before any stream capture. A host
 * that destroys the device's primary context (cudaDeviceReset) invalidates
 * that address and must reload the library before calling again. Sizes outside 1 <= n, m <= 2^22 return
 * CVO_ERR_INVALID_ARG; so do NULL pointers and invalid parameters (a
 * color_mode other than NONE, KERNEL or DOT; ell_color <= 0 for KERNEL or
 * color_scale <= 0 for DOT when features are used). The detail
 * message of a failed call is returned by cvo_last_error(NULL) on the same
 * host thread. */
int cvo_eval_gradient_static(const float* d_x, const float* d_fx, int64_t n, const float* d_z,
                             const float* d_fz, int64_t m, const cvo_params* params,
                             const double P[16], double ell, double* d_out, void* stream);

/* Name of a status code (static string). */
const char* cvo_strerror(int status);

/* Detail message of the last failed call on this context (static until the
 * next call on the context; "" if none). With ctx == NULL: the message of the
 * last failed context-free call (cvo_eval_gradient_static) on this thread. */
const char* cvo_last_error(cvo_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CVO_H */
