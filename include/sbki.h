/* sbki.h - C ABI of libsbki, a GB300 (sm_103a) implementation of the
 * semantic Bayesian kernel inference (S-BKI) map update of Gan et al.,
 * "Bayesian Spatial Kernel Smoothing for Scalable Dense Semantic Mapping".
 *
 * The map holds, for every voxel of every allocated block, the Dirichlet
 * concentrations alpha[K+1] of Eq. (alpha_kernel): class 0 is the free class,
 * classes 1..K are the occupied semantic classes.  A scan update turns a
 * labelled point cloud into training points (Sec. III: hits plus free-space
 * samples interpolated along each beam, then voxel downsampling) and adds
 * k(x_*, x_i) y_i into every voxel centre x_* within the support l of a
 * training point x_i, with the sparse kernel of Eq. (kernel); the update is
 * recursive over scans (Sec. IV).  Read-off follows Eq. (mode), Eq. (variance)
 * and the occupancy rule of Sec. V-C.  A map can instead run the paper's
 * counting sensor model (S-CSM, Eq. (alpha); params.sensor_model = 1): the
 * same training points, each adding 1 to class y of the voxel containing it.
 *
 * Conventions shared by every entry point
 *  - Buffers are owned by the caller.  Pointer arguments may be host or device
 *    memory of the map's device (detected with cudaPointerGetAttributes);
 *    device buffers are read/written in stream order on params.cuda_stream.
 *  - Coordinates are float32, row-major [n,3] (x, y, z).  Poses are float64
 *    4x4 row-major world_from_sensor matrices.
 *  - No function aborts or traps.  Every failure is a returned sbki_status;
 *    sbki_last_error() gives a message.  On SBKI_ERR_CAPACITY and
 *    SBKI_ERR_LABEL_RANGE an insert leaves the map unchanged.
 *  - Device-side waits are bounded; nothing spins without a limit.
 */
#ifndef SBKI_H
#define SBKI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SBKI_OK = 0,
  SBKI_ERR_INVALID_ARG = 1, /* null/negative/unsupported argument or parameter */
  SBKI_ERR_LABEL_RANGE = 2, /* a label outside 1..K (scans) or 0..K (training sets) */
  SBKI_ERR_CAPACITY = 3,    /* a fixed-size pool, hash or scratch buffer would overflow */
  SBKI_ERR_CUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
  SBKI_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  SBKI_ERR_NOT_FOUND = 6    /* lookup of something that does not exist */
} sbki_status;

/* Parameters.  Defaults (sbki_default_params) follow Table (parameters):
 * l = 0.3 m, sigma0 = 0.1, alpha0 = 0.001; Sec. V-A: res = 0.1 m, free and
 * occupied thresholds 0.47 and 0.6.  Start from sbki_default_params and
 * override fields: a zeroed struct is refused (sigma0_scale must be > 0). */
typedef struct sbki_params {
  double res;          /* voxel edge [m] */
  double length_scale; /* kernel support l [m], Eq. (kernel); 0 < l <= 0.75 * block edge * res */
  double sigma0;       /* kernel scale sigma0, Eq. (kernel) */
  double alpha0;       /* Dirichlet prior alpha_0^k, equal for all K+1 classes */
  double free_step;    /* spacing of free-space samples along a beam [m], Sec. III */
  double ds_res;       /* downsampling cell edge [m]; <= 0 means res */
  double min_range;    /* hits closer than this to the sensor are dropped [m] */
  double max_range;    /* hits farther than this are dropped [m]; must be finite */
  double free_thresh;  /* p_occ below this reads as free (Sec. V-A) */
  double occ_thresh;   /* p_occ above this reads as occupied (Sec. V-A) */
  int32_t num_classes; /* K occupied classes; alpha has K+1 entries; K+1 <= 32 */
  int32_t block_edge;  /* voxels per block edge: 4 or 8 */
  int64_t pool_blocks; /* capacity of the block pool (alpha storage) */
  int64_t sample_capacity; /* max hits + free samples of one scan */
  int32_t track_pairs; /* nonzero: keep per-voxel in-support pair counts (parity aid) */
  int32_t device;      /* CUDA device ordinal */
  int32_t accumulate_mode; /* step a5 form: 0 point-major (one warp per training
                            * point, global reductions; default), 1 block-major
                            * (one CTA per touched block, shared-memory tile;
                            * also counts touched voxels in sbki_stats) */
  int32_t num_maps;    /* independent maps held by the handle (1..64, default 1);
                        * they share the block pool; see sbki_select_map and
                        * sbki_insert_batch */
  void* cuda_stream;   /* cudaStream_t for every launch and copy; NULL = legacy default stream */
  int32_t sensor_model; /* 0: kernel inference, Eq. (alpha_kernel) (default); 1: counting sensor
                         * model, Eq. (alpha): every training point adds 1 to alpha^{y_i} of the
                         * voxel floor(x * fp32(1/res)) that contains it (exact FP32 counts below
                         * 2^24 per voxel and class); length_scale and sigma0 do not enter it.
                         * Needs accumulate_mode 0; sbki_backward, sbki_backward_scales and
                         * sbki_grad refuse it */
  double sigma0_scale[32]; /* per-class kernel scale: class k's kernel is sigma0 * sigma0_scale[k]
                            * * f(d/l) (the paper's class-dependent signal variance, Sec. V);
                            * entries 0..K must be finite and > 0; sbki_default_params sets 1,
                            * which is Eq. (kernel) as printed.  Unused by the counting model */
  int32_t association; /* which (voxel, training point) pairs Eq. (alpha_kernel) sums (Sec. IV):
                        * 0 (default) every voxel centre within l of the point; 1 the paper's
                        * extended block: a voxel of block b takes the points whose own voxel lies
                        * in b or one of b's six face neighbours, so pairs reaching b from an edge
                        * or corner neighbour are left out even when d < l.  Both accumulation
                        * forms honour it; sbki_backward, sbki_backward_scales and sbki_grad
                        * refuse 1.  The counting model ignores it */
  double l_scale[32];  /* per-class length scale: class k's kernel is sigma0 sigma0_scale[k]
                        * f(d/l_k) with support d < l_k = length_scale * l_scale[k] (Sec. V and VI
                        * name class-dependent parameters; reading K16).  Entries 0..K finite and
                        * > 0, l_k <= 0.75 * block_edge * res; sbki_default_params sets 1 (the
                        * common l).  With any entry other than 1 the update takes the general
                        * weighted accumulation; the block-major form, extended-block association
                        * and the differentiable entry points refuse it */
} sbki_params;

/* Per-insert counters (all for the last insert). */
typedef struct sbki_stats {
  int64_t hits;           /* input points kept (finite, within range) */
  int64_t dropped;        /* input points dropped */
  int64_t free_samples;   /* free-space samples generated (Sec. III) */
  int64_t train_points;   /* training points after downsampling */
  int64_t touched_blocks; /* blocks with at least one in-support pair (counting model: holding a point) */
  int64_t new_blocks;     /* blocks allocated by this insert */
  int64_t pairs;          /* in-support (voxel, training point) pairs, Eq. (alpha_kernel); counting
                           * model: training points counted (one voxel each) */
  int64_t touched_voxels; /* voxels whose alpha changed (block-major mode only; 0 otherwise) */
  int64_t total_blocks;   /* blocks allocated in the map after the insert */
} sbki_stats;

typedef struct sbki_map sbki_map;

/* Fills *p with the defaults above (K = 10, block edge 8, pool 2^16 blocks,
 * 2^24 samples per scan, device 0, default stream). */
sbki_status sbki_default_params(sbki_params* p);

/* Allocates the map (block hash, alpha pool and per-scan scratch) on
 * params->device.  *out receives the handle; release with sbki_destroy_map. */
sbki_status sbki_create_map(const sbki_params* params, sbki_map** out);
void sbki_destroy_map(sbki_map* map);

/* One scan update, Sec. III + Eq. (alpha_kernel) + Sec. IV:
 *   points [n,3] sensor frame, labels [n] in 1..K, sensor_pose = world_from_sensor.
 * Hits that are non-finite or outside [min_range, max_range] are dropped and
 * counted, not an error.  Free samples lie at distance r - j*free_step from
 * the sensor origin for j >= 1 while positive.  Hits and free samples are
 * grouped per (downsampling cell, label) into centroids, and every centroid
 * adds sigma0 * f(d/l) into class y of every voxel centre with d < l (the
 * counting model: 1 into class y of its own voxel, Eq. (alpha)).
 * Synchronises the stream before returning (stats may be NULL). */
sbki_status sbki_insert_scan(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                             const double sensor_pose[16], sbki_stats* stats);

/* Same update, without the final synchronisation: errors raised on the device
 * surface at the next sbki_sync or synchronising call.  Buffers must stay
 * valid until then. */
sbki_status sbki_insert_scan_async(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                                   const double sensor_pose[16]);
/* Waits for the map's stream and returns the first pending error (and the
 * stats of the last insert, if stats is not NULL). */
sbki_status sbki_sync(sbki_map* map, sbki_stats* stats);

/* Steps a1-a3 only (Sec. III): the training set of a scan, without touching
 * the map.  xyzl_out [cap,4] float32 = (x, y, z, label as float), ordered by
 * (downsampling tile, cell, label); *count receives the number of points (if
 * count > cap only cap are written and SBKI_ERR_CAPACITY is returned). */
sbki_status sbki_training_set(sbki_map* map, const float* points, const int32_t* labels, int64_t n,
                              const double sensor_pose[16], float* xyzl_out, int64_t cap, int64_t* count);

/* Soft labels (Sec. III takes the network's most probable class; the paper's
 * discussion names the softmax output as the richer input; reading K15):
 * every hit carries a probability vector probs [n,K] float32 over the
 * occupied classes 1..K (row i for point i; entries finite in [0, 1], at least
 * one > 0) instead of one label.  Free samples stay class 0 with weight 1.
 * Downsampling groups hits and samples by (cell, most probable class, ties to
 * the lowest), so one-hot vectors give the groups of sbki_insert_scan; a
 * group's representative is the exact centroid with, per class 0..K, the
 * exact mean of its members' weights rounded once to FP32; the accumulation
 * adds sigma0 sigma0_scale[k] f(d/l_k) w^k into every class k of every voxel
 * centre within l_k (Eq. (alpha_kernel) with the one-hot y_i replaced by w).
 * points and probs may be host or device memory; synchronises the stream.
 * Needs accumulate_mode 0, association 0 and the common l (all l_scale 1);
 * stats as sbki_insert_scan (pairs: voxel-point pairs, each counted once). */
sbki_status sbki_insert_scan_soft(sbki_map* map, const float* points, const float* probs, int64_t n,
                                  const double sensor_pose[16], sbki_stats* stats);
/* Steps a1-a3 of sbki_insert_scan_soft only: xyz_out [cap,3] float32 and
 * w_out [cap,K+1] float32 (host or device, both or neither), ordered as
 * sbki_training_set; *count as sbki_training_set. */
sbki_status sbki_training_set_soft(sbki_map* map, const float* points, const float* probs, int64_t n,
                                   const double sensor_pose[16], float* xyz_out, float* w_out, int64_t cap,
                                   int64_t* count);

/* The training set of one scan (steps a1-a3, same result as
 * sbki_training_set) with no device allocation and no map.  The paper has no
 * counterpart: this is a deployment variant for callers that cannot allocate
 * device memory while they run - a real-time mapping loop that reserves all of
 * its memory at start-up (a cudaMalloc can stall or fail mid-run), or a
 * framework that owns the device heap through its own pool allocator.
 *   params: as for sbki_create_map (pool_blocks, sample_capacity and
 *     track_pairs are ignored); work runs on params->device and, in stream
 *     order, on params->cuda_stream; the call synchronises that stream.
 *   points [n,3] float32 and labels [n] int32 (1..K): DEVICE memory of
 *     params->device; xyzl_out [cap,4] float32: DEVICE memory, written as for
 *     sbki_training_set; *count (host) receives the number of points.
 * Every intermediate buffer lives in one fixed device array of about 11 MB
 * that each GPU loading the library holds until the process exits; nothing
 * is allocated per call (no cudaMalloc, cudaFree or allocating library call).
 * Limits: n <= 16384 points (else SBKI_ERR_INVALID_ARG before any GPU work)
 * and at most 131072 hits + free samples (else SBKI_ERR_CAPACITY after the
 * counting step); count > cap writes cap points and returns SBKI_ERR_CAPACITY.
 * All calls share the array and it keeps the last call's contents (its
 * counters are cleared at the start of each call): calls that overlap on the
 * GPU - other streams, other host threads - race and must be serialised.
 * The first call on a device looks up the array's device address with that
 * device current; make it before any stream capture.  Errors are reported by
 * sbki_last_error(NULL). */
sbki_status sbki_training_set_noalloc(const sbki_params* params, const float* points, const int32_t* labels,
                                      int64_t n, const double sensor_pose[16], float* xyzl_out, int64_t cap,
                                      int64_t* count);

/* One scan of a batched update. */
typedef struct sbki_scan {
  const float* points;   /* [n,3] sensor frame (host or device) */
  const int32_t* labels; /* [n] in 1..K (host or device) */
  int64_t n;
  double pose[16];       /* world_from_sensor, row-major */
  int32_t map_id;        /* target map of the handle, 0..num_maps-1 */
} sbki_scan;

/* Batched form of the update (Sec. III + Eq. (alpha_kernel) + Sec. IV for
 * every scan): scans[0..count) (count <= 64), each into map scans[i].map_id
 * of the handle, go through one pass of the device pipeline - one launch per
 * stage for all scans together (persistent kernels over the concatenated
 * points, items and training points; every scan is downsampled on its own,
 * as sbki_insert_scan would) with no host round trip between stages.  The
 * stage sequence is recorded once per batch size as a CUDA graph and replayed
 * on later calls with the same count.  Scans into the same map add up as
 * consecutive sbki_insert_scan calls would (up to the order of FP32 sums).
 * The sum of n must fit the staging capacity (grown on demand, outside the
 * graph) and the hits + free samples of all scans must fit sample_capacity.
 * Synchronises the stream once, at the end; stats are totals over the batch
 * (touched_voxels 0).  On any error no map changes. */
sbki_status sbki_insert_batch(sbki_map* map, const sbki_scan* scans, int32_t count, sbki_stats* stats);

/* Launch shapes of the update's kernels (all persistent grids): CTAs per SM
 * for the accumulation (0 = as many as fit), training points per warp chunk
 * in the accumulation (1..64), CTAs per SM for the touched-block pass and for
 * the ingest kernels (transform, samples, segments, centroids).  Results do
 * not depend on them; speed does.  sbki_set_tuning drops the recorded
 * batched updates (they are recorded again with the new shapes). */
typedef struct sbki_tuning {
  int32_t accumulate_ctas_per_sm;
  int32_t accumulate_chunk;
  int32_t touch_ctas_per_sm;
  int32_t ingest_ctas_per_sm;
} sbki_tuning;
sbki_status sbki_get_tuning(const sbki_map* map, sbki_tuning* out);
sbki_status sbki_set_tuning(sbki_map* map, const sbki_tuning* tuning);

/* Selects the map of the handle (0..num_maps-1) that sbki_insert_scan,
 * sbki_insert_scan_async, sbki_insert_training, sbki_query_probs,
 * sbki_voxel_count, sbki_export and the differentiable calls act on. */
sbki_status sbki_select_map(sbki_map* map, int32_t map_id);

/* Eq. (alpha_kernel) for a given training set (no sampling or downsampling):
 * xyzl [p,4] float32 world (x, y, z, label as float) with labels 0..K. */
sbki_status sbki_insert_training(sbki_map* map, const float* xyzl, int64_t p, sbki_stats* stats);

/* Read-off at world points xyz [q,3] (Eq. mode, Eq. variance, Sec. V-C): the
 * voxel containing each point is looked up; a voxel never reached reads as
 * the prior.  probs [q,K+1] = E[theta] (required); var [q,K+1] = V[theta];
 * mode [q,K+1] = (alpha^k - 1)/(sum alpha - (K+1)) where every alpha^k > 1,
 * else NaN; label [q] = argmax alpha (ties to the lowest class); p_occ [q] =
 * sum of the occupied-class probabilities; state [q] = 0 free / 1 unknown /
 * 2 occupied (a voxel with no kernel mass is unknown).  All but probs may be
 * NULL. */
sbki_status sbki_query_probs(const sbki_map* map, const float* xyz, int64_t q, float* probs, float* var,
                             float* mode, int32_t* label, float* p_occ, int32_t* state);

/* The same contents as sbki_export, computed on the device and written in
 * pool order (blocks in allocation order; within a block x fastest, then y,
 * z): keys [cap,3] int64 and alpha [cap,K+1] float32 with prior, each host or
 * device memory (device buffers get no host copy; the call synchronises the
 * stream to read the row count).  count-only when both are NULL. */
sbki_status sbki_export_blocks(const sbki_map* map, int64_t* keys, float* alpha, int64_t cap, int64_t* count);

/* Number of allocated voxels (blocks * block_edge^3). */
sbki_status sbki_voxel_count(const sbki_map* map, int64_t* count);

/* Every voxel of every allocated block, sorted by voxel index (x, y, z)
 * lexicographically: keys [cap,3] int64 voxel indices (centre = (key+0.5)*res),
 * alpha [cap,K+1] float32 including alpha0, pairs [cap] in-support pair counts
 * (NULL, or requires track_pairs).  Host buffers only. */
sbki_status sbki_export(const sbki_map* map, int64_t* keys, float* alpha, int32_t* pairs, int64_t cap,
                        int64_t* count);

/* Per-stage device timing and launch counting (tracing aid).  With profiling
 * on, each insert records CUDA events on the map's stream around step a1-a3
 * (sampling + downsampling), a4 (block hash) and a5 (accumulation) and adds
 * the elapsed times: a synchronous insert at its end, an asynchronous one
 * (sbki_insert_scan_async) at the next synchronising call on the map (two
 * sets of events, so back-to-back asynchronous inserts are all timed);
 * launches counts every kernel the library launched on the map since
 * creation (profiling on or off).  A reset drops an asynchronous insert not
 * yet read. */
typedef struct sbki_profile_data {
  int64_t inserts;     /* inserts timed since the last reset */
  int64_t launches;    /* kernels launched by this map since creation */
  double ingest_ms;    /* a1-a3 */
  double blocks_ms;    /* a4 */
  double accumulate_ms;/* a5 */
  int64_t readback_bytes; /* device-to-host bytes of one scan update: the counter block, read once */
} sbki_profile_data;
sbki_status sbki_profile(sbki_map* map, int32_t enable, int32_t reset);
sbki_status sbki_profile_read(const sbki_map* map, sbki_profile_data* out);

/* The sparse kernel of Eq. (kernel): f[i] = f(r[i]) for r = d/l (f = 0 for
 * r >= 1), so k(d) = sigma0 * f(d/l).  method 0 is the form the update uses
 * (u^5 Q(u^2), u = 1 - r, Q a Chebyshev interpolant), method 1 the textbook
 * trigonometric form.  r and f are device buffers of n floats; synchronises
 * `stream` (a cudaStream_t, NULL = legacy default stream).  Diagnostic aid. */
sbki_status sbki_kernel_values(const float* r, int64_t n, float* f, int32_t method, void* stream);

/* ------------------------------------------------------------------------
 * Differentiable form.  alpha is a smooth function of the training points,
 * of l and of sigma0 (Eq. alpha_kernel with Eq. kernel, which has zero slope
 * at d = l, so the support boundary adds no term).  A map holds a gradient
 * buffer G = dL/dalpha with the layout of alpha, allocated on first use
 * (pool_blocks x (K+1) x block_edge^3 floats); the calls below fill it and
 * pull it back through every in-support pair, recomputing the kernel.
 * Gradients refer to the training set inserted with sbki_insert_training:
 * pass the same xyzl to sbki_backward.
 * ------------------------------------------------------------------------ */

/* Sets G to zero on every allocated block. */
sbki_status sbki_grad_clear(sbki_map* map);

/* Held-out log-likelihood of labelled points, the Dirichlet mean of Eq.
 * (variance) used as the predictive probability at the voxel containing each
 * point: LL = sum_h log(alpha^{y_h} / sum_k alpha^k) (alpha with prior; a
 * voxel outside every block reads the prior).  xyz [h,3] world, labels [h] in
 * 0..K (host or device).  If accumulate_grad != 0, dLL/dalpha is added into G
 * (only on allocated blocks: no pair reaches the others).  *loglik on host. */
sbki_status sbki_heldout_loglik(sbki_map* map, const float* xyz, const int32_t* labels, int64_t h,
                                int32_t accumulate_grad, double* loglik);

/* Adds an upstream gradient given per voxel: keys [count,3] int64 voxel
 * indices, grad_alpha [count,K+1] float32 (host or device).  Rows whose voxel
 * lies outside every allocated block are skipped and counted in *missed
 * (nullable): no pair reaches them. */
sbki_status sbki_grad_add_alpha(sbki_map* map, const int64_t* keys, const float* grad_alpha, int64_t count,
                                int64_t* missed);

/* Backward pass of Eq. (alpha_kernel) through Eq. (kernel) for the training
 * set xyzl [p,4] (world x, y, z, label as float; host or device) that was
 * inserted: with r = d/l and G = G_v^{y_i} per in-support pair,
 *   grad_sigma0 = sum G f(r),  grad_l = sum G sigma0 f'(r) (-d/l^2),
 *   grad_xyz[i] = sum_v G sigma0 f'(r) (x_i - c_v)/(l d)   ([p,3], nullable,
 *   host or device; 0 where d = 0).
 * grad_l and grad_sigma0 (host, nullable) are summed in FP64 from FP32 pair
 * terms.  A counting-model map (piecewise constant in x, no l or sigma0)
 * returns SBKI_ERR_INVALID_ARG. */
sbki_status sbki_backward(sbki_map* map, const float* xyzl, int64_t p, double* grad_l, double* grad_sigma0,
                          float* grad_xyz);

/* The same pass for the per-class kernel scales: grad_scale[k] = dL/d
 * sigma0_scale[k] = sum over the in-support pairs of class-k points of
 * G sigma0 f(r) (host, [K+1], summed in FP64 from FP32 pair terms).  Same
 * inputs and errors as sbki_backward. */
sbki_status sbki_backward_scales(sbki_map* map, const float* xyzl, int64_t p, double* grad_scale);

/* Stateless forms (they create and destroy a map of `params` inside the call,
 * so they allocate): alpha of a training set at every voxel of the blocks it
 * reaches (as sbki_export: keys_out [cap,3], alpha_out [cap,K+1], host
 * memory, sorted by key, count-only when both are NULL), and the gradient of
 * L with respect to l, sigma0 and the points for dL/dalpha given at voxel
 * keys.  Errors are reported by sbki_last_error(NULL). */
sbki_status sbki_forward_alpha(const sbki_params* params, const float* xyzl, int64_t p, int64_t* keys_out,
                               float* alpha_out, int64_t cap, int64_t* count);
sbki_status sbki_grad(const sbki_params* params, const float* xyzl, int64_t p, const int64_t* keys,
                      const float* grad_alpha, int64_t count, double* grad_l, double* grad_sigma0, float* grad_xyz);

/* Eq. (alpha_kernel) at arbitrary points of space (Sec. IV: the model can be
 * queried at any resolution, not only at voxel centres), stateless, from a
 * training set:  alpha_out[j, k] = alpha0 + sum over training points i with
 * |pts_j - x_i| < l and label k of sigma0 sigma0_scale[k] f(|pts_j - x_i| / l)
 * (every point within l: the exact association, whatever params->association
 * says).  xyzl [p,4] float32 (x, y, z, label as float, labels 0..K); pts [q,3]
 * float32 world; alpha_out [q,K+1] float32.  Each of the three may be host or
 * device memory (device pointers are used in stream order on
 * params->cuda_stream); the call allocates its own work buffers and
 * synchronises the stream.  Membership as in the map update (exact); sums in
 * FP32.  The counting model is refused (SBKI_ERR_INVALID_ARG); errors are
 * reported by sbki_last_error(NULL). */
sbki_status sbki_query_points(const sbki_params* params, const float* xyzl, int64_t p, const float* pts, int64_t q,
                              float* alpha_out);

/* Restores contents written by sbki_export into the selected map (a snapshot
 * and resume path): keys [count,3] int64 voxel indices, alpha [count,K+1]
 * float32 with prior (host or device).  The block of every key is created if
 * missing and the voxel's increments are set to alpha - alpha0 (one FP32
 * subtraction, so a re-export equals the snapshot to an ulp); other voxels of
 * created blocks read the prior, voxels not listed keep their values.  An
 * increment below half an ulp of alpha0 is already lost in the exported alpha
 * (alpha0 + increment rounds to alpha0), so such a voxel is restored with no
 * kernel mass and reads as unknown.  Pair counts are not restored.
 * SBKI_ERR_CAPACITY (pool full) leaves the block set unchanged. */
sbki_status sbki_import(sbki_map* map, const int64_t* keys, const float* alpha, int64_t count);

/* Failure-detection self-test on `device` (diagnostic): runs one digit pass
 * of the downsampling step's radix sort, then the one-pass prefix sum of the
 * sample offsets, each over three tiles whose first tile is never processed,
 * so every bounded wait of the others on it runs out (about a second each);
 * the kernels report SBKI_ERR_TIMEOUT instead of spinning, and the context
 * stays usable.  *device_status: SBKI_ERR_TIMEOUT when the waits of both ran
 * out, else the first other status.  Returns SBKI_OK when the test itself
 * ran. */
sbki_status sbki_selftest_bounded_wait(int32_t device, int32_t* device_status);

/* Message of the last failure on this map (or of the last sbki_create_map
 * failure when map is NULL). */
const char* sbki_last_error(const sbki_map* map);
const char* sbki_status_string(sbki_status s);

#ifdef __cplusplus
}
#endif
#endif /* SBKI_H */
