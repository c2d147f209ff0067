/* rapid.h — C ABI of the GB300 (sm_103a) implementation of the coarse-to-fine
 * topology-preserving superpixel refinement of RAPID ("RAPID" Regions-of-Interest
 * Detection in Big Histopathological Images, Sulimowicz & Ahmad, ICME 2017).
 *
 * The calls follow the paper's statement of the problem: an RGB image goes in; the label
 * matrix L (one superpixel id per pixel) and the per-superpixel statistics S (size, mean
 * colour, mean position; Algorithm RAPID) come out.  Every step runs in CUDA kernels on
 * one GPU; the library owns all device memory it allocates and keeps no caller pointer
 * after a call returns.
 *
 * Conventions
 *  - Every call returns a rapid_status and never throws.  The first CUDA error is sticky:
 *    later calls on the same context return RAPID_ECUDA until rapid_destroy.
 *  - Work is enqueued on the context's stream (borrowed, never destroyed by the library;
 *    0 = the legacy default stream).  Calls that return data to the host synchronise that
 *    stream first.  A device wait that gives up (see spin_limit_ns) is reported as
 *    RAPID_ETIMEOUT by the next synchronising call.
 *  - Labels are int32 in [0, M).  They are stable: a superpixel merged away keeps its id
 *    retired (size 0) and ids are never reused.
 *  - Coordinates are 0-based full-resolution pixels; x = column, y = row.  Images are
 *    row-major, interleaved RGB, one byte per channel.
 *  - Floating-point energies are IEEE binary64 evaluated in a fixed operation order with
 *    no fused multiply-add; all sums are exact int64.  Results are therefore reproducible
 *    bit for bit.
 */
#ifndef RAPID_H
#define RAPID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rapid_status {
  RAPID_OK = 0,
  RAPID_EINVAL = 1,   /* bad argument (NULL pointer, size out of range, bad parameter) */
  RAPID_ENOMEM = 2,   /* device or host allocation failed */
  RAPID_ECUDA = 3,    /* a CUDA runtime call or kernel failed (sticky) */
  RAPID_ESTATE = 4,   /* call out of order (e.g. refine before seeding, split after the last stage) */
  RAPID_ETIMEOUT = 5, /* a bounded device-side wait (grid barrier) gave up; results are invalid */
  RAPID_ERANGE = 6    /* exactness limit exceeded (an int64 sum could pass 2^53, too many stages) */
} rapid_status;

typedef struct rapid_ctx rapid_ctx; /* opaque; owns every device buffer it allocates */

/* Parameters of the method.  rapid_default_params() fills the defaults listed here. */
typedef struct rapid_params {
  int32_t num_levels;      /* L >= 1 image levels (Sec. 2.2); level l (1 = coarsest) is the
                              image box-summed by f_l = C^(L-l).  Default 1. */
  int32_t ratio_C;         /* compression ratio C between levels, power of two >= 2
                              (Eq. eq:mu).  Default 4. */
  int32_t init_block;      /* initial block side in full-res pixels, power of two.  Default 16. */
  int32_t final_grain;     /* final block side ("grain", Sec. 4.3), power of two.  Default 1. */
  int32_t K;               /* requested number of superpixels (seed grid, Algorithm RAPID).
                              Default 200. */
  int32_t size_mode;       /* E_size handling (Sec. 3.1): 0 = none (lambda_s = 0), 1 = hard
                              lower bound (lambda_s = inf), 2 = merge (the paper's
                              regularity optimisation).  Default 2. */
  double lambda_pos0;      /* position weight: lambda_pos = lambda_pos0 * M / (H*W).  Default 400. */
  double lambda_b;         /* boundary-length weight per 4-adjacent full-res pixel pair
                              (Eq. equa:energy1, Eq. bound).  Default 50. */
  int32_t lo_num, lo_den;  /* lower size bound l = lo_num/lo_den (Sec. 3.1).  Default 1/4. */
  int32_t hi_num, hi_den;  /* upper size bound u = hi_num/hi_den (Eq. condtion).  Default 3/2. */
  int32_t predict;         /* 1: predict at level 2 and refine only boundary superpixels
                              afterwards (Sec. 3.2, Eq. predict, Eq. new_bound).  Default 0. */
  int32_t reuse;           /* 1: carry S across levels (Eq. eq:mu); 0: recompute S at every
                              level entry (multi-scale baseline).  Same results.  Default 1. */
  int32_t importance_rule; /* 0: a block is refined when its superpixel is a boundary
                              superpixel; 1: when a 4-neighbour has a different label of the
                              other class (Eq. new_bound read pairwise).  Default 0. */
  int32_t max_sweeps;      /* sweeps per stage before giving up on convergence.  Default 64. */
  int64_t h_T;             /* brightness threshold of the integer stand-in classifier
                              h(k) = 3 h_T N_k - (R_k + G_k + B_k) (Eq. predict).  Default 150. */
  int64_t spin_limit_ns;   /* give-up time of each device-side barrier wait; 0 gives up at
                              once (used by tests).  Default 2e9 (2 s). */
  int32_t use_filter;      /* 1: decide blocks in single precision with a certified error
                              bound and fall back to binary64 when it cannot decide (same
                              results as 0, faster).  Default 1. */
  int32_t skip_tiles;      /* 1: skip tiles none of whose labels changed since their last scan
                              (same results and counters as 0, faster).  Default 1. */
  int32_t verify_filter;   /* 1: also decide every block in binary64 and count disagreements
                              with the single-precision decisions (testing).  Default 0. */
  int32_t schedule;        /* which blocks a phase visits (Sec. 2.1, the boundary queue):
                              0 = every block of the phase class, every sweep (default);
                              1 = frontier queue: every block is queued when a stage starts, a
                              phase pops the queued blocks of its class, and a move (or an
                              accepted merge, at its first requesting block) pushes the
                              block's 4-neighbours.  Results differ from 0; the stage still
                              ends after a sweep without changes (the queue is then empty).
                              Not combinable with the learned scorer (RAPID_EINVAL). */
} rapid_params;

#define RAPID_MAX_STAGES 32

/* Per-superpixel statistics S (Algorithm RAPID), index = label id.  Means are sums / n. */
typedef struct rapid_sp_stats {
  int64_t n;          /* pixel count (0 = retired by a merge) */
  int64_t sum_r, sum_g, sum_b;
  int64_t sum_x, sum_y;
  int64_t init_size;  /* InitSize: pixel count right after seeding (Sec. 3.1) */
  int32_t y;          /* class from Eq. predict: +1 ROI, -1 non-ROI, 0 before prediction */
  int32_t important;  /* 1 when a boundary superpixel (Eq. new_bound), else 0 */
} rapid_sp_stats;

typedef struct rapid_stage_counters {
  int32_t level;           /* image level l of the stage */
  int32_t block;           /* block side s in full-res pixels */
  int32_t sweeps;          /* 9-phase sweeps run (<= max_sweeps) */
  int32_t pad;
  int64_t eligible;        /* block evaluations that passed the boundary / importance test */
  int64_t evaluated;       /* ... and the topology test (energies computed) */
  int64_t moves;           /* blocks relabelled */
  int64_t merge_requests;  /* moves replaced by a merge request (size bound hit) */
  int64_t merges;          /* merges accepted */
  int64_t fp64_fallbacks;  /* evaluations the single-precision bound could not decide */
  int64_t filter_mismatches; /* with verify_filter: single-precision decisions that differ
                              from binary64 (must be 0) */
  int64_t tiles_scanned;   /* sweep schedule: blocks visited by the bitmap walk (their bit
                              was set); queue schedule: tile-phase scans ... */
  int64_t tiles_skipped;   /* sweep schedule: blocks that passed the tests and skipped the
                              decision because nothing in their window changed since their
                              previous visit; queue schedule: tiles skipped because none of
                              their blocks of the phase class was queued (its sparse phases
                              take listed blocks, not tiles, and count neither) */
  int64_t merge_searches;  /* merge-target searches that scanned the label map ... */
  int64_t merge_cache_hits; /* ... and requests answered by a still-valid earlier failure */
  float kernel_ms;         /* device time of the stage's refinement launch when profiling is
                              on (rapid_set_profiling), else -1 */
  float section_ms[5];     /* with profiling on, as seen by the launch's first CTA: block
                              evaluation, wait after it, statistics commit, wait after it,
                              merge resolution (with its waits); else 0 */
  float pad2;
} rapid_stage_counters;

typedef struct rapid_counters {
  int32_t num_stages;      /* stages of the schedule */
  int32_t M;               /* label ids in use (seeded superpixels) */
  int64_t launches;        /* kernels this context has launched since creation */
  rapid_stage_counters stage[RAPID_MAX_STAGES];
} rapid_counters;

/* Fill *p with the defaults documented in rapid_params.  NULL-safe. */
void rapid_default_params(rapid_params *p);

/* Create a context bound to the current CUDA device.  p is copied; cuda_stream is a
 * cudaStream_t borrowed for the context's lifetime (0 = legacy default stream).
 * EINVAL on a bad parameter, ENOMEM, ECUDA. */
rapid_status rapid_create(const rapid_params *p, void *cuda_stream, rapid_ctx **out);

/* Copy an H x W interleaved RGB image into the context (Algorithm RAPID input I).
 * rgb: host or device (rgb_is_device) pointer, rows row_pitch_bytes apart
 * (>= 3*W).  The caller keeps ownership; the copy is complete when the call returns for
 * host input and stream-ordered for device input.  Allocates the per-image buffers;
 * resets the context to "image set, not seeded".  EINVAL (H or W < 1, H*W >= 2^31, or
 * H*W*max(H,W) >= 2^53, which would break exact double conversion of position sums),
 * ERANGE (a level factor f with min(f,W)*min(f,H)*255 > 2^31 - 1: the level's int32
 * colour sums would overflow), ENOMEM, ECUDA. */
rapid_status rapid_set_image(rapid_ctx *ctx, const uint8_t *rgb, int32_t H, int32_t W,
                             int64_t row_pitch_bytes, int32_t rgb_is_device);

/* Build the level images (exact box sums, Sec. 2.2) and seed the regular grid of
 * superpixels (Algorithm RAPID, "initialize superpixels to be regular grids"): gx =
 * round(sqrt(K W / H)), gy = round(K / gx), clamped to the first stage's block grid;
 * compute S and InitSize.  *M_out (may be NULL) receives gx*gy.  ESTATE without an image. */
rapid_status rapid_seed_grid(rapid_ctx *ctx, int32_t *M_out);

/* Refine the current stage (Sec. 2.1 and Algorithm RAPID's queue loop): 9-phase sweeps of
 * boundary-block relabelling (Eq. operation) under the topology constraint, with the size
 * term of size_mode, until a sweep changes nothing or max_sweeps.  Out-pointers may be
 * NULL; when any is non-NULL the call synchronises and fills them.  ESTATE before
 * seeding; ETIMEOUT / ECUDA as above. */
rapid_status rapid_refine_stage(rapid_ctx *ctx, int32_t *sweeps_out, int64_t *moves_out,
                                int64_t *merges_out);

/* Advance to the next stage: predict on entering level 2 (when enabled), split every block
 * into 2x2 blocks that keep its label (Algorithm RAPID, "map superpixels' labels"), and
 * with reuse off recompute S from the new level.  ESTATE before seeding or after the last
 * stage. */
rapid_status rapid_split(rapid_ctx *ctx);

/* The whole schedule on the context's image(s): level images, seeding, then refine / split
 * through every stage.  Enqueue only; a later synchronising call reports errors.  With
 * graph mode on (rapid_set_graph) the first call captures these launches into a CUDA
 * graph and every call launches that graph. */
rapid_status rapid_run(rapid_ctx *ctx);

/* ---- Batches: many images refined together (the data partitioning of Sec. 3.3) ----
 * A context may hold up to RAPID_MAX_BATCH images of any sizes.  Every stage then refines
 * all of them in one persistent launch; each image keeps its own block grid, seed grid
 * (from its own K), lambda_pos and sweep count (an image stops sweeping a stage after its
 * own sweep without change), so each image's labels, statistics and counters are exactly
 * those of refining it alone with the same parameters.  The single-image calls above act
 * on image 0. */
#define RAPID_MAX_BATCH 64

/* Copy n images into the context (replacing any previous ones).  rgb[i]: H[i] x W[i]
 * interleaved RGB, host or device (rgb_is_device), rows row_pitch_bytes[i] apart (>= 3 W[i]).
 * K: requested superpixels per image (NULL = params.K for all).  The caller keeps
 * ownership; host input is copied before the call returns.  EINVAL as for
 * rapid_set_image (per image) or n < 1; ERANGE for n > RAPID_MAX_BATCH, an overflowing
 * level sum, or more than 2^31 - 1 blocks or labels over the batch; ENOMEM, ECUDA. */
rapid_status rapid_set_images(rapid_ctx *ctx, int32_t n, const uint8_t *const *rgb, const int32_t *H,
                              const int32_t *W, const int64_t *row_pitch_bytes, const int32_t *K,
                              int32_t rgb_is_device);

/* Size and superpixel count M of image i (any pointer may be NULL).  EINVAL for a bad i. */
rapid_status rapid_get_image_info(rapid_ctx *ctx, int32_t i, int32_t *H, int32_t *W, int32_t *M);

/* Image i's full-resolution label map (ids 0 .. M_i - 1, layout as rapid_read_labels),
 * statistics (as rapid_read_stats) and per-stage counters (as rapid_read_counters; the
 * section times and kernel_ms are those of the whole launch).  All synchronise. */
rapid_status rapid_read_image_labels(rapid_ctx *ctx, int32_t i, int32_t *dst, int64_t row_pitch_bytes,
                                     int32_t dst_is_device);
rapid_status rapid_read_image_stats(rapid_ctx *ctx, int32_t i, rapid_sp_stats *dst, int64_t capacity,
                                    int64_t *M_out);
rapid_status rapid_read_image_counters(rapid_ctx *ctx, int32_t i, rapid_counters *dst);

/* Launch geometry.  Results never depend on it (a phase's decisions are independent and
 * merges are ordered by block index), only the time does.
 * rapid_set_stage_grids: CTAs of each stage's launch for stages 0 .. n-1 (0 = the full
 *   co-resident grid, larger values are capped to it; the others reset to 0).  A single
 *   image's stage of 2 to 16 CTAs runs as one thread-block cluster, whose hardware barrier
 *   replaces the grid barrier, where the device can co-schedule such a cluster (else, and
 *   for batches, as a cooperative launch).
 * rapid_set_stage_shapes: evaluation-tile shape of each stage, an index into
 *   {32 x 16, 32 x 8, 64 x 16} blocks with 1024 threads per CTA (0, 1, 2) or with 512 threads
 *   per CTA (3, 4, 5) (default 0; the others reset to 0).
 * rapid_autotune: time the whole schedule on the context's current images once per tile
 *   shape (full grid), then once per grid size (the full grid halved down to one CTA, and
 *   the cluster sizes 16 and 8) with the chosen shapes; keep per stage the fastest and write them to grids_out and
 *   shapes_out (RAPID_MAX_STAGES entries each, either may be NULL).  Synchronises; the
 *   context's results afterwards are those of a normal run.
 * EINVAL on a negative grid or an unknown shape, ESTATE without images. */
rapid_status rapid_set_stage_grids(rapid_ctx *ctx, const int32_t *grids, int32_t n);
rapid_status rapid_set_stage_shapes(rapid_ctx *ctx, const int32_t *shapes, int32_t n);
rapid_status rapid_autotune(rapid_ctx *ctx, int32_t *grids_out, int32_t *shapes_out);

/* ---- Learned block scorer (pruning of the boundary-block queue) ----
 * A 3-layer 3x3 convolutional net over 9 per-block features (colour gain of moving to each
 * of the up to 4 neighbour labels, boundary count, level, coarse importance, block side,
 * misfit to the own label) predicts which boundary blocks will move in a stage.  It only
 * prunes which eligible blocks the exact topology and energy tests evaluate; every move is
 * still decided by the exact test (Eq. operation).  Weights and activations are bf16 with
 * fp32 sums.  Weights are RAPID_SCORER_PARAMS floats in the order W1[16][9][3][3], b1[16],
 * W2[16][16][3][3], b2[16], W3[16][3][3], b3 (conv weights [out][in][ky][kx], zero padding
 * outside the image at every layer). */
#define RAPID_SCORER_PARAMS 3777
#define RAPID_SCORER_FEATURES 9

/* ---- Superpixel features and a linear classifier for Eq. predict ----
 * With theta (host, 5 doubles; NULL = off, the default) the prediction at the entry to
 * level 2 evaluates h = theta[0] + theta[1] f1 + theta[2] f2 + theta[3] f3 + theta[4] f4
 * (binary64, left to right) over each superpixel's features on the last level-1 block grid
 * (the F in R^4 of Sec. 4.1), and y = 1 when h >= 0; without theta it uses the brightness
 * stand-in 3 h_T N - (R + G + B).  With b the mean brightness (R + G + B) / (3 N) and c the
 * mean colour:
 *   f1 absolute brightness b;
 *   f2 comparative brightness: b minus the mean, over the superpixel's 4-adjacent block
 *      pairs with other superpixels, of their b (each as floor(2^16 b) / 2^16);
 *   f3 extra-region dissimilarity: the mean over those pairs of |c - c_other| (each
 *      truncated to a multiple of 2^-16);
 *   f4 intra-region dissimilarity: sqrt of the pixel-weighted mean over its blocks of
 *      |c_block - c|^2 (each block's term truncated to a multiple of 2^-16).
 * theta = (3 h_T, -3, 0, 0, 0) reproduces the stand-in exactly.  EINVAL on a non-finite
 * theta.  rapid_read_features copies image i's features of the last prediction made with
 * a classifier (M_i x 4 doubles, host dst; ESTATE when no classifier was set).
 * Synchronises. */
rapid_status rapid_set_classifier(rapid_ctx *ctx, const double *theta5);
rapid_status rapid_read_features(rapid_ctx *ctx, int32_t i, double *dst_host);

/* Pruned refinement: with weights (host, RAPID_SCORER_PARAMS floats; NULL = off) every stage
 * first scores its blocks (score = sigmoid of the net's output) and sweeps only over the
 * eligible blocks scoring >= threshold until a sweep changes nothing; then it sweeps over
 * every block until a sweep changes nothing (the full sweep is the fallback), within
 * max_sweeps in all.  Results then differ from the plain method's (quality is judged
 * against it); with threshold 0 they are the same.  Synchronises. */
rapid_status rapid_set_scorer(rapid_ctx *ctx, const float *weights, float threshold);

/* The stages the scorer prunes: on[i] = 1 prunes stage i, 0 sweeps it in full without
 * scoring; stages from n on are pruned (n = 0: every stage, the default).  EINVAL on a flag
 * other than 0 and 1 or n outside [0, RAPID_MAX_STAGES]. */
rapid_status rapid_set_scorer_stages(rapid_ctx *ctx, const int32_t *on, int32_t n);

/* Pruned refinement with keep masks the caller gives instead of the scorer's: the same
 * pruned sweeps as rapid_set_scorer runs (a stage sweeps testing and deciding only the kept
 * eligible blocks until a sweep changes nothing, then sweeps every block until a sweep
 * changes nothing, within max_sweeps), with the boundary-superpixel pruning of Sec. 3.2
 * generalised to an arbitrary per-block mask.  It lets the pruned machinery be checked
 * against a reference on the same masks, and serves callers with a pruning rule of their
 * own.  mask: image i's mask for stage s, n = nbx * nby bytes of that stage's block grid
 * (row-major, nonzero = kept), host memory or device memory by mask_is_device (1), copied
 * before return.  A stage with a mask set for any image sweeps pruned; the images without
 * one at that stage keep every block.  rapid_set_keep_mask(ctx, -1, -1, NULL, 0, 0) clears
 * every mask; rapid_set_images clears them too.  ESTATE before rapid_set_images; EINVAL on
 * a wrong size, image or stage index, under the queue schedule (schedule 1) or while a
 * scorer is set (rapid_set_scorer likewise refuses while masks are set).  Synchronises. */
rapid_status rapid_set_keep_mask(rapid_ctx *ctx, int32_t i, int32_t s, const uint8_t *mask, int64_t n,
                                 int32_t mask_is_device);

/* The current stage's features of image i ([nby][nbx][RAPID_SCORER_FEATURES] fp32, device
 * buffer dst of nby*nbx*9 floats), and scores ([nby][nbx] fp32, device buffer) under the
 * given weights (host).  Stream-ordered.  ESTATE before seeding. */
rapid_status rapid_scorer_features(rapid_ctx *ctx, int32_t i, float *dst_dev);
rapid_status rapid_scorer_scores(rapid_ctx *ctx, int32_t i, const float *weights, float *dst_dev);

/* Training data and training.  A trainer holds up to `capacity` samples on the device.
 * While a context logs into it (rapid_set_logging), every stage appends one sample per
 * block that was a boundary block at the stage start: its 7x7 patch of features (the net's
 * receptive field) and y = 1 when the block's label changed during the stage.  Blocks with
 * y = 0 are kept with probability neg_rate (a hash of image, stage and block decides).
 * rapid_trainer_fit trains the net on the samples with Adam (fp32 master weights, bf16
 * forward) on the loss pos_weight * y * -log p + (1 - y) * -log(1 - p), in minibatches of
 * `batch` over `epochs` shuffled passes (shuffle seeded by `seed`), starting from `init`
 * (host, NULL = a seeded random start) and writes the weights to `weights_out` (host) and
 * the mean loss of each epoch to `epoch_loss` (host, `epochs` floats, may be NULL).
 * Both are deterministic: samples take their slots in a fixed order (not by thread
 * timing), and gradients are summed in a fixed order, so the same runs and the same seed
 * give bit-identical weights.  Synchronises. */
typedef struct rapid_trainer rapid_trainer;
rapid_status rapid_trainer_create(int64_t capacity, float neg_rate, rapid_trainer **out);
rapid_status rapid_set_logging(rapid_ctx *ctx, rapid_trainer *t);
rapid_status rapid_trainer_count(rapid_trainer *t, int64_t *samples, int64_t *positives);
rapid_status rapid_trainer_fit(rapid_trainer *t, int32_t epochs, int32_t batch, float lr, float pos_weight,
                               uint64_t seed, const float *init, float *weights_out, float *epoch_loss);
void rapid_trainer_destroy(rapid_trainer *t);

/* The stored samples first .. first + count - 1 (in the order logging appended them:
 * logged stage by logged stage, image by image, blocks in row-major order, so the same
 * runs log the same samples in the same slots): their feature patches (count x 7 x 7 x 9
 * floats, host x_out), in-image masks (bit p = patch position p is inside the image, host
 * inb_out) and labels (host y_out); any of the three may be NULL.  ERANGE past the stored
 * samples.  Synchronises. */
rapid_status rapid_trainer_samples(rapid_trainer *t, int64_t first, int32_t count, float *x_out, uint64_t *inb_out,
                                   float *y_out);

/* The gradient rapid_trainer_fit follows, for checking it: the sum over the samples first
 * .. first + count - 1 of the gradient of their loss (as in rapid_trainer_fit) at the master
 * weights `weights` (host, RAPID_SCORER_PARAMS floats; bf16-rounded for the forward pass as
 * in training), written to grad_out (host, RAPID_SCORER_PARAMS floats, same layout), and
 * the summed loss to loss_out (host, may be NULL).  The sums are taken in a fixed order, so
 * the result does not depend on thread timing.  ERANGE past the stored samples, EINVAL on
 * non-finite weights.  Synchronises. */
rapid_status rapid_trainer_gradient(rapid_trainer *t, const float *weights, int64_t first, int32_t count,
                                    float pos_weight, float *grad_out, float *loss_out);

/* Input generator (not part of the method: it makes the synthetic stand-in for the
 * paper's whole-slide images at full size on the device).  Writes the counter-based
 * synthetic H&E-like slide of H x W pixels into rgb_dev (device, interleaved RGB uint8,
 * rows rgb_pitch_bytes apart) and, when regions_dev is not NULL, its ground-truth region
 * ids (device int32, rows regions_pitch_bytes apart): Voronoi tissue cells (one per
 * px_per_cell pixels, white_frac of them white background), nuclei (nucleus_density per
 * pixel), fold bands covering about fold_frac of the area, Gaussian noise of sigma 6.
 * The definition is in k_synth.cu; paper_1704_02083_gb300.synth.slide_gen gives the same
 * bytes on the host for any window.  Stream-ordered on cuda_stream.  EINVAL on bad
 * arguments, ERANGE beyond 8 seeds or 64 nuclei per 128 x 128 bucket, 1024 bands or 2^31
 * ids. */
typedef struct {
  int64_t H, W;
  uint64_t seed;
  int32_t px_per_cell;
  int32_t pad;
  double white_frac, fold_frac, nucleus_density;
} rapid_synth_params;
rapid_status rapid_synth_slide(const rapid_synth_params *p, uint8_t *rgb_dev, int64_t rgb_pitch_bytes,
                               int32_t *regions_dev, int64_t regions_pitch_bytes, void *cuda_stream);

/* Whole slide.  The slide (device, H x W interleaved RGB, rows rgb_pitch_bytes apart; any
 * size) is cut into tiles by even row and column bands of at most max_tile pixels
 * (startRow = H i / n, Eq. parallel_spit, on both axes); the tiles, as views into the
 * slide, are refined on ctx in batches of up to RAPID_MAX_BATCH tiles and at most 2^30
 * pixels (a batch's block and label indices are 32-bit; a larger tile forms a batch alone;
 * each with
 * K = max(1, area / px_per_superpixel) and ctx's parameters), and every tile's labels are
 * written into labels_dev (device, H x W int32, rows labels_pitch_bytes apart) as
 * slide-wide ids: the tiles' superpixels numbered one after another, tile by tile in
 * row-major order.  Superpixels never cross a tile edge.  stats_dev (device, may be NULL)
 * receives the statistics of every slide-wide id (capacity entries; EINVAL when too few).
 * With autotune, the launch geometry is tuned on the first batch and kept; otherwise ctx's
 * geometry is used.  *M_out and *tiles_out (may be NULL) receive the superpixel and tile
 * counts.  ctx's images are replaced; it can serve further calls.  Synchronises.  EINVAL on
 * bad arguments (max_tile in [16, 46340]), ERANGE beyond 2^24 tiles or 2^31 - 1
 * superpixels. */
rapid_status rapid_refine_slide(rapid_ctx *ctx, const uint8_t *rgb_dev, int64_t H, int64_t W,
                                int64_t rgb_pitch_bytes, int32_t max_tile, int32_t px_per_superpixel,
                                int32_t autotune, int32_t *labels_dev, int64_t labels_pitch_bytes,
                                rapid_sp_stats *stats_dev, int64_t stats_capacity, int64_t *M_out,
                                int32_t *tiles_out);

/* Graph mode (0 = off, the default): rapid_run captures the schedule into a CUDA graph on
 * its first call after rapid_set_images and replays it afterwards (profiling events are
 * captured as event-record nodes, so kernel_ms keeps working).  Needs a non-default stream
 * (EINVAL with stream 0). */
rapid_status rapid_set_graph(rapid_ctx *ctx, int32_t on);

/* Current position in the schedule: stage index (-1 before seeding), its level and block
 * side, and M.  Host-side only (no synchronisation).  Any pointer may be NULL. */
rapid_status rapid_get_state(rapid_ctx *ctx, int32_t *stage, int32_t *level, int32_t *block,
                             int32_t *M);

/* Full-resolution label map (H x W int32, rows row_pitch_bytes apart, >= 4*W) into a host
 * or device (dst_is_device) buffer owned by the caller.  Synchronises.  ESTATE before
 * seeding. */
rapid_status rapid_read_labels(rapid_ctx *ctx, int32_t *dst, int64_t row_pitch_bytes,
                               int32_t dst_is_device);

/* The current stage's block-resolution label map (nby x nbx int32, row-major, nbx =
 * ceil(W/s), nby = ceil(H/s)) into a host buffer of `capacity` elements.  *nbx_out and
 * *nby_out may be NULL.  Synchronises.  EINVAL when the buffer is too small. */
rapid_status rapid_read_block_labels(rapid_ctx *ctx, int32_t *dst, int64_t capacity,
                                     int32_t *nbx_out, int32_t *nby_out);

/* Statistics S of every label id (host buffer of `capacity` entries).  *M_out (may be
 * NULL) receives M.  Synchronises.  EINVAL when capacity < M. */
rapid_status rapid_read_stats(rapid_ctx *ctx, rapid_sp_stats *dst, int64_t capacity,
                              int64_t *M_out);

/* Per-stage counters of the current run (host struct).  Synchronises. */
rapid_status rapid_read_counters(rapid_ctx *ctx, rapid_counters *dst);

/* Time each stage's refinement launch with CUDA events (0 = off, the default). */
rapid_status rapid_set_profiling(rapid_ctx *ctx, int32_t on);

/* Synchronise the context's stream and return the context's status (ETIMEOUT if a device
 * wait gave up, ECUDA on a CUDA error). */
rapid_status rapid_sync(rapid_ctx *ctx);

/* Topology test table computed by the device code: out[m] = 1 when removing a block whose
 * 3x3 neighbourhood mask is m keeps its superpixel connected (E_topo, Eq. equa:energy1).
 * Bit i of m is neighbour i in the order NW, N, NE, E, SE, S, SW, W (1 = same label).
 * Host buffer of 256 bytes; runs a kernel on the current device and synchronises. */
rapid_status rapid_simple_table(uint8_t *out256);

/* Whole refinement of one small image without allocating any GPU memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call cudaMalloc, such as
 * services whose device memory is fully reserved up front by their own pool allocator, or
 * latency-critical paths where cudaMalloc / cudaFree (which can synchronise the device)
 * are not allowed.  It runs the same kernels as rapid_run (same results, bit for bit), but
 * every byte of working memory comes from one fixed 16 MiB __device__ array inside the
 * library; every GPU that loads the library holds that array until the process exits.
 *
 * p: parameters as for rapid_create (schedule 0 or 1; the prediction uses the brightness
 * stand-in: a context's classifier, scorer and tile shapes do not apply here, and every
 * stage uses the 32 x 16-block tiles).  rgb_dev: H x W interleaved RGB in device memory, rows
 * rgb_pitch_bytes apart (>= 3*W), read only.  labels_dev: device H x W int32 output, rows
 * labels_pitch_bytes apart (>= 4*W, multiple of 4).  stats_dev: device output of
 * stats_capacity entries (>= M), index = label id.  *M_out (host, may be NULL) receives M.
 * cuda_stream: the stream to run on (0 = legacy default).  All buffers belong to the
 * caller.  The call synchronises the stream before returning.
 *
 * Limits: H*W <= RAPID_STATIC_MAX_PIXELS and M <= RAPID_STATIC_MAX_LABELS, and the image's
 * level sums, label maps and per-label arrays must fit the fixed array; otherwise
 * RAPID_ERANGE, with nothing launched.  EINVAL on a bad argument, ECUDA, ETIMEOUT as above.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it for that device, so make the first call on each device before capturing
 * any stream work.  All calls on a device share the array and it keeps the last call's
 * contents; each call re-initialises what must start at zero.  Calls whose GPU work
 * overlaps in time (other streams or host threads) race on the array: serialise them. */
#define RAPID_STATIC_MAX_PIXELS (1 << 19)
#define RAPID_STATIC_MAX_LABELS (1 << 13)
rapid_status rapid_run_static(const rapid_params *p, const uint8_t *rgb_dev, int32_t H, int32_t W,
                              int64_t rgb_pitch_bytes, int32_t *labels_dev, int64_t labels_pitch_bytes,
                              rapid_sp_stats *stats_dev, int64_t stats_capacity, int32_t *M_out,
                              void *cuda_stream);

/* Race check (a debug mode): with on = 1 every label write of a phase also stamps its
 * block with the phase, and a write counts a violation when its block is not of the
 * phase's class, was already written in the phase, or has a block within distance 2
 * written in the same phase -- the independence the 9-phase schedule relies on (two blocks
 * deciding together never share a 3 x 3 window).  rapid_read_race_violations returns the
 * count since the check was first turned on (synchronises); rapid_race_selftest runs the
 * check on three scripted write sequences and returns their counts (expected 0, 2, 1).
 * Costs one stamp per block of device memory and some atomics per move. */
rapid_status rapid_set_race_check(rapid_ctx *ctx, int32_t on);
rapid_status rapid_read_race_violations(rapid_ctx *ctx, int64_t *out);
rapid_status rapid_race_selftest(int64_t *violations3);

/* Test hook for failure handling: the n-th device allocation the library attempts from
 * now on fails as if the device were out of memory (n = 1: the next one); n <= 0 turns it
 * off.  Process-wide; the calls that meet the failure return RAPID_ENOMEM and the context
 * stays destroyable.  Not for production use. */
void rapid_debug_fail_alloc(int64_t n);

/* Human-readable name of a status.  Never NULL. */
const char *rapid_status_string(rapid_status s);

/* Free everything the context owns.  NULL-safe.  Synchronises its stream first. */
void rapid_destroy(rapid_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* RAPID_H */
