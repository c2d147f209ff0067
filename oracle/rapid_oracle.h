/* CPU oracle for the coarse-to-fine topology-preserving superpixel refinement of
 * "RAPID: Regions-of-Interest Detection in Big Histopathological Images"
 * (Sulimowicz & Ahmad, ICME 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct restatement of
 * the method used to check the CUDA path; only the tests, the package smoke check and
 * the bench's CPU-baseline leg may load it.  It shares no code with the CUDA path.
 *
 * Sections followed: Sec. 2.1 (energy Eq. equa:energy1, boundary indicator Eq. bound,
 * block relabel Eq. operation, coarse-to-fine block stages), Sec. 2.2 (multi-scale
 * levels), Sec. 3.1 (size regularity by merging, Eqs. eqa:merge / condtion, energy
 * difference of a merge), Sec. 3.2 (Algorithm RAPID, prediction Eq. predict, boundary
 * superpixels Eq. new_bound, reuse of the coarsest statistics Eq. eq:mu).
 */
#ifndef RAPID_ORACLE_H
#define RAPID_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
  int32_t num_levels;      /* L >= 1; level l (1 = coarsest) has factor f_l = C^(L-l) */
  int32_t ratio_C;         /* compression ratio C (power of two >= 2) */
  int32_t init_block;      /* initial block side, full-res pixels (power of two) */
  int32_t final_grain;     /* stop once the block side would fall below this (power of two) */
  int32_t K;               /* requested superpixel count */
  int32_t size_mode;       /* 0: no size term, 1: hard lower bound, 2: merge (Sec. 3.1) */
  double lambda_pos0;      /* lambda_pos = lambda_pos0 * M / (H*W) */
  double lambda_b;         /* boundary weight per full-res 4-adjacent pixel pair */
  int32_t lo_num, lo_den;  /* lower size bound l = lo_num/lo_den (1/4) */
  int32_t hi_num, hi_den;  /* upper size bound u = hi_num/hi_den (3/2) */
  int32_t predict;         /* 1: prediction and boundary superpixels from level 2 on */
  int32_t reuse;           /* 1: carry the statistics across levels (Eq. eq:mu); 0: recompute */
  int32_t importance_rule; /* 0: block's superpixel must be a boundary superpixel; 1: pair rule */
  int32_t max_sweeps;      /* per stage */
  int64_t h_T;             /* brightness threshold of the stand-in classifier */
  int32_t schedule;        /* 0: a phase visits every block of its class; 1: frontier queue
                              (every block queued at the start of a stage refinement; a phase
                              pops the queued blocks of its class; a move, or an accepted
                              merge at its first requesting block, queues the block's
                              4-neighbours) */
  int32_t pad;
} orc_params;

typedef struct orc_state orc_state;

/* Per-stage counters, 8 int64 each: level, block side, sweeps, eligible, evaluated,
 * moves, merge requests, merges. */
#define ORC_NCOUNT 8

orc_state *orc_create(const uint8_t *rgb, int32_t H, int32_t W, const orc_params *p, int32_t *status);
void orc_destroy(orc_state *st);
int32_t orc_num_stages(const orc_state *st);
int32_t orc_stage_info(const orc_state *st, int32_t i, int32_t *level, int32_t *side);
int32_t orc_seed(orc_state *st);
int32_t orc_phase(orc_state *st, int32_t phase, int64_t *moves, int64_t *merges);
/* the two halves of orc_phase, exposed so tests can inspect the state between them */
int32_t orc_phase_moves(orc_state *st, int32_t phase, int64_t *moves, int64_t *requests);
int32_t orc_phase_merges(orc_state *st, int64_t *merges);
int32_t orc_pending_requests(const orc_state *st, int64_t *blk, int32_t *lab, int64_t cap);
int32_t orc_refine_stage(orc_state *st);
int32_t orc_next_stage(orc_state *st);
int32_t orc_run(orc_state *st);
int32_t orc_get_grid(const orc_state *st, int32_t *stage, int32_t *nbx, int32_t *nby, int32_t *side,
                     int32_t *level, int32_t *M);
int32_t orc_read_block_labels(const orc_state *st, int32_t *dst);
int32_t orc_read_labels(const orc_state *st, int32_t *dst);
int32_t orc_read_stats(const orc_state *st, int64_t *dst7, int8_t *y, uint8_t *important);
int32_t orc_read_counters(const orc_state *st, int64_t *dst);
int32_t orc_read_pyramid(const orc_state *st, int32_t level, int64_t *dst6);
int32_t orc_level_dims(const orc_state *st, int32_t level, int32_t *Wl, int32_t *Hl, int32_t *f);
double orc_lambda_pos(const orc_state *st);
int32_t orc_simple_lut(uint8_t *dst256);
/* Threads of the phase decisions in a build with ORC_OPENMP (the all-core baseline): n > 0
 * sets them; returns the number in use (1 in the plain build).  Results do not depend on
 * it. */
int32_t orc_set_threads(int32_t n);
int32_t orc_run_fifo(orc_state *st);
/* Eq. predict with the linear classifier theta[0] + theta[1..4] . F over the features F of
 * each superpixel (NULL: the integer brightness stand-in), and the features of the last
 * prediction (M x 4: absolute brightness, comparative brightness, extra-region and
 * intra-region dissimilarity). */
int32_t orc_set_classifier(orc_state *st, const double *theta5);
/* Pruned sweeps (the pruning that the learned block scorer drives): keep mask of stage i
 * over its block grid (nbx * nby bytes, nonzero = kept), or NULL for full sweeps.  The
 * stage then sweeps testing and deciding only the kept eligible blocks until a sweep
 * changes nothing, then full sweeps until a full sweep changes nothing, within max_sweeps.
 * Sweep schedule only. */
int32_t orc_set_keep_mask(orc_state *st, int32_t i, const uint8_t *mask, int64_t n);
int32_t orc_read_features(const orc_state *st, double *dst4);

#ifdef __cplusplus
}
#endif
#endif
