/* CPU oracle for the coarse-to-fine topology-preserving superpixel refinement (CTFTPS)
 * with the size-regularity merge, prediction and coarsest-level reuse of RAPID
 * (Sulimowicz & Ahmad, ICME 2017).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow and literal, written to be checked by eye against
 * the paper.  Only the tests, the package smoke check and the bench's CPU-baseline leg use
 * it.  It shares no code with the CUDA path.  Build with -ffp-contract=off: every
 * floating-point operation below is a separately rounded IEEE double operation in the
 * order written.
 *
 * Conventions (the readings of the paper this file implements):
 *  - Colour is raw RGB (Sec. 2.1 "colour intensity"); positions are 0-based full-res
 *    pixel coordinates; all sums are exact int64.
 *  - Level l (1 = coarsest) is the image box-summed by f_l = C^(L-l) (Sec. 2.2 "resizes").
 *    A coarse pixel keeps the exact sums (count, R, G, B, x, y) of its f x f footprint, so
 *    every energy is in full-res units at every level and the statistics carry over
 *    unchanged from level to level; this is Eq. eq:mu exactly (reuse, Sec. 3.2).
 *  - A stage works on square blocks of side s full-res pixels; s halves from stage to
 *    stage ("each block with smaller regular grid", Algorithm RAPID) from the initial block
 *    down to the final grain; stage s belongs to the coarsest level whose factor divides it.
 *  - Boundary blocks are relabelled in a 9-phase schedule: phase (py,px) takes the blocks
 *    with by%3==py and bx%3==px; all of them decide against a snapshot of the statistics
 *    taken at the start of the phase, then the moves are applied together.  (The paper's
 *    queue updates after every move; the sequential FIFO variant orc_run_fifo keeps that
 *    order for quality comparison.)
 *  - With schedule 1 the phases work through a queue instead (the boundary queue of
 *    Sec. 2.1 kept as a set of flags, one per block): every block is queued when the
 *    refinement of a stage starts, a phase takes the queued blocks of its class off the
 *    queue and evaluates those, and each block that moves -- and each accepted merge, at
 *    the block whose request was accepted -- puts its 4-neighbours on the queue.
 */
#include "rapid_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXL 8
#define MAXSTAGES 64

struct orc_state {
  orc_params p;
  int32_t H, W;
  uint8_t *rgb;
  int32_t L;
  int32_t f[MAXL + 1];
  int32_t Wl[MAXL + 1], Hl[MAXL + 1];
  int64_t *pyr[MAXL + 1]; /* 6 sums per coarse pixel: count, R, G, B, x, y (NULL when f==1) */
  int32_t nstages;
  int32_t st_level[MAXSTAGES], st_side[MAXSTAGES];
  int32_t cur; /* current stage, -1 before seeding */
  int32_t *lab;
  int32_t nbx, nby, side, level;
  int32_t M;
  int64_t *N, *R, *G, *B, *X, *Y, *init;
  int8_t *y;
  uint8_t *imp;
  int32_t imp_on;
  double lam_pos, lam_b2;
  uint8_t lut[256];
  int64_t cnt[MAXSTAGES][ORC_NCOUNT];
  int64_t *req_blk; /* merge requests of the current phase, ascending block order */
  int32_t *req_lab;
  int64_t nreq, req_cap;
  int64_t phase_moves;
  uint32_t *visit; /* flood-fill marks: visit[i] == visit_id means visited in this fill */
  uint32_t visit_id;
  int64_t *queue;
  uint8_t *queued; /* schedule 1: 1 when the block is on the queue */
  int32_t use_theta; /* 1: Eq. predict evaluates the linear classifier theta on F */
  double theta[5];
  double *feat;      /* M x 4 features of the last prediction */
  uint8_t *keep[MAXSTAGES]; /* pruned sweeps: the stage's keep mask over its block grid (NULL: none) */
  int32_t pruned;           /* 1 while the current stage sweeps with its keep mask */
};

enum { C_LEVEL, C_SIDE, C_SWEEPS, C_ELIG, C_EVAL, C_MOVES, C_REQ, C_MERGES };

/* ---------------------------------------------------------------- simple-point test */
/* Eq. equa:energy1, E_topo: a superpixel must stay one connected component.  Removing a
 * block p from its label a keeps a connected when the neighbours of p labelled a that are
 * 4-adjacent to p exist and are all joined to each other by 4-paths through the other
 * a-labelled cells of the 3x3 window (centre excluded).  Bit i of the mask is neighbour i
 * in the order NW, N, NE, E, SE, S, SW, W; a set bit means "labelled a".  Decided here by
 * a breadth-first search over the 3x3 grid. */
static const int RING_DX[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
static const int RING_DY[8] = {-1, -1, -1, 0, 1, 1, 1, 0};

static int simple_by_bfs(unsigned mask) {
  int grid[3][3];
  memset(grid, 0, sizeof grid);
  for (int i = 0; i < 8; i++)
    if (mask & (1u << i)) grid[1 + RING_DY[i]][1 + RING_DX[i]] = 1;
  /* 4-neighbours of the centre: N (0,-1), E (1,0), S (0,1), W (-1,0) */
  const int fx[4] = {0, 1, 0, -1}, fy[4] = {-1, 0, 1, 0};
  int start = -1;
  for (int j = 0; j < 4; j++)
    if (grid[1 + fy[j]][1 + fx[j]]) { start = j; break; }
  if (start < 0) return 0;
  int seen[3][3];
  memset(seen, 0, sizeof seen);
  int qx[9], qy[9], qh = 0, qt = 0;
  qx[qt] = 1 + fx[start]; qy[qt] = 1 + fy[start]; qt++;
  seen[1 + fy[start]][1 + fx[start]] = 1;
  while (qh < qt) {
    int cx = qx[qh], cy = qy[qh]; qh++;
    for (int j = 0; j < 4; j++) {
      int nx = cx + fx[j], ny = cy + fy[j];
      if (nx < 0 || nx > 2 || ny < 0 || ny > 2) continue;
      if (nx == 1 && ny == 1) continue; /* the centre is being removed */
      if (!grid[ny][nx] || seen[ny][nx]) continue;
      seen[ny][nx] = 1;
      qx[qt] = nx; qy[qt] = ny; qt++;
    }
  }
  for (int j = 0; j < 4; j++)
    if (grid[1 + fy[j]][1 + fx[j]] && !seen[1 + fy[j]][1 + fx[j]]) return 0;
  return 1;
}

/* Threads of the phase decisions (an ORC_OPENMP build; ignored otherwise); returns the
 * number in use. */
#ifdef ORC_OPENMP
#include <omp.h>
#endif
int32_t orc_set_threads(int32_t n) {
#ifdef ORC_OPENMP
  if (n > 0) omp_set_num_threads(n);
  return (int32_t)omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int32_t orc_simple_lut(uint8_t *dst256) {
  for (unsigned m = 0; m < 256; m++) dst256[m] = (uint8_t)simple_by_bfs(m);
  return 0;
}

/* ---------------------------------------------------------------- helpers */
static int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
static int32_t ceil_div(int32_t a, int32_t b) { return (a + b - 1) / b; }
static int is_pow2(int32_t v) { return v > 0 && (v & (v - 1)) == 0; }

/* Sums of one coarse pixel (X,Y) of level l: count, R, G, B, x, y over its footprint. */
static void cell_sums(const orc_state *st, int32_t l, int32_t X, int32_t Y, int64_t c[6]) {
  if (st->f[l] == 1) {
    const uint8_t *px = st->rgb + 3 * ((int64_t)Y * st->W + X);
    c[0] = 1; c[1] = px[0]; c[2] = px[1]; c[3] = px[2]; c[4] = X; c[5] = Y;
  } else {
    const int64_t *q = st->pyr[l] + 6 * ((int64_t)Y * st->Wl[l] + X);
    for (int i = 0; i < 6; i++) c[i] = q[i];
  }
}

/* Sums of block (bx,by) of the current stage: the sum of the level-l coarse pixels it
 * covers (a block of side s covers (s/f_l)^2 of them, clipped at the image edge). */
static void block_sums(const orc_state *st, int32_t bx, int32_t by, int64_t out[6]) {
  int32_t l = st->level, k = st->side / st->f[l];
  for (int i = 0; i < 6; i++) out[i] = 0;
  for (int32_t Y = by * k; Y < by * k + k && Y < st->Hl[l]; Y++)
    for (int32_t X = bx * k; X < bx * k + k && X < st->Wl[l]; X++) {
      int64_t c[6];
      cell_sums(st, l, X, Y, c);
      for (int i = 0; i < 6; i++) out[i] += c[i];
    }
}

/* Block geometry in full-res pixels (ragged at the right and bottom edges). */
static int32_t block_w(const orc_state *st, int32_t bx) {
  return (int32_t)imin64((int64_t)st->side * (bx + 1), st->W) - st->side * bx;
}
static int32_t block_h(const orc_state *st, int32_t by) {
  return (int32_t)imin64((int64_t)st->side * (by + 1), st->H) - st->side * by;
}

/* ---------------------------------------------------------------- create / schedule */
orc_state *orc_create(const uint8_t *rgb, int32_t H, int32_t W, const orc_params *p, int32_t *status) {
  *status = 1;
  if (!rgb || !p || H <= 0 || W <= 0) return NULL;
  if (p->num_levels < 1 || p->num_levels > MAXL) return NULL;
  if (p->num_levels > 1 && (!is_pow2(p->ratio_C) || p->ratio_C < 2)) return NULL;
  if (!is_pow2(p->init_block) || !is_pow2(p->final_grain) || p->K < 1) return NULL;
  if (p->size_mode < 0 || p->size_mode > 2 || p->max_sweeps < 1) return NULL;
  if (p->lo_den <= 0 || p->hi_den <= 0 || p->lo_num < 0 || p->hi_num < 0) return NULL;
  orc_state *st = (orc_state *)calloc(1, sizeof *st);
  if (!st) { *status = 2; return NULL; }
  st->p = *p;
  st->H = H; st->W = W;
  st->rgb = (uint8_t *)malloc((size_t)H * W * 3);
  if (!st->rgb) { free(st); *status = 2; return NULL; }
  memcpy(st->rgb, rgb, (size_t)H * W * 3);
  st->L = p->num_levels;
  for (int32_t l = 1; l <= st->L; l++) {
    int32_t f = 1;
    for (int32_t i = 0; i < st->L - l; i++) f *= (st->L > 1 ? p->ratio_C : 1);
    st->f[l] = f;
    st->Wl[l] = ceil_div(W, f);
    st->Hl[l] = ceil_div(H, f);
  }
  /* Level images (Sec. 2.2): literal box sums over every full-res pixel. */
  for (int32_t l = 1; l <= st->L; l++) {
    if (st->f[l] == 1) continue;
    int64_t *q = (int64_t *)calloc((size_t)st->Wl[l] * st->Hl[l] * 6, sizeof(int64_t));
    if (!q) { orc_destroy(st); *status = 2; return NULL; }
    st->pyr[l] = q;
    for (int32_t y = 0; y < H; y++)
      for (int32_t x = 0; x < W; x++) {
        int64_t *c = q + 6 * ((int64_t)(y / st->f[l]) * st->Wl[l] + x / st->f[l]);
        const uint8_t *px = rgb + 3 * ((int64_t)y * W + x);
        c[0] += 1; c[1] += px[0]; c[2] += px[1]; c[3] += px[2]; c[4] += x; c[5] += y;
      }
  }
  /* Stages: block side halves from the initial block (at least f_1) to the final grain;
   * each side belongs to the coarsest level whose factor is <= the side. */
  int32_t s = p->init_block < st->f[1] ? st->f[1] : p->init_block;
  st->nstages = 0;
  while (s >= 1 && s >= p->final_grain && st->nstages < MAXSTAGES) {
    int32_t lev = 0;
    for (int32_t l = 1; l <= st->L; l++)
      if (st->f[l] <= s) { lev = l; break; }
    if (lev == 0) break; /* finer than full resolution */
    st->st_level[st->nstages] = lev;
    st->st_side[st->nstages] = s;
    st->nstages++;
    s /= 2;
  }
  if (st->nstages == 0) { /* final grain above the initial block: seed only */
    st->st_level[0] = 1;
    st->st_side[0] = p->init_block < st->f[1] ? st->f[1] : p->init_block;
    st->nstages = 1;
  }
  int32_t s0 = st->st_side[0];
  size_t cap = (size_t)ceil_div(W, st->st_side[st->nstages - 1]) * ceil_div(H, st->st_side[st->nstages - 1]);
  (void)s0;
  st->lab = (int32_t *)malloc(cap * sizeof(int32_t));
  st->visit = (uint32_t *)calloc(cap, sizeof(uint32_t));
  st->queue = (int64_t *)malloc(cap * sizeof(int64_t));
  st->queued = (uint8_t *)malloc(cap);
  orc_simple_lut(st->lut);
  st->cur = -1;
  if (!st->lab || !st->visit || !st->queue || !st->queued) { orc_destroy(st); *status = 2; return NULL; }
  *status = 0;
  return st;
}

void orc_destroy(orc_state *st) {
  if (!st) return;
  free(st->rgb);
  for (int l = 0; l <= MAXL; l++) free(st->pyr[l]);
  free(st->lab);
  free(st->visit);
  free(st->queue);
  free(st->queued);
  free(st->req_blk);
  free(st->req_lab);
  free(st->N); free(st->R); free(st->G); free(st->B); free(st->X); free(st->Y); free(st->init);
  free(st->y); free(st->imp); free(st->feat);
  for (int i = 0; i < MAXSTAGES; i++) free(st->keep[i]);
  free(st);
}

int32_t orc_num_stages(const orc_state *st) { return st->nstages; }

int32_t orc_stage_info(const orc_state *st, int32_t i, int32_t *level, int32_t *side) {
  if (i < 0 || i >= st->nstages) return 1;
  *level = st->st_level[i];
  *side = st->st_side[i];
  return 0;
}

static void set_stage_grid(orc_state *st, int32_t i) {
  st->cur = i;
  st->pruned = st->keep[i] != NULL; /* a stage with a keep mask starts with pruned sweeps */
  st->level = st->st_level[i];
  st->side = st->st_side[i];
  st->nbx = ceil_div(st->W, st->side);
  st->nby = ceil_div(st->H, st->side);
  st->cnt[i][C_LEVEL] = st->level;
  st->cnt[i][C_SIDE] = st->side;
  memset(st->queued, 1, (size_t)st->nbx * st->nby);
}

/* Schedule 1: the 4-neighbours of block blk that lie on the grid go on the queue. */
static void queue_neighbours(orc_state *st, int64_t blk) {
  int32_t bx = (int32_t)(blk % st->nbx), by = (int32_t)(blk / st->nbx);
  if (by > 0) st->queued[blk - st->nbx] = 1;
  if (bx > 0) st->queued[blk - 1] = 1;
  if (bx + 1 < st->nbx) st->queued[blk + 1] = 1;
  if (by + 1 < st->nby) st->queued[blk + st->nbx] = 1;
}

/* Statistics S of every label recomputed from the label map and the current level
 * (Algorithm RAPID, "compute initial mu and c ... store in S"). */
static void recompute_stats(orc_state *st) {
  for (int32_t k = 0; k < st->M; k++) st->N[k] = st->R[k] = st->G[k] = st->B[k] = st->X[k] = st->Y[k] = 0;
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++) {
      int64_t s[6];
      block_sums(st, bx, by, s);
      int32_t k = st->lab[(int64_t)by * st->nbx + bx];
      st->N[k] += s[0]; st->R[k] += s[1]; st->G[k] += s[2]; st->B[k] += s[3]; st->X[k] += s[4]; st->Y[k] += s[5];
    }
}

/* Seeding (Algorithm RAPID, "initialize superpixels to be regular grids"): gx x gy grid
 * cells over the first stage's block grid, gx = round(sqrt(K W / H)), gy = round(K / gx),
 * clamped to the block grid. */
int32_t orc_seed(orc_state *st) {
  memset(st->cnt, 0, sizeof st->cnt);
  set_stage_grid(st, 0);
  double gxd = sqrt((double)st->p.K * (double)st->W / (double)st->H);
  int32_t gx = (int32_t)floor(gxd + 0.5);
  if (gx < 1) gx = 1;
  int32_t gy = (int32_t)floor((double)st->p.K / (double)gx + 0.5);
  if (gy < 1) gy = 1;
  if (gx > st->nbx) gx = st->nbx;
  if (gy > st->nby) gy = st->nby;
  st->M = gx * gy;
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++)
      st->lab[(int64_t)by * st->nbx + bx] =
          (int32_t)(((int64_t)by * gy / st->nby) * gx + ((int64_t)bx * gx / st->nbx));
  size_t M = (size_t)st->M;
  free(st->N); free(st->R); free(st->G); free(st->B); free(st->X); free(st->Y); free(st->init);
  free(st->y); free(st->imp); free(st->feat);
  st->feat = (double *)calloc(M * 4, 8);
  st->N = (int64_t *)calloc(M, 8); st->R = (int64_t *)calloc(M, 8); st->G = (int64_t *)calloc(M, 8);
  st->B = (int64_t *)calloc(M, 8); st->X = (int64_t *)calloc(M, 8); st->Y = (int64_t *)calloc(M, 8);
  st->init = (int64_t *)calloc(M, 8);
  st->y = (int8_t *)calloc(M, 1);
  st->imp = (uint8_t *)calloc(M, 1);
  if (!st->N || !st->R || !st->G || !st->B || !st->X || !st->Y || !st->init || !st->y || !st->imp || !st->feat)
    return 2;
  recompute_stats(st);
  for (int32_t k = 0; k < st->M; k++) st->init[k] = st->N[k];
  /* lambda_pos scales with the initial superpixel area H*W/M (position energy per pixel
   * is then independent of image size). */
  st->lam_pos = st->p.lambda_pos0 * ((double)st->M / ((double)st->H * (double)st->W));
  st->lam_b2 = 2.0 * st->p.lambda_b; /* Eq. equa:energy1 sums E_b over p and q in N4(p): each pair twice */
  st->imp_on = 0;
  return 0;
}

double orc_lambda_pos(const orc_state *st) { return st->lam_pos; }

/* ---------------------------------------------------------------- energy */
/* Block energy of block sums b (count w, colour S, position P) under label means
 * (c, mu), up to a label-independent constant (Eq. equa:energy1):
 *   sum_pixels |I - c|^2 = sum I^2 - 2 S.c + w |c|^2   (E_col)
 *   sum_pixels |p - mu|^2 = sum p^2 - 2 P.mu + w |mu|^2 (E_pos)
 * plus the boundary-length term 2 lambda_b Bk, Bk = full-res 4-adjacent pixel pairs across
 * the block perimeter whose other side is not labelled k. */
static double block_energy(const int64_t b[6], double cR, double cG, double cB, double mx, double my,
                           int64_t Bk, double lam_pos, double lam_b2) {
  double w = (double)b[0];
  double eR = (w * cR) * cR - (double)(2 * b[1]) * cR;
  double eG = (w * cG) * cG - (double)(2 * b[2]) * cG;
  double eB = (w * cB) * cB - (double)(2 * b[3]) * cB;
  double ec = (eR + eG) + eB;
  double ex = (w * mx) * mx - (double)(2 * b[4]) * mx;
  double ey = (w * my) * my - (double)(2 * b[5]) * my;
  double ep = ex + ey;
  return (ec + lam_pos * ep) + lam_b2 * (double)Bk;
}

/* Merge cost of labels a and n (Sec. 3.1: the energy change of a merge involves only the
 * two superpixels; for the colour and position terms it is the Ward increase
 * Na Nn / (Na + Nn) (|ca - cn|^2 + lambda_pos |mua - mun|^2)). */
static double ward(const orc_state *st, int32_t a, int32_t n) {
  double ca0 = (double)st->R[a] / (double)st->N[a], ca1 = (double)st->G[a] / (double)st->N[a];
  double ca2 = (double)st->B[a] / (double)st->N[a];
  double ma0 = (double)st->X[a] / (double)st->N[a], ma1 = (double)st->Y[a] / (double)st->N[a];
  double cn0 = (double)st->R[n] / (double)st->N[n], cn1 = (double)st->G[n] / (double)st->N[n];
  double cn2 = (double)st->B[n] / (double)st->N[n];
  double mn0 = (double)st->X[n] / (double)st->N[n], mn1 = (double)st->Y[n] / (double)st->N[n];
  double t = ((double)st->N[a] * (double)st->N[n]) / (double)(st->N[a] + st->N[n]);
  double d0 = ca0 - cn0, d1 = ca1 - cn1, d2 = ca2 - cn2;
  double dc = (d0 * d0 + d1 * d1) + d2 * d2;
  double e0 = ma0 - mn0, e1 = ma1 - mn1;
  double dm = e0 * e0 + e1 * e1;
  return t * (dc + st->lam_pos * dm);
}

/* ---------------------------------------------------------------- one phase */
typedef struct { int64_t blk; int32_t a, k; } move_t;

static int32_t label_at(const orc_state *st, int32_t bx, int32_t by) {
  if (bx < 0 || by < 0 || bx >= st->nbx || by >= st->nby) return -1;
  return st->lab[(int64_t)by * st->nbx + bx];
}

/* Eligibility of block p (Eq. bound; from level 2 on with prediction also Eq. new_bound /
 * the boundary-superpixel rule): returns 1 when p is queued. */
static int eligible(const orc_state *st, int32_t bx, int32_t by, int32_t a) {
  int32_t nb[4] = {label_at(st, bx, by - 1), label_at(st, bx - 1, by), label_at(st, bx + 1, by),
                   label_at(st, bx, by + 1)};
  int boundary = 0;
  for (int j = 0; j < 4; j++)
    if (nb[j] >= 0 && nb[j] != a) boundary = 1;
  if (!boundary) return 0;
  if (!st->imp_on) return 1;
  if (st->p.importance_rule == 0) return st->imp[a] != 0;
  for (int j = 0; j < 4; j++)
    if (nb[j] >= 0 && nb[j] != a && st->y[nb[j]] != st->y[a]) return 1;
  return 0;
}

static unsigned neighbour_mask(const orc_state *st, int32_t bx, int32_t by, int32_t a) {
  unsigned m = 0;
  for (int i = 0; i < 8; i++)
    if (label_at(st, bx + RING_DX[i], by + RING_DY[i]) == a) m |= 1u << i;
  return m;
}

/* Decide block p against the means (c, mu) and counts N0: returns 0 no move, 1 move to
 * *k_out, 2 merge request (size bound hit, size_mode 2). */
static int decide(const orc_state *st, int32_t bx, int32_t by, const double *cR, const double *cG,
                  const double *cB, const double *mX, const double *mY, const int64_t *N0, int32_t *k_out,
                  int64_t *elig, int64_t *eval) {
  int32_t a = st->lab[(int64_t)by * st->nbx + bx];
  if (!eligible(st, bx, by, a)) return 0;
  (*elig)++;
  /* pruned sweeps: an eligible block that the stage's keep mask leaves out gets neither
   * the topology test nor a decision (it stays as it is) */
  if (st->pruned && !st->keep[st->cur][(int64_t)by * st->nbx + bx]) return 0;
  if (!st->lut[neighbour_mask(st, bx, by, a)]) return 0;
  (*eval)++;
  int64_t b[6];
  block_sums(st, bx, by, b);
  int32_t bw = block_w(st, bx), bh = block_h(st, by);
  /* 4-neighbours N, W, E, S and the full-res edge each shares with p */
  int32_t nb[4] = {label_at(st, bx, by - 1), label_at(st, bx - 1, by), label_at(st, bx + 1, by),
                   label_at(st, bx, by + 1)};
  int32_t len[4] = {bw, bh, bh, bw};
  int64_t Ba = 0;
  for (int j = 0; j < 4; j++)
    if (nb[j] >= 0 && nb[j] != a) Ba += len[j];
  double ea = block_energy(b, cR[a], cG[a], cB[a], mX[a], mY[a], Ba, st->lam_pos, st->lam_b2);
  int32_t bestk = -1;
  double best = 0.0;
  for (int j = 0; j < 4; j++) {
    int32_t k = nb[j];
    if (k < 0 || k == a) continue;
    int dup = 0;
    for (int i = 0; i < j; i++)
      if (nb[i] == k) dup = 1;
    if (dup) continue;
    int64_t Bk = 0;
    for (int i = 0; i < 4; i++)
      if (nb[i] >= 0 && nb[i] != k) Bk += len[i];
    double dE = block_energy(b, cR[k], cG[k], cB[k], mX[k], mY[k], Bk, st->lam_pos, st->lam_b2) - ea;
    if (bestk < 0 || dE < best || (dE == best && k < bestk)) {
      best = dE;
      bestk = k;
    }
  }
  if (bestk < 0 || !(best < 0.0)) return 0; /* Eq. operation: keep the label unless a neighbour lowers E */
  if (st->p.size_mode != 0 &&
      (int64_t)st->p.lo_den * (N0[a] - b[0]) < (int64_t)st->p.lo_num * st->init[a]) {
    /* Sec. 3.1: the superpixel would fall below l * InitSize */
    return st->p.size_mode == 2 ? 2 : 0;
  }
  *k_out = bestk;
  return 1;
}

static void apply_move(orc_state *st, int64_t blk, int32_t a, int32_t k) {
  int32_t bx = (int32_t)(blk % st->nbx), by = (int32_t)(blk / st->nbx);
  int64_t b[6];
  block_sums(st, bx, by, b);
  st->lab[blk] = k;
  st->N[a] -= b[0]; st->R[a] -= b[1]; st->G[a] -= b[2]; st->B[a] -= b[3]; st->X[a] -= b[4]; st->Y[a] -= b[5];
  st->N[k] += b[0]; st->R[k] += b[1]; st->G[k] += b[2]; st->B[k] += b[3]; st->X[k] += b[4]; st->Y[k] += b[5];
}

/* Merge target for label a (Eqs. eqa:merge, condtion): over N_s(a), the labels
 * 4-adjacent to a, those whose size after taking a stays within u * InitSize, the least
 * merge cost; ties to the smaller id; -1 if none.  Superpixel a is one 4-connected
 * component (E_topo; seeding, moves, splits and merges all keep it so), so a flood fill
 * from any block of a visits all of a. */
static int32_t merge_target(const orc_state *st, int32_t a, int64_t from_blk) {
  int32_t best = -1;
  double bw = 0.0;
  const int dx[4] = {0, -1, 1, 0}, dy[4] = {-1, 0, 0, 1};
  int64_t nb = (int64_t)st->nbx * st->nby;
  orc_state *ms = (orc_state *)st; /* the fill marks are scratch, not state */
  uint32_t id = ++ms->visit_id;
  if (id == 0) { /* wrapped: clear the marks */
    memset(ms->visit, 0, sizeof(uint32_t) * (size_t)nb);
    id = ++ms->visit_id;
  }
  uint32_t *seen = ms->visit;
  int64_t *q = ms->queue;
  int64_t qh = 0, qt = 0;
  q[qt++] = from_blk;
  seen[from_blk] = id;
  while (qh < qt) {
    int64_t i = q[qh++];
    int32_t bx = (int32_t)(i % st->nbx), by = (int32_t)(i / st->nbx);
    for (int j = 0; j < 4; j++) {
      int32_t n = label_at(st, bx + dx[j], by + dy[j]);
      if (n < 0) continue;
      int64_t ni = (int64_t)(by + dy[j]) * st->nbx + (bx + dx[j]);
      if (n == a) {
        if (seen[ni] != id) { seen[ni] = id; q[qt++] = ni; }
        continue;
      }
      if ((int64_t)st->p.hi_den * (st->N[n] + st->N[a]) > (int64_t)st->p.hi_num * st->init[n]) continue;
      double w = ward(st, a, n);
      if (best < 0 || w < bw || (w == bw && n < best)) {
        bw = w;
        best = n;
      }
    }
  }
  return best;
}

/* First half of a phase: every block of the phase decides against a snapshot of the
 * statistics taken at the start of the phase; the moves are then applied together
 * (Algorithm RAPID, "update mu and c") and the merge requests are kept for the second
 * half. */
int32_t orc_phase_moves(orc_state *st, int32_t phase, int64_t *moves_out, int64_t *requests_out) {
  if (st->cur < 0 || phase < 0 || phase > 8) return 4;
  int32_t py = phase / 3, px = phase % 3, M = st->M;
  double *cR = (double *)malloc(sizeof(double) * M), *cG = (double *)malloc(sizeof(double) * M);
  double *cB = (double *)malloc(sizeof(double) * M), *mX = (double *)malloc(sizeof(double) * M);
  double *mY = (double *)malloc(sizeof(double) * M);
  int64_t *N0 = (int64_t *)malloc(sizeof(int64_t) * M);
  for (int32_t k = 0; k < M; k++) {
    N0[k] = st->N[k];
    if (st->N[k] > 0) {
      double n = (double)st->N[k];
      cR[k] = (double)st->R[k] / n; cG[k] = (double)st->G[k] / n; cB[k] = (double)st->B[k] / n;
      mX[k] = (double)st->X[k] / n; mY[k] = (double)st->Y[k] / n;
    } else {
      cR[k] = cG[k] = cB[k] = mX[k] = mY[k] = 0.0;
    }
  }
  int64_t nph = (int64_t)ceil_div(st->nbx - px > 0 ? st->nbx - px : 0, 3) * ceil_div(st->nby - py > 0 ? st->nby - py : 0, 3);
  if (nph < 1) nph = 1;
  move_t *mv = (move_t *)malloc(sizeof(move_t) * (size_t)nph);
  if (st->req_cap < nph) {
    free(st->req_blk); free(st->req_lab);
    st->req_blk = (int64_t *)malloc(sizeof(int64_t) * (size_t)nph);
    st->req_lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)nph);
    st->req_cap = nph;
  }
  int64_t nmv = 0;
  st->nreq = 0;
  int64_t *c = st->cnt[st->cur];
  /* Every block of the phase decides on its own (their windows are disjoint and all read
   * the phase snapshot): outcome r[j] and target k[j] of the class's j-th block, listed
   * afterwards in block order.  Built with ORC_OPENMP the decisions run on all cores; the
   * result is the same for any thread count. */
  int64_t ncx = ceil_div(st->nbx - px > 0 ? st->nbx - px : 0, 3), ncy = ceil_div(st->nby - py > 0 ? st->nby - py : 0, 3);
  int8_t *r = (int8_t *)malloc((size_t)nph);
  int32_t *kk = (int32_t *)malloc(sizeof(int32_t) * (size_t)nph);
  int64_t elig = 0, eval = 0;
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(static) reduction(+ : elig, eval)
#endif
  for (int64_t j = 0; j < ncx * ncy; j++) {
    int32_t by = py + 3 * (int32_t)(j / ncx), bx = px + 3 * (int32_t)(j % ncx);
    int64_t blk = (int64_t)by * st->nbx + bx;
    r[j] = 0;
    kk[j] = -1;
    if (st->p.schedule == 1) { /* only queued blocks, which leave the queue */
      if (!st->queued[blk]) continue;
      st->queued[blk] = 0;
    }
    int64_t e = 0, v = 0;
    r[j] = (int8_t)decide(st, bx, by, cR, cG, cB, mX, mY, N0, &kk[j], &e, &v);
    elig += e;
    eval += v;
  }
  c[C_ELIG] += elig;
  c[C_EVAL] += eval;
  for (int64_t j = 0; j < ncx * ncy; j++) {
    int64_t blk = (int64_t)(py + 3 * (j / ncx)) * st->nbx + px + 3 * (j % ncx);
    if (r[j] == 1) { mv[nmv].blk = blk; mv[nmv].a = st->lab[blk]; mv[nmv].k = kk[j]; nmv++; }
    if (r[j] == 2) { st->req_blk[st->nreq] = blk; st->req_lab[st->nreq] = st->lab[blk]; st->nreq++; }
  }
  free(r);
  free(kk);
  for (int64_t i = 0; i < nmv; i++) {
    apply_move(st, mv[i].blk, mv[i].a, mv[i].k);
    if (st->p.schedule == 1) queue_neighbours(st, mv[i].blk);
  }
  c[C_MOVES] += nmv;
  c[C_REQ] += st->nreq;
  st->phase_moves = nmv;
  if (moves_out) *moves_out = nmv;
  if (requests_out) *requests_out = st->nreq;
  free(cR); free(cG); free(cB); free(mX); free(mY); free(N0); free(mv);
  return 0;
}

/* Second half of a phase, the merges (Sec. 3.1): each request's target is chosen against
 * the state after the moves; requests are accepted in ascending block order unless the
 * source or the target already took part in an accepted merge of this phase; accepted
 * merges are applied together (relabel a -> n, S_n += S_a, S_a = 0). */
int32_t orc_phase_merges(orc_state *st, int64_t *merges_out) {
  if (st->cur < 0) return 4;
  int32_t M = st->M;
  int64_t nmerge = 0;
  if (st->nreq > 0) {
    int32_t *tgt = (int32_t *)malloc(sizeof(int32_t) * (size_t)st->nreq);
#ifdef ORC_OPENMP
    /* all-core build: one search per requested label (every block of a connected label
     * reaches the same neighbours, so the target depends on the label alone) */
    int32_t *memo = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    for (int32_t k = 0; k < M; k++) memo[k] = -2;
    for (int64_t i = 0; i < st->nreq; i++) {
      int32_t a = st->req_lab[i];
      if (memo[a] == -2) memo[a] = merge_target(st, a, st->req_blk[i]);
      tgt[i] = memo[a];
    }
    free(memo);
#else
    for (int64_t i = 0; i < st->nreq; i++) tgt[i] = merge_target(st, st->req_lab[i], st->req_blk[i]);
#endif
    uint8_t *inv = (uint8_t *)calloc((size_t)M, 1);
    int32_t *to = (int32_t *)malloc(sizeof(int32_t) * M);
    for (int32_t k = 0; k < M; k++) to[k] = -1;
    for (int64_t i = 0; i < st->nreq; i++) {
      int32_t a = st->req_lab[i], n = tgt[i];
      if (n < 0 || inv[a] || inv[n]) continue;
      inv[a] = inv[n] = 1;
      to[a] = n;
      nmerge++;
      if (st->p.schedule == 1) queue_neighbours(st, st->req_blk[i]);
    }
    if (nmerge > 0) {
      for (int64_t i = 0; i < (int64_t)st->nbx * st->nby; i++)
        if (to[st->lab[i]] >= 0) st->lab[i] = to[st->lab[i]];
      for (int32_t a = 0; a < M; a++) {
        int32_t n = to[a];
        if (n < 0) continue;
        st->N[n] += st->N[a]; st->R[n] += st->R[a]; st->G[n] += st->G[a]; st->B[n] += st->B[a];
        st->X[n] += st->X[a]; st->Y[n] += st->Y[a];
        st->N[a] = st->R[a] = st->G[a] = st->B[a] = st->X[a] = st->Y[a] = 0;
      }
    }
    free(tgt); free(inv); free(to);
  }
  st->nreq = 0;
  st->cnt[st->cur][C_MERGES] += nmerge;
  if (merges_out) *merges_out = nmerge;
  return 0;
}

int32_t orc_pending_requests(const orc_state *st, int64_t *blk, int32_t *lab, int64_t cap) {
  int64_t n = st->nreq < cap ? st->nreq : cap;
  for (int64_t i = 0; i < n; i++) { blk[i] = st->req_blk[i]; lab[i] = st->req_lab[i]; }
  return (int32_t)n;
}

int32_t orc_phase(orc_state *st, int32_t phase, int64_t *moves_out, int64_t *merges_out) {
  int32_t r = orc_phase_moves(st, phase, moves_out, NULL);
  if (r) return r;
  return orc_phase_merges(st, merges_out);
}

/* Sweeps of the current stage until one makes no move and no merge ("until the queue is
 * empty"), or max_sweeps.  A stage with a keep mask first sweeps pruned (only the kept
 * eligible blocks are tested and decided) until a pruned sweep changes nothing, then goes
 * on with full sweeps until a full sweep changes nothing; all sweeps count against
 * max_sweeps. */
int32_t orc_refine_stage(orc_state *st) {
  if (st->cur < 0) return 4;
  memset(st->queued, 1, (size_t)st->nbx * st->nby); /* schedule 1: every block queued */
  for (int32_t s = 0; s < st->p.max_sweeps; s++) {
    int64_t changes = 0;
    for (int32_t ph = 0; ph < 9; ph++) {
      int64_t mv = 0, mg = 0;
      orc_phase(st, ph, &mv, &mg);
      changes += mv + mg;
    }
    st->cnt[st->cur][C_SWEEPS]++;
    if (changes == 0) {
      if (!st->pruned) break;
      st->pruned = 0; /* the fallback: full sweeps from here on */
    }
  }
  return 0;
}

/* Keep mask of stage i (nbx * nby bytes of that stage's block grid, row-major; nonzero =
 * kept), or NULL to sweep the stage in full.  The schedule of the pruned sweeps is the
 * sweep schedule (schedule 0). */
int32_t orc_set_keep_mask(orc_state *st, int32_t i, const uint8_t *mask, int64_t n) {
  if (i < 0 || i >= st->nstages) return 1;
  free(st->keep[i]);
  st->keep[i] = NULL;
  if (!mask) return 0;
  if (st->p.schedule != 0) return 1;
  int64_t nb = (int64_t)ceil_div(st->W, st->st_side[i]) * ceil_div(st->H, st->st_side[i]);
  if (n != nb) return 1;
  st->keep[i] = (uint8_t *)malloc((size_t)nb);
  if (!st->keep[i]) return 2;
  memcpy(st->keep[i], mask, (size_t)nb);
  if (st->cur == i) st->pruned = 1;
  return 0;
}

/* Superpixel features at the prediction point (the F in R^4 of Sec. 4.1: absolute and
 * comparative brightness, extra- and intra-region dissimilarity), over the current block
 * grid.  With b_k = (R_k + G_k + B_k) / (3 N_k) and c_k = (R_k, G_k, B_k) / N_k:
 *   f1 = b_k;
 *   f2 = b_k - the mean of b_j over the 4-adjacent block pairs (p, q), p in k, q in j != k,
 *        each b_j taken as floor(2^16 b_j) / 2^16 (an exact integer quotient);
 *   f3 = the mean over the same pairs of |c_k - c_j|, each truncated to a multiple of 2^-16;
 *   f4 = sqrt(sum over k's blocks p of w_p |c_p - c_k|^2, each term truncated to a multiple
 *        of 2^-16, divided by N_k), c_p the block's mean colour.
 * Pairs and blocks are summed as integers, so the summation order does not matter; a
 * label without neighbours has f2 = f3 = 0. */
static void features(orc_state *st) {
  int32_t M = st->M;
  double *cr = (double *)calloc((size_t)M, 8), *cg = (double *)calloc((size_t)M, 8);
  double *cb = (double *)calloc((size_t)M, 8);
  int64_t *sb = (int64_t *)calloc((size_t)M, 8), *sd = (int64_t *)calloc((size_t)M, 8);
  int64_t *si = (int64_t *)calloc((size_t)M, 8), *np = (int64_t *)calloc((size_t)M, 8);
  for (int32_t k = 0; k < M; k++)
    if (st->N[k] > 0) {
      double n = (double)st->N[k];
      cr[k] = (double)st->R[k] / n; cg[k] = (double)st->G[k] / n; cb[k] = (double)st->B[k] / n;
    }
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++) {
      int32_t a = label_at(st, bx, by);
      int64_t s6[6];
      block_sums(st, bx, by, s6);
      double w = (double)s6[0];
      double dr = (double)s6[1] / w - cr[a], dg = (double)s6[2] / w - cg[a], db = (double)s6[3] / w - cb[a];
      double v = w * (dr * dr + dg * dg + db * db);
      si[a] += (int64_t)(v * 65536.0);
      int32_t nb[2] = {label_at(st, bx + 1, by), label_at(st, bx, by + 1)};
      for (int j = 0; j < 2; j++) {
        int32_t b = nb[j];
        if (b < 0 || b == a) continue;
        sb[a] += ((st->R[b] + st->G[b] + st->B[b]) << 16) / (3 * st->N[b]);
        sb[b] += ((st->R[a] + st->G[a] + st->B[a]) << 16) / (3 * st->N[a]);
        np[a]++;
        np[b]++;
        double er = cr[a] - cr[b], eg = cg[a] - cg[b], eb = cb[a] - cb[b];
        int64_t dq = (int64_t)(sqrt(er * er + eg * eg + eb * eb) * 65536.0);
        sd[a] += dq;
        sd[b] += dq;
      }
    }
  for (int32_t k = 0; k < M; k++) {
    double *f = st->feat + 4 * (int64_t)k;
    f[0] = f[1] = f[2] = f[3] = 0.0;
    if (st->N[k] == 0) continue;
    f[0] = (double)(st->R[k] + st->G[k] + st->B[k]) / (double)(3 * st->N[k]);
    if (np[k] > 0) {
      f[1] = f[0] - ((double)sb[k] / (double)np[k]) / 65536.0;
      f[2] = ((double)sd[k] / (double)np[k]) / 65536.0;
    }
    f[3] = sqrt(((double)si[k] / 65536.0) / (double)st->N[k]);
  }
  free(cr); free(cg); free(cb); free(sb); free(sd); free(si); free(np);
}

/* Prediction at the start of level 2 (Algorithm RAPID; Eq. predict): y_k = 1 when
 * h(k) >= 0, else -1.  h is the linear classifier theta_0 + theta . F(k) when one is set
 * (orc_set_classifier), else the integer stand-in h(k) = 3 T N_k - (R_k + G_k + B_k)
 * (ROI = dark superpixels).  Boundary superpixels (Eq. new_bound; "blocks located in
 * boundary superpixel"): labels 4-adjacent to a label of the other class. */
static void predict(orc_state *st) {
  features(st);
  for (int32_t k = 0; k < st->M; k++) {
    int32_t pos;
    if (st->use_theta) {
      const double *f = st->feat + 4 * (int64_t)k, *t = st->theta;
      double h = (((t[0] + t[1] * f[0]) + t[2] * f[1]) + t[3] * f[2]) + t[4] * f[3];
      pos = h >= 0.0;
    } else {
      int64_t h = 3 * st->p.h_T * st->N[k] - (st->R[k] + st->G[k] + st->B[k]);
      pos = h >= 0;
    }
    st->y[k] = (int8_t)(pos ? 1 : -1);
    st->imp[k] = 0;
  }
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++) {
      int32_t a = label_at(st, bx, by);
      int32_t e = label_at(st, bx + 1, by), s = label_at(st, bx, by + 1);
      if (e >= 0 && e != a && st->y[e] != st->y[a]) st->imp[a] = st->imp[e] = 1;
      if (s >= 0 && s != a && st->y[s] != st->y[a]) st->imp[a] = st->imp[s] = 1;
    }
  st->imp_on = 1;
}

int32_t orc_set_classifier(orc_state *st, const double *theta5) {
  st->use_theta = theta5 != NULL;
  for (int i = 0; i < 5; i++) st->theta[i] = theta5 ? theta5[i] : 0.0;
  return 0;
}

int32_t orc_read_features(const orc_state *st, double *dst4) {
  if (st->cur < 0) return 4;
  memcpy(dst4, st->feat, sizeof(double) * 4 * (size_t)st->M);
  return 0;
}

/* Next stage: prediction on entering level 2, then each block splits into 2x2 blocks
 * that keep its label ("map superpixels' labels", Algorithm RAPID).  With reuse off the
 * statistics are recomputed from the new level (the multi-scale baseline, Sec. 2.2). */
int32_t orc_next_stage(orc_state *st) {
  if (st->cur < 0 || st->cur + 1 >= st->nstages) return 4;
  int32_t prev_level = st->level, onbx = st->nbx;
  int32_t nxt = st->cur + 1;
  if (st->p.predict && st->st_level[nxt] >= 2 && prev_level < 2) predict(st);
  int32_t *old = (int32_t *)malloc(sizeof(int32_t) * (size_t)st->nbx * st->nby);
  if (!old) return 2;
  memcpy(old, st->lab, sizeof(int32_t) * (size_t)st->nbx * st->nby);
  int32_t ratio = st->side / st->st_side[nxt];
  set_stage_grid(st, nxt);
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++)
      st->lab[(int64_t)by * st->nbx + bx] = old[(int64_t)(by / ratio) * onbx + bx / ratio];
  free(old);
  if (!st->p.reuse && st->level != prev_level) recompute_stats(st);
  return 0;
}

int32_t orc_run(orc_state *st) {
  int32_t r = orc_seed(st);
  if (r) return r;
  orc_refine_stage(st);
  while (st->cur + 1 < st->nstages) {
    r = orc_next_stage(st);
    if (r) return r;
    orc_refine_stage(st);
  }
  return 0;
}

/* ---------------------------------------------------------------- sequential FIFO variant */
/* The paper's own order (Sec. 2.1, Algorithm RAPID): boundary blocks are queued, popped
 * one at a time, and the statistics are updated after every move; the 4-neighbours of a
 * moved block are pushed (N, W, E, S) when not already queued.  Used only to compare
 * quality with the phased schedule. */
static void fifo_stage(orc_state *st) {
  st->pruned = 0; /* keep masks belong to the phased sweeps only */
  int64_t nb = (int64_t)st->nbx * st->nby;
  int64_t cap = nb + 1;
  int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  uint8_t *inq = (uint8_t *)calloc((size_t)nb, 1);
  int64_t head = 0, tail = 0, count = 0, pops = 0, limit = (int64_t)st->p.max_sweeps * nb;
  int64_t *c = st->cnt[st->cur];
  for (int32_t by = 0; by < st->nby; by++)
    for (int32_t bx = 0; bx < st->nbx; bx++)
      if (eligible(st, bx, by, label_at(st, bx, by))) {
        int64_t i = (int64_t)by * st->nbx + bx;
        q[tail] = i; tail = (tail + 1) % cap; count++; inq[i] = 1;
      }
  int32_t M = st->M;
  double *mr = (double *)malloc(sizeof(double) * M), *mg = (double *)malloc(sizeof(double) * M);
  double *mb = (double *)malloc(sizeof(double) * M), *mx = (double *)malloc(sizeof(double) * M);
  double *my = (double *)malloc(sizeof(double) * M);
  while (count > 0 && pops < limit) {
    int64_t i = q[head]; head = (head + 1) % cap; count--; inq[i] = 0; pops++;
    int32_t bx = (int32_t)(i % st->nbx), by = (int32_t)(i / st->nbx);
    int32_t a = st->lab[i];
    /* live means of the labels involved */
    int32_t nbl[5] = {a, label_at(st, bx, by - 1), label_at(st, bx - 1, by), label_at(st, bx + 1, by),
                      label_at(st, bx, by + 1)};
    for (int j = 0; j < 5; j++) {
      int32_t k = nbl[j];
      if (k < 0 || st->N[k] == 0) continue;
      double n = (double)st->N[k];
      mr[k] = (double)st->R[k] / n; mg[k] = (double)st->G[k] / n; mb[k] = (double)st->B[k] / n;
      mx[k] = (double)st->X[k] / n; my[k] = (double)st->Y[k] / n;
    }
    int32_t k = -1;
    int r = decide(st, bx, by, mr, mg, mb, mx, my, st->N, &k, &c[C_ELIG], &c[C_EVAL]);
    if (r == 0) continue;
    if (r == 2) {
      c[C_REQ]++;
      int32_t n = merge_target(st, a, i);
      if (n < 0) continue;
      for (int64_t j = 0; j < nb; j++)
        if (st->lab[j] == a) st->lab[j] = n;
      st->N[n] += st->N[a]; st->R[n] += st->R[a]; st->G[n] += st->G[a]; st->B[n] += st->B[a];
      st->X[n] += st->X[a]; st->Y[n] += st->Y[a];
      st->N[a] = st->R[a] = st->G[a] = st->B[a] = st->X[a] = st->Y[a] = 0;
      c[C_MERGES]++;
    } else {
      apply_move(st, i, a, k);
      c[C_MOVES]++;
    }
    const int dx[4] = {0, -1, 1, 0}, dy[4] = {-1, 0, 0, 1};
    for (int j = 0; j < 4; j++) {
      int32_t nx = bx + dx[j], ny = by + dy[j];
      if (nx < 0 || ny < 0 || nx >= st->nbx || ny >= st->nby) continue;
      int64_t ni = (int64_t)ny * st->nbx + nx;
      if (inq[ni]) continue;
      q[tail] = ni; tail = (tail + 1) % cap; count++; inq[ni] = 1;
    }
  }
  c[C_SWEEPS] = pops;
  free(q); free(inq); free(mr); free(mg); free(mb); free(mx); free(my);
}

int32_t orc_run_fifo(orc_state *st) {
  int32_t r = orc_seed(st);
  if (r) return r;
  fifo_stage(st);
  while (st->cur + 1 < st->nstages) {
    r = orc_next_stage(st);
    if (r) return r;
    fifo_stage(st);
  }
  return 0;
}

/* ---------------------------------------------------------------- readers */
int32_t orc_get_grid(const orc_state *st, int32_t *stage, int32_t *nbx, int32_t *nby, int32_t *side,
                     int32_t *level, int32_t *M) {
  *stage = st->cur; *nbx = st->nbx; *nby = st->nby; *side = st->side; *level = st->level; *M = st->M;
  return 0;
}

int32_t orc_read_block_labels(const orc_state *st, int32_t *dst) {
  if (st->cur < 0) return 4;
  memcpy(dst, st->lab, sizeof(int32_t) * (size_t)st->nbx * st->nby);
  return 0;
}

int32_t orc_read_labels(const orc_state *st, int32_t *dst) {
  if (st->cur < 0) return 4;
  for (int32_t y = 0; y < st->H; y++)
    for (int32_t x = 0; x < st->W; x++)
      dst[(int64_t)y * st->W + x] = st->lab[(int64_t)(y / st->side) * st->nbx + x / st->side];
  return 0;
}

int32_t orc_read_stats(const orc_state *st, int64_t *dst7, int8_t *y, uint8_t *important) {
  if (st->cur < 0) return 4;
  for (int32_t k = 0; k < st->M; k++) {
    int64_t *d = dst7 + 7 * (int64_t)k;
    d[0] = st->N[k]; d[1] = st->R[k]; d[2] = st->G[k]; d[3] = st->B[k]; d[4] = st->X[k]; d[5] = st->Y[k];
    d[6] = st->init[k];
    if (y) y[k] = st->y[k];
    if (important) important[k] = st->imp[k];
  }
  return 0;
}

int32_t orc_read_counters(const orc_state *st, int64_t *dst) {
  memcpy(dst, st->cnt, sizeof(int64_t) * ORC_NCOUNT * (size_t)st->nstages);
  return 0;
}

int32_t orc_level_dims(const orc_state *st, int32_t level, int32_t *Wl, int32_t *Hl, int32_t *f) {
  if (level < 1 || level > st->L) return 1;
  *Wl = st->Wl[level]; *Hl = st->Hl[level]; *f = st->f[level];
  return 0;
}

int32_t orc_read_pyramid(const orc_state *st, int32_t level, int64_t *dst6) {
  if (level < 1 || level > st->L) return 1;
  for (int32_t Y = 0; Y < st->Hl[level]; Y++)
    for (int32_t X = 0; X < st->Wl[level]; X++) cell_sums(st, level, X, Y, dst6 + 6 * ((int64_t)Y * st->Wl[level] + X));
  return 0;
}
