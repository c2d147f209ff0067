// rapid_dev.cuh — device-side data layout and helpers shared by the kernels of the
// coarse-to-fine topology-preserving superpixel refinement (RAPID, ICME 2017).
//
// Layout in HBM (all row-major):
//   image   H x W interleaved RGB bytes, rows img_pitch bytes apart
//   level   for each image level with factor f > 1: ceil(H/f) x ceil(W/f) int4 = exact
//           (R, G, B, 0) sums of the f x f full-res footprint (Sec. 2.2, box "resize")
//   labels  two int32 maps sized for the finest stage; the current stage uses nby x nbx
//   S       structure of arrays over label ids: count, R, G, B, x, y, InitSize (int64),
//           the phase-start snapshot of the count, snapshot means (5 doubles) and their
//           single-precision hi/lo splits, last-change stamps, class y (int8),
//           boundary-superpixel flag (uint8), conservative bounding box (int4)
//   bitmaps sweep schedule: per phase class, one bit per block that may be eligible, and
//           one per block that requested a merge at its last evaluation
//   queue   queue schedule: per (tile, phase class) queue bits, and per-class worklists
// Position sums of a block are not stored: a block is an axis-aligned rectangle of
// full-res pixels, so its count and x/y sums follow from its corners.
//
// A context refines a batch of images together (a single image is a batch of one): every
// image keeps its own block grid, label map and sum levels, its labels are a contiguous
// range of one global id space (so S and the merge state are shared arrays), and its
// tiles are a contiguous range of one global tile index space.  Images never share a
// label, so each evolves exactly as it would alone.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rapid {

enum { CNT_LEVEL = 0, CNT_SIDE, CNT_SWEEPS, CNT_ELIG, CNT_EVAL, CNT_MOVES, CNT_REQ, CNT_MERGES,
       CNT_FALLBACK, CNT_MISMATCH, CNT_SCANNED, CNT_SKIPPED, CNT_SEARCHES, CNT_CACHE_HITS, CNT_N };

// Sections timed by the first CTA when profiling is on.
enum { PROF_EVAL = 0, PROF_SYNC1, PROF_COMMIT, PROF_SYNC2, PROF_MERGE, PROF_N };

// Device error word values (0 = fine).
enum { DERR_TIMEOUT = 1 };

// Evaluation tiles of the queue schedule's dense phases: one warp takes a tile of w x h
// blocks.  The stage kernel is compiled for each shape below, with `threads` per CTA: 1024
// threads hold 64 registers each (some spill), 512 hold 128 (none spill, half the warps
// per SM).  A launch uses one shape; the result never depends on it.  (The sweep schedule
// uses only the thread count.)
struct TileShape {
  int w, h, threads;
};
constexpr int kNumShapes = 6;
constexpr TileShape kShapes[kNumShapes] = {{32, 16, 1024}, {32, 8, 1024}, {64, 16, 1024},
                                           {32, 16, 512},  {32, 8, 512},  {64, 16, 512}};
constexpr int kCacheLabels = 16;           // neighbour labels remembered by a failed merge

struct DevStats {
  long long *N, *R, *G, *B, *X, *Y, *init;  // S; moves add into it during a phase
  long long *mN;                            // count N at the start of the phase (snapshot)
  double *mR, *mG, *mB, *mX, *mY;
  float4 *fhi, *flo;  // single-precision (hi, lo) of cR, cG, cB, mX
  float2 *fy;         // (hi, lo) of mY
  int *chg;           // stamp of the last change of S_k in this stage (2g: moves of phase g,
                      // 2g + 1: merges of phase g; 0 = before the stage)
  int *adj;           // stamp (2g) of the last move of a block of label k or 4-adjacent to one
  unsigned char *dirty;
  signed char *y;
  unsigned char *imp;
  int4 *bbox;  // inclusive full-res pixel box: x0, y0, x1, y1
  // prediction with a linear classifier: per-label integer sums over block pairs (brightness
  // in 2^-16 units, colour distance in 2^-16 units, pair count) and over blocks (squared
  // colour deviation in 2^-16 units), and the 4 features of the last prediction
  long long *fsb, *fsd, *fsi;
  int *fnp;
  double *feat;  // [M * 4]
  int M;
};

struct DevMerge {
  int *req_count;   // [2] requests (distinct labels) of the phase, slot = phase parity
  int *found_count; // [2] requests whose target search found a target, slot = phase parity
  int *found;       // [M] those requested labels

  int *req_list;    // [M] requested label ids
  // [M] smallest request key per label: (0xFFFFFFFF - phase) << 32 | global block index, so
  // that a later phase's key always wins the atomicMin and nothing has to be cleared
  unsigned long long *req_min;
  int *req_flag;    // [M] phase number in which the label was last put in req_list (0 = never)
  int *target;      // [M] chosen merge target (or -1)
  int *order;       // [M] scratch: requests sorted by req_min
  int2 *acc;        // [M] accepted (source, target) pairs of the phase
  int *acc_count;
  unsigned char *involved;  // [M]
  int *cache_stamp; // [M] stamp of the last target search that found no target (0 = none)
  int *cache_n;     // [M] number of neighbour labels it saw (-1 = too many to remember)
  int *cache_nb;    // [M * kCacheLabels] those neighbour labels
};

__device__ __forceinline__ unsigned long long req_key(int g, long long blk) {
  return ((unsigned long long)(0xFFFFFFFFu - (unsigned)g) << 32) | (unsigned long long)(unsigned)blk;
}
// the requesting block of a key of the current phase
__device__ __forceinline__ int req_block(unsigned long long key) { return (int)(unsigned)(key & 0xFFFFFFFFull); }

// Images one context refines together (one launch per stage covers all of them).
constexpr int kMaxBatch = 64;
// 32-bit words of the frontier queue per (tile, phase class): enough for the largest tile
// shape's class lattice (22 x 6 blocks of a 64 x 16 tile)
constexpr int kQueueWords = 5;

struct DevCtl {
  unsigned int *bar;             // grid-barrier arrivals (monotone within a launch; own line)
  int *err;                      // first device error (0 = none)
  long long spin_ns;             // give-up time of one barrier wait
  unsigned long long *changes;   // [nimg][3] moves + merges of the sweep per image, rotating slots
  int *last_merge;               // [nimg] stamp (2g + 1) of the image's last accepted merge
  long long *cnt;                // image 0's counters of this stage [CNT_N]; image i at + i * cnt_stride
  long long *prof;               // this stage's section times [PROF_N] in ns, or null
};

// Control block of a context: error word (8), merge counts (16..36), barrier counter (128,
// a line of its own: every CTA polls it), per-image merge stamps and sweep changes,
// per-(image, stage) counters, per-stage section times.  Every launch clears [16,
// reset_end), which holds the barrier counter; the error word persists.
struct CtlLayout {
  size_t bar, last_merge, changes, cnt, prof, reset_end, total;
};
inline CtlLayout ctl_layout(int nimg) {
  CtlLayout c;
  c.bar = 128;
  c.last_merge = 256;
  c.changes = (c.last_merge + 4 * (size_t)nimg + 7) / 8 * 8;
  c.reset_end = c.changes + 24 * (size_t)nimg;
  c.cnt = (c.reset_end + 255) / 256 * 256;
  c.prof = c.cnt + sizeof(long long) * CNT_N * 32 * (size_t)nimg;
  c.total = c.prof + sizeof(long long) * PROF_N * 32;
  return c;
}
constexpr int kCntStride = CNT_N * 32;  // counters of one image: 32 stages x CNT_N

// One image of a stage launch.
struct ImageDesc {
  int H, W;           // full-res image
  int nbx, nby;       // block grid ceil(W/s) x ceil(H/s)
  int ntx, nty;       // tile grid
  int Wl, Hl;         // dims of the sum level the stage reads
  int tile0;          // first global tile index
  int label0, M;      // global label ids label0 .. label0 + M - 1
  int blk0;           // first global block index (orders merge requests)
  int use_filter;     // 1: single-precision decisions with certified bounds, binary64 when undecided
  int pad;
  const unsigned char *img;
  long long img_pitch;
  const int4 *pyr;    // sum level (f > 1), else unused
  int *lab;           // nby x nbx labels (global ids)
  const unsigned char *mask;  // nby x nbx: 1 = the scorer keeps the block (pruned launches only)
  double lam_pos;
  float lam_pos_f;
  float pad2;
  int cw0[9];         // sweep schedule: first word of this image's bitmap of each phase class
  int pad3;
};

struct StageArgs {
  int side;           // block side s (full-res px)
  int level, f, k;    // level, the sum level's factor, its cells per block side (s / f)
  const ImageDesc *imgs;  // [nimg] in device memory
  ImageDesc img0;         // imgs[0] (a launch over one image reads it from here)
  int nimg;
  int ntiles;         // tiles of all images
  DevStats st;
  DevMerge mg;
  DevCtl ctl;
  int imp_on, imp_rule;
  double lam_b2;
  float lam_b2_f;
  int verify_filter;  // 1: also decide every block in binary64 and count disagreements
  int skip_tiles;     // 1: skip decisions whose inputs did not change since their last evaluation
  int size_mode, lo_num, lo_den, hi_num, hi_den;
  int max_sweeps;
  int prune;          // 1: sweep with the scorer's masks until a sweep changes nothing, then in full
  int frontier;       // 1: a phase visits only the queued blocks of its class (schedule 1)
  unsigned *qbits;    // frontier queue [ntiles * 9 * kQueueWords]: bit j of (tile, class) =
                      // the class's j-th block of the tile (row-major over the class lattice)
  int *wl;            // frontier worklists [9 * wl_cap]: global block indices queued since
                      // their class's last phase (each listed once)
  int *wl_count;      // [9] entries of each class's worklist
  int wl_cap;         // entries one class can hold (its blocks over all images)
  // sweep schedule: per phase class, one bit per block of the class lattice (class_words
  // below), class-major over the images: class c's words are [cwb[c], cwb[c + 1])
  int *wstamp;        // race check (null when off): per block of the stage, the phase that last wrote it
  unsigned long long *race;  // race check: violations found
  unsigned *cbits;    // 1 = the block may be eligible (a superset of the eligible blocks)
  unsigned *rbits;    // 1 = the block requested a merge at its last evaluation
  int cwb[10];
};

// Which schedule a stage-kernel instantiation runs: the sweeps only, the queue only, or the
// one a.frontier names (the build with both, whose register allocation measured faster
// for batches under the sweep schedule).
enum { kSchedSweeps = 0, kSchedQueue = 1, kSchedRuntime = 2 };
template <int kSched>
__device__ __forceinline__ bool queue_schedule(const StageArgs &a) {
  return kSched == kSchedQueue || (kSched == kSchedRuntime && a.frontier);
}


// Sweep-schedule bitmaps.  Phase class c = py * 3 + px holds the blocks (px + 3 i, py + 3 j)
// of a block grid nbx x nby, i < class_cols, j < class_rows; lattice row j is class_wpr
// 32-bit words, bit (i & 31) of word j * class_wpr + i / 32.  Bits past class_cols in a
// row's last word belong to no block.
__host__ __device__ inline int class_cols(int nbx, int px) { return nbx > px ? (nbx - px + 2) / 3 : 0; }
__host__ __device__ inline int class_rows(int nby, int py) { return nby > py ? (nby - py + 2) / 3 : 0; }
__host__ __device__ inline int class_wpr(int nbx, int px) { return (class_cols(nbx, px) + 31) >> 5; }
__host__ __device__ inline long long class_words(int nbx, int nby, int c) {
  return (long long)class_rows(nby, c / 3) * class_wpr(nbx, c % 3);
}

__host__ __device__ inline int popc32(unsigned v) {
#ifdef __CUDA_ARCH__
  return __popc(v);
#else
  int c = 0;
  for (; v; v &= v - 1u) c++;
  return c;
#endif
}

// Position of the k-th (0-based) set bit of m, which has more than k set bits: a binary
// search over the halves by their set-bit counts.
__host__ __device__ inline int select_bit(unsigned m, int k) {
  int pos = 0;
  for (int h = 16; h > 0; h >>= 1) {
    const int c = popc32(m & ((1u << h) - 1u));
    if (k >= c) {
      k -= c;
      m >>= h;
      pos += h;
    }
  }
  return pos;
}

// Box-sum levels kept for block sums: the method's level factors (> 1) plus 4, 16 and 64
// when a stage block is at least that large, so a block's colour sum never needs more than
// a few cells (the sums are exact integers whichever level supplies them).  Returns the
// count; out[] ascending.
constexpr int kMaxSumLevels = 12;
inline int sum_factors(const int *level_f, int L, int max_side, int *out) {
  int n = 0;
  auto add = [&](int v) {
    if (v <= 1 || v > max_side) return;
    for (int i = 0; i < n; i++)
      if (out[i] == v) return;
    if (n < kMaxSumLevels) out[n++] = v;
  };
  for (int l = 1; l <= L; l++) add(level_f[l]);
  add(4);
  add(16);
  add(64);
  for (int i = 1; i < n; i++)  // insertion sort, ascending
    for (int j = i; j > 0 && out[j - 1] > out[j]; j--) {
      const int t = out[j];
      out[j] = out[j - 1];
      out[j - 1] = t;
    }
  return n;
}

// Stage schedule handed to the counter initialiser (by value).
struct Schedule {
  int n;
  int level[32];
  int side[32];
};

#ifdef __CUDACC__

// ---------------------------------------------------------------- topology test
// Removing the centre from its label keeps the label 4-connected iff the label's ring
// cells that are 4-neighbours of the centre all lie in one 4-connected arc of the 3x3
// ring (E_topo of Eq. equa:energy1).  Ring order NW, N, NE, E, SE, S, SW, W: consecutive
// ring cells are 4-adjacent and no others are, so the ring's 4-components are the cyclic
// runs of set bits; a run without a 4-neighbour bit is an isolated corner.
__host__ __device__ inline int popc8(unsigned v) {
  v &= 0xFFu;
  v = v - ((v >> 1) & 0x55u);
  v = (v & 0x33u) + ((v >> 2) & 0x33u);
  return (int)((v + (v >> 4)) & 0x0Fu);
}

__host__ __device__ inline bool simple_mask(unsigned m) {
  m &= 0xFFu;
  if ((m & 0xAAu) == 0) return false;  // no 4-neighbour keeps the label
  if (m == 0xFFu) return true;
  unsigned prev = ((m << 1) | (m >> 7)) & 0xFFu;  // bit i holds ring bit i-1
  unsigned next = ((m >> 1) | (m << 7)) & 0xFFu;  // bit i holds ring bit i+1
  int runs = popc8(m & ~prev);
  int lone_corners = popc8(m & 0x55u & ~prev & ~next);
  return runs - lone_corners == 1;
}

// ---------------------------------------------------------------- race check
// A phase may write only labels of blocks of its class (by % 3, bx % 3), each once, and
// these are at least 3 apart (Chebyshev), so no two deciding blocks share a 3 x 3 window.
// With the check on, every label write of a phase (a move) stamps its block (global index
// idx) with the phase number g and counts a violation when the block is not of the class
// `phase`, was already stamped in this phase, or finds a block within distance 2 stamped in
// this phase (whichever of two conflicting writes comes second sees the first).
__device__ inline void race_check(unsigned long long *race, int *wstamp, long long blk0, int nbx, int nby, int bx,
                                  int by, int g, int phase) {
  if ((by % 3) * 3 + bx % 3 != phase) atomicAdd(race, 1ull);
  if (atomicExch(wstamp + blk0 + (long long)by * nbx + bx, g) == g) atomicAdd(race, 1ull);
  for (int dy = -2; dy <= 2; dy++)
    for (int dx = -2; dx <= 2; dx++) {
      const int x = bx + dx, y = by + dy;
      if ((dx == 0 && dy == 0) || x < 0 || y < 0 || x >= nbx || y >= nby) continue;
      if (atomicAdd(wstamp + blk0 + (long long)y * nbx + x, 0) == g) atomicAdd(race, 1ull);
    }
}

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// All CTAs of a co-resident (cooperative) grid meet here.  The arrival counter only grows
// during a launch: barrier number `epoch` (counted by every CTA) is complete when it reaches
// (epoch + 1) * gridDim.x.  Thread 0 arrives (after the CTA barrier) with a release add that
// does not wait for its result, then polls the counter with acquire loads: every arrival is
// a read-modify-write of the counter, so the final count lies in the release sequence of
// every CTA's arrival and the acquire that reads it synchronises with all of them.  (Polling
// the counter itself measured 1.30 us per barrier on 152 CTAs, against 1.85 us for an
// acquire-release add whose last arriver opens a separate flag.)  Every wait is bounded by
// ctl.spin_ns (and an iteration cap); on give-up the CTA records DERR_TIMEOUT and the whole
// grid returns false, so no kernel can hang.
//
// A kernel launched as one thread-block cluster (kCluster: the single-image kernels built
// for it) meets at the cluster's hardware
// barrier instead: every thread arrives with release and waits with acquire semantics at
// cluster scope, which orders the global-memory accesses of all the cluster's threads as
// the counter does for a grid.  The wait cannot time out and every CTA passes the same
// barriers (all control flow between barriers is uniform over the grid), so it returns true.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
template <bool kCluster = false>
__device__ inline bool grid_sync(const DevCtl &c, unsigned &epoch) {
  if constexpr (kCluster) {
    cluster_barrier();
    epoch++;
    return true;
  }
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int good = 1;
    const unsigned target = (epoch + 1) * gridDim.x;
    red_release_add_u32(&c.bar[0], 1u);
    if (ld_acquire_u32(c.bar) < target) {
      const unsigned long long t0 = global_ns();
      long long iters = 0;
      while (ld_acquire_u32(c.bar) < target) {
        if (ld_volatile_i32(c.err) != 0) {
          good = 0;
          break;
        }
        if ((long long)(global_ns() - t0) > c.spin_ns || ++iters > (1ll << 28)) {
          atomicCAS(c.err, 0, (int)DERR_TIMEOUT);
          good = 0;
          break;
        }
      }
    }
    ok = good;
  }
  __syncthreads();
  epoch++;
  return ok != 0;
}

// ---------------------------------------------------------------- block sums
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ unsigned ld_u8_hint(const unsigned char *p, unsigned long long pol) {
  unsigned v;
  asm volatile("ld.global.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

struct BlockSums {
  long long w, r, g, b, x, y;
  int bw, bh;
};

// Sums of block (bx, by) of image im at the current stage: colour from the sum level's
// cells (or the image at f = 1), count and position from the block rectangle
// [s bx, min(s bx + s, W)) x [s by, min(s by + s, H)).
__device__ inline BlockSums block_sums(const StageArgs &a, const ImageDesc &im, int bx, int by) {
  BlockSums o;
  int x0 = bx * a.side, y0 = by * a.side;
  int x1 = min(x0 + a.side, im.W), y1 = min(y0 + a.side, im.H);
  o.bw = x1 - x0;
  o.bh = y1 - y0;
  o.w = (long long)o.bw * o.bh;
  o.x = (long long)o.bh * (((long long)(x0 + x1 - 1) * o.bw) >> 1);
  o.y = (long long)o.bw * (((long long)(y0 + y1 - 1) * o.bh) >> 1);
  long long r = 0, g = 0, b = 0;
  if (a.f == 1) {
    // the image is read sparsely (boundary blocks only): mark its lines first to leave L2,
    // ahead of the label map and tile records that every phase re-reads
    const unsigned long long pol = l2_evict_first_policy();
    for (int yy = y0; yy < y1; yy++) {
      const unsigned char *row = im.img + (long long)yy * im.img_pitch + 3ll * x0;
      for (int xx = 0; xx < o.bw; xx++) {
        r += ld_u8_hint(row + 3 * xx, pol);
        g += ld_u8_hint(row + 3 * xx + 1, pol);
        b += ld_u8_hint(row + 3 * xx + 2, pol);
      }
    }
  } else {
    int X0 = bx * a.k, Y0 = by * a.k;
    int X1 = min(X0 + a.k, im.Wl), Y1 = min(Y0 + a.k, im.Hl);
    for (int Y = Y0; Y < Y1; Y++)
      for (int X = X0; X < X1; X++) {
        int4 c = im.pyr[(long long)Y * im.Wl + X];
        r += c.x;
        g += c.y;
        b += c.z;
      }
  }
  o.r = r;
  o.g = g;
  o.b = b;
  return o;
}

// ---------------------------------------------------------------- energies (binary64)
// Block energy under label means (c, mu), up to a label-independent constant
// (Eq. equa:energy1 summed over the block's pixels):
//   sum_ch [(w c) c - (2 S) c] + lambda_pos sum_d [(w mu) mu - (2 P) mu] + 2 lambda_b B
// evaluated with explicitly rounded operations in exactly this order (never fused).
__device__ __forceinline__ double blk_energy(double w, double r2, double g2, double b2, double x2,
                                             double y2, double cR, double cG, double cB, double mX,
                                             double mY, double Bk, double lam_pos, double lam_b2) {
  double eR = __dsub_rn(__dmul_rn(__dmul_rn(w, cR), cR), __dmul_rn(r2, cR));
  double eG = __dsub_rn(__dmul_rn(__dmul_rn(w, cG), cG), __dmul_rn(g2, cG));
  double eB = __dsub_rn(__dmul_rn(__dmul_rn(w, cB), cB), __dmul_rn(b2, cB));
  double ec = __dadd_rn(__dadd_rn(eR, eG), eB);
  double ex = __dsub_rn(__dmul_rn(__dmul_rn(w, mX), mX), __dmul_rn(x2, mX));
  double ey = __dsub_rn(__dmul_rn(__dmul_rn(w, mY), mY), __dmul_rn(y2, mY));
  double ep = __dadd_rn(ex, ey);
  return __dadd_rn(__dadd_rn(ec, __dmul_rn(lam_pos, ep)), __dmul_rn(lam_b2, Bk));
}

// Snapshot means of label k from its exact sums: c = S / N (IEEE division), plus their
// single-precision hi/lo splits (hi = nearest float, lo = nearest float of the rest).
__device__ __forceinline__ void split_f(double v, float &hi, float &lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(__dsub_rn(v, (double)hi));
}

__device__ __forceinline__ void set_means(const DevStats &s, int k) {
  long long n = s.N[k];
  s.mN[k] = n;
  double cr = 0.0, cg = 0.0, cb = 0.0, mx = 0.0, my = 0.0;
  if (n > 0) {
    double dn = __ll2double_rn(n);
    cr = __ddiv_rn(__ll2double_rn(s.R[k]), dn);
    cg = __ddiv_rn(__ll2double_rn(s.G[k]), dn);
    cb = __ddiv_rn(__ll2double_rn(s.B[k]), dn);
    mx = __ddiv_rn(__ll2double_rn(s.X[k]), dn);
    my = __ddiv_rn(__ll2double_rn(s.Y[k]), dn);
  }
  s.mR[k] = cr;
  s.mG[k] = cg;
  s.mB[k] = cb;
  s.mX[k] = mx;
  s.mY[k] = my;
  float4 hi, lo;
  float2 fy;
  split_f(cr, hi.x, lo.x);
  split_f(cg, hi.y, lo.y);
  split_f(cb, hi.z, lo.z);
  split_f(mx, hi.w, lo.w);
  split_f(my, fy.x, fy.y);
  s.fhi[k] = hi;
  s.flo[k] = lo;
  s.fy[k] = fy;
}

// Merge cost of labels a and n (Sec. 3.1): the Ward increase of the colour and position
// energy, Na Nn / (Na + Nn) * (|ca - cn|^2 + lambda_pos |mua - mun|^2).
// The means are taken from S itself (the state after the phase's moves), with the same
// operations as set_means, so they equal the snapshot means the next phase will use.
__device__ __forceinline__ double mean_of(const long long *sum, const long long *cnt, int k) {
  return __ddiv_rn(__ll2double_rn(sum[k]), __ll2double_rn(cnt[k]));
}
// am: a's means (R, G, B, X, Y) as mean_of gives them.
__device__ __forceinline__ double ward_cost(const DevStats &s, int a, const double *am, int n, double lam_pos) {
  double t = __ddiv_rn(__dmul_rn(__ll2double_rn(s.N[a]), __ll2double_rn(s.N[n])),
                       __ll2double_rn(s.N[a] + s.N[n]));
  double d0 = __dsub_rn(am[0], mean_of(s.R, s.N, n));
  double d1 = __dsub_rn(am[1], mean_of(s.G, s.N, n));
  double d2 = __dsub_rn(am[2], mean_of(s.B, s.N, n));
  double dc = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  double e0 = __dsub_rn(am[3], mean_of(s.X, s.N, n));
  double e1 = __dsub_rn(am[4], mean_of(s.Y, s.N, n));
  double dm = __dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1));
  return __dmul_rn(t, __dadd_rn(dc, __dmul_rn(lam_pos, dm)));
}

__device__ __forceinline__ void atomic_add_i64(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

#endif  // __CUDACC__

// Learned block scorer (k_scorer.cu): device weights and the training-sample store.
struct ScorerDev {
  const void *w1, *w2;  // bf16 [tap][co][ci] (ci padded to 16)
  const float *w3, *b1, *b2;
  float b3;
};
struct TrainSet {
  float *x;                 // [cap][7 * 7 * 9] feature patches
  unsigned long long *inb;  // [cap] bit p: patch position p lies inside the image
  float *y;                 // [cap] 1 = the block moved in its stage
  int *count;               // samples appended (may exceed cap: the extra ones are dropped)
  long long cap;
};
constexpr int kScorerPatchFloats = 7 * 7 * 9;
cudaError_t scorer_upload(const float *weights, void *buf, ScorerDev *out, cudaStream_t s);
size_t scorer_dev_bytes();
cudaError_t launch_features(const StageArgs &a, const ImageDesc &im, int L, float *out, cudaStream_t s);
cudaError_t launch_score(const StageArgs &a, const ImageDesc &im, int L, const ScorerDev &W, float threshold,
                         float *score, unsigned char *mask, cudaStream_t s);
// Training samples of one logged stage of one image, appended in block order (scratch:
// collect_scratch_ints(nbx * nby) ints of device memory).
size_t collect_scratch_ints(long long blocks);
cudaError_t launch_collect(const float *feat, const int *before, const int *after, int nbx, int nby, int img,
                           int stage, float neg_rate, const TrainSet &ts, int *scratch, cudaStream_t s);
// One minibatch: samples order[(off + b) % n], b < batch; grad = the sum of their gradients
// at the master weights w (summed in a fixed order), *loss += the sum of their losses.
// part: train_max_ctas() * RAPID_SCORER_PARAMS floats, part_loss: train_max_ctas() floats.
int train_max_ctas();
cudaError_t launch_train_step(const TrainSet &ts, int n, const float *w, const int *order, int off, int batch,
                              float pos_weight, float *part, float *part_loss, float *grad, float *loss,
                              cudaStream_t s);
cudaError_t launch_adam(float *w, float *m, float *v, float *grad, float lr, float bc1, float bc2, float inv_batch,
                        cudaStream_t s);

// Host-side launchers (defined in the .cu files).
cudaError_t launch_stage(const StageArgs &a, int grid, int block, cudaStream_t s, int shape);
// Largest grid that runs as one thread-block cluster (the non-portable cluster size limit).
constexpr int kMaxCluster = 16;
// Whether stage kernel fn (block threads per CTA) can run as one cluster of `grid` CTAs on
// the current device: decided once per kernel and device (cluster sizes 16 and 8 are
// queried) and remembered; while the stream is being captured an unknown kernel counts as
// not (a cooperative launch is always correct).
bool cluster_launch_ok(const void *fn, int grid, int block, cudaStream_t s);
int stage_block_threads(int shape);
const void *stage_kernel_ptr(bool batch, bool frontier, int shape);
// the single-image kernel of a shape built for a launch as one thread-block cluster
const void *stage_cluster_kernel_ptr(bool frontier, int shape);

// Carve the per-label arrays of M labels from `base` (256-byte aligned pieces); returns the
// bytes used, or 0 when they do not fit in `cap` bytes.  label_arrays_bytes(M) is the size.
size_t carve_label_arrays(void *base, size_t cap, int M, DevStats *st, DevMerge *mg);
size_t label_arrays_bytes(int M);

}  // namespace rapid
