// k_synth.cu — the counter-based whole-slide generator on the device (input data only: it
// holds none of the refinement's arithmetic).  It makes the synthetic H&E-like slide that
// stands in for the paper's NLST whole-slide images at their full size (100000 x 80000 RGB,
// 24 GB), which the host generator would take most of an hour to make.
//
// Definition (restated pixel for pixel by paper_1704_02083_gb300.synth.slide_gen, which
// must give the same bytes): every random quantity is h(seed, stream, index) = mix(mix(
// mix(seed) ^ stream) ^ index), mix being the SplitMix64 output function, and every
// geometric test is exact integer arithmetic.
//   * Buckets of 128 x 128 px (clipped at the right and bottom edges).
//   * Voronoi cells: kc seeds per bucket (id = bucket * kc + j) at hashed positions inside
//     the bucket; a pixel takes the seed of least squared distance, ties to the smaller id
//     (every bucket holds a seed, so the nearest lies within two buckets).
//   * Cell class (white / purple / pink by thresholds on a hash mod 10000) and mean colour
//     (base + a hashed offset in [-15, 15], white [-5, 5]).
//   * Nuclei: kn per bucket, hashed centre, radius 3..8 and colour; kept when the centre's
//     cell is not white; the largest covering id wins.
//   * Folds: nf straight bands with hashed width, direction, centre, length and colour; a
//     pixel is inside when 4 (a.d)^2 <= length^2 |a|^2 and 4 (a x d)^2 <= width^2 |a|^2;
//     the largest band id wins over nuclei and cells.
//   * Noise: a discrete Gaussian (sigma 6) per channel by table inversion of the upper 32
//     bits of a per-(pixel, channel) hash; the sum is clamped to [0, 255].
//
// Layout: one CTA per bucket, kThreads threads.  The CTA first gathers, in shared memory,
// the seeds of the 7 x 7 buckets around it (every pixel's candidates, and those of the
// nucleus centres that can reach it), the nuclei of the 3 x 3 buckets around it (painting
// the kept ones into a per-pixel id map with atomicMax) and the folds whose bounding box
// meets the bucket; then each thread colours its pixels.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "../../include/rapid.h"

namespace {

constexpr int kB = 128;           // bucket side
constexpr int kThreads = 256;
constexpr int kMaxKc = 8;         // seeds per bucket
constexpr int kMaxKn = 64;        // nuclei per bucket
constexpr int kMaxFolds = 1024;   // bands per slide
constexpr int kSeedRing = 7;      // the 7 x 7 buckets whose seeds a CTA gathers

__constant__ unsigned c_noise_cdf[60];  // the discrete Gaussian's cumulative thresholds (x 2^32)

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Gen {
  uint64_t key[40];  // mix(mix(seed) ^ stream) for streams 0..39
  int64_t H, W;
  int nbx, nby, kc, kn, nf;
  int n_white, n_purple;
  int64_t n_cells, n_nuclei;
};

__device__ __forceinline__ uint64_t hh(const Gen &g, int stream, uint64_t idx) { return mix64(g.key[stream] ^ idx); }

struct Seed {
  int x, y;
  int64_t id;
};

struct Nucleus {
  int x, y, r2;
  int64_t id;
  int col[3];
};

struct Fold {
  int64_t cx, cy, ax, ay, n2w, n2l;  // centre, direction, width^2 |a|^2 and length^2 |a|^2
  int col[3];
  int id;
};

struct Smem {
  Seed seeds[kSeedRing * kSeedRing * kMaxKc];
  Nucleus nuc[9 * kMaxKn];
  Fold folds[kMaxFolds];
  int nfold;
  int nuc_map[kB * kB];  // per pixel of the bucket: index into nuc (max id), -1 none
};

// Nearest seed of pixel (x, y) among the gathered seeds of the 5 x 5 buckets around its
// bucket (pbx, pby); (gx0, gy0) is the first gathered bucket.
__device__ int64_t nearest_seed(const Gen &g, const Smem &S, int64_t x, int64_t y, int gx0, int gy0) {
  const int pbx = (int)(x / kB), pby = (int)(y / kB);
  int64_t best_d = INT64_MAX, best_id = -1;
  for (int dby = -2; dby <= 2; dby++)
    for (int dbx = -2; dbx <= 2; dbx++) {
      const int qbx = pbx + dbx, qby = pby + dby;
      if (qbx < 0 || qby < 0 || qbx >= g.nbx || qby >= g.nby) continue;
      const int lx = qbx - gx0, ly = qby - gy0;  // within the gathered 7 x 7 ring
      for (int j = 0; j < g.kc; j++) {
        const Seed &sd = S.seeds[(ly * kSeedRing + lx) * g.kc + j];
        const int64_t dx = sd.x - x, dy = sd.y - y;
        const int64_t d = dx * dx + dy * dy;
        if (d < best_d || (d == best_d && sd.id < best_id)) {
          best_d = d;
          best_id = sd.id;
        }
      }
    }
  return best_id;
}

// class (0 pink, 1 purple, 2 white) and mean colour of cell id
__device__ int cell_colour(const Gen &g, int64_t id, int col[3]) {
  const int u = (int)(hh(g, 3, (uint64_t)id) % 10000ull);
  const int cls = u < g.n_white ? 2 : (u < g.n_white + g.n_purple ? 1 : 0);
  const int base[3][3] = {{230, 150, 190}, {120, 70, 150}, {245, 245, 245}};
  for (int c = 0; c < 3; c++) {
    const uint64_t v = hh(g, 4 + c, (uint64_t)id);
    col[c] = base[cls][c] + (cls == 2 ? (int)(v % 11ull) - 5 : (int)(v % 31ull) - 15);
  }
  return cls;
}

__global__ void __launch_bounds__(kThreads) synth_slide_kernel(Gen g, uint8_t *rgb, int64_t pitch, int32_t *regions,
                                                                int64_t rpitch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &S = *reinterpret_cast<Smem *>(smem_raw);
  const int bx = blockIdx.x, by = blockIdx.y;
  const int gx0 = bx - kSeedRing / 2, gy0 = by - kSeedRing / 2;
  // 1. the seeds of the 7 x 7 buckets around (outside the grid: never read)
  for (int t = threadIdx.x; t < kSeedRing * kSeedRing * g.kc; t += blockDim.x) {
    const int j = t % g.kc, cell = t / g.kc, lx = cell % kSeedRing, ly = cell / kSeedRing;
    const int qbx = gx0 + lx, qby = gy0 + ly;
    Seed sd = {0, 0, -1};
    if (qbx >= 0 && qby >= 0 && qbx < g.nbx && qby < g.nby) {
      const int64_t q = (int64_t)qby * g.nbx + qbx;
      const int64_t id = q * g.kc + j;
      const int bw = (int)min((int64_t)kB, g.W - (int64_t)kB * qbx), bh = (int)min((int64_t)kB, g.H - (int64_t)kB * qby);
      sd.x = kB * qbx + (int)(hh(g, 1, (uint64_t)id) % (uint64_t)bw);
      sd.y = kB * qby + (int)(hh(g, 2, (uint64_t)id) % (uint64_t)bh);
      sd.id = id;
    }
    S.seeds[t] = sd;
  }
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) S.nuc_map[t] = -1;
  if (threadIdx.x == 0) S.nfold = 0;
  __syncthreads();
  // 2. the nuclei of the 3 x 3 buckets around, kept when their centre's cell is not white
  for (int t = threadIdx.x; t < 9 * g.kn; t += blockDim.x) {
    const int j = t % g.kn, cell = t / g.kn;
    const int qbx = bx - 1 + cell % 3, qby = by - 1 + cell / 3;
    Nucleus n;
    n.id = -1;
    if (qbx >= 0 && qby >= 0 && qbx < g.nbx && qby < g.nby) {
      const int64_t q = (int64_t)qby * g.nbx + qbx;
      const int64_t id = q * g.kn + j;
      const int bw = (int)min((int64_t)kB, g.W - (int64_t)kB * qbx), bh = (int)min((int64_t)kB, g.H - (int64_t)kB * qby);
      n.x = kB * qbx + (int)(hh(g, 10, (uint64_t)id) % (uint64_t)bw);
      n.y = kB * qby + (int)(hh(g, 11, (uint64_t)id) % (uint64_t)bh);
      const int r = 3 + (int)(hh(g, 12, (uint64_t)id) % 6ull);
      n.r2 = r * r;
      const int nucleus[3] = {60, 30, 90};
      for (int c = 0; c < 3; c++) n.col[c] = nucleus[c] + (int)(hh(g, 13 + c, (uint64_t)id) % 21ull) - 10;
      int cc[3];
      if (cell_colour(g, nearest_seed(g, S, n.x, n.y, gx0, gy0), cc) != 2) n.id = id;
    }
    S.nuc[t] = n;
  }
  // 3. the folds whose bounding box meets this bucket
  const int64_t X0 = (int64_t)kB * bx, Y0 = (int64_t)kB * by;
  const int64_t X1 = min(X0 + kB, g.W), Y1 = min(Y0 + kB, g.H);
  for (int b = threadIdx.x; b < g.nf; b += blockDim.x) {
    const int64_t fw = 20 + (int64_t)(hh(g, 30, (uint64_t)b) % 61ull);
    int64_t ax = (int64_t)(hh(g, 31, (uint64_t)b) % 2049ull) - 1024;
    int64_t ay = (int64_t)(hh(g, 32, (uint64_t)b) % 2049ull) - 1024;
    if (ax == 0 && ay == 0) ax = 1;
    const int64_t cx = (int64_t)(hh(g, 33, (uint64_t)b) % (uint64_t)g.W), cy = (int64_t)(hh(g, 34, (uint64_t)b) % (uint64_t)g.H);
    const int64_t len = min(g.H, g.W) * (300 + (int64_t)(hh(g, 35, (uint64_t)b) % 701ull)) / 1000;
    const int64_t ext = (len + fw) / 2 + 2;
    if (cx + ext < X0 || cx - ext >= X1 || cy + ext < Y0 || cy - ext >= Y1) continue;
    const int slot = atomicAdd(&S.nfold, 1);
    Fold &f = S.folds[slot];
    f.cx = cx;
    f.cy = cy;
    f.ax = ax;
    f.ay = ay;
    const int64_t n2 = ax * ax + ay * ay;
    f.n2w = fw * fw * n2;
    f.n2l = len * len * n2;
    const int fold[3] = {80, 40, 110};
    for (int c = 0; c < 3; c++) f.col[c] = fold[c] + (int)(hh(g, 36 + c, (uint64_t)b) % 21ull) - 10;
    f.id = b;
  }
  __syncthreads();
  // paint the kept nuclei's discs into the bucket's id map (largest id wins)
  for (int t = threadIdx.x; t < 9 * g.kn * 289; t += blockDim.x) {
    const int k = t / 289, o = t % 289;
    const Nucleus &n = S.nuc[k];
    if (n.id < 0) continue;
    const int x = n.x - 8 + o % 17, y = n.y - 8 + o / 17;
    if (x < X0 || x >= X1 || y < Y0 || y >= Y1) continue;
    const int dx = x - n.x, dy = y - n.y;
    if (dx * dx + dy * dy > n.r2) continue;
    const int cell = (y - (int)Y0) * kB + (x - (int)X0);
    // compare by nucleus id: the map holds indices into S.nuc, whose ids grow with the index
    atomicMax(&S.nuc_map[cell], k);
  }
  __syncthreads();
  // 4. every pixel of the bucket
  const int nfold = S.nfold;
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int64_t x = X0 + t % kB, y = Y0 + t / kB;
    if (x >= X1 || y >= Y1) continue;
    int col[3];
    int64_t region;
    // the largest fold id that covers the pixel
    int best_f = -1, fi = -1;
    for (int i = 0; i < nfold; i++) {
      const Fold &f = S.folds[i];
      if (f.id <= best_f) continue;
      const int64_t dx = x - f.cx, dy = y - f.cy;
      const int64_t along = f.ax * dx + f.ay * dy, across = f.ay * dx - f.ax * dy;
      if (4 * along * along <= f.n2l && 4 * across * across <= f.n2w) {
        best_f = f.id;
        fi = i;
      }
    }
    if (fi >= 0) {
      for (int c = 0; c < 3; c++) col[c] = S.folds[fi].col[c];
      region = g.n_cells + g.n_nuclei + best_f;
    } else {
      const int k = S.nuc_map[t];
      if (k >= 0) {
        for (int c = 0; c < 3; c++) col[c] = S.nuc[k].col[c];
        region = g.n_cells + S.nuc[k].id;
      } else {
        region = nearest_seed(g, S, x, y, gx0, gy0);
        cell_colour(g, region, col);
      }
    }
    uint8_t *px = rgb + y * pitch + 3 * x;
    const uint64_t pix = (uint64_t)(y * g.W + x) * 3ull;
    for (int c = 0; c < 3; c++) {
      const unsigned u = (unsigned)(hh(g, 20, pix + c) >> 32);
      int lo = 0, hi = 60;  // #{thresholds <= u}
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c_noise_cdf[mid] <= u) lo = mid + 1;
        else hi = mid;
      }
      const int v = col[c] + (lo - 30);
      px[c] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
    }
    if (regions) regions[y * rpitch + x] = (int32_t)region;
  }
}

const unsigned kNoiseCdf[60] = {
    1064u,       3479u,       8809u,       20251u,      44139u,      92645u,      188445u,     372463u,
    716254u,     1340945u,    2444952u,    4342595u,    7515037u,    12673366u,   20830933u,   33378184u,
    52148550u,   79459272u,   118107525u,  171301547u,  242510082u,  335222422u,  452625448u,  597221792u,
    770431245u,  972231699u,  1200901570u, 1452919839u, 1723061373u, 2004696593u, 2290270703u, 2571905923u,
    2842047457u, 3094065726u, 3322735597u, 3524536051u, 3697745504u, 3842341848u, 3959744874u, 4052457214u,
    4123665749u, 4176859771u, 4215508024u, 4242818746u, 4261589112u, 4274136363u, 4282293930u, 4287452259u,
    4290624701u, 4292522344u, 4293626351u, 4294251042u, 4294594833u, 4294778851u, 4294874651u, 4294923157u,
    4294947045u, 4294958487u, 4294963817u, 4294966232u};

}  // namespace

extern "C" rapid_status rapid_synth_slide(const rapid_synth_params *p, uint8_t *rgb_dev, int64_t rgb_pitch_bytes,
                                          int32_t *regions_dev, int64_t regions_pitch_bytes, void *cuda_stream) {
  if (!p || !rgb_dev || p->H < 1 || p->W < 1 || rgb_pitch_bytes < 3 * p->W) return RAPID_EINVAL;
  if (regions_dev && (regions_pitch_bytes < 4 * p->W || regions_pitch_bytes % 4)) return RAPID_EINVAL;
  if (p->px_per_cell < 1 || !(p->white_frac >= 0.0 && p->white_frac <= 1.0) ||
      !(p->fold_frac >= 0.0 && p->fold_frac <= 1.0) || !(p->nucleus_density >= 0.0 && p->nucleus_density <= 1.0))
    return RAPID_EINVAL;
  if (p->H > (1ll << 31) || p->W > (1ll << 31)) return RAPID_ERANGE;
  Gen g;
  for (int s = 0; s < 40; s++) g.key[s] = mix64(mix64(p->seed) ^ (uint64_t)s);
  g.H = p->H;
  g.W = p->W;
  g.nbx = (int)((p->W + kB - 1) / kB);
  g.nby = (int)((p->H + kB - 1) / kB);
  // the counts, rounded to nearest (ties to even) as the host generator rounds them
  const double kcd = std::nearbyint((double)(kB * kB) / (double)p->px_per_cell);
  g.kc = kcd < 1.0 ? 1 : (int)kcd;
  g.kn = (int)std::nearbyint((double)(kB * kB) * p->nucleus_density);
  const double nfd = std::nearbyint(p->fold_frac * (double)p->H * (double)p->W /
                                    (50.0 * 0.65 * (double)(p->H < p->W ? p->H : p->W)));
  g.nf = nfd < 1.0 ? 1 : (nfd > kMaxFolds ? kMaxFolds + 1 : (int)nfd);
  if (g.kc > kMaxKc || g.kn > kMaxKn || g.nf > kMaxFolds) return RAPID_ERANGE;
  g.n_white = (int)std::nearbyint(p->white_frac * 10000.0);
  g.n_purple = (int)std::nearbyint((1.0 - p->white_frac) * 0.4375 * 10000.0);
  g.n_cells = (int64_t)g.nbx * g.nby * g.kc;
  g.n_nuclei = (int64_t)g.nbx * g.nby * g.kn;
  if (g.n_cells + g.n_nuclei + g.nf > INT32_MAX) return RAPID_ERANGE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemcpyToSymbolAsync(c_noise_cdf, kNoiseCdf, sizeof kNoiseCdf, 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return RAPID_ECUDA;
  const size_t smem = sizeof(Smem);
  if (cudaFuncSetAttribute(synth_slide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RAPID_ECUDA;
  synth_slide_kernel<<<dim3(g.nbx, g.nby), kThreads, smem, s>>>(g, rgb_dev, rgb_pitch_bytes, regions_dev,
                                                                regions_pitch_bytes / 4);
  return cudaGetLastError() == cudaSuccess ? RAPID_OK : RAPID_ECUDA;
}
