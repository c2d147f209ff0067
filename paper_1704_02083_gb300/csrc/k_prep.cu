// k_prep.cu — the non-sweep kernels: level images (box sums), seeding, stage split,
// prediction, statistics recomputation and the readers.
#include <climits>

#include "../../include/rapid.h"
#include "rapid_dev.cuh"

namespace rapid {

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Level image of factor f (Sec. 2.2): coarse cell (X, Y) holds the exact R, G, B sums of
// full-res [fX, min(fX + f, W)) x [fY, min(fY + f, H)).
//
// The finest sum level is read from the image: a CTA takes f rows and kPyrCells cells of
// them (f * kPyrCells pixels per row), stages those rows in shared memory with 16-byte loads
// when the image rows allow it (16-byte aligned base and pitch), and each thread sums one
// cell from shared memory.  Every coarser level (its factor a multiple of the previous one's:
// all are powers of two) is summed from the previous level's cells, never from the image.
constexpr int kPyrCells = 256;
constexpr int kPyrMaxF = 16;  // finest factor staged in shared memory (larger: per-thread sums)

__global__ void __launch_bounds__(kPyrCells) pyramid_rows_kernel(const unsigned char *img, long long pitch, int H,
                                                                  int W, int f, int Wl, int4 *out, int vec) {
  extern __shared__ __align__(16) unsigned char rows[];  // f rows of 3 f kPyrCells bytes
  const int Y = blockIdx.y, X0 = blockIdx.x * kPyrCells;
  const int x0 = X0 * f, y0 = Y * f;
  const int nrow = min(f, H - y0);
  const int span = min(f * kPyrCells, W - x0);  // pixels of this CTA's rows
  const int bytes = 3 * span, stride = 3 * f * kPyrCells;
  if (vec) {  // 16-byte loads; the last chunk may read up to 15 bytes past the row, within its pitch
    const int chunks = (bytes + 15) / 16;
    for (int t = threadIdx.x; t < nrow * chunks; t += blockDim.x) {
      const int r = t / chunks, c = t % chunks;
      const uint4 v = *reinterpret_cast<const uint4 *>(img + (long long)(y0 + r) * pitch + 3ll * x0 + 16 * c);
      *reinterpret_cast<uint4 *>(rows + r * stride + 16 * c) = v;
    }
  } else {
    for (int t = threadIdx.x; t < nrow * bytes; t += blockDim.x) {
      const int r = t / bytes, c = t % bytes;
      rows[r * stride + c] = img[(long long)(y0 + r) * pitch + 3ll * x0 + c];
    }
  }
  __syncthreads();
  const int X = X0 + threadIdx.x;
  if (X >= Wl) return;
  const int cx0 = threadIdx.x * f, cw = min(f, span - cx0);
  int r = 0, g = 0, b = 0;
  for (int yy = 0; yy < nrow; yy++) {
    const unsigned char *row = rows + yy * stride + 3 * cx0;
    for (int x = 0; x < cw; x++) {
      r += row[3 * x];
      g += row[3 * x + 1];
      b += row[3 * x + 2];
    }
  }
  out[(long long)Y * Wl + X] = make_int4(r, g, b, 0);
}

// Per-thread sums straight from the image (factors too large to stage their rows).
__global__ void pyramid_kernel(const unsigned char *img, long long pitch, int H, int W, int f, int Wl, int Hl,
                               int4 *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Wl * Hl) return;
  const int X = (int)(i % Wl), Y = (int)(i / Wl);
  const int x0 = X * f, y0 = Y * f, x1 = min(x0 + f, W), y1 = min(y0 + f, H);
  int r = 0, g = 0, b = 0;
  for (int y = y0; y < y1; y++) {
    const unsigned char *row = img + (long long)y * pitch + 3ll * x0;
    for (int x = 0; x < x1 - x0; x++) {
      r += row[3 * x];
      g += row[3 * x + 1];
      b += row[3 * x + 2];
    }
  }
  out[i] = make_int4(r, g, b, 0);
}

// Coarser level: cell (X, Y) = the sum of the finer level's cells [mX, mX + m) x [mY, mY + m)
// (clipped to the finer level), m = the ratio of the two factors.
__global__ void pyramid_merge_kernel(const int4 *fine, int Wf, int Hf, int m, int Wl, int Hl, int4 *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Wl * Hl) return;
  const int X = (int)(i % Wl), Y = (int)(i / Wl);
  const int x1 = min(X * m + m, Wf), y1 = min(Y * m + m, Hf);
  int r = 0, g = 0, b = 0;
  for (int y = Y * m; y < y1; y++)
    for (int x = X * m; x < x1; x++) {
      const int4 c = fine[(long long)y * Wf + x];
      r += c.x;
      g += c.y;
      b += c.z;
    }
  out[i] = make_int4(r, g, b, 0);
}

cudaError_t launch_pyramid(const unsigned char *img, long long pitch, int H, int W, int f, int Wl, int Hl,
                           int4 *out, cudaStream_t s) {
  if (f > kPyrMaxF || Hl > 65535) {
    const long long n = (long long)Wl * Hl;
    pyramid_kernel<<<blocks_for(n, 256), 256, 0, s>>>(img, pitch, H, W, f, Wl, Hl, out);
    return cudaGetLastError();
  }
  const int vec = ((uintptr_t)img % 16 == 0 && pitch % 16 == 0) ? 1 : 0;
  const size_t smem = (size_t)f * 3 * f * kPyrCells + 16;
  if (smem > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(pyramid_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  pyramid_rows_kernel<<<dim3((Wl + kPyrCells - 1) / kPyrCells, Hl), kPyrCells, smem, s>>>(img, pitch, H, W, f, Wl,
                                                                                         out, vec);
  return cudaGetLastError();
}

cudaError_t launch_pyramid_merge(const int4 *fine, int Wf, int Hf, int m, int Wl, int Hl, int4 *out, cudaStream_t s) {
  const long long n = (long long)Wl * Hl;
  pyramid_merge_kernel<<<blocks_for(n, 256), 256, 0, s>>>(fine, Wf, Hf, m, Wl, Hl, out);
  return cudaGetLastError();
}

// Regular seed grid (Algorithm RAPID): block (bx, by) of the first stage gets label
// floor(by gy / nby) gx + floor(bx gx / nbx); its sums go to S and its rectangle to the
// label's bounding box.
__global__ void seed_kernel(StageArgs a, ImageDesc im, int gx, int gy) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)im.nbx * im.nby) return;
  const int bx = (int)(i % im.nbx), by = (int)(i / im.nbx);
  const int lbl = im.label0 + (int)(((long long)by * gy / im.nby) * gx + ((long long)bx * gx / im.nbx));
  im.lab[i] = lbl;
  const BlockSums bs = block_sums(a, im, bx, by);
  atomic_add_i64(&a.st.N[lbl], bs.w);
  atomic_add_i64(&a.st.R[lbl], bs.r);
  atomic_add_i64(&a.st.G[lbl], bs.g);
  atomic_add_i64(&a.st.B[lbl], bs.b);
  atomic_add_i64(&a.st.X[lbl], bs.x);
  atomic_add_i64(&a.st.Y[lbl], bs.y);
  const int x0 = bx * a.side, y0 = by * a.side;
  atomicMin(&a.st.bbox[lbl].x, x0);
  atomicMin(&a.st.bbox[lbl].y, y0);
  atomicMax(&a.st.bbox[lbl].z, x0 + bs.bw - 1);
  atomicMax(&a.st.bbox[lbl].w, y0 + bs.bh - 1);
}

__global__ void reset_labels_kernel(DevStats st, DevMerge mg) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= st.M) return;
  st.N[k] = st.R[k] = st.G[k] = st.B[k] = st.X[k] = st.Y[k] = st.init[k] = 0;
  st.mN[k] = 0;
  st.dirty[k] = 0;
  st.y[k] = 0;
  st.imp[k] = 0;
  st.bbox[k] = make_int4(INT_MAX, INT_MAX, INT_MIN, INT_MIN);
  mg.req_min[k] = ~0ull;
  mg.req_flag[k] = 0;
  mg.target[k] = -1;
  mg.involved[k] = 0;
}

__global__ void init_size_kernel(DevStats st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < st.M) st.init[k] = st.N[k];
}

// Seeding of a batch: every label cleared, each image's grid (gx[i] x gy[i] labels from
// its label0) with its sums, then InitSize = N.  ims: host copies of the stage-0 images.
cudaError_t launch_seed(const StageArgs &a, const ImageDesc *ims, const int *gx, const int *gy, int n,
                        cudaStream_t s, int *launches) {
  reset_labels_kernel<<<blocks_for(a.st.M, 256), 256, 0, s>>>(a.st, a.mg);
  for (int i = 0; i < n; i++) {
    const long long nb = (long long)ims[i].nbx * ims[i].nby;
    seed_kernel<<<blocks_for(nb, 256), 256, 0, s>>>(a, ims[i], gx[i], gy[i]);
  }
  init_size_kernel<<<blocks_for(a.st.M, 256), 256, 0, s>>>(a.st);
  *launches += 2 + n;
  return cudaGetLastError();
}

// S recomputed from the label map at the current stage's level (the multi-scale
// baseline's per-level statistics; identical to the carried S).
__global__ void zero_stats_kernel(DevStats st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < st.M) st.N[k] = st.R[k] = st.G[k] = st.B[k] = st.X[k] = st.Y[k] = 0;
}

__global__ void accumulate_stats_kernel(StageArgs a, ImageDesc im) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)im.nbx * im.nby) return;
  const int bx = (int)(i % im.nbx), by = (int)(i / im.nbx);
  const int lbl = im.lab[i];
  const BlockSums bs = block_sums(a, im, bx, by);
  atomic_add_i64(&a.st.N[lbl], bs.w);
  atomic_add_i64(&a.st.R[lbl], bs.r);
  atomic_add_i64(&a.st.G[lbl], bs.g);
  atomic_add_i64(&a.st.B[lbl], bs.b);
  atomic_add_i64(&a.st.X[lbl], bs.x);
  atomic_add_i64(&a.st.Y[lbl], bs.y);
}

cudaError_t launch_recompute(const StageArgs &a, const ImageDesc *ims, int n, cudaStream_t s, int *launches) {
  zero_stats_kernel<<<blocks_for(a.st.M, 256), 256, 0, s>>>(a.st);
  for (int i = 0; i < n; i++)
    accumulate_stats_kernel<<<blocks_for((long long)ims[i].nbx * ims[i].nby, 256), 256, 0, s>>>(a, ims[i]);
  *launches += 1 + n;
  return cudaGetLastError();
}

// Stage split: each block becomes 2x2 blocks with its label ("map superpixels' labels").
__global__ void split_kernel(const int *src, int snbx, int *dst, int dnbx, int dnby) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)dnbx * dnby) return;
  const int cx = (int)(i % dnbx), cy = (int)(i / dnbx);
  dst[i] = src[(long long)(cy >> 1) * snbx + (cx >> 1)];
}

cudaError_t launch_split(const int *src, int snbx, int *dst, int dnbx, int dnby, cudaStream_t s) {
  split_kernel<<<blocks_for((long long)dnbx * dnby, 256), 256, 0, s>>>(src, snbx, dst, dnbx, dnby);
  return cudaGetLastError();
}

// Prediction at the start of level 2 (Eq. predict) with the integer stand-in classifier
// h(k) = 3 T N_k - (R_k + G_k + B_k); y = 1 when h >= 0.
__global__ void classify_kernel(DevStats st, long long hT) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= st.M) return;
  const long long h = 3 * hT * st.N[k] - (st.R[k] + st.G[k] + st.B[k]);
  st.y[k] = h >= 0 ? 1 : -1;
  st.imp[k] = 0;
}

// Boundary superpixels (Eq. new_bound): labels 4-adjacent to a label of the other class.
__global__ void importance_kernel(const int *lab, int nbx, int nby, DevStats st) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nbx * nby) return;
  const int bx = (int)(i % nbx), by = (int)(i / nbx);
  const int a = lab[i];
  if (bx + 1 < nbx) {
    const int e = lab[i + 1];
    if (e != a && st.y[e] != st.y[a]) {
      st.imp[a] = 1;
      st.imp[e] = 1;
    }
  }
  if (by + 1 < nby) {
    const int b = lab[i + nbx];
    if (b != a && st.y[b] != st.y[a]) {
      st.imp[a] = 1;
      st.imp[b] = 1;
    }
  }
}

// ---------------------------------------------------------------- features (Sec. 4.1's F)
// The features of a superpixel at the prediction point, with b_k = (R_k + G_k + B_k) /
// (3 N_k) and c_k its mean colour: f1 = b_k; f2 = b_k minus the mean over k's 4-adjacent
// block pairs (p in k, q in j != k) of b_j taken as floor(2^16 b_j) / 2^16; f3 = the mean over
// those pairs of |c_k - c_j| truncated to 2^-16; f4 = sqrt(sum over k's blocks of w_p
// |c_p - c_k|^2, each truncated to 2^-16, over N_k).  Every pair and block term is an
// integer, so the atomic sums do not depend on their order, and the binary64 operations
// are those of the definition in the order written.

// Sums cleared; the mean colours go to feat[4k .. 4k + 2] for the pass over the blocks.
__global__ void feature_init_kernel(DevStats st) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= st.M) return;
  st.fsb[k] = st.fsd[k] = st.fsi[k] = 0;
  st.fnp[k] = 0;
  const long long n = st.N[k];
  double *f = st.feat + 4ll * k;
  if (n > 0) {
    const double dn = __ll2double_rn(n);
    f[0] = __ddiv_rn(__ll2double_rn(st.R[k]), dn);
    f[1] = __ddiv_rn(__ll2double_rn(st.G[k]), dn);
    f[2] = __ddiv_rn(__ll2double_rn(st.B[k]), dn);
  } else {
    f[0] = f[1] = f[2] = 0.0;
  }
  f[3] = 0.0;
}

__device__ __forceinline__ long long brightness_q16(const DevStats &st, int j) {
  return ((st.R[j] + st.G[j] + st.B[j]) << 16) / (3 * st.N[j]);
}

// One thread per block of the prediction grid: its squared deviation, and its pairs with
// the E and S neighbours.
__global__ void feature_pass_kernel(StageArgs a, ImageDesc im, DevStats st) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)im.nbx * im.nby) return;
  const int bx = (int)(i % im.nbx), by = (int)(i / im.nbx);
  const int k = im.lab[i];
  const double *ck = st.feat + 4ll * k;
  const BlockSums bs = block_sums(a, im, bx, by);
  const double w = __ll2double_rn(bs.w);
  const double dr = __dsub_rn(__ddiv_rn(__ll2double_rn(bs.r), w), ck[0]);
  const double dg = __dsub_rn(__ddiv_rn(__ll2double_rn(bs.g), w), ck[1]);
  const double db = __dsub_rn(__ddiv_rn(__ll2double_rn(bs.b), w), ck[2]);
  const double v = __dmul_rn(w, __dadd_rn(__dadd_rn(__dmul_rn(dr, dr), __dmul_rn(dg, dg)), __dmul_rn(db, db)));
  atomicAdd((unsigned long long *)&st.fsi[k], (unsigned long long)__double2ll_rz(__dmul_rn(v, 65536.0)));
  const int q[2] = {bx + 1 < im.nbx ? im.lab[i + 1] : -1, by + 1 < im.nby ? im.lab[i + im.nbx] : -1};
  for (int t = 0; t < 2; t++) {
    const int j = q[t];
    if (j < 0 || j == k) continue;
    atomicAdd((unsigned long long *)&st.fsb[k], (unsigned long long)brightness_q16(st, j));
    atomicAdd((unsigned long long *)&st.fsb[j], (unsigned long long)brightness_q16(st, k));
    atomicAdd(&st.fnp[k], 1);
    atomicAdd(&st.fnp[j], 1);
    const double *cj = st.feat + 4ll * j;
    const double er = __dsub_rn(ck[0], cj[0]), eg = __dsub_rn(ck[1], cj[1]), eb = __dsub_rn(ck[2], cj[2]);
    const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(er, er), __dmul_rn(eg, eg)), __dmul_rn(eb, eb)));
    const unsigned long long dq = (unsigned long long)__double2ll_rz(__dmul_rn(d, 65536.0));
    atomicAdd((unsigned long long *)&st.fsd[k], dq);
    atomicAdd((unsigned long long *)&st.fsd[j], dq);
  }
}

// The features from the sums, then Eq. predict with h = t0 + t1 f1 + t2 f2 + t3 f3 + t4 f4
// (summed left to right): y = 1 when h >= 0.
__global__ void classify_linear_kernel(DevStats st, double t0, double t1, double t2, double t3, double t4) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= st.M) return;
  const long long n = st.N[k];
  double f1 = 0.0, f2 = 0.0, f3 = 0.0, f4 = 0.0;
  if (n > 0) {
    f1 = __ddiv_rn(__ll2double_rn(st.R[k] + st.G[k] + st.B[k]), __ll2double_rn(3 * n));
    const int np = st.fnp[k];
    if (np > 0) {
      const double dnp = (double)np;
      f2 = __dsub_rn(f1, __ddiv_rn(__ddiv_rn(__ll2double_rn(st.fsb[k]), dnp), 65536.0));
      f3 = __ddiv_rn(__ddiv_rn(__ll2double_rn(st.fsd[k]), dnp), 65536.0);
    }
    f4 = __dsqrt_rn(__ddiv_rn(__ddiv_rn(__ll2double_rn(st.fsi[k]), 65536.0), __ll2double_rn(n)));
  }
  double *f = st.feat + 4ll * k;
  f[0] = f1;
  f[1] = f2;
  f[2] = f3;
  f[3] = f4;
  const double h =
      __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(t0, __dmul_rn(t1, f1)), __dmul_rn(t2, f2)), __dmul_rn(t3, f3)),
                __dmul_rn(t4, f4));
  st.y[k] = h >= 0.0 ? 1 : -1;
  st.imp[k] = 0;
}

// Prediction with the linear classifier theta over the features; a: the launch arguments
// of the stage whose block grid the prediction reads (for the block sums).
cudaError_t launch_predict_linear(const StageArgs &a, const ImageDesc *ims, int n, const double *theta,
                                  cudaStream_t s, int *launches) {
  const DevStats &st = a.st;
  feature_init_kernel<<<blocks_for(st.M, 256), 256, 0, s>>>(st);
  for (int i = 0; i < n; i++)
    feature_pass_kernel<<<blocks_for((long long)ims[i].nbx * ims[i].nby, 256), 256, 0, s>>>(a, ims[i], st);
  classify_linear_kernel<<<blocks_for(st.M, 256), 256, 0, s>>>(st, theta[0], theta[1], theta[2], theta[3],
                                                                 theta[4]);
  for (int i = 0; i < n; i++)
    importance_kernel<<<blocks_for((long long)ims[i].nbx * ims[i].nby, 256), 256, 0, s>>>(ims[i].lab, ims[i].nbx,
                                                                                           ims[i].nby, st);
  *launches += 2 + 2 * n;
  return cudaGetLastError();
}

cudaError_t launch_predict(const ImageDesc *ims, int n, const DevStats &st, long long hT, cudaStream_t s,
                           int *launches) {
  classify_kernel<<<blocks_for(st.M, 256), 256, 0, s>>>(st, hT);
  for (int i = 0; i < n; i++)
    importance_kernel<<<blocks_for((long long)ims[i].nbx * ims[i].nby, 256), 256, 0, s>>>(ims[i].lab, ims[i].nbx,
                                                                                           ims[i].nby, st);
  *launches += 1 + n;
  return cudaGetLastError();
}

// Full-resolution label map from a block-resolution one, as image-local ids (global id -
// label0).
__global__ void upsample_kernel(const int *lab, int nbx, int side, int H, int W, int label0, int *dst,
                                long long pitch_elems) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)H * W) return;
  const int x = (int)(i % W), y = (int)(i / W);
  dst[(long long)y * pitch_elems + x] = lab[(long long)(y / side) * nbx + x / side] - label0;
}

cudaError_t launch_upsample(const int *lab, int nbx, int side, int H, int W, int label0, int *dst,
                            long long pitch_elems, cudaStream_t s) {
  upsample_kernel<<<blocks_for((long long)H * W, 256), 256, 0, s>>>(lab, nbx, side, H, W, label0, dst, pitch_elems);
  return cudaGetLastError();
}

// rapid_sp_stats records of the labels label0 .. label0 + M - 1 (entry k - label0).
__global__ void pack_stats_kernel(DevStats st, int label0, int M, rapid_sp_stats *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int k = label0 + j;
  rapid_sp_stats v;
  v.n = st.N[k];
  v.sum_r = st.R[k];
  v.sum_g = st.G[k];
  v.sum_b = st.B[k];
  v.sum_x = st.X[k];
  v.sum_y = st.Y[k];
  v.init_size = st.init[k];
  v.y = st.y[k];
  v.important = st.imp[k];
  out[j] = v;
}

cudaError_t launch_pack_stats(const DevStats &st, int label0, int M, rapid_sp_stats *out, cudaStream_t s) {
  pack_stats_kernel<<<blocks_for(M, 256), 256, 0, s>>>(st, label0, M, out);
  return cudaGetLastError();
}

// Counters of n images x 32 stages: level and side of every stage, the rest zero.
__global__ void init_counters_kernel(long long *cnt, Schedule sch, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * RAPID_MAX_STAGES) return;
  const int st = i % RAPID_MAX_STAGES;
  long long *c = cnt + (long long)i * CNT_N;
  for (int j = 0; j < CNT_N; j++) c[j] = 0;
  if (st < sch.n) {
    c[CNT_LEVEL] = sch.level[st];
    c[CNT_SIDE] = sch.side[st];
  }
}

cudaError_t launch_init_counters(long long *cnt, const Schedule &sch, int n, cudaStream_t s) {
  init_counters_kernel<<<blocks_for((long long)n * RAPID_MAX_STAGES, 128), 128, 0, s>>>(cnt, sch, n);
  return cudaGetLastError();
}

__global__ void simple_table_kernel(unsigned char *out) {
  const unsigned m = threadIdx.x;
  out[m] = simple_mask(m) ? 1 : 0;
}

cudaError_t launch_simple_table(unsigned char *out, cudaStream_t s) {
  simple_table_kernel<<<1, 256, 0, s>>>(out);
  return cudaGetLastError();
}

}  // namespace rapid

namespace rapid {

// Per-label arrays, each in its own 256-byte aligned piece.
static size_t carve_impl(char *base, size_t cap, int M, DevStats *st, DevMerge *mg) {
  const size_t m = (size_t)M;
  size_t used = 0;
  bool ok = true;
  auto take = [&](size_t n) -> void * {
    n = (n + 255) / 256 * 256;
    if (used + n > cap) {
      ok = false;
      return nullptr;
    }
    void *r = base ? base + used : nullptr;
    used += n;
    return r;
  };
  long long **i64[] = {&st->N, &st->R, &st->G, &st->B, &st->X, &st->Y, &st->init,
                       &st->mN};
  for (long long **q : i64) *q = (long long *)take(m * 8);
  double **f64[] = {&st->mR, &st->mG, &st->mB, &st->mX, &st->mY};
  for (double **q : f64) *q = (double *)take(m * 8);
  st->fhi = (float4 *)take(m * 16);
  st->flo = (float4 *)take(m * 16);
  st->fy = (float2 *)take(m * 8);
  st->bbox = (int4 *)take(m * 16);
  st->chg = (int *)take(m * 4);
  st->adj = (int *)take(m * 4);
  st->fsb = (long long *)take(m * 8);
  st->fsd = (long long *)take(m * 8);
  st->fsi = (long long *)take(m * 8);
  st->fnp = (int *)take(m * 4);
  st->feat = (double *)take(m * 32);
  mg->acc = (int2 *)take(m * 8);
  mg->req_min = (unsigned long long *)take(m * 8);
  int **i32[] = {&mg->req_list, &mg->req_flag, &mg->target, &mg->order, &mg->cache_stamp, &mg->cache_n};
  for (int **q : i32) *q = (int *)take(m * 4);
  mg->cache_nb = (int *)take(m * 4 * kCacheLabels);
  mg->found = (int *)take(m * 4);

  st->dirty = (unsigned char *)take(m);
  st->y = (signed char *)take(m);
  st->imp = (unsigned char *)take(m);
  mg->involved = (unsigned char *)take(m);
  st->M = M;
  return ok ? used : 0;
}

size_t label_arrays_bytes(int M) {
  DevStats st;
  DevMerge mg;
  return carve_impl(nullptr, (size_t)-1, M, &st, &mg);
}

size_t carve_label_arrays(void *base, size_t cap, int M, DevStats *st, DevMerge *mg) {
  return carve_impl((char *)base, cap, M, st, mg);
}

}  // namespace rapid
