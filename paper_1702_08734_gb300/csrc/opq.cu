// Training of the OPQ pre-rotation (the optimized product quantization of the paper's
// DEEP1B / YFCC100M runs, sections 1 and 6.4; the paper cites it and does not specify it).
// Non-parametric OPQ alternates two steps on the training vectors x (rows):
//   1. with R fixed, the product quantizer of the rotated vectors x R^T: one 256-centroid
//      k-means per block of d/M dimensions, and every rotated vector's reconstruction y^;
//   2. with the reconstructions fixed, the orthogonal R minimising ||x R^T - Y^||_F: the
//      orthogonal Procrustes solution R = U V^T for A = Y^T x = U S V^T (the polar factor
//      of A), computed here in double precision by the scaled Newton iteration
//      X <- (g X + X^{-T} / g) / 2, g = (||X^{-1}||_F / ||X||_F)^(1/2) (Higham), which
//      converges quadratically whatever the conditioning of A, the inverse by Gauss-Jordan
//      elimination with partial pivoting; two Newton-Schulz steps
//      X <- X (3 I - X^T X) / 2 polish the orthogonality at the end.
// The result is installed as the index's rotation (as gbk_ivfpq_set_rotation does).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ivf.cuh"
#include "ivf_index.cuh"
#include "knn.cuh"

namespace gbk {

gbk_status pq_encode_run(const float* x, int64_t n, int d, int M, const float* coarse,
                         const int32_t* lists, const float* pq, uint8_t* codes, cudaStream_t st);

namespace {

// y[i][m*dsub + t] = books[m][codes[i][m]][t]
__global__ void reconstruct_kernel(const uint8_t* __restrict__ codes, const float* __restrict__ books,
                                   int64_t n, int d, int M, float* __restrict__ y) {
  const int dsub = d / M;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int t = (int)(e % d), m = t / dsub;
    y[e] = books[((int64_t)m * 256 + codes[i * M + m]) * dsub + (t % dsub)];
  }
}

// Partial A[s] = sum over rows i of split s of y[i]^T x[i] (d x d, double), one 32 x 32
// output tile per block (blockIdx.x: tile, blockIdx.y: split); rows in increasing order.
__global__ void cross_partial_kernel(const float* __restrict__ y, const float* __restrict__ x,
                                     int64_t n, int d, int64_t rows_per_split,
                                     double* __restrict__ part) {
  const int tiles = (d + 31) / 32;
  const int ti = blockIdx.x / tiles, tj = blockIdx.x % tiles;
  const int64_t r0 = blockIdx.y * rows_per_split;
  const int64_t r1 = min(n, r0 + rows_per_split);
  __shared__ float ys[32][33], xs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8 threads, 4 outputs each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t b = r0; b < r1; b += 32) {
    for (int l = threadIdx.x; l < 32 * 32; l += blockDim.x) {
      const int rr = l / 32, cc = l % 32;
      const int64_t row = b + rr;
      const int ci = ti * 32 + cc, cj = tj * 32 + cc;
      ys[rr][cc] = (row < r1 && ci < d) ? y[row * d + ci] : 0.f;
      xs[rr][cc] = (row < r1 && cj < d) ? x[row * d + cj] : 0.f;
    }
    __syncthreads();
    for (int rr = 0; rr < 32; rr++) {
      const double xv = xs[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] += (double)ys[rr][ty * 4 + q] * xv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int i = ti * 32 + ty * 4 + q, j = tj * 32 + tx;
    if (i < d && j < d) part[((int64_t)blockIdx.y * d + i) * d + j] = acc[q];
  }
}

// A = sum of the split partials in split order; also ||A||_F^2 into *fro (one block).
__global__ void cross_reduce_kernel(const double* __restrict__ part, int splits, int d,
                                    double* __restrict__ A) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; k++) s += part[(int64_t)k * d * d + e];
    A[e] = s;
  }
}

// C = alpha * op(A) B + beta * Cin for d x d row-major doubles, op(A) = A or A^T; 16 x 16 tiles
__global__ void gemm_f64_kernel(const double* __restrict__ A, const double* __restrict__ B, int d,
                                bool transA, double alpha, const double* __restrict__ Cin,
                                double beta, double* __restrict__ C) {
  __shared__ double as[16][17], bs[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < d; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    as[ty][tx] = (i < d && ka < d) ? (transA ? A[(int64_t)ka * d + i] : A[(int64_t)i * d + ka]) : 0.0;
    bs[ty][tx] = (kb < d && j < d) ? B[(int64_t)kb * d + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) acc += as[ty][kk] * bs[kk][tx];
    __syncthreads();
  }
  if (i < d && j < d) {
    const int64_t e = (int64_t)i * d + j;
    C[e] = alpha * acc + (Cin ? beta * Cin[e] : 0.0);
  }
}

// One block: inverse of the d x d matrix X (row-major doubles) by Gauss-Jordan elimination
// with partial pivoting on the workspace W [d][2d] = [X | I]; Xinv out.  *singular = 1 when
// a pivot is zero (Xinv then undefined).
__global__ void __launch_bounds__(1024) gauss_jordan_kernel(const double* __restrict__ X, int d,
                                                          double* __restrict__ W,
                                                          double* __restrict__ Xinv,
                                                          int* __restrict__ singular) {
  const int tid = threadIdx.x, nt = blockDim.x, w2 = 2 * d;
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int piv;
  __shared__ double pval;
  for (int e = tid; e < d * w2; e += nt) {
    const int r = e / w2, c = e % w2;
    W[e] = c < d ? X[(int64_t)r * d + c] : (c - d == r ? 1.0 : 0.0);
  }
  if (tid == 0) *singular = 0;
  __syncthreads();
  for (int c = 0; c < d; c++) {
    // pivot: the row r >= c with the largest |W[r][c]| (lowest r on ties)
    double bv = -1.0;
    int bi = c;
    for (int r = c + tid; r < d; r += nt) {
      const double v = fabs(W[(int64_t)r * w2 + c]);
      if (v > bv) {
        bv = v;
        bi = r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      red_v[tid >> 5] = bv;
      red_i[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double v = red_v[0];
      int i = red_i[0];
      for (int w = 1; w < (nt + 31) / 32; w++)
        if (red_v[w] > v || (red_v[w] == v && red_i[w] < i)) {
          v = red_v[w];
          i = red_i[w];
        }
      piv = i;
      if (!(v > 0.0)) *singular = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != c)
      for (int j = tid; j < w2; j += nt) {
        const double t = W[(int64_t)c * w2 + j];
        W[(int64_t)c * w2 + j] = W[(int64_t)p * w2 + j];
        W[(int64_t)p * w2 + j] = t;
      }
    __syncthreads();
    if (tid == 0) pval = W[(int64_t)c * w2 + c];
    __syncthreads();
    const double inv = pval != 0.0 ? 1.0 / pval : 0.0;
    for (int j = tid; j < w2; j += nt) W[(int64_t)c * w2 + j] *= inv;
    __syncthreads();
    // eliminate column c from every other row (factors read before any row changes)
    for (int e = tid; e < d * w2; e += nt) {
      const int r = e / w2, j = e % w2;
      if (r == c || j == c) continue;
      W[e] -= W[(int64_t)r * w2 + c] * W[(int64_t)c * w2 + j];
    }
    __syncthreads();
    for (int r = tid; r < d; r += nt)
      if (r != c) W[(int64_t)r * w2 + c] = 0.0;
    __syncthreads();
  }
  for (int e = tid; e < d * d; e += nt) {
    const int r = e / d, j = e % d;
    Xinv[e] = W[(int64_t)r * w2 + d + j];
  }
}

// X <- (g X + Xinv^T / g) / 2 with g = sqrt(||Xinv||_F / ||X||_F) (one block)
__global__ void newton_step_kernel(double* __restrict__ X, const double* __restrict__ Xinv, int d) {
  __shared__ double sa[256], sb[256];
  double a = 0.0, b = 0.0;
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    a += X[e] * X[e];
    b += Xinv[e] * Xinv[e];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double g = sqrt(sqrt(sb[0]) / sqrt(sa[0]));
  __syncthreads();
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int r = e / d, c = e % d;
    X[e] = 0.5 * (g * X[e] + Xinv[(int64_t)c * d + r] / g);
  }
}

__global__ void to_float_kernel(const double* __restrict__ Z, int n, float* __restrict__ R) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    R[e] = (float)Z[e];
}

__global__ void identity_kernel(int d, float* __restrict__ R) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * d; e += gridDim.x * blockDim.x)
    R[e] = (e / d == e % d) ? 1.f : 0.f;
}

// Polar factor of the d x d matrix A (device doubles) into R (float): `iters` scaled
// Newton steps from X = A, then two Newton-Schulz steps.  GBK_EINVAL if A is singular.
gbk_status polar_run(const double* A, int d, int iters, float* R, cudaStream_t st) {
  gbk_status r;
  Scratch X, Xi, W, T, X2, sing;
  const size_t b = sizeof(double) * (size_t)d * d;
  if ((r = X.alloc(b, st)) != GBK_OK || (r = Xi.alloc(b, st)) != GBK_OK ||
      (r = W.alloc(2 * b, st)) != GBK_OK || (r = T.alloc(b, st)) != GBK_OK ||
      (r = X2.alloc(b, st)) != GBK_OK || (r = sing.alloc(sizeof(int), st)) != GBK_OK)
    return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(X.p, A, b, cudaMemcpyDeviceToDevice, st));
  for (int it = 0; it < iters; it++) {
    gauss_jordan_kernel<<<1, 1024, 0, st>>>(X.as<double>(), d, W.as<double>(), Xi.as<double>(),
                                            sing.as<int>());
    newton_step_kernel<<<1, 256, 0, st>>>(X.as<double>(), Xi.as<double>(), d);
  }
  GBK_LAUNCH_CHECK();
  int singular = 0;
  GBK_CUDA_CHECK(cudaMemcpyAsync(&singular, sing.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (singular)
    return set_error(GBK_EINVAL, "gbk_ivfpq_train_rotation: singular cross-covariance (degenerate training data)");
  const dim3 grid((d + 15) / 16, (d + 15) / 16);
  double* x = X.as<double>();
  double* x2 = X2.as<double>();
  for (int it = 0; it < 2; it++) {
    gemm_f64_kernel<<<grid, 256, 0, st>>>(x, x, d, true, 1.0, nullptr, 0.0, T.as<double>());
    gemm_f64_kernel<<<grid, 256, 0, st>>>(x, T.as<double>(), d, false, -0.5, x, 1.5, x2);
    std::swap(x, x2);
  }
  to_float_kernel<<<(d * d + 255) / 256, 256, 0, st>>>(x, d * d, R);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_ivfpq_train_rotation(gbk_index* ix, const float* x, int64_t n,
                                    const gbk_opq_opts* opts, float* R_out, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && x, "gbk_ivfpq_train_rotation: NULL argument");
  GBK_REQUIRE(!ix->trained && ix->n_staged == 0,
              "gbk_ivfpq_train_rotation: must run before training and adding");
  GBK_REQUIRE(n >= 256 && n < (int64_t(1) << 31), "gbk_ivfpq_train_rotation: need 256 <= n < 2^31");
  GBK_REQUIRE(ix->d <= 1024, "gbk_ivfpq_train_rotation: d <= 1024");
  const int niter = opts && opts->niter > 0 ? opts->niter : 10;
  const int pq_niter = opts && opts->pq_niter > 0 ? opts->pq_niter : 4;
  const int ns_iters = opts && opts->polar_iters > 0 ? opts->polar_iters : 12;
  std::vector<int64_t> pinit(256);
  for (int i = 0; i < 256; i++) pinit[i] = opts && opts->pq_init ? opts->pq_init[i] : i;
  for (int64_t v : pinit)
    GBK_REQUIRE(v >= 0 && v < n, "gbk_ivfpq_train_rotation: pq_init out of range");
  cudaStream_t st = as_stream(stream);
  const int d = ix->d, M = ix->M, dsub = ix->dsub;
  gbk_status r;
  if ((r = ix->rot.alloc(sizeof(float) * (size_t)d * d)) != GBK_OK) return r;
  identity_kernel<<<(d * d + 255) / 256, 256, 0, st>>>(d, ix->rot.as<float>());
  GBK_LAUNCH_CHECK();
  ix->rotated = true;
  Scratch pi, zero_c, zero_l, books, codes, y, part, A;
  if ((r = pi.alloc(sizeof(int64_t) * 256, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(pi.p, pinit.data(), sizeof(int64_t) * 256, cudaMemcpyHostToDevice,
                                 st));
  if ((r = zero_c.alloc(sizeof(float) * d, st)) != GBK_OK) return r;
  if ((r = zero_l.alloc(sizeof(int32_t) * (size_t)n, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemsetAsync(zero_c.p, 0, sizeof(float) * d, st));
  GBK_CUDA_CHECK(cudaMemsetAsync(zero_l.p, 0, sizeof(int32_t) * (size_t)n, st));
  if ((r = books.alloc(sizeof(float) * (size_t)M * 256 * dsub, st)) != GBK_OK) return r;
  if ((r = codes.alloc((size_t)n * M, st)) != GBK_OK) return r;
  if ((r = y.alloc(sizeof(float) * (size_t)n * d, st)) != GBK_OK) return r;
  const int tiles = (d + 31) / 32;
  const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(
      (int64_t)(4 * device_info().sm_count) / (tiles * tiles) + 1, (n + 4095) / 4096));
  const int64_t rows_per_split = ((n + splits - 1) / splits + 31) / 32 * 32;
  if ((r = part.alloc(sizeof(double) * (size_t)splits * d * d, st)) != GBK_OK) return r;
  if ((r = A.alloc(sizeof(double) * (size_t)d * d, st)) != GBK_OK) return r;
  ProfScope prof("opq_train", st);
  for (int it = 0; it < niter; it++) {
    Scratch xr;
    const float* xrot = x;
    if ((r = rotate_rows(ix, x, n, xr, &xrot, st)) != GBK_OK) return r;
    // 1. product quantizer of the rotated vectors and their reconstructions
    for (int m = 0; m < M; m++) {
      if ((r = kmeans_run(xrot + m * dsub, n, dsub, d, 256, pq_niter, pi.as<int64_t>(),
                          books.as<float>() + (size_t)m * 256 * dsub, nullptr, nullptr, true,
                          st)) != GBK_OK)
        return r;
    }
    if ((r = pq_encode_run(xrot, n, d, M, zero_c.as<float>(), zero_l.as<int32_t>(),
                           books.as<float>(), codes.as<uint8_t>(), st)) != GBK_OK)
      return r;
    reconstruct_kernel<<<(unsigned)std::min<int64_t>((n * d + 255) / 256, 65536), 256, 0, st>>>(
        codes.as<uint8_t>(), books.as<float>(), n, d, M, y.as<float>());
    GBK_LAUNCH_CHECK();
    // 2. orthogonal Procrustes: R = polar(Y^T x)
    cross_partial_kernel<<<dim3(tiles * tiles, splits), 256, 0, st>>>(
        y.as<float>(), x, n, d, rows_per_split, part.as<double>());
    cross_reduce_kernel<<<(d * d + 255) / 256, 256, 0, st>>>(part.as<double>(), splits, d,
                                                            A.as<double>());
    GBK_LAUNCH_CHECK();
    if ((r = polar_run(A.as<double>(), d, ns_iters, ix->rot.as<float>(), st)) != GBK_OK) return r;
  }
  if (R_out)
    GBK_CUDA_CHECK(cudaMemcpyAsync(R_out, ix->rot.p, sizeof(float) * (size_t)d * d,
                                   cudaMemcpyDefault, st));
  return GBK_OK;
}

}  // extern "C"
