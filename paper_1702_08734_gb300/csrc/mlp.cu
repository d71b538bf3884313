// Learned nprobe: a small MLP (query features -> per-query nprobe class) trained on the GPU
// with the library's own forward, backward and Adam kernels.
//
//   h1 = relu(W1 f + b1),  h2 = relu(W2 h1 + b2),  z = W3 h2 + b3,  loss = mean CE(z, y)
// Weights live as a float32 master copy; every forward/backward pass reads them rounded to
// BF16 (round-to-nearest-even), with float32 accumulation.  Adam (Kingma & Ba 2015) updates
// the master copy.  The batch reductions of the weight gradients run in a fixed order, so a
// training run is bit-reproducible.  The layers are tiny (at most 256 x 256), so the
// contractions are tiled SIMT kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gbk {

namespace {

__device__ __forceinline__ float bf16r(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// Row-wise softmax cross-entropy: dz = (softmax(z) - onehot(y)) / B; loss_row out.
__global__ void softmax_ce_kernel(const float* __restrict__ z, const int32_t* __restrict__ y,
                                  int64_t B, int C, float* __restrict__ dz,
                                  float* __restrict__ loss_row) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const float* zr = z + r * C;
  float mx = zr[0];
  for (int c = 1; c < C; c++) mx = fmaxf(mx, zr[c]);
  float se = 0.f;
  for (int c = 0; c < C; c++) se += expf(zr[c] - mx);
  const float lse = mx + logf(se);
  loss_row[r] = lse - zr[y[r]];
  for (int c = 0; c < C; c++) {
    const float p = expf(zr[c] - lse);
    dz[r * C + c] = (p - (c == y[r] ? 1.f : 0.f)) / (float)B;
  }
}

// dA = dH * (A > 0) in place on dH (A = pre-activation, kept as relu output h > 0 test).
__global__ void relu_bwd_kernel(float* __restrict__ dh, const float* __restrict__ h, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(h[i] > 0.f)) dh[i] = 0.f;
}

// db[n] = sum over rows of dY[r][n], fixed order.
__global__ void colsum_kernel(const float* __restrict__ dy, int64_t B, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int64_t r = 0; r < B; r++) s += dy[r * N + n];
  db[n] = s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void argmax_kernel(const float* __restrict__ z, int64_t B, int C, int32_t* __restrict__ cls) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  int best = 0;
  for (int c = 1; c < C; c++)
    if (z[r * C + c] > z[r * C + best]) best = c;
  cls[r] = best;
}

// Smallest class whose softmax cumulative probability reaches alpha (classes ordered by
// cost, as the nprobe classes are): a confidence level for routing instead of the argmax.
__global__ void quantile_class_kernel(const float* __restrict__ z, int64_t B, int C, float alpha,
                                      int32_t* __restrict__ cls) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const float* zr = z + r * C;
  float mx = zr[0];
  for (int c = 1; c < C; c++) mx = fmaxf(mx, zr[c]);
  float se = 0.f;
  for (int c = 0; c < C; c++) se += expf(zr[c] - mx);
  float cum = 0.f;
  int c = 0;
  for (; c < C - 1; c++) {
    cum += expf(zr[c] - mx) / se;
    if (cum >= alpha) break;
  }
  cls[r] = c;
}

__global__ void loss_sum_kernel(const float* __restrict__ lr, int64_t B, float* __restrict__ out) {
  // single block, fixed order: per-thread strided partials then a tree
  __shared__ float part[256];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < B; i += 256) s += lr[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0] / (float)B;
}

int grid1(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// C[M][N] = sum_k A(m, k) * B(k, n) (+ bias[n]) (relu optional); accumulate into C when acc.
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// RB: round B elements to BF16 (weights).  Each output is summed over k in increasing
// order with fmaf (a fixed order).  64 x 64 block tiles, 4 x 4 outputs per thread: 16 FMAs
// per pair of 16-byte shared-memory reads.
constexpr int BT = 64, BK = 16;
template <bool TA, bool TB, bool RB>
__global__ void __launch_bounds__(256)
    gemm64(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B,
           int ldb, float* __restrict__ C, int ldc, const float* __restrict__ bias, int relu,
           int acc) {
  __shared__ __align__(16) float As[BK][BT + 4];
  __shared__ __align__(16) float Bs[BK][BT + 4];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int m0 = blockIdx.y * BT, n0 = blockIdx.x * BT;
  float s[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const int i = t + 256 * r;
      const int km = TA ? i / BT : i % BK, mm = TA ? i % BT : i / BK;
      const int gm = m0 + mm, gk = k0 + km;
      As[km][mm] = (gm < M && gk < K) ? (TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk])
                                      : 0.f;
      const int kn = TB ? i % BK : i / BT, nn = TB ? i / BK : i % BT;
      const int gn = n0 + nn, gk2 = k0 + kn;
      const float b = (gn < N && gk2 < K) ? (TB ? B[(int64_t)gn * ldb + gk2] : B[(int64_t)gk2 * ldb + gn])
                                          : 0.f;
      Bs[kn][nn] = RB ? bf16r(b) : b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) s[i][j] = fmaf(av[i], bv[j], s[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = s[i][j];
      if (bias) v += bias[n];
      if (relu) v = fmaxf(v, 0.f);
      float* c = C + (int64_t)m * ldc + n;
      *c = acc ? *c + v : v;
    }
  }
}

template <bool TA, bool TB, bool RB>
void mm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
        const float* bias, bool relu, bool acc, cudaStream_t st) {
  dim3 grd((N + BT - 1) / BT, (M + BT - 1) / BT);
  gemm64<TA, TB, RB><<<grd, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu ? 1 : 0,
                                          acc ? 1 : 0);
}

}  // namespace

}  // namespace gbk

// Parameter layout (one float array, in this order): W1 [h1][in], b1 [h1], W2 [h2][h1],
// b2 [h2], W3 [out][h2], b3 [out].
// Parameter e drawn from U(-bound, bound), bound = 1/sqrt(fan-in) of its layer (W1, b1:
// n_in; W2, b2: h1; W3, b3: h2), from the 24 high bits of a SplitMix64 hash of (seed, e).
__global__ void init_uniform_kernel(float* __restrict__ p, int64_t n, int64_t off2, int64_t off4,
                                    float bound1, float bound2, float bound3, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed * 0x9e3779b97f4a7c15ull + (uint64_t)(e + 1) * 0xd1b54a32d192ed03ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    const float u = (float)(z >> 40) * (1.f / 16777216.f);
    const float bound = e < off2 ? bound1 : (e < off4 ? bound2 : bound3);
    p[e] = (2.f * u - 1.f) * bound;
  }
}

struct gbk_mlp {
  int n_in, h1, h2, n_out;
  int64_t nparam;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int64_t step = 0;
  int64_t off[6];
  ~gbk_mlp() {
    if (p) cudaFree(p);
    if (g) cudaFree(g);
    if (m) cudaFree(m);
    if (v) cudaFree(v);
  }
};

using namespace gbk;

namespace {

// Forward over B rows; activations (h1, h2, z) into caller scratch.
gbk_status mlp_forward(gbk_mlp* n, const float* X, int64_t B, float* h1, float* h2, float* z,
                       cudaStream_t st) {
  const float* W1 = n->p + n->off[0];
  const float* b1 = n->p + n->off[1];
  const float* W2 = n->p + n->off[2];
  const float* b2 = n->p + n->off[3];
  const float* W3 = n->p + n->off[4];
  const float* b3 = n->p + n->off[5];
  mm<false, true, true>((int)B, n->h1, n->n_in, X, n->n_in, W1, n->n_in, h1, n->h1, b1, true, false, st);
  mm<false, true, true>((int)B, n->h2, n->h1, h1, n->h1, W2, n->h1, h2, n->h2, b2, true, false, st);
  mm<false, true, true>((int)B, n->n_out, n->h2, h2, n->h2, W3, n->h2, z, n->n_out, b3, false, false,
                        st);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status mlp_grad(gbk_mlp* n, const float* X, const int32_t* y, int64_t B, float* loss,
                    cudaStream_t st) {
  gbk_status r;
  Scratch sh1, sh2, sz, sdz, sdh2, sdh1, slr;
  if ((r = sh1.alloc(sizeof(float) * B * n->h1, st)) != GBK_OK) return r;
  if ((r = sh2.alloc(sizeof(float) * B * n->h2, st)) != GBK_OK) return r;
  if ((r = sz.alloc(sizeof(float) * B * n->n_out, st)) != GBK_OK) return r;
  if ((r = sdz.alloc(sizeof(float) * B * n->n_out, st)) != GBK_OK) return r;
  if ((r = sdh2.alloc(sizeof(float) * B * n->h2, st)) != GBK_OK) return r;
  if ((r = sdh1.alloc(sizeof(float) * B * n->h1, st)) != GBK_OK) return r;
  if ((r = slr.alloc(sizeof(float) * B, st)) != GBK_OK) return r;
  float *h1 = sh1.as<float>(), *h2 = sh2.as<float>(), *z = sz.as<float>(), *dz = sdz.as<float>();
  float *dh2 = sdh2.as<float>(), *dh1 = sdh1.as<float>();
  if ((r = mlp_forward(n, X, B, h1, h2, z, st)) != GBK_OK) return r;
  softmax_ce_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(z, y, B, n->n_out, dz,
                                                                slr.as<float>());
  if (loss) loss_sum_kernel<<<1, 256, 0, st>>>(slr.as<float>(), B, loss);
  float* g = n->g;
  const float* W2 = n->p + n->off[2];
  const float* W3 = n->p + n->off[4];
  // layer 3: dW3 = dz^T h2, db3 = colsum dz, dh2 = dz W3
  mm<true, false, false>(n->n_out, n->h2, (int)B, dz, n->n_out, h2, n->h2, g + n->off[4], n->h2,
                         nullptr, false, false, st);
  colsum_kernel<<<(n->n_out + 127) / 128, 128, 0, st>>>(dz, B, n->n_out, g + n->off[5]);
  mm<false, false, true>((int)B, n->h2, n->n_out, dz, n->n_out, W3, n->h2, dh2, n->h2, nullptr,
                         false, false, st);
  relu_bwd_kernel<<<grid1(B * n->h2), 256, 0, st>>>(dh2, h2, B * n->h2);
  // layer 2
  mm<true, false, false>(n->h2, n->h1, (int)B, dh2, n->h2, h1, n->h1, g + n->off[2], n->h1,
                         nullptr, false, false, st);
  colsum_kernel<<<(n->h2 + 127) / 128, 128, 0, st>>>(dh2, B, n->h2, g + n->off[3]);
  mm<false, false, true>((int)B, n->h1, n->h2, dh2, n->h2, W2, n->h1, dh1, n->h1, nullptr, false,
                         false, st);
  relu_bwd_kernel<<<grid1(B * n->h1), 256, 0, st>>>(dh1, h1, B * n->h1);
  // layer 1
  mm<true, false, false>(n->h1, n->n_in, (int)B, dh1, n->h1, X, n->n_in, g + n->off[0], n->n_in,
                         nullptr, false, false, st);
  colsum_kernel<<<(n->h1 + 127) / 128, 128, 0, st>>>(dh1, B, n->h1, g + n->off[1]);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace

namespace gbk {
int mlp_inputs(const gbk_mlp* n) { return n ? n->n_in : 0; }
int mlp_outputs(const gbk_mlp* n) { return n ? n->n_out : 0; }

gbk_status mlp_forward_classes(gbk_mlp* n, const float* X, int64_t B, int32_t* cls,
                               cudaStream_t st, float alpha) {
  ProfScope prof("mlp_forward", st);
  gbk_status r;
  Scratch sh1, sh2, sz;
  if ((r = sh1.alloc(sizeof(float) * B * n->h1, st)) != GBK_OK) return r;
  if ((r = sh2.alloc(sizeof(float) * B * n->h2, st)) != GBK_OK) return r;
  if ((r = sz.alloc(sizeof(float) * B * n->n_out, st)) != GBK_OK) return r;
  if ((r = mlp_forward(n, X, B, sh1.as<float>(), sh2.as<float>(), sz.as<float>(), st)) != GBK_OK)
    return r;
  if (alpha > 0.f)
    quantile_class_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(sz.as<float>(), B, n->n_out,
                                                                       alpha, cls);
  else
    argmax_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(sz.as<float>(), B, n->n_out, cls);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}
}  // namespace gbk

extern "C" {

gbk_status gbk_mlp_create(int32_t n_in, int32_t h1, int32_t h2, int32_t n_out,
                          const float* init_params, gbk_mlp** out) {
  clear_error();
  GBK_REQUIRE(out && n_in >= 1 && h1 >= 1 && h2 >= 1 && n_out >= 2, "gbk_mlp_create: bad sizes");
  gbk_mlp* n = new gbk_mlp();
  n->n_in = n_in;
  n->h1 = h1;
  n->h2 = h2;
  n->n_out = n_out;
  const int64_t sz[6] = {(int64_t)h1 * n_in, h1, (int64_t)h2 * h1, h2, (int64_t)n_out * h2, n_out};
  int64_t o = 0;
  for (int i = 0; i < 6; i++) {
    n->off[i] = o;
    o += sz[i];
  }
  n->nparam = o;
  const size_t b = sizeof(float) * (size_t)o;
  if (cudaMalloc(&n->p, b) != cudaSuccess || cudaMalloc(&n->g, b) != cudaSuccess ||
      cudaMalloc(&n->m, b) != cudaSuccess || cudaMalloc(&n->v, b) != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return set_error(GBK_ENOMEM, "gbk_mlp_create: cudaMalloc failed");
  }
  cudaMemset(n->m, 0, b);
  cudaMemset(n->v, 0, b);
  cudaMemset(n->g, 0, b);
  if (init_params)
    cudaMemcpy(n->p, init_params, b, cudaMemcpyDefault);
  else
    cudaMemset(n->p, 0, b);
  *out = n;
  return GBK_OK;
}

gbk_status gbk_mlp_init_uniform(gbk_mlp* n, uint64_t seed, void* stream) {
  clear_error();
  GBK_REQUIRE(n, "gbk_mlp_init_uniform: NULL network");
  cudaStream_t st = as_stream(stream);
  const int64_t fan[3] = {n->n_in, n->h1, n->h2};
  init_uniform_kernel<<<grid1(n->nparam), 256, 0, st>>>(n->p, n->nparam, n->off[2], n->off[4],
                                                        1.f / sqrtf((float)fan[0]),
                                                        1.f / sqrtf((float)fan[1]),
                                                        1.f / sqrtf((float)fan[2]), seed);
  GBK_LAUNCH_CHECK();
  const size_t b = sizeof(float) * (size_t)n->nparam;
  GBK_CUDA_CHECK(cudaMemsetAsync(n->m, 0, b, st));
  GBK_CUDA_CHECK(cudaMemsetAsync(n->v, 0, b, st));
  n->step = 0;
  return GBK_OK;
}

void gbk_mlp_destroy(gbk_mlp* n) { delete n; }

int64_t gbk_mlp_num_params(const gbk_mlp* n) { return n ? n->nparam : 0; }

gbk_status gbk_mlp_params(gbk_mlp* n, float* params_out, float* grads_out, void* stream) {
  clear_error();
  GBK_REQUIRE(n, "gbk_mlp_params: NULL network");
  cudaStream_t st = as_stream(stream);
  const size_t b = sizeof(float) * (size_t)n->nparam;
  if (params_out) GBK_CUDA_CHECK(cudaMemcpyAsync(params_out, n->p, b, cudaMemcpyDefault, st));
  if (grads_out) GBK_CUDA_CHECK(cudaMemcpyAsync(grads_out, n->g, b, cudaMemcpyDefault, st));
  return GBK_OK;
}

gbk_status gbk_mlp_forward(gbk_mlp* n, const float* X, int64_t B, float* logits, int32_t* cls,
                           void* stream) {
  clear_error();
  GBK_REQUIRE(n && X && B >= 0 && B < (int64_t(1) << 31), "gbk_mlp_forward: bad arguments");
  if (B == 0) return GBK_OK;
  cudaStream_t st = as_stream(stream);
  ProfScope prof("mlp_forward", st);
  gbk_status r;
  Scratch sh1, sh2, sz;
  if ((r = sh1.alloc(sizeof(float) * B * n->h1, st)) != GBK_OK) return r;
  if ((r = sh2.alloc(sizeof(float) * B * n->h2, st)) != GBK_OK) return r;
  float* z = logits;
  if (!z) {
    if ((r = sz.alloc(sizeof(float) * B * n->n_out, st)) != GBK_OK) return r;
    z = sz.as<float>();
  }
  if ((r = mlp_forward(n, X, B, sh1.as<float>(), sh2.as<float>(), z, st)) != GBK_OK) return r;
  if (cls) {
    argmax_kernel<<<(unsigned)((B + 127) / 128), 128, 0, st>>>(z, B, n->n_out, cls);
    GBK_LAUNCH_CHECK();
  }
  return GBK_OK;
}

gbk_status gbk_mlp_train_step(gbk_mlp* n, const float* X, const int32_t* labels, int64_t B,
                              float lr, int32_t update, float* loss, void* stream) {
  clear_error();
  GBK_REQUIRE(n && X && labels && B >= 1 && B < (int64_t(1) << 31), "gbk_mlp_train_step: bad arguments");
  cudaStream_t st = as_stream(stream);
  ProfScope prof("mlp_train_step", st);
  gbk_status r;
  if ((r = mlp_grad(n, X, labels, B, loss, st)) != GBK_OK) return r;
  if (update) {
    n->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
    adam_kernel<<<grid1(n->nparam), 256, 0, st>>>(n->p, n->g, n->m, n->v, n->nparam, lr, b1, b2,
                                                  1e-8f, c1, c2);
    GBK_LAUNCH_CHECK();
  }
  return GBK_OK;
}

}  // extern "C"
