// Exact float32 re-rank of low-precision candidates, with a per-query certificate.
//
// The BF16 / FP8 distance GEMM selects k' >= k candidates per query; this kernel
// recomputes their distances directly (sum of (x_t - y_t)^2, or sum of x_t y_t) in
// float32, keeps the best k in the library's total order, and states for each query
// whether the result provably equals the float32 top-k:
//   every non-candidate y has a low-precision distance >= that of the k'-th candidate
//   (d'_k'), and |low(y) - exact(y)| <= eps_q, so exact(y) >= d'_k' - eps_q;  if
//   d'_k' - eps_q > (exact k-th distance) no non-candidate can enter the top k.
// eps_q bounds the inner-product error of the quantised operands: with x~ = x + e_x,
// |<x~,y~> - <x,y>| <= |e_x| |y~| + |x| |e_y| (Cauchy-Schwarz) plus float32 accumulation,
// using the largest database norm and quantisation error.  (Inner product: mirror image.)
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "ivf.cuh"
#include "knn.cuh"
#include "select_core.cuh"

namespace gbk {

namespace {

// Block per query: groups of 8 lanes take candidates (4 per warp, 2 such sets in flight),
// each lane summing every 8th float4 (or float) of the row; the group then butterfly-sums
// its partials.  Composites are then sorted in shared memory (bitonic, KP >= k').  v4:
// rows are 16-byte aligned float4 rows (d % 4 == 0, aligned base), checked by the host.
template <int KP>
__global__ void __launch_bounds__(256)
    rerank_kernel(const float* __restrict__ xq, const float* __restrict__ xb, int d, int kprime,
                  int k, int largest, const int64_t* __restrict__ Ic,
                  const float* __restrict__ Dc, const float* __restrict__ eps,
                  float* __restrict__ D, int64_t* __restrict__ I,
                  int32_t* __restrict__ certified, int all_candidates, int v4) {
  constexpr int U = 2;
  __shared__ uint64_t keys[KP];
  extern __shared__ __align__(16) float xs[];  // the query, d floats
  const int64_t q = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int grp = lane >> 3, sub = lane & 7;
  for (int t = threadIdx.x; t < d; t += blockDim.x) xs[t] = xq[q * d + t];
  for (int j = threadIdx.x; j < KP; j += blockDim.x) keys[j] = ~0ull;
  __syncthreads();
  for (int c0 = warp * 4 * U; c0 < kprime; c0 += nw * 4 * U) {
    int64_t id[U];
    float s[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int c = c0 + u * 4 + grp;
      id[u] = c < kprime ? Ic[q * kprime + c] : -1;
      s[u] = 0.f;
    }
    if (v4) {
      const int nf = d >> 2;
      const float4* y4 = reinterpret_cast<const float4*>(xb);
      for (int f = sub; f < nf; f += 8) {
        const float4 xv = reinterpret_cast<const float4*>(xs)[f];
        float4 yv[U];
#pragma unroll
        for (int u = 0; u < U; u++)
          yv[u] = id[u] >= 0 ? __ldg(y4 + id[u] * nf + f) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; u++) {
          if (largest) {
            s[u] = fmaf(xv.x, yv[u].x, s[u]);
            s[u] = fmaf(xv.y, yv[u].y, s[u]);
            s[u] = fmaf(xv.z, yv[u].z, s[u]);
            s[u] = fmaf(xv.w, yv[u].w, s[u]);
          } else {
            float e = xv.x - yv[u].x;
            s[u] = fmaf(e, e, s[u]);
            e = xv.y - yv[u].y;
            s[u] = fmaf(e, e, s[u]);
            e = xv.z - yv[u].z;
            s[u] = fmaf(e, e, s[u]);
            e = xv.w - yv[u].w;
            s[u] = fmaf(e, e, s[u]);
          }
        }
      }
    } else {
      for (int t = sub; t < d; t += 8) {
        const float xv = xs[t];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const float yv = id[u] >= 0 ? __ldg(xb + id[u] * d + t) : 0.f;
          if (largest) {
            s[u] = fmaf(xv, yv, s[u]);
          } else {
            const float e = xv - yv;
            s[u] = fmaf(e, e, s[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      s[u] += __shfl_xor_sync(FULL_MASK, s[u], 4);
      s[u] += __shfl_xor_sync(FULL_MASK, s[u], 2);
      s[u] += __shfl_xor_sync(FULL_MASK, s[u], 1);
      const int c = c0 + u * 4 + grp;
      if (sub == 0 && id[u] >= 0)
        keys[c] = composite(ordered_key(s[u], largest != 0), (uint32_t)id[u]);
    }
  }
  __syncthreads();
  for (int size = 2; size <= KP; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < KP / 2; t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        const uint64_t a = keys[lo], b = keys[hi];
        if ((a > b) == asc) {
          keys[lo] = b;
          keys[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const uint64_t e = keys[j];
    if (e == ~0ull) {
      D[q * k + j] = largest ? -INFINITY : INFINITY;
      I[q * k + j] = -1;
    } else {
      D[q * k + j] = key_value((uint32_t)(e >> 32), largest != 0);
      I[q * k + j] = (int64_t)(uint32_t)e;
    }
  }
  if (certified && threadIdx.x == 0) {
    int ok = all_candidates;
    const uint64_t ek = keys[k - 1];
    if (!ok && ek != ~0ull) {
      const float exact_k = key_value((uint32_t)(ek >> 32), largest != 0);
      const float low_kp = Dc[q * kprime + kprime - 1];
      const float e = eps[q];
      ok = largest ? (low_kp + e < exact_k) : (low_kp - e > exact_k);
    }
    certified[q] = ok;
  }
}

// eps_q for every query (see file comment).  ymax = max ||y||, yerr = max quantisation
// error norm over the database, u = unit roundoff of the format.
__global__ void rerank_eps_kernel(const float* __restrict__ xnorm2, const float* __restrict__ qscale,
                                  int64_t nq, int d, float u, float sub, const float* __restrict__ stats,
                                  int largest, float* __restrict__ eps) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float xn = sqrtf(xnorm2[q]);
  const float ymax = stats[0], yerr = stats[1];
  const float ex = u * xn + (qscale ? qscale[q] * sub * sqrtf((float)d) : 0.f);
  const float ip_err = ex * (ymax + yerr) + xn * yerr + (float)d * 1.2e-7f * xn * ymax;
  eps[q] = (largest ? 1.f : 2.f) * ip_err * 1.0001f + 1e-30f;
}

// stats[0] = max ||y||, stats[1] = max quantisation error bound of y (u ||y|| + s sub sqrt(d)).
__global__ void db_stats_kernel(const float* __restrict__ ynorm2, const float* __restrict__ bscale,
                                int64_t nb, int d, float u, float sub, float* __restrict__ stats) {
  float m0 = 0.f, m1 = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float yn = sqrtf(ynorm2[i]);
    m0 = fmaxf(m0, yn);
    m1 = fmaxf(m1, u * yn + (bscale ? bscale[i] * sub * sqrtf((float)d) : 0.f));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(FULL_MASK, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(FULL_MASK, m1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(reinterpret_cast<unsigned int*>(&stats[0]), __float_as_uint(m0));  // >= 0 floats
    atomicMax(reinterpret_cast<unsigned int*>(&stats[1]), __float_as_uint(m1));
  }
}

template <int KP>
gbk_status launch_rerank(const float* xq, const float* xb, int64_t nq, int d, int kprime, int k,
                         int largest, const int64_t* Ic, const float* Dc, const float* eps,
                         float* D, int64_t* I, int32_t* cert, int all, cudaStream_t st) {
  const int v4 = (d & 3) == 0 && (reinterpret_cast<uintptr_t>(xb) & 15) == 0;
  rerank_kernel<KP><<<(unsigned)nq, 256, sizeof(float) * (size_t)d, st>>>(
      xq, xb, d, kprime, k, largest, Ic, Dc, eps, D, I, cert, all, v4);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace

gbk_status rerank_run(const float* xq, const float* xb, int64_t nq, int64_t nb, int d,
                      int kprime, int k, bool largest, int prec, const float* xnorm2,
                      const float* qscale, const float* ynorm2, const float* bscale,
                      const int64_t* Ic, const float* Dc, float* D, int64_t* I,
                      int32_t* certified, float* eps_out, cudaStream_t st) {
  if (d > 8192) return set_error(GBK_EUNSUPPORTED, "re-rank supports d <= 8192");
  // unit roundoff of the format; `sub` = half the smallest subnormal step relative to scale
  const float u = prec == GBK_PREC_BF16 ? 0.00390625f /* 2^-8 */ : 0.0625f /* 2^-4 */;
  const float sub = prec == GBK_PREC_FP8 ? 0.0009765625f /* 2^-10 */ : 0.f;
  Scratch stats, eps;
  gbk_status r;
  if ((r = stats.alloc(2 * sizeof(float), st)) != GBK_OK) return r;
  float* epsp = eps_out;
  if (!epsp) {
    if ((r = eps.alloc(sizeof(float) * (size_t)nq, st)) != GBK_OK) return r;
    epsp = eps.as<float>();
  }
  GBK_CUDA_CHECK(cudaMemsetAsync(stats.p, 0, 2 * sizeof(float), st));
  db_stats_kernel<<<std::min<int64_t>(1024, (nb + 255) / 256), 256, 0, st>>>(
      ynorm2, prec == GBK_PREC_FP8 ? bscale : nullptr, nb, d, u, sub, stats.as<float>());
  GBK_LAUNCH_CHECK();
  rerank_eps_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(
      xnorm2, prec == GBK_PREC_FP8 ? qscale : nullptr, nq, d, u, sub, stats.as<float>(),
      largest ? 1 : 0, epsp);
  GBK_LAUNCH_CHECK();
  const int all = nb <= kprime ? 1 : 0;
  ProfScope prof("rerank", st);
  const int lg = largest ? 1 : 0;
  if (kprime <= 64)
    return launch_rerank<64>(xq, xb, nq, d, kprime, k, lg, Ic, Dc, epsp, D, I, certified, all, st);
  if (kprime <= 256)
    return launch_rerank<256>(xq, xb, nq, d, kprime, k, lg, Ic, Dc, epsp, D, I, certified, all, st);
  return launch_rerank<1024>(xq, xb, nq, d, kprime, k, lg, Ic, Dc, epsp, D, I, certified, all, st);
}

gbk_status rerank_rows_run(const float* xq, const float* xb, int64_t nq, int d, int kprime,
                           int k, const int64_t* rows, float* D, int64_t* I, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  if (d > 8192) return set_error(GBK_EUNSUPPORTED, "re-rank supports d <= 8192");
  ProfScope prof("rerank", st);
  if (kprime <= 64)
    return launch_rerank<64>(xq, xb, nq, d, kprime, k, 0, rows, nullptr, nullptr, D, I, nullptr, 0, st);
  if (kprime <= 256)
    return launch_rerank<256>(xq, xb, nq, d, kprime, k, 0, rows, nullptr, nullptr, D, I, nullptr, 0, st);
  return launch_rerank<1024>(xq, xb, nq, d, kprime, k, 0, rows, nullptr, nullptr, D, I, nullptr, 0, st);
}

}  // namespace gbk
