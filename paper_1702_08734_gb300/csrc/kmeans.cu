// Lloyd's k-means (the coarse quantizer q1 of Eq. (3) is "trained via k-means", section
// 2; section 6.2 runs the assignment as exact search with k = 1).
//
// Each iteration: assignment (tensor-core k-NN with k = 1, or direct float32 distances for
// the small sub-vectors of the product quantizer), then the update.  The update sums each
// cluster's members in double precision in increasing member index (stable bucketing gives
// that order), one thread per dimension, and rounds the mean to float32 once.  When there
// are few clusters for the GPU's size, each cluster's members are cut into S equal
// segments summed in parallel and the S partial sums are added in segment order: the
// double sum then differs from a sequential loop's by rounding far below float32's.  Empty clusters are re-seeded,
// in increasing index, by splitting the currently most populated cluster (lowest index on
// ties): c_e = c_s (1 + g/1024), c_s = c_s (1 - g/1024) with g = +1 on even and -1 on odd
// dimensions; its count is halved between the two.
#include <algorithm>

#include "common.cuh"
#include "ivf.cuh"
#include "knn.cuh"

namespace gbk {

namespace {

__global__ void gather_rows_kernel(const float* __restrict__ x, int ldx, int d,
                                   const int64_t* __restrict__ idx, int nc, float* __restrict__ out) {
  const int c = blockIdx.x;
  const int64_t r = idx[c];
  for (int t = threadIdx.x; t < d; t += blockDim.x) out[(int64_t)c * d + t] = x[r * ldx + t];
}

__global__ void to_i32_kernel(const int64_t* __restrict__ a, int64_t n, int32_t* __restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (int32_t)a[i];
}

// Member sums of cluster c = blockIdx.x over segment blockIdx.y of S equal parts of its
// members (in increasing member order, double precision, one thread per dimension, 8 rows
// in flight).  S == 1 writes the mean directly; otherwise the partial sums go to
// part[c][s][d] and update_combine_kernel adds them in segment order.
__global__ void update_partial_kernel(const float* __restrict__ x, int ldx, int d,
                                      const int64_t* __restrict__ offsets,
                                      const int64_t* __restrict__ order, int S,
                                      double* __restrict__ part, float* __restrict__ cent,
                                      long long* __restrict__ counts) {
  const int c = blockIdx.x, sg = blockIdx.y;
  const int64_t o0 = offsets[c], cnt = offsets[c + 1] - o0;
  if (sg == 0 && threadIdx.x == 0) counts[c] = cnt;
  const int64_t len = (cnt + S - 1) / S;
  const int64_t j0 = min(cnt, (int64_t)sg * len), j1 = min(cnt, j0 + len);
  const int64_t* ord = order + o0;
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    double acc = 0.0;
    int64_t j = j0;
    for (; j + 8 <= j1; j += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; u++) v[u] = __ldg(x + ord[j + u] * ldx + t);
#pragma unroll
      for (int u = 0; u < 8; u++) acc += (double)v[u];
    }
    for (; j < j1; j++) acc += (double)__ldg(x + ord[j] * ldx + t);
    if (S == 1) {
      if (cnt > 0) cent[(int64_t)c * d + t] = (float)(acc / (double)cnt);
    } else {
      part[((int64_t)c * S + sg) * d + t] = acc;
    }
  }
}

__global__ void update_combine_kernel(const double* __restrict__ part, int S, int d,
                                      const int64_t* __restrict__ offsets,
                                      float* __restrict__ cent) {
  const int c = blockIdx.x;
  const int64_t cnt = offsets[c + 1] - offsets[c];
  if (cnt == 0) return;
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    double acc = 0.0;
    for (int sg = 0; sg < S; sg++) acc += part[((int64_t)c * S + sg) * d + t];
    cent[(int64_t)c * d + t] = (float)(acc / (double)cnt);
  }
}

// Single block: re-seed empty clusters in increasing index order.
__global__ void __launch_bounds__(1024)
    empty_split_kernel(float* __restrict__ cent, int d, long long* __restrict__ counts, int nc,
                       long long* __restrict__ n_split) {
  __shared__ long long best_v[32];
  __shared__ int best_i[32];
  __shared__ int s_sel;
  __shared__ int e_cur;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long splits = 0;
  for (int base = 0; base < nc; base += blockDim.x) {
    // empties in this slice, handled one by one in index order
    const int e = base + tid;
    const bool empty = e < nc && counts[e] == 0;
    __syncthreads();
    unsigned any = __syncthreads_or(empty);
    if (!any) continue;
    for (int j = 0; j < (int)blockDim.x && base + j < nc; j++) {
      if (tid == 0) e_cur = counts[base + j] == 0 ? base + j : -1;
      __syncthreads();
      const int ec = e_cur;
      __syncthreads();  // everyone has read e_cur before thread 0 may rewrite it
      if (ec < 0) continue;
      // argmax of counts, lowest index on ties
      long long bv = -1;
      int bi = 0x7fffffff;
      for (int i = tid; i < nc; i += blockDim.x) {
        const long long v = counts[i];
        if (v > bv || (v == bv && i < bi)) {
          bv = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        best_v[warp] = bv;
        best_i[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        long long v = best_v[0];
        int ii = best_i[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++)
          if (best_v[w] > v || (best_v[w] == v && best_i[w] < ii)) {
            v = best_v[w];
            ii = best_i[w];
          }
        s_sel = ii;
      }
      __syncthreads();
      const int s = s_sel;
      for (int t = tid; t < d; t += blockDim.x) {
        const double g = (t % 2 == 0) ? 1.0 : -1.0;
        const double cs = (double)cent[(int64_t)s * d + t];
        cent[(int64_t)ec * d + t] = (float)(cs * (1.0 + g / 1024.0));
        cent[(int64_t)s * d + t] = (float)(cs * (1.0 - g / 1024.0));
      }
      __syncthreads();
      if (tid == 0) {
        counts[ec] = counts[s] / 2;
        counts[s] -= counts[ec];
      }
      splits++;
      __syncthreads();
    }
  }
  if (tid == 0 && n_split) *n_split += splits;
}

__global__ void sum_dist_kernel(const float* __restrict__ dist, int64_t n, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += (double)dist[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Direct float32 squared distances to at most 256 centroids of dimension <= 32.
__global__ void __launch_bounds__(256)
    assign_direct_kernel(const float* __restrict__ x, int64_t n, int ldx, int d,
                         const float* __restrict__ cent, int nc, int32_t* __restrict__ a,
                         float* __restrict__ dist) {
  __shared__ float C[256 * 32];
  for (int i = threadIdx.x; i < nc * d; i += blockDim.x) C[i] = cent[i];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xv[32];
#pragma unroll
  for (int t = 0; t < 32; t++) xv[t] = t < d ? x[i * ldx + t] : 0.f;
  float best = __int_as_float(0x7f800000);
  int bc = 0;
  for (int c = 0; c < nc; c++) {
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < 32; t++) {
      if (t < d) {
        const float e = xv[t] - C[c * d + t];
        s = fmaf(e, e, s);
      }
    }
    if (s < best) {
      best = s;
      bc = c;
    }
  }
  a[i] = bc;
  if (dist) dist[i] = best;
}

}  // namespace

gbk_status assign_direct_run(const float* x, int64_t n, int ldx, int d, const float* cent, int nc,
                             int32_t* a, float* dist, cudaStream_t st) {
  if (d > 32 || nc > 256) return set_error(GBK_EUNSUPPORTED, "direct assignment: d<=32, nc<=256");
  if (n == 0) return GBK_OK;
  ProfScope prof("assign_direct", st);
  assign_direct_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, ldx, d, cent, nc, a,
                                                                    dist);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status kmeans_run(const float* x, int64_t n, int d, int ldx, int nc, int niter,
                      const int64_t* init_idx, float* cent, double* objective, long long* n_split,
                      bool assign_direct, cudaStream_t st) {
  if (!assign_direct && ldx != d)
    return set_error(GBK_EINVAL, "k-means: tensor-core assignment needs contiguous rows");
  gbk_status r;
  Scratch a64, a32, dist, offs, order, counts;
  if ((r = a32.alloc(sizeof(int32_t) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = dist.alloc(sizeof(float) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = offs.alloc(sizeof(int64_t) * (size_t)(nc + 1), st)) != GBK_OK) return r;
  if ((r = order.alloc(sizeof(int64_t) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = counts.alloc(sizeof(long long) * (size_t)nc, st)) != GBK_OK) return r;
  if (!assign_direct && (r = a64.alloc(sizeof(int64_t) * (size_t)n, st)) != GBK_OK) return r;
  gather_rows_kernel<<<nc, 128, 0, st>>>(x, ldx, d, init_idx, nc, cent);
  GBK_LAUNCH_CHECK();
  if (objective) GBK_CUDA_CHECK(cudaMemsetAsync(objective, 0, sizeof(double) * (size_t)niter, st));
  if (n_split) GBK_CUDA_CHECK(cudaMemsetAsync(n_split, 0, sizeof(long long), st));
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_info().sm_count * 8);
  // update split: S segments per cluster when clusters are few and large (enough blocks to
  // fill the GPU), each segment at least 256 members
  const int64_t want = ((int64_t)device_info().sm_count * 16 + nc - 1) / nc;
  const int S = (int)std::max<int64_t>(1, std::min<int64_t>({want, 64, n / ((int64_t)nc * 256)}));
  Scratch part;
  if (S > 1 && (r = part.alloc(sizeof(double) * (size_t)nc * S * d, st)) != GBK_OK) return r;
  for (int it = 0; it < niter; it++) {
    if (assign_direct) {
      if ((r = assign_direct_run(x, n, ldx, d, cent, nc, a32.as<int32_t>(), dist.as<float>(), st)) !=
          GBK_OK)
        return r;
    } else {
      KnnPlan plan;
      if ((r = knn_run(x, n, cent, nc, d, 1, GBK_METRIC_L2, dist.as<float>(), a64.as<int64_t>(),
                       plan, st)) != GBK_OK)
        return r;
      to_i32_kernel<<<grid, 256, 0, st>>>(a64.as<int64_t>(), n, a32.as<int32_t>());
      GBK_LAUNCH_CHECK();
    }
    if (objective) {
      sum_dist_kernel<<<grid, 256, 0, st>>>(dist.as<float>(), n, objective + it);
      GBK_LAUNCH_CHECK();
    }
    if ((r = bucket_stable(a32.as<int32_t>(), n, nc, offs.as<int64_t>(), order.as<int64_t>(), st)) !=
        GBK_OK)
      return r;
    {
      ProfScope prof("kmeans_update", st);
      const int threads = std::min(1024, (d + 31) / 32 * 32);
      update_partial_kernel<<<dim3((unsigned)nc, (unsigned)S), threads, 0, st>>>(
          x, ldx, d, offs.as<int64_t>(), order.as<int64_t>(), S, part.as<double>(), cent,
          counts.as<long long>());
      if (S > 1)
        update_combine_kernel<<<nc, threads, 0, st>>>(part.as<double>(), S, d, offs.as<int64_t>(),
                                                      cent);
      empty_split_kernel<<<1, 1024, 0, st>>>(cent, d, counts.as<long long>(), nc, n_split);
      GBK_LAUNCH_CHECK();
    }
  }
  return GBK_OK;
}

}  // namespace gbk
