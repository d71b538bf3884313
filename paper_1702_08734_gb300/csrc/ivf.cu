// IVFADC index (section 2 "Compressed-domain search", section 5.2-5.3): coarse quantizer
// q1 trained by k-means, product quantizer q2 on the residuals, inverted lists stored as
// two arrays (codes, ids), and the batch search of Algorithm 4.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ivf.cuh"
#include "ivf_index.cuh"
#include "knn.cuh"

namespace gbk {

gbk_status ivf_scan_run(int M, int64_t nq, int nprobe, int k, const int64_t* cl_I,
                        const float* cl_D, const float* s1, const float* t3, const float* xq,
                        const float* coarse, const float* pq, int d, bool direct,
                        const int64_t* list_off, const uint8_t* codes, const int64_t* ids,
                        float* D, int64_t* I, cudaStream_t st, const int32_t* kq = nullptr,
                        const int32_t* npq = nullptr, const int64_t* out_off = nullptr,
                        const int64_t* order = nullptr, unsigned long long* counter = nullptr,
                        ScanTuning tun = ScanTuning());
gbk_status scan_cost_run(const int64_t* cl_I, int64_t nq, int nprobe, const int32_t* npq,
                         const int64_t* off, int32_t* key, cudaStream_t st);
gbk_status pq_encode_run(const float* x, int64_t n, int d, int M, const float* coarse,
                         const int32_t* lists, const float* pq, uint8_t* codes, cudaStream_t st);
gbk_status term1_run(const float* coarse, const float* pq, int nlist, int d, int M, float* T,
                     cudaStream_t st);
gbk_status term3_run(const float* xq, int64_t nq, const float* pq, int d, int M, float* t3,
                     cudaStream_t st);

namespace {

__global__ void residual_kernel(const float* __restrict__ x, int64_t n, int d,
                                const float* __restrict__ coarse, const int64_t* __restrict__ a,
                                float* __restrict__ r) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int t = (int)(e % d);
    r[e] = x[e] - coarse[a[i] * d + t];
  }
}

__global__ void stage_lists_kernel(const int64_t* __restrict__ a, int64_t n,
                                   int32_t* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (int32_t)a[i];
}

__global__ void stage_ids_kernel(const int64_t* __restrict__ ids, int64_t n, int64_t first,
                                 int64_t* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = ids ? ids[i] : first + i;
}

// codes/ids in list order: position j takes staged vector order[j]; its code is stored
// rotated by r = ((j - start of its list) mod 32) mod M (byte s = sub-quantizer (s + r) mod
// M, the layout the scan's conflict-free look-ups need: a lane knows its position modulo
// the warp width; for M <= 32, a divisor of 32, r is the position mod M) and, with the
// term-1 table T [nlist][256][M]
// given, s1[j] = sum_m T[L][code_m][m] is formed in sub-quantizer order.
__global__ void gather_codes_kernel(const uint8_t* __restrict__ in, const int64_t* __restrict__ order,
                                    int64_t n, int M, const int32_t* __restrict__ st_list,
                                    const int64_t* __restrict__ list_off,
                                    const float* __restrict__ T, uint8_t* __restrict__ out,
                                    float* __restrict__ s1, const int64_t* __restrict__ ids_in,
                                    int64_t* __restrict__ ids_out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t src = order[j];
    const int64_t L = st_list[src];
    const int r = (int)(((j - list_off[L]) & 31) % M);
    const uint8_t* c = in + src * M;
    for (int m = 0; m < M; m++) out[j * M + m] = c[(m + r) % M];
    if (T) {
      const float* TL = T + L * 256 * M;
      float acc = 0.f;
      for (int m = 0; m < M; m++) acc += TL[(int)c[m] * M + m];
      s1[j] = acc;
    }
    ids_out[j] = ids_in[src];
  }
}

// Inverse of the rotation above: out[j] = the code of position j in sub-quantizer order.
__global__ void unrotate_codes_kernel(const uint8_t* __restrict__ in, int64_t n, int M, int nlist,
                                      const int64_t* __restrict__ list_off,
                                      uint8_t* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nlist;  // list of position j: the last L with list_off[L] <= j
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (list_off[mid] <= j) lo = mid;
      else hi = mid;
    }
    const int r = (int)(((j - list_off[lo]) & 31) % M);
    for (int m = 0; m < M; m++) out[j * M + (m + r) % M] = in[j * M + m];
  }
}

int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256,
                                                     (int64_t)device_info().sm_count * 16));
}

}  // namespace

gbk_status finalize_index(gbk_index* ix, cudaStream_t st) {
  if (!ix->dirty) return GBK_OK;
  gbk_status r;
  const int64_t n = ix->n_staged;
  if ((r = ix->list_off.alloc(sizeof(int64_t) * (size_t)(ix->nlist + 1))) != GBK_OK) return r;
  if ((r = ix->codes.alloc((size_t)std::max<int64_t>(n, 1) * ix->M)) != GBK_OK) return r;
  if ((r = ix->ids.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1))) != GBK_OK) return r;
  Scratch order;
  if ((r = order.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1), st)) != GBK_OK) return r;
  if ((r = bucket_stable(ix->st_list.as<int32_t>(), n, ix->nlist, ix->list_off.as<int64_t>(),
                         order.as<int64_t>(), st)) != GBK_OK)
    return r;
  const bool tables = ix->use_precomputed && ix->T.p;
  if (tables && (r = ix->s1.alloc(sizeof(float) * (size_t)std::max<int64_t>(n, 1))) != GBK_OK)
    return r;
  if (n > 0) {
    gather_codes_kernel<<<grid_for(n), 256, 0, st>>>(
        ix->st_codes.as<uint8_t>(), order.as<int64_t>(), n, ix->M, ix->st_list.as<int32_t>(),
        ix->list_off.as<int64_t>(), tables ? ix->T.as<float>() : nullptr,
        ix->codes.as<uint8_t>(), tables ? ix->s1.as<float>() : nullptr,
        ix->st_ids.as<int64_t>(), ix->ids.as<int64_t>());
    GBK_LAUNCH_CHECK();
  }
  if (ix->keep_vectors) {
    if ((r = ix->vecs.alloc(sizeof(float) * (size_t)std::max<int64_t>(n, 1) * ix->d)) != GBK_OK)
      return r;
    if ((r = gather_rows_run(ix->st_vecs.as<float>(), order.as<int64_t>(), n, ix->d,
                             ix->vecs.as<float>(), st)) != GBK_OK)
      return r;
  }
  ix->ntotal = n;
  ix->dirty = false;
  return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_ivfpq_create(int32_t d, int32_t nlist, int32_t M, int32_t nbits, int32_t metric,
                            gbk_index** out) {
  clear_error();
  GBK_REQUIRE(out, "gbk_ivfpq_create: out is NULL");
  GBK_REQUIRE(d >= 1 && nlist >= 1 && nlist < (1 << 30), "gbk_ivfpq_create: bad d or nlist");
  GBK_REQUIRE(M >= 1 && d % M == 0, "gbk_ivfpq_create: M must divide d");
  if (nbits != 8) return set_error(GBK_EUNSUPPORTED, "gbk_ivfpq_create: only 8-bit codes");
  if (metric != GBK_METRIC_L2)
    return set_error(GBK_EUNSUPPORTED, "gbk_ivfpq_create: IVFADC is defined for L2 (Eq. 6)");
  if (M % 4 != 0 || M > 64)
    return set_error(GBK_EUNSUPPORTED, "gbk_ivfpq_create: M must be a multiple of 4 up to 64");
  if (d / M > 32) return set_error(GBK_EUNSUPPORTED, "gbk_ivfpq_create: d/M must be <= 32");
  gbk_index* ix = new gbk_index();
  ix->d = d;
  ix->nlist = nlist;
  ix->M = M;
  ix->dsub = d / M;
  *out = ix;
  return GBK_OK;
}

void gbk_ivfpq_destroy(gbk_index* ix) { delete ix; }

gbk_status gbk_ivfpq_train(gbk_index* ix, const float* x_in, int64_t n,
                           const gbk_train_opts* opts, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && x_in, "gbk_ivfpq_train: NULL argument");
  GBK_REQUIRE(n >= ix->nlist && n >= 256 && n < (int64_t(1) << 31),
              "gbk_ivfpq_train: need max(nlist, 256) <= n < 2^31 training vectors");
  cudaStream_t st = as_stream(stream);
  const int niter = opts && opts->niter > 0 ? opts->niter : 20;
  const int pq_niter = opts && opts->pq_niter > 0 ? opts->pq_niter : niter;
  std::vector<int64_t> cinit(ix->nlist), pinit(256);
  for (int i = 0; i < ix->nlist; i++) cinit[i] = opts && opts->coarse_init ? opts->coarse_init[i] : i;
  for (int i = 0; i < 256; i++) pinit[i] = opts && opts->pq_init ? opts->pq_init[i] : i;
  for (int64_t v : cinit) GBK_REQUIRE(v >= 0 && v < n, "gbk_ivfpq_train: coarse_init out of range");
  for (int64_t v : pinit) GBK_REQUIRE(v >= 0 && v < n, "gbk_ivfpq_train: pq_init out of range");
  if (opts) ix->use_precomputed = opts->use_precomputed;
  gbk_status r;
  Scratch xr;
  const float* x = x_in;
  if ((r = rotate_rows(ix, x_in, n, xr, &x, st)) != GBK_OK) return r;
  const int d = ix->d, M = ix->M, dsub = ix->dsub;
  if ((r = ix->coarse.alloc(sizeof(float) * (size_t)ix->nlist * d)) != GBK_OK) return r;
  if ((r = ix->pq.alloc(sizeof(float) * (size_t)M * 256 * dsub)) != GBK_OK) return r;
  Scratch ci, pi, a, dist, res, sub;
  if ((r = ci.alloc(sizeof(int64_t) * ix->nlist, st)) != GBK_OK) return r;
  if ((r = pi.alloc(sizeof(int64_t) * 256, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ci.p, cinit.data(), sizeof(int64_t) * ix->nlist,
                                 cudaMemcpyHostToDevice, st));
  GBK_CUDA_CHECK(cudaMemcpyAsync(pi.p, pinit.data(), sizeof(int64_t) * 256, cudaMemcpyHostToDevice,
                                 st));
  // coarse quantizer q1 (Eq. 3) by k-means, assignment on the tensor cores
  if ((r = kmeans_run(x, n, d, d, ix->nlist, niter, ci.as<int64_t>(), ix->coarse.as<float>(),
                      nullptr, nullptr, false, st)) != GBK_OK)
    return r;
  // residuals y - q1(y)
  if ((r = a.alloc(sizeof(int64_t) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = dist.alloc(sizeof(float) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = res.alloc(sizeof(float) * (size_t)n * d, st)) != GBK_OK) return r;
  KnnPlan plan;
  if ((r = knn_run(x, n, ix->coarse.as<float>(), ix->nlist, d, 1, GBK_METRIC_L2, dist.as<float>(),
                   a.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  residual_kernel<<<grid_for(n * d), 256, 0, st>>>(x, n, d, ix->coarse.as<float>(),
                                                    a.as<int64_t>(), res.as<float>());
  GBK_LAUNCH_CHECK();
  // product quantizer: 256-centroid k-means per sub-vector block (section 2)
  for (int m = 0; m < M; m++) {
    if ((r = kmeans_run(res.as<float>() + m * dsub, n, dsub, d, 256, pq_niter, pi.as<int64_t>(),
                        ix->pq.as<float>() + (size_t)m * 256 * dsub, nullptr, nullptr, true,
                        st)) != GBK_OK)
      return r;
  }
  // term-1 table (Eq. 11)
  if (ix->use_precomputed) {
    if ((r = ix->T.alloc(sizeof(float) * (size_t)ix->nlist * M * 256)) != GBK_OK) return r;
    if ((r = term1_run(ix->coarse.as<float>(), ix->pq.as<float>(), ix->nlist, d, M,
                       ix->T.as<float>(), st)) != GBK_OK)
      return r;
  }
  ix->trained = true;
  ix->dirty = true;
  return GBK_OK;
}

gbk_status gbk_ivfpq_set_quantizers(gbk_index* ix, const float* coarse, const float* pq,
                                    int32_t use_precomputed, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && coarse && pq, "gbk_ivfpq_set_quantizers: NULL argument");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  const size_t cb = sizeof(float) * (size_t)ix->nlist * ix->d;
  const size_t pb = sizeof(float) * (size_t)ix->M * 256 * ix->dsub;
  if ((r = ix->coarse.alloc(cb)) != GBK_OK) return r;
  if ((r = ix->pq.alloc(pb)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ix->coarse.p, coarse, cb, cudaMemcpyDefault, st));
  GBK_CUDA_CHECK(cudaMemcpyAsync(ix->pq.p, pq, pb, cudaMemcpyDefault, st));
  ix->use_precomputed = use_precomputed;
  if (use_precomputed) {
    if ((r = ix->T.alloc(sizeof(float) * (size_t)ix->nlist * ix->M * 256)) != GBK_OK) return r;
    if ((r = term1_run(ix->coarse.as<float>(), ix->pq.as<float>(), ix->nlist, ix->d, ix->M,
                       ix->T.as<float>(), st)) != GBK_OK)
      return r;
  }
  ix->trained = true;
  ix->dirty = true;
  return GBK_OK;
}

gbk_status gbk_ivfpq_add(gbk_index* ix, const float* x_in, int64_t n, const int64_t* ids,
                         void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_add: NULL index");
  GBK_REQUIRE(ix->trained, "gbk_ivfpq_add: index not trained");
  GBK_REQUIRE(n >= 0, "gbk_ivfpq_add: n < 0");
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x_in, "gbk_ivfpq_add: NULL x");
  GBK_REQUIRE(ix->n_staged + n <= (int64_t(1) << 32) - (int64_t(1) << 16),
              "gbk_ivfpq_add: index full (2^32 - 2^16 vectors)");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  Scratch xr;
  const float* x = x_in;
  if ((r = rotate_rows(ix, x_in, n, xr, &x, st)) != GBK_OK) return r;
  const int64_t need = ix->n_staged + n;
  if (need > ix->cap_staged) {
    int64_t cap = std::max<int64_t>(need, ix->cap_staged * 2);
    const size_t keep = (size_t)ix->n_staged;
    if ((r = ix->st_list.grow(sizeof(int32_t) * cap, sizeof(int32_t) * keep, st)) != GBK_OK) return r;
    if ((r = ix->st_codes.grow((size_t)cap * ix->M, keep * ix->M, st)) != GBK_OK) return r;
    if ((r = ix->st_ids.grow(sizeof(int64_t) * cap, sizeof(int64_t) * keep, st)) != GBK_OK) return r;
    if (ix->keep_vectors &&
        (r = ix->st_vecs.grow(sizeof(float) * ix->d * cap, sizeof(float) * ix->d * keep, st)) !=
            GBK_OK)
      return r;
    ix->cap_staged = cap;
  }
  if (ix->keep_vectors)
    GBK_CUDA_CHECK(cudaMemcpyAsync(ix->st_vecs.as<float>() + (size_t)ix->n_staged * ix->d, x,
                                   sizeof(float) * ix->d * (size_t)n, cudaMemcpyDeviceToDevice, st));
  Scratch a, dist;
  if ((r = a.alloc(sizeof(int64_t) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = dist.alloc(sizeof(float) * (size_t)n, st)) != GBK_OK) return r;
  KnnPlan plan;
  // q1(y): nearest coarse centroid (exact, k = 1)
  if ((r = knn_run(x, n, ix->coarse.as<float>(), ix->nlist, ix->d, 1, GBK_METRIC_L2,
                   dist.as<float>(), a.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  int32_t* lists = ix->st_list.as<int32_t>() + ix->n_staged;
  stage_lists_kernel<<<grid_for(n), 256, 0, st>>>(a.as<int64_t>(), n, lists);
  stage_ids_kernel<<<grid_for(n), 256, 0, st>>>(ids, n, ix->n_staged,
                                                ix->st_ids.as<int64_t>() + ix->n_staged);
  GBK_LAUNCH_CHECK();
  if ((r = pq_encode_run(x, n, ix->d, ix->M, ix->coarse.as<float>(), lists, ix->pq.as<float>(),
                         ix->st_codes.as<uint8_t>() + (size_t)ix->n_staged * ix->M, st)) != GBK_OK)
    return r;
  ix->n_staged += n;
  ix->dirty = true;
  return GBK_OK;
}

gbk_status gbk_ivfpq_search(gbk_index* ix, const float* xq, int64_t nq, int32_t k, int32_t nprobe,
                            float* D, int64_t* I, void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_search: NULL index");
  GBK_REQUIRE(ix->trained, "gbk_ivfpq_search: index not trained");
  GBK_REQUIRE(k >= 1 && k <= GBK_MAX_K, "gbk_ivfpq_search: k out of [1, %d]", GBK_MAX_K);
  GBK_REQUIRE(nprobe >= 1 && nprobe <= ix->nlist && nprobe <= GBK_MAX_K,
              "gbk_ivfpq_search: nprobe out of [1, min(nlist, %d)]", GBK_MAX_K);
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "gbk_ivfpq_search: nq out of range");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && D && I, "gbk_ivfpq_search: NULL pointer");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  return gbk::search_run(ix, xq, nq, k, nprobe, D, I, st);
}

gbk_status gbk_ivfpq_set_coarse_precision(gbk_index* ix, int32_t precision) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_set_coarse_precision: NULL index");
  GBK_REQUIRE(precision == GBK_PREC_FP32 || precision == GBK_PREC_BF16 ||
                  precision == GBK_PREC_FP8 || precision == GBK_PREC_TF32X3,
              "gbk_ivfpq_set_coarse_precision: bad precision");
  ix->coarse_prec = precision;
  return GBK_OK;
}

gbk_status gbk_ivfpq_set_learned_route(gbk_index* ix, float alpha, int32_t shift) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_set_learned_route: NULL index");
  GBK_REQUIRE(shift >= -16 && shift <= 16, "gbk_ivfpq_set_learned_route: shift out of [-16, 16]");
  GBK_REQUIRE(alpha >= 0.f && alpha <= 1.f, "gbk_ivfpq_set_learned_route: alpha out of [0, 1]");
  ix->class_shift = shift;
  ix->route_alpha = alpha;
  return GBK_OK;
}

gbk_status gbk_ivfpq_keep_vectors(gbk_index* ix, int32_t keep) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_keep_vectors: NULL index");
  GBK_REQUIRE(ix->n_staged == 0 || (keep != 0) == ix->keep_vectors,
              "gbk_ivfpq_keep_vectors: must be set before the first add");
  ix->keep_vectors = keep != 0;
  return GBK_OK;
}

gbk_status gbk_ivfpq_set_rotation(gbk_index* ix, const float* R, void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_set_rotation: NULL index");
  GBK_REQUIRE(!ix->trained && ix->n_staged == 0,
              "gbk_ivfpq_set_rotation: must be set before training and adding");
  if (!R) {
    ix->rot.release();
    ix->rotated = false;
    return GBK_OK;
  }
  gbk_status r;
  const size_t b = sizeof(float) * (size_t)ix->d * ix->d;
  if ((r = ix->rot.alloc(b)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ix->rot.p, R, b, cudaMemcpyDefault, as_stream(stream)));
  ix->rotated = true;
  return GBK_OK;
}

gbk_status gbk_ivfpq_rotate(gbk_index* ix, const float* x, int64_t n, float* out, void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_rotate: NULL index");
  GBK_REQUIRE(n >= 0 && n < (int64_t(1) << 31), "gbk_ivfpq_rotate: n out of range");
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x && out, "gbk_ivfpq_rotate: NULL pointer");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  Scratch xr;
  const float* y = x;
  if ((r = rotate_rows(ix, x, n, xr, &y, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(out, y, sizeof(float) * (size_t)n * ix->d,
                                 cudaMemcpyDeviceToDevice, st));
  return GBK_OK;
}

gbk_status gbk_ivfpq_search_refine(gbk_index* ix, const float* xq, int64_t nq, int32_t k,
                                   int32_t nprobe, int32_t kprime, float* D, int64_t* I,
                                   void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_search_refine: NULL index");
  GBK_REQUIRE(ix->trained, "gbk_ivfpq_search_refine: index not trained");
  GBK_REQUIRE(ix->keep_vectors,
              "gbk_ivfpq_search_refine: the index keeps no vectors (gbk_ivfpq_keep_vectors)");
  GBK_REQUIRE(k >= 1 && kprime >= k && kprime <= GBK_MAX_K,
              "gbk_ivfpq_search_refine: need 1 <= k <= kprime <= %d", GBK_MAX_K);
  GBK_REQUIRE(nprobe >= 1 && nprobe <= ix->nlist && nprobe <= GBK_MAX_K,
              "gbk_ivfpq_search_refine: nprobe out of [1, min(nlist, %d)]", GBK_MAX_K);
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "gbk_ivfpq_search_refine: nq out of range");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && D && I, "gbk_ivfpq_search_refine: NULL pointer");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  Scratch Dc, Ic;
  if ((r = Dc.alloc(sizeof(float) * (size_t)nq * kprime, st)) != GBK_OK) return r;
  if ((r = Ic.alloc(sizeof(int64_t) * (size_t)nq * kprime, st)) != GBK_OK) return r;
  // k' ADC candidates as list positions, exact distances from the stored vectors, top k
  Scratch xr;
  const float* xqr = xq;
  if ((r = rotate_rows(ix, xq, nq, xr, &xqr, st)) != GBK_OK) return r;
  if ((r = gbk::search_run(ix, xqr, nq, kprime, nprobe, Dc.as<float>(), Ic.as<int64_t>(), st,
                           true, true)) != GBK_OK)
    return r;
  if ((r = rerank_rows_run(xqr, ix->vecs.as<float>(), nq, ix->d, kprime, k, Ic.as<int64_t>(), D,
                           I, st)) != GBK_OK)
    return r;
  return rows_to_ids_run(I, nq * (int64_t)k, ix->ids.as<int64_t>(), st);
}

}  // extern "C"

namespace gbk {
// Algorithm 4 for a validated, finalized index.
gbk_status rotate_rows(const gbk_index* ix, const float* x, int64_t n, Scratch& buf,
                       const float** out, cudaStream_t st) {
  if (!ix->rotated || n == 0) {
    *out = x;
    return GBK_OK;
  }
  gbk_status r;
  const int d = ix->d;
  if ((r = buf.alloc(sizeof(float) * (size_t)n * d, st)) != GBK_OK) return r;
  PreparedOperand Rp;
  if ((r = prepare_operand(ix->rot.as<float>(), d, d, GBK_PREC_FP32, (d + 127) / 128 * 128, 0.f,
                           &Rp, st)) != GBK_OK)
    return r;
  const int64_t CH = int64_t(1) << 20;
  for (int64_t r0 = 0; r0 < n; r0 += CH) {
    const int64_t c = std::min(CH, n - r0);
    PreparedOperand Q;
    if ((r = prepare_operand(x + r0 * d, c, d, GBK_PREC_FP32, c, 0.f, &Q, st)) != GBK_OK) return r;
    if ((r = pairwise_run(Q, Rp, true, buf.as<float>() + r0 * d, d, st)) != GBK_OK) return r;
  }
  *out = buf.as<float>();
  return GBK_OK;
}

// key[q] = the nearest probed list of query q (0 when it has none)
__global__ void first_list_kernel(const int64_t* __restrict__ cl_I, int64_t nq, int nprobe,
                                  int32_t* __restrict__ key) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) key[q] = (int32_t)max(cl_I[q * nprobe], (int64_t)0);
}

gbk_status search_run(gbk_index* ix, const float* xq_in, int64_t nq, int k, int nprobe, float* D,
                      int64_t* I, cudaStream_t st, bool positions, bool prerotated) {
  gbk_status r;
  Scratch clD, clI, t3, xr;
  const float* xq = xq_in;
  if (!prerotated && (r = rotate_rows(ix, xq_in, nq, xr, &xq, st)) != GBK_OK) return r;
  if ((r = clD.alloc(sizeof(float) * (size_t)nq * nprobe, st)) != GBK_OK) return r;
  if ((r = clI.alloc(sizeof(int64_t) * (size_t)nq * nprobe, st)) != GBK_OK) return r;
  // L_IVF (Eq. 5): the nprobe nearest coarse centroids, with term 2 = ||x - c||^2
  KnnPlan plan;
  plan.prec = ix->coarse_prec;
  if ((r = knn_run(xq, nq, ix->coarse.as<float>(), ix->nlist, ix->d, nprobe, GBK_METRIC_L2,
                   clD.as<float>(), clI.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  const bool direct = !ix->use_precomputed;
  if (!direct) {
    if ((r = t3.alloc(sizeof(float) * (size_t)nq * ix->M * 256, st)) != GBK_OK) return r;
    if ((r = term3_run(xq, nq, ix->pq.as<float>(), ix->d, ix->M, t3.as<float>(), st)) != GBK_OK)
      return r;
  }
  // queries taken in the order of their nearest list, so that queries probing the same
  // lists run at the same time and share those lists' codes in L2
  Scratch key, order, offs, counter;
  const bool by_list = ix->tuning.list_order && nq > 1;
  if (by_list) {
    if ((r = key.alloc(sizeof(int32_t) * (size_t)nq, st)) != GBK_OK) return r;
    if ((r = order.alloc(sizeof(int64_t) * (size_t)nq, st)) != GBK_OK) return r;
    if ((r = offs.alloc(sizeof(int64_t) * (size_t)(ix->nlist + 1), st)) != GBK_OK) return r;
    if ((r = counter.alloc(sizeof(unsigned long long), st)) != GBK_OK) return r;
    first_list_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(clI.as<int64_t>(), nq, nprobe,
                                                                     key.as<int32_t>());
    GBK_LAUNCH_CHECK();
    if ((r = bucket_stable(key.as<int32_t>(), nq, ix->nlist, offs.as<int64_t>(),
                           order.as<int64_t>(), st)) != GBK_OK)
      return r;
    GBK_CUDA_CHECK(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), st));
  }
  return ivf_scan_run(ix->M, nq, nprobe, k, clI.as<int64_t>(), clD.as<float>(), ix->s1.as<float>(),
                      t3.as<float>(), xq, ix->coarse.as<float>(), ix->pq.as<float>(), ix->d,
                      direct, ix->list_off.as<int64_t>(), ix->codes.as<uint8_t>(),
                      positions ? nullptr : ix->ids.as<int64_t>(), D, I, st, nullptr, nullptr,
                      nullptr, by_list ? order.as<int64_t>() : nullptr,
                      by_list ? counter.as<unsigned long long>() : nullptr, ix->tuning);
}
}  // namespace gbk
extern "C" {

gbk_status gbk_ivfpq_info(gbk_index* ix, int64_t* ntotal, int32_t* nlist, int32_t* d, int32_t* M,
                          void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_info: NULL index");
  gbk_status r;
  if (ix->trained && (r = finalize_index(ix, as_stream(stream))) != GBK_OK) return r;
  if (ntotal) *ntotal = ix->n_staged;
  if (nlist) *nlist = ix->nlist;
  if (d) *d = ix->d;
  if (M) *M = ix->M;
  return GBK_OK;
}

gbk_status gbk_ivfpq_export(gbk_index* ix, float* coarse, float* pq, int64_t* list_off,
                            uint8_t* codes, int64_t* ids, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained, "gbk_ivfpq_export: index missing or not trained");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  if (coarse)
    GBK_CUDA_CHECK(cudaMemcpyAsync(coarse, ix->coarse.p, ix->coarse.bytes, cudaMemcpyDefault, st));
  if (pq) GBK_CUDA_CHECK(cudaMemcpyAsync(pq, ix->pq.p, ix->pq.bytes, cudaMemcpyDefault, st));
  if (list_off)
    GBK_CUDA_CHECK(cudaMemcpyAsync(list_off, ix->list_off.p, sizeof(int64_t) * (ix->nlist + 1),
                                   cudaMemcpyDefault, st));
  if (codes && ix->ntotal) {
    Scratch plain;
    if ((r = plain.alloc((size_t)ix->ntotal * ix->M, st)) != GBK_OK) return r;
    unrotate_codes_kernel<<<grid_for(ix->ntotal), 256, 0, st>>>(
        ix->codes.as<uint8_t>(), ix->ntotal, ix->M, ix->nlist, ix->list_off.as<int64_t>(),
        plain.as<uint8_t>());
    GBK_LAUNCH_CHECK();
    GBK_CUDA_CHECK(cudaMemcpyAsync(codes, plain.p, (size_t)ix->ntotal * ix->M, cudaMemcpyDefault,
                                   st));
  }
  if (ids && ix->ntotal)
    GBK_CUDA_CHECK(cudaMemcpyAsync(ids, ix->ids.p, sizeof(int64_t) * ix->ntotal, cudaMemcpyDefault,
                                   st));
  return GBK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ save / load

namespace gbk {
namespace {

// File layout (little-endian): this header, then coarse f32 [nlist][d], pq f32 [M][256][d/M],
// the rotation f32 [d][d] when `rotated`, list_off i64 [nlist+1], codes u8 [ntotal][M]
// (sub-quantizer m in byte m), ids i64 [ntotal], and the kept vectors f32 [ntotal][d] when
// `keep_vectors`.  Term-1 tables and sums, the rotated code layout and the staging arrays
// are rebuilt on load from these, by the same kernels, so a loaded index searches exactly
// as the saved one did.
struct FileHeader {
  char magic[8];
  uint32_t version;
  int32_t d, nlist, M, nbits, use_precomputed, coarse_prec, keep_vectors, rotated;
  int32_t codes_per_thread, blocks_per_sm, list_order, scan_threads, class_shift;
  float route_alpha;
  int64_t ntotal;
  int64_t reserved[4];
};
constexpr char kMagic[8] = {'G', 'B', 'K', 'I', 'V', 'F', 'P', 'Q'};

struct File {
  std::FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

gbk_status write_block(std::FILE* f, const void* dev, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return GBK_OK;
  std::vector<unsigned char> h(bytes);
  GBK_CUDA_CHECK(cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, st));
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (std::fwrite(h.data(), 1, bytes, f) != bytes)
    return set_error(GBK_EINVAL, "gbk_ivfpq_save: write failed");
  return GBK_OK;
}

gbk_status read_block(std::FILE* f, DevBuf& dst, size_t bytes, cudaStream_t st) {
  gbk_status r;
  if ((r = dst.alloc(std::max<size_t>(bytes, 1))) != GBK_OK) return r;
  if (bytes == 0) return GBK_OK;
  std::vector<unsigned char> h(bytes);
  if (std::fread(h.data(), 1, bytes, f) != bytes)
    return set_error(GBK_EINVAL, "gbk_ivfpq_load: file truncated");
  GBK_CUDA_CHECK(cudaMemcpyAsync(dst.p, h.data(), bytes, cudaMemcpyHostToDevice, st));
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  return GBK_OK;
}

// staged list of position j = the list whose range holds j (list-ordered input)
__global__ void lists_of_positions_kernel(const int64_t* __restrict__ off, int nlist, int64_t n,
                                          int32_t* __restrict__ lst) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nlist;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (off[mid] <= j) lo = mid;
      else hi = mid;
    }
    lst[j] = lo;
  }
}

}  // namespace
}  // namespace gbk

extern "C" {

gbk_status gbk_ivfpq_save(gbk_index* ix, const char* path, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained && path, "gbk_ivfpq_save: index missing, not trained, or no path");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  File file;
  file.f = std::fopen(path, "wb");
  if (!file.f) return set_error(GBK_EINVAL, "gbk_ivfpq_save: cannot open %s", path);
  FileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.version = 1;
  h.d = ix->d;
  h.nlist = ix->nlist;
  h.M = ix->M;
  h.nbits = 8;
  h.use_precomputed = ix->use_precomputed;
  h.coarse_prec = ix->coarse_prec;
  h.keep_vectors = ix->keep_vectors ? 1 : 0;
  h.rotated = ix->rotated ? 1 : 0;
  h.codes_per_thread = ix->tuning.codes_per_thread;
  h.blocks_per_sm = ix->tuning.blocks_per_sm;
  h.list_order = ix->tuning.list_order;
  h.scan_threads = ix->tuning.threads;
  h.class_shift = ix->class_shift;
  h.route_alpha = ix->route_alpha;
  h.ntotal = ix->ntotal;
  if (std::fwrite(&h, sizeof(h), 1, file.f) != 1)
    return set_error(GBK_EINVAL, "gbk_ivfpq_save: write failed");
  const size_t n = (size_t)ix->ntotal;
  if ((r = write_block(file.f, ix->coarse.p, sizeof(float) * (size_t)ix->nlist * ix->d, st)) ||
      (r = write_block(file.f, ix->pq.p, sizeof(float) * (size_t)ix->M * 256 * ix->dsub, st)) ||
      (ix->rotated && (r = write_block(file.f, ix->rot.p, sizeof(float) * (size_t)ix->d * ix->d, st))) ||
      (r = write_block(file.f, ix->list_off.p, sizeof(int64_t) * (size_t)(ix->nlist + 1), st)))
    return r;
  if (n) {
    Scratch plain;
    if ((r = plain.alloc(n * ix->M, st)) != GBK_OK) return r;
    unrotate_codes_kernel<<<grid_for((int64_t)n), 256, 0, st>>>(
        ix->codes.as<uint8_t>(), (int64_t)n, ix->M, ix->nlist, ix->list_off.as<int64_t>(),
        plain.as<uint8_t>());
    GBK_LAUNCH_CHECK();
    if ((r = write_block(file.f, plain.p, n * ix->M, st)) ||
        (r = write_block(file.f, ix->ids.p, sizeof(int64_t) * n, st)) ||
        (ix->keep_vectors && (r = write_block(file.f, ix->vecs.p, sizeof(float) * n * ix->d, st))))
      return r;
  }
  if (std::fflush(file.f) != 0) return set_error(GBK_EINVAL, "gbk_ivfpq_save: write failed");
  return GBK_OK;
}

gbk_status gbk_ivfpq_load(const char* path, gbk_index** out, void* stream) {
  clear_error();
  GBK_REQUIRE(path && out, "gbk_ivfpq_load: NULL argument");
  cudaStream_t st = as_stream(stream);
  File file;
  file.f = std::fopen(path, "rb");
  if (!file.f) return set_error(GBK_EINVAL, "gbk_ivfpq_load: cannot open %s", path);
  FileHeader h;
  if (std::fread(&h, sizeof(h), 1, file.f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0 ||
      h.version != 1)
    return set_error(GBK_EINVAL, "gbk_ivfpq_load: %s is not a gbknn IVFPQ file (version 1)", path);
  gbk_index* ix = nullptr;
  gbk_status r = gbk_ivfpq_create(h.d, h.nlist, h.M, h.nbits, GBK_METRIC_L2, &ix);
  if (r != GBK_OK) return r;
  struct Guard {
    gbk_index* p;
    ~Guard() { delete p; }
  } guard{ix};
  GBK_REQUIRE(h.ntotal >= 0 && h.ntotal <= (int64_t(1) << 32) - (int64_t(1) << 16),
              "gbk_ivfpq_load: bad vector count");
  GBK_REQUIRE(h.coarse_prec >= GBK_PREC_FP32 && h.coarse_prec <= GBK_PREC_TF32X3 &&
                  (h.codes_per_thread == 2 || h.codes_per_thread == 4 || h.codes_per_thread == 8) &&
                  h.blocks_per_sm >= 1 && h.blocks_per_sm <= 8 &&
                  (h.scan_threads == 256 || h.scan_threads == 384 || h.scan_threads == 512) &&
                  h.class_shift >= -16 && h.class_shift <= 16 && h.route_alpha >= 0.f &&
                  h.route_alpha <= 1.f,
              "gbk_ivfpq_load: bad settings in the header");
  const int64_t n = h.ntotal;
  ix->use_precomputed = h.use_precomputed ? 1 : 0;
  ix->coarse_prec = h.coarse_prec;
  ix->keep_vectors = h.keep_vectors != 0;
  ix->tuning.codes_per_thread = h.codes_per_thread;
  ix->tuning.blocks_per_sm = h.blocks_per_sm;
  ix->tuning.list_order = h.list_order ? 1 : 0;
  ix->tuning.threads = h.scan_threads;
  ix->class_shift = h.class_shift;
  ix->route_alpha = h.route_alpha;
  DevBuf off;
  if ((r = read_block(file.f, ix->coarse, sizeof(float) * (size_t)h.nlist * h.d, st)) ||
      (r = read_block(file.f, ix->pq, sizeof(float) * (size_t)h.M * 256 * (h.d / h.M), st)) ||
      (h.rotated && (r = read_block(file.f, ix->rot, sizeof(float) * (size_t)h.d * h.d, st))) ||
      (r = read_block(file.f, off, sizeof(int64_t) * (size_t)(h.nlist + 1), st))) {
    off.release();
    return r;
  }
  ix->rotated = h.rotated != 0;
  std::vector<int64_t> offh(h.nlist + 1);
  if (cudaMemcpy(offh.data(), off.p, sizeof(int64_t) * offh.size(), cudaMemcpyDeviceToHost) !=
      cudaSuccess) {
    off.release();
    return set_error(GBK_ECUDA, "gbk_ivfpq_load: copy failed");
  }
  bool ok = offh[0] == 0 && offh[h.nlist] == n;
  for (int L = 0; L < h.nlist && ok; L++) ok = offh[L] <= offh[L + 1];
  if (!ok) {
    off.release();
    return set_error(GBK_EINVAL, "gbk_ivfpq_load: inconsistent list offsets");
  }
  // the lists become the staging arrays (insertion order = list order), rebuilt at first use
  if ((r = read_block(file.f, ix->st_codes, (size_t)n * h.M, st)) ||
      (r = read_block(file.f, ix->st_ids, sizeof(int64_t) * (size_t)n, st)) ||
      (ix->keep_vectors &&
       (r = read_block(file.f, ix->st_vecs, sizeof(float) * (size_t)n * h.d, st)))) {
    off.release();
    return r;
  }
  if ((r = ix->st_list.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1))) != GBK_OK) {
    off.release();
    return r;
  }
  if (n > 0) {
    lists_of_positions_kernel<<<grid_for(n), 256, 0, st>>>(off.as<int64_t>(), h.nlist, n,
                                                           ix->st_list.as<int32_t>());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      off.release();
      return set_error(GBK_ECUDA, "gbk_ivfpq_load: launch: %s", cudaGetErrorString(e));
    }
  }
  off.release();
  ix->n_staged = ix->cap_staged = n;
  if (ix->use_precomputed) {
    if ((r = ix->T.alloc(sizeof(float) * (size_t)ix->nlist * ix->M * 256)) != GBK_OK) return r;
    if ((r = term1_run(ix->coarse.as<float>(), ix->pq.as<float>(), ix->nlist, ix->d, ix->M,
                       ix->T.as<float>(), st)) != GBK_OK)
      return r;
  }
  ix->trained = true;
  ix->dirty = true;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  guard.p = nullptr;
  *out = ix;
  return GBK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ mixed batches

namespace gbk {
namespace {

// F[q] = [x_q, d_i / max(d_0, 1e-12) - 1 for the nfeat nearest coarse distances d_i]
__global__ void nprobe_features_kernel(const float* __restrict__ xq, int64_t nq, int d,
                                       const float* __restrict__ clD, int tau, int nfeat,
                                       float* __restrict__ F) {
  const int64_t q = blockIdx.x;
  const int nf = d + nfeat;
  const float d0 = fmaxf(clD[q * tau], 1e-12f);
  for (int t = threadIdx.x; t < nf; t += blockDim.x)
    F[q * nf + t] = t < d ? xq[q * d + t] : clD[q * tau + (t - d)] / d0 - 1.f;
}

// nprobe of each query from the class chosen by the network: class c -> 2^c, capped.
__global__ void class_to_nprobe_kernel(const int32_t* __restrict__ cls, int64_t nq, int cap,
                                       int shift, int32_t* __restrict__ np) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nq) np[q] = min(1 << min(max(cls[q] + shift, 0), 30), cap);
}

__global__ void recall_counts_kernel(const int64_t* __restrict__ I, const int64_t* __restrict__ G,
                                     int64_t nq, int k, int kg, int32_t* __restrict__ cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int c = 0;
  for (int i = 0; i < k; i++) {
    const int64_t v = I[q * k + i];
    if (v < 0) continue;
    for (int j = 0; j < kg; j++)
      if (G[q * kg + j] == v) {
        c++;
        break;
      }
  }
  cnt[q] = c;
}

}  // namespace

gbk_status nprobe_features_run(const float* xq, int64_t nq, int d, const float* clD, int tau,
                               int nfeat, float* F, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  ProfScope prof("nprobe_features", st);
  nprobe_features_kernel<<<(unsigned)nq, 128, 0, st>>>(xq, nq, d, clD, tau, nfeat, F);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

// kq / out_off may be null (every query max_k results at q * max_k); positions: list
// positions out instead of ids; prerotated: xq already in the index's rotated space.
gbk_status batched_run(gbk_index* ix, const float* xq_in, int64_t nq, const int32_t* kq,
                       int max_k, const int32_t* npq_in, int max_nprobe, gbk_mlp* mlp,
                       const int64_t* out_off, float* D, int64_t* I, int32_t* np_used,
                       cudaStream_t st, bool positions, bool prerotated) {
  gbk_status r;
  Scratch xr;
  const float* xq = xq_in;
  if (!prerotated && (r = rotate_rows(ix, xq_in, nq, xr, &xq, st)) != GBK_OK) return r;
  const int nfeat = 64;
  const int tau = std::min(ix->nlist, mlp ? std::max(max_nprobe, nfeat) : max_nprobe);
  Scratch clD, clI, t3, npq_s, F, cls, key, order, off32, counter;
  if ((r = clD.alloc(sizeof(float) * (size_t)nq * tau, st)) != GBK_OK) return r;
  if ((r = clI.alloc(sizeof(int64_t) * (size_t)nq * tau, st)) != GBK_OK) return r;
  KnnPlan plan;
  plan.prec = ix->coarse_prec;
  // L_IVF (Eq. 5) for the largest nprobe of the batch, with term 2
  if ((r = knn_run(xq, nq, ix->coarse.as<float>(), ix->nlist, ix->d, tau, GBK_METRIC_L2,
                   clD.as<float>(), clI.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  const int32_t* npq = npq_in;
  if (!npq) {
    // learned nprobe: features -> network -> class -> nprobe
    if ((r = npq_s.alloc(sizeof(int32_t) * (size_t)nq, st)) != GBK_OK) return r;
    if ((r = F.alloc(sizeof(float) * (size_t)nq * (ix->d + nfeat), st)) != GBK_OK) return r;
    if ((r = cls.alloc(sizeof(int32_t) * (size_t)nq, st)) != GBK_OK) return r;
    if ((r = nprobe_features_run(xq, nq, ix->d, clD.as<float>(), tau, std::min(nfeat, tau),
                                 F.as<float>(), st)) != GBK_OK)
      return r;
    if ((r = mlp_forward_classes(mlp, F.as<float>(), nq, cls.as<int32_t>(), st,
                                 ix->route_alpha)) != GBK_OK)
      return r;
    class_to_nprobe_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(
        cls.as<int32_t>(), nq, max_nprobe, ix->class_shift, npq_s.as<int32_t>());
    GBK_LAUNCH_CHECK();
    npq = npq_s.as<int32_t>();
  }
  if (np_used)
    GBK_CUDA_CHECK(cudaMemcpyAsync(np_used, npq, sizeof(int32_t) * (size_t)nq,
                                   cudaMemcpyDeviceToDevice, st));
  const bool direct = !ix->use_precomputed;
  if (!direct) {
    if ((r = t3.alloc(sizeof(float) * (size_t)nq * ix->M * 256, st)) != GBK_OK) return r;
    if ((r = term3_run(xq, nq, ix->pq.as<float>(), ix->d, ix->M, t3.as<float>(), st)) != GBK_OK)
      return r;
  }
  // longest-first work order for the persistent scan (uneven lists, mixed nprobe)
  if ((r = key.alloc(sizeof(int32_t) * (size_t)nq, st)) != GBK_OK) return r;
  if ((r = order.alloc(sizeof(int64_t) * (size_t)nq, st)) != GBK_OK) return r;
  if ((r = off32.alloc(sizeof(int64_t) * 33, st)) != GBK_OK) return r;
  if ((r = counter.alloc(sizeof(unsigned long long), st)) != GBK_OK) return r;
  if ((r = scan_cost_run(clI.as<int64_t>(), nq, tau, npq, ix->list_off.as<int64_t>(),
                         key.as<int32_t>(), st)) != GBK_OK)
    return r;
  if ((r = bucket_stable(key.as<int32_t>(), nq, 32, off32.as<int64_t>(), order.as<int64_t>(), st)) !=
      GBK_OK)
    return r;
  GBK_CUDA_CHECK(cudaMemsetAsync(counter.p, 0, sizeof(unsigned long long), st));
  return ivf_scan_run(ix->M, nq, tau, max_k, clI.as<int64_t>(), clD.as<float>(), ix->s1.as<float>(),
                      t3.as<float>(), xq, ix->coarse.as<float>(), ix->pq.as<float>(), ix->d, direct,
                      ix->list_off.as<int64_t>(), ix->codes.as<uint8_t>(),
                      positions ? nullptr : ix->ids.as<int64_t>(), D, I, st, kq, npq, out_off,
                      order.as<int64_t>(), counter.as<unsigned long long>(), ix->tuning);
}

}  // namespace gbk

struct gbk_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~gbk_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

extern "C" {

static gbk_status batched_check(gbk_index* ix, const float* xq, int64_t nq, const int32_t* kq,
                                int32_t max_k, const int32_t* npq, int32_t max_nprobe,
                                gbk_mlp* mlp, const int64_t* out_off, float* D, int64_t* I) {
  GBK_REQUIRE(ix && ix->trained, "batched search: index missing or not trained");
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "batched search: nq out of range");
  GBK_REQUIRE(max_k >= 1 && max_k <= GBK_MAX_K, "batched search: max_k out of [1, %d]", GBK_MAX_K);
  GBK_REQUIRE(max_nprobe >= 1 && max_nprobe <= ix->nlist && max_nprobe <= GBK_MAX_K,
              "batched search: max_nprobe out of range");
  GBK_REQUIRE(npq || mlp, "batched search: give nprobe_per_q or a network");
  if (!npq) {
    GBK_REQUIRE(ix->nlist >= 64, "learned nprobe needs nlist >= 64 (64 coarse-distance features)");
    GBK_REQUIRE(gbk::mlp_inputs(mlp) == ix->d + 64,
                "learned nprobe: network inputs must be d + 64 = %d", ix->d + 64);
  }
  GBK_REQUIRE(nq == 0 || (xq && kq && out_off && D && I), "batched search: NULL pointer");
  return GBK_OK;
}

gbk_status gbk_ivfpq_search_batched(gbk_index* ix, const float* xq, int64_t nq,
                                    const int32_t* k_per_q, int32_t max_k,
                                    const int32_t* nprobe_per_q, int32_t max_nprobe,
                                    gbk_mlp* mlp, const int64_t* out_offsets, float* D,
                                    int64_t* I, int32_t* nprobe_used, void* stream) {
  clear_error();
  gbk_status r = batched_check(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp,
                               out_offsets, D, I);
  if (r != GBK_OK || nq == 0) return r;
  cudaStream_t st = as_stream(stream);
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  return batched_run(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp, out_offsets, D, I,
                     nprobe_used, st);
}

gbk_status gbk_ivfpq_search_batched_refine(gbk_index* ix, const float* xq, int64_t nq,
                                           int32_t k, int32_t kprime,
                                           const int32_t* nprobe_per_q, int32_t max_nprobe,
                                           gbk_mlp* mlp, float* D, int64_t* I,
                                           int32_t* nprobe_used, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained, "batched refine: index missing or not trained");
  GBK_REQUIRE(ix->keep_vectors, "batched refine: the index keeps no vectors");
  GBK_REQUIRE(k >= 1 && kprime >= k && kprime <= GBK_MAX_K,
              "batched refine: need 1 <= k <= kprime <= %d", GBK_MAX_K);
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "batched refine: nq out of range");
  GBK_REQUIRE(max_nprobe >= 1 && max_nprobe <= ix->nlist && max_nprobe <= GBK_MAX_K,
              "batched refine: max_nprobe out of range");
  GBK_REQUIRE(nprobe_per_q || mlp, "batched refine: give nprobe_per_q or a network");
  if (!nprobe_per_q) {
    GBK_REQUIRE(ix->nlist >= 64, "learned nprobe needs nlist >= 64 (64 coarse-distance features)");
    GBK_REQUIRE(gbk::mlp_inputs(mlp) == ix->d + 64,
                "learned nprobe: network inputs must be d + 64 = %d", ix->d + 64);
  }
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && D && I, "batched refine: NULL pointer");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  Scratch xr, Dc, Ic;
  const float* xqr = xq;
  if ((r = rotate_rows(ix, xq, nq, xr, &xqr, st)) != GBK_OK) return r;
  if ((r = Dc.alloc(sizeof(float) * (size_t)nq * kprime, st)) != GBK_OK) return r;
  if ((r = Ic.alloc(sizeof(int64_t) * (size_t)nq * kprime, st)) != GBK_OK) return r;
  // k' ADC candidates per query (list positions) from the mixed-nprobe scan, then the exact
  // float32 re-rank from the kept vectors and the ids of the k winners
  if ((r = batched_run(ix, xqr, nq, nullptr, kprime, nprobe_per_q, max_nprobe, mlp, nullptr,
                       Dc.as<float>(), Ic.as<int64_t>(), nprobe_used, st, true, true)) != GBK_OK)
    return r;
  if ((r = rerank_rows_run(xqr, ix->vecs.as<float>(), nq, ix->d, kprime, k, Ic.as<int64_t>(), D,
                           I, st)) != GBK_OK)
    return r;
  return rows_to_ids_run(I, nq * (int64_t)k, ix->ids.as<int64_t>(), st);
}

gbk_status gbk_ivfpq_batched_graph(gbk_index* ix, const float* xq, int64_t nq,
                                   const int32_t* k_per_q, int32_t max_k,
                                   const int32_t* nprobe_per_q, int32_t max_nprobe, gbk_mlp* mlp,
                                   const int64_t* out_offsets, float* D, int64_t* I,
                                   int32_t* nprobe_used, gbk_graph** out, void* stream) {
  clear_error();
  GBK_REQUIRE(out, "gbk_ivfpq_batched_graph: out is NULL");
  gbk_status r = batched_check(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp,
                               out_offsets, D, I);
  if (r != GBK_OK) return r;
  GBK_REQUIRE(nq > 0, "gbk_ivfpq_batched_graph: empty batch");
  cudaStream_t st = as_stream(stream);
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  if (!device_status()) return set_error(GBK_ECUDA, "device status word unavailable");
  GBK_CUDA_CHECK(cudaStreamSynchronize(st));
  cudaStream_t cs;
  GBK_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  gbk_graph* g = new gbk_graph();
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    r = batched_run(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp, out_offsets, D, I,
                    nprobe_used, cs);
    e = cudaStreamEndCapture(cs, &g->graph);
  }
  if (e == cudaSuccess && r == GBK_OK) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  cudaStreamDestroy(cs);
  if (r != GBK_OK || e != cudaSuccess) {
    delete g;
    cudaGetLastError();
    return r != GBK_OK ? r : set_error(GBK_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  *out = g;
  return GBK_OK;
}

gbk_status gbk_graph_launch(gbk_graph* g, void* stream) {
  clear_error();
  GBK_REQUIRE(g && g->exec, "gbk_graph_launch: NULL graph");
  GBK_CUDA_CHECK(cudaGraphLaunch(g->exec, as_stream(stream)));
  return GBK_OK;
}

void gbk_graph_destroy(gbk_graph* g) { delete g; }

gbk_status gbk_recall_counts(const int64_t* I, const int64_t* G, int64_t nq, int32_t k, int32_t kg,
                             int32_t* counts, void* stream) {
  clear_error();
  GBK_REQUIRE(nq >= 0 && k >= 1 && kg >= 1, "gbk_recall_counts: bad sizes");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(I && G && counts, "gbk_recall_counts: NULL pointer");
  recall_counts_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, as_stream(stream)>>>(I, G, nq, k, kg,
                                                                                   counts);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status gbk_nprobe_features(const float* xq, int64_t nq, int32_t d, const float* coarse_dist,
                               int32_t tau, int32_t nfeat, float* F, void* stream) {
  clear_error();
  GBK_REQUIRE(nq >= 0 && d >= 1 && nfeat >= 1 && tau >= nfeat, "gbk_nprobe_features: bad sizes");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && coarse_dist && F, "gbk_nprobe_features: NULL pointer");
  nprobe_features_kernel<<<(unsigned)nq, 128, 0, as_stream(stream)>>>(xq, nq, d, coarse_dist, tau,
                                                                      nfeat, F);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ k-NN graph (section 6.5)

namespace gbk {
namespace {

// Row r of the (k+1)-NN lists without the query's own id: the first occurrence of `self`
// is dropped (a duplicate vector with another id stays a neighbour); when the row does not
// contain it, its first k entries are kept.
__global__ void drop_self_kernel(const float* __restrict__ D1, const int64_t* __restrict__ I1,
                                 int64_t n, int k, const int64_t* __restrict__ self_ids,
                                 int64_t id0, float* __restrict__ GD, int64_t* __restrict__ G) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t self = self_ids ? self_ids[r] : id0 + r;
  const float* d = D1 + r * (k + 1);
  const int64_t* id = I1 + r * (k + 1);
  bool dropped = false;
  int j = 0;
  for (int i = 0; i <= k && j < k; i++) {
    if (!dropped && id[i] == self) {
      dropped = true;
      continue;
    }
    if (GD) GD[r * k + j] = d[i];
    G[r * k + j] = id[i];
    j++;
  }
}

__global__ void fill_graph_args_kernel(int64_t n, int kk, int32_t* kq, int64_t* off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) kq[i] = kk;
  if (i <= n) off[i] = i * kk;
}

}  // namespace
}  // namespace gbk

extern "C" {

static gbk_status knn_graph_run(gbk_index* ix, const float* x, int64_t n, const int64_t* self_ids,
                                int32_t k, int32_t nprobe, int32_t kprime, gbk_mlp* mlp,
                                int64_t batch, float* GD, int64_t* G, void* stream) {
  GBK_REQUIRE(ix && ix->trained, "gbk_ivfpq_knn_graph: index missing or not trained");
  GBK_REQUIRE(k >= 1 && k < GBK_MAX_K, "gbk_ivfpq_knn_graph: k out of [1, %d)", GBK_MAX_K);
  GBK_REQUIRE(nprobe >= 1 && nprobe <= ix->nlist && nprobe <= GBK_MAX_K,
              "gbk_ivfpq_knn_graph: nprobe out of range");
  GBK_REQUIRE(kprime == 0 || (kprime > k && kprime <= GBK_MAX_K && ix->keep_vectors),
              "gbk_ivfpq_knn_graph: re-rank needs k < kprime <= %d and kept vectors", GBK_MAX_K);
  GBK_REQUIRE(n >= 0, "gbk_ivfpq_knn_graph: n < 0");
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x && G, "gbk_ivfpq_knn_graph: NULL pointer");
  if (mlp) {
    GBK_REQUIRE(ix->nlist >= 64, "learned nprobe needs nlist >= 64 (64 coarse-distance features)");
    GBK_REQUIRE(gbk::mlp_inputs(mlp) == ix->d + 64,
                "learned nprobe: network inputs must be d + 64 = %d", ix->d + 64);
  }
  const int kk = k + 1;
  const int kc = kprime > 0 ? kprime : kk;  // candidates per query from the scan
  if (batch <= 0) batch = int64_t(1) << 20;
  batch = std::min<int64_t>(batch, std::min<int64_t>(n, (int64_t(1) << 31) / (kc + 1) - 1));
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  Scratch D1, I1, Dc, Ic, kq, off;
  if ((r = D1.alloc(sizeof(float) * (size_t)batch * kk, st)) != GBK_OK) return r;
  if ((r = I1.alloc(sizeof(int64_t) * (size_t)batch * kk, st)) != GBK_OK) return r;
  if (kprime > 0) {
    if ((r = Dc.alloc(sizeof(float) * (size_t)batch * kc, st)) != GBK_OK) return r;
    if ((r = Ic.alloc(sizeof(int64_t) * (size_t)batch * kc, st)) != GBK_OK) return r;
  }
  if (mlp && kprime == 0) {
    if ((r = kq.alloc(sizeof(int32_t) * (size_t)batch, st)) != GBK_OK) return r;
    if ((r = off.alloc(sizeof(int64_t) * (size_t)(batch + 1), st)) != GBK_OK) return r;
    gbk::fill_graph_args_kernel<<<(unsigned)((batch + 256) / 256), 256, 0, st>>>(
        batch, kk, kq.as<int32_t>(), off.as<int64_t>());
    GBK_LAUNCH_CHECK();
  }
  ProfScope prof("knn_graph", st);
  for (int64_t b0 = 0; b0 < n; b0 += batch) {
    const int64_t nb = std::min(batch, n - b0);
    const float* xb = x + b0 * ix->d;
    if (kprime > 0) {
      // k' ADC candidates as list positions, exact float32 re-rank from the kept vectors
      Scratch xr;
      const float* xbr = xb;
      if ((r = gbk::rotate_rows(ix, xb, nb, xr, &xbr, st)) != GBK_OK) return r;
      if (mlp)
        r = gbk::batched_run(ix, xbr, nb, nullptr, kc, nullptr, nprobe, mlp, nullptr,
                             Dc.as<float>(), Ic.as<int64_t>(), nullptr, st, true, true);
      else
        r = gbk::search_run(ix, xbr, nb, kc, nprobe, Dc.as<float>(), Ic.as<int64_t>(), st, true,
                            true);
      if (r != GBK_OK) return r;
      if ((r = gbk::rerank_rows_run(xbr, ix->vecs.as<float>(), nb, ix->d, kc, kk,
                                    Ic.as<int64_t>(), D1.as<float>(), I1.as<int64_t>(), st)) !=
          GBK_OK)
        return r;
      if ((r = gbk::rows_to_ids_run(I1.as<int64_t>(), nb * (int64_t)kk, ix->ids.as<int64_t>(),
                                    st)) != GBK_OK)
        return r;
    } else if (mlp) {
      r = gbk::batched_run(ix, xb, nb, kq.as<int32_t>(), kk, nullptr, nprobe, mlp,
                           off.as<int64_t>(), D1.as<float>(), I1.as<int64_t>(), nullptr, st);
    } else {
      r = gbk::search_run(ix, xb, nb, kk, nprobe, D1.as<float>(), I1.as<int64_t>(), st);
    }
    if (r != GBK_OK) return r;
    gbk::drop_self_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
        D1.as<float>(), I1.as<int64_t>(), nb, k, self_ids ? self_ids + b0 : nullptr, b0,
        GD ? GD + b0 * k : nullptr, G + b0 * k);
    GBK_LAUNCH_CHECK();
  }
  return GBK_OK;
}

gbk_status gbk_ivfpq_knn_graph(gbk_index* ix, const float* x, int64_t n, const int64_t* self_ids,
                               int32_t k, int32_t nprobe, gbk_mlp* mlp, int64_t batch,
                               float* GD, int64_t* G, void* stream) {
  clear_error();
  return knn_graph_run(ix, x, n, self_ids, k, nprobe, 0, mlp, batch, GD, G, stream);
}

gbk_status gbk_ivfpq_knn_graph_refine(gbk_index* ix, const float* x, int64_t n,
                                      const int64_t* self_ids, int32_t k, int32_t nprobe,
                                      int32_t kprime, gbk_mlp* mlp, int64_t batch, float* GD,
                                      int64_t* G, void* stream) {
  clear_error();
  GBK_REQUIRE(kprime >= 1, "gbk_ivfpq_knn_graph_refine: kprime < 1");
  return knn_graph_run(ix, x, n, self_ids, k, nprobe, kprime, mlp, batch, GD, G, stream);
}

}  // extern "C"

// ------------------------------------------------------------------ scan autotuning

extern "C" {

gbk_status gbk_ivfpq_set_tuning(gbk_index* ix, int32_t codes_per_thread, int32_t blocks_per_sm) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_set_tuning: NULL index");
  GBK_REQUIRE(codes_per_thread == 2 || codes_per_thread == 4 || codes_per_thread == 8,
              "gbk_ivfpq_set_tuning: codes per thread must be 2, 4 or 8");
  GBK_REQUIRE(blocks_per_sm >= 1 && blocks_per_sm <= 8,
              "gbk_ivfpq_set_tuning: blocks per SM must be in [1, 8]");
  ix->tuning.codes_per_thread = codes_per_thread;
  ix->tuning.blocks_per_sm = blocks_per_sm;
  return GBK_OK;
}

gbk_status gbk_ivfpq_set_scan_options(gbk_index* ix, int32_t threads_per_block, int32_t by_list) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_set_scan_options: NULL index");
  GBK_REQUIRE(threads_per_block == 256 || threads_per_block == 384 || threads_per_block == 512,
              "gbk_ivfpq_set_scan_options: threads per block must be 256, 384 or 512");
  ix->tuning.threads = threads_per_block;
  ix->tuning.list_order = by_list ? 1 : 0;
  return GBK_OK;
}

gbk_status gbk_ivfpq_get_tuning(const gbk_index* ix, int32_t* codes_per_thread,
                                int32_t* blocks_per_sm) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfpq_get_tuning: NULL index");
  if (codes_per_thread) *codes_per_thread = ix->tuning.codes_per_thread;
  if (blocks_per_sm) *blocks_per_sm = ix->tuning.blocks_per_sm;
  return GBK_OK;
}

gbk_status gbk_ivfpq_autotune(gbk_index* ix, const float* xq, int64_t nq, const int32_t* k_per_q,
                              int32_t max_k, const int32_t* nprobe_per_q, int32_t max_nprobe,
                              gbk_mlp* mlp, const int64_t* out_offsets, float* D, int64_t* I,
                              int32_t reps, float* best_ms, void* stream) {
  clear_error();
  gbk_status r = batched_check(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp,
                               out_offsets, D, I);
  if (r != GBK_OK) return r;
  GBK_REQUIRE(nq > 0, "gbk_ivfpq_autotune: empty batch");
  if (reps < 1) reps = 3;
  cudaStream_t st = as_stream(stream);
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  cudaEvent_t e0, e1;
  GBK_CUDA_CHECK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(GBK_ECUDA, "gbk_ivfpq_autotune: cudaEventCreate failed");
  }
  const gbk::ScanTuning keep = ix->tuning;
  gbk::ScanTuning best = keep;
  float best_t = -1.f;
  // block size x codes per thread (the shapes that keep two blocks per SM) x blocks per SM
  static const int SHAPES[6][2] = {{256, 2}, {256, 4}, {256, 8}, {384, 2}, {384, 4}, {512, 2}};
  const int nshape = ix->use_precomputed ? 6 : 3;  // the direct-table scan has 256 threads
  for (int si = 0; si < nshape && r == GBK_OK; si++) {
    for (int bps = 1; bps <= 2 && r == GBK_OK; bps++) {
      ix->tuning.threads = SHAPES[si][0];
      ix->tuning.codes_per_thread = SHAPES[si][1];
      ix->tuning.blocks_per_sm = bps;
      // one untimed run (first-use set-up), then `reps` timed runs of the whole batch
      r = gbk::batched_run(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp,
                           out_offsets, D, I, nullptr, st);
      if (r != GBK_OK) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) {
        r = set_error(GBK_ECUDA, "gbk_ivfpq_autotune: event record failed");
        break;
      }
      for (int i = 0; i < reps && r == GBK_OK; i++)
        r = gbk::batched_run(ix, xq, nq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp,
                             out_offsets, D, I, nullptr, st);
      if (r != GBK_OK) break;
      float ms = 0.f;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        r = set_error(GBK_ECUDA, "gbk_ivfpq_autotune: event timing failed");
        break;
      }
      ms /= (float)reps;
      if (best_t < 0.f || ms < best_t) {
        best_t = ms;
        best = ix->tuning;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ix->tuning = r == GBK_OK ? best : keep;
  if (r == GBK_OK && best_ms) *best_ms = best_t;
  return r;
}

}  // extern "C"

