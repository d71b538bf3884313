// IVF-Flat: the inverted file of section 2 ("Compressed-domain search") with uncompressed
// lists.  The coarse quantizer q1 (Eq. 3) and its search (Eq. 5) are those of IVFADC; the
// lists hold the float32 vectors themselves, so the list scan computes exact squared
// distances (Eq. 1) instead of ADC look-ups, and the k-selection is the same block
// selection as every other kernel of the library.  Section 5.1 names this exact stage as a
// component of many indexes; here it also serves the exact re-rank of IVFADC candidates
// from stored vectors.
//
// List scan layout: a block per query, 8 lanes per vector (each lane sums the squared
// differences of every 8th float4 of the row), 4 vectors per warp and 4 such groups in
// flight per thread, so one step reads 128 rows; the lanes of a group then butterfly-sum
// their partials and one of them offers the result to the selection.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "ivf.cuh"
#include "knn.cuh"
#include "select_core.cuh"

namespace gbk {

namespace {

__global__ void gather_rows_kernel(const float* __restrict__ in, const int64_t* __restrict__ order,
                                   int64_t n, int d, float* __restrict__ out) {
  const bool v4 = (d & 3) == 0;
  const int w = v4 ? d / 4 : d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * w;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / w;
    const int t = (int)(e % w);
    const int64_t src = order[j];
    if (v4)
      reinterpret_cast<float4*>(out)[j * w + t] = reinterpret_cast<const float4*>(in)[src * w + t];
    else
      out[j * d + t] = in[src * d + t];
  }
}

__global__ void rows_to_ids_kernel(int64_t* __restrict__ I, int64_t n,
                                   const int64_t* __restrict__ ids) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = I[j];
    if (r >= 0) I[j] = ids[r];
  }
}

struct FlatArgs {
  int64_t nq;
  int d, nprobe, k;
  const float* xq;
  const int64_t* cl_I;      // [nq][nprobe] probed lists (-1 = none)
  const int64_t* list_off;  // [nlist + 1]
  const float* vecs;        // [ntotal][d] list order
  const int64_t* ids;       // [ntotal] or null (positions out)
  float* D;
  int64_t* I;
};

template <int KP, bool V4>
__global__ void __launch_bounds__(256) ivf_flat_scan_kernel(const FlatArgs a) {
  constexpr int THREADS = 256, CAP = 2048, U = 4, STEP = 32 * U;
  using Sel = BlockSelect<THREADS, KP, CAP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* xs = reinterpret_cast<float*>(smem_raw);  // the query, d floats (16-byte padded)
  typename Sel::Smem& s =
      *reinterpret_cast<typename Sel::Smem*>(smem_raw + ((size_t)a.d * 4 + 15) / 16 * 16);
  const int64_t q = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sub = lane & 7, grp = lane >> 3;
  for (int t = tid; t < a.d; t += THREADS) xs[t] = a.xq[q * a.d + t];
  Sel::init(s);
  __syncthreads();
  ValueFilter f;
  f.set(NAN_KEY, false);
  for (int p = 0; p < a.nprobe; p++) {
    const int64_t L = a.cl_I[q * a.nprobe + p];
    if (L < 0) continue;  // uniform across the block
    const int64_t o0 = a.list_off[L], o1 = a.list_off[L + 1];
    for (int64_t b0 = o0; b0 < o1; b0 += STEP) {
      float acc[U];
#pragma unroll
      for (int u = 0; u < U; u++) acc[u] = 0.f;
      if (V4) {
        const int nf = a.d >> 2;
        const float4* x4 = reinterpret_cast<const float4*>(xs);
        const float4* y4 = reinterpret_cast<const float4*>(a.vecs);
        for (int fi = sub; fi < nf; fi += 8) {
          const float4 xv = x4[fi];
          float4 yv[U];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const int64_t v = b0 + u * 32 + warp * 4 + grp;
            yv[u] = v < o1 ? __ldg(y4 + v * nf + fi) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < U; u++) {
            float e = xv.x - yv[u].x;
            acc[u] = fmaf(e, e, acc[u]);
            e = xv.y - yv[u].y;
            acc[u] = fmaf(e, e, acc[u]);
            e = xv.z - yv[u].z;
            acc[u] = fmaf(e, e, acc[u]);
            e = xv.w - yv[u].w;
            acc[u] = fmaf(e, e, acc[u]);
          }
        }
      } else {
        for (int t = sub; t < a.d; t += 8) {
          const float xv = xs[t];
#pragma unroll
          for (int u = 0; u < U; u++) {
            const int64_t v = b0 + u * 32 + warp * 4 + grp;
            const float e = v < o1 ? xv - __ldg(a.vecs + v * a.d + t) : 0.f;
            acc[u] = fmaf(e, e, acc[u]);
          }
        }
      }
      uint32_t mask = 0;
      uint64_t cc[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        acc[u] += __shfl_xor_sync(FULL_MASK, acc[u], 4);
        acc[u] += __shfl_xor_sync(FULL_MASK, acc[u], 2);
        acc[u] += __shfl_xor_sync(FULL_MASK, acc[u], 1);
        const int64_t v = b0 + u * 32 + warp * 4 + grp;
        cc[u] = ~0ull;
        if (sub == u && v < o1 && f.pass(acc[u])) {
          mask |= 1u << u;
          cc[u] = composite(ordered_key(acc[u], false), (uint32_t)v);
        }
      }
      Sel::template push<U>(s, mask, cc);
      __syncthreads();
      if (s.n_buf > CAP - STEP) {
        Sel::compact(s, a.k);
        f.set((uint32_t)(s.thr >> 32), false);
      }
    }
  }
  Sel::finish(s, a.k);
  for (int j = tid; j < a.k; j += THREADS) {
    const uint64_t e = s.top[j];
    const int64_t o = q * a.k + j;
    if (e == ~0ull) {
      a.D[o] = __int_as_float(0x7f800000);
      a.I[o] = -1;
    } else {
      a.D[o] = key_value((uint32_t)(e >> 32), false);
      a.I[o] = a.ids ? a.ids[(uint32_t)e] : (int64_t)(uint32_t)e;
    }
  }
}

template <int KP>
gbk_status launch_flat(const FlatArgs& a, cudaStream_t st) {
  using Sel = BlockSelect<256, KP, 2048>;
  const size_t smem = ((size_t)a.d * 4 + 15) / 16 * 16 + sizeof(typename Sel::Smem);
  if ((a.d & 3) == 0)
    ivf_flat_scan_kernel<KP, true><<<(unsigned)a.nq, 256, smem, st>>>(a);
  else
    ivf_flat_scan_kernel<KP, false><<<(unsigned)a.nq, 256, smem, st>>>(a);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256,
                                                     (int64_t)device_info().sm_count * 16));
}

}  // namespace

gbk_status gather_rows_run(const float* in, const int64_t* order, int64_t n, int d, float* out,
                           cudaStream_t st) {
  if (n == 0) return GBK_OK;
  const int64_t w = (d & 3) == 0 ? d / 4 : d;
  gather_rows_kernel<<<grid_for(n * w), 256, 0, st>>>(in, order, n, d, out);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status rows_to_ids_run(int64_t* I, int64_t n, const int64_t* ids, cudaStream_t st) {
  if (n == 0) return GBK_OK;
  rows_to_ids_kernel<<<grid_for(n), 256, 0, st>>>(I, n, ids);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

gbk_status ivf_flat_scan_run(const float* xq, int64_t nq, int d, int nprobe, int k,
                             const int64_t* cl_I, const int64_t* list_off, const float* vecs,
                             const int64_t* ids, float* D, int64_t* I, cudaStream_t st) {
  if (nq == 0) return GBK_OK;
  if (d > 4096) return set_error(GBK_EUNSUPPORTED, "IVF-Flat scan supports d <= 4096");
  FlatArgs a{nq, d, nprobe, k, xq, cl_I, list_off, vecs, ids, D, I};
  ProfScope prof("ivf_flat_scan", st);
  if (k <= 32) return launch_flat<32>(a, st);
  if (k <= 128) return launch_flat<128>(a, st);
  if (k <= 256) return launch_flat<256>(a, st);
  return launch_flat<1024>(a, st);
}

}  // namespace gbk

// ---------------------------------------------------------------------------- the index

struct gbk_ivfflat {
  int d = 0, nlist = 0;
  bool trained = false;
  gbk::DevBuf coarse;
  // insertion-order staging: every added vector's list, the vector, its id
  gbk::DevBuf st_list, st_vecs, st_ids;
  int64_t n_staged = 0, cap_staged = 0;
  // inverted file in list order (rebuilt from the staging arrays on demand)
  gbk::DevBuf list_off, vecs, ids;
  int64_t ntotal = 0;
  bool dirty = true;
  ~gbk_ivfflat() {
    coarse.release();
    st_list.release();
    st_vecs.release();
    st_ids.release();
    list_off.release();
    vecs.release();
    ids.release();
  }
};

namespace gbk {
namespace {

__global__ void flat_stage_kernel(const int64_t* __restrict__ a, const int64_t* __restrict__ ids,
                                  int64_t n, int64_t first, int32_t* __restrict__ lists,
                                  int64_t* __restrict__ ids_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    lists[i] = (int32_t)a[i];
    ids_out[i] = ids ? ids[i] : first + i;
  }
}

__global__ void flat_ids_kernel(const int64_t* __restrict__ order, int64_t n,
                                const int64_t* __restrict__ in, int64_t* __restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = in[order[j]];
}

gbk_status flat_finalize(gbk_ivfflat* ix, cudaStream_t st) {
  if (!ix->dirty) return GBK_OK;
  gbk_status r;
  const int64_t n = ix->n_staged;
  if ((r = ix->list_off.alloc(sizeof(int64_t) * (size_t)(ix->nlist + 1))) != GBK_OK) return r;
  if ((r = ix->vecs.alloc(sizeof(float) * (size_t)std::max<int64_t>(n, 1) * ix->d)) != GBK_OK)
    return r;
  if ((r = ix->ids.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1))) != GBK_OK) return r;
  Scratch order;
  if ((r = order.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(n, 1), st)) != GBK_OK) return r;
  if ((r = bucket_stable(ix->st_list.as<int32_t>(), n, ix->nlist, ix->list_off.as<int64_t>(),
                         order.as<int64_t>(), st)) != GBK_OK)
    return r;
  if (n > 0) {
    if ((r = gather_rows_run(ix->st_vecs.as<float>(), order.as<int64_t>(), n, ix->d,
                             ix->vecs.as<float>(), st)) != GBK_OK)
      return r;
    flat_ids_kernel<<<grid_for(n), 256, 0, st>>>(order.as<int64_t>(), n,
                                                 ix->st_ids.as<int64_t>(), ix->ids.as<int64_t>());
    GBK_LAUNCH_CHECK();
  }
  ix->ntotal = n;
  ix->dirty = false;
  return GBK_OK;
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_ivfflat_create(int32_t d, int32_t nlist, int32_t metric, gbk_ivfflat** out) {
  clear_error();
  GBK_REQUIRE(out, "gbk_ivfflat_create: out is NULL");
  GBK_REQUIRE(d >= 1 && d <= 4096 && nlist >= 1 && nlist < (1 << 30),
              "gbk_ivfflat_create: need 1 <= d <= 4096 and 1 <= nlist < 2^30");
  if (metric != GBK_METRIC_L2)
    return set_error(GBK_EUNSUPPORTED, "gbk_ivfflat_create: the inverted file is built for L2");
  gbk_ivfflat* ix = new gbk_ivfflat();
  ix->d = d;
  ix->nlist = nlist;
  *out = ix;
  return GBK_OK;
}

void gbk_ivfflat_destroy(gbk_ivfflat* ix) { delete ix; }

gbk_status gbk_ivfflat_train(gbk_ivfflat* ix, const float* x, int64_t n,
                             const gbk_train_opts* opts, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && x, "gbk_ivfflat_train: NULL argument");
  GBK_REQUIRE(n >= ix->nlist && n < (int64_t(1) << 31),
              "gbk_ivfflat_train: need nlist <= n < 2^31 training vectors");
  cudaStream_t st = as_stream(stream);
  const int niter = opts && opts->niter > 0 ? opts->niter : 20;
  std::vector<int64_t> cinit(ix->nlist);
  for (int i = 0; i < ix->nlist; i++) cinit[i] = opts && opts->coarse_init ? opts->coarse_init[i] : i;
  for (int64_t v : cinit) GBK_REQUIRE(v >= 0 && v < n, "gbk_ivfflat_train: coarse_init out of range");
  gbk_status r;
  if ((r = ix->coarse.alloc(sizeof(float) * (size_t)ix->nlist * ix->d)) != GBK_OK) return r;
  Scratch ci;
  if ((r = ci.alloc(sizeof(int64_t) * ix->nlist, st)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ci.p, cinit.data(), sizeof(int64_t) * ix->nlist,
                                 cudaMemcpyHostToDevice, st));
  // q1 (Eq. 3) by k-means, assignment on the tensor cores
  if ((r = kmeans_run(x, n, ix->d, ix->d, ix->nlist, niter, ci.as<int64_t>(),
                      ix->coarse.as<float>(), nullptr, nullptr, false, st)) != GBK_OK)
    return r;
  ix->trained = true;
  return GBK_OK;
}

gbk_status gbk_ivfflat_set_centroids(gbk_ivfflat* ix, const float* coarse, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && coarse, "gbk_ivfflat_set_centroids: NULL argument");
  gbk_status r;
  const size_t cb = sizeof(float) * (size_t)ix->nlist * ix->d;
  if ((r = ix->coarse.alloc(cb)) != GBK_OK) return r;
  GBK_CUDA_CHECK(cudaMemcpyAsync(ix->coarse.p, coarse, cb, cudaMemcpyDefault, as_stream(stream)));
  ix->trained = true;
  return GBK_OK;
}

gbk_status gbk_ivfflat_add(gbk_ivfflat* ix, const float* x, int64_t n, const int64_t* ids,
                           void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfflat_add: NULL index");
  GBK_REQUIRE(ix->trained, "gbk_ivfflat_add: index not trained");
  GBK_REQUIRE(n >= 0, "gbk_ivfflat_add: n < 0");
  if (n == 0) return GBK_OK;
  GBK_REQUIRE(x, "gbk_ivfflat_add: NULL x");
  GBK_REQUIRE(ix->n_staged + n < (int64_t(1) << 32) - 1, "gbk_ivfflat_add: index full (2^32)");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  const int64_t need = ix->n_staged + n;
  const size_t row = sizeof(float) * (size_t)ix->d;
  if (need > ix->cap_staged) {
    const int64_t cap = std::max<int64_t>(need, ix->cap_staged * 2);
    const size_t keep = (size_t)ix->n_staged;
    if ((r = ix->st_list.grow(sizeof(int32_t) * cap, sizeof(int32_t) * keep, st)) != GBK_OK) return r;
    if ((r = ix->st_vecs.grow(row * cap, row * keep, st)) != GBK_OK) return r;
    if ((r = ix->st_ids.grow(sizeof(int64_t) * cap, sizeof(int64_t) * keep, st)) != GBK_OK) return r;
    ix->cap_staged = cap;
  }
  Scratch a, dist;
  if ((r = a.alloc(sizeof(int64_t) * (size_t)n, st)) != GBK_OK) return r;
  if ((r = dist.alloc(sizeof(float) * (size_t)n, st)) != GBK_OK) return r;
  KnnPlan plan;
  // q1(y): nearest coarse centroid (exact, k = 1, ties to the lowest list)
  if ((r = knn_run(x, n, ix->coarse.as<float>(), ix->nlist, ix->d, 1, GBK_METRIC_L2,
                   dist.as<float>(), a.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  flat_stage_kernel<<<grid_for(n), 256, 0, st>>>(a.as<int64_t>(), ids, n, ix->n_staged,
                                                 ix->st_list.as<int32_t>() + ix->n_staged,
                                                 ix->st_ids.as<int64_t>() + ix->n_staged);
  GBK_LAUNCH_CHECK();
  GBK_CUDA_CHECK(cudaMemcpyAsync(ix->st_vecs.as<char>() + row * ix->n_staged, x, row * n,
                                 cudaMemcpyDeviceToDevice, st));
  ix->n_staged += n;
  ix->dirty = true;
  return GBK_OK;
}

gbk_status gbk_ivfflat_search(gbk_ivfflat* ix, const float* xq, int64_t nq, int32_t k,
                              int32_t nprobe, float* D, int64_t* I, void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfflat_search: NULL index");
  GBK_REQUIRE(ix->trained, "gbk_ivfflat_search: index not trained");
  GBK_REQUIRE(k >= 1 && k <= GBK_MAX_K, "gbk_ivfflat_search: k out of [1, %d]", GBK_MAX_K);
  GBK_REQUIRE(nprobe >= 1 && nprobe <= ix->nlist && nprobe <= GBK_MAX_K,
              "gbk_ivfflat_search: nprobe out of [1, min(nlist, %d)]", GBK_MAX_K);
  GBK_REQUIRE(nq >= 0 && nq < (int64_t(1) << 31), "gbk_ivfflat_search: nq out of range");
  if (nq == 0) return GBK_OK;
  GBK_REQUIRE(xq && D && I, "gbk_ivfflat_search: NULL pointer");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = flat_finalize(ix, st)) != GBK_OK) return r;
  Scratch clD, clI;
  if ((r = clD.alloc(sizeof(float) * (size_t)nq * nprobe, st)) != GBK_OK) return r;
  if ((r = clI.alloc(sizeof(int64_t) * (size_t)nq * nprobe, st)) != GBK_OK) return r;
  // Eq. 5: the nprobe nearest coarse centroids
  KnnPlan plan;
  if ((r = knn_run(xq, nq, ix->coarse.as<float>(), ix->nlist, ix->d, nprobe, GBK_METRIC_L2,
                   clD.as<float>(), clI.as<int64_t>(), plan, st)) != GBK_OK)
    return r;
  return ivf_flat_scan_run(xq, nq, ix->d, nprobe, k, clI.as<int64_t>(),
                           ix->list_off.as<int64_t>(), ix->vecs.as<float>(),
                           ix->ids.as<int64_t>(), D, I, st);
}

gbk_status gbk_ivfflat_info(gbk_ivfflat* ix, int64_t* ntotal, int32_t* nlist, int32_t* d,
                            void* stream) {
  clear_error();
  GBK_REQUIRE(ix, "gbk_ivfflat_info: NULL index");
  if (ntotal) *ntotal = ix->n_staged;
  if (nlist) *nlist = ix->nlist;
  if (d) *d = ix->d;
  (void)stream;
  return GBK_OK;
}

gbk_status gbk_ivfflat_export(gbk_ivfflat* ix, float* coarse, int64_t* list_off, int64_t* ids,
                              void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained, "gbk_ivfflat_export: index missing or not trained");
  cudaStream_t st = as_stream(stream);
  gbk_status r;
  if ((r = flat_finalize(ix, st)) != GBK_OK) return r;
  if (coarse)
    GBK_CUDA_CHECK(cudaMemcpyAsync(coarse, ix->coarse.p, ix->coarse.bytes, cudaMemcpyDefault, st));
  if (list_off)
    GBK_CUDA_CHECK(cudaMemcpyAsync(list_off, ix->list_off.p, sizeof(int64_t) * (ix->nlist + 1),
                                   cudaMemcpyDefault, st));
  if (ids && ix->ntotal)
    GBK_CUDA_CHECK(cudaMemcpyAsync(ids, ix->ids.p, sizeof(int64_t) * ix->ntotal, cudaMemcpyDefault,
                                   st));
  return GBK_OK;
}

}  // extern "C"
