// Learned nprobe, training side: labels from exact search and the training loop of the
// per-query nprobe network, both inside the library (the search itself is section 5.3's
// Algorithm 4 with the number of probed lists chosen per query; the network is not part
// of the paper).
//
// Label of a training query: with classes c = 0 .. C-1 probing tau_c = min(2^c, nlist)
// lists, r_c = |top-k of the search at tau_c  intersect  exact top-k| (the k-recall@k of
// that query), the label is the smallest c with r_c >= min(ceil(target k), r_{C-1}): the
// fewest lists that reach the target, or the query's own ceiling when the target is out
// of reach at any tau.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "ivf.cuh"
#include "ivf_index.cuh"
#include "knn.cuh"

namespace gbk {
namespace {

// cnt[q] = |{I[q][i] : i < k, I >= 0} intersect {G[q][j] : j < k}|; G has row stride ldg
__global__ void overlap_kernel(const int64_t* __restrict__ I, const int64_t* __restrict__ G,
                               int64_t nq, int k, int ldg, int32_t* __restrict__ cnt) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  int c = 0;
  for (int i = 0; i < k; i++) {
    const int64_t v = I[q * k + i];
    if (v < 0) continue;
    for (int j = 0; j < k; j++)
      if (G[q * ldg + j] == v) {
        c++;
        break;
      }
  }
  cnt[q] = c;
}

// label[q] = smallest c with cnt[c][q] >= min(need, cnt[C-1][q])
__global__ void label_kernel(const int32_t* __restrict__ cnt, int64_t n, int C, int need,
                             int32_t* __restrict__ label) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int goal = min(need, cnt[(int64_t)(C - 1) * n + q]);
  int c = 0;
  while (c < C - 1 && cnt[(int64_t)c * n + q] < goal) c++;
  label[q] = c;
}

__global__ void gather_labels_kernel(const int32_t* __restrict__ y, const int64_t* __restrict__ idx,
                                     int64_t n, int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = y[idx[i]];
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct TrainCfg {
  int C, k, kprime, epochs, batch;
  float target, lr;
  uint64_t seed;
  int64_t chunk;
};

TrainCfg cfg_of(const gbk_nprobe_train_opts* o) {
  TrainCfg c;
  c.C = o && o->n_classes > 0 ? o->n_classes : 9;
  c.k = o && o->k > 0 ? o->k : 10;
  c.kprime = o ? o->kprime : 0;
  c.epochs = o && o->epochs > 0 ? o->epochs : 15;
  c.batch = o && o->batch > 0 ? o->batch : 4096;
  c.target = o && o->target > 0.f ? o->target : 0.95f;
  c.lr = o && o->lr > 0.f ? o->lr : 1e-3f;
  c.seed = o ? o->seed : 0;
  c.chunk = o && o->chunk > 0 ? o->chunk : 20000;
  return c;
}

gbk_status check_cfg(const gbk_index* ix, const TrainCfg& c, const int64_t* gt, int kgt) {
  GBK_REQUIRE(c.C >= 1 && c.C <= 11, "nprobe training: n_classes must be in [1, 11]");
  GBK_REQUIRE(c.k >= 1 && c.k <= GBK_MAX_K, "nprobe training: k out of [1, %d]", GBK_MAX_K);
  GBK_REQUIRE(c.target > 0.f && c.target <= 1.f, "nprobe training: target must be in (0, 1]");
  GBK_REQUIRE(c.kprime == 0 || (c.kprime > c.k && c.kprime <= GBK_MAX_K && ix->keep_vectors),
              "nprobe training: kprime needs k < kprime <= %d and kept vectors", GBK_MAX_K);
  GBK_REQUIRE(gt ? kgt >= c.k : ix->keep_vectors,
              "nprobe training: give the exact neighbours (kgt >= k) or keep the vectors");
  return GBK_OK;
}

// Recall counts cnt [C][n] and labels [n] of the training queries xq (rotated space when
// the index has a rotation: search_run applies it itself).
gbk_status labels_run(gbk_index* ix, const float* xq, int64_t n, const int64_t* gt, int kgt,
                      const TrainCfg& c, int32_t* labels, int32_t* cnt, cudaStream_t st) {
  gbk_status r;
  const int64_t chunk = std::min<int64_t>(c.chunk, n);
  const int kk = c.k;
  Scratch G, D, I, Dc, Ic, Dg, xr;
  if ((r = D.alloc(sizeof(float) * (size_t)chunk * kk, st)) != GBK_OK) return r;
  if ((r = I.alloc(sizeof(int64_t) * (size_t)chunk * kk, st)) != GBK_OK) return r;
  if (!gt) {
    if ((r = G.alloc(sizeof(int64_t) * (size_t)chunk * kk, st)) != GBK_OK) return r;
    if ((r = Dg.alloc(sizeof(float) * (size_t)chunk * kk, st)) != GBK_OK) return r;
  }
  if (c.kprime > 0) {
    if ((r = Dc.alloc(sizeof(float) * (size_t)chunk * c.kprime, st)) != GBK_OK) return r;
    if ((r = Ic.alloc(sizeof(int64_t) * (size_t)chunk * c.kprime, st)) != GBK_OK) return r;
  }
  ProfScope prof("nprobe_labels", st);
  for (int64_t q0 = 0; q0 < n; q0 += chunk) {
    const int64_t nb = std::min(chunk, n - q0);
    const float* xb = xq + q0 * ix->d;
    const float* xbr = xb;  // rotated queries (for the kept vectors and the re-rank)
    if ((r = rotate_rows(ix, xb, nb, xr, &xbr, st)) != GBK_OK) return r;
    const int64_t* g = gt ? gt + q0 * kgt : G.as<int64_t>();
    const int ldg = gt ? kgt : kk;
    if (!gt) {  // exact top-k over the kept vectors (Eq. 1), rows mapped to ids
      KnnPlan plan;
      if ((r = knn_run(xbr, nb, ix->vecs.as<float>(), ix->ntotal, ix->d, kk, GBK_METRIC_L2,
                       Dg.as<float>(), G.as<int64_t>(), plan, st)) != GBK_OK)
        return r;
      if ((r = rows_to_ids_run(G.as<int64_t>(), nb * kk, ix->ids.as<int64_t>(), st)) != GBK_OK)
        return r;
    }
    for (int cl = 0; cl < c.C; cl++) {
      const int tau = std::min(1 << cl, std::min(ix->nlist, GBK_MAX_K));
      if (c.kprime > 0) {
        if ((r = search_run(ix, xbr, nb, c.kprime, tau, Dc.as<float>(), Ic.as<int64_t>(), st,
                            true, true)) != GBK_OK)
          return r;
        if ((r = rerank_rows_run(xbr, ix->vecs.as<float>(), nb, ix->d, c.kprime, kk,
                                 Ic.as<int64_t>(), D.as<float>(), I.as<int64_t>(), st)) != GBK_OK)
          return r;
        if ((r = rows_to_ids_run(I.as<int64_t>(), nb * kk, ix->ids.as<int64_t>(), st)) != GBK_OK)
          return r;
      } else if ((r = search_run(ix, xbr, nb, kk, tau, D.as<float>(), I.as<int64_t>(), st, false,
                                 true)) != GBK_OK) {
        return r;
      }
      overlap_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
          I.as<int64_t>(), g, nb, kk, ldg, cnt + (int64_t)cl * n + q0);
      GBK_LAUNCH_CHECK();
    }
  }
  const int need = (int)std::ceil((double)c.target * kk - 1e-9);
  label_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cnt, n, c.C, need, labels);
  GBK_LAUNCH_CHECK();
  return GBK_OK;
}

}  // namespace
}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_nprobe_labels(gbk_index* ix, const float* xq, int64_t n, const int64_t* gt,
                             int32_t kgt, const gbk_nprobe_train_opts* opts, int32_t* labels,
                             int32_t* counts, void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained, "gbk_nprobe_labels: index missing or not trained");
  GBK_REQUIRE(n >= 0 && n < (int64_t(1) << 31), "gbk_nprobe_labels: n out of range");
  const TrainCfg c = cfg_of(opts);
  gbk_status r = check_cfg(ix, c, gt, kgt);
  if (r != GBK_OK || n == 0) return r;
  GBK_REQUIRE(xq && labels, "gbk_nprobe_labels: NULL pointer");
  cudaStream_t st = as_stream(stream);
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  Scratch cnt;
  int32_t* cp = counts;
  if (!cp) {
    if ((r = cnt.alloc(sizeof(int32_t) * (size_t)n * c.C, st)) != GBK_OK) return r;
    cp = cnt.as<int32_t>();
  }
  return labels_run(ix, xq, n, gt, kgt, c, labels, cp, st);
}

gbk_status gbk_nprobe_mlp_train(gbk_index* ix, gbk_mlp* net, const float* xq, int64_t n,
                                const int32_t* labels, const int64_t* gt, int32_t kgt,
                                const gbk_nprobe_train_opts* opts, float* epoch_loss,
                                void* stream) {
  clear_error();
  GBK_REQUIRE(ix && ix->trained && net, "gbk_nprobe_mlp_train: index or network missing");
  GBK_REQUIRE(n >= 1 && n < (int64_t(1) << 31) && xq, "gbk_nprobe_mlp_train: bad queries");
  const TrainCfg c = cfg_of(opts);
  GBK_REQUIRE(ix->nlist >= 64, "learned nprobe needs nlist >= 64 (64 coarse-distance features)");
  GBK_REQUIRE(mlp_inputs(net) == ix->d + 64, "gbk_nprobe_mlp_train: network inputs must be d + 64");
  GBK_REQUIRE(mlp_outputs(net) == c.C, "gbk_nprobe_mlp_train: network outputs must be n_classes");
  GBK_REQUIRE(c.batch <= n, "gbk_nprobe_mlp_train: batch larger than the training set");
  gbk_status r;
  if (!labels && (r = check_cfg(ix, c, gt, kgt)) != GBK_OK) return r;
  cudaStream_t st = as_stream(stream);
  if ((r = finalize_index(ix, st)) != GBK_OK) return r;
  const int d = ix->d, nf = d + 64;
  Scratch lab, cnt, F, clD, clI, xr, perm, Fb, yb, loss;
  const int32_t* y = labels;
  if (!y) {
    if ((r = lab.alloc(sizeof(int32_t) * (size_t)n, st)) != GBK_OK) return r;
    if ((r = cnt.alloc(sizeof(int32_t) * (size_t)n * c.C, st)) != GBK_OK) return r;
    if ((r = labels_run(ix, xq, n, gt, kgt, c, lab.as<int32_t>(), cnt.as<int32_t>(), st)) !=
        GBK_OK)
      return r;
    y = lab.as<int32_t>();
  }
  // features: the query (rotated space) and its 64 nearest coarse distances (Eq. 5)
  if ((r = F.alloc(sizeof(float) * (size_t)n * nf, st)) != GBK_OK) return r;
  {
    const int64_t chunk = std::min<int64_t>(c.chunk, n);
    if ((r = clD.alloc(sizeof(float) * (size_t)chunk * 64, st)) != GBK_OK) return r;
    if ((r = clI.alloc(sizeof(int64_t) * (size_t)chunk * 64, st)) != GBK_OK) return r;
    for (int64_t q0 = 0; q0 < n; q0 += chunk) {
      const int64_t nb = std::min(chunk, n - q0);
      const float* xbr = xq + q0 * d;
      if ((r = rotate_rows(ix, xq + q0 * d, nb, xr, &xbr, st)) != GBK_OK) return r;
      KnnPlan plan;
      plan.prec = ix->coarse_prec;
      if ((r = knn_run(xbr, nb, ix->coarse.as<float>(), ix->nlist, d, 64, GBK_METRIC_L2,
                       clD.as<float>(), clI.as<int64_t>(), plan, st)) != GBK_OK)
        return r;
      if ((r = nprobe_features_run(xbr, nb, d, clD.as<float>(), 64, 64,
                                   F.as<float>() + q0 * nf, st)) != GBK_OK)
        return r;
    }
  }
  // epochs of Adam over a seeded permutation of the samples (whole batches only)
  const int64_t nbatch = n / c.batch;
  if ((r = perm.alloc(sizeof(int64_t) * (size_t)n * c.epochs, st)) != GBK_OK) return r;
  if ((r = Fb.alloc(sizeof(float) * (size_t)c.batch * nf, st)) != GBK_OK) return r;
  if ((r = yb.alloc(sizeof(int32_t) * (size_t)c.batch, st)) != GBK_OK) return r;
  if ((r = loss.alloc(sizeof(float) * (size_t)std::max<int64_t>(1, nbatch * c.epochs), st)) !=
      GBK_OK)
    return r;
  std::vector<int64_t> order((size_t)n * c.epochs);
  for (int ep = 0; ep < c.epochs; ep++) {  // Fisher-Yates with a counter-based generator
    int64_t* o = order.data() + (size_t)ep * n;
    for (int64_t i = 0; i < n; i++) o[i] = i;
    for (int64_t i = n - 1; i > 0; i--) {
      const uint64_t h = mix64(c.seed * 0x9e3779b97f4a7c15ull + (uint64_t)ep * 0xd1b54a32d192ed03ull +
                               (uint64_t)i);
      const int64_t j = (int64_t)(h % (uint64_t)(i + 1));
      std::swap(o[i], o[j]);
    }
  }
  GBK_CUDA_CHECK(cudaMemcpyAsync(perm.p, order.data(), sizeof(int64_t) * order.size(),
                                 cudaMemcpyHostToDevice, st));
  ProfScope prof("nprobe_mlp_train", st);
  for (int ep = 0; ep < c.epochs; ep++) {
    for (int64_t b = 0; b < nbatch; b++) {
      const int64_t* idx = perm.as<int64_t>() + (int64_t)ep * n + b * c.batch;
      if ((r = gather_rows_run(F.as<float>(), idx, c.batch, nf, Fb.as<float>(), st)) != GBK_OK)
        return r;
      gather_labels_kernel<<<(unsigned)((c.batch + 255) / 256), 256, 0, st>>>(y, idx, c.batch,
                                                                               yb.as<int32_t>());
      GBK_LAUNCH_CHECK();
      if ((r = gbk_mlp_train_step(net, Fb.as<float>(), yb.as<int32_t>(), c.batch, c.lr, 1,
                                  loss.as<float>() + (int64_t)ep * nbatch + b, st)) != GBK_OK)
        return r;
    }
  }
  if (epoch_loss) {
    std::vector<float> h((size_t)std::max<int64_t>(1, nbatch * c.epochs));
    GBK_CUDA_CHECK(cudaMemcpyAsync(h.data(), loss.p, sizeof(float) * h.size(),
                                   cudaMemcpyDeviceToHost, st));
    GBK_CUDA_CHECK(cudaStreamSynchronize(st));
    for (int ep = 0; ep < c.epochs; ep++) {
      double s = 0.0;
      for (int64_t b = 0; b < nbatch; b++) s += h[(size_t)(ep * nbatch + b)];
      epoch_loss[ep] = nbatch ? (float)(s / (double)nbatch) : 0.f;
    }
  }
  return GBK_OK;
}

}  // extern "C"
