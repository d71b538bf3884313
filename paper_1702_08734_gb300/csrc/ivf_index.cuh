// The IVFADC index object and the internal steps shared by its translation units.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "ivf.cuh"

struct gbk_mlp;

struct gbk_index {
  int d = 0, nlist = 0, M = 0, dsub = 0;
  bool trained = false;
  int use_precomputed = 1;
  gbk::DevBuf coarse, pq, T;
  // insertion-order staging: every added vector's list, code and id
  gbk::DevBuf st_list, st_codes, st_ids;
  int64_t n_staged = 0, cap_staged = 0;
  // inverted file (built from the staging arrays on demand): codes rotated by list position
  // (byte s of the code at position r of its list = sub-quantizer (s + r) mod M), and with
  // precomputed tables the term-1 sum s1 of every stored code (Eq. 11)
  gbk::DevBuf list_off, codes, ids, s1;
  // optional float32 copies of the added vectors (exact re-rank): staged, then list order
  bool keep_vectors = false;
  gbk::DevBuf st_vecs, vecs;
  // optional OPQ pre-rotation R [d][d]: every input vector y is replaced by R y
  gbk::DevBuf rot;
  bool rotated = false;
  // arithmetic of the coarse search of queries (Eq. 5); low precision over-fetches and
  // re-ranks the candidate lists in float32, so term 2 stays exact
  int coarse_prec = GBK_PREC_FP32;
  // learned nprobe: the network's class c (argmax, or with route_alpha > 0 the smallest
  // class of cumulative probability >= route_alpha) probes 2^max(c + class_shift, 0) lists
  int class_shift = 0;
  float route_alpha = 0.f;
  int64_t ntotal = 0;
  bool dirty = true;
  int64_t max_list = 0;
  gbk::ScanTuning tuning;  // list-scan launch shape (gbk_ivfpq_autotune / set_tuning)
  ~gbk_index() {
    coarse.release();
    pq.release();
    T.release();
    st_list.release();
    st_codes.release();
    st_ids.release();
    list_off.release();
    codes.release();
    ids.release();
    s1.release();
    st_vecs.release();
    vecs.release();
    rot.release();
  }
};

namespace gbk {

// Algorithm 4 for a validated, finalized index (below).
gbk_status search_run(gbk_index* ix, const float* xq, int64_t nq, int k, int nprobe, float* D,
                      int64_t* I, cudaStream_t st, bool positions = false,
                      bool prerotated = false);

// Rows of x replaced by R y (the OPQ pre-rotation) as the inner-product GEMM x R^T on the
// tensor cores (float32-accurate), in chunks of 2^20 rows; without a rotation *out = x.
gbk_status rotate_rows(const gbk_index* ix, const float* x, int64_t n, Scratch& buf,
                       const float** out, cudaStream_t st);

// Builds the inverted file from the staging arrays when vectors were added since the last
// build (stable by insertion order within a list; codes rotated by list position; term-1
// sums with precomputed tables).
gbk_status finalize_index(gbk_index* ix, cudaStream_t st);

// Mixed batch of Algorithm 4 (per-query k and nprobe, or nprobe from the network mlp).
gbk_status batched_run(gbk_index* ix, const float* xq, int64_t nq, const int32_t* kq, int max_k,
                       const int32_t* npq, int max_nprobe, gbk_mlp* mlp, const int64_t* out_off,
                       float* D, int64_t* I, int32_t* np_used, cudaStream_t st,
                       bool positions = false, bool prerotated = false);

// Network inputs / outputs and argmax classes of a forward pass (mlp.cu).
int mlp_inputs(const gbk_mlp* n);
int mlp_outputs(const gbk_mlp* n);
// alpha > 0: the smallest class whose cumulative softmax probability reaches alpha;
// otherwise the argmax (ties to the lower class).
gbk_status mlp_forward_classes(gbk_mlp* net, const float* X, int64_t B, int32_t* cls,
                               cudaStream_t st, float alpha = 0.f);

// Learned-nprobe features of Eq. 5's nearest coarse distances (ivf.cu):
// F[q] = [x_q, d_i / max(d_0, 1e-12) - 1 for i < nfeat]
gbk_status nprobe_features_run(const float* xq, int64_t nq, int d, const float* clD, int tau,
                               int nfeat, float* F, cudaStream_t st);

}  // namespace gbk
