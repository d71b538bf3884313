/*
 * CPU oracle for "Billion-scale similarity search with GPUs" (Johnson, Douze, Jegou,
 * arXiv 1702.08734).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the library's compute path never does.
 *
 * Plain, slow and obviously correct: every quantity is evaluated from its definition
 * in double precision from the float32 inputs, with no blocking, fusion or
 * reordering.  It shares no code, header or constant with the CUDA library.
 *
 * Total order used by every selection below (the paper leaves the order of equal
 * keys unspecified, section 2 "k-selection"): a candidate is better than another if
 * its key is smaller (larger for the "largest" comparator), NaN keys are worse than
 * every number in both directions, -0 equals +0, and equal keys are ordered by the
 * lower index / id.
 *
 * Work is split statically over rows or queries onto POSIX threads; the result of
 * each row does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

/* ------------------------------------------------------------------ threads */

typedef void (*range_fn)(void* ctx, int64_t begin, int64_t end);

typedef struct {
  range_fn fn;
  void* ctx;
  int64_t begin, end;
} range_job;

static void* run_range(void* p) {
  range_job* j = (range_job*)p;
  if (j->begin < j->end) j->fn(j->ctx, j->begin, j->end);
  return NULL;
}

int or_default_threads(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n < 1 ? 1 : (int)n;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (nthreads <= 0) nthreads = or_default_threads();
  if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads <= 1) {
    if (n > 0) fn(ctx, 0, n);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  range_job* jobs = (range_job*)malloc(sizeof(range_job) * nthreads);
  for (int t = 0; t < nthreads; t++) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].begin = n * t / nthreads;
    jobs[t].end = n * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, run_range, &jobs[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------- ordering of candidates */

/* Is candidate (va, ia) strictly worse than (vb, ib)?  `largest` flips the value
 * order; NaN is worst in both directions; ties go to the lower index. */
static int worse(double va, int64_t ia, double vb, int64_t ib, int largest) {
  int na = isnan(va), nb = isnan(vb);
  if (na != nb) return na;
  if (!na) {
    if (va != vb) return largest ? (va < vb) : (va > vb);
  }
  return ia > ib;
}

/* Max-heap of the k best candidates seen so far: the root is the worst kept one. */
typedef struct {
  double* v;
  int64_t* id;
  int32_t size, cap;
  int largest;
} kheap;

static void heap_sift_down(kheap* h, int32_t i) {
  for (;;) {
    int32_t l = 2 * i + 1, r = l + 1, w = i;
    if (l < h->size && worse(h->v[l], h->id[l], h->v[w], h->id[w], h->largest)) w = l;
    if (r < h->size && worse(h->v[r], h->id[r], h->v[w], h->id[w], h->largest)) w = r;
    if (w == i) return;
    double tv = h->v[i];
    h->v[i] = h->v[w];
    h->v[w] = tv;
    int64_t ti = h->id[i];
    h->id[i] = h->id[w];
    h->id[w] = ti;
    i = w;
  }
}

static void heap_sift_up(kheap* h, int32_t i) {
  while (i > 0) {
    int32_t p = (i - 1) / 2;
    if (!worse(h->v[i], h->id[i], h->v[p], h->id[p], h->largest)) return;
    double tv = h->v[i];
    h->v[i] = h->v[p];
    h->v[p] = tv;
    int64_t ti = h->id[i];
    h->id[i] = h->id[p];
    h->id[p] = ti;
    i = p;
  }
}

/* Offer a candidate; returns 1 if it entered the kept set (a "successive min-k"
 * event in the Appendix's terminology). */
static int heap_push(kheap* h, double v, int64_t id) {
  if (h->size < h->cap) {
    h->v[h->size] = v;
    h->id[h->size] = id;
    h->size++;
    heap_sift_up(h, h->size - 1);
    return 1;
  }
  if (h->cap == 0 || !worse(h->v[0], h->id[0], v, id, h->largest)) return 0;
  h->v[0] = v;
  h->id[0] = id;
  heap_sift_down(h, 0);
  return 1;
}

/* Pop everything, best first, into (outv, outid); pads the tail with (pad, -1). */
static void heap_drain_sorted(kheap* h, double* outv, int64_t* outid, int32_t k, double pad) {
  int32_t n = h->size;
  for (int32_t j = n; j < k; j++) {
    outv[j] = pad;
    outid[j] = -1;
  }
  for (int32_t j = n - 1; j >= 0; j--) {
    outv[j] = h->v[0];
    outid[j] = h->id[0];
    h->size--;
    if (h->size > 0) {
      h->v[0] = h->v[h->size];
      h->id[0] = h->id[h->size];
      heap_sift_down(h, 0);
    }
  }
}

/* ------------------------------------------------------------- k-selection */
/* Section 2, "k-selection": the k lowest (or highest) valued elements of each
 * row, sorted, with their indices.  method 0: size-k heap over a single pass;
 * method 1: full sort of (value, index) pairs, first k.  Both obey `worse`. */

typedef struct {
  double v;
  int64_t i;
  int largest;
} vi_pair;

static int cmp_pair_small(const void* a, const void* b) {
  const vi_pair* x = (const vi_pair*)a;
  const vi_pair* y = (const vi_pair*)b;
  if (worse(x->v, x->i, y->v, y->i, 0)) return 1;
  if (worse(y->v, y->i, x->v, x->i, 0)) return -1;
  return 0;
}
static int cmp_pair_large(const void* a, const void* b) {
  const vi_pair* x = (const vi_pair*)a;
  const vi_pair* y = (const vi_pair*)b;
  if (worse(x->v, x->i, y->v, y->i, 1)) return 1;
  if (worse(y->v, y->i, x->v, x->i, 1)) return -1;
  return 0;
}

typedef struct {
  const float* vals;
  int64_t len;
  int32_t k, largest, method;
  float* outD;
  int64_t* outI;
  int64_t* events; /* per-row count of heap entries, may be NULL */
} ksel_ctx;

static void ksel_rows(void* p, int64_t r0, int64_t r1) {
  ksel_ctx* c = (ksel_ctx*)p;
  int32_t k = c->k;
  if (c->method == 1) {
    vi_pair* a = (vi_pair*)malloc(sizeof(vi_pair) * (size_t)(c->len > 0 ? c->len : 1));
    for (int64_t r = r0; r < r1; r++) {
      const float* row = c->vals + r * c->len;
      for (int64_t i = 0; i < c->len; i++) {
        a[i].v = row[i];
        a[i].i = i;
      }
      qsort(a, (size_t)c->len, sizeof(vi_pair), c->largest ? cmp_pair_large : cmp_pair_small);
      for (int32_t j = 0; j < k; j++) {
        if (j < c->len) {
          c->outD[r * k + j] = row[a[j].i];
          c->outI[r * k + j] = a[j].i;
        } else {
          c->outD[r * k + j] = NAN;
          c->outI[r * k + j] = -1;
        }
      }
    }
    free(a);
    return;
  }
  kheap h;
  h.v = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
  double* tv = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  h.cap = k;
  h.largest = c->largest;
  for (int64_t r = r0; r < r1; r++) {
    const float* row = c->vals + r * c->len;
    h.size = 0;
    int64_t ev = 0;
    for (int64_t i = 0; i < c->len; i++) ev += heap_push(&h, (double)row[i], i);
    if (c->events) c->events[r] = ev;
    heap_drain_sorted(&h, tv, c->outI + r * k, k, NAN);
    for (int32_t j = 0; j < k; j++) {
      int64_t ix = c->outI[r * k + j];
      c->outD[r * k + j] = ix >= 0 ? row[ix] : NAN; /* the input's own bits */
    }
  }
  free(h.v);
  free(h.id);
  free(tv);
}

int or_kselect(const float* vals, int64_t rows, int64_t len, int32_t k, int32_t largest,
               int32_t method, float* outD, int64_t* outI, int64_t* events, int nthreads) {
  if (rows < 0 || len < 0 || k < 0) return OR_EINVAL;
  ksel_ctx c = {vals, len, k, largest, method, outD, outI, events};
  parallel_for(rows, nthreads, ksel_rows, &c);
  return OR_OK;
}

/* ---------------------------------------------------- exact k-NN, Eq. (1) */
/* The full distance ||x - y||^2 (or <x, y> for the inner-product metric) is
 * evaluated directly for every pair, in double precision - not through the
 * norm decomposition of Eq. (2) that the GPU path uses. */

typedef struct {
  const float *xq, *xb;
  int64_t nb;
  int32_t d, k, metric;
  double* outD;
  int64_t* outI;
} knn_ctx;

static void knn_rows(void* p, int64_t q0, int64_t q1) {
  knn_ctx* c = (knn_ctx*)p;
  kheap h;
  int32_t k = c->k;
  h.v = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
  h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
  h.cap = k;
  h.largest = (c->metric == 1);
  for (int64_t q = q0; q < q1; q++) {
    const float* x = c->xq + q * c->d;
    h.size = 0;
    for (int64_t i = 0; i < c->nb; i++) {
      const float* y = c->xb + i * c->d;
      double s = 0.0;
      if (c->metric == 1) {
        for (int32_t t = 0; t < c->d; t++) s += (double)x[t] * (double)y[t];
      } else {
        for (int32_t t = 0; t < c->d; t++) {
          double e = (double)x[t] - (double)y[t];
          s += e * e;
        }
      }
      heap_push(&h, s, i);
    }
    heap_drain_sorted(&h, c->outD + q * k, c->outI + q * k, k,
                      c->metric == 1 ? -INFINITY : INFINITY);
  }
  free(h.v);
  free(h.id);
}

int or_knn(const float* xq, int64_t nq, const float* xb, int64_t nb, int32_t d, int32_t k,
           int32_t metric, double* outD, int64_t* outI, int nthreads) {
  if (nq < 0 || nb < 0 || d <= 0 || k < 0 || (metric != 0 && metric != 1)) return OR_EINVAL;
  knn_ctx c = {xq, xb, nb, d, k, metric, outD, outI};
  parallel_for(nq, nthreads, knn_rows, &c);
  return OR_OK;
}

/* Exact distances of given (query, database id) pairs, one by one. */
int or_pair_dist(const float* xq, const float* xb, int32_t d, const int64_t* qi,
                 const int64_t* bi, int64_t n, int32_t metric, double* out) {
  for (int64_t p = 0; p < n; p++) {
    const float* x = xq + qi[p] * d;
    const float* y = xb + bi[p] * d;
    double s = 0.0;
    for (int32_t t = 0; t < d; t++) {
      if (metric == 1) {
        s += (double)x[t] * (double)y[t];
      } else {
        double e = (double)x[t] - (double)y[t];
        s += e * e;
      }
    }
    out[p] = s;
  }
  return OR_OK;
}

/* ------------------------------------------------- nearest-centroid assign */
/* argmin_j ||x_i - c_j||^2 in double, ties to the lowest j (k-means assignment,
 * the coarse quantizer q1 of Eq. (3), and the first step of Eq. (5) with tau=1). */

typedef struct {
  const float *x, *c;
  int32_t d, nc;
  int64_t* assign;
  double* dist;
} assign_ctx;

static void assign_rows(void* p, int64_t i0, int64_t i1) {
  assign_ctx* a = (assign_ctx*)p;
  for (int64_t i = i0; i < i1; i++) {
    const float* x = a->x + i * a->d;
    double best = INFINITY;
    int64_t bj = -1;
    for (int32_t j = 0; j < a->nc; j++) {
      const float* c = a->c + (int64_t)j * a->d;
      double s = 0.0;
      for (int32_t t = 0; t < a->d; t++) {
        double e = (double)x[t] - (double)c[t];
        s += e * e;
      }
      if (bj < 0 || s < best) {
        best = s;
        bj = j;
      }
    }
    a->assign[i] = bj;
    if (a->dist) a->dist[i] = best;
  }
}

int or_assign(const float* x, int64_t n, int32_t d, const float* cent, int32_t nc,
              int64_t* assign, double* dist, int nthreads) {
  if (n < 0 || d <= 0 || nc <= 0) return OR_EINVAL;
  assign_ctx a = {x, cent, d, nc, assign, dist};
  parallel_for(n, nthreads, assign_rows, &a);
  return OR_OK;
}

/* ------------------------------------------------------ Lloyd's k-means */
/* Section 2 ("trained via k-means") and section 6.2 (assignment = exact search
 * with k=1).  Centroids are float32 between iterations; each update is the double
 * precision mean of the members, rounded once.  Readings where the paper is
 * silent: initial centroids are given rows of x (a seeded permutation's prefix);
 * an empty cluster e (in ascending order) is re-seeded by splitting the cluster s
 * with the largest member count (ties: lowest index): for every dimension t with
 * sign g_t = +1 (t even) or -1 (t odd), c_e[t] = c_s[t]*(1 + g_t/1024) and
 * c_s[t] = c_s[t]*(1 - g_t/1024), then count_e = count_s/2, count_s -= count_e. */

int or_kmeans(const float* x, int64_t n, int32_t d, int32_t nc, int32_t niter,
              const int64_t* init_idx, float* centroids, double* objective,
              int64_t* n_split, int nthreads) {
  if (n < 1 || d <= 0 || nc <= 0 || niter < 0) return OR_EINVAL;
  for (int32_t j = 0; j < nc; j++) {
    if (init_idx[j] < 0 || init_idx[j] >= n) return OR_EINVAL;
    memcpy(centroids + (int64_t)j * d, x + init_idx[j] * d, sizeof(float) * (size_t)d);
  }
  int64_t* assign = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  double* dist = (double*)malloc(sizeof(double) * (size_t)n);
  double* sum = (double*)malloc(sizeof(double) * (size_t)nc * (size_t)d);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)nc);
  if (!assign || !dist || !sum || !cnt) return OR_ENOMEM;
  int64_t splits = 0;
  for (int32_t it = 0; it < niter; it++) {
    or_assign(x, n, d, centroids, nc, assign, dist, nthreads);
    double obj = 0.0;
    for (int64_t i = 0; i < n; i++) obj += dist[i];
    if (objective) objective[it] = obj;
    memset(sum, 0, sizeof(double) * (size_t)nc * (size_t)d);
    memset(cnt, 0, sizeof(int64_t) * (size_t)nc);
    for (int64_t i = 0; i < n; i++) {
      int64_t j = assign[i];
      cnt[j]++;
      for (int32_t t = 0; t < d; t++) sum[j * d + t] += (double)x[i * d + t];
    }
    for (int32_t j = 0; j < nc; j++) {
      if (cnt[j] == 0) continue;
      for (int32_t t = 0; t < d; t++)
        centroids[(int64_t)j * d + t] = (float)(sum[(int64_t)j * d + t] / (double)cnt[j]);
    }
    for (int32_t e = 0; e < nc; e++) {
      if (cnt[e] != 0) continue;
      int32_t s = 0;
      for (int32_t j = 1; j < nc; j++)
        if (cnt[j] > cnt[s]) s = j;
      for (int32_t t = 0; t < d; t++) {
        double g = (t % 2 == 0) ? 1.0 : -1.0;
        double cs = (double)centroids[(int64_t)s * d + t];
        centroids[(int64_t)e * d + t] = (float)(cs * (1.0 + g / 1024.0));
        centroids[(int64_t)s * d + t] = (float)(cs * (1.0 - g / 1024.0));
      }
      cnt[e] = cnt[s] / 2;
      cnt[s] -= cnt[e];
      splits++;
    }
  }
  if (n_split) *n_split = splits;
  free(assign);
  free(dist);
  free(sum);
  free(cnt);
  return OR_OK;
}

/* ------------------------------------------- IVFADC encoding, Eq. (3) + PQ */
/* q1(y) = nearest coarse centroid; residual r = y - q1(y) (in double); the product
 * quantizer splits r into M sub-vectors of d/M consecutive dimensions and byte m of
 * the code is the nearest of the 256 centroids of sub-quantizer m (section 2,
 * "Product quantizer"; ties to the lowest centroid).  pq is [M][256][d/M]. */

typedef struct {
  const float *x, *coarse, *pq;
  int32_t d, nlist, M;
  int64_t* list_of;
  uint8_t* codes;
} enc_ctx;

static void enc_rows(void* p, int64_t i0, int64_t i1) {
  enc_ctx* e = (enc_ctx*)p;
  int32_t dsub = e->d / e->M;
  double* r = (double*)malloc(sizeof(double) * (size_t)e->d);
  for (int64_t i = i0; i < i1; i++) {
    const float* y = e->x + i * e->d;
    int64_t L = -1;
    double best = INFINITY;
    for (int32_t j = 0; j < e->nlist; j++) {
      const float* c = e->coarse + (int64_t)j * e->d;
      double s = 0.0;
      for (int32_t t = 0; t < e->d; t++) {
        double df = (double)y[t] - (double)c[t];
        s += df * df;
      }
      if (L < 0 || s < best) {
        best = s;
        L = j;
      }
    }
    e->list_of[i] = L;
    const float* cL = e->coarse + L * e->d;
    for (int32_t t = 0; t < e->d; t++) r[t] = (double)y[t] - (double)cL[t];
    for (int32_t m = 0; m < e->M; m++) {
      int32_t bc = -1;
      double bd = INFINITY;
      for (int32_t c = 0; c < 256; c++) {
        const float* C = e->pq + ((int64_t)m * 256 + c) * dsub;
        double s = 0.0;
        for (int32_t t = 0; t < dsub; t++) {
          double df = r[m * dsub + t] - (double)C[t];
          s += df * df;
        }
        if (bc < 0 || s < bd) {
          bd = s;
          bc = c;
        }
      }
      e->codes[i * e->M + m] = (uint8_t)bc;
    }
  }
  free(r);
}

int or_ivfpq_encode(const float* x, int64_t n, int32_t d, const float* coarse, int32_t nlist,
                    const float* pq, int32_t M, int64_t* list_of, uint8_t* codes, int nthreads) {
  if (n < 0 || d <= 0 || M <= 0 || d % M != 0 || nlist <= 0) return OR_EINVAL;
  enc_ctx e = {x, coarse, pq, d, nlist, M, list_of, codes};
  parallel_for(n, nthreads, enc_rows, &e);
  return OR_OK;
}

/* Inverted file (section 2): list L holds, in insertion order, the positions of
 * the vectors with q1 = L.  offsets has nlist+1 entries; order[offsets[L]..] are
 * positions 0..n-1 of the added batch. */
int or_ivf_bucket(const int64_t* list_of, int64_t n, int32_t nlist, int64_t* offsets,
                  int64_t* order) {
  if (nlist <= 0 || n < 0) return OR_EINVAL;
  for (int32_t L = 0; L <= nlist; L++) offsets[L] = 0;
  for (int64_t i = 0; i < n; i++) {
    if (list_of[i] < 0 || list_of[i] >= nlist) return OR_EINVAL;
    offsets[list_of[i] + 1]++;
  }
  for (int32_t L = 0; L < nlist; L++) offsets[L + 1] += offsets[L];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nlist);
  for (int32_t L = 0; L < nlist; L++) fill[L] = offsets[L];
  for (int64_t i = 0; i < n; i++) order[fill[list_of[i]]++] = i;
  free(fill);
  return OR_OK;
}

/* ------------------------------------------- IVFADC search, Algorithm 4 */
/* For each query: L_IVF = the nprobe nearest coarse centroids (Eq. 5; exact double
 * distances, ties to the lower list number); every vector of every probed list gets
 * the ADC distance ||x - q(y)||^2 (Eq. 6 with Eq. 3).  form 0 evaluates it as the
 * distance to the reconstruction q1(y) + q2(y - q1(y)); form 1 as the sum of b
 * look-ups in tables T_m[c] = ||(x - q1(y))^m - C_m[c]||^2 (Eq. 10).  The k
 * smallest (distance, id) pairs are kept; missing results are (+inf, -1). */

typedef struct {
  const float *xq, *coarse, *pq;
  int32_t d, nlist, M, k, nprobe, form;
  const int64_t* offsets;
  const uint8_t* codes;
  const int64_t* ids;
  double* outD;
  int64_t* outI;
  int64_t* probes; /* [nq][nprobe] chosen lists, may be NULL */
} ivf_ctx;

static void ivf_rows(void* p, int64_t q0, int64_t q1) {
  ivf_ctx* c = (ivf_ctx*)p;
  int32_t d = c->d, M = c->M, dsub = d / M;
  kheap coarse_h, h;
  coarse_h.v = (double*)malloc(sizeof(double) * (size_t)c->nprobe);
  coarse_h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->nprobe);
  coarse_h.cap = c->nprobe;
  coarse_h.largest = 0;
  h.v = (double*)malloc(sizeof(double) * (size_t)(c->k > 0 ? c->k : 1));
  h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(c->k > 0 ? c->k : 1));
  h.cap = c->k;
  h.largest = 0;
  double* cd = (double*)malloc(sizeof(double) * (size_t)c->nprobe);
  int64_t* cl = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->nprobe);
  double* xr = (double*)malloc(sizeof(double) * (size_t)d);
  double* T = (double*)malloc(sizeof(double) * (size_t)M * 256);
  for (int64_t q = q0; q < q1; q++) {
    const float* x = c->xq + q * d;
    coarse_h.size = 0;
    for (int32_t L = 0; L < c->nlist; L++) {
      const float* cc = c->coarse + (int64_t)L * d;
      double s = 0.0;
      for (int32_t t = 0; t < d; t++) {
        double e = (double)x[t] - (double)cc[t];
        s += e * e;
      }
      heap_push(&coarse_h, s, L);
    }
    heap_drain_sorted(&coarse_h, cd, cl, c->nprobe, INFINITY);
    if (c->probes) memcpy(c->probes + q * c->nprobe, cl, sizeof(int64_t) * (size_t)c->nprobe);
    h.size = 0;
    for (int32_t pi = 0; pi < c->nprobe; pi++) {
      int64_t L = cl[pi];
      if (L < 0) continue;
      const float* cL = c->coarse + L * d;
      for (int32_t t = 0; t < d; t++) xr[t] = (double)x[t] - (double)cL[t];
      if (c->form == 1) {
        for (int32_t m = 0; m < M; m++)
          for (int32_t cc = 0; cc < 256; cc++) {
            const float* C = c->pq + ((int64_t)m * 256 + cc) * dsub;
            double s = 0.0;
            for (int32_t t = 0; t < dsub; t++) {
              double e = xr[m * dsub + t] - (double)C[t];
              s += e * e;
            }
            T[m * 256 + cc] = s;
          }
      }
      for (int64_t j = c->offsets[L]; j < c->offsets[L + 1]; j++) {
        const uint8_t* code = c->codes + j * M;
        double s = 0.0;
        if (c->form == 1) {
          for (int32_t m = 0; m < M; m++) s += T[m * 256 + code[m]];
        } else {
          for (int32_t m = 0; m < M; m++) {
            const float* C = c->pq + ((int64_t)m * 256 + code[m]) * dsub;
            for (int32_t t = 0; t < dsub; t++) {
              /* x - (q1(y) + q2(residual)) */
              double e = (double)x[m * dsub + t] - ((double)cL[m * dsub + t] + (double)C[t]);
              s += e * e;
            }
          }
        }
        heap_push(&h, s, c->ids[j]);
      }
    }
    heap_drain_sorted(&h, c->outD + q * c->k, c->outI + q * c->k, c->k, INFINITY);
  }
  free(coarse_h.v);
  free(coarse_h.id);
  free(h.v);
  free(h.id);
  free(cd);
  free(cl);
  free(xr);
  free(T);
}

int or_ivfadc_search(const float* xq, int64_t nq, int32_t d, const float* coarse, int32_t nlist,
                     const float* pq, int32_t M, const int64_t* offsets, const uint8_t* codes,
                     const int64_t* ids, int32_t k, int32_t nprobe, int32_t form, double* outD,
                     int64_t* outI, int64_t* probes, int nthreads) {
  if (nq < 0 || d <= 0 || M <= 0 || d % M != 0 || k < 0 || nprobe < 1 || nprobe > nlist)
    return OR_EINVAL;
  ivf_ctx c = {xq, coarse, pq, d, nlist, M, k, nprobe, form, offsets, codes, ids,
               outD, outI, probes};
  parallel_for(nq, nthreads, ivf_rows, &c);
  return OR_OK;
}

/* ------------------------------------------------------------------ IVF-Flat search */
/* The inverted file of section 2 with the vectors themselves in the lists: the nprobe
 * nearest centroids by exact double distance (ties to the lower list), then Eq. (1)
 * evaluated directly for every vector of those lists, k smallest by (distance, id). */
typedef struct {
  const float *xq, *coarse, *vecs;
  int32_t d, nlist, k, nprobe;
  const int64_t* offsets;
  const int64_t* ids;
  double* outD;
  int64_t* outI;
} flat_ctx;

static void flat_rows(void* p, int64_t q0, int64_t q1) {
  flat_ctx* c = (flat_ctx*)p;
  const int32_t d = c->d;
  kheap coarse_h, h;
  coarse_h.v = (double*)malloc(sizeof(double) * (size_t)c->nprobe);
  coarse_h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->nprobe);
  coarse_h.cap = c->nprobe;
  coarse_h.largest = 0;
  h.v = (double*)malloc(sizeof(double) * (size_t)(c->k > 0 ? c->k : 1));
  h.id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(c->k > 0 ? c->k : 1));
  h.cap = c->k;
  h.largest = 0;
  double* cd = (double*)malloc(sizeof(double) * (size_t)c->nprobe);
  int64_t* cl = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->nprobe);
  for (int64_t q = q0; q < q1; q++) {
    const float* x = c->xq + q * d;
    coarse_h.size = 0;
    for (int32_t L = 0; L < c->nlist; L++) {
      const float* cc = c->coarse + (int64_t)L * d;
      double s = 0.0;
      for (int32_t t = 0; t < d; t++) {
        double e = (double)x[t] - (double)cc[t];
        s += e * e;
      }
      heap_push(&coarse_h, s, L);
    }
    heap_drain_sorted(&coarse_h, cd, cl, c->nprobe, INFINITY);
    h.size = 0;
    for (int32_t pi = 0; pi < c->nprobe; pi++) {
      const int64_t L = cl[pi];
      if (L < 0) continue;
      for (int64_t j = c->offsets[L]; j < c->offsets[L + 1]; j++) {
        const float* y = c->vecs + j * d;
        double s = 0.0;
        for (int32_t t = 0; t < d; t++) {
          double e = (double)x[t] - (double)y[t];
          s += e * e;
        }
        heap_push(&h, s, c->ids[j]);
      }
    }
    heap_drain_sorted(&h, c->outD + q * c->k, c->outI + q * c->k, c->k, INFINITY);
  }
  free(coarse_h.v);
  free(coarse_h.id);
  free(h.v);
  free(h.id);
  free(cd);
  free(cl);
}

int or_ivfflat_search(const float* xq, int64_t nq, int32_t d, const float* coarse, int32_t nlist,
                      const int64_t* offsets, const float* vecs, const int64_t* ids, int32_t k,
                      int32_t nprobe, double* outD, int64_t* outI, int nthreads) {
  if (nq < 0 || d <= 0 || k < 0 || nprobe < 1 || nprobe > nlist) return OR_EINVAL;
  flat_ctx c = {xq, coarse, vecs, d, nlist, k, nprobe, offsets, ids, outD, outI};
  parallel_for(nq, nthreads, flat_rows, &c);
  return OR_OK;
}
