// Pruning and selection pipeline (Sections 3.4, 4 and 5).
//
// Device: normalisation of the benchmark table, k-means clustering of the
// normalised performance vectors (one thread block per seeded restart), and
// the held-out geometric-mean score.  Host (offline, microseconds): cluster
// representatives, the Top-N baseline and CART training of the classifier
// whose nodes the launcher walks.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ks {

// ------------------------------------------------------------------ Section 3.4
__global__ void normalise_kernel(int64_t n_rows, int n_cols, const float* perf, float* out, int mode) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n_rows) return;
  const float* p = perf + row * n_cols;
  float best = 0.f;
  for (int c = lane; c < n_cols; c += 32) best = fmaxf(best, p[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(0xffffffffu, best, o));
  for (int c = lane; c < n_cols; c += 32) {
    float x = best > 0.f ? p[c] / best : 0.f;
    if (mode == 1) {
      x = x < 0.9f ? 0.f : x;
    } else if (mode == 2) {
      x = x < 0.9f ? 0.f : (x - 0.9f) / 0.1f;
    } else if (mode == 3) {
      x = 1.f / (1.f + expf(50.f * (0.85f - x)));
    }
    out[row * n_cols + c] = x;
  }
}

// ------------------------------------------------------------------ Section 4.1
constexpr int kKmThreads = 512;

struct KmArgs {
  int n, d, k, max_iter;
  float tol;
  const float* X;
  const uint32_t* draws;  // n_init x k
  float* centres;         // n_init x k x d
  float* newc;            // n_init x k x d
  int* labels;            // n_init x n
  float* d2;              // n_init x n
  float* inertia;         // n_init
  int* iters;             // n_init
};

__device__ float km_block_sum(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? sh[l] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[32] = v;
  }
  __syncthreads();
  return sh[32];
}

__device__ __forceinline__ float sqdist(const float* x, const float* c, int d) {
  float s = 0.f;
  for (int j = 0; j < d; ++j) {
    const float t = x[j] - c[j];
    s = fmaf(t, t, s);
  }
  return s;
}

__global__ void __launch_bounds__(kKmThreads) kmeans_kernel(const KmArgs a) {
  __shared__ float sh[33];
  __shared__ float scan[kKmThreads];
  __shared__ int pick_sh;
  extern __shared__ int counts[];  // k
  const int r = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
  const int n = a.n, d = a.d, k = a.k;
  const float* X = a.X;
  float* C = a.centres + (int64_t)r * k * d;
  float* NC = a.newc + (int64_t)r * k * d;
  int* lab = a.labels + (int64_t)r * n;
  float* d2 = a.d2 + (int64_t)r * n;
  const uint32_t* u = a.draws + (int64_t)r * k;

  // tol_abs = tol * mean over dimensions of the population variance.
  float vsum = 0.f;
  for (int j = tid; j < d; j += T) {
    float m = 0.f;
    for (int i = 0; i < n; ++i) m += X[(int64_t)i * d + j];
    m /= (float)n;
    float v = 0.f;
    for (int i = 0; i < n; ++i) {
      const float t = X[(int64_t)i * d + j] - m;
      v = fmaf(t, t, v);
    }
    vsum += v / (float)n;
  }
  const float tol_abs = a.tol * km_block_sum(vsum, sh) / (float)d;

  // k-means++ seeding (Arthur & Vassilvitskii) from the given draws.
  int idx = (int)(((uint64_t)u[0] * (uint64_t)n) >> 32);
  for (int j = tid; j < d; j += T) C[j] = X[(int64_t)idx * d + j];
  __syncthreads();
  for (int i = tid; i < n; i += T) d2[i] = sqdist(X + (int64_t)i * d, C, d);
  __syncthreads();
  const int chunk = (n + T - 1) / T;
  for (int c = 1; c < k; ++c) {
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    float s = 0.f;
    for (int i = lo; i < hi; ++i) s += d2[i];
    scan[tid] = s;
    __syncthreads();
    if (tid == 0) {  // exclusive scan of the per-thread chunk sums, in thread order
      float run = 0.f;
      for (int t = 0; t < T; ++t) {
        const float v = scan[t];
        scan[t] = run;
        run += v;
      }
      sh[32] = run;
      pick_sh = -1;
    }
    __syncthreads();
    const float total = sh[32];
    int pick;
    if (total > 0.f) {
      const float target = (float)u[c] * 2.3283064365386963e-10f * total;
      float run = scan[tid];
      if (lo < hi && run <= target && run + s > target) {
        for (int i = lo; i < hi; ++i) {
          run += d2[i];
          if (run > target) {
            pick_sh = i;
            break;
          }
        }
      }
      __syncthreads();
      pick = pick_sh < 0 ? n - 1 : pick_sh;
    } else {
      pick = (int)(((uint64_t)u[c] * (uint64_t)n) >> 32);
    }
    for (int j = tid; j < d; j += T) C[(int64_t)c * d + j] = X[(int64_t)pick * d + j];
    __syncthreads();
    for (int i = tid; i < n; i += T) d2[i] = fminf(d2[i], sqdist(X + (int64_t)i * d, C + (int64_t)c * d, d));
    __syncthreads();
  }

  // Lloyd's iterations.
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    for (int i = tid; i < n; i += T) {
      const float* x = X + (int64_t)i * d;
      int best = 0;
      float bd = sqdist(x, C, d);
      for (int c = 1; c < k; ++c) {
        const float t = sqdist(x, C + (int64_t)c * d, d);
        if (t < bd) { bd = t; best = c; }
      }
      lab[i] = best;
    }
    for (int c = tid; c < k; c += T) counts[c] = 0;
    __syncthreads();
    for (int i = tid; i < n; i += T) atomicAdd(&counts[lab[i]], 1);
    __syncthreads();
    float shift = 0.f;
    for (int j = tid; j < d; j += T) {  // each thread owns dimension j of every centre
      for (int c = 0; c < k; ++c) NC[(int64_t)c * d + j] = 0.f;
      for (int i = 0; i < n; ++i) NC[(int64_t)lab[i] * d + j] += X[(int64_t)i * d + j];
      for (int c = 0; c < k; ++c) {
        const float old = C[(int64_t)c * d + j];
        const float nv = counts[c] > 0 ? NC[(int64_t)c * d + j] / (float)counts[c] : old;
        shift = fmaf(nv - old, nv - old, shift);
        C[(int64_t)c * d + j] = nv;
      }
    }
    shift = km_block_sum(shift, sh);
    if (shift <= tol_abs) break;
  }
  if (it > a.max_iter) it = a.max_iter;
  float in = 0.f;
  for (int i = tid; i < n; i += T) {
    const float* x = X + (int64_t)i * d;
    int best = 0;
    float bd = sqdist(x, C, d);
    for (int c = 1; c < k; ++c) {
      const float t = sqdist(x, C + (int64_t)c * d, d);
      if (t < bd) { bd = t; best = c; }
    }
    lab[i] = best;
    in += bd;
  }
  in = km_block_sum(in, sh);
  if (tid == 0) {
    a.inertia[r] = in;
    a.iters[r] = it;
  }
}

// ------------------------------------------------------------------ Section 4.3
constexpr int kScoreThreads = 256;

struct ScoreArgs {
  int n_rows, n_cols, n_deployed;
  int deployed[GEMM_MAX_DEPLOYED];
  const float* perf;
  const int* chosen;  // column per row, or null
  float floor_;
  float* out;  // [geomean, mean, clamped]
};

__global__ void __launch_bounds__(kScoreThreads) score_kernel(const ScoreArgs a) {
  __shared__ float sh[33];
  float slog = 0.f, s = 0.f, cl = 0.f;
  for (int r = threadIdx.x; r < a.n_rows; r += blockDim.x) {
    const float* p = a.perf + (int64_t)r * a.n_cols;
    float best = 0.f;
    for (int c = 0; c < a.n_cols; ++c) best = fmaxf(best, p[c]);
    float got;
    if (a.chosen) {
      got = p[a.chosen[r]];
    } else if (a.n_deployed > 0) {
      got = 0.f;
      for (int q = 0; q < a.n_deployed; ++q) got = fmaxf(got, p[a.deployed[q]]);
    } else {
      got = best;
    }
    const float ratio = best > 0.f ? got / best : 0.f;
    s += ratio;
    cl += ratio < a.floor_ ? 1.f : 0.f;
    slog += logf(fmaxf(ratio, a.floor_));
  }
  slog = km_block_sum(slog, sh);
  s = km_block_sum(s, sh);
  cl = km_block_sum(cl, sh);
  if (threadIdx.x == 0) {
    a.out[0] = expf(slog / (float)a.n_rows);
    a.out[1] = s / (float)a.n_rows;
    a.out[2] = cl;
  }
}

// ------------------------------------------------------------------ k-NN (Section 5.1 comparison)
constexpr int kKnnMax = 16;

// One thread per query: the k nearest training points (squared Euclidean
// distance over d features; ties to the lower training index), then the
// majority label (ties to the label of the nearest among the tied).
__global__ void knn_kernel(int n_train, int n_query, int d, const float* train, const int* labels,
                           const float* query, int k, int* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_query) return;
  float bd[kKnnMax];
  int bi[kKnnMax];
  for (int j = 0; j < k; ++j) {
    bd[j] = CUDART_INF_F;
    bi[j] = -1;
  }
  const float* x = query + (int64_t)q * d;
  for (int i = 0; i < n_train; ++i) {
    const float* t = train + (int64_t)i * d;
    float dist = 0.f;
    for (int f = 0; f < d; ++f) {
      const float u = x[f] - t[f];
      dist = fmaf(u, u, dist);
    }
    if (dist < bd[k - 1]) {  // insert, keeping (distance, index) order; equal distances keep the earlier point
      int j = k - 1;
      while (j > 0 && bd[j - 1] > dist) {
        bd[j] = bd[j - 1];
        bi[j] = bi[j - 1];
        --j;
      }
      bd[j] = dist;
      bi[j] = i;
    }
  }
  int best = -1, best_count = 0;
  for (int j = 0; j < k; ++j) {  // candidates in nearest-first order
    if (bi[j] < 0) continue;
    const int lab = labels[bi[j]];
    int c = 0;
    for (int m = 0; m < k; ++m)
      if (bi[m] >= 0 && labels[bi[m]] == lab) ++c;
    if (c > best_count) {
      best = lab;
      best_count = c;
    }
  }
  out[q] = best;
}

static gemm_status_t cuda_fail(cudaError_t e) {
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
}

// ------------------------------------------------------------------ cluster geometric means (Section 4.2)
// One thread per (cluster, configuration): log-mean over the cluster's rows in row order.
__global__ void cluster_geomean_kernel(int n, int d, const float* X, const int32_t* labels, int k, float floor,
                                       float* out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)k * d;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / d), j = (int)(t - (int64_t)c * d);
    double acc = 0.0;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
      if (labels[i] != c) continue;
      acc += log((double)fmaxf(X[(int64_t)i * d + j], floor));
      ++cnt;
    }
    out[t] = cnt ? (float)exp(acc / cnt) : 0.f;
  }
}

// ------------------------------------------------------------------ CART (Section 5.1)
struct TreeBuilder {
  const double* F;
  const int32_t* y;
  int n_classes, max_depth, min_leaf, max_nodes;
  std::vector<gemm_tree_node_t> nodes;
  bool overflow = false;
  static constexpr int kF = GEMM_TREE_FEATURES;
  int max_features = kF;            // < kF: random-forest node feature subsets
  const uint32_t* draws = nullptr;  // kF per node, in node (preorder) order

  // 1 - sum_c (cnt_c / n)^2, summed in class order.
  double gini(const std::vector<double>& cnt, double n) const {
    double s = 0.0;
    for (int c = 0; c < n_classes; ++c) {
      const double p = cnt[c] / n;
      s = s + p * p;
    }
    return 1.0 - s;
  }

  int grow(std::vector<int>& idx, int depth) {
    std::vector<int> counts(n_classes, 0);
    for (int i : idx) counts[y[i]]++;
    int label = 0;
    for (int c = 1; c < n_classes; ++c)
      if (counts[c] > counts[label]) label = c;
    const int me = (int)nodes.size();
    if (me >= max_nodes) {
      overflow = true;
      return me;
    }
    nodes.push_back(gemm_tree_node_t{-1, -1, -1, label, 0.0});
    const int n = (int)idx.size();
    if (counts[label] == n || (max_depth >= 0 && depth >= max_depth)) return me;
    // Features this node may split on: all, or the first max_features entries of a
    // partial Fisher-Yates shuffle driven by the node's draws, taken in order.
    bool allowed[kF];
    for (int f = 0; f < kF; ++f) allowed[f] = true;
    if (max_features < kF) {
      int perm[kF];
      for (int f = 0; f < kF; ++f) perm[f] = f;
      for (int t = 0; t < max_features; ++t) {
        const int j = t + (int)(draws[kF * (size_t)me + t] % (uint32_t)(kF - t));
        std::swap(perm[t], perm[j]);
      }
      for (int f = 0; f < kF; ++f) allowed[f] = false;
      for (int t = 0; t < max_features; ++t) allowed[perm[t]] = true;
    }
    // Best split: features in order, thresholds ascending, first best kept.
    int bf = -1;
    double bt = 0.0, bw = 0.0;
    std::vector<int> order(idx);
    std::vector<double> cl(n_classes), cr(n_classes);
    for (int f = 0; f < kF; ++f) {
      if (!allowed[f]) continue;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return F[kF * a + f] < F[kF * b + f]; });
      std::fill(cl.begin(), cl.end(), 0.0);
      for (int c = 0; c < n_classes; ++c) cr[c] = counts[c];
      for (int p = 0; p + 1 < n; ++p) {
        const int c = y[order[p]];
        cl[c] += 1.0;
        cr[c] -= 1.0;
        const double xa = F[kF * order[p] + f], xb = F[kF * order[p + 1] + f];
        if (!(xa < xb)) continue;
        const double nl = (double)(p + 1), nr = (double)(n - p - 1);
        if (nl < min_leaf || nr < min_leaf) continue;
        const double w = (nl * gini(cl, nl) + nr * gini(cr, nr)) / (double)n;
        if (bf < 0 || w < bw) {
          bf = f;
          bw = w;
          bt = (xa + xb) / 2.0;
        }
      }
    }
    if (bf < 0) return me;
    std::vector<int> left, right;
    for (int i : idx) (F[kF * i + bf] <= bt ? left : right).push_back(i);
    nodes[me].feature = bf;
    nodes[me].threshold = bt;
    const int l = grow(left, depth + 1);
    nodes[me].left = l;
    const int r = grow(right, depth + 1);
    nodes[me].right = r;
    return me;
  }
};

// ------------------------------------------------------------------ regression tree (Section 4.1)
// Multi-output regression tree from sizes to performance vectors, grown
// best-first to a leaf budget.  Within a node the rows are centred on the
// node mean, so the squared error a split removes is the between-part sum
// sum_j S_j^2 (1 / n_left + 1 / n_right), S_j the left part's column sums.
// A candidate replaces the best so far only if its gain is larger by more than
// this relative amount: splits that cut a node the same way through different
// features then tie exactly as they do in exact arithmetic.
constexpr double kGainTie = 1e-9;

struct RegressionTree {
  static constexpr int kF = GEMM_TREE_FEATURES;
  const double* F;
  const float* Y;
  int d;
  struct Split {
    double gain = 0.0;
    int f = -1;
    double thr = 0.0;
  };

  double sse(const std::vector<int>& idx) const {
    const int n = (int)idx.size();
    double total = 0.0;
    for (int j = 0; j < d; ++j) {
      double m = 0.0;
      for (int i : idx) m += Y[(size_t)i * d + j];
      m /= n;
      for (int i : idx) {
        const double e = Y[(size_t)i * d + j] - m;
        total += e * e;
      }
    }
    return total;
  }

  Split best(const std::vector<int>& idx) const {
    Split b;
    const int n = (int)idx.size();
    if (n < 2) return b;
    std::vector<double> mean(d, 0.0), L(d);
    for (int i : idx)
      for (int j = 0; j < d; ++j) mean[j] += Y[(size_t)i * d + j];
    for (int j = 0; j < d; ++j) mean[j] /= n;
    std::vector<int> order(idx);
    for (int f = 0; f < kF; ++f) {
      std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return F[kF * a + f] < F[kF * c + f]; });
      std::fill(L.begin(), L.end(), 0.0);
      for (int p = 0; p + 1 < n; ++p) {
        const float* row = Y + (size_t)order[p] * d;
        for (int j = 0; j < d; ++j) L[j] += (double)row[j] - mean[j];
        const double xa = F[kF * order[p] + f], xb = F[kF * order[p + 1] + f];
        if (!(xa < xb)) continue;
        double s2 = 0.0;
        for (int j = 0; j < d; ++j) s2 += L[j] * L[j];
        const double gain = s2 * (1.0 / (p + 1) + 1.0 / (n - p - 1));
        if (b.f < 0 || gain > b.gain * (1.0 + kGainTie)) {
          b.gain = gain;
          b.f = f;
          b.thr = (xa + xb) / 2.0;
        }
      }
    }
    return b;
  }
};

}  // namespace ks

using namespace ks;

extern "C" {

gemm_status_t kselect_normalise(int64_t n_rows, int32_t n_cols, const float* perf, float* out, int32_t mode,
                                void* stream) {
  if (n_rows < 0 || n_cols < 0 || mode < 0 || mode > 3) return GEMM_ERR_INVALID_ARG;
  if (n_rows == 0 || n_cols == 0) return GEMM_OK;
  if (!perf || !out) return GEMM_ERR_INVALID_ARG;
  const int rows_per_block = 8;
  normalise_kernel<<<(unsigned)((n_rows + rows_per_block - 1) / rows_per_block), 32 * rows_per_block, 0,
                     static_cast<cudaStream_t>(stream)>>>(n_rows, n_cols, perf, out, mode);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : cuda_fail(e);
}

gemm_status_t kselect_kmeans(int32_t n, int32_t d, int32_t k, int32_t n_init, const float* X, const uint32_t* draws,
                             int32_t max_iter, float tol, float* centres_out, int32_t* labels_out,
                             double* inertia_out, int32_t* iters_out, void* stream) {
  if (n < 1 || d < 1 || k < 1 || k > n || n_init < 1 || max_iter < 1 || !(tol >= 0.f)) return GEMM_ERR_INVALID_ARG;
  if (!X || !draws || !centres_out || !labels_out || !inertia_out) return GEMM_ERR_INVALID_ARG;
  if (k > 1024 || n_init > 1024) return GEMM_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t kd = (size_t)k * d;
  const size_t bytes = sizeof(float) * 2 * kd * n_init + sizeof(int) * (size_t)n * n_init +
                       sizeof(float) * (size_t)n * n_init + sizeof(float) * n_init + sizeof(int) * n_init +
                       sizeof(uint32_t) * (size_t)n_init * k + 64 * 8;
  char* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s);
  if (e != cudaSuccess) return cuda_fail(e);
  auto carve = [&](size_t nbytes) {
    char* p = ws;
    ws += (nbytes + 63) / 64 * 64;
    return p;
  };
  char* base = ws;
  KmArgs a;
  a.n = n; a.d = d; a.k = k; a.max_iter = max_iter; a.tol = tol; a.X = X;
  a.centres = reinterpret_cast<float*>(carve(sizeof(float) * kd * n_init));
  a.newc = reinterpret_cast<float*>(carve(sizeof(float) * kd * n_init));
  a.labels = reinterpret_cast<int*>(carve(sizeof(int) * (size_t)n * n_init));
  a.d2 = reinterpret_cast<float*>(carve(sizeof(float) * (size_t)n * n_init));
  a.inertia = reinterpret_cast<float*>(carve(sizeof(float) * n_init));
  a.iters = reinterpret_cast<int*>(carve(sizeof(int) * n_init));
  uint32_t* draws_dev = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * (size_t)n_init * k));
  a.draws = draws_dev;
  std::vector<float> inert(n_init);
  std::vector<int> its(n_init);
  e = cudaMemcpyAsync(draws_dev, draws, sizeof(uint32_t) * (size_t)n_init * k, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    kmeans_kernel<<<n_init, kKmThreads, sizeof(int) * k, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(inert.data(), a.inertia, sizeof(float) * n_init, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(its.data(), a.iters, sizeof(int) * n_init, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int best = 0;
  if (e == cudaSuccess) {
    for (int r = 1; r < n_init; ++r)
      if (inert[r] < inert[best]) best = r;
    e = cudaMemcpyAsync(centres_out, a.centres + kd * best, sizeof(float) * kd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(labels_out, a.labels + (size_t)n * best, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
  }
  cudaFreeAsync(base, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  *inertia_out = inert[best];
  if (iters_out) *iters_out = its[best];
  return GEMM_OK;
}

gemm_status_t kselect_score(int32_t n_rows, int32_t n_cols, const float* perf, int32_t n_deployed,
                            const int32_t* deployed_cols, const int32_t* chosen, float floor_, double out[3],
                            void* stream) {
  if (n_rows < 1 || n_cols < 1 || !perf || !out || n_deployed < 0 || n_deployed > GEMM_MAX_DEPLOYED ||
      (n_deployed > 0 && !deployed_cols) || !(floor_ > 0.f))
    return GEMM_ERR_INVALID_ARG;
  ScoreArgs a;
  a.n_rows = n_rows; a.n_cols = n_cols; a.n_deployed = chosen ? 0 : n_deployed;
  for (int q = 0; q < GEMM_MAX_DEPLOYED; ++q) a.deployed[q] = q < n_deployed ? deployed_cols[q] : 0;
  for (int q = 0; q < n_deployed; ++q)
    if (deployed_cols[q] < 0 || deployed_cols[q] >= n_cols) return GEMM_ERR_INVALID_ARG;
  a.perf = perf; a.chosen = chosen; a.floor_ = floor_;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* dout = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dout), 3 * sizeof(float), s);
  if (e != cudaSuccess) return cuda_fail(e);
  a.out = dout;
  score_kernel<<<1, kScoreThreads, 0, s>>>(a);
  e = cudaGetLastError();
  float h[3] = {0.f, 0.f, 0.f};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(dout, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  out[0] = h[0]; out[1] = h[1]; out[2] = h[2];
  return GEMM_OK;
}

gemm_status_t kselect_knn(int32_t n_train, int32_t n_query, int32_t d, const float* train, const int32_t* labels,
                          const float* query, int32_t k, int32_t* out, void* stream) {
  if (n_train < 1 || n_query < 0 || d < 1 || k < 1 || k > kKnnMax || k > n_train || !train || !labels ||
      (n_query > 0 && (!query || !out)))
    return GEMM_ERR_INVALID_ARG;
  if (n_query == 0) return GEMM_OK;
  knn_kernel<<<(n_query + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n_train, n_query, d, train, labels,
                                                                                  query, k, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : cuda_fail(e);
}

// Section 4.2: the best configuration of each centre, clusters in descending
// size (lower index first on ties); with dedupe, a cluster whose best is taken
// gets its best unused configuration, otherwise it is dropped.
gemm_status_t kselect_representatives(int32_t k, int32_t d, const float* centres, int32_t n, const int32_t* labels,
                                      int32_t dedupe, int32_t* out_cols, int32_t* out_count) {
  if (k < 1 || d < 1 || n < 0 || !centres || (n > 0 && !labels) || !out_cols || !out_count) return GEMM_ERR_INVALID_ARG;
  std::vector<int> sizes(k, 0);
  for (int i = 0; i < n; ++i) {
    if (labels[i] < 0 || labels[i] >= k) return GEMM_ERR_INVALID_ARG;
    sizes[labels[i]]++;
  }
  std::vector<int> order(k);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return sizes[a] > sizes[b]; });
  std::vector<char> taken(d, 0);
  int cnt = 0;
  for (int c : order) {
    const float* row = centres + (size_t)c * d;
    int pick = -1;
    for (int j = 0; j < d; ++j) {
      if (dedupe && taken[j]) continue;
      if (pick < 0 || row[j] > row[pick]) pick = j;
    }
    if (pick < 0) continue;
    if (!dedupe && taken[pick]) continue;
    taken[pick] = 1;
    out_cols[cnt++] = pick;
  }
  *out_count = cnt;
  return GEMM_OK;
}

// Section 4.2 baseline: the configurations that are best for the most rows
// (lowest index on ties); if fewer than n ever win, the rest by highest mean
// standard-normalised performance.
gemm_status_t kselect_top_n(int32_t n_rows, int32_t n_cols, const float* perf, int32_t n, int32_t* out_cols) {
  if (n_rows < 1 || n_cols < 1 || !perf || n < 1 || n > n_cols || !out_cols) return GEMM_ERR_INVALID_ARG;
  std::vector<int> wins(n_cols, 0);
  std::vector<double> mean(n_cols, 0.0);
  for (int r = 0; r < n_rows; ++r) {
    const float* p = perf + (size_t)r * n_cols;
    int b = 0;
    for (int c = 1; c < n_cols; ++c)
      if (p[c] > p[b]) b = c;
    wins[b]++;
    if (p[b] > 0.f)
      for (int c = 0; c < n_cols; ++c) mean[c] += (double)p[c] / (double)p[b];
  }
  std::vector<int> order(n_cols);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wins[a] > wins[b]; });
  std::vector<char> used(n_cols, 0);
  int cnt = 0;
  for (int c : order) {
    if (cnt == n || wins[c] == 0) break;
    out_cols[cnt++] = c;
    used[c] = 1;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mean[a] > mean[b]; });
  std::sort(order.begin(), order.end(), [&](int a, int b) { return mean[a] > mean[b] || (mean[a] == mean[b] && a < b); });
  for (int c : order) {
    if (cnt == n) break;
    if (!used[c]) out_cols[cnt++] = c;
  }
  return GEMM_OK;
}

// Section 5.1 classifier comparison: one random-forest tree (CART restricted to
// per-node feature subsets drawn from `draws`, GEMM_TREE_FEATURES uint32 per node).
gemm_status_t kselect_tree_train_rf(int32_t n, const double* features, const int32_t* labels, int32_t n_classes,
                                    int32_t max_depth, int32_t min_leaf, int32_t max_features, const uint32_t* draws,
                                    gemm_tree_node_t* out_nodes, int32_t max_nodes, int32_t* out_n_nodes) {
  if (n < 1 || !features || !labels || n_classes < 1 || min_leaf < 1 || !out_nodes || max_nodes < 1 ||
      !out_n_nodes || max_features < 1 || max_features > GEMM_TREE_FEATURES ||
      (max_features < GEMM_TREE_FEATURES && !draws))
    return GEMM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (labels[i] < 0 || labels[i] >= n_classes) return GEMM_ERR_INVALID_ARG;
    for (int f = 0; f < GEMM_TREE_FEATURES; ++f)
      if (!std::isfinite(features[GEMM_TREE_FEATURES * i + f])) return GEMM_ERR_INVALID_ARG;
  }
  TreeBuilder tb{features, labels, n_classes, max_depth, min_leaf, max_nodes, {}, false, max_features, draws};
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  tb.grow(idx, 0);
  if (tb.overflow) return GEMM_ERR_UNSUPPORTED;
  std::memcpy(out_nodes, tb.nodes.data(), tb.nodes.size() * sizeof(gemm_tree_node_t));
  *out_n_nodes = (int32_t)tb.nodes.size();
  return GEMM_OK;
}

// Section 5.1: the selector's feature rows of a list of sizes.
gemm_status_t kselect_selector_features(int32_t n, const int64_t* sizes, double* out) {
  if (n < 0 || (n > 0 && (!sizes || !out))) return GEMM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int64_t* r = sizes + 4 * (size_t)i;
    if (r[0] < 0 || r[1] < 0 || r[2] < 0 || r[3] < 0) return GEMM_ERR_INVALID_ARG;
    selector_features(r[0], r[1], r[2], r[3], out + GEMM_TREE_FEATURES * (size_t)i);
  }
  return GEMM_OK;
}

// Section 5.1: each training size is labelled with its best deployed kernel.
gemm_status_t kselect_best_labels(int32_t n_rows, int32_t n_cols, const double* perf, int32_t n_sel,
                                  const int32_t* cols, int32_t* labels_out) {
  if (n_rows < 1 || n_cols < 1 || n_sel < 1 || !perf || !cols || !labels_out) return GEMM_ERR_INVALID_ARG;
  for (int j = 0; j < n_sel; ++j)
    if (cols[j] < 0 || cols[j] >= n_cols) return GEMM_ERR_INVALID_ARG;
  for (int i = 0; i < n_rows; ++i) {
    const double* row = perf + (size_t)i * n_cols;
    int best = 0;
    for (int j = 0; j < n_sel; ++j) {
      if (std::isnan(row[cols[j]])) return GEMM_ERR_INVALID_ARG;
      if (row[cols[j]] > row[cols[best]]) best = j;
    }
    labels_out[i] = best;
  }
  return GEMM_OK;
}

// Section 5.1: CART classifier from the sizes' feature rows to a deployed kernel.
gemm_status_t kselect_tree_train(int32_t n, const double* features, const int32_t* labels, int32_t n_classes,
                                 int32_t max_depth, int32_t min_leaf, gemm_tree_node_t* out_nodes, int32_t max_nodes,
                                 int32_t* out_n_nodes) {
  if (n < 1 || !features || !labels || n_classes < 1 || min_leaf < 1 || !out_nodes || max_nodes < 1 ||
      !out_n_nodes)
    return GEMM_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (labels[i] < 0 || labels[i] >= n_classes) return GEMM_ERR_INVALID_ARG;
    for (int f = 0; f < GEMM_TREE_FEATURES; ++f)
      if (!std::isfinite(features[GEMM_TREE_FEATURES * i + f])) return GEMM_ERR_INVALID_ARG;
  }
  TreeBuilder tb{features, labels, n_classes, max_depth, min_leaf, max_nodes, {}, false};
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  tb.grow(idx, 0);
  if (tb.overflow) return GEMM_ERR_UNSUPPORTED;
  std::memcpy(out_nodes, tb.nodes.data(), tb.nodes.size() * sizeof(gemm_tree_node_t));
  *out_n_nodes = (int32_t)tb.nodes.size();
  return GEMM_OK;
}

gemm_status_t kselect_cluster_geomean(int32_t n, int32_t d, const float* X, const int32_t* labels, int32_t k,
                                      float floor, float* out, void* stream) {
  if (n < 0 || d < 1 || k < 1 || !(floor > 0.f) || !out || (n > 0 && (!X || !labels))) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)k * d;
  const int grid = (int)std::min<int64_t>((total + 127) / 128, 152 * 16);
  cluster_geomean_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, d, X, labels, k, floor, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : cuda_fail(e);
}

// Section 4.1 "Decision tree" pruning: partition of the training sizes by a
// regression tree with at most max_leaves leaves.
gemm_status_t kselect_tree_regress(int32_t n, int32_t d, const double* features, const float* Y, int32_t max_leaves,
                                   int32_t* labels_out, float* centres_out, int32_t* n_leaves_out) {
  if (n < 1 || d < 1 || !features || !Y || max_leaves < 1 || !labels_out || !centres_out || !n_leaves_out)
    return GEMM_ERR_INVALID_ARG;
  for (int64_t i = 0; i < (int64_t)n * GEMM_TREE_FEATURES; ++i)
    if (!std::isfinite(features[i])) return GEMM_ERR_INVALID_ARG;
  for (int64_t i = 0; i < (int64_t)n * d; ++i)
    if (!std::isfinite(Y[i])) return GEMM_ERR_INVALID_ARG;
  RegressionTree rt{features, Y, d};
  std::vector<std::vector<int>> leaves(1, std::vector<int>(n));
  std::iota(leaves[0].begin(), leaves[0].end(), 0);
  std::vector<RegressionTree::Split> splits{rt.best(leaves[0])};
  const double tol = 1e-12 * rt.sse(leaves[0]);
  while ((int)leaves.size() < max_leaves) {
    int pick = -1;
    for (int i = 0; i < (int)leaves.size(); ++i)
      if (splits[i].f >= 0 && splits[i].gain > tol &&
          (pick < 0 || splits[i].gain > splits[pick].gain * (1.0 + kGainTie)))
        pick = i;
    if (pick < 0) break;
    const RegressionTree::Split sp = splits[pick];
    std::vector<int> left, right;
    for (int i : leaves[pick]) (features[GEMM_TREE_FEATURES * i + sp.f] <= sp.thr ? left : right).push_back(i);
    leaves[pick] = std::move(left);
    leaves.push_back(std::move(right));
    splits[pick] = rt.best(leaves[pick]);
    splits.push_back(rt.best(leaves.back()));
  }
  for (int c = 0; c < (int)leaves.size(); ++c) {
    for (int j = 0; j < d; ++j) {
      double m = 0.0;
      for (int i : leaves[c]) m += Y[(size_t)i * d + j];
      centres_out[(size_t)c * d + j] = (float)(m / leaves[c].size());
    }
    for (int i : leaves[c]) labels_out[i] = c;
  }
  *n_leaves_out = (int32_t)leaves.size();
  return GEMM_OK;
}

}  // extern "C"
