// Principal component analysis of normalised performance vectors (Section 3.3,
// and the PCA + k-means pruning of Section 4.1).
//
// Covariance C = Xc^T Xc / (n - 1) of the centred data comes from the
// library's own FP32 SIMT GEMM; the dominant r-dimensional subspace from
// subspace (orthogonal) iteration W = C V, V = orth(W) with a one-block
// modified Gram-Schmidt kernel; Ritz values and vectors from the r x r
// projection V^T C V, solved on the host by cyclic Jacobi rotations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace ks {
gemm_status_t launch_by_id(int id, const GemmArgs& a, cudaStream_t s);
gemm_status_t make_launch_args(int id, char transA, char transB, int64_t M, int64_t N, int64_t K, float alpha,
                               const void* A, int64_t lda, const void* B, int64_t ldb, float beta, float* C,
                               int64_t ldc, int64_t batch, GemmArgs* a, bool* noop);

namespace {
// TM 8, TN 8, WX 16, WY 8, BK 16, staged: a large-tile FP32 config
constexpr int kPcaGemmConfig = ((((3 * 4 + 3) * 6 + 4) * 3 + 1) * 2 + 1);

__global__ void center_kernel(int n, int d, const float* X, float* mean, float* Xc) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += X[(int64_t)i * d + j];
    const float m = s / (float)n;
    mean[j] = m;
    for (int i = 0; i < n; ++i) Xc[(int64_t)i * d + j] = X[(int64_t)i * d + j] - m;
  }
}

__device__ float block_sum(float v, float* sh) {
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

// Modified Gram-Schmidt on the r columns of V (d x r, row-major), one block.
__global__ void mgs_kernel(int d, int r, float* V) {
  __shared__ float sh[33];
  for (int j = 0; j < r; ++j) {
    for (int q = 0; q < j; ++q) {
      float part = 0.f;
      for (int i = threadIdx.x; i < d; i += blockDim.x) part = fmaf(V[i * r + q], V[i * r + j], part);
      const float proj = block_sum(part, sh);
      for (int i = threadIdx.x; i < d; i += blockDim.x) V[i * r + j] = fmaf(-proj, V[i * r + q], V[i * r + j]);
      __syncthreads();
    }
    float part = 0.f;
    for (int i = threadIdx.x; i < d; i += blockDim.x) part = fmaf(V[i * r + j], V[i * r + j], part);
    const float nrm = sqrtf(block_sum(part, sh));
    const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    for (int i = threadIdx.x; i < d; i += blockDim.x) V[i * r + j] *= inv;
    __syncthreads();
  }
}

__global__ void backproject_kernel(int k, int d, int r, const float* cent, const float* V, const float* mean,
                                   float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * d) return;
  const int c = t / d, j = t % d;
  float x = mean[j];
  for (int q = 0; q < r; ++q) x = fmaf(cent[c * r + q], V[j * r + q], x);
  out[t] = x;
}

__global__ void trace_kernel(int d, const float* C, float* out) {
  __shared__ float sh[33];
  float part = 0.f;
  for (int i = threadIdx.x; i < d; i += blockDim.x) part += C[(int64_t)i * d + i];
  const float t = block_sum(part, sh);
  if (threadIdx.x == 0) *out = t;
}

gemm_status_t fail(cudaError_t e) {
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
}

// ---- spectral embedding (Section 4.1, spectral clustering)
__global__ void diag_kernel(int n, const float* G, float* sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) sq[i] = G[(int64_t)i * n + i];
}

// G (the Gram matrix X X^T) becomes the RBF adjacency, zero diagonal.
__global__ void affinity_kernel(int n, float gamma, const float* sq, float* G) {
  const int64_t total = (int64_t)n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
    const float d2 = fmaxf(sq[i] + sq[j] - 2.f * G[t], 0.f);
    G[t] = (i == j) ? 0.f : expf(-gamma * d2);
  }
}

// s_i = deg_i^-1/2 (0 for an isolated row), one block per row.
__global__ void inv_sqrt_degree_kernel(int n, const float* A, float* s) {
  __shared__ float sh[33];
  const int i = blockIdx.x;
  float part = 0.f;
  for (int j = threadIdx.x; j < n; j += blockDim.x) part += A[(int64_t)i * n + j];
  const float deg = block_sum(part, sh);
  if (threadIdx.x == 0) s[i] = deg > 0.f ? rsqrtf(deg) : 0.f;
}

// A <- D^-1/2 A D^-1/2 + I: the shift puts the spectrum in [0, 2], so the
// subspace iteration converges to the largest (not the largest-magnitude) eigenvalues.
__global__ void normalise_shift_kernel(int n, const float* s, float* A) {
  const int64_t total = (int64_t)n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (int64_t)i * n);
    A[t] = s[i] * A[t] * s[j] + (i == j ? 1.f : 0.f);
  }
}

// Rows of U (n x k) scaled to unit length; zero rows stay zero.
__global__ void row_unit_kernel(int n, int k, float* U) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float q = 0.f;
    for (int j = 0; j < k; ++j) q = fmaf(U[i * k + j], U[i * k + j], q);
    const float inv = q > 0.f ? rsqrtf(q) : 0.f;
    for (int j = 0; j < k; ++j) U[i * k + j] *= inv;
  }
}

int grid_of(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 16); }

// C[M x N] = alpha * op(A) * op(B) with the library's SIMT kernel.
gemm_status_t mm(char ta, char tb, int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb,
                 float* C, int ldc, cudaStream_t s) {
  GemmArgs a;
  bool noop = false;
  gemm_status_t st = make_launch_args(kPcaGemmConfig, ta, tb, M, N, K, alpha, A, lda, B, ldb, 0.f, C, ldc, 1, &a,
                                      &noop);
  if (st != GEMM_OK || noop) return st;
  return launch_by_id(kPcaGemmConfig, a, s);
}

// Cyclic Jacobi eigen-decomposition of a symmetric r x r matrix (row-major).
void jacobi(int r, std::vector<double>& A, std::vector<double>& Q) {
  Q.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) Q[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) off += A[(size_t)p * r + q] * A[(size_t)p * r + q];
    if (off < 1e-30) break;
    for (int p = 0; p < r; ++p)
      for (int q = p + 1; q < r; ++q) {
        const double apq = A[(size_t)p * r + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * r + p], aqq = A[(size_t)q * r + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < r; ++k) {  // columns p, q
          const double akp = A[(size_t)k * r + p], akq = A[(size_t)k * r + q];
          A[(size_t)k * r + p] = c * akp - sn * akq;
          A[(size_t)k * r + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < r; ++k) {  // rows p, q
          const double apk = A[(size_t)p * r + k], aqk = A[(size_t)q * r + k];
          A[(size_t)p * r + k] = c * apk - sn * aqk;
          A[(size_t)q * r + k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < r; ++k) {
          const double qkp = Q[(size_t)k * r + p], qkq = Q[(size_t)k * r + q];
          Q[(size_t)k * r + p] = c * qkp - sn * qkq;
          Q[(size_t)k * r + q] = sn * qkp + c * qkq;
        }
      }
  }
}
}  // namespace
}  // namespace ks

using namespace ks;

extern "C" gemm_status_t kselect_pca(int32_t n, int32_t d, const float* X, int32_t r, int32_t iters, const float* V0,
                                     float* mean_out, float* V_out, float* Y_out, double* evals_out,
                                     double* total_var_out, void* stream) {
  if (n < 2 || d < 1 || r < 1 || r > d || r > 256 || iters < 1 || !X || !V0 || !mean_out || !V_out || !evals_out ||
      !total_var_out)
    return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fXc = (size_t)n * d, fC = (size_t)d * d, fW = (size_t)d * r, fT = (size_t)r * r;
  float* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), sizeof(float) * (fXc + fC + 2 * fW + fT + 64), s);
  if (e != cudaSuccess) return fail(e);
  float *Xc = ws, *C = Xc + fXc, *W = C + fC, *V = W + fW, *T = V + fW, *tr = T + fT;
  gemm_status_t st = GEMM_OK;
  center_kernel<<<(d + 127) / 128, 128, 0, s>>>(n, d, X, mean_out, Xc);
  if ((e = cudaGetLastError()) != cudaSuccess) st = fail(e);
  // C = Xc^T Xc / (n - 1)
  if (st == GEMM_OK) st = mm('T', 'N', d, d, n, 1.f / (float)(n - 1), Xc, d, Xc, d, C, d, s);
  if (st == GEMM_OK) {
    trace_kernel<<<1, 256, 0, s>>>(d, C, tr);
    e = cudaMemcpyAsync(V, V0, sizeof(float) * fW, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  }
  for (int it = 0; it < iters && st == GEMM_OK; ++it) {
    st = mm('N', 'N', d, r, d, 1.f, C, d, V, r, W, r, s);  // W = C V
    if (st != GEMM_OK) break;
    mgs_kernel<<<1, 256, 0, s>>>(d, r, W);
    e = cudaMemcpyAsync(V, W, sizeof(float) * fW, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  }
  // Rayleigh-Ritz: T = V^T C V, T = Q diag Q^T, V <- V Q (columns by descending value)
  if (st == GEMM_OK) st = mm('N', 'N', d, r, d, 1.f, C, d, V, r, W, r, s);
  if (st == GEMM_OK) st = mm('T', 'N', r, r, d, 1.f, V, r, W, r, T, r, s);
  std::vector<float> Th(fT);
  float trh = 0.f;
  if (st == GEMM_OK) {
    e = cudaMemcpyAsync(Th.data(), T, sizeof(float) * fT, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&trh, tr, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(e);
  }
  if (st == GEMM_OK) {
    std::vector<double> A(fT), Q;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) A[(size_t)i * r + j] = 0.5 * ((double)Th[(size_t)i * r + j] + Th[(size_t)j * r + i]);
    jacobi(r, A, Q);
    std::vector<int> order(r);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return A[(size_t)a * r + a] > A[(size_t)b * r + b]; });
    std::vector<float> Qs(fT);
    for (int j = 0; j < r; ++j) {
      evals_out[j] = A[(size_t)order[j] * r + order[j]];
      for (int i = 0; i < r; ++i) Qs[(size_t)i * r + j] = (float)Q[(size_t)i * r + order[j]];
    }
    *total_var_out = trh;
    e = cudaMemcpyAsync(T, Qs.data(), sizeof(float) * fT, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = fail(e);
    if (st == GEMM_OK) st = mm('N', 'N', d, r, r, 1.f, V, r, T, r, V_out, r, s);  // V_out = V Q
    if (st == GEMM_OK && Y_out) st = mm('N', 'N', n, r, d, 1.f, Xc, d, V_out, r, Y_out, r, s);  // Y = Xc V
    if (st == GEMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail(e);
  }
  cudaFreeAsync(ws, s);
  cudaStreamSynchronize(s);
  return st;
}

// out (k x d) = mean + cent (k x r) V^T: centres found in PCA coordinates,
// expressed again as performance vectors over the d configurations.
extern "C" gemm_status_t kselect_pca_backproject(int32_t k, int32_t d, int32_t r, const float* cent, const float* V,
                                                 const float* mean, float* out, void* stream) {
  if (k < 1 || d < 1 || r < 1 || !cent || !V || !mean || !out) return GEMM_ERR_INVALID_ARG;
  backproject_kernel<<<(k * d + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(k, d, r, cent, V, mean, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

// Section 4.1, spectral clustering: the k leading eigenvectors of
// S = D^-1/2 A D^-1/2 for the RBF adjacency A_ij = exp(-gamma |x_i - x_j|^2)
// (zero diagonal) of the n rows of X, i.e. those of the normalised Laplacian
// I - S with the smallest eigenvalues, by subspace iteration on S + I with an
// r-column block (r >= k) and Rayleigh-Ritz; rows then scaled to unit length.
extern "C" gemm_status_t kselect_spectral_embedding(int32_t n, int32_t d, const float* X, float gamma, int32_t k,
                                                    int32_t r, int32_t iters, const float* V0, float* U_out,
                                                    double* evals_out, void* stream) {
  if (n < 2 || d < 1 || k < 1 || r < k || r > n || r > 256 || iters < 1 || !(gamma > 0.f) || !std::isfinite(gamma) ||
      !X || !V0 || !U_out || !evals_out)
    return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fA = (size_t)n * n, fW = (size_t)n * r, fT = (size_t)r * r;
  float* ws = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), sizeof(float) * (fA + 2 * fW + fT + 2 * (size_t)n), s);
  if (e != cudaSuccess) return fail(e);
  float *A = ws, *W = A + fA, *V = W + fW, *T = V + fW, *sq = T + fT, *sc = sq + n;
  gemm_status_t st = mm('N', 'T', n, n, d, 1.f, X, d, X, d, A, n, s);  // Gram matrix
  if (st == GEMM_OK) {
    diag_kernel<<<grid_of(n), 256, 0, s>>>(n, A, sq);
    affinity_kernel<<<grid_of((int64_t)n * n), 256, 0, s>>>(n, gamma, sq, A);
    inv_sqrt_degree_kernel<<<n, 256, 0, s>>>(n, A, sc);
    normalise_shift_kernel<<<grid_of((int64_t)n * n), 256, 0, s>>>(n, sc, A);
    e = cudaMemcpyAsync(V, V0, sizeof(float) * fW, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  }
  for (int it = 0; it < iters && st == GEMM_OK; ++it) {
    st = mm('N', 'N', n, r, n, 1.f, A, n, V, r, W, r, s);  // W = (S + I) V
    if (st != GEMM_OK) break;
    mgs_kernel<<<1, 256, 0, s>>>(n, r, W);
    e = cudaMemcpyAsync(V, W, sizeof(float) * fW, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = fail(e);
  }
  if (st == GEMM_OK) st = mm('N', 'N', n, r, n, 1.f, A, n, V, r, W, r, s);
  if (st == GEMM_OK) st = mm('T', 'N', r, r, n, 1.f, V, r, W, r, T, r, s);  // V^T (S + I) V
  std::vector<float> Th(fT);
  if (st == GEMM_OK) {
    e = cudaMemcpyAsync(Th.data(), T, sizeof(float) * fT, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(e);
  }
  if (st == GEMM_OK) {
    std::vector<double> Am(fT), Q;
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < r; ++j) Am[(size_t)i * r + j] = 0.5 * ((double)Th[(size_t)i * r + j] + Th[(size_t)j * r + i]);
    jacobi(r, Am, Q);
    std::vector<int> order(r);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return Am[(size_t)a * r + a] > Am[(size_t)b * r + b]; });
    std::vector<float> Qk((size_t)r * k);
    for (int j = 0; j < k; ++j) {
      evals_out[j] = Am[(size_t)order[j] * r + order[j]] - 1.0;  // undo the shift
      for (int i = 0; i < r; ++i) Qk[(size_t)i * k + j] = (float)Q[(size_t)i * r + order[j]];
    }
    e = cudaMemcpyAsync(T, Qk.data(), sizeof(float) * Qk.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) st = fail(e);
    if (st == GEMM_OK) st = mm('N', 'N', n, k, r, 1.f, V, r, T, k, U_out, k, s);  // U = V Q_k
    if (st == GEMM_OK) {
      row_unit_kernel<<<grid_of(n), 256, 0, s>>>(n, k, U_out);
      if ((e = cudaGetLastError()) != cudaSuccess) st = fail(e);
    }
    if (st == GEMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = fail(e);
  }
  cudaFreeAsync(ws, s);
  cudaStreamSynchronize(s);
  return st;
}
