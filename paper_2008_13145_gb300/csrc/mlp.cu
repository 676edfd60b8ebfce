// Learned selector: a 7-64-64-8 MLP performance model trained and served by
// the library's own kernels.
//
// Training (full batch): mlp_grad_kernel computes, for a chunk of samples per
// block, the forward pass, the masked squared-error gradient and the block's
// partial parameter gradient; mlp_reduce_kernel sums the partials over blocks
// in block order (deterministic) and mlp_adam_kernel applies Adam.  The three
// launches of one step are captured once in a CUDA graph and replayed, the
// Adam step counter living in device memory.
// Serving: mlp_select_kernel gives one thread per queued GEMM; the weights sit
// in shared memory and the second hidden layer is consumed unit by unit, so
// each thread keeps only 64 + 8 activations in registers.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace ks {
namespace mlp {

constexpr int NI = 7, NH = 64, NO = 8, NP = GEMM_MLP_PARAMS;
constexpr int OW1 = 0, OB1 = OW1 + NI * NH, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH * NO;
static_assert(OB3 + NO == NP, "parameter layout");

constexpr int kChunk = 32;     // samples per block in training
constexpr int kThreads = 256;

struct GradArgs {
  int n;
  const float* P;
  const float* X;
  const float* T;
  const float* mask;
  const float* count;  // device scalar: number of measured outputs
  float* partials;     // nblocks x NP
  float* loss_part;    // nblocks
  int* step;           // Adam step counter, incremented by block 0 (may be null)
};

__global__ void __launch_bounds__(kThreads) mlp_grad_kernel(const GradArgs a) {
  extern __shared__ float sm[];
  float* P = sm;                      // NP
  float* x = P + NP;                  // kChunk x NI
  float* z1 = x + kChunk * NI;        // kChunk x NH
  float* z2 = z1 + kChunk * NH;       // kChunk x NH
  float* dy = z2 + kChunk * NH;       // kChunk x NO
  float* d2 = dy + kChunk * NO;       // kChunk x NH
  float* d1 = d2 + kChunk * NH;       // kChunk x NH
  __shared__ float red[kThreads / 32];
  const int tid = threadIdx.x, s0 = blockIdx.x * kChunk;
  if (a.step && blockIdx.x == 0 && tid == 0) atomicAdd(a.step, 1);
  for (int p = tid; p < NP; p += kThreads) P[p] = a.P[p];
  for (int e = tid; e < kChunk * NI; e += kThreads) {
    const int s = s0 + e / NI;
    x[e] = s < a.n ? a.X[(int64_t)s * NI + e % NI] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * NH; e += kThreads) {
    const int s = e / NH, j = e % NH;
    float z = P[OB1 + j];
    for (int i = 0; i < NI; ++i) z = fmaf(x[s * NI + i], P[OW1 + i * NH + j], z);
    z1[e] = z;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * NH; e += kThreads) {
    const int s = e / NH, j = e % NH;
    float z = P[OB2 + j];
    for (int i = 0; i < NH; ++i) z = fmaf(fmaxf(z1[s * NH + i], 0.f), P[OW2 + i * NH + j], z);
    z2[e] = z;
  }
  __syncthreads();
  const float inv = 1.f / *a.count;
  float lsum = 0.f;
  for (int e = tid; e < kChunk * NO; e += kThreads) {
    const int s = e / NO, o = e % NO, gs = s0 + s;
    float y = P[OB3 + o];
    for (int i = 0; i < NH; ++i) y = fmaf(fmaxf(z2[s * NH + i], 0.f), P[OW3 + i * NO + o], y);
    float r = 0.f;
    if (gs < a.n) {
      const float m = a.mask ? a.mask[(int64_t)gs * NO + o] : 1.f;
      r = (y - a.T[(int64_t)gs * NO + o]) * m;
    }
    lsum = fmaf(r, r, lsum);
    dy[e] = 2.f * r * inv;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * NH; e += kThreads) {
    const int s = e / NH, i = e % NH;
    float g = 0.f;
    for (int o = 0; o < NO; ++o) g = fmaf(dy[s * NO + o], P[OW3 + i * NO + o], g);
    d2[e] = z2[e] > 0.f ? g : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * NH; e += kThreads) {
    const int s = e / NH, i = e % NH;
    float g = 0.f;
    for (int j = 0; j < NH; ++j) g = fmaf(d2[s * NH + j], P[OW2 + i * NH + j], g);
    d1[e] = z1[e] > 0.f ? g : 0.f;
  }
  __syncthreads();
  float* out = a.partials + (int64_t)blockIdx.x * NP;
  for (int p = tid; p < NP; p += kThreads) {
    float g = 0.f;
    if (p < OB1) {
      const int i = p / NH, j = p % NH;
      for (int s = 0; s < kChunk; ++s) g = fmaf(x[s * NI + i], d1[s * NH + j], g);
    } else if (p < OW2) {
      const int j = p - OB1;
      for (int s = 0; s < kChunk; ++s) g += d1[s * NH + j];
    } else if (p < OB2) {
      const int i = (p - OW2) / NH, j = (p - OW2) % NH;
      for (int s = 0; s < kChunk; ++s) g = fmaf(fmaxf(z1[s * NH + i], 0.f), d2[s * NH + j], g);
    } else if (p < OW3) {
      const int j = p - OB2;
      for (int s = 0; s < kChunk; ++s) g += d2[s * NH + j];
    } else if (p < OB3) {
      const int i = (p - OW3) / NO, o = (p - OW3) % NO;
      for (int s = 0; s < kChunk; ++s) g = fmaf(fmaxf(z2[s * NH + i], 0.f), dy[s * NO + o], g);
    } else {
      const int o = p - OB3;
      for (int s = 0; s < kChunk; ++s) g += dy[s * NO + o];
    }
    out[p] = g;
  }
  // block loss partial (sum of squared masked residuals / count)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    a.loss_part[blockIdx.x] = t * inv;
  }
}

__global__ void mlp_reduce_kernel(const float* partials, const float* loss_part, int nblocks, float* grad,
                                  float* loss, float* loss_hist, const int* step, int t0) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NP) {
    float g = 0.f;
    for (int b = 0; b < nblocks; ++b) g += partials[(int64_t)b * NP + p];
    grad[p] = g;
  }
  if (p == 0) {
    float l = 0.f;
    for (int b = 0; b < nblocks; ++b) l += loss_part[b];
    if (loss) *loss = l;
    if (loss_hist && step) loss_hist[*step - t0 - 1] = l;
  }
}

__global__ void mlp_count_kernel(const float* mask, int64_t total, float* count) {
  __shared__ float red[32];
  float c = 0.f;
  for (int64_t i = threadIdx.x; i < total; i += blockDim.x) c += mask ? mask[i] : 1.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *count = t > 0.f ? t : 1.f;
  }
}

__global__ void mlp_adam_kernel(float* P, const float* g, float* m, float* v, const int* step_dev, int step_host,
                                float lr, float b1, float b2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NP) return;
  const int t = step_dev ? *step_dev : step_host;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.f - b1) * gp;
  const float vp = b2 * v[p] + (1.f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float mh = mp / (1.f - powf(b1, (float)t));
  const float vh = vp / (1.f - powf(b2, (float)t));
  P[p] -= lr * mh / (sqrtf(vh) + eps);
}

__device__ __forceinline__ float feature(int q, const int64_t* sh) {
  switch (q) {
    case 0: return log2f((float)sh[0]) / 12.f;
    case 1: return log2f((float)sh[1]) / 12.f;
    case 2: return log2f((float)sh[2]) / 12.f;
    case 3: return log2f((float)sh[3]) / 4.f;
    case 4: return (float)sh[4];
    case 5: return (float)sh[5];
    default: return (float)sh[6] / 3.f;
  }
}

// Training targets: per row of an n x d throughput table, log(perf / row max)
// over the measured (perf > 0) entries, 0 elsewhere, and the mask of measured
// entries (a row with none measured is all masked).
__global__ void mlp_targets_kernel(int n, int d, const float* perf, float* T, float* mask) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float* p = perf + (int64_t)r * d;
  float mx = 0.f;
  for (int j = 0; j < d; ++j) mx = fmaxf(mx, p[j]);
  for (int j = 0; j < d; ++j) {
    const bool ok = p[j] > 0.f;
    T[(int64_t)r * d + j] = ok ? logf(p[j] / mx) : 0.f;
    mask[(int64_t)r * d + j] = ok ? 1.f : 0.f;
  }
}

__global__ void mlp_features_kernel(int n, const int64_t* shapes, float* X) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
#pragma unroll
  for (int q = 0; q < NI; ++q) X[(int64_t)r * NI + q] = feature(q, shapes + (int64_t)r * 7);
}

// One thread per row: y = network(x); optionally pick argmax over the first n_out outputs.
template <bool FROM_SHAPES>
__global__ void __launch_bounds__(128) mlp_forward_kernel(int n, const float* Pg, const float* X, const int64_t* shapes,
                                                          float* Y, int n_out, const int32_t* ids, int32_t* ids_out) {
  __shared__ float P[NP];
  for (int p = threadIdx.x; p < NP; p += blockDim.x) P[p] = Pg[p];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float x[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) x[i] = FROM_SHAPES ? feature(i, shapes + (int64_t)r * 7) : X[(int64_t)r * NI + i];
  float h1[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float z = P[OB1 + j];
#pragma unroll
    for (int i = 0; i < NI; ++i) z = fmaf(x[i], P[OW1 + i * NH + j], z);
    h1[j] = fmaxf(z, 0.f);
  }
  float y[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) y[o] = P[OB3 + o];
#pragma unroll 1
  for (int j = 0; j < NH; ++j) {
    float z = P[OB2 + j];
#pragma unroll
    for (int i = 0; i < NH; ++i) z = fmaf(h1[i], P[OW2 + i * NH + j], z);
    const float h = fmaxf(z, 0.f);
#pragma unroll
    for (int o = 0; o < NO; ++o) y[o] = fmaf(h, P[OW3 + j * NO + o], y[o]);
  }
  if (Y) {
#pragma unroll
    for (int o = 0; o < NO; ++o) Y[(int64_t)r * NO + o] = y[o];
  }
  if (ids_out) {
    int best = 0;
    for (int o = 1; o < n_out; ++o)
      if (y[o] > y[best]) best = o;
    ids_out[r] = ids[best];
  }
}

struct Ids {
  int32_t v[GEMM_MAX_DEPLOYED];
};

gemm_status_t fail(cudaError_t e) {
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
}

constexpr size_t kGradSmem = sizeof(float) * (NP + kChunk * NI + 4 * kChunk * NH + kChunk * NO);

cudaError_t ensure_attr() {
  static unsigned long long done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
  if (e == cudaSuccess) __atomic_fetch_or(&done, bit, __ATOMIC_ACQ_REL);
  return e;
}

// Scratch for one training configuration: partials, loss partials, count, grad, loss, step.
struct Workspace {
  float* partials;
  float* loss_part;
  float* count;
  float* grad;
  float* loss;
  int* step;
  char* base;
};

cudaError_t ws_alloc(int nblocks, cudaStream_t s, Workspace* w) {
  const size_t bytes = sizeof(float) * ((size_t)nblocks * NP + nblocks + 1 + NP + 1) + sizeof(int) + 6 * 256;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&w->base), bytes, s);
  if (e != cudaSuccess) return e;
  char* p = w->base;
  auto carve = [&](size_t nb) {
    char* r = p;
    p += (nb + 255) / 256 * 256;
    return r;
  };
  w->partials = reinterpret_cast<float*>(carve(sizeof(float) * (size_t)nblocks * NP));
  w->loss_part = reinterpret_cast<float*>(carve(sizeof(float) * nblocks));
  w->count = reinterpret_cast<float*>(carve(sizeof(float)));
  w->grad = reinterpret_cast<float*>(carve(sizeof(float) * NP));
  w->loss = reinterpret_cast<float*>(carve(sizeof(float)));
  w->step = reinterpret_cast<int*>(carve(sizeof(int)));
  return cudaSuccess;
}

// ---------------------------------------------------------------- allocation-free loss/gradient
// Scratch of mlp_loss_grad_noalloc: per-block gradient partials for up to
// kNoAllocMaxSamples samples, then the per-block losses, then the count of
// measured outputs.  Every device that loads the library holds this array
// (about 5.3 MB) until the process exits.
constexpr int kNoAllocMaxSamples = 8192;
constexpr int kNoAllocMaxBlocks = kNoAllocMaxSamples / kChunk;
constexpr size_t kNoAllocFloats = (size_t)kNoAllocMaxBlocks * NP + kNoAllocMaxBlocks + 64;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side stand-in, so the address is looked up
// once per device and cached.
float* noalloc_scratch(cudaError_t* err) {
  static float* addr[64] = {nullptr};
  static std::mutex mu;
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = static_cast<float*>(p);
  }
  return addr[dev];
}

}  // namespace mlp
}  // namespace ks

using namespace ks;
using namespace ks::mlp;

extern "C" {

gemm_status_t mlp_features(int32_t n, const int64_t* shapes, float* X, void* stream) {
  if (n < 0 || (n > 0 && (!shapes || !X))) return GEMM_ERR_INVALID_ARG;
  if (n == 0) return GEMM_OK;
  mlp_features_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, shapes, X);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_targets(int32_t n, int32_t d, const float* perf, float* T, float* mask, void* stream) {
  if (n < 0 || d < 1 || (n > 0 && (!perf || !T || !mask))) return GEMM_ERR_INVALID_ARG;
  if (n == 0) return GEMM_OK;
  mlp_targets_kernel<<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, d, perf, T, mask);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_forward(int32_t n, const float* P, const float* X, float* Y, void* stream) {
  if (n < 0 || (n > 0 && (!P || !X || !Y))) return GEMM_ERR_INVALID_ARG;
  if (n == 0) return GEMM_OK;
  mlp_forward_kernel<false><<<(n + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(n, P, X, nullptr, Y, 0,
                                                                                            nullptr, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_loss_grad(int32_t n, const float* P, const float* X, const float* T, const float* mask,
                            float* grad, float* loss, void* stream) {
  if (n < 1 || !P || !X || !T || !grad || !loss) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_attr();
  if (e != cudaSuccess) return fail(e);
  const int nb = (n + kChunk - 1) / kChunk;
  Workspace w;
  if ((e = ws_alloc(nb, s, &w)) != cudaSuccess) return fail(e);
  mlp_count_kernel<<<1, 256, 0, s>>>(mask, (int64_t)n * NO, w.count);
  GradArgs a{n, P, X, T, mask, w.count, w.partials, w.loss_part, nullptr};
  mlp_grad_kernel<<<nb, kThreads, kGradSmem, s>>>(a);
  mlp_reduce_kernel<<<(NP + 255) / 256, 256, 0, s>>>(w.partials, w.loss_part, nb, grad, loss, nullptr, nullptr, 0);
  e = cudaGetLastError();
  cudaFreeAsync(w.base, s);
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_loss_grad_noalloc(int32_t n, const float* P, const float* X, const float* T, const float* mask,
                                    float* grad, float* loss, void* stream) {
  if (n < 1 || !P || !X || !T || !grad || !loss) return GEMM_ERR_INVALID_ARG;
  if (n > kNoAllocMaxSamples) return GEMM_ERR_UNSUPPORTED;  // beyond the static scratch
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_attr();
  if (e != cudaSuccess) return fail(e);
  float* base = noalloc_scratch(&e);
  if (!base) return fail(e);
  float* partials = base;
  float* loss_part = base + (size_t)kNoAllocMaxBlocks * NP;
  float* count = loss_part + kNoAllocMaxBlocks;
  // Every scratch value read below is written earlier in this call (count, then
  // the partials and losses of blocks 0..nb-1), so nothing needs clearing.
  const int nb = (n + kChunk - 1) / kChunk;
  mlp_count_kernel<<<1, 256, 0, s>>>(mask, (int64_t)n * NO, count);
  GradArgs a{n, P, X, T, mask, count, partials, loss_part, nullptr};
  mlp_grad_kernel<<<nb, kThreads, kGradSmem, s>>>(a);
  mlp_reduce_kernel<<<(NP + 255) / 256, 256, 0, s>>>(partials, loss_part, nb, grad, loss, nullptr, nullptr, 0);
  e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_adam_step(float* P, const float* g, float* m, float* v, int32_t t, float lr, float b1, float b2,
                            float eps, void* stream) {
  if (!P || !g || !m || !v || t < 1 || !(lr > 0.f)) return GEMM_ERR_INVALID_ARG;
  mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(P, g, m, v, nullptr, t, lr, b1,
                                                                                   b2, eps);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t mlp_train(int32_t n, float* P, const float* X, const float* T, const float* mask, float* m, float* v,
                        int32_t t0, int32_t steps, float lr, float b1, float b2, float eps, float* loss_hist,
                        void* stream) {
  if (n < 1 || !P || !X || !T || !m || !v || t0 < 0 || steps < 0 || !(lr > 0.f)) return GEMM_ERR_INVALID_ARG;
  if (steps == 0) return GEMM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_attr();
  if (e != cudaSuccess) return fail(e);
  const int nb = (n + kChunk - 1) / kChunk;
  Workspace w;
  if ((e = ws_alloc(nb, s, &w)) != cudaSuccess) return fail(e);
  mlp_count_kernel<<<1, 256, 0, s>>>(mask, (int64_t)n * NO, w.count);
  e = cudaMemcpyAsync(w.step, &t0, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    GradArgs a{n, P, X, T, mask, w.count, w.partials, w.loss_part, w.step};
    mlp_grad_kernel<<<nb, kThreads, kGradSmem, cap>>>(a);
    mlp_reduce_kernel<<<(NP + 255) / 256, 256, 0, cap>>>(w.partials, w.loss_part, nb, w.grad, w.loss, loss_hist,
                                                         w.step, t0);
    mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, cap>>>(P, w.grad, m, v, w.step, 0, lr, b1, b2, eps);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    e = (e2 != cudaSuccess) ? e2 : cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  for (int i = 0; i < steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  cudaFreeAsync(w.base, s);
  cudaStreamSynchronize(s);
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

gemm_status_t select_kernels_batched(gemm_handle_t h, int32_t n, const int64_t* shapes, int32_t* ids_out,
                                     float* pred, void* stream) {
  if (!h || n < 0 || (n > 0 && (!shapes || !ids_out))) return GEMM_ERR_INVALID_ARG;
  if (h->mlp.empty()) return GEMM_ERR_UNSUPPORTED;
  if ((int)h->ids.size() > NO) return GEMM_ERR_UNSUPPORTED;
  if (n == 0) return GEMM_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return fail(e);
  float* P = nullptr;
  {
    std::lock_guard<std::mutex> g(h->dev_mu);
    if (!h->dev_mlp[dev]) {
      float* p = nullptr;
      if ((e = cudaMalloc(&p, sizeof(float) * NP)) != cudaSuccess) return fail(e);
      if ((e = cudaMemcpy(p, h->mlp.data(), sizeof(float) * NP, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(p);
        return fail(e);
      }
      h->dev_mlp[dev] = p;
    }
    P = h->dev_mlp[dev];
  }
  Ids ids{};
  for (size_t i = 0; i < h->ids.size(); ++i) ids.v[i] = h->ids[i];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* dids = nullptr;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(&dids), sizeof(ids.v), s)) != cudaSuccess) return fail(e);
  e = cudaMemcpyAsync(dids, ids.v, sizeof(ids.v), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    mlp_forward_kernel<true><<<(n + 127) / 128, 128, 0, s>>>(n, P, nullptr, shapes, pred, (int)h->ids.size(), dids,
                                                           ids_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dids, s);
  return e == cudaSuccess ? GEMM_OK : fail(e);
}

}  // extern "C"
