// The layers around the GEMMs of a convolutional network (Section 6: VGG16
// inference with the library's matrix multiply).  Activations are NHWC, so a
// 3x3 convolution is im2col (rows = output pixels, columns = (kh, kw, c))
// times the weights (Cout x 9 Cin, i.e. op(B) = B^T), and the GEMM's output
// rows are already the next NHWC activation.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"

namespace ks {
namespace {

// out[(n, h, w), (kh * 3 + kw) * C + c] = x[n, h + kh - 1, w + kw - 1, c], zero outside.
// V = 4 moves 4 channels per thread (C % 4 == 0, 16-byte aligned rows); the
// index type I is 32-bit whenever the element count allows, which keeps the
// per-element index arithmetic cheap on this memory-bound copy.
template <int V, typename I>
__global__ void im2col3x3_kernel(const float* __restrict__ x, int N, int H, int W, int C, float* __restrict__ out,
                                 int64_t ld) {
  const int CV = C / V;
  const I per_row = (I)9 * CV;
  const I total = (I)N * H * W * per_row;
  for (I t = (I)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
    const I row = t / per_row;
    const int q = (int)(t - row * per_row);
    const int tap = q / CV, c = (q - tap * CV) * V;
    const int kh = tap / 3, kw = tap - kh * 3;
    const I hw = row % ((I)H * W);
    const int n = (int)(row / ((I)H * W)), h = (int)(hw / W), w = (int)(hw - (I)h * W);
    const int hh = h + kh - 1, ww = w + kw - 1;
    float* dst = out + (int64_t)row * ld + tap * C + c;
    const bool inside = hh >= 0 && hh < H && ww >= 0 && ww < W;
    const float* src = x + (((int64_t)n * H + hh) * W + ww) * C + c;
    if constexpr (V == 4) {
      *reinterpret_cast<float4*>(dst) = inside ? __ldg(reinterpret_cast<const float4*>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      *dst = inside ? __ldg(src) : 0.f;
    }
  }
}

// y[r, j] = act(y[r, j] + bias[j]) over rows x cols with leading dimension ld, V columns per thread.
template <int V, typename I>
__global__ void bias_act_kernel(float* y, int64_t rows, int cols, int64_t ld, const float* bias, int relu) {
  const int cv = cols / V;
  const I total = (I)rows * cv;
  for (I t = (I)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
    const I r = t / cv;
    const int j = (int)(t - r * cv) * V;
    float* p = y + (int64_t)r * ld + j;
    if constexpr (V == 4) {
      float4 v = *reinterpret_cast<float4*>(p);
      if (bias) {
        const float4 b = __ldg(reinterpret_cast<const float4*>(bias + j));
        v.x += b.x; v.y += b.y; v.z += b.z; v.w += b.w;
      }
      if (relu) { v.x = fmaxf(v.x, 0.f); v.y = fmaxf(v.y, 0.f); v.z = fmaxf(v.z, 0.f); v.w = fmaxf(v.w, 0.f); }
      *reinterpret_cast<float4*>(p) = v;
    } else {
      float v = *p + (bias ? bias[j] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      *p = v;
    }
  }
}

// 2 x 2, stride 2 max pooling of NHWC x (H, W even), V channels per thread.
template <int V, typename I>
__global__ void maxpool2x2_kernel(const float* __restrict__ x, int N, int H, int W, int C, float* __restrict__ out) {
  const int Ho = H / 2, Wo = W / 2, CV = C / V;
  const I total = (I)N * Ho * Wo * CV;
  for (I t = (I)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
    const I p = t / CV;
    const int c = (int)(t - p * CV) * V;
    const I hw = p % ((I)Ho * Wo);
    const int n = (int)(p / ((I)Ho * Wo)), ho = (int)(hw / Wo), wo = (int)(hw - (I)ho * Wo);
    const float* b = x + (((int64_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
    const int64_t rs = (int64_t)W * C;
    if constexpr (V == 4) {
      const float4 a0 = __ldg(reinterpret_cast<const float4*>(b)), a1 = __ldg(reinterpret_cast<const float4*>(b + C));
      const float4 a2 = __ldg(reinterpret_cast<const float4*>(b + rs));
      const float4 a3 = __ldg(reinterpret_cast<const float4*>(b + rs + C));
      *reinterpret_cast<float4*>(out + (int64_t)p * C + c) =
          make_float4(fmaxf(fmaxf(a0.x, a1.x), fmaxf(a2.x, a3.x)), fmaxf(fmaxf(a0.y, a1.y), fmaxf(a2.y, a3.y)),
                      fmaxf(fmaxf(a0.z, a1.z), fmaxf(a2.z, a3.z)), fmaxf(fmaxf(a0.w, a1.w), fmaxf(a2.w, a3.w)));
    } else {
      out[(int64_t)p * C + c] = fmaxf(fmaxf(b[0], b[C]), fmaxf(b[rs], b[rs + C]));
    }
  }
}

// The same im2col from NCHW activations (the GEMM-batched layout of Section 6,
// where each image's output is Cout x (H W)): out[(n, h, w), (kh * 3 + kw) * C + c]
// = x[n, c, h + kh - 1, w + kw - 1].  Consecutive threads write consecutive columns.
template <typename I>
__global__ void im2col3x3_nchw_kernel(const float* __restrict__ x, int N, int C, int H, int W,
                                      float* __restrict__ out, int64_t ld) {
  const I per_row = (I)9 * C;
  const I total = (I)N * H * W * per_row;
  for (I t = (I)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
    const I row = t / per_row;
    const int q = (int)(t - row * per_row);
    const int tap = q / C, c = q - tap * C;
    const int kh = tap / 3, kw = tap - kh * 3;
    const I hw = row % ((I)H * W);
    const int n = (int)(row / ((I)H * W)), h = (int)(hw / W), w = (int)(hw - (I)h * W);
    const int hh = h + kh - 1, ww = w + kw - 1;
    const bool inside = hh >= 0 && hh < H && ww >= 0 && ww < W;
    out[(int64_t)row * ld + q] = inside ? __ldg(x + (((int64_t)n * C + c) * H + hh) * W + ww) : 0.f;
  }
}

// y[n, c, p] = act(y[n, c, p] + bias[c]) for NCHW activations (p over H W).
template <typename I>
__global__ void bias_act_nchw_kernel(float* y, int N, int C, int64_t HW, const float* bias, int relu) {
  const I total = (I)N * C * HW;
  for (I t = (I)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (I)gridDim.x * blockDim.x) {
    const int c = (int)((t / (I)HW) % C);
    float v = y[t] + (bias ? __ldg(bias + c) : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    y[t] = v;
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int grid_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

gemm_status_t done(cudaError_t e) {
  if (e == cudaSuccess) return GEMM_OK;
  set_last_cuda_error(e);
  return GEMM_ERR_CUDA;
}
}  // namespace
}  // namespace ks

using namespace ks;

extern "C" {

gemm_status_t kselect_im2col3x3(const float* x, int32_t N, int32_t H, int32_t W, int32_t C, float* out, int64_t ld,
                                void* stream) {
  if (N < 0 || H < 0 || W < 0 || C < 1 || ld < 9LL * C) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)N * H * W * 9 * C;
  if (total == 0) return GEMM_OK;
  if (!x || !out) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vec = C % 4 == 0 && ld % 4 == 0 && aligned16(x) && aligned16(out);
  const int64_t work = vec ? total / 4 : total;
  const bool small = work < ((int64_t)1 << 31) - 152LL * 32 * 256;
  if (vec && small) im2col3x3_kernel<4, int32_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out, ld);
  else if (vec) im2col3x3_kernel<4, int64_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out, ld);
  else if (small) im2col3x3_kernel<1, int32_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out, ld);
  else im2col3x3_kernel<1, int64_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out, ld);
  return done(cudaGetLastError());
}

gemm_status_t kselect_bias_act(float* y, int64_t rows, int32_t cols, int64_t ld, const float* bias, int32_t relu,
                               void* stream) {
  if (rows < 0 || cols < 0 || ld < cols) return GEMM_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return GEMM_OK;
  if (!y) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vec = cols % 4 == 0 && ld % 4 == 0 && aligned16(y) && (!bias || aligned16(bias));
  const int64_t work = vec ? rows * (cols / 4) : rows * cols;
  const bool small = work < ((int64_t)1 << 31) - 152LL * 32 * 256;
  if (vec && small) bias_act_kernel<4, int32_t><<<grid_for(work), 256, 0, s>>>(y, rows, cols, ld, bias, relu);
  else if (vec) bias_act_kernel<4, int64_t><<<grid_for(work), 256, 0, s>>>(y, rows, cols, ld, bias, relu);
  else if (small) bias_act_kernel<1, int32_t><<<grid_for(work), 256, 0, s>>>(y, rows, cols, ld, bias, relu);
  else bias_act_kernel<1, int64_t><<<grid_for(work), 256, 0, s>>>(y, rows, cols, ld, bias, relu);
  return done(cudaGetLastError());
}

gemm_status_t kselect_maxpool2x2(const float* x, int32_t N, int32_t H, int32_t W, int32_t C, float* out,
                                 void* stream) {
  if (N < 0 || H < 0 || W < 0 || C < 1 || (H % 2) || (W % 2)) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)N * (H / 2) * (W / 2) * C;
  if (total == 0) return GEMM_OK;
  if (!x || !out) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vec = C % 4 == 0 && aligned16(x) && aligned16(out);
  const int64_t work = vec ? total / 4 : total;
  const bool small = work < ((int64_t)1 << 31) - 152LL * 32 * 256;
  if (vec && small) maxpool2x2_kernel<4, int32_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out);
  else if (vec) maxpool2x2_kernel<4, int64_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out);
  else if (small) maxpool2x2_kernel<1, int32_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out);
  else maxpool2x2_kernel<1, int64_t><<<grid_for(work), 256, 0, s>>>(x, N, H, W, C, out);
  return done(cudaGetLastError());
}

gemm_status_t kselect_im2col3x3_nchw(const float* x, int32_t N, int32_t C, int32_t H, int32_t W, float* out,
                                     int64_t ld, void* stream) {
  if (N < 0 || H < 0 || W < 0 || C < 1 || ld < 9LL * C) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)N * H * W * 9 * C;
  if (total == 0) return GEMM_OK;
  if (!x || !out) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (total < ((int64_t)1 << 31) - 152LL * 32 * 256)
    im2col3x3_nchw_kernel<int32_t><<<grid_for(total), 256, 0, s>>>(x, N, C, H, W, out, ld);
  else
    im2col3x3_nchw_kernel<int64_t><<<grid_for(total), 256, 0, s>>>(x, N, C, H, W, out, ld);
  return done(cudaGetLastError());
}

gemm_status_t kselect_bias_act_nchw(float* y, int32_t N, int32_t C, int64_t HW, const float* bias, int32_t relu,
                                    void* stream) {
  if (N < 0 || C < 1 || HW < 0) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)N * C * HW;
  if (total == 0) return GEMM_OK;
  if (!y) return GEMM_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (total < ((int64_t)1 << 31) - 152LL * 32 * 256)
    bias_act_nchw_kernel<int32_t><<<grid_for(total), 256, 0, s>>>(y, N, C, HW, bias, relu);
  else
    bias_act_nchw_kernel<int64_t><<<grid_for(total), 256, 0, s>>>(y, N, C, HW, bias, relu);
  return done(cudaGetLastError());
}

}  // extern "C"
