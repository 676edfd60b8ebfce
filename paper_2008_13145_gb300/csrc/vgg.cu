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
__global__ void im2col3x3_kernel(const float* __restrict__ x, int N, int H, int W, int C, float* __restrict__ out,
                                 int64_t ld) {
  const int64_t K = 9LL * C;
  const int64_t total = (int64_t)N * H * W * K;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / K;
    const int col = (int)(t - row * K);
    const int c = col % C, tap = col / C, kw = tap % 3, kh = tap / 3;
    const int w = (int)(row % W), h = (int)((row / W) % H), n = (int)(row / ((int64_t)W * H));
    const int hh = h + kh - 1, ww = w + kw - 1;
    float v = 0.f;
    if (hh >= 0 && hh < H && ww >= 0 && ww < W) v = x[(((int64_t)n * H + hh) * W + ww) * C + c];
    out[row * ld + col] = v;
  }
}

// y[r, j] = act(y[r, j] + bias[j]) over rows x cols with leading dimension ld.
__global__ void bias_act_kernel(float* y, int64_t rows, int cols, int64_t ld, const float* bias, int relu) {
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols;
    const int j = (int)(t - r * cols);
    float v = y[r * ld + j] + (bias ? bias[j] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    y[r * ld + j] = v;
  }
}

// 2 x 2, stride 2 max pooling of NHWC x (H, W even).
__global__ void maxpool2x2_kernel(const float* __restrict__ x, int N, int H, int W, int C, float* __restrict__ out) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)N * Ho * Wo * C;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % C);
    const int64_t p = t / C;
    const int wo = (int)(p % Wo), ho = (int)((p / Wo) % Ho), n = (int)(p / ((int64_t)Wo * Ho));
    const float* b = x + (((int64_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
    const int64_t rs = (int64_t)W * C;
    out[t] = fmaxf(fmaxf(b[0], b[C]), fmaxf(b[rs], b[rs + C]));
  }
}

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
  im2col3x3_kernel<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, N, H, W, C, out, ld);
  return done(cudaGetLastError());
}

gemm_status_t kselect_bias_act(float* y, int64_t rows, int32_t cols, int64_t ld, const float* bias, int32_t relu,
                               void* stream) {
  if (rows < 0 || cols < 0 || ld < cols) return GEMM_ERR_INVALID_ARG;
  if (rows == 0 || cols == 0) return GEMM_OK;
  if (!y) return GEMM_ERR_INVALID_ARG;
  bias_act_kernel<<<grid_for(rows * cols), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, rows, cols, ld, bias, relu);
  return done(cudaGetLastError());
}

gemm_status_t kselect_maxpool2x2(const float* x, int32_t N, int32_t H, int32_t W, int32_t C, float* out,
                                 void* stream) {
  if (N < 0 || H < 0 || W < 0 || C < 1 || (H % 2) || (W % 2)) return GEMM_ERR_INVALID_ARG;
  const int64_t total = (int64_t)N * (H / 2) * (W / 2) * C;
  if (total == 0) return GEMM_OK;
  if (!x || !out) return GEMM_ERR_INVALID_ARG;
  maxpool2x2_kernel<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, N, H, W, C, out);
  return done(cudaGetLastError());
}

}  // extern "C"
