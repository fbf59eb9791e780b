// The temporal-visibility record (Sec. 3.3, "Temporal separation"):
//   RECORD   Eq. 5: l_s = min(l_s, t), l_e = max(l_e, t) where M_t[i];
//   FINALIZE Eq. 6: v = (l_s - 0.1, l_e + 0.1), in FP32;
//   RESET    v = (-1, 1), l = (1, -1): visible at all times, empty life.
// A plain streaming pass, one Gaussian (one 8-byte pair per array) per
// thread, so that sub-ranges starting at any index can be passed.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

__global__ void k_vis(int64_t n, float t, const uint32_t* __restrict__ mask, float2* life,
                      float2* vis, int mode) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mode == S3R_VIS_RESET) {
      vis[i] = make_float2(-1.f, 1.f);
      life[i] = make_float2(1.f, -1.f);
    } else if (mode == S3R_VIS_FINALIZE) {
      const float2 l = life[i];
      vis[i] = make_float2(l.x - 0.1f, l.y + 0.1f);
    } else if ((mask[i >> 5] >> (i & 31)) & 1u) {
      float2 l = life[i];
      l.x = fminf(l.x, t);
      l.y = fmaxf(l.y, t);
      life[i] = l;
    }
  }
}

// Mean absolute error and its gradient; one block-reduced atomic per CTA.
__global__ void k_l1(int64_t n, const float* __restrict__ pred, const float* __restrict__ target,
                     float* __restrict__ grad, float* loss) {
  __shared__ float s_part[8];
  const float inv_n = 1.f / (float)n;
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = pred[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
    atomicAdd(loss, t * inv_n);
  }
}

}  // namespace

cudaError_t launch_l1_loss(int64_t n, const float* pred, const float* target, float* grad,
                           float* loss, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_l1<<<(unsigned)blocks, 256, 0, st>>>(n, pred, target, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_visibility(int64_t n, float t, const uint32_t* mask, float* life, float* vis,
                              int mode, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_vis<<<(unsigned)blocks, 256, 0, st>>>(n, t, mask, reinterpret_cast<float2*>(life),
                                          reinterpret_cast<float2*>(vis), mode);
  return cudaGetLastError();
}

}  // namespace s3r
