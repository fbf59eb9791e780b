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

// Fused Adam over up to 8 tensors laid end to end in one index space of work
// units: four elements (one 128-bit access per array) where all four arrays of
// a tensor are 16-byte aligned, else one element.
struct AdamSet {
  s3r_adam_tensor t[S3R_ADAM_MAX_TENSORS];
  int64_t ustart[S3R_ADAM_MAX_TENSORS + 1];   // first work unit of each tensor
  int vec[S3R_ADAM_MAX_TENSORS];
  int count;
  float lr, b1, b2, eps, inv_bc1, inv_sqrt_bc2;
  const uint32_t* gate;   // optional device word: the step is skipped unless it reads 0
};

__device__ __forceinline__ void adam1(const AdamSet& s, float& p, float g, float& m, float& v) {
  m = fmaf(s.b1, m, (1.f - s.b1) * g);
  v = fmaf(s.b2, v, (1.f - s.b2) * g * g);
  p -= s.lr * (m * s.inv_bc1) / (sqrtf(v) * s.inv_sqrt_bc2 + s.eps);
}

__global__ void k_adam(const __grid_constant__ AdamSet s) {
  if (s.gate && *s.gate != 0u) return;   // an earlier call of the step failed: change nothing
  const int64_t total = s.ustart[s.count];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < total;
       u += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (u >= s.ustart[k + 1]) ++k;
    const s3r_adam_tensor& t = s.t[k];
    if (s.vec[k]) {
      const int64_t e = 4 * (u - s.ustart[k]);
      if (e + 4 <= t.n) {
        float4 p = *reinterpret_cast<const float4*>(t.param + e);
        const float4 g = *reinterpret_cast<const float4*>(t.grad + e);
        float4 m = *reinterpret_cast<const float4*>(t.exp_avg + e);
        float4 v = *reinterpret_cast<const float4*>(t.exp_avg_sq + e);
        adam1(s, p.x, g.x, m.x, v.x);
        adam1(s, p.y, g.y, m.y, v.y);
        adam1(s, p.z, g.z, m.z, v.z);
        adam1(s, p.w, g.w, m.w, v.w);
        *reinterpret_cast<float4*>(t.param + e) = p;
        *reinterpret_cast<float4*>(t.exp_avg + e) = m;
        *reinterpret_cast<float4*>(t.exp_avg_sq + e) = v;
      } else {
        for (int64_t i = e; i < t.n; ++i) adam1(s, t.param[i], t.grad[i], t.exp_avg[i], t.exp_avg_sq[i]);
      }
    } else {
      const int64_t i = u - s.ustart[k];
      adam1(s, t.param[i], t.grad[i], t.exp_avg[i], t.exp_avg_sq[i]);
    }
  }
}

}  // namespace

cudaError_t launch_adam(const s3r_adam_tensor* t, int count, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, const uint32_t* gate, cudaStream_t st) {
  AdamSet s;
  s.count = count;
  s.gate = gate;
  s.ustart[0] = 0;
  for (int k = 0; k < count; ++k) {
    s.t[k] = t[k];
    const bool al = ((reinterpret_cast<uintptr_t>(t[k].param) | reinterpret_cast<uintptr_t>(t[k].grad) |
                      reinterpret_cast<uintptr_t>(t[k].exp_avg) |
                      reinterpret_cast<uintptr_t>(t[k].exp_avg_sq)) & 15u) == 0;
    s.vec[k] = al ? 1 : 0;
    s.ustart[k + 1] = s.ustart[k] + (al ? (t[k].n + 3) / 4 : t[k].n);
  }
  for (int k = count; k < S3R_ADAM_MAX_TENSORS; ++k) {
    s.t[k] = s3r_adam_tensor{nullptr, nullptr, nullptr, nullptr, 0};
    s.vec[k] = 0;
    s.ustart[k + 1] = s.ustart[count];
  }
  s.lr = lr; s.b1 = b1; s.b2 = b2; s.eps = eps;
  s.inv_bc1 = 1.f / bc1;
  s.inv_sqrt_bc2 = 1.f / sqrtf(bc2);
  const int64_t total = s.ustart[count];
  if (total == 0) return cudaSuccess;
  // four 256-thread blocks per SM: on the GB300 a grid-stride stream of
  // this mix (four 16-byte loads, three 16-byte stores per thread and step)
  // measured 6.7 TB/s with four blocks per SM against 5.9 TB/s with six to
  // eight (fewer concurrent DRAM streams) and 6.3 TB/s with two vector units
  // per thread
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)sm_count() * 4) blocks = (int64_t)sm_count() * 4;
  k_adam<<<(unsigned)blocks, 256, 0, st>>>(s);
  return cudaGetLastError();
}

namespace {
__global__ void k_zero(uint4* p4, int64_t n4, uint32_t* tail, int tail_words) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x)
    p4[i] = make_uint4(0u, 0u, 0u, 0u);
  if (blockIdx.x == 0 && (int)threadIdx.x < tail_words) tail[threadIdx.x] = 0u;
}
}  // namespace

cudaError_t launch_zero(void* p, int64_t words, cudaStream_t st) {
  if (words <= 0) return cudaSuccess;
  const int64_t n4 = words / 4;
  int64_t blocks = (n4 + 255) / 256;
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  if (blocks < 1) blocks = 1;
  k_zero<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<uint4*>(p), n4,
                                           reinterpret_cast<uint32_t*>(p) + 4 * n4,
                                           (int)(words - 4 * n4));
  return cudaGetLastError();
}

cudaError_t launch_l1_loss(int64_t n, const float* pred, const float* target, float* grad,
                           float* loss, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // the blocks add their partial sums to *loss: start it at zero
  cudaError_t e = launch_zero(loss, 1, st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  k_l1<<<(unsigned)blocks, 256, 0, st>>>(n, pred, target, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_visibility(int64_t n, float t, const uint32_t* mask, float* life, float* vis,
                              int mode, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sm_count() * 64) blocks = (int64_t)sm_count() * 64;
  k_vis<<<(unsigned)blocks, 256, 0, st>>>(n, t, mask, reinterpret_cast<float2*>(life),
                                          reinterpret_cast<float2*>(vis), mode);
  return cudaGetLastError();
}

}  // namespace s3r
