// Front-to-back alpha blending of every 16x16 tile (Eq. 2) and its exact
// adjoint.
//
// Forward: one CTA of 256 threads per tile, one pixel per thread. The tile's
// front-to-back splat list is consumed in batches of 256: each thread gathers
// one splat record (uv, conic+opacity, rgb) into shared memory, then every
// thread blends the batch for its pixel. alpha = min(0.99, o G) is skipped
// below 1/255, and a pixel stops before its transmittance would fall under
// 1e-4; the CTA stops when all its pixels have stopped. The final
// transmittance and the count of visited splats up to the last blended one
// are stored per pixel.
//
// Backward: the same tiles walked back to front, starting at each pixel's
// last blended splat. The transmittance before each splat is recovered from
// the stored final value as T <- T / (1 - alpha), so no per-pixel lists are
// kept. Per splat the nine adjoints (uv, conic, opacity, rgb) are summed over
// the warp with shuffles, then over the CTA in shared memory, and flushed to
// global memory with one vector atomic per four floats.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kThreads = kTilePixels;   // 256
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

struct BlendArgs {
  const uint2* ranges;
  const uint32_t* sorted_splats;
  const float2* sp_xy;
  const float4* sp_conic_o;
  const float4* sp_rgb_d;
  const float* bg;
  const float* dL;        // backward only
  float* out;             // forward only
  float* final_T;
  uint32_t* n_contrib;
  float* sp_grad;         // backward only, [S*12]
  unsigned long long* pairs;  // forward only: evaluated (pixel, splat) pairs
};

__device__ __forceinline__ int view_of_tile(const ViewSet& vs, int tile) {
  int v = 0;
  while (v + 1 < vs.n_views && vs.v[v + 1].tile_base <= tile) ++v;
  return v;
}

__global__ void __launch_bounds__(kThreads) k_blend_fwd(const __grid_constant__ ViewSet vs,
                                                        BlendArgs a) {
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_co[kThreads];
  __shared__ float4 s_rgb[kThreads];
  const int tile = blockIdx.x;
  const int v = view_of_tile(vs, tile);
  const ViewInfo& vi = vs.v[v];
  const int lt = tile - vi.tile_base;
  const int tx = lt % vi.gx, ty = lt / vi.gx;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < vi.width && py < vi.height;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const uint2 range = a.ranges[tile];
  const int n = (int)(range.y - range.x);

  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t contributor = 0, last = 0;
  bool done = !inside;
  for (int b0 = 0; b0 < n; b0 += kThreads) {
    if (__syncthreads_count(done) == kThreads) break;
    const int i = b0 + threadIdx.x;
    if (i < n) {
      const uint32_t s = a.sorted_splats[range.x + i];
      s_xy[threadIdx.x] = a.sp_xy[s];
      s_co[threadIdx.x] = a.sp_conic_o[s];
      s_rgb[threadIdx.x] = a.sp_rgb_d[s];
    }
    __syncthreads();
    const int m = min(kThreads, n - b0);
    for (int j = 0; j < m && !done; ++j) {
      ++contributor;
      const float2 xy = s_xy[j];
      const float4 co = s_co[j];
      const float dx = xy.x - fx, dy = xy.y - fy;
      const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
      if (power > 0.f) continue;
      const float alpha = fminf(kAlphaMax, co.w * __expf(power));
      if (alpha < kAlphaMin) continue;
      const float nT = T * (1.f - alpha);
      if (nT < kTStop) {
        done = true;
        break;
      }
      const float4 c = s_rgb[j];
      const float w = alpha * T;
      C0 = fmaf(c.x, w, C0);
      C1 = fmaf(c.y, w, C1);
      C2 = fmaf(c.z, w, C2);
      T = nT;
      last = contributor;
    }
  }
  // work accounting: one 64-bit atomic per warp
  unsigned long long visited = contributor;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) visited += __shfl_xor_sync(0xffffffffu, visited, o);
  if ((threadIdx.x & 31) == 0 && visited) atomicAdd(a.pairs, visited);
  if (inside) {
    const int64_t plane = (int64_t)vi.width * vi.height;
    const int64_t pix = (int64_t)py * vi.width + px;
    float* o = a.out + 3 * (int64_t)vi.pix_base + pix;
    o[0] = fmaf(T, a.bg[0], C0);
    o[plane] = fmaf(T, a.bg[1], C1);
    o[2 * plane] = fmaf(T, a.bg[2], C2);
    a.final_T[vi.pix_base + pix] = T;
    a.n_contrib[vi.pix_base + pix] = last;
  }
}

// Sum eight values over the warp with 9 shuffles instead of 8 x 5: at each
// butterfly level every lane keeps half of its remaining values and sends the
// other half to its partner. On return, lane l holds the warp total of value
// index 4*bit4(l) + 2*bit3(l) + bit2(l); lanes 4m (m = 0..7) hold value m.
__device__ __forceinline__ float warp_sum8_transposed(const float v[8], uint32_t lane) {
  const bool b4 = lane & 16u, b3 = lane & 8u, b2 = lane & 4u;
  float k4[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = b4 ? v[j] : v[j + 4];
    const float keep = b4 ? v[j + 4] : v[j];
    k4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float k2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = b3 ? k4[j] : k4[j + 2];
    const float keep = b3 ? k4[j + 2] : k4[j];
    k2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = b2 ? k2[0] : k2[1];
  float k1 = (b2 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
  return k1;
}

__device__ __forceinline__ void red_v4(float* p, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z),
               "f"(w)
               : "memory");
}

__global__ void __launch_bounds__(kThreads) k_blend_bwd(const __grid_constant__ ViewSet vs,
                                                        BlendArgs a) {
  __shared__ float2 s_xy[kThreads];
  __shared__ float4 s_co[kThreads];
  __shared__ float4 s_rgb[kThreads];
  __shared__ uint32_t s_id[kThreads];
  __shared__ float s_g[kThreads][9];
  __shared__ uint32_t s_max;
  const int tile = blockIdx.x;
  const int v = view_of_tile(vs, tile);
  const ViewInfo& vi = vs.v[v];
  const int lt = tile - vi.tile_base;
  const int tx = lt % vi.gx, ty = lt / vi.gx;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < vi.width && py < vi.height;
  const float fx = px + 0.5f, fy = py + 0.5f;
  const uint2 range = a.ranges[tile];

  float T = 1.f, d0 = 0.f, d1 = 0.f, d2 = 0.f;
  uint32_t last = 0;
  if (threadIdx.x == 0) s_max = 0;
  if (inside) {
    const int64_t plane = (int64_t)vi.width * vi.height;
    const int64_t pix = (int64_t)py * vi.width + px;
    const float* g = a.dL + 3 * (int64_t)vi.pix_base + pix;
    d0 = g[0];
    d1 = g[plane];
    d2 = g[2 * plane];
    T = a.final_T[vi.pix_base + pix];
    last = a.n_contrib[vi.pix_base + pix];
  }
  __syncthreads();
  if (last) atomicMax(&s_max, last);
  const float T_final = T;
  const float bg_dot = a.bg[0] * d0 + a.bg[1] * d1 + a.bg[2] * d2;
  float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;          // colour behind the current splat
  float last_alpha = 0.f, lc0 = 0.f, lc1 = 0.f, lc2 = 0.f;
  __syncthreads();
  const int n = (int)s_max;
  const uint32_t lane = lane_id();

  for (int hi = n; hi > 0; hi -= kThreads) {
    const int lo = max(0, hi - kThreads);
    const int m = hi - lo;
    __syncthreads();
    if (threadIdx.x < m) {
      const uint32_t s = a.sorted_splats[range.x + lo + threadIdx.x];
      s_id[threadIdx.x] = s;
      s_xy[threadIdx.x] = a.sp_xy[s];
      s_co[threadIdx.x] = a.sp_conic_o[s];
      s_rgb[threadIdx.x] = a.sp_rgb_d[s];
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) s_g[threadIdx.x][q] = 0.f;
    __syncthreads();
    for (int j = m - 1; j >= 0; --j) {
      const int pos = lo + j;
      bool act = inside && pos < (int)last;
      float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f;
      float g_r = 0.f, g_g = 0.f, g_bl = 0.f;
      if (act) {
        const float2 xy = s_xy[j];
        const float4 co = s_co[j];
        const float dx = xy.x - fx, dy = xy.y - fy;
        const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
        const float G = __expf(power);
        const float raw = co.w * G;
        const float alpha = fminf(kAlphaMax, raw);
        act = !(power > 0.f) && !(alpha < kAlphaMin);
        if (act) {
          const float4 c = s_rgb[j];
          const float one_m = 1.f - alpha;
          T = T / one_m;
          const float w = alpha * T;
          g_r = w * d0;
          g_g = w * d1;
          g_bl = w * d2;
          acc0 = last_alpha * lc0 + (1.f - last_alpha) * acc0;
          acc1 = last_alpha * lc1 + (1.f - last_alpha) * acc1;
          acc2 = last_alpha * lc2 + (1.f - last_alpha) * acc2;
          lc0 = c.x; lc1 = c.y; lc2 = c.z;
          float dalpha = (c.x - acc0) * d0 + (c.y - acc1) * d1 + (c.z - acc2) * d2;
          dalpha *= T;
          last_alpha = alpha;
          dalpha -= T_final / one_m * bg_dot;
          if (!(raw > kAlphaMax)) {
            g_o = G * dalpha;
            const float dpow = co.w * G * dalpha;
            g_u = dpow * (-co.x * dx - co.y * dy);
            g_v = dpow * (-co.z * dy - co.y * dx);
            g_a = dpow * (-0.5f * dx * dx);
            g_b = dpow * (-dx * dy);
            g_c = dpow * (-0.5f * dy * dy);
          }
        }
      }
      if (__any_sync(0xffffffffu, act)) {
        const float eight[8] = {g_u, g_v, g_a, g_b, g_c, g_o, g_r, g_g};
        const float tot = warp_sum8_transposed(eight, lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g_bl += __shfl_xor_sync(0xffffffffu, g_bl, o);
        if ((lane & 3u) == 0) atomicAdd(&s_g[j][lane >> 2], tot);
        if (lane == 0) atomicAdd(&s_g[j][8], g_bl);
      }
    }
    __syncthreads();
    if (threadIdx.x < m) {
      const float* sg = s_g[threadIdx.x];
      bool any = false;
#pragma unroll
      for (int q = 0; q < 9; ++q) any |= sg[q] != 0.f;
      if (any) {
        float* dst = a.sp_grad + 12 * (size_t)s_id[threadIdx.x];
        red_v4(dst, sg[0], sg[1], sg[2], sg[3]);
        red_v4(dst + 4, sg[4], sg[5], sg[6], sg[7]);
        atomicAdd(dst + 8, sg[8]);
      }
    }
  }
}

// Zero the per-splat adjoints of the splats written by the last projection.
__global__ void k_zero_grads(float4* g, const uint32_t* ctr, int64_t cap) {
  const int64_t n = 3 * min((int64_t)ctr[kCtrSplats], cap);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

static BlendArgs make_args(s3r_workspace* ws) {
  BlendArgs a;
  a.ranges = ws->ranges;
  a.sorted_splats = ws->dup_val[ws->dup_final];
  a.sp_xy = ws->sp_xy;
  a.sp_conic_o = ws->sp_conic_o;
  a.sp_rgb_d = ws->sp_rgb_d;
  a.final_T = ws->final_T;
  a.n_contrib = ws->n_contrib;
  a.sp_grad = ws->sp_grad;
  a.pairs = reinterpret_cast<unsigned long long*>(ws->ctr + kCtrPairs);
  a.bg = nullptr;
  a.dL = nullptr;
  a.out = nullptr;
  return a;
}

cudaError_t launch_render_fwd(s3r_workspace* ws, const float* bg, float* out, cudaStream_t st) {
  BlendArgs a = make_args(ws);
  a.bg = bg;
  a.out = out;
  if (ws->views.total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.pairs, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  KernelTimer timer(ws, kKBlendFwd, st);
  k_blend_fwd<<<ws->views.total_tiles, kThreads, 0, st>>>(ws->views, a);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(s3r_workspace* ws, const float* bg, const float* dL,
                              cudaStream_t st) {
  BlendArgs a = make_args(ws);
  a.bg = bg;
  a.dL = dL;
  {
    KernelTimer timer(ws, kKZeroGrads, st);
    k_zero_grads<<<ws->num_sms * 4, 256, 0, st>>>(reinterpret_cast<float4*>(ws->sp_grad), ws->ctr,
                                                  ws->cap.max_splats);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ws->views.total_tiles == 0) return cudaSuccess;
  KernelTimer timer(ws, kKBlendBwd, st);
  k_blend_bwd<<<ws->views.total_tiles, kThreads, 0, st>>>(ws->views, a);
  return cudaGetLastError();
}

}  // namespace s3r
