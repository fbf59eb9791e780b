// Temporal selection (Sec. 3.3, "Temporal separation"): the ascending list of
// Gaussians whose visibility window [v_s, v_e] contains t, as one streaming
// pass over the record.
//
// Each warp owns 512 consecutive Gaussians and reads them as 8 rounds of
// 128-bit loads (one float4 = two (v_s, v_e) pairs per lane). A warp ballot
// per round gives every selected Gaussian its rank; a block scan over the 8
// warps and a single-pass decoupled look-back over tiles give the global
// offset, so the output is written once, in order, coalesced.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 8;                            // float4 loads per lane
constexpr int kWarpSpan = kRounds * 32 * 2;           // Gaussians per warp
constexpr int kTileSpan = kWarps * kWarpSpan;         // 4096 Gaussians per tile

__global__ void k_begin(uint32_t* ctr, uint32_t* hist) {
  // one block: zero the per-call counters and histograms, bump the epoch
  for (int i = threadIdx.x; i < kHistCount * kRadix; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x < kCtrCount && threadIdx.x != kCtrStatus && threadIdx.x != kCtrEpoch &&
      threadIdx.x != kCtrPairs && threadIdx.x != kCtrPairs + 1)
    ctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) ctr[kCtrEpoch] = ctr[kCtrEpoch] + 1;
}

__global__ void __launch_bounds__(kThreads) k_compact(const float* __restrict__ vis, int64_t n,
                                                      float t, uint32_t* __restrict__ sel,
                                                      uint32_t* ctr,
                                                      unsigned long long* lookback) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_base;
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const uint32_t tag = stage_tag(ctr[kCtrEpoch], kStageCompact);
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ctr + kCtrTileBase + kStageCompact, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) return;
    const int64_t g0 = tile * kTileSpan + (int64_t)warp * kWarpSpan;

    uint32_t b0[kRounds], b1[kRounds];
    uint32_t count = 0;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t g = g0 + 2 * (r * 32 + (int64_t)lane);
      float4 w = make_float4(1.f, -1.f, 1.f, -1.f);  // empty windows
      if (g + 1 < n) {
        w = __ldcs(reinterpret_cast<const float4*>(vis + 2 * g));
      } else if (g < n) {
        const float2 h = __ldcs(reinterpret_cast<const float2*>(vis + 2 * g));
        w.x = h.x; w.y = h.y;
      }
      const bool f0 = (w.x <= t) && (t <= w.y);
      const bool f1 = (w.z <= t) && (t <= w.w);
      b0[r] = __ballot_sync(0xffffffffu, f0);
      b1[r] = __ballot_sync(0xffffffffu, f1);
      count += __popc(b0[r]) + __popc(b1[r]);
    }
    if (lane == 0) s_warp[warp] = count;
    __syncthreads();
    if (warp == 0) {
      const uint32_t c = lane < kWarps ? s_warp[lane] : 0u;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t prefix = warp_lookback(lookback, tile, tag, total, ctr);
      if (lane < kWarps) s_warp[lane] = incl - c;
      if (lane == 0) {
        s_base = prefix;
        if (tile == n_tiles - 1) ctr[kCtrSelected] = prefix + total;
      }
    }
    __syncthreads();
    uint32_t out = s_base + s_warp[warp];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t g = g0 + 2 * (r * 32 + (int64_t)lane);
      const uint32_t before = __popc(b0[r] & lt) + __popc(b1[r] & lt);
      const bool f0 = (b0[r] >> lane) & 1u;
      const bool f1 = (b1[r] >> lane) & 1u;
      if (f0) sel[out + before] = (uint32_t)g;
      if (f1) sel[out + before + (f0 ? 1u : 0u)] = (uint32_t)(g + 1);
      out += __popc(b0[r]) + __popc(b1[r]);
    }
    __syncthreads();  // s_tile / s_warp reuse
  }
}

}  // namespace

cudaError_t launch_begin(s3r_workspace* ws, cudaStream_t st) {
  KernelTimer timer(ws, kKBegin, st);
  k_begin<<<1, 256, 0, st>>>(ws->ctr, ws->hist);
  return cudaGetLastError();
}

cudaError_t launch_compact(s3r_workspace* ws, const float* vis, int64_t n, float t,
                           cudaStream_t st) {
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  int64_t grid = ws->num_sms * 8;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  KernelTimer timer(ws, kKCompact, st);
  k_compact<<<(unsigned)grid, kThreads, 0, st>>>(vis, n, t, ws->selected, ws->ctr, ws->lookback);
  return cudaGetLastError();
}

}  // namespace s3r
