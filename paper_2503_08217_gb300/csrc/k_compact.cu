// Temporal selection (Sec. 3.3, "Temporal separation"): the ascending list of
// Gaussians whose visibility window [v_s, v_e] contains t, as one streaming
// pass over the record.
//
// Each warp owns 512 consecutive Gaussians and reads them as 8 rounds of
// 128-bit loads (one float4 = two (v_s, v_e) pairs per lane). A warp ballot
// per round gives every selected Gaussian its rank; a block scan over the 8
// warps and a single-pass decoupled look-back over tiles give the global
// offset, so the output is written once, in order, coalesced.
#include <mutex>
#include <string>

#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 8;                            // float4 loads per lane
constexpr int kWarpSpan = kRounds * 32 * 2;           // Gaussians per warp
constexpr int kTileSpan = kWarps * kWarpSpan;         // 4096 Gaussians per tile

__global__ void k_begin(uint32_t* ctr, uint32_t* hist, unsigned long long* lookback,
                        int64_t lookback_words) {
  // one block: zero the per-call counters and histograms, bump the epoch
  for (int i = threadIdx.x; i < kHistCount * kRadix; i += blockDim.x) hist[i] = 0;
  const uint32_t epoch = ctr[kCtrEpoch] + 1;
  __syncthreads();   // every thread has read the old epoch
  // the status word, the epoch and the blend pair counts (which describe the
  // last counted render) survive
  if (threadIdx.x < kCtrCount && threadIdx.x != kCtrStatus && threadIdx.x != kCtrEpoch &&
      (threadIdx.x < kCtrPairs || threadIdx.x > kCtrEvalBwd + 1))
    ctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) ctr[kCtrEpoch] = epoch;
  // look-back tags keep the epoch's low 26 bits: when they wrap, words of the
  // call 2^26 calls ago would carry the current tags, so every word is
  // cleared (once per 67,108,864 calls)
  if ((epoch & ((1u << 26) - 1u)) == 0u)
    for (int64_t i = threadIdx.x; i < lookback_words; i += blockDim.x) lookback[i] = 0ull;
}

// Bits 2m (even) and 2m + 1 (odd) of a 32-bit word from bit m of the low
// halves of `even` and `odd`: the ballots of a round cover its Gaussians
// 2 lane and 2 lane + 1.
__device__ __forceinline__ uint32_t interleave16(uint32_t even, uint32_t odd) {
  auto spread = [](uint32_t x) {
    x &= 0xffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
  };
  return spread(even) | (spread(odd) << 1);
}

// sel_bits (may be null): bit i of word i / 32 set iff Gaussian i is
// selected; every word of every tile is written (zeros past n).
__global__ void __launch_bounds__(kThreads) k_compact(const float* __restrict__ vis, int64_t n,
                                                      float t, uint32_t* __restrict__ sel,
                                                      uint32_t* ctr,
                                                      unsigned long long* lookback,
                                                      uint32_t* __restrict__ sel_bits) {
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
    if (sel_bits && lane < 2 * kRounds) {
      // round r covers Gaussians g0 + 64 r .. + 63: two words, lanes 2r and 2r + 1
      uint32_t e = 0, o = 0;
#pragma unroll
      for (int r = 0; r < kRounds; ++r)
        if ((int)(lane >> 1) == r) { e = b0[r]; o = b1[r]; }
      const uint32_t sh = (lane & 1u) * 16u;
      sel_bits[(g0 >> 5) + lane] = interleave16(e >> sh, o >> sh);
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
  k_begin<<<1, 256, 0, st>>>(ws->ctr, ws->hist, ws->lookback, ws->lookback_words);
  return cudaGetLastError();
}

cudaError_t launch_compact(s3r_workspace* ws, const float* vis, int64_t n, float t,
                           cudaStream_t st) {
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  int64_t grid = (int64_t)ws->num_sms * 8;
  if (grid > n_tiles) grid = n_tiles;
  if (grid < 1) grid = 1;
  KernelTimer timer(ws, kKCompact, st);
  k_compact<<<(unsigned)grid, kThreads, 0, st>>>(vis, n, t, ws->selected, ws->ctr, ws->lookback,
                                                 ws->kept_bits);
  return cudaGetLastError();
}

}  // namespace s3r

namespace s3r {

// ---- allocation-free variant --------------------------------------------
// The same k_compact kernel, run on scratch that lives in a fixed array of
// the library's device image instead of a workspace: look-back words for up
// to S3R_STATIC_MAX_GAUSSIANS / 4096 tiles and the counters the kernel uses.
namespace {

constexpr int64_t kStaticTiles = S3R_STATIC_MAX_GAUSSIANS / kTileSpan;   // 16,384

struct StaticScratch {
  unsigned long long lookback[kStaticTiles];   // 128 KB
  uint32_t ctr[kCtrCount];
};

static __device__ __align__(256) StaticScratch g_static_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
StaticScratch* g_static_ptr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};

// Device address of the scratch array on the current device and the
// device's SM count, looked up once per device (host code cannot use the
// symbol itself as a device pointer).
s3r_status static_scratch(StaticScratch** out, int* sms) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_last_error(S3R_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return set_last_error(S3R_ERR_INVALID, "s3r_select_visible_static: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      const std::string msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return set_last_error(S3R_ERR_CUDA, msg.c_str());
    }
    int n_sms = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n_sms < 1) {
      const std::string msg = std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e);
      return set_last_error(S3R_ERR_CUDA, msg.c_str());
    }
    g_static_sms[dev] = n_sms;
    g_static_ptr[dev] = static_cast<StaticScratch*>(p);
  }
  *out = g_static_ptr[dev];
  *sms = g_static_sms[dev];
  return S3R_OK;
}

// The list length, or 0xffffffff where a look-back wait of the call gave up
// (the list is then not valid): the status word is only in the scratch, so
// the call reports it through its output.
__global__ void k_static_finish(const uint32_t* ctr, uint32_t* out_count) {
  *out_count = (ctr[kCtrStatus] & kStatusTimeout) ? 0xffffffffu : ctr[kCtrSelected];
}

}  // namespace
}  // namespace s3r

extern "C" s3r_status s3r_select_visible_static(int64_t n, float t, const float* vis_window,
                                                uint32_t* out_idx, uint32_t* out_count,
                                                void* stream) {
  using namespace s3r;
  if (n < 0 || n > S3R_STATIC_MAX_GAUSSIANS)
    return set_last_error(S3R_ERR_INVALID,
                          "s3r_select_visible_static: n must be in [0, 2^26] (the fixed scratch "
                          "holds look-back words for at most 67,108,864 Gaussians)");
  if (!out_count || ((uintptr_t)out_count & 3u))
    return set_last_error(S3R_ERR_INVALID, "s3r_select_visible_static: out_count must be a device uint32");
  if (n > 0 && (!vis_window || !out_idx || ((uintptr_t)vis_window & 15u) || ((uintptr_t)out_idx & 3u)))
    return set_last_error(S3R_ERR_INVALID,
                          "s3r_select_visible_static: vis_window (16-byte aligned) and out_idx are required");
  if (!(t == t)) return set_last_error(S3R_ERR_INVALID, "s3r_select_visible_static: t is NaN");
  StaticScratch* sc = nullptr;
  int sms = 0;
  s3r_status st = static_scratch(&sc, &sms);
  if (st != S3R_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  // the array keeps the previous call's contents: clear the counters and the
  // look-back words this call will use
  cudaError_t e = cudaMemsetAsync(sc->ctr, 0, sizeof(sc->ctr), s);
  if (e == cudaSuccess && n_tiles > 0)
    e = cudaMemsetAsync(sc->lookback, 0, sizeof(unsigned long long) * (size_t)n_tiles, s);
  if (e == cudaSuccess) {
    int64_t grid = (int64_t)sms * 8;
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    k_compact<<<(unsigned)grid, kThreads, 0, s>>>(vis_window, n, t, out_idx, sc->ctr, sc->lookback,
                                                   nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_static_finish<<<1, 1, 0, s>>>(sc->ctr, out_count);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_last_error(S3R_ERR_CUDA, cudaGetErrorString(e));
  return S3R_OK;
}
