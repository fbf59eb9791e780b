// Temporal selection (Sec. 3.3, "Temporal separation"): the ascending list of
// Gaussians whose visibility window [v_s, v_e] contains t, as one streaming
// pass over the record.
//
// A tile is 4096 consecutive Gaussians; each warp owns 512 of them and reads
// them as 8 rounds of 128-bit loads (one float4 = two (v_s, v_e) pairs per
// lane). A warp ballot per round gives every selected Gaussian its rank. A
// CTA takes a chunk of consecutive tiles, keeps their ballots in shared
// memory, and gets the chunk's global offset from the counts that all earlier
// chunks published (chunk_prefix), so the output is written once, in order,
// coalesced.
#include <mutex>
#include <string>

#include "s3r_math.cuh"

namespace s3r {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRounds = 8;                            // float4 loads per lane
constexpr int kWarpSpan = kRounds * 32 * 2;           // Gaussians per warp
constexpr int kTileSpan = kWarps * kWarpSpan;         // 4096 Gaussians per tile
constexpr int kChunkTiles = kThreads / kWarps;        // tiles a CTA holds (one offset per thread)

// W_v * P_k for every segment k of view v (k = 0: identity pose), and the
// camera centre in the segment's frame, computed in FP64 once per call; the
// block's threads stride over the segments.
__device__ __forceinline__ void compose_view(const ViewSet& vs, int v,
                                             const float4* __restrict__ pose_q,
                                             const float* __restrict__ pose_t, int n_inst,
                                             InstMat* __restrict__ out) {
  const int nk = n_inst + 1;
  const float* Vf = vs.v[v].V;
  double V[12];
  for (int i = 0; i < 12; ++i) V[i] = Vf[i];
  for (int k = threadIdx.x; k < nk; k += blockDim.x) {
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t[3] = {0, 0, 0};
    if (k > 0) {
      const float4 qf = pose_q[k - 1];
      double w = qf.x, x = qf.y, y = qf.z, z = qf.w;
      const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
      w *= inv; x *= inv; y *= inv; z *= inv;
      R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
      R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
      R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
      for (int r = 0; r < 3; ++r) t[r] = pose_t[3 * (k - 1) + r];
    }
    double A[9], b[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c)
        A[3 * r + c] = V[4 * r] * R[c] + V[4 * r + 1] * R[3 + c] + V[4 * r + 2] * R[6 + c];
      b[r] = V[4 * r] * t[0] + V[4 * r + 1] * t[1] + V[4 * r + 2] * t[2] + V[4 * r + 3];
    }
    // c = -A^{-1} b by cofactors
    const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8],
                 c02 = A[3] * A[7] - A[4] * A[6];
    const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    const double Ai[9] = {c00 / det, (A[2] * A[7] - A[1] * A[8]) / det, (A[1] * A[5] - A[2] * A[4]) / det,
                          c01 / det, (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                          c02 / det, (A[1] * A[6] - A[0] * A[7]) / det, (A[0] * A[4] - A[1] * A[3]) / det};
    InstMat m;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) m.m[4 * r + c] = (float)A[3 * r + c];
      m.m[4 * r + 3] = (float)b[r];
      const double cr = -(Ai[3 * r] * b[0] + Ai[3 * r + 1] * b[1] + Ai[3 * r + 2] * b[2]);
      m.c[r] = (float)cr;
      m.c_lo[r] = (float)(cr - (double)m.c[r]);
    }
    double f2 = 0.0;
    for (int i = 0; i < 9; ++i) f2 += A[i] * A[i];
    m.a_frob2 = (float)(f2 * (1.0 + 1e-6));
    m.pad = 0.f;
    out[v * nk + k] = m;
  }
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

// The first launch of a call sequence also does the call's set-up, so that
// it needs no launch of its own: its first CTAs compose the instance
// matrices of the views (for the projection that follows), and the last CTA
// to finish zeroes the per-call counters, histograms and tile-class counts,
// bumps the call counter (epoch) and resets the compaction's tile counter.
// The compaction's look-back words carry the tag of the new epoch, read by
// every CTA before the last one finishes.
struct CallSetup {
  int n_views;                       // 0: no matrices to compose
  const float4* pose_q;
  const float* pose_t;
  int n_inst;
  InstMat* mats;
  uint32_t* hist;                    // null: no histograms
  uint32_t* tile_class_cnt;          // null: no tile classes
  int64_t lookback_words;
};

__device__ void call_setup_last(uint32_t* ctr, unsigned long long* lookback, const CallSetup& c,
                                int64_t n_tiles) {
  if (c.hist)
    for (int i = threadIdx.x; i < kHistCount * kRadix; i += blockDim.x) c.hist[i] = 0;
  if (c.tile_class_cnt && threadIdx.x < kTileClasses) c.tile_class_cnt[threadIdx.x] = 0;
  const uint32_t epoch = ctr[kCtrEpoch] + 1;
  __syncthreads();   // every thread has read the old epoch
  // kept: the status word, the epoch, the selection count just written, the
  // blend pair counts (they describe the last counted render)
  if (threadIdx.x < kCtrCount && threadIdx.x != kCtrStatus && threadIdx.x != kCtrEpoch &&
      threadIdx.x != kCtrSelected && (threadIdx.x < kCtrPairs || threadIdx.x > kCtrEvalBwd + 1))
    ctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    ctr[kCtrEpoch] = epoch;
    if (n_tiles == 0) ctr[kCtrSelected] = 0;
  }
  // look-back tags keep the epoch's low 26 bits: before the call whose tags
  // wrap around, every word is cleared (once per 67,108,864 calls)
  if (((epoch + 1u) & ((1u << 26) - 1u)) == 0u)
    for (int64_t i = threadIdx.x; i < c.lookback_words; i += blockDim.x) lookback[i] = 0ull;
}

// The tiles are dealt out in chunks of `per` consecutive tiles, one chunk per
// claim of the CTA counter. A CTA streams its chunk's windows, keeping the
// ballots (one bit per Gaussian) in shared memory, publishes the chunk's
// count, sums the counts of ALL earlier chunks at once (its 256 threads read
// them in parallel: one round trip, where a walk back over the tiles in
// flight took one dependent round trip per 32 tiles) and then writes its
// indices from the ballots. A chunk only waits for chunks claimed before it,
// whose CTAs are running, so no residency assumption is needed.
//
// sel_bits (may be null): bit i of word i / 32 set iff Gaussian i is
// selected; every word of every tile is written (zeros past n).
__global__ void __launch_bounds__(kThreads, 4) k_compact(const __grid_constant__ ViewSet vs,
                                                      const float* __restrict__ vis, int64_t n,
                                                      float t, int per,
                                                      uint32_t* __restrict__ sel,
                                                      uint32_t* ctr,
                                                      unsigned long long* lookback,
                                                      uint32_t* __restrict__ sel_bits,
                                                      const CallSetup setup) {
  __shared__ uint32_t s_bits[kChunkTiles][kWarps][2 * kRounds];   // ballots of the chunk
  __shared__ uint32_t s_off[kChunkTiles * kWarps];   // per (tile, warp): count -> offset in chunk
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_chunk;
  __shared__ bool s_last;
  for (int v = blockIdx.x; v < setup.n_views; v += gridDim.x)
    compose_view(vs, v, setup.pose_q, setup.pose_t, setup.n_inst, setup.mats);
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const uint32_t tag = stage_tag(ctr[kCtrEpoch] + 1u, kStageCompact);
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  const int64_t n_chunks = (n_tiles + per - 1) / per;
  // the windows of a tile: lane reads Gaussians 2 (32 r + lane) + {0, 1} of
  // its warp's span, round r (one float4 per round)
  auto load = [&](int64_t tile, float4 (&w)[kRounds]) {
    const int64_t g0 = tile * kTileSpan + (int64_t)warp * kWarpSpan;
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t g = g0 + 2 * (r * 32 + (int64_t)lane);
      w[r] = make_float4(1.f, -1.f, 1.f, -1.f);  // empty windows
      if (g + 1 < n) {
        w[r] = __ldcs(reinterpret_cast<const float4*>(vis + 2 * g));
      } else if (g < n) {
        const float2 h = __ldcs(reinterpret_cast<const float2*>(vis + 2 * g));
        w[r].x = h.x;
        w[r].y = h.y;
      }
    }
  };
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(ctr + kCtrTileBase + kStageCompact, 1u);
    __syncthreads();
    const int64_t chunk = s_chunk;
    if (chunk >= n_chunks) break;
    const int64_t t0 = chunk * per;
    const int nt = (int)min((int64_t)per, n_tiles - t0);
    // 1. ballots of the chunk's tiles (the next tile's loads issued first)
    float4 w[kRounds];
    load(t0, w);
    for (int i = 0; i < nt; ++i) {
      uint32_t b[2 * kRounds];
      uint32_t count = 0;
#pragma unroll
      for (int r = 0; r < kRounds; ++r) {
        b[r] = __ballot_sync(0xffffffffu, (w[r].x <= t) && (t <= w[r].y));
        b[kRounds + r] = __ballot_sync(0xffffffffu, (w[r].z <= t) && (t <= w[r].w));
        count += __popc(b[r]) + __popc(b[kRounds + r]);
      }
      if (i + 1 < nt) load(t0 + i + 1, w);
      // lane m < 16 keeps ballot m (rounds' even Gaussians, then odd ones)
      uint32_t mine = 0;
#pragma unroll
      for (int m = 0; m < 2 * kRounds; ++m)
        if ((int)lane == m) mine = b[m];
      if (lane < 2 * kRounds) s_bits[i][warp][lane] = mine;
      if (sel_bits && lane < 2 * kRounds) {
        // round r covers Gaussians g0 + 64 r .. + 63: two words, lanes 2r and 2r + 1
        const int r = (int)(lane >> 1);
        uint32_t e = 0, o = 0;
#pragma unroll
        for (int q = 0; q < kRounds; ++q)
          if (r == q) { e = b[q]; o = b[kRounds + q]; }
        const uint32_t sh = (lane & 1u) * 16u;
        const int64_t g0 = (t0 + i) * kTileSpan + (int64_t)warp * kWarpSpan;
        sel_bits[(g0 >> 5) + lane] = interleave16(e >> sh, o >> sh);
      }
      if (lane == 0) s_off[i * kWarps + warp] = count;
    }
    __syncthreads();
    // 2. offsets of the (tile, warp) spans within the chunk: one entry per
    //    thread (per * kWarps <= kThreads)
    const uint32_t c = threadIdx.x < nt * kWarps ? s_off[threadIdx.x] : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      const uint32_t y = s_tmp[q];
      if (q < warp) wbase += y;
      total += y;
    }
    if (threadIdx.x < nt * kWarps) s_off[threadIdx.x] = wbase + incl - c;
    // 3. publish the chunk's count and sum every earlier chunk's count
    if (threadIdx.x == 0) lookback_publish(lookback, 1, chunk, tag, 1u, total);
    const uint32_t prefix = chunk_prefix<kWarps>(lookback, chunk, tag, ctr, s_tmp);
    if (threadIdx.x == 0 && chunk == n_chunks - 1) ctr[kCtrSelected] = prefix + total;
    // 4. the chunk's indices, in order, from the ballots
    const uint32_t lt = lanemask_lt();
    for (int i = 0; i < nt; ++i) {
      const int64_t g0 = (t0 + i) * kTileSpan + (int64_t)warp * kWarpSpan;
      uint32_t out = prefix + s_off[i * kWarps + warp];
#pragma unroll
      for (int r = 0; r < kRounds; ++r) {
        const uint32_t b0 = s_bits[i][warp][r], b1 = s_bits[i][warp][kRounds + r];
        const int64_t g = g0 + 2 * (r * 32 + (int64_t)lane);
        const uint32_t before = __popc(b0 & lt) + __popc(b1 & lt);
        const bool f0 = (b0 >> lane) & 1u;
        const bool f1 = (b1 >> lane) & 1u;
        if (f0) sel[out + before] = (uint32_t)g;
        if (f1) sel[out + before + (f0 ? 1u : 0u)] = (uint32_t)(g + 1);
        out += __popc(b0) + __popc(b1);
      }
    }
    __syncthreads();   // s_chunk / s_bits / s_off reuse
  }
  // the last CTA to finish does the call's set-up for the launches after it
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ctr + kCtrCompactExits, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    call_setup_last(ctr, lookback, setup, n_tiles);
    if (threadIdx.x == 0) ctr[kCtrCompactExits] = 0u;
  }
}

// Chunk length and grid for n Gaussians on `sms` SMs: one chunk per resident
// CTA where a chunk of at most kChunkTiles tiles allows it, else as many
// chunks of kChunkTiles tiles as needed (the CTAs then take several).
struct CompactGrid {
  int per;
  unsigned grid;
};
CompactGrid compact_grid(int64_t n, int sms) {
  // occupancy is queried once (outside any graph capture: the first call)
  static int per_sm = 0;
  if (!per_sm) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_compact, kThreads, 0) != cudaSuccess ||
        b < 1)
      b = 1;
    per_sm = b;
  }
  const int64_t n_tiles = (n + kTileSpan - 1) / kTileSpan;
  const int64_t resident = scan_ctas((int64_t)(sms > 0 ? sms : 1) * per_sm);
  int64_t per = (n_tiles + resident - 1) / resident;
  per = per < 1 ? 1 : (per > kChunkTiles ? kChunkTiles : per);
  const int64_t n_chunks = (n_tiles + per - 1) / per;
  int64_t grid = n_chunks < resident ? n_chunks : resident;
  if (grid < 1) grid = 1;
  return {(int)per, (unsigned)grid};
}

}  // namespace

cudaError_t launch_compact(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                           const float* vis, float t, cudaStream_t st) {
  const int64_t n = sc->n;
  const CompactGrid cg = compact_grid(n, ws->num_sms);
  CallSetup c;
  c.n_views = ws->n_views;
  c.pose_q = reinterpret_cast<const float4*>(poses ? poses->quat : nullptr);
  c.pose_t = poses ? poses->trans : nullptr;
  c.n_inst = sc->n_inst;
  c.mats = reinterpret_cast<InstMat*>(ws->mats);
  c.hist = ws->hist;
  c.tile_class_cnt = ws->tile_class_cnt;
  c.lookback_words = ws->lookback_words;
  KernelTimer timer(ws, kKCompact, st);
  k_compact<<<cg.grid, kThreads, 0, st>>>(ws->views, vis, n, t, cg.per, ws->selected, ws->ctr,
                                          ws->lookback, ws->kept_bits, c);
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
const ViewSet g_no_views = {};   // the selection composes no matrices
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
    const CompactGrid cg = compact_grid(n, sms);
    CallSetup none = {0, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0};
    k_compact<<<cg.grid, kThreads, 0, s>>>(g_no_views, vis_window, n, t, cg.per, out_idx, sc->ctr,
                                            sc->lookback, nullptr, none);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_static_finish<<<1, 1, 0, s>>>(sc->ctr, out_count);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_last_error(S3R_ERR_CUDA, cudaGetErrorString(e));
  return S3R_OK;
}
