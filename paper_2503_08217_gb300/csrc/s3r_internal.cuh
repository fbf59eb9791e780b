// Internal declarations shared by the CUDA translation units of libs3r.
// Not part of the public ABI (that is include/s3r.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "s3r.h"

namespace s3r {

constexpr int kTile = S3R_TILE;            // 16x16 pixel tiles
constexpr int kTilePixels = kTile * kTile;

// ---- device counters (uint32 slots of ws->ctr) -----------------------------
enum Ctr : int {
  kCtrSelected = 0,   // Gaussians whose window contains t
  kCtrSplats = 1,     // kept (Gaussian, view) pairs (may exceed capacity)
  kCtrDups = 2,       // (tile, splat) pairs (may exceed capacity)
  kCtrStatus = 3,     // latched error bits
  kCtrEpoch = 4,      // bumped once per s3r_project; tags look-back words
  kCtrFrustum = 5,    // selected Gaussians inside >= 1 frustum
  kCtrKept = 6,       // selected Gaussians kept in >= 1 view (length of kept_list)
  kCtrTileBase = 8,   // 16 dynamic tile-acquisition counters, one per stage
  kCtrPairs = 24,     // 64-bit: (pixel, splat) list pairs the forward walked (counting mode)
  kCtrEvalFwd = 26,   // 64-bit: (pixel, splat) pairs the forward evaluated (counting mode)
  kCtrEvalBwd = 28,   // 64-bit: (pixel, splat) pairs the backward evaluated (counting mode)
  kCtrRows = 30,      // 64-bit: row-table entries requested by the tile counts of the sort
  kCtrBlendFwdCursor = 32,   // persistent blend queues: next tile, and CTAs that left
  kCtrBlendFwdExits = 33,
  kCtrBlendBwdCursor = 34,
  kCtrBlendBwdExits = 35,
  kCtrProjBwdExits = 36,     // CTAs of the projection backward that finished
  kCtrCompactExits = 38,     // CTAs of the compaction that finished
  kCtrCount = 40
};
// Tile classes of the blend queue: class c = clz(pairs) holds the tiles with
// [2^(31-c), 2^(32-c)) pairs (class 0 the longest lists), class 32 the empty.
constexpr int kTileClasses = 33;
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Look-back stages (each has its own tile counter and status tag).
enum Stage : int {
  kStageCompact = 0,
  kStageProject = 1,
  kStageDup = 2,
  kStageDepth0 = 3,   // 3..6: depth radix passes
  kStageTile0 = 7,    // 7..10: tile radix passes
  kStageProjectBwd = 11,
  kStageExpand = 12,  // chunk counter of the duplication expansion
  kStageCount = 13
};
// Look-back tag stage of the bounded-wait test hook (k_probe.cu): no pass
// uses it, so no word the hook writes can ever match a pass's tag.
constexpr int kStageProbe = 15;
static_assert(kStageCount <= kStageProbe && kStageProbe < 16, "stage tags carry 4 bits");

// Bounded spin: after this many polls a wait gives up, latches
// kStatusTimeout and carries on (results are then invalid, nothing hangs).
constexpr int kSpinLimit = 1 << 22;

// ---- per-call camera set, passed by value in kernel parameters -------------
struct ViewInfo {
  int32_t width, height, gx, gy;
  int32_t tile_base, pix_base;
  float fx, fy, cx, cy, near_z, limx, limy;
  float jc;                   // fx^2 (1 + limx^2) + fy^2 (1 + limy^2): bounds |J|_F^2 z^2
  float V[12];
};

struct ViewSet {
  int32_t n_views;
  int32_t total_tiles;
  int32_t total_pixels;
  int32_t pad;
  ViewInfo v[S3R_MAX_VIEWS];
};

// ---- packed splat record ----------------------------------------------------
// A splat's position, conic, opacity and tile extent in one 32-byte record,
// written by the splat writer: (u, v, conic a, conic b), (conic c, opacity,
// x0 | y0 << 16, w | h << 13 | view << 26 | moved << 31), with w, h the
// rectangle's tile extent. The tile-count kernel, which visits the splats in
// depth order, and the blend's staging, which visits them in each tile's
// order, gather one sector per splat for all of it. Views whose tile grid is wider or higher than S3R_TIN_MAX_GRID
// (8190, the most the 13-bit fields hold without ever giving the all-ones
// word) do not fit that last word; it is then all ones and the kernel reads
// the separate arrays. A build with S3R_TIN_MAX_GRID 0 takes that path for
// every view (a variant the parity tests run).
#ifndef S3R_TIN_MAX_GRID
#define S3R_TIN_MAX_GRID 8190
#endif
static_assert(S3R_TIN_MAX_GRID >= 0 && S3R_TIN_MAX_GRID <= 8190, "13-bit tile extents");
constexpr uint32_t kTinFallback = 0xffffffffu;
constexpr int kTinMaxGrid = S3R_TIN_MAX_GRID;

// ---- chunked scans ----------------------------------------------------------
// S3R_SCAN_CTAS: at most this many CTAs run the chunked scans (compaction,
// splat offsets, pair offsets); 0, the default, means every resident CTA. A
// small value makes every chunk span many tiles and every CTA take several
// chunks, a launch shape the parity tests also run.
#ifndef S3R_SCAN_CTAS
#define S3R_SCAN_CTAS 0
#endif
static_assert(S3R_SCAN_CTAS >= 0, "a CTA cap, or 0 for none");
inline int64_t scan_ctas(int64_t resident) {
  return (S3R_SCAN_CTAS > 0 && resident > S3R_SCAN_CTAS) ? (int64_t)S3R_SCAN_CTAS : resident;
}

// ---- radix sort geometry ----------------------------------------------------
// S3R_SORT_ITEMS (keys per thread per tile) and S3R_SORT_BLOCKS (resident
// onesweep blocks per SM) are build-time defines the autotuner varies; the
// tile's keys and values take 8 * 256 * S3R_SORT_ITEMS bytes of shared memory.
#ifndef S3R_SORT_ITEMS
#define S3R_SORT_ITEMS 15
#endif
#ifndef S3R_SORT_BLOCKS
#define S3R_SORT_BLOCKS 2
#endif
constexpr int kSortThreads = 256;
constexpr int kSortItems = S3R_SORT_ITEMS;
constexpr int kSortTileKeys = kSortThreads * kSortItems;  // 3840 at 15
static_assert(kSortItems >= 1 && kSortItems <= 18,
              "above 18 keys per thread the onesweep tile exceeds 48 KB of static shared memory");
static_assert(S3R_SORT_BLOCKS >= 1 && S3R_SORT_BLOCKS * kSortThreads <= 2048,
              "an SM holds at most 2048 threads");
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
// digit histograms: 4 depth passes + up to 4 tile passes
constexpr int kHistDepth = 0;
constexpr int kHistTile = 4;
constexpr int kHistCount = 8;
constexpr int kDupChunkMin = 1024;   // smallest output chunk of the pair expansion

// Kernel ids for the per-kernel timing hook.
enum KernelId : int {
  kKCompact = 0, kKProject, kKSplatScan, kKProjectSplats, kKDepth0, kKDepth1, kKDepth2, kKDepth3, kKDuplicate,
  kKTile0, kKTile1, kKTile2, kKTile3, kKTileRanges, kKExpand, kKBlendFwd, kKZeroGrads, kKBlendBwd,
  kKProjectBwd, kKSplatTiles, kKCount
};

}  // namespace s3r

// The workspace: every intermediate of one call sequence, allocated once.
struct s3r_workspace {
  int device;
  s3r_capacity cap;
  int num_sms;
  // device buffers
  uint32_t* ctr;            // [kCtrCount]
  uint32_t* hist;           // [kHistCount][256]
  unsigned long long* lookback;  // tagged look-back words
  int64_t lookback_words;
  uint32_t* selected;       // [N]
  uint32_t* frustum_mask;   // [N]
  uint32_t* keep_mask;      // [N]
  uint32_t* splat_start;    // [N]
  uint2* kept_list;         // [N] (compacted index, Gaussian id) of those kept in >= 1 view (any order)
  uint32_t* kept_bits;      // [ceil(N / 4096) * 128] bit per Gaussian id: selected and kept in >= 1 view
  int64_t kept_words;
  float4* sp_rgb_d;         // [S]
  uint2* sp_rect;           // [S]
  uint8_t* sp_view;         // [S]
  uint32_t* sp_tin;         // [S] x 8: position, conic, opacity and tile extent (one 32-byte record)
  uint32_t* depth_key[2];   // [S]
  uint32_t* depth_val[2];   // [S]
  uint32_t* dup_key[2];     // [K]
  uint32_t* dup_val[2];     // [K]
  uint2* ranges;            // [tiles]
  uint32_t* tile_class_cnt; // [64] tiles per class of pair count (kTileClasses used)
  uint32_t* tile_class_list;  // [kTileClasses][max_tiles] tile ids per class
  float* final_T;           // [P]
  uint32_t* n_contrib;      // [P]
  float* sp_grad;           // [S*12] per-splat 2D adjoints summed by the blend backward
  int sp_grad_clean;        // host: the last render_fwd zeroed sp_grad and no backward used it since
  float* pose_dM;           // [views*(inst+1)*12], zero between backward calls
  float* world_acc;         // [(inst+1) * world_acc_floats()] pose sums of s3r_to_world_bwd, zero between calls
  float* mats;              // composed matrices [views*(inst+1)] x 20 floats
  uint32_t* dup_excl;       // [S+1] first pair of each depth-sorted splat
  uint32_t* dup_meta;       // [S] x 8: expansion record of each splat, depth order
  uint32_t* sp_tiles;       // [S] tiles of its rectangle a splat's alpha region reaches, depth order
  float* sp_region;         // [S] x 8: that region, where the row table had no room
  uint32_t* row_spans;      // [rows_cap] column interval of one rectangle row
  int64_t rows_cap;
  uint32_t* dup_chunk;      // [K/kDupChunkMin + 2] sorted splat holding the first pair of each expansion chunk
  uint32_t* contrib;        // [4][K/32 + 2] bit per (warp block, sorted pair): blended in the forward
  int64_t contrib_words;    // words per warp block
  int64_t bytes;
  // host-side state of the current call sequence
  s3r::ViewSet views;
  int n_views;
  int n_inst;
  int sh_degree;
  int64_t n;
  int stage_done;           // 0 none, 1 projected, 2 sorted, 3 rendered
  int depth_final;          // which buffer holds the depth-sorted splats
  int dup_final;            // which buffer holds the tile-sorted pairs
  int tile_passes;
  s3r_lod_params lod;       // mode S3R_LOD_THRESHOLD unless s3r_set_lod said otherwise
  int counting;             // blend kernels count their pairs (s3r_set_counting)
  int grad_mode;            // S3R_GRAD_ACCUMULATE or S3R_GRAD_OVERWRITE (s3r_set_grad_mode)
  // per-kernel timing hook
  int timing;
  cudaEvent_t ev[2 * s3r::kKCount];
  int ev_used[s3r::kKCount];
};

namespace s3r {
// Records a CUDA event before a kernel launch and another after it when the
// workspace's timing hook is on. The events are recorded as external events,
// so under stream capture they become event-record nodes of the graph and
// time every replay.
struct KernelTimer {
  s3r_workspace* ws;
  int id;
  cudaStream_t st;
  unsigned flags = 0;
  KernelTimer(s3r_workspace* w, int kid, cudaStream_t s) : ws(w), id(kid), st(s) {
    if (!ws->timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags(ws->ev[2 * id], st, flags);
  }
  ~KernelTimer() {
    if (ws->timing) {
      cudaEventRecordWithFlags(ws->ev[2 * id + 1], st, flags);
      ws->ev_used[id] = 1;
    }
  }
};
}  // namespace s3r

namespace s3r {

// ---- launchers (one translation unit each) ---------------------------------
cudaError_t launch_compact(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                           const float* vis, float t, cudaStream_t st);
cudaError_t launch_project(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                           float t, float* life, float lod, cudaStream_t st);
cudaError_t launch_sort(s3r_workspace* ws, cudaStream_t st);
cudaError_t launch_to_world(const s3r_scene* sc, const s3r_poses* poses, float* means_out,
                            float* quats_out, float* sh_out, int64_t n_dynamic, int num_sms,
                            cudaStream_t st);
cudaError_t launch_to_world_bwd(const s3r_scene* sc, const s3r_poses* poses, const s3r_grads* g,
                                float* acc, int64_t n_dynamic, int num_sms, cudaStream_t st);
int world_acc_floats();
cudaError_t launch_render_fwd(s3r_workspace* ws, const float* bg, float* out, cudaStream_t st);
cudaError_t launch_render_bwd(s3r_workspace* ws, const float* bg, const float* dL,
                              const s3r_grads* grads, cudaStream_t st);
cudaError_t launch_project_bwd(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                               const s3r_grads* g, cudaStream_t st);
cudaError_t launch_adam(const s3r_adam_tensor* t, int count, float lr, float b1, float b2,
                        float eps, float bc1, float bc2, const uint32_t* gate, cudaStream_t st);
// SM count of the current device (queried once per device, then cached).
int sm_count();
// Zero `words` 32-bit words at a 16-byte aligned device address with a
// kernel (no copy-engine memset: a captured step then overlaps host-to-device
// copies on another stream).
cudaError_t launch_zero(void* p, int64_t words, cudaStream_t st);
cudaError_t launch_l1_loss(int64_t n, const float* pred, const float* target, float* grad,
                           float* loss, cudaStream_t st);
cudaError_t launch_visibility(int64_t n, float t, const uint32_t* mask, float* life, float* vis,
                              int mode, cudaStream_t st);
cudaError_t launch_wait_probe(s3r_workspace* ws, int max_polls, cudaStream_t st);
int64_t ode_param_count(int embed_dim);
cudaError_t launch_ode_fwd(const s3r_ode_net* net, int n_inst, const float* z0, const float* times,
                           int n_times, int substeps, float* states, float* quat, float* trans,
                           cudaStream_t st);
cudaError_t launch_ode_bwd(const s3r_ode_net* net, int n_inst, const float* times, int n_times,
                           int substeps, const float* states, const float* g_quat,
                           const float* g_trans, float* g_params, float* g_embed, float* g_z0,
                           cudaStream_t st);
// Record `msg` as the calling thread's last error and return `st`.
s3r_status set_last_error(s3r_status st, const char* msg);

// ---- small device helpers ----------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tagged look-back word: [tag:30][flag:2][value:32]. flag 1 = this tile's
// aggregate only, 2 = inclusive prefix through this tile.
__device__ __forceinline__ unsigned long long lb_word(uint32_t tag, uint32_t flag, uint32_t v) {
  return ((unsigned long long)tag << 34) | ((unsigned long long)flag << 32) | v;
}
__device__ __forceinline__ uint32_t stage_tag(uint32_t epoch, int stage) {
  return ((epoch << 4) | (uint32_t)stage) & 0x3fffffffu;
}

// Decoupled look-back over tiles for one running sum (one digit): `words`
// points at the sum's word of tile 0, consecutive tiles `stride` words apart.
// A tile first publishes its own aggregate (flag 1, lookback_publish), then
// walks back over its predecessors, adding aggregates until it meets an
// inclusive prefix (flag 2), and publishes its own inclusive prefix. The walk
// reads kLookbackBatch predecessors per round trip (independent loads), so a
// chain of w unfinished predecessors costs about w / kLookbackBatch dependent
// loads. Bounded: after max_polls rounds without progress it latches
// kStatusTimeout into ctr and returns the partial sum.
constexpr int kLookbackBatch = 8;

__device__ __forceinline__ void lookback_publish(unsigned long long* words, int64_t stride,
                                                 int64_t tile, uint32_t tag, uint32_t flag,
                                                 uint32_t value) {
  st_relaxed(words + tile * stride, lb_word(tag, flag, value));
}

template <int kBatch = kLookbackBatch>
__device__ __forceinline__ uint32_t lookback_walk(unsigned long long* words, int64_t stride,
                                                  int64_t tile, uint32_t tag, uint32_t* ctr,
                                                  int max_polls = kSpinLimit) {
  uint32_t prefix = 0;
  int64_t k = tile - 1;
  int spins = 0;
  while (k >= 0) {
    unsigned long long w[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      w[j] = k - j >= 0 ? ld_relaxed(words + (k - j) * stride) : lb_word(tag, 2u, 0u);
    uint32_t acc = 0;
    int used = 0;
    bool stop = false, done = false;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const uint32_t flag = (uint32_t)(w[j] >> 34) == tag ? (uint32_t)(w[j] >> 32) & 3u : 0u;
      const bool take = !stop && flag != 0u;
      acc += take ? (uint32_t)w[j] : 0u;
      used += take ? 1 : 0;
      done = done || (take && flag == 2u);
      stop = stop || flag != 1u;
    }
    prefix += acc;
    k -= used;
    if (done) break;
    if (used == 0) {
      if (++spins > max_polls) {
        atomicOr(ctr + kCtrStatus, kStatusTimeout);
        break;
      }
      __nanosleep(20);
    }
  }
  return prefix;
}

// Publish, walk and publish the inclusive value in one call (one thread per
// running sum); returns the exclusive prefix of `tile`.
__device__ __forceinline__ uint32_t lookback_prefix(unsigned long long* words, int64_t stride,
                                                     int64_t tile, uint32_t tag, uint32_t aggregate,
                                                     uint32_t* ctr, int max_polls = kSpinLimit) {
  if (tile == 0) {
    lookback_publish(words, stride, 0, tag, 2u, aggregate);
    return 0;
  }
  lookback_publish(words, stride, tile, tag, 1u, aggregate);
  const uint32_t prefix = lookback_walk(words, stride, tile, tag, ctr, max_polls);
  lookback_publish(words, stride, tile, tag, 2u, prefix + aggregate);
  return prefix;
}

// Saturating sum for running sums that may pass 2^32 (the pair offsets):
// values at or above kSat mean "more than any capacity" and stay there. For
// operands <= kSat the 64-bit sum cannot wrap, and min(a + b, kSat) is
// associative, so any summation order gives min(exact sum, kSat).
constexpr uint32_t kSat = 0x80000000u;
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
  const unsigned long long s = (unsigned long long)a + b;
  return s > kSat ? kSat : (uint32_t)s;
}

// Chunked single-pass scan: once a block has published its chunk's aggregate
// (flag 1, lookback_publish at stride 1), it sums the aggregates of ALL
// earlier chunks, its threads reading them in parallel (one round trip, where
// a walk back over the chunks in flight takes one per batch of
// predecessors). Chunks are claimed in order from a counter, so a chunk only
// waits for chunks whose blocks are running. Every thread of the block calls
// it (it synchronises twice); returns the exclusive prefix in every thread.
// s_red: kWarpsB words. Bounded like lookback_walk. kSaturate: sat_add sums.
template <int kWarpsB, bool kSaturate = false>
__device__ __forceinline__ uint32_t chunk_prefix(const unsigned long long* words, int64_t chunk,
                                                 uint32_t tag, uint32_t* ctr, uint32_t* s_red,
                                                 int max_polls = kSpinLimit) {
  auto add = [](uint32_t a, uint32_t b) { return kSaturate ? sat_add(a, b) : a + b; };
  uint32_t part = 0;
  for (int64_t k = threadIdx.x; k < chunk; k += kWarpsB * 32) {
    unsigned long long x = ld_relaxed(words + k);
    int spins = 0;
    while ((uint32_t)(x >> 34) != tag) {
      if (++spins > max_polls) {
        atomicOr(ctr + kCtrStatus, kStatusTimeout);
        x = 0;
        break;
      }
      __nanosleep(32);
      x = ld_relaxed(words + k);
    }
    part = add(part, (uint32_t)x);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part = add(part, __shfl_xor_sync(0xffffffffu, part, o));
  __syncthreads();   // s_red may still be read by the caller's previous step
  if ((threadIdx.x & 31u) == 0) s_red[threadIdx.x >> 5] = part;
  __syncthreads();
  uint32_t prefix = 0;
#pragma unroll
  for (int w = 0; w < kWarpsB; ++w) prefix = add(prefix, s_red[w]);
  return prefix;
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Hardware approximations (about 1 ulp); deterministic, so two kernels that
// evaluate the same expression with them get the same bits.
__device__ __forceinline__ float approx_sqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float approx_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ------------------------------------------------------- alpha-region bounds
// The blend keeps a (pixel, splat) pair iff alpha = min(0.99, o G) >= 1/255
// with G = exp(-q / 2), q = A dx^2 + 2 B dx dy + C dy^2 (the conic), i.e. iff q
// <= 2 ln(255 o) up to the FP32 rounding of the per-pixel evaluation. Its
// error grows with the conic's eigenvalue ratio (cancellation between the
// terms along a thin splat): about 2^-24 L ratio in units of q. Below a ratio
// of kMaxConicRatio that is under 0.02, far inside the margins of the cull
// tests; above it the tests give up and keep everything.
constexpr float kMaxConicRatio = 3e4f;

// det(conic) lowered by a bound on the rounding of A C - B^2 (so that the
// ellipse built from it contains the exact one); -1 where the splat is too
// anisotropic for the cull tests, or the conic is not positive definite.
__device__ __forceinline__ float conic_det_lower(float A, float B, float C) {
  const float bb = __fmul_rn(B, B);
  const float det = __fmaf_rn(A, C, -bb);
  const float lo = __fsub_rn(__fmul_rn(det, 1.f - 0x1p-20f), __fmul_rn(bb, 0x1p-20f));
  const float tr = __fadd_rn(A, C);
  const bool ok = (A > 0.f) & (C > 0.f) & (lo > 0.f) & (__fmul_rn(tr, tr) <= __fmul_rn(kMaxConicRatio, lo));
  return ok ? lo : -1.f;
}
#endif

}  // namespace s3r
