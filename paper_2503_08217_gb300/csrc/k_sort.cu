// Tile|depth key duplication and the radix sort that orders every tile's
// splats front to back (the rasteriser of Eq. 2), then per-tile ranges.
//
// The sorted order is the one of a stable LSD radix sort on the 64-bit key
// (view-tile id << 32 | FP32 depth bits) over the duplicated pairs in
// projection order. Duplicates of one splat share its depth, so the four
// depth-digit passes run on the splats BEFORE duplication (S keys instead of
// K); the splats are then expanded into (tile, splat) pairs in depth order,
// and the one or two tile-digit passes finish the sort. Every pass is a
// single-pass "onesweep" kernel: persistent CTAs take 3840-key tiles from an
// atomic counter, rank digits with warp match.any, get each digit's global
// offset from a precomputed histogram plus a decoupled look-back over tiles,
// reorder the tile in shared memory and write it out coalesced.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kWarpKeys = kSortItems * 32;   // 480 keys per warp per tile

struct PassArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;   // null: values are the input positions
  uint32_t* keys_out;
  uint32_t* vals_out;
  const uint32_t* count;     // device count of keys
  int64_t cap;
  int shift;
  const uint32_t* hist;      // [256] global digit histogram of this pass
  uint32_t* ctr;
  unsigned long long* lookback;
  int stage;
};

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_tmp /*[8]*/,
                                                    uint32_t* total) {
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_tmp[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_tmp[w];
    if (w < warp) wbase += c;
    tot += c;
  }
  __syncthreads();
  if (total) *total = tot;
  return wbase + incl - x;
}

__global__ void __launch_bounds__(kSortThreads) k_onesweep(PassArgs a) {
  __shared__ uint32_t s_keys[kSortTileKeys];
  __shared__ uint32_t s_vals[kSortTileKeys];
  __shared__ uint32_t s_cnt[kWarps][kRadix];   // per-warp digit counts -> exclusive offsets
  __shared__ uint32_t s_gbase[kRadix];         // exclusive scan of the global histogram
  __shared__ uint32_t s_dst[kRadix];           // global start of each digit for this tile
  __shared__ uint32_t s_loc[kRadix];           // tile-local start of each digit
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_tile;

  const int64_t n = min((int64_t)*a.count, a.cap);
  const int64_t n_tiles = (n + kSortTileKeys - 1) / kSortTileKeys;
  const uint32_t tag = stage_tag(a.ctr[kCtrEpoch], a.stage);
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  const int d_me = threadIdx.x;   // the digit this thread scans / looks back on

  s_gbase[d_me] = block_excl_scan(a.hist[d_me], s_tmp, nullptr);

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr + kCtrTileBase + a.stage, 1u);
    for (int i = lane; i < kRadix; i += 32) s_cnt[warp][i] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;
    const int64_t base = tile * kSortTileKeys + (int64_t)warp * kWarpKeys;

    uint32_t key[kSortItems], val[kSortItems];
    uint32_t rank[kSortItems];
    // all loads first, so that each thread has 2 x 15 requests in flight
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      const bool valid = idx < n;
      key[r] = valid ? __ldcs(a.keys_in + idx) : 0xffffffffu;
      val[r] = valid ? (a.vals_in ? __ldcs(a.vals_in + idx) : (uint32_t)idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      const bool valid = idx < n;
      const uint32_t d = (key[r] >> a.shift) & (kRadix - 1);
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : kRadix);
      uint32_t before = 0;
      if (valid) before = s_cnt[warp][d];
      rank[r] = before + __popc(peers & lt);
      __syncwarp();
      if (valid && (peers & lt) == 0) s_cnt[warp][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();

    // per digit: exclusive offsets over warps, tile count, look-back
    uint32_t tile_cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_cnt[w][d_me];
      s_cnt[w][d_me] = tile_cnt;
      tile_cnt += c;
    }
    const uint32_t prefix =
        lookback_prefix(a.lookback + d_me, kRadix, tile, tag, tile_cnt, a.ctr);
    s_dst[d_me] = s_gbase[d_me] + prefix;
    s_loc[d_me] = block_excl_scan(tile_cnt, s_tmp, nullptr);
    __syncthreads();

    // reorder in shared memory by digit (stable)
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      if (idx < n) {
        const uint32_t d = (key[r] >> a.shift) & (kRadix - 1);
        const uint32_t pos = s_loc[d] + s_cnt[warp][d] + rank[r];
        s_keys[pos] = key[r];
        s_vals[pos] = val[r];
      }
    }
    __syncthreads();
    const int64_t tile_n = min((int64_t)kSortTileKeys, n - tile * kSortTileKeys);
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
      const uint32_t k = s_keys[i];
      const uint32_t d = (k >> a.shift) & (kRadix - 1);
      const uint32_t dst = s_dst[d] + (uint32_t)i - s_loc[d];
      __stcs(a.keys_out + dst, k);
      __stcs(a.vals_out + dst, s_vals[i]);
    }
    __syncthreads();
  }
}

// Expand depth-sorted splats into (view-tile id, splat) pairs, in two kernels
// so that the work is balanced by OUTPUT count: the nearest splats come first
// in depth order and may each cover hundreds of tiles.
//  k_dup_scan:   per sorted splat, its tile count and a compact descriptor
//                (splat id, first tile id, grid width | rect width << 16,
//                1/width); a block scan + decoupled look-back over 1024-splat
//                tiles gives every splat its first output position.
//  k_dup_expand: persistent CTAs take fixed chunks of 4096 outputs; a warp
//                finds the chunk's first splat by a 32-ary search of the
//                offsets, each thread expands 16 consecutive outputs (binary
//                search in shared memory, then an incremental cursor), the
//                pairs are staged in shared memory and written coalesced. The
//                tile id of output r of a splat of rectangle width w is
//                first + (r / w) * gx + r % w, r / w from a float reciprocal
//                with one integer correction step.
constexpr int kDupThreads = 256;
constexpr int kDupPer = 4;                            // splats per thread in the scan
constexpr int kDupSplats = kDupThreads * kDupPer;     // 1024 per scan tile
constexpr int kExpItems = 16;                         // outputs per thread per chunk
constexpr int kExpChunk = kDupThreads * kExpItems;    // 4096 outputs per chunk

struct DupArgs {
  const uint32_t* sorted_splats;
  const uint2* sp_rect;
  const uint8_t* sp_view;
  uint32_t* dup_key;
  uint32_t* dup_val;
  uint32_t* dup_excl;    // [S+1] first output of each sorted splat
  uint4* dup_meta;       // [S] descriptors
  int64_t cap_splats, cap_dups;
  uint32_t* ctr;
  unsigned long long* lookback;
};

__global__ void __launch_bounds__(kDupThreads) k_dup_scan(const __grid_constant__ ViewSet vs,
                                                          DupArgs a) {
  __shared__ uint32_t s_tmp[8];
  __shared__ uint32_t s_tile, s_base;
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap_splats);
  const int64_t n_tiles = (n + kDupSplats - 1) / kDupSplats;
  const uint32_t tag = stage_tag(a.ctr[kCtrEpoch], kStageDup);
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr + kCtrTileBase + kStageDup, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;
    const int64_t i0 = tile * kDupSplats + (int64_t)threadIdx.x * kDupPer;
    uint32_t sp[kDupPer], cnt[kDupPer], run = 0;
#pragma unroll
    for (int k = 0; k < kDupPer; ++k) sp[k] = i0 + k < n ? a.sorted_splats[i0 + k] : 0u;
    uint2 rect[kDupPer];
    int view[kDupPer];
#pragma unroll
    for (int k = 0; k < kDupPer; ++k) {
      rect[k] = i0 + k < n ? a.sp_rect[sp[k]] : make_uint2(0u, 0u);
      view[k] = i0 + k < n ? a.sp_view[sp[k]] : 0;
    }
#pragma unroll
    for (int k = 0; k < kDupPer; ++k) {
      const uint32_t x0 = rect[k].x & 0xffffu, y0 = rect[k].x >> 16;
      const uint32_t w = (rect[k].y & 0xffffu) - x0, h = (rect[k].y >> 16) - y0;
      cnt[k] = w * h;
      run += cnt[k];
      if (i0 + k < n) {
        const ViewInfo& vi = vs.v[view[k]];
        const uint32_t first = (uint32_t)vi.tile_base + y0 * (uint32_t)vi.gx + x0;
        a.dup_meta[i0 + k] = make_uint4(sp[k], first, (uint32_t)vi.gx | (w << 16),
                                        __float_as_uint(w ? 1.f / (float)w : 1.f));
      }
    }
    uint32_t total;
    uint32_t ex = block_excl_scan(run, s_tmp, &total);
    if (threadIdx.x < 32) {
      const uint32_t prefix = warp_lookback(a.lookback, tile, tag, total, a.ctr);
      if (threadIdx.x == 0) {
        s_base = prefix;
        if (tile == n_tiles - 1) {
          a.ctr[kCtrDups] = prefix + total;
          a.dup_excl[n] = prefix + total;              // sentinel
          if ((int64_t)prefix + total > a.cap_dups) atomicOr(a.ctr + kCtrStatus, kStatusCapacity);
        }
      }
    }
    __syncthreads();
    ex += s_base;
#pragma unroll
    for (int k = 0; k < kDupPer; ++k) {
      if (i0 + k < n) a.dup_excl[i0 + k] = ex;
      ex += cnt[k];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kDupThreads) k_dup_expand(DupArgs a) {
  __shared__ uint32_t s_excl[kExpChunk + 1];
  __shared__ uint32_t s_key[kExpChunk];
  __shared__ uint32_t s_val[kExpChunk];
  __shared__ uint32_t s_chunk, s_q0, s_q1;
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap_splats);
  const int64_t total = min((int64_t)a.ctr[kCtrDups], a.cap_dups);
  const int64_t n_chunks = (total + kExpChunk - 1) / kExpChunk;
  const uint32_t lane = lane_id();
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(a.ctr + kCtrTileBase + kStageExpand, 1u);
    __syncthreads();
    const int64_t chunk = s_chunk;
    if (chunk >= n_chunks) break;
    const uint32_t O0 = (uint32_t)(chunk * kExpChunk);
    const uint32_t O1 = (uint32_t)min((int64_t)O0 + kExpChunk, total);   // exclusive
    if (threadIdx.x < 32) {
      // last q with excl[q] <= O0, and last q with excl[q] <= O1 - 1: 32-ary search
      for (int which = 0; which < 2; ++which) {
        const uint32_t target = which ? O1 - 1 : O0;
        int64_t lo = 0, hi = n;          // excl[lo] <= target < excl[hi] (excl[n] = total)
        while (hi - lo > 1) {
          const int64_t step = (hi - lo + 31) / 32;
          const int64_t probe = lo + (int64_t)(lane + 1) * step;
          const bool le = probe < hi && a.dup_excl[probe] <= target;
          const uint32_t m = __ballot_sync(0xffffffffu, le);
          const int c = __popc(m);                      // probes that are <= target (a prefix)
          const int64_t nlo = lo + (int64_t)c * step;
          const int64_t nhi = min(hi, lo + (int64_t)(c + 1) * step);
          lo = nlo;
          hi = nhi;
        }
        if (lane == 0) (which ? s_q1 : s_q0) = (uint32_t)lo;
      }
    }
    __syncthreads();
    const int q0 = (int)s_q0, nq = (int)s_q1 - q0 + 1;
    for (int i = threadIdx.x; i <= nq; i += kDupThreads) s_excl[i] = a.dup_excl[q0 + i];
    __syncthreads();
    // 16 consecutive outputs per thread
    const uint32_t o0 = O0 + threadIdx.x * kExpItems;
    if (o0 < O1) {
      int lo = 0, hi = nq;            // last local q with s_excl[q] <= o0
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_excl[mid] <= o0) lo = mid; else hi = mid;
      }
      int q = lo;
      uint32_t q_end = s_excl[q + 1];
      uint4 meta = a.dup_meta[q0 + q];
      const uint32_t oe = min(o0 + kExpItems, O1);
      for (uint32_t o = o0; o < oe; ++o) {
        while (o >= q_end) {
          ++q;
          q_end = s_excl[q + 1];
          meta = a.dup_meta[q0 + q];
        }
        const uint32_t rr = o - s_excl[q];
        const uint32_t w = meta.z >> 16, gx = meta.z & 0xffffu;
        uint32_t row = (uint32_t)(((float)rr + 0.5f) * __uint_as_float(meta.w));
        row -= (row * w > rr) ? 1u : 0u;
        row += ((row + 1u) * w <= rr) ? 1u : 0u;
        s_key[o - O0] = meta.y + row * gx + (rr - row * w);
        s_val[o - O0] = meta.x;
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < O1 - O0; i += kDupThreads) {
      __stcs(a.dup_key + O0 + i, s_key[i]);
      __stcs(a.dup_val + O0 + i, s_val[i]);
    }
    (void)lane;
  }
}

// Per-tile pair counts from the projection's difference array (+1 / -1 at
// the two ends of every covered tile row), their exclusive scan (the [start,
// end) range of every tile in the sorted pair array, clamped to capacity),
// and the digit histograms of the tile-id radix passes. One CTA; three walks
// over the tiles (sum of differences, sum of counts, output).
constexpr int kCountThreads = 1024;

__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t x, uint32_t* s_tmp /*[32]*/) {
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) s_tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = s_tmp[lane];
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (uint32_t)o) wi += y;
    }
    s_tmp[lane] = wi - w;
  }
  __syncthreads();
  const uint32_t r = s_tmp[warp] + incl - x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kCountThreads) k_tile_counts(const int32_t* __restrict__ diff,
                                                               int tiles, int passes, int64_t cap,
                                                               uint2* __restrict__ ranges,
                                                               uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[4][kRadix];
  __shared__ uint32_t s_tmp[32];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  const int per = (tiles + kCountThreads - 1) / kCountThreads;
  const int t0 = min(tiles, (int)threadIdx.x * per), t1 = min(tiles, t0 + per);
  int32_t dsum = 0;
  for (int t = t0; t < t1; ++t) dsum += diff[t];
  const int32_t enter = (int32_t)block_excl_scan_1024((uint32_t)dsum, s_tmp);   // count entering t0
  uint32_t csum = 0;
  int32_t c = enter;
  for (int t = t0; t < t1; ++t) {
    c += diff[t];
    csum += (uint32_t)c;
  }
  uint32_t start = block_excl_scan_1024(csum, s_tmp);
  c = enter;
  for (int t = t0; t < t1; ++t) {
    c += diff[t];
    const uint32_t cnt = (uint32_t)c;
    const uint32_t b = (uint32_t)min((int64_t)start, cap), e = (uint32_t)min((int64_t)start + cnt, cap);
    ranges[t] = cnt ? make_uint2(b, e) : make_uint2(0u, 0u);   // empty tiles: [0, 0)
    start += cnt;
    if (cnt)
      for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][((uint32_t)t >> (8 * p)) & 0xffu], cnt);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) hist[i] = (&s_hist[0][0])[i];
}

int per_sm_for(const void* fn, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

}  // namespace

cudaError_t launch_sort(s3r_workspace* ws, cudaStream_t st) {
  cudaError_t e;
  // occupancy is queried once (outside any graph capture: the first call)
  static thread_local int sweep_per_sm = 0, dup_per_sm = 0, exp_per_sm = 0;
  if (!sweep_per_sm) sweep_per_sm = per_sm_for((const void*)k_onesweep, kSortThreads);
  if (!dup_per_sm) dup_per_sm = per_sm_for((const void*)k_dup_scan, kDupThreads);
  if (!exp_per_sm) exp_per_sm = per_sm_for((const void*)k_dup_expand, kDupThreads);
  const int g_sweep = ws->num_sms * sweep_per_sm;
  // depth digits on the splats: 4 passes, result back in buffer 0
  for (int p = 0; p < 4; ++p) {
    PassArgs a;
    a.keys_in = ws->depth_key[p & 1];
    a.vals_in = p == 0 ? nullptr : ws->depth_val[p & 1];
    a.keys_out = ws->depth_key[(p + 1) & 1];
    a.vals_out = ws->depth_val[(p + 1) & 1];
    a.count = ws->ctr + kCtrSplats;
    a.cap = ws->cap.max_splats;
    a.shift = 8 * p;
    a.hist = ws->hist + (kHistDepth + p) * kRadix;
    a.ctr = ws->ctr;
    a.lookback = ws->lookback;
    a.stage = kStageDepth0 + p;
    KernelTimer timer(ws, kKDepth0 + p, st);
    k_onesweep<<<g_sweep, kSortThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  ws->depth_final = 0;
  // expand into (tile, splat) pairs in depth order
  DupArgs d;
  d.sorted_splats = ws->depth_val[0];
  d.sp_rect = ws->sp_rect;
  d.sp_view = ws->sp_view;
  d.dup_key = ws->dup_key[0];
  d.dup_val = ws->dup_val[0];
  d.dup_excl = ws->dup_excl;
  d.dup_meta = reinterpret_cast<uint4*>(ws->dup_meta);
  d.cap_splats = ws->cap.max_splats;
  d.cap_dups = ws->cap.max_duplicates;
  d.ctr = ws->ctr;
  d.lookback = ws->lookback;
  {
    KernelTimer timer(ws, kKTileCounts, st);
    k_tile_counts<<<1, kCountThreads, 0, st>>>(ws->tile_diff, ws->views.total_tiles, ws->tile_passes,
                                               ws->cap.max_duplicates, ws->ranges,
                                               ws->hist + kHistTile * kRadix);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKDuplicate, st);
    k_dup_scan<<<ws->num_sms * dup_per_sm, kDupThreads, 0, st>>>(ws->views, d);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKExpand, st);
    k_dup_expand<<<ws->num_sms * exp_per_sm, kDupThreads, 0, st>>>(d);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // tile digits on the pairs
  for (int p = 0; p < ws->tile_passes; ++p) {
    PassArgs a;
    a.keys_in = ws->dup_key[p & 1];
    a.vals_in = ws->dup_val[p & 1];
    a.keys_out = ws->dup_key[(p + 1) & 1];
    a.vals_out = ws->dup_val[(p + 1) & 1];
    a.count = ws->ctr + kCtrDups;
    a.cap = ws->cap.max_duplicates;
    a.shift = 8 * p;
    a.hist = ws->hist + (kHistTile + p) * kRadix;
    a.ctr = ws->ctr;
    a.lookback = ws->lookback;
    a.stage = kStageTile0 + p;
    KernelTimer timer(ws, kKTile0 + p, st);
    k_onesweep<<<g_sweep, kSortThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  ws->dup_final = ws->tile_passes & 1;
  return cudaSuccess;
}

}  // namespace s3r
