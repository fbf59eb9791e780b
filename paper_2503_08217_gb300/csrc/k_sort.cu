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
// atomic counter, rank digits with nine warp ballots per key (faster here than
// match.any, which queues on the address-divergence unit), get each digit's global
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

__global__ void __launch_bounds__(kSortThreads, 3) k_onesweep(PassArgs a) {
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
      // peers with the same digit: the AND over the digit's eight bits of the
      // ballot or its complement. Slots past the end hold key 0xffffffff
      // (digit 255) and are counted with it: they are the tile's last slots,
      // so they only follow the valid keys of that digit and are never written
      const uint32_t d = (key[r] >> a.shift) & (kRadix - 1);
      uint32_t peers = 0xffffffffu;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
      }
      const uint32_t before = s_cnt[warp][d];
      rank[r] = before + __popc(peers & lt);
      __syncwarp();
      if ((peers & lt) == 0) s_cnt[warp][d] = before + __popc(peers);
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
  uint32_t* hist;        // tile-digit histograms of the radix passes that follow
  int tile_passes;
  const uint32_t* sorted_splats;
  const uint2* sp_rect;
  const uint8_t* sp_view;
  uint32_t* dup_key;
  uint32_t* dup_val;
  uint32_t* dup_excl;    // [S+1] first output of each sorted splat
  uint4* dup_meta;       // [S] descriptors
  uint32_t* dup_chunk;   // [chunks+1] splat holding each chunk's first output; last: final splat
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
      view[k] = i0 + k < n ? (a.sp_view[sp[k]] & 0x7f) : 0;   // bit 7: Eq. 7 moved
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
      if (i0 + k < n) {
        a.dup_excl[i0 + k] = ex;
        // every chunk boundary inside this splat's outputs [ex, ex + cnt)
        // (below capacity) starts with this splat
        const uint64_t e1 = min((uint64_t)ex + cnt[k], (uint64_t)a.cap_dups);
        for (uint64_t c = ((uint64_t)ex + kExpChunk - 1) / kExpChunk; c * kExpChunk < e1; ++c)
          a.dup_chunk[c] = (uint32_t)(i0 + k);
      }
      ex += cnt[k];
    }
    if (tile == n_tiles - 1 && threadIdx.x == 0) {
      // after the last chunk: the last splat (chunks end at an inclusive splat bound)
      const uint64_t tot = min((uint64_t)s_base + total, (uint64_t)a.cap_dups);
      a.dup_chunk[(tot + kExpChunk - 1) / kExpChunk] = (uint32_t)(n - 1);
    }
    __syncthreads();
  }
}

// Per-thread run-length counting of the radix digits of a key sequence: one
// shared atomic per run of equal digits (consecutive outputs walk a tile
// row, so the higher digits repeat for many outputs).
struct DigitRuns {
  uint32_t d[4], n[4];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int p = 0; p < 4; ++p) { d[p] = 0; n[p] = 0; }
  }
  __device__ __forceinline__ void add(uint32_t (*s_hist)[kRadix], uint32_t key, int passes) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (p >= passes) break;
      const uint32_t dg = (key >> (8 * p)) & 0xffu;
      if (dg != d[p]) {
        if (n[p]) atomicAdd(&s_hist[p][d[p]], n[p]);
        d[p] = dg;
        n[p] = 0;
      }
      ++n[p];
    }
  }
  __device__ __forceinline__ void flush(uint32_t (*s_hist)[kRadix], int passes) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
      if (p < passes && n[p]) atomicAdd(&s_hist[p][d[p]], n[p]);
  }
};

__global__ void __launch_bounds__(kDupThreads) k_dup_expand(DupArgs a) {
  __shared__ uint32_t s_excl[kExpChunk + 1];
  __shared__ uint32_t s_key[kExpChunk];
  __shared__ uint32_t s_val[kExpChunk];
  __shared__ uint32_t s_chunk, s_q0, s_q1;
  __shared__ uint32_t s_hist[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += kDupThreads) (&s_hist[0][0])[i] = 0;
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
    // the chunk's splats: from the one holding its first output to (at most)
    // the one holding the next chunk's first output, from the scan's map
    if (threadIdx.x == 0) {
      s_q0 = a.dup_chunk[chunk];
      s_q1 = a.dup_chunk[chunk + 1];
    }
    __syncthreads();
    // at most one splat per output has outputs here, and splats without any
    // sort after all of them, so kExpChunk bounds the count
    const int q0 = (int)s_q0, nq = min((int)s_q1 - q0 + 1, kExpChunk);
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
      DigitRuns runs;
      runs.init();
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
        const uint32_t key = meta.y + row * gx + (rr - row * w);
        s_key[o - O0] = key;
        s_val[o - O0] = meta.x;
        runs.add(s_hist, key, a.tile_passes);
      }
      runs.flush(s_hist, a.tile_passes);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < O1 - O0; i += kDupThreads) {
      __stcs(a.dup_key + O0 + i, s_key[i]);
      __stcs(a.dup_val + O0 + i, s_val[i]);
    }
    (void)lane;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < a.tile_passes * kRadix; i += kDupThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(a.hist + i, c);
  }
}

// Tile ranges by boundary detection in the sorted pair keys: the first and
// one-past-last position of every tile id present; tiles without pairs keep
// the [0, 0) written by the memset before the sort. Each thread takes
// kRangeItems consecutive keys plus the one after them.
constexpr int kRangeThreads = 256;
constexpr int kRangeItems = 8;

__global__ void __launch_bounds__(kRangeThreads) k_tile_ranges(const uint32_t* __restrict__ keys,
                                                               const uint32_t* ctr, int64_t cap,
                                                               uint2* __restrict__ ranges) {
  const int64_t K = min((int64_t)ctr[kCtrDups], cap);
  const int64_t per = (int64_t)kRangeThreads * kRangeItems;
  for (int64_t base = (int64_t)blockIdx.x * per; base < K; base += (int64_t)gridDim.x * per) {
    const int64_t i0 = base + (int64_t)threadIdx.x * kRangeItems;
    if (i0 >= K) continue;
    uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
    uint32_t cur = keys[i0];
#pragma unroll
    for (int k = 0; k < kRangeItems; ++k) {
      const int64_t i = i0 + k;
      if (i >= K) break;
      const uint32_t next = i + 1 < K ? keys[i + 1] : 0xffffffffu;
      if (cur != prev) ranges[cur].x = (uint32_t)i;
      if (cur != next) ranges[cur].y = (uint32_t)(i + 1);
      prev = cur;
      cur = next;
    }
  }
}

// Blend schedule: the tiles in descending order of their pair count (by
// power-of-two bucket, any order inside a bucket), so that the longest lists
// start first and do not trail the launch. One CTA.
constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const uint2* __restrict__ ranges,
                                                              int tiles,
                                                              uint32_t* __restrict__ order) {
  __shared__ uint32_t s_cnt[33];
  if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    atomicAdd(&s_cnt[len ? __clz(len) : 32], 1u);   // bucket 0 = longest
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = 0; b < 33; ++b) {
      const uint32_t c = s_cnt[b];
      s_cnt[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    order[atomicAdd(&s_cnt[len ? __clz(len) : 32], 1u)] = (uint32_t)t;
  }
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
  d.dup_chunk = ws->dup_chunk;
  d.cap_splats = ws->cap.max_splats;
  d.cap_dups = ws->cap.max_duplicates;
  d.ctr = ws->ctr;
  d.lookback = ws->lookback;
  d.hist = ws->hist + kHistTile * kRadix;
  d.tile_passes = ws->tile_passes;
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
  // ranges of the tiles present in the sorted pairs; the rest stay [0, 0)
  if ((e = launch_zero(ws->ranges, 2 * (int64_t)ws->views.total_tiles, st)) != cudaSuccess) return e;
  {
    static thread_local int range_per_sm = 0;
    if (!range_per_sm) range_per_sm = per_sm_for((const void*)k_tile_ranges, kRangeThreads);
    KernelTimer timer(ws, kKTileRanges, st);
    k_tile_ranges<<<ws->num_sms * range_per_sm, kRangeThreads, 0, st>>>(
        ws->dup_key[ws->dup_final], ws->ctr, ws->cap.max_duplicates, ws->ranges);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKTileOrder, st);
    k_tile_order<<<1, kOrderThreads, 0, st>>>(ws->ranges, ws->views.total_tiles, ws->tile_order);
  }
  return cudaGetLastError();
}

}  // namespace s3r
