// Tile|depth key duplication and the radix sort that orders every tile's
// splats front to back (the rasteriser of Eq. 2), then per-tile ranges.
//
// The sorted order is the one of a stable LSD radix sort on the 64-bit key
// (view-tile id << 32 | FP32 depth bits) over the duplicated pairs in
// projection order (the pairs of the tiles a splat's alpha region reaches,
// see the expansion below). Duplicates of one splat share its depth, so the four
// depth-digit passes run on the splats BEFORE duplication (S keys instead of
// K); the splats are then expanded into (tile, splat) pairs in depth order,
// and the one or two tile-digit passes finish the sort. Every pass is a
// single-pass "onesweep" kernel: persistent CTAs take tiles of kSortTileKeys
// keys (3840 by default) from an atomic counter, rank digits with eight warp
// ballots per key (faster here than match.any, which queues on the
// address-divergence unit), get each digit's global offset from a
// precomputed histogram plus a decoupled look-back over tiles, reorder the
// tile in shared memory and write it out coalesced.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kWarpKeys = kSortItems * 32;   // keys per warp per tile
// Predecessor words a digit's look-back reads per round trip (build-time
// define the autotuner varies).
#ifndef S3R_SORT_LOOKBACK
#define S3R_SORT_LOOKBACK 8
#endif
constexpr int kSortLookback = S3R_SORT_LOOKBACK;
static_assert(kSortLookback >= 1 && kSortLookback <= 64, "look-back batch of 1..64 words");

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

// Keys (and values, or their positions) of one radix tile: warp w reads its
// kWarpKeys consecutive keys as kSortItems coalesced rounds. Slots past the
// end get key 0xffffffff (digit 255) and are never written out.
__device__ __forceinline__ void load_tile(const PassArgs& a, int64_t n, int64_t tile, int warp,
                                          uint32_t lane, uint32_t (&key)[kSortItems],
                                          uint32_t (&val)[kSortItems]) {
  const int64_t first = tile * kSortTileKeys + (int64_t)warp * kWarpKeys + lane;
  // items of this lane below n (one 64-bit compare; the rounds then compare
  // small constants against it), and one base pointer per array
  const int64_t left = n - first;
  const int avail = left <= 0 ? 0 : (left >= (int64_t)kWarpKeys ? kWarpKeys : (int)left);
  const uint32_t* kp = a.keys_in + first;
  const uint32_t* vp = a.vals_in ? a.vals_in + first : nullptr;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = r * 32 < avail;
    key[r] = valid ? __ldcs(kp + r * 32) : 0xffffffffu;
    val[r] = valid ? (vp ? __ldcs(vp + r * 32) : (uint32_t)(first + r * 32)) : 0u;
  }
}

// One LSD pass. Per tile: rank the digits (eight warp ballots per key),
// publish the tile's digit counts for the look-back, reorder the tile by digit
// in shared memory, take the next tile and start its loads, then walk the
// look-back for the global offsets (thread d for digit d, eight predecessors
// per round trip) while those loads are in flight, and write the reordered
// tile out.
__global__ void __launch_bounds__(kSortThreads, S3R_SORT_BLOCKS) k_onesweep(PassArgs a) {
  __shared__ uint32_t s_keys[kSortTileKeys];
  __shared__ uint32_t s_vals[kSortTileKeys];
  __shared__ uint32_t s_cnt[kWarps][kRadix];   // per-warp digit counts -> exclusive offsets
  __shared__ uint32_t s_gbase[kRadix];         // exclusive scan of the global histogram
  __shared__ uint32_t s_loc[kRadix];           // tile-local start of each digit
  __shared__ uint32_t s_dst[kRadix];           // global start of each digit minus its local start
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_tile;

  const int64_t n = min((int64_t)*a.count, a.cap);
  const int64_t n_tiles = (n + kSortTileKeys - 1) / kSortTileKeys;
  const uint32_t tag = stage_tag(a.ctr[kCtrEpoch], a.stage);
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  const int d_me = threadIdx.x;   // the digit this thread scans / looks back on

  if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr + kCtrTileBase + a.stage, 1u);
  s_gbase[d_me] = block_excl_scan(a.hist[d_me], s_tmp, nullptr);   // synchronises
  int64_t tile = s_tile;
  uint32_t key[kSortItems], val[kSortItems];
  if (tile < n_tiles) load_tile(a, n, tile, warp, lane, key, val);

  while (tile < n_tiles) {
    for (int i = lane; i < kRadix; i += 32) s_cnt[warp][i] = 0;
    __syncwarp();
    uint32_t rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      // peers with the same digit: the AND over the digit's eight bits of the
      // ballot or its complement (padding keys rank last within digit 255)
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

    // per digit: exclusive offsets over warps and the tile's count, published
    // at once for the successors' look-back
    uint32_t tile_cnt = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_cnt[w][d_me];
      s_cnt[w][d_me] = tile_cnt;
      tile_cnt += c;
    }
    lookback_publish(a.lookback + d_me, kRadix, tile, tag, tile == 0 ? 2u : 1u, tile_cnt);
    const uint32_t loc = block_excl_scan(tile_cnt, s_tmp, nullptr);   // synchronises
    s_loc[d_me] = loc;
    __syncthreads();

    // reorder in shared memory by digit (stable)
    const int64_t base = tile * kSortTileKeys + (int64_t)warp * kWarpKeys;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      if (base + r * 32 + lane < n) {
        const uint32_t d = (key[r] >> a.shift) & (kRadix - 1);
        const uint32_t pos = s_loc[d] + s_cnt[warp][d] + rank[r];
        s_keys[pos] = key[r];
        s_vals[pos] = val[r];
      }
    }
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr + kCtrTileBase + a.stage, 1u);
    __syncthreads();
    const int64_t next = s_tile;
    // the next tile's loads overlap this tile's look-back and write-out
    if (next < n_tiles) load_tile(a, n, next, warp, lane, key, val);

    uint32_t prefix = 0;
    if (tile > 0) {
      prefix = lookback_walk<kSortLookback>(a.lookback + d_me, kRadix, tile, tag, a.ctr);
      lookback_publish(a.lookback + d_me, kRadix, tile, tag, 2u, prefix + tile_cnt);
    }
    s_dst[d_me] = s_gbase[d_me] + prefix - loc;
    __syncthreads();
    const int tile_n = (int)min((int64_t)kSortTileKeys, n - tile * kSortTileKeys);
    for (int i = threadIdx.x; i < tile_n; i += kSortThreads) {
      const uint32_t k = s_keys[i];
      const uint32_t dst = s_dst[(k >> a.shift) & (kRadix - 1)] + (uint32_t)i;
      __stcs(a.keys_out + dst, k);
      __stcs(a.vals_out + dst, s_vals[i]);
    }
    __syncthreads();   // shared arrays and s_tile are reused
    tile = next;
  }
}

// Expand depth-sorted splats into (view-tile id, splat) pairs, in two kernels
// so that the work is balanced by OUTPUT count: the nearest splats come first
// in depth order and may each cover hundreds of tiles.
//
// A splat is listed in the tiles of its 3-sigma rectangle (the record's rect)
// that its alpha >= 1/255 region reaches: the blend skips every pixel outside
// that region, so the other tiles of the rectangle would only lengthen the
// lists (they are 40-50 % of the rectangle's tiles on the rig workload). With
// the conic q = A dx^2 + 2 B dx dy + C dy^2 the region is the ellipse q <= L,
// L = 2 ln(255 o). A row of tiles is a strip of pixel-centre rows, and the
// ellipse's extent in x within a strip is one interval: its left end
//   x_l(dy) = (-B dy - sqrt(L A - det dy^2)) / A
// is convex in dy with its minimum -sqrt(L C / det) (the ellipse's leftmost
// point) at dy = s = B sqrt(L A / (det (det + B^2))); over a strip it is that
// minimum if s lies in the strip, else the smaller value at the strip's ends.
// The right end is the mirror image (-s, +sqrt(L C / det)). L is raised
// (1.02 L + 0.1), det lowered by a bound on its rounding, the square roots and
// the strip padded, so every interval only grows: a tile is dropped only when
// none of its pixel centres can pass the blend's FP32 test. Splats too
// anisotropic for that guarantee keep their whole rectangle. The square roots
// and reciprocals are the hardware approximations (errors of about 1 ulp, far
// inside the margins), deterministic like the rest of the arithmetic.
//
//  k_splat_tiles: per splat, in depth order (its packed 32-byte record
//                gathered by the sorted id), its tile count (one interval per row of its
//                rectangle) and a 32-byte record for the expansion: the splat
//                id, the tile id of the rectangle's corner, grid and
//                rectangle widths, rectangle height, and its rows: the first
//                kInlineRows in the record, the others 4 bytes each in a row
//                table (offsets from a warp-aggregated bump counter; the warp
//                computes a tall splat's rows together, one per lane), so
//                that the expansion reads most splats' rows without a
//                dependent load. A splat that no longer fits the table
//                stores its region (32 bytes, by splat id) instead, and the
//                expansion recomputes its later rows from it with the same
//                function. Outside the scan below, which would otherwise
//                wait on the few splats with tens of rows.
//  k_dup_scan:   the exclusive scan of the counts (saturating) gives every
//                splat its first output, and every expansion chunk its first
//                splat.
//  k_dup_expand: persistent CTAs take fixed chunks of 256 * kExpItems outputs
//                (2048 at 8); each thread expands kExpItems consecutive
//                outputs (binary search of the chunk's splat offsets in
//                shared memory, a walk over the splat's rows to the first
//                one, then an incremental cursor over rows and splats); the
//                pairs are staged in shared memory and written coalesced.
constexpr int kDupThreads = 256;
#ifndef S3R_DUP_EXPAND_ITEMS
#define S3R_DUP_EXPAND_ITEMS 8   // build-time define the autotuner varies
#endif
constexpr int kExpItems = S3R_DUP_EXPAND_ITEMS;       // outputs per thread per chunk
constexpr int kExpChunk = kDupThreads * kExpItems;    // outputs per chunk
static_assert(kExpChunk >= kDupChunkMin, "the chunk map is sized for chunks of kDupChunkMin");
static_assert(kExpItems <= 14, "above 14 outputs per thread the staged chunk exceeds 48 KB of shared memory");

constexpr float kSpanPad = 0.05f;        // pixels, on the strips and the column bounds

// The alpha >= 1/255 region of a splat in the frame of its rectangle's
// top-left pixel corner. Stored as two float4: (u, v, B, 1/A), (L A, det, ye, xe).
struct Region {
  float u, v, B, inv_A;
  float LA, det;        // det < 0: no usable bound, every tile of a row
  float ye, xe;         // half-extents in y and x; ye < 0: reaches no pixel
  float s;              // dy of the leftmost point (-s: the rightmost)
};

__device__ __forceinline__ void region_store(const Region& g, float4* dst) {
  dst[0] = make_float4(g.u, g.v, g.B, g.inv_A);
  dst[1] = make_float4(g.LA, g.det, g.ye, g.xe);
}

// The stationary point s from the stored fields, so that the scan and the
// expansion derive it identically.
__device__ __forceinline__ void region_finish(Region& g) {
  g.s = (g.det > 0.f && g.ye > 0.f)
            ? __fmul_rn(__fmul_rn(g.B, g.ye), approx_rcp(approx_sqrt(__fmaf_rn(g.B, g.B, g.det))))
            : 0.f;
}

__device__ __forceinline__ Region region_load(const float4 a, const float4 b) {
  Region g;
  g.u = a.x; g.v = a.y; g.B = a.z; g.inv_A = a.w;
  g.LA = b.x; g.det = b.y; g.ye = b.z; g.xe = b.w;
  region_finish(g);
  return g;
}

__device__ __forceinline__ Region region_of(const float2 xy, const float4 co, uint32_t x0,
                                            uint32_t y0) {
  const float A = co.x, B = co.y, C = co.z, o = co.w;
  Region g;
  g.u = __fsub_rn(xy.x, 16.f * (float)x0);
  g.v = __fsub_rn(xy.y, 16.f * (float)y0);
  g.B = B;
  g.inv_A = A > 0.f ? approx_rcp(A) : 0.f;
  g.det = conic_det_lower(A, B, C);
  const float L = __fmaf_rn(2.04f, __logf(__fmul_rn(255.f, o)), 0.1f);   // 1.02 * 2 ln(255 o) + 0.1
  g.LA = __fmul_rn(L, A);
  g.ye = g.xe = 0.f;
  if (g.det > 0.f) {
    if (L > 0.f) {
      g.ye = __fmaf_rn(approx_sqrt(__fmul_rn(g.LA, approx_rcp(g.det))), 1.00001f, kSpanPad);
      g.xe = __fmaf_rn(approx_sqrt(__fmul_rn(__fmul_rn(L, C), approx_rcp(g.det))), 1.00001f, kSpanPad);
    } else {
      g.ye = -1.f;
    }
  }
  region_finish(g);
  return g;
}

// Columns [first, second) (relative to the rectangle, clamped to [0, w)) of
// the tiles in row r of the rectangle that the region reaches.
__device__ __forceinline__ uint2 row_span(const Region& g, uint32_t r, uint32_t w) {
  if (!(g.det > 0.f)) return make_uint2(0u, w);
  const float top = 16.f * (float)r;
  const float lo = fmaxf(__fsub_rn(__fadd_rn(top, 0.5f - kSpanPad), g.v), -g.ye);
  const float hi = fminf(__fsub_rn(__fadd_rn(top, 15.5f + kSpanPad), g.v), g.ye);
  if (!(lo <= hi)) return make_uint2(0u, 0u);
  const float pad = __fmul_rn(4e-6f, g.LA);
  const float rl = approx_sqrt(__fadd_rn(fmaxf(__fmaf_rn(__fmul_rn(-g.det, lo), lo, g.LA), 0.f), pad));
  const float rh = approx_sqrt(__fadd_rn(fmaxf(__fmaf_rn(__fmul_rn(-g.det, hi), hi, g.LA), 0.f), pad));
  const float bl = __fmul_rn(-g.B, lo), bh = __fmul_rn(-g.B, hi);
  float xl = __fmul_rn(fminf(__fsub_rn(bl, rl), __fsub_rn(bh, rh)), g.inv_A);
  float xr = __fmul_rn(fmaxf(__fadd_rn(bl, rl), __fadd_rn(bh, rh)), g.inv_A);
  if (lo <= g.s && g.s <= hi) xl = fminf(xl, -g.xe);
  if (lo <= -g.s && -g.s <= hi) xr = fmaxf(xr, g.xe);
  // tile c holds the pixel centres 16 c + 0.5 .. 16 c + 15.5
  const float ca = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(g.u, xl), 15.5f + kSpanPad), 0.0625f));
  const float cb = floorf(__fmul_rn(__fsub_rn(__fadd_rn(g.u, xr), 0.5f - kSpanPad), 0.0625f)) + 1.f;
  const float fw = (float)w;
  const float a = ca > 0.f ? fminf(ca, fw) : 0.f;           // NaN: 0
  const float b = cb < fw ? fmaxf(cb, 0.f) : fw;            // NaN: w
  return a < b ? make_uint2((uint32_t)a, (uint32_t)b) : make_uint2(0u, 0u);
}

struct DupArgs {
  uint32_t* hist;        // tile-digit histograms of the radix passes that follow
  int tile_passes;
  const uint32_t* sorted_splats;
  const uint2* sp_rect;
  const uint8_t* sp_view;
  const uint32_t* sp_cnt;      // [S] tiles each splat reaches, by depth position
  const uint32_t* row_spans;   // per row of a rectangle: first | end << 16 (columns)
  const float4* sp_region;     // [S][2] region, by splat id, where sp_rowoff is kNoRows
  uint32_t* dup_key;
  uint32_t* dup_val;
  uint32_t* dup_excl;    // [S+1] first output of each sorted splat
  uint4* dup_meta;       // [S][2] records in depth order: (splat, corner tile, gx | w << 16, h),
                         // (first row-table entry or kNoRows, rows 0..2)
  uint32_t* dup_chunk;   // [chunks+1] splat holding each chunk's first output; last: final splat
  int64_t cap_splats, cap_dups;
  uint32_t* ctr;
  unsigned long long* lookback;
};

constexpr int kTilesThreads = 256;
constexpr uint32_t kNoRows = 0xffffffffu;
constexpr int kInlineRows = 3;

struct TilesArgs {
  const uint32_t* sorted;   // depth order -> splat id
  const uint4* tin;         // [S][2] packed splat records (rect and view below: fallback)
  const uint2* rect;
  const uint8_t* view;
  uint32_t* ctr;
  int64_t cap;
  uint32_t* cnt;            // [S] tiles reached, by depth position
  uint4* meta;              // [S][2] expansion records, by depth position
  uint32_t* row_spans;
  int64_t rows_cap;
  float4* region;           // [S][2] by splat id
};

__global__ void __launch_bounds__(kTilesThreads) k_splat_tiles(const __grid_constant__ ViewSet vs,
                                                              TilesArgs a) {
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap);
  const uint32_t lane = lane_id();
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;   // depth position
    const bool live = i < n;
    const uint32_t sp = live ? a.sorted[i] : 0u;
    // the packed inputs: one 32-byte sector per splat
    uint4 t0 = make_uint4(0u, 0u, 0u, 0u), t1 = make_uint4(0u, 0u, 0u, 0u);
    if (live) {
      t0 = a.tin[2 * (size_t)sp];
      t1 = a.tin[2 * (size_t)sp + 1];
    }
    const float2 sxy = make_float2(__uint_as_float(t0.x), __uint_as_float(t0.y));
    const float4 sco = make_float4(__uint_as_float(t0.z), __uint_as_float(t0.w),
                                   __uint_as_float(t1.x), __uint_as_float(t1.y));
    uint32_t x0 = t1.z & 0xffffu, y0 = t1.z >> 16;
    uint32_t w = t1.w & 0x1fffu, h = (t1.w >> 13) & 0x1fffu;
    uint32_t sview = ((t1.w >> 26) & 0x1fu) | ((t1.w >> 31) ? 0x80u : 0u);   // bit 7: moved
    if (live && t1.w == kTinFallback) {   // a view too large for the packed extent
      const uint2 rc = a.rect[sp];
      x0 = rc.x & 0xffffu;
      y0 = rc.x >> 16;
      w = (rc.y & 0xffffu) - x0;
      h = (rc.y >> 16) - y0;
      sview = a.view[sp];
    }
    // table entries for the rows past the inline ones, one atomic per warp
    const uint32_t need = (live && w != 0 && h > kInlineRows) ? h - kInlineRows : 0u;
    uint32_t incl = need;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += t;
    }
    unsigned long long wbase = 0;
    if (lane == 31 && incl)
      wbase = atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr + kCtrRows),
                        (unsigned long long)incl);
    wbase = __shfl_sync(0xffffffffu, wbase, 31);
    const uint64_t off = wbase + incl - need;
    const bool table = off + need <= (uint64_t)a.rows_cap;
    Region g = {};
    if (live) g = region_of(sxy, sco, x0, y0);
    // each lane: the inline rows of its own splat
    uint32_t cnt = 0;
    uint32_t head[kInlineRows] = {0u, 0u, 0u};
    if (live && w != 0)
#pragma unroll
      for (uint32_t r = 0; r < (uint32_t)kInlineRows; ++r)
        if (r < h) {
          const uint2 c = row_span(g, r, w);
          head[r] = c.x | (c.y << 16);
          cnt += c.y - c.x;
        }
    // the warp: the further rows of its taller splats, one splat at a time,
    // one row per lane (a per-lane loop would wait on the tallest splat)
    uint32_t tall = __ballot_sync(0xffffffffu, need != 0u);
    while (tall) {
      const int b = __ffs(tall) - 1;
      tall &= tall - 1;
      Region gb;
      gb.u = __shfl_sync(0xffffffffu, g.u, b);
      gb.v = __shfl_sync(0xffffffffu, g.v, b);
      gb.B = __shfl_sync(0xffffffffu, g.B, b);
      gb.inv_A = __shfl_sync(0xffffffffu, g.inv_A, b);
      gb.LA = __shfl_sync(0xffffffffu, g.LA, b);
      gb.det = __shfl_sync(0xffffffffu, g.det, b);
      gb.ye = __shfl_sync(0xffffffffu, g.ye, b);
      gb.xe = __shfl_sync(0xffffffffu, g.xe, b);
      gb.s = __shfl_sync(0xffffffffu, g.s, b);
      const uint32_t wb = __shfl_sync(0xffffffffu, w, b), hb = __shfl_sync(0xffffffffu, h, b);
      const uint64_t ob = __shfl_sync(0xffffffffu, (unsigned long long)off, b);
      const bool tb = __shfl_sync(0xffffffffu, (int)table, b) != 0;
      uint32_t part = 0;
      for (uint32_t r = kInlineRows + lane; r < hb; r += 32) {
        const uint2 c = row_span(gb, r, wb);
        part += c.y - c.x;
        if (tb) a.row_spans[ob + (r - kInlineRows)] = c.x | (c.y << 16);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == (uint32_t)b) cnt += part;
    }
    if (!live) continue;
    const ViewInfo& vi = vs.v[sview & 0x7f];   // bit 7: Eq. 7 moved
    const uint32_t corner = (uint32_t)vi.tile_base + y0 * (uint32_t)vi.gx + x0;
    // a rectangle without columns (an Eq. 7 splat moved out of the frustum)
    // has no rows either for the expansion, which then reads no row table
    a.cnt[i] = cnt;
    a.meta[2 * i] = make_uint4(sp, corner, (uint32_t)vi.gx | (w << 16), w != 0 ? h : 0u);
    a.meta[2 * i + 1] = make_uint4(table ? (uint32_t)off : kNoRows, head[0], head[1], head[2]);
    if (!table) region_store(g, a.region + 2 * sp);
  }
}

// Exclusive saturating scan (sat_add) of one value per thread across a
// 256-thread block; inputs <= kSat.
__device__ __forceinline__ uint32_t block_excl_scan_sat(uint32_t x, uint32_t* s_tmp /*[8]*/,
                                                        uint32_t* total) {
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl = sat_add(incl, y);
  }
  uint32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0;
  if (lane == 31) s_tmp[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kDupThreads / 32; ++w) {
    const uint32_t c = s_tmp[w];
    if (w < warp) wbase = sat_add(wbase, c);
    tot = sat_add(tot, c);
  }
  __syncthreads();
  *total = tot;
  return sat_add(wbase, excl);
}

// Pair offsets saturate at kSat (above every capacity, which is < 2^31), so a
// real pair count of 2^32 or more cannot wrap into a small one: it latches
// the capacity status like any other overflow.
//
// The counts are in depth order already (k_splat_tiles), so this is a plain
// scan: 4096-count tiles, 16 consecutive counts per thread (128-bit loads and
// stores); a CTA scans the tiles of its chunk in the block, gets the chunk's
// offset from the counts all earlier chunks published (chunk_prefix), and
// reads its counts again (from L2) to write the offsets and the expansion
// chunks' first splats.
constexpr int kDupScanItems = 16;
constexpr int kDupScanTile = kDupThreads * kDupScanItems;   // 4096
constexpr int kDupScanChunkTiles = 16;

__global__ void __launch_bounds__(kDupThreads) k_dup_scan(DupArgs a) {
  __shared__ uint32_t s_ex[kDupScanChunkTiles][kDupThreads];   // thread's offset within the chunk
  __shared__ uint32_t s_tmp[kDupThreads / 32];
  __shared__ uint32_t s_chunk;
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap_splats);
  const int64_t n_tiles = (n + kDupScanTile - 1) / kDupScanTile;
  // one chunk per CTA of the grid where kDupScanChunkTiles tiles allow it (the
  // count is on the device, so every CTA derives the same chunk length)
  const int per = (int)max((int64_t)1, min((int64_t)kDupScanChunkTiles,
                                           (n_tiles + gridDim.x - 1) / (int64_t)gridDim.x));
  const int64_t n_chunks = (n_tiles + per - 1) / per;
  const uint32_t tag = stage_tag(a.ctr[kCtrEpoch], kStageDup);
  auto load = [&](int64_t tile, uint32_t (&c)[kDupScanItems]) {
    const int64_t i0 = tile * kDupScanTile + (int64_t)threadIdx.x * kDupScanItems;
    if (i0 + kDupScanItems <= n) {
      const uint4* p = reinterpret_cast<const uint4*>(a.sp_cnt + i0);
#pragma unroll
      for (int q = 0; q < kDupScanItems / 4; ++q) {
        const uint4 v = p[q];
        c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kDupScanItems; ++k) c[k] = i0 + k < n ? a.sp_cnt[i0 + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kDupScanItems; ++k) c[k] = min(c[k], kSat);
  };
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(a.ctr + kCtrTileBase + kStageDup, 1u);
    __syncthreads();
    const int64_t chunk = s_chunk;
    if (chunk >= n_chunks) break;
    const int64_t t0 = chunk * per;
    const int nt = (int)min((int64_t)per, n_tiles - t0);
    // 1. per tile: the threads' sums, scanned over the block and carried over
    //    the chunk (the next tile's loads issued first)
    uint32_t c[kDupScanItems];
    load(t0, c);
    uint32_t carry = 0;
    for (int i = 0; i < nt; ++i) {
      uint32_t run = 0;
#pragma unroll
      for (int k = 0; k < kDupScanItems; ++k) run = sat_add(run, c[k]);
      if (i + 1 < nt) load(t0 + i + 1, c);
      uint32_t total;
      const uint32_t ex = block_excl_scan_sat(run, s_tmp, &total);   // synchronises
      s_ex[i][threadIdx.x] = sat_add(carry, ex);
      carry = sat_add(carry, total);
    }
    // 2. the chunk's count, published, and every earlier chunk's count
    if (threadIdx.x == 0) lookback_publish(a.lookback, 1, chunk, tag, 1u, carry);
    const uint32_t prefix =
        chunk_prefix<kDupThreads / 32, true>(a.lookback, chunk, tag, a.ctr, s_tmp);
    if (threadIdx.x == 0 && chunk == n_chunks - 1) {
      const uint32_t all = sat_add(prefix, carry);
      a.ctr[kCtrDups] = all;
      a.dup_excl[n] = all;                          // sentinel
      if ((int64_t)all > a.cap_dups) atomicOr(a.ctr + kCtrStatus, kStatusCapacity);
      // after the last chunk: the last splat (chunks end at an inclusive splat bound)
      const uint64_t tot = min((uint64_t)all, (uint64_t)a.cap_dups);
      a.dup_chunk[(tot + kExpChunk - 1) / kExpChunk] = (uint32_t)(n - 1);
    }
    // 3. every splat's first output, and the expansion chunks starting in it
    load(t0, c);
    for (int i = 0; i < nt; ++i) {
      const int64_t i0 = (t0 + i) * kDupScanTile + (int64_t)threadIdx.x * kDupScanItems;
      uint32_t o[kDupScanItems];
      uint32_t ex = sat_add(prefix, s_ex[i][threadIdx.x]);
#pragma unroll
      for (int k = 0; k < kDupScanItems; ++k) {
        o[k] = ex;
        if (i0 + k < n) {
          // every chunk boundary inside this splat's outputs [ex, ex + c)
          // (below capacity) starts with this splat
          const uint64_t e1 = min((uint64_t)ex + c[k], (uint64_t)a.cap_dups);
          for (uint64_t q = ((uint64_t)ex + kExpChunk - 1) / kExpChunk; q * kExpChunk < e1; ++q)
            a.dup_chunk[q] = (uint32_t)(i0 + k);
        }
        ex = sat_add(ex, c[k]);
      }
      if (i + 1 < nt) load(t0 + i + 1, c);
      if (i0 + kDupScanItems <= n) {
        uint4* p = reinterpret_cast<uint4*>(a.dup_excl + i0);
#pragma unroll
        for (int q = 0; q < kDupScanItems / 4; ++q)
          p[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < kDupScanItems; ++k)
          if (i0 + k < n) a.dup_excl[i0 + k] = o[k];
      }
    }
    __syncthreads();   // s_chunk / s_ex reuse
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

// Position in the expansion of one splat: row r of its rectangle, column c in
// the row's interval [.., ce). Rows past the rectangle (an inconsistent count,
// which the shared row function rules out) stay on its last row, so every key
// is a tile of the splat's view.
struct Cursor {
  const uint32_t* row_spans;
  const float4* region;
  uint32_t sp, corner, gx, w, h, off;
  uint32_t head[kInlineRows];
  uint32_t r, c, ce, row_tile;
  __device__ __forceinline__ void load(const uint4* m, const DupArgs& a) {
    row_spans = a.row_spans;
    region = a.sp_region;
    const uint4 d = m[0], e = m[1];
    sp = d.x;
    corner = d.y;
    gx = d.z & 0xffffu;
    w = d.z >> 16;
    h = d.w;
    off = e.x;
    head[0] = e.y;
    head[1] = e.z;
    head[2] = e.w;
  }
  // rows past the inline ones: the row table, or (where it had no room) the
  // stored region through the same function that counted them
  __device__ __forceinline__ uint32_t far_row(uint32_t row) const {
    if (off != kNoRows) return row_spans[off + row - kInlineRows];
    const Region g = region_load(region[2 * (size_t)sp], region[2 * (size_t)sp + 1]);
    const uint2 s = row_span(g, row, w);
    return s.x | (s.y << 16);
  }
  __device__ __forceinline__ void set_row(uint32_t rr) {
    r = rr;
    const uint32_t row = min(r, h - 1u);
    static_assert(kInlineRows == 3, "the selects below take rows 0..2 from registers");
    const uint32_t e = row == 0 ? head[0] : row == 1 ? head[1] : row == 2 ? head[2] : far_row(row);
    c = e & 0xffffu;
    ce = e >> 16;
    row_tile = corner + row * gx;
  }
  // the k-th output of the splat (k < its count)
  __device__ __forceinline__ void seek(uint32_t k) {
    set_row(0);
    while (r + 1 < h && k >= ce - c) {
      k -= ce - c;
      set_row(r + 1);
    }
    c += min(k, ce > c ? ce - c - 1 : 0u);
  }
  __device__ __forceinline__ void next() {
    if (++c < ce) return;
    do {
      set_row(r + 1);
    } while (c >= ce && r + 1 < h);
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
    // kExpItems consecutive outputs per thread
    const uint32_t o0 = O0 + threadIdx.x * kExpItems;
    if (o0 < O1) {
      int lo = 0, hi = nq;            // last local q with s_excl[q] <= o0
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_excl[mid] <= o0) lo = mid; else hi = mid;
      }
      int q = lo;
      const uint32_t oe = min(o0 + kExpItems, O1);
      // cursor: splat q, its row r with columns [c, ce), tile id of column 0 of row r
      Cursor cur;
      cur.load(a.dup_meta + 2 * (q0 + q), a);
      cur.seek(o0 - s_excl[q]);
      uint32_t q_end = s_excl[q + 1];
      DigitRuns runs;
      runs.init();
      for (uint32_t o = o0; o < oe; ++o) {
        while (o >= q_end) {
          ++q;
          q_end = s_excl[q + 1];
          cur.load(a.dup_meta + 2 * (q0 + q), a);
          cur.seek(0);
        }
        const uint32_t key = cur.row_tile + cur.c;
        s_key[o - O0] = key;
        s_val[o - O0] = cur.sp;
        runs.add(s_hist, key, a.tile_passes);
        cur.next();
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

// Tile ranges and the blend queue's classes, one thread per tile: the
// tile's first pair is the lower bound of its id in the sorted pair keys
// (binary search), its end the next tile's first pair (the neighbouring lane's
// search). Every tile's [start, end) is written ([0, 0) for a tile without
// pairs), and the tile is filed under class clz(end - start) (32 for the
// empty ones): a shared count per class, one global atomic per class and
// block for the block's slots, then the ids. The same launch clears the
// forward's contributor bits.
constexpr int kRangeThreads = 256;

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* __restrict__ keys, uint32_t n,
                                                    uint32_t v) {
  uint32_t lo = 0, len = n;
  while (len > 0) {
    const uint32_t half = len >> 1;
    if (__ldg(keys + lo + half) < v) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

__global__ void __launch_bounds__(kRangeThreads) k_tile_ranges(
    const uint32_t* __restrict__ keys, const uint32_t* ctr, int64_t cap, int tiles,
    uint2* __restrict__ ranges, uint32_t* class_cnt, uint32_t* __restrict__ class_list,
    uint32_t* __restrict__ contrib, int64_t contrib_words) {
  __shared__ uint32_t s_cnt[kTileClasses], s_base[kTileClasses];
  const uint32_t K = (uint32_t)min((int64_t)ctr[kCtrDups], cap);
  const uint32_t lane = lane_id();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < contrib_words;
       i += (int64_t)gridDim.x * blockDim.x)
    contrib[i] = 0u;
  for (int base = blockIdx.x * kRangeThreads; base < tiles; base += gridDim.x * kRangeThreads) {
    if (threadIdx.x < kTileClasses) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int t = base + (int)threadIdx.x;
    const bool live = t < tiles;
    const uint32_t start = live ? lower_bound_u32(keys, K, (uint32_t)t) : K;
    uint32_t end = __shfl_down_sync(0xffffffffu, start, 1);
    if (live && (lane == 31 || t + 1 >= tiles)) end = lower_bound_u32(keys, K, (uint32_t)t + 1u);
    int cls = 0;
    uint32_t slot = 0;
    if (live) {
      const uint32_t len = end - start;
      ranges[t] = len ? make_uint2(start, end) : make_uint2(0u, 0u);
      cls = len ? __clz(len) : 32;
      slot = atomicAdd(&s_cnt[cls], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kTileClasses && s_cnt[threadIdx.x])
      s_base[threadIdx.x] = atomicAdd(class_cnt + threadIdx.x, s_cnt[threadIdx.x]);
    __syncthreads();
    if (live) class_list[(size_t)cls * tiles + s_base[cls] + slot] = (uint32_t)t;
    __syncthreads();
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
  d.sp_cnt = ws->sp_tiles;
  d.row_spans = ws->row_spans;
  d.sp_region = reinterpret_cast<const float4*>(ws->sp_region);
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
    static thread_local int tiles_per_sm = 0;
    if (!tiles_per_sm) tiles_per_sm = per_sm_for((const void*)k_splat_tiles, kTilesThreads);
    KernelTimer timer(ws, kKSplatTiles, st);
    TilesArgs t;
    t.rect = ws->sp_rect;
    t.view = ws->sp_view;
    t.ctr = ws->ctr;
    t.cap = ws->cap.max_splats;
    t.sorted = ws->depth_val[0];
    t.tin = reinterpret_cast<const uint4*>(ws->sp_tin);
    t.cnt = ws->sp_tiles;
    t.meta = reinterpret_cast<uint4*>(ws->dup_meta);
    t.row_spans = ws->row_spans;
    t.rows_cap = ws->rows_cap;
    t.region = reinterpret_cast<float4*>(ws->sp_region);
    k_splat_tiles<<<ws->num_sms * tiles_per_sm, kTilesThreads, 0, st>>>(ws->views, t);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKDuplicate, st);
    k_dup_scan<<<(unsigned)scan_ctas((int64_t)ws->num_sms * dup_per_sm), kDupThreads, 0, st>>>(d);
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
  // every tile's range and class (the blend queue), and the cleared
  // contributor bits of the forward
  {
    const int tiles = ws->views.total_tiles;
    int64_t grid = (tiles + kRangeThreads - 1) / kRangeThreads;
    if (grid > (int64_t)ws->num_sms * 8) grid = (int64_t)ws->num_sms * 8;
    if (grid < 1) grid = 1;
    KernelTimer timer(ws, kKTileRanges, st);
    k_tile_ranges<<<(unsigned)grid, kRangeThreads, 0, st>>>(
        ws->dup_key[ws->dup_final], ws->ctr, ws->cap.max_duplicates, tiles, ws->ranges,
        ws->tile_class_cnt, ws->tile_class_list, ws->contrib, 2 * ws->contrib_words);
  }
  return cudaGetLastError();
}

}  // namespace s3r
