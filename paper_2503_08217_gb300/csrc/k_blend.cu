// Front-to-back alpha blending of every 16x16 tile (Eq. 2) and its exact
// adjoint.
//
// Forward: one CTA of two warps per tile, each warp a 16x8 band, four pixels
// per lane, the two of a column evaluated as one packed f32x2 pair. The
// tile's front-to-back splat list is consumed in batches (64 by default) staged in
// shared memory (uv, base-2 conic, opacity, rgb as duplicated pairs, and the
// box where the splat can reach alpha >= 1/255); per 32 splats a warp ballots which of
// them can reach alpha >= 1/255 somewhere in its band (box, then the exact
// ellipse-rectangle test) and evaluates only those. alpha = min(0.99, o G) is
// skipped below 1/255, and a pixel stops before its transmittance would fall
// under 1e-4; a warp stops when all its pixels have stopped. The final
// transmittance and the position of the last blended splat are stored per
// pixel, and the splats blended into at least one pixel of a band are
// recorded as bits for the backward.
//
// Backward: the same tiles and bands walked back to front, starting at each
// warp's last blended splat and visiting only the recorded splats. The
// transmittance before each splat is recovered from the stored final value as
// T <- T / (1 - alpha), so no per-pixel lists are kept; a lane's two pixels
// of a column again form one packed pair. Per splat the nine
// adjoints (uv, conic, opacity, rgb) are summed over the warp with shuffles,
// then over the CTA in shared memory (one shared atomic per splat and warp),
// and flushed to global memory with one vector atomic per four floats.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

// Launch shapes. Each is a build-time define, so that the autotuner
// (autotune.py beside this package's build script) can build and time
// alternatives; the values here are its choice at the surround-rig workload.
#ifndef S3R_BLEND_FWD_BATCH
#define S3R_BLEND_FWD_BATCH 64    // splats staged per batch (forward)
#endif
#ifndef S3R_BLEND_FWD_BLOCKS
#define S3R_BLEND_FWD_BLOCKS 20   // resident forward blocks per SM (register budget)
#endif
#ifndef S3R_BLEND_BWD_BATCH
#define S3R_BLEND_BWD_BATCH 64    // splats staged per batch (backward)
#endif
#ifndef S3R_BLEND_BWD_BLOCKS
#define S3R_BLEND_BWD_BLOCKS 16   // resident backward blocks per SM (register budget)
#endif

constexpr int kBatchBwd = S3R_BLEND_BWD_BATCH;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

// Persistent tile queue: a launch of (SMs x resident blocks) CTAs takes
// positions from an atomic cursor. Tiles come longest lists first
// (k_tile_ranges files every tile under class clz(length), class 0 the
// longest, 32 the empty tiles). Chunks of memory-bound zeroing are spread
// evenly between the tiles (position i is a chunk when floor((i+1) C / P)
// > floor(i C / P), C chunks among P positions), so that their stores run
// while other CTAs of the SM blend: the forward clears the per-splat adjoints
// the backward sums into, the backward in overwrite mode clears the caller's
// gradient arrays. The last CTA to leave resets the cursor for the next launch.
struct TileQueue {
  uint32_t* cursor;
  uint32_t* exits;
};

// Overwrite mode of the backward: the arrays of 1-4 floats per Gaussian are
// zeroed in full (the projection backward, which runs next, writes the kept
// rows), the SH rows only of the Gaussians that no view kept.
constexpr int kZeroChunk = 2048;   // Gaussians (or splats) per chunk (64 words of the kept bitmap)
struct GradZero {
  const uint32_t* kept_bits;
  int64_t n;                       // 0: nothing to zero (accumulate mode)
  s3r_grads g;
  int sh_floats;                   // 3 (K + 1)^2
};

struct BlendArgs {
  const uint2* ranges;
  const uint32_t* class_cnt;    // [kTileClasses] tiles per class
  const uint32_t* class_list;   // [kTileClasses][tiles] tile ids per class
  int tiles;
  TileQueue fwd_queue, bwd_queue;
  GradZero zero;          // backward only
  const uint32_t* sorted_splats;
  const uint4* sp_tin;     // [S][2] packed splat record: (u, v, conic a, b), (conic c, opacity, ..)
  const float4* sp_rgb_d;
  const float* bg;
  const float* dL;        // backward only
  float* out;             // forward only
  float* final_T;
  uint32_t* n_contrib;
  float* sp_grad;         // [S*12]: zeroed by the forward (chunks in its queue), summed by the backward
  const uint32_t* ctr;
  int64_t cap_splats;
  unsigned long long* pairs;     // counting mode: list pairs the forward walked
  unsigned long long* eval_fwd;  // counting mode: pairs the forward evaluated
  unsigned long long* eval_bwd;  // counting mode: pairs the backward evaluated
  uint32_t* contrib;          // [bands][contrib_words]: pair blended into >= 1 pixel of the band
  int64_t contrib_words;
};

// Set the bits of `bits` (positions gp .. gp+31 of the sorted pairs) in a
// bit array; the window may straddle two words (shared with a neighbour tile).
__device__ __forceinline__ void or_bits(uint32_t* arr, uint32_t gp, uint32_t bits) {
  const uint32_t w = gp >> 5, sh = gp & 31u;
  atomicOr(arr + w, bits << sh);
  if (sh) atomicOr(arr + w + 1, bits >> (32u - sh));
}
__device__ __forceinline__ uint32_t get_bits(const uint32_t* arr, uint32_t gp) {
  const uint32_t w = gp >> 5, sh = gp & 31u;
  return __funnelshift_r(arr[w], arr[w + 1], sh);
}

// Class starts of the queue (exclusive scan of the class counts) and the
// number of zeroing chunks, once per CTA; thread 0 takes the CTA's first
// queue position.
__device__ __forceinline__ void queue_init(const BlendArgs& a, const TileQueue& q, uint32_t* s_cstart,
                                           uint32_t n_chunks, uint32_t& pending) {
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int c = 0; c < kTileClasses; ++c) {
      s_cstart[c] = run;
      run += a.class_cnt[c];
    }
    s_cstart[kTileClasses] = run;
    s_cstart[kTileClasses + 1] = n_chunks;
    pending = atomicAdd(q.cursor, 1u);
  }
  __syncthreads();
}

// The CTA's next work item (block-uniform): a tile id (>= 0), a zeroing
// chunk c as -2 - c, or -1 when the queue is empty. Thread 0 holds the
// position taken one item ahead, so that the atomic's round trip overlaps
// the current item's work.
__device__ __forceinline__ int queue_next(const BlendArgs& a, const TileQueue& q,
                                          const uint32_t* s_cstart, int* s_tile, uint32_t& pending) {
  if (threadIdx.x == 0) {
    const uint32_t i = pending;
    const uint64_t T = s_cstart[kTileClasses], C = s_cstart[kTileClasses + 1];
    const uint64_t P = T + C;
    int t = -1;
    if (i < P) {
      pending = atomicAdd(q.cursor, 1u);
      const uint64_t cb = C ? (uint64_t)i * C / P : 0u;              // chunks before position i
      const uint64_t cb1 = C ? ((uint64_t)i + 1u) * C / P : 0u;
      if (cb1 > cb) {
        t = -2 - (int)cb;
      } else {
        const uint32_t ti = (uint32_t)(i - cb);                          // tiles before position i
        int c = 0;
        while (ti >= s_cstart[c + 1]) ++c;
        t = (int)a.class_list[(size_t)c * a.tiles + (ti - s_cstart[c])];
      }
    }
    *s_tile = t;
  }
  __syncthreads();
  return *s_tile;
}

// Every CTA has taken its last item: the last one to leave resets the cursor.
__device__ __forceinline__ void queue_exit(const TileQueue& q) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(q.exits, 1u) == gridDim.x - 1) {
      *q.cursor = 0u;
      *q.exits = 0u;
      __threadfence();
    }
  }
}

__device__ __forceinline__ void zero_span(float* p, int64_t lo, int64_t hi) {
  if (!p) return;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) p[i] = 0.f;
}

template <int SHF>
__device__ __forceinline__ void zero_sh_unkept(const GradZero& z, int64_t w0, int64_t w1) {
  const uint32_t lane = threadIdx.x & 31u;
  const int nwarps = (int)(blockDim.x >> 5);
  for (int64_t w = w0 + (threadIdx.x >> 5); w < w1; w += nwarps) {
    const int64_t g0 = w * 32;
    const int cnt = (int)min((int64_t)32, z.n - g0);
    const uint32_t live = cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u);
    const uint32_t zero = ~z.kept_bits[w] & live;
    if (!zero) continue;
    if constexpr (SHF % 4 == 0) {
      constexpr int W4 = SHF / 4;
      float4* p = reinterpret_cast<float4*>(z.g.sh) + g0 * W4;
      for (int i = (int)lane; i < W4 * cnt; i += 32)
        if ((zero >> (i / W4)) & 1u) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      float* p = z.g.sh + g0 * SHF;
      for (int i = (int)lane; i < SHF * cnt; i += 32)
        if ((zero >> (i / SHF)) & 1u) p[i] = 0.f;
    }
  }
}

// Zeroing chunk c of the forward: the per-splat adjoints (12 floats per
// splat) of splats [c kZeroChunk, (c + 1) kZeroChunk).
__device__ __forceinline__ uint32_t splat_grad_chunks(const BlendArgs& a) {
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap_splats);
  return (uint32_t)((n + kZeroChunk - 1) / kZeroChunk);
}
__device__ void splat_grad_zero_chunk(const BlendArgs& a, int64_t c) {
  const int64_t n = min((int64_t)a.ctr[kCtrSplats], a.cap_splats);
  float4* g = reinterpret_cast<float4*>(a.sp_grad);
  const int64_t lo = 3 * c * kZeroChunk, hi = 3 * min(n, (c + 1) * kZeroChunk);
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Zeroing chunk c of the backward: Gaussians [c kZeroChunk, (c + 1) kZeroChunk).
__device__ __forceinline__ uint32_t grad_chunks(const GradZero& z) {
  return (uint32_t)((z.n + kZeroChunk - 1) / kZeroChunk);
}
__device__ void grad_zero_chunk(const GradZero& z, int64_t c) {
  const int64_t g0 = c * kZeroChunk, g1 = min(z.n, g0 + kZeroChunk);
  zero_span(z.g.means, 3 * g0, 3 * g1);
  zero_span(z.g.log_scales, 3 * g0, 3 * g1);
  zero_span(z.g.quats, 4 * g0, 4 * g1);
  zero_span(z.g.opacity_logits, g0, g1);
  if (z.g.sh) {
    const int64_t w0 = g0 / 32, w1 = (g1 + 31) / 32;
    switch (z.sh_floats) {
      case 3: zero_sh_unkept<3>(z, w0, w1); break;
      case 12: zero_sh_unkept<12>(z, w0, w1); break;
      case 27: zero_sh_unkept<27>(z, w0, w1); break;
      default: zero_sh_unkept<48>(z, w0, w1); break;
    }
  }
}

__device__ __forceinline__ int view_of_tile(const ViewSet& vs, int tile) {
  int v = 0;
  while (v + 1 < vs.n_views && vs.v[v + 1].tile_base <= tile) ++v;
  return v;
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two FP32 values in one 64-bit register for the packed .f32x2 instructions
// (sm_100 and later): one instruction does the same IEEE operation on both
// halves, so the pixel pairs of a lane cost half the issue slots of scalar
// code with bit-identical results.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Shared-memory form of a splat for the blend: the conic is pre-scaled so that
// the exponent is evaluated directly in base 2:
//   a = (u, v, A2, B2), b = (C2, opacity, r, g), c = b-channel, with
//   A2 = -A/2 log2(e), B2 = -B log2(e), C2 = -C/2 log2(e)
// so that power * log2(e) = dx (A2 dx + B2 dy) + C2 dy^2 and G = 2^that.
__device__ __forceinline__ void stage_splat(const float2 xy, const float4 co, const float4 rgb,
                                            float4& a, float4& b, float& c) {
  a = make_float4(xy.x, xy.y, -0.5f * kLog2e * co.x, -kLog2e * co.y);
  b = make_float4(-0.5f * kLog2e * co.z, co.w, rgb.x, rgb.y);
  c = rgb.z;
}

// Exponent (base 2) and alpha of a staged splat at pixel centre (fx, fy), as
// both blend kernels evaluate them (in packed pairs, with these operations in
// this order, so that both take the same FP32 decisions):
//   dx = u - fx, dy = v - fy, p = fma(dx, fma(A2, dx, B2 dy), (C2 dy) dy),
//   G = 2^p (ex2.approx), raw = o G, alpha = min(0.99, raw);
// the pixel takes the splat iff p <= 0 and alpha >= 1/255.

// Bounding box of the region where a staged splat can reach alpha >= 1/255:
// the ellipse d^T Q d <= 2 ln(255 o) (Q the conic), grown by a small relative
// and absolute margin so that FP32 rounding of the exact test can never fall
// outside it. Empty (xmin = +inf) when o < 1/255; unbounded for a splat too
// anisotropic for that guarantee (the per-pixel test then decides alone).
__device__ __forceinline__ float4 alpha_box(const float2 xy, const float4 co) {
  const float o = co.w;
  if (!(o * 255.f > 1.f)) return make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
  const float det = conic_det_lower(co.x, co.y, co.z);
  if (det < 0.f) return make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
  const float L2 = 2.f * __logf(255.f * o);
  const float ex = sqrtf(fmaxf(L2 * co.z / det, 0.f)) * 1.002f + 0.02f;
  const float ey = sqrtf(fmaxf(L2 * co.x / det, 0.f)) * 1.002f + 0.02f;
  return make_float4(xy.x - ex, xy.x + ex, xy.y - ey, xy.y + ey);
}

// The blend kernels run kBandWarps warps per tile; warp r covers the band of
// 16 / kBandWarps rows starting at row r * 16 / kBandWarps, and lane (x, y) =
// (l & 7, l >> 3) owns the pixels (x + 8c, y + 4k) of that band, c = 0, 1.
// The forward's footprint test and contributor bits are per band, and the
// backward walks a band's bits. Neighbouring 8x8 blocks share almost all their
// contributors (a 16x8 band's set is 3 % larger than an 8x8 block's at the rig
// workload), while the per-splat work of a warp (the footprint ballot, the
// loop and the loads; in the backward the nine-value warp sum, its dominant
// cost) is shared by 2 * (4 / kBandWarps) pixels per lane.
constexpr int kBandWarps = 2;
constexpr int kBandThreads = 32 * kBandWarps;
constexpr int kBandRows = 4 / kBandWarps;       // pixel rows per lane and column
constexpr int kBandPix = 2 * kBandRows;         // pixels per lane
static_assert(S3R_BLEND_FWD_BATCH % 32 == 0 && S3R_BLEND_FWD_BATCH <= 256 &&
                  S3R_BLEND_BWD_BATCH % 32 == 0 && S3R_BLEND_BWD_BATCH <= 256,
              "batches are whole 32-splat ballots and stay within static shared memory");
static_assert(S3R_BLEND_FWD_BLOCKS >= 1 && S3R_BLEND_FWD_BLOCKS * kBandThreads <= 2048 &&
                  S3R_BLEND_BWD_BLOCKS >= 1 && S3R_BLEND_BWD_BLOCKS * kBandThreads <= 2048,
              "an SM holds at most 2048 threads");

struct Band {
  int X0, Y0;              // pixel (0, 0) of this lane
  float fx[2], fy[kBandRows];
  float bx0, bx1, by0, by1;   // pixel-centre extent of the warp's band
};
__device__ __forceinline__ Band band_pixels(const ViewInfo& vi, int lt, int warp, uint32_t lane) {
  Band b;
  const int bx = (lt % vi.gx) * kTile, by = (lt / vi.gx) * kTile + warp * (kTile / kBandWarps);
  b.X0 = bx + (int)(lane & 7u);
  b.Y0 = by + (int)(lane >> 3);
#pragma unroll
  for (int c = 0; c < 2; ++c) b.fx[c] = (float)(b.X0 + 8 * c) + 0.5f;
#pragma unroll
  for (int r = 0; r < kBandRows; ++r) b.fy[r] = (float)(b.Y0 + 4 * r) + 0.5f;
  b.bx0 = bx + 0.5f;
  b.bx1 = bx + 15.5f;
  b.by0 = by + 0.5f;
  b.by1 = by + (kTile / kBandWarps) - 0.5f;
  return b;
}

// Whether a staged splat can reach alpha >= 1/255 at some pixel centre of the
// band. The base-2 exponent p = dx (A2 dx + B2 dy) + C2 dy^2 (dx = u - px,
// dy = v - py) is concave, so its maximum over the band's pixel-centre
// rectangle is 0 if the centre lies inside and otherwise lies on an edge, at
// the clamped stationary point of that edge (dy = -B2 X / (2 C2) on the edge
// dx = X, dx = -B2 Y / (2 A2) on dy = Y). The splat passes if that maximum
// reaches log2(1 / (255 o)) less a margin far above FP32 rounding, so that no
// splat the per-pixel test would keep is dropped. Most splats are small and
// anisotropic, and their bounding box touches many bands that the ellipse
// itself misses.
__device__ __forceinline__ bool ellipse_reaches(const float4 a, const float4 b, const Band& t) {
  // the staged conic is (A, B, C) scaled by -log2(e) (A2 = -A/2, B2 = -B, C2 = -C/2)
  if (conic_det_lower(-a.z, -0.5f * a.w, -b.x) < 0.f) return true;
  const float dx0 = a.x - t.bx1, dx1 = a.x - t.bx0;
  const float dy0 = a.y - t.by1, dy1 = a.y - t.by0;
  const bool inside = (dx0 <= 0.f) & (dx1 >= 0.f) & (dy0 <= 0.f) & (dy1 >= 0.f);
  const float A2 = a.z, B2 = a.w, C2 = b.x;
  const float kx = -0.5f * B2 * rcp_approx(C2), ky = -0.5f * B2 * rcp_approx(A2);
  float best = -INFINITY;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const float X = s ? dx1 : dx0;
    const float dy = fminf(fmaxf(kx * X, dy0), dy1);
    best = fmaxf(best, fmaf(X, fmaf(A2, X, B2 * dy), C2 * dy * dy));
    const float Y = s ? dy1 : dy0;
    const float dx = fminf(fmaxf(ky * Y, dx0), dx1);
    best = fmaxf(best, fmaf(dx, fmaf(A2, dx, B2 * Y), C2 * Y * Y));
  }
  const float thr = -__log2f(255.f * b.y);
  return inside | (best >= thr - (0.05f + 1e-3f * fabsf(thr)));
}

__device__ __forceinline__ bool box_misses(const float4 b, const Band& t) {
  return b.x > t.bx1 || b.y < t.bx0 || b.z > t.by1 || b.w < t.by0;
}

// kCount: also count the (pixel, splat) pairs walked (list positions up to
// each pixel's stop) and evaluated (footprint test passed, pixel not stopped).
//
// A lane's two pixels of a column (rows y and y + 4) are evaluated as one
// packed pair: the splat's values are staged in shared memory as duplicated
// pairs (A2 A2 B2 B2 | C2 C2 o o | r r g g | b b v v | u u), so every operand
// of the packed arithmetic comes straight from a 64-bit shared load. The
// arithmetic is the exponent and alpha of stage_splat's comment, in that
// order, so the backward's recomputation takes the same decisions.
constexpr int kBatchFwd = S3R_BLEND_FWD_BATCH;
// One splat of the forward's walk over a warp's four pixels per lane (two
// packed pairs). kClamp: the splat's opacity exceeds 0.99, so alpha = o G may
// reach the 0.99 cap; for o <= 0.99 it cannot (G = 2^p <= 1 where p <= 0, up
// to the last ulp of ex2.approx at p = 0), and the clamp is left out. The
// backward takes the same branch per splat, and the FP64 o G of the exact
// definition never reaches the cap for those splats either.
template <bool kCount, bool kClamp>
__device__ __forceinline__ void fwd_splat(const float4 q0, const float4 q1, const float4 q2,
                                          const float4 q3, const float2 qu, const f2 FY,
                                          const f2 (&FX)[2], const f2 ONE, int pos, f2 (&T2)[2],
                                          f2 (&C2)[2][3], int (&last)[kBandPix],
                                          int (&endp)[kBandPix], bool (&done)[kBandPix],
                                          uint32_t& n_eval, bool& any_blend) {
  // a blended pixel takes alpha >= 1/255 > 0, a skipped one 0: the splat was
  // blended somewhere in the lane's pixels iff the applied alphas sum above 0
  f2 ab_sum = pk(0.f, 0.f);
  const f2 A2 = pk(q0.x, q0.y), B2 = pk(q0.z, q0.w), C2c = pk(q1.x, q1.y), O2 = pk(q1.z, q1.w);
  const f2 R2 = pk(q2.x, q2.y), G2 = pk(q2.z, q2.w), Bl2 = pk(q3.x, q3.y), V2 = pk(q3.z, q3.w);
  const f2 U2 = pk(qu.x, qu.y);
  // the rows' dy and the dy terms of the exponent, shared by both columns
  const f2 dy = sub2(V2, FY);
  const f2 bdy = mul2(B2, dy);
  const f2 cdy = mul2(mul2(C2c, dy), dy);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const f2 dx = sub2(U2, FX[c]);
    const f2 pw = fma2(dx, fma2(A2, dx, bdy), cdy);
    float p[2], G[2];
    upk(pw, p[0], p[1]);
    G[0] = ex2_approx(p[0]);
    G[1] = ex2_approx(p[1]);
    float raw[2];
    upk(mul2(O2, pk(G[0], G[1])), raw[0], raw[1]);
    float al[2], ab[2];
    bool blend[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k = c * kBandRows + r;
      al[r] = kClamp ? fminf(kAlphaMax, raw[r]) : raw[r];
      if constexpr (kCount) n_eval += done[k] ? 0u : 1u;
      blend[r] = !done[k] && !(p[r] > 0.f) && !(al[r] < kAlphaMin);
    }
    float nT[2];
    upk(mul2(T2[c], sub2(ONE, pk(al[0], al[1]))), nT[0], nT[1]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k = c * kBandRows + r;
      const bool stop = blend[r] && (nT[r] < kTStop);
      blend[r] = blend[r] && !stop;
      // one select: T (1 - 0) = T exactly where the splat is not blended
      ab[r] = blend[r] ? al[r] : 0.f;
      last[k] = blend[r] ? pos : last[k];
      if constexpr (kCount) endp[k] = stop ? pos : endp[k];
      done[k] = done[k] || stop;
    }
    const f2 AB = pk(ab[0], ab[1]);
    ab_sum = add2(ab_sum, AB);
    const f2 w = mul2(AB, T2[c]);
    C2[c][0] = fma2(R2, w, C2[c][0]);
    C2[c][1] = fma2(G2, w, C2[c][1]);
    C2[c][2] = fma2(Bl2, w, C2[c][2]);
    T2[c] = mul2(T2[c], sub2(ONE, AB));
  }
  float s0, s1;
  upk(ab_sum, s0, s1);
  any_blend = s0 + s1 > 0.f;
}

// S3R_BLEND_FWD_BLOCKS: 20 blocks per SM (48 registers, a small spill)
// measured fastest: 16 (64 registers) 6 % slower, 22 and 24 11 % slower.
template <bool kCount>
__global__ void __launch_bounds__(kBandThreads, S3R_BLEND_FWD_BLOCKS) k_blend_fwd(const __grid_constant__ ViewSet vs,
                                                            BlendArgs a) {
  static_assert(kBandRows == 2, "the packed forward pairs the two rows of a lane's column");
  __shared__ float4 s_p0[kBatchFwd];   // A2 A2 B2 B2
  __shared__ float4 s_p1[kBatchFwd];   // C2 C2 o o
  __shared__ float4 s_p2[kBatchFwd];   // r r g g
  __shared__ float4 s_p3[kBatchFwd];   // b b v v
  __shared__ float2 s_u[kBatchFwd];    // u u
  __shared__ float4 s_box[kBatchFwd];
  __shared__ uint32_t s_cstart[kTileClasses + 2];
  __shared__ int s_tile;
  uint32_t pending = 0;
  queue_init(a, a.fwd_queue, s_cstart, threadIdx.x == 0 ? splat_grad_chunks(a) : 0u, pending);
  for (;;) {
    const int tile = queue_next(a, a.fwd_queue, s_cstart, &s_tile, pending);
    if (tile == -1) break;
    if (tile < -1) {
      splat_grad_zero_chunk(a, -2 - (int64_t)tile);
      __syncthreads();   // s_tile is rewritten by the next queue_next
      continue;
    }
    const int v = view_of_tile(vs, tile);
    const ViewInfo& vi = vs.v[v];
    const int lt = tile - vi.tile_base;
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const Band P = band_pixels(vi, lt, warp, lane);
    const uint2 range = a.ranges[tile];
    const int n = (int)(range.y - range.x);
    const f2 FY = pk(P.fy[0], P.fy[1]);
    const f2 FX[2] = {pk(P.fx[0], P.fx[0]), pk(P.fx[1], P.fx[1])};
    const f2 ONE = pk(1.f, 1.f);

    // per column c: the pair (row 0, row 1); scalar per-pixel state k = 2c + r
    f2 T2[2], C2[2][3];
    int last[kBandPix], endp[kBandPix];
    bool done[kBandPix];
    uint32_t n_eval = 0;
    bool all_done = true;
  #pragma unroll
    for (int c = 0; c < 2; ++c) {
      T2[c] = ONE;
      C2[c][0] = C2[c][1] = C2[c][2] = pk(0.f, 0.f);
  #pragma unroll
      for (int r = 0; r < kBandRows; ++r) {
        const int k = c * kBandRows + r;
        last[k] = 0;
        done[k] = !(P.X0 + 8 * c < vi.width && P.Y0 + 4 * r < vi.height);
        endp[k] = done[k] ? 0 : n;      // positions walked
        all_done = all_done && done[k];
      }
    }
    uint32_t* wbits = a.contrib + warp * a.contrib_words;
    for (int b0 = 0; b0 < n; b0 += kBatchFwd) {
      // the pixels' done flags are folded once per chunk and batch, not per splat
  #pragma unroll
      for (int k = 0; k < kBandPix; ++k) all_done = all_done && done[k];
      if (__syncthreads_count(all_done) == kBandThreads) break;
      for (int i = threadIdx.x; i < kBatchFwd && b0 + i < n; i += kBandThreads) {
        const uint32_t s = a.sorted_splats[range.x + b0 + i];
        const uint4 t0 = a.sp_tin[2 * (size_t)s], t1 = a.sp_tin[2 * (size_t)s + 1];
        const float2 xy = make_float2(__uint_as_float(t0.x), __uint_as_float(t0.y));
        const float4 co = make_float4(__uint_as_float(t0.z), __uint_as_float(t0.w),
                                      __uint_as_float(t1.x), __uint_as_float(t1.y));
        const float4 rgb = a.sp_rgb_d[s];
        float4 sa, sb;
        float sc;
        stage_splat(xy, co, rgb, sa, sb, sc);
        s_p0[i] = make_float4(sa.z, sa.z, sa.w, sa.w);
        s_p1[i] = make_float4(sb.x, sb.x, sb.y, sb.y);
        s_p2[i] = make_float4(sb.z, sb.z, sb.w, sb.w);
        s_p3[i] = make_float4(sc, sc, sa.y, sa.y);
        s_u[i] = make_float2(sa.x, sa.x);
        s_box[i] = alpha_box(xy, co);
      }
      __syncthreads();
      const int m = min(kBatchFwd, n - b0);
      for (int c0 = 0; c0 < m; c0 += 32) {
        all_done = true;
  #pragma unroll
        for (int k = 0; k < kBandPix; ++k) all_done = all_done && done[k];
        if (__all_sync(0xffffffffu, all_done)) break;
        // which of the next 32 splats can reach alpha >= 1/255 in this warp's band
        const int jl = c0 + (int)lane;
        bool reach = false;
        if (jl < m) {
          const float4 p0 = s_p0[jl], p1 = s_p1[jl], p3 = s_p3[jl];
          const float4 ea = make_float4(s_u[jl].x, p3.z, p0.x, p0.z);
          const float4 eb = make_float4(p1.x, p1.z, 0.f, 0.f);
          reach = !box_misses(s_box[jl], P) && ellipse_reaches(ea, eb, P);
        }
        uint32_t todo = __ballot_sync(0xffffffffu, reach);
        uint32_t blended = 0;     // splats of this chunk blended into some pixel of the band
        while (todo) {
          const int j = c0 + __ffs(todo) - 1;
          todo &= todo - 1;
          const float4 q0 = s_p0[j], q1 = s_p1[j], q2 = s_p2[j], q3 = s_p3[j];
          const float2 qu = s_u[j];
          const int pos = b0 + j + 1;
          bool any_blend = false;
          // warp-uniform: every lane walks the same splat
          if (q1.z > kAlphaMax)
            fwd_splat<kCount, true>(q0, q1, q2, q3, qu, FY, FX, ONE, pos, T2, C2, last, endp, done,
                                    n_eval, any_blend);
          else
            fwd_splat<kCount, false>(q0, q1, q2, q3, qu, FY, FX, ONE, pos, T2, C2, last, endp, done,
                                     n_eval, any_blend);
          if (__any_sync(0xffffffffu, any_blend)) blended |= 1u << (j - c0);
        }
        if (lane == 0 && blended) or_bits(wbits, range.x + b0 + c0, blended);
      }
    }
    if constexpr (kCount) {
      // work accounting, one 64-bit atomic per warp and counter
      unsigned long long walked = 0;
  #pragma unroll
      for (int k = 0; k < kBandPix; ++k) walked += (unsigned long long)endp[k];
      unsigned long long evald = n_eval;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        walked += __shfl_xor_sync(0xffffffffu, walked, o);
        evald += __shfl_xor_sync(0xffffffffu, evald, o);
      }
      if (lane == 0 && walked) atomicAdd(a.pairs, walked);
      if (lane == 0 && evald) atomicAdd(a.eval_fwd, evald);
    }
    const int64_t plane = (int64_t)vi.width * vi.height;
  #pragma unroll
    for (int c = 0; c < 2; ++c) {
      float T[2], Cr[2], Cg[2], Cb[2];
      upk(T2[c], T[0], T[1]);
      upk(C2[c][0], Cr[0], Cr[1]);
      upk(C2[c][1], Cg[0], Cg[1]);
      upk(C2[c][2], Cb[0], Cb[1]);
  #pragma unroll
      for (int r = 0; r < kBandRows; ++r) {
        const int k = c * kBandRows + r;
        const int px = P.X0 + 8 * c, py = P.Y0 + 4 * r;
        if (px < vi.width && py < vi.height) {
          const int64_t pix = (int64_t)py * vi.width + px;
          float* o = a.out + 3 * (int64_t)vi.pix_base + pix;
          o[0] = fmaf(T[r], a.bg[0], Cr[r]);
          o[plane] = fmaf(T[r], a.bg[1], Cg[r]);
          o[2 * plane] = fmaf(T[r], a.bg[2], Cb[r]);
          a.final_T[vi.pix_base + pix] = T[r];
          a.n_contrib[vi.pix_base + pix] = (uint32_t)last[k];
        }
      }
    }
    __syncthreads();   // shared staging is reused by the next tile
  }
  queue_exit(a.fwd_queue);
}

// a ? x : y as one selp. Written out because the compiler turned the
// lane-dependent selects of the warp sum below into divergent branches around
// the shuffles (57 branch instructions per splat in the backward), which made
// the sum several times dearer than its 14 shuffles.
__device__ __forceinline__ float select_f(bool a, float x, float y) {
  float r;
  asm("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\tselp.f32 %0, %1, %2, p;\n\t}"
      : "=f"(r)
      : "f"(x), "f"(y), "r"((int)a));
  return r;
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
    const float send = select_f(b4, v[j], v[j + 4]);
    const float keep = select_f(b4, v[j + 4], v[j]);
    k4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float k2[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = select_f(b3, k4[j], k4[j + 2]);
    const float keep = select_f(b3, k4[j + 2], k4[j]);
    k2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send = select_f(b2, k2[0], k2[1]);
  float k1 = select_f(b2, k2[1], k2[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
  k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
  return k1;
}

__device__ __forceinline__ void red_shared(float* addr, float v) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(addr);
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(sa), "f"(v) : "memory");
}

__device__ __forceinline__ void red_v4(float* p, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z),
               "f"(w)
               : "memory");
}

// Per-pixel state of the reverse walk: the recovered transmittance in front
// of the current splat, and the colour already composited behind it, dotted
// with dL/dC and in absolute terms,
//   Bd = T_final (bg . d) + sum over blended splats k behind of (c_k . d) alpha_k T_k,
// so that dL/dalpha_i = T_i (c_i . d) - Bd / (1 - alpha_i) (Eq. 2 differentiated).
struct BwdPixel {
  float T, Bd, d0, d1, d2;
  int last;
};

// One splat's contribution to the adjoints at one pixel (reverse order), with
// act = the forward blended it there: T <- T / (1 - alpha) where act;
// cd = c . d; dL/dalpha = T cd - Bd / (1 - alpha); w = act ? alpha T : 0;
// Bd += cd w; dL/dopacity = (act and raw <= 0.99 ? G : 0) dL/dalpha (alpha =
// 0.99 is constant); dpow = o dL/dopacity is dL/d(power). The per-splat sums
// are kept in moment form over the warp's pixels,
//   g0 = sum dpow dx, g1 = sum dpow dy, g2 = sum dpow dx^2, g3 = sum dpow dx dy,
//   g4 = sum dpow dy^2, g5 = sum dL/dopacity, g6..8 = sum w dL/dC,
// (a column's pixels share dx, so g0..g3 take its sums of dpow and dpow dy)
// and turned into the adjoints of (u, v, conic) once per splat at the flush.

__device__ __forceinline__ void bwd_init(BwdPixel& q, const BlendArgs& a, const ViewInfo& vi,
                                         int px, int py, bool inside) {
  q.T = 1.f; q.d0 = q.d1 = q.d2 = 0.f; q.last = 0;
  if (inside) {
    const int64_t plane = (int64_t)vi.width * vi.height;
    const int64_t pix = (int64_t)py * vi.width + px;
    const float* g = a.dL + 3 * (int64_t)vi.pix_base + pix;
    q.d0 = g[0];
    q.d1 = g[plane];
    q.d2 = g[2 * plane];
    q.T = a.final_T[vi.pix_base + pix];
    q.last = (int)a.n_contrib[vi.pix_base + pix];
  }
  q.Bd = q.T * (a.bg[0] * q.d0 + a.bg[1] * q.d1 + a.bg[2] * q.d2);
}

// One splat of the backward's walk (see above) over a lane's two packed
// pixel pairs: updates T and Bd, returns the lane's shares of the nine sums
// (g0..g3 scalar, g4..g8 as row pairs). kClamp as for fwd_splat, per splat.
template <bool kCount, bool kClamp>
__device__ __forceinline__ void bwd_splat(const float4 q0, const float4 q1, const float4 q2,
                                          const float4 q3, const float2 qu, const f2 FY,
                                          const f2 (&FX)[2], const f2 ONE, int pos,
                                          const int (&last)[kBandPix], f2 (&T2)[2], f2 (&Bd2)[2],
                                          const f2 (&Q0)[2], const f2 (&Q1)[2], const f2 (&Q2)[2],
                                          uint32_t& n_eval, float (&g)[4], f2& g4, f2& g5, f2& g6,
                                          f2& g7, f2& g8) {
  constexpr int kRows = kBandRows;
  const f2 A2 = pk(q0.x, q0.y), B2 = pk(q0.z, q0.w), C2c = pk(q1.x, q1.y), O2 = pk(q1.z, q1.w);
  const f2 R2 = pk(q2.x, q2.y), G2 = pk(q2.z, q2.w), Bl2 = pk(q3.x, q3.y), V2 = pk(q3.z, q3.w);
  const f2 U2 = pk(qu.x, qu.y);
  const f2 dy = sub2(V2, FY);
  const f2 bdy = mul2(B2, dy);
  const f2 cdy = mul2(mul2(C2c, dy), dy);
  float dyv[2];
  upk(dy, dyv[0], dyv[1]);
  g[0] = g[1] = g[2] = g[3] = 0.f;
  g4 = g5 = g6 = g7 = g8 = pk(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const f2 dx2 = sub2(U2, FX[c]);
    const f2 pw = fma2(dx2, fma2(A2, dx2, bdy), cdy);
    float p[2], G[2], raw[2], al[2], inv[2];
    bool act[2], live[2];
    upk(pw, p[0], p[1]);
    G[0] = ex2_approx(p[0]);
    G[1] = ex2_approx(p[1]);
    upk(mul2(O2, pk(G[0], G[1])), raw[0], raw[1]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int k = c * kRows + r;
      al[r] = kClamp ? fminf(kAlphaMax, raw[r]) : raw[r];
      if constexpr (kCount) n_eval += pos < last[k] ? 1u : 0u;
      act[r] = (pos < last[k]) && !(p[r] > 0.f) && !(al[r] < kAlphaMin);
      // alpha = 0.99 is constant in o; without the cap alpha = o G throughout
      live[r] = kClamp ? act[r] && !(raw[r] > kAlphaMax) : act[r];
    }
    const f2 AL = pk(al[0], al[1]);
    upk(sub2(ONE, AL), inv[0], inv[1]);
    inv[0] = rcp_approx(inv[0]);
    inv[1] = rcp_approx(inv[1]);
    // T before this splat where it was blended; Bd the colour behind it
    float Tn[2], Tc[2];
    upk(mul2(T2[c], pk(inv[0], inv[1])), Tn[0], Tn[1]);
    upk(T2[c], Tc[0], Tc[1]);
    Tc[0] = select_f(act[0], Tn[0], Tc[0]);
    Tc[1] = select_f(act[1], Tn[1], Tc[1]);
    T2[c] = pk(Tc[0], Tc[1]);
    const f2 cd = fma2(R2, Q0[c], fma2(G2, Q1[c], mul2(Bl2, Q2[c])));
    const f2 dal = fma2(T2[c], cd, mul2(Bd2[c], pk(-inv[0], -inv[1])));   // dL/dalpha
    float wv[2];
    upk(mul2(AL, T2[c]), wv[0], wv[1]);
    wv[0] = select_f(act[0], wv[0], 0.f);
    wv[1] = select_f(act[1], wv[1], 0.f);
    const f2 w = pk(wv[0], wv[1]);
    Bd2[c] = fma2(cd, w, Bd2[c]);
    const f2 gd = mul2(pk(select_f(live[0], G[0], 0.f), select_f(live[1], G[1], 0.f)), dal);
    const f2 dpow = mul2(O2, gd);                       // dL/d(power), natural units
    const f2 pdy = mul2(dpow, dy);
    g4 = fma2(pdy, dy, g4);
    g5 = add2(g5, gd);
    g6 = fma2(w, Q0[c], g6);
    g7 = fma2(w, Q1[c], g7);
    g8 = fma2(w, Q2[c], g8);
    // the column's sums of dpow and dpow * dy (dx is shared by its rows)
    float dp[2], pd[2];
    upk(dpow, dp[0], dp[1]);
    upk(pdy, pd[0], pd[1]);
    const float D = dp[0] + dp[1];
    const float E = fmaf(dp[1], dyv[1], pd[0]);
    float dx, dxh;
    upk(dx2, dx, dxh);
    const float t = dx * D;
    g[0] += t;
    g[1] += E;
    g[2] = fmaf(t, dx, g[2]);
    g[3] = fmaf(dx, E, g[3]);
  }
}

// The reverse walk evaluates a lane's two pixels of a column (rows y and
// y + 4) as one packed pair, like the forward: the splat is staged as
// duplicated pairs, the per-pixel state (T, Bd, dL/dC) is held as pairs per
// column, and the recomputation, the recovery of T and dL/dalpha are the
// scalar expressions in the same order. Only the order in which a lane adds
// up its four pixels' shares of the nine sums differs from a scalar walk.
template <bool kCount>
__global__ void __launch_bounds__(kBandThreads, S3R_BLEND_BWD_BLOCKS) k_blend_bwd(
    const __grid_constant__ ViewSet vs, BlendArgs a) {
  static_assert(kBandRows == 2, "the packed backward pairs the two rows of a lane's column");
  constexpr int kT = kBandThreads;
  constexpr int kRows = kBandRows;
  constexpr int kPix = kBandPix;
  __shared__ float4 s_p0[kBatchBwd];   // A2 A2 B2 B2
  __shared__ float4 s_p1[kBatchBwd];   // C2 C2 o o
  __shared__ float4 s_p2[kBatchBwd];   // r r g g
  __shared__ float4 s_p3[kBatchBwd];   // b b v v
  __shared__ float2 s_u[kBatchBwd];    // u u
  __shared__ uint32_t s_id[kBatchBwd];
  __shared__ float s_g[kBatchBwd][9];
  __shared__ float s_sink[kBandThreads];   // target of the lanes with no sum to add
  __shared__ int s_max;
  __shared__ uint32_t s_cstart[kTileClasses + 2];
  __shared__ int s_tile;
  uint32_t pending = 0;
  queue_init(a, a.bwd_queue, s_cstart, grad_chunks(a.zero), pending);
  for (;;) {
    const int tile = queue_next(a, a.bwd_queue, s_cstart, &s_tile, pending);
    if (tile == -1) break;
    if (tile < -1) {
      grad_zero_chunk(a.zero, -2 - (int64_t)tile);
      __syncthreads();   // s_tile is rewritten by the next queue_next
      continue;
    }
    const int v = view_of_tile(vs, tile);
    const ViewInfo& vi = vs.v[v];
    const int lt = tile - vi.tile_base;
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const int X0 = (lt % vi.gx) * kTile + (int)(lane & 7u);
    const int Y0 = (lt / vi.gx) * kTile + warp * (kTile / kBandWarps) + (int)(lane >> 3);
    const uint2 range = a.ranges[tile];

    float fx[2], fy[kRows];
  #pragma unroll
    for (int c = 0; c < 2; ++c) fx[c] = (float)(X0 + 8 * c) + 0.5f;
  #pragma unroll
    for (int r = 0; r < kRows; ++r) fy[r] = (float)(Y0 + 4 * r) + 0.5f;
    const f2 FY = pk(fy[0], fy[1]);
    const f2 FX[2] = {pk(fx[0], fx[0]), pk(fx[1], fx[1])};
    const f2 ONE = pk(1.f, 1.f);
    // per column c: (row 0, row 1) pairs of T, Bd and dL/dC; scalar last contributor
    f2 T2[2], Bd2[2], Q0[2], Q1[2], Q2[2];
    int last[kPix];
    int wlast = 0;
  #pragma unroll
    for (int c = 0; c < 2; ++c) {
      BwdPixel qq[kRows];
  #pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int px = X0 + 8 * c, py = Y0 + 4 * r;
        bwd_init(qq[r], a, vi, px, py, px < vi.width && py < vi.height);
        last[c * kRows + r] = qq[r].last;
        wlast = max(wlast, qq[r].last);
      }
      T2[c] = pk(qq[0].T, qq[1].T);
      Bd2[c] = pk(qq[0].Bd, qq[1].Bd);
      Q0[c] = pk(qq[0].d0, qq[1].d0);
      Q1[c] = pk(qq[0].d1, qq[1].d1);
      Q2[c] = pk(qq[0].d2, qq[1].d2);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
  #pragma unroll
    for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
    if (lane == 0 && wlast) atomicMax(&s_max, wlast);
    __syncthreads();
    const int n = s_max;
    uint32_t n_eval = 0;   // counting mode: pairs inside their pixel's walk
    // the forward recorded its contributors per band, with the same bands
    const uint32_t* wbits = a.contrib + warp * a.contrib_words;

    for (int hi = n; hi > 0; hi -= kBatchBwd) {
      const int lo = max(0, hi - kBatchBwd);
      const int m = hi - lo;
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += kT) {
        const uint32_t s = a.sorted_splats[range.x + lo + i];
        s_id[i] = s;
        const uint4 t0 = a.sp_tin[2 * (size_t)s], t1 = a.sp_tin[2 * (size_t)s + 1];
        const float2 xy = make_float2(__uint_as_float(t0.x), __uint_as_float(t0.y));
        const float4 co = make_float4(__uint_as_float(t0.z), __uint_as_float(t0.w),
                                      __uint_as_float(t1.x), __uint_as_float(t1.y));
        float4 sa, sb;
        float sc;
        stage_splat(xy, co, a.sp_rgb_d[s], sa, sb, sc);
        s_p0[i] = make_float4(sa.z, sa.z, sa.w, sa.w);
        s_p1[i] = make_float4(sb.x, sb.x, sb.y, sb.y);
        s_p2[i] = make_float4(sb.z, sb.z, sb.w, sb.w);
        s_p3[i] = make_float4(sc, sc, sa.y, sa.y);
        s_u[i] = make_float2(sa.x, sa.x);
      }
      for (int i = threadIdx.x; i < kBatchBwd * 9; i += kT) (&s_g[0][0])[i] = 0.f;
      __syncthreads();
      // this warp's splats end at its own last contributor; walk them back to
      // front, 32 at a time, visiting only the splats the forward blended into
      // at least one pixel of the band (recorded bits)
      for (int c1 = min(m, wlast - lo) - 1; c1 >= 0; c1 -= 32) {
        const int c0 = max(0, c1 - 31);
        uint32_t todo = get_bits(wbits, range.x + lo + c0);
        const int span = c1 - c0 + 1;
        if (span < 32) todo &= (1u << span) - 1u;
        // as a ballot result the mask is warp-uniform to the compiler as well
        todo = __ballot_sync(0xffffffffu, (todo >> lane) & 1u);
        while (todo) {
          const int bit = 31 - __clz(todo);
          todo &= ~(1u << bit);
          const int j = c0 + bit;
          const float4 q0 = s_p0[j], q1 = s_p1[j], q2 = s_p2[j], q3 = s_p3[j];
          const float2 qu = s_u[j];
          const int pos = lo + j;
          float g[4];
          f2 g4, g5, g6, g7, g8;
          // warp-uniform: every lane walks the same splat
          if (q1.z > kAlphaMax)
            bwd_splat<kCount, true>(q0, q1, q2, q3, qu, FY, FX, ONE, pos, last, T2, Bd2, Q0, Q1, Q2,
                                    n_eval, g, g4, g5, g6, g7, g8);
          else
            bwd_splat<kCount, false>(q0, q1, q2, q3, qu, FY, FX, ONE, pos, last, T2, Bd2, Q0, Q1, Q2,
                                     n_eval, g, g4, g5, g6, g7, g8);
          float gs[9] = {g[0], g[1], g[2], g[3], 0.f, 0.f, 0.f, 0.f, 0.f};
          {
            float lo4, hi4;
            upk(g4, lo4, hi4); gs[4] = lo4 + hi4;
            upk(g5, lo4, hi4); gs[5] = lo4 + hi4;
            upk(g6, lo4, hi4); gs[6] = lo4 + hi4;
            upk(g7, lo4, hi4); gs[7] = lo4 + hi4;
            upk(g8, lo4, hi4); gs[8] = lo4 + hi4;
          }
          const float tot = warp_sum8_transposed(gs, lane);
          float g8s = gs[8];
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) g8s += __shfl_xor_sync(0xffffffffu, g8s, o);
          // one shared atomic per warp: lanes 4m add value m, lane 1 the ninth
          // sum, the rest add to their own sink word. Predicated atomics compiled
          // to divergent branches (two per splat).
          const bool own = (lane & 3u) == 0;
          float* dst = own ? &s_g[j][lane >> 2] : (lane == 1 ? &s_g[j][8] : &s_sink[threadIdx.x]);
          red_shared(dst, select_f(own, tot, g8s));
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += kT) {
        const float* sg = s_g[i];
        bool any = false;
  #pragma unroll
        for (int r = 0; r < 9; ++r) any |= sg[r] != 0.f;
        if (any) {
          float* dst = a.sp_grad + 12 * (size_t)s_id[i];
          // moments -> adjoints: power*log2(e) = dx (A2 dx + B2 dy) + C2 dy^2 with
          // dx = u - px, so d/du = ln 2 (2 A2 g0 + B2 g1), d/dv = ln 2 (B2 g0 + 2 C2 g1)
          const float A2 = s_p0[i].x, B2 = s_p0[i].z, C2 = s_p1[i].x;
          const float gu = kLn2 * fmaf(2.f * A2, sg[0], B2 * sg[1]);
          const float gv = kLn2 * fmaf(B2, sg[0], 2.f * C2 * sg[1]);
          red_v4(dst, gu, gv, -0.5f * sg[2], -sg[3]);
          red_v4(dst + 4, -0.5f * sg[4], sg[5], sg[6], sg[7]);
          atomicAdd(dst + 8, sg[8]);
        }
      }
    }
    if constexpr (kCount) {
      unsigned long long evald = n_eval;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) evald += __shfl_xor_sync(0xffffffffu, evald, o);
      if (lane == 0 && evald) atomicAdd(a.eval_bwd, evald);
    }
    __syncthreads();   // shared staging is reused by the next tile
  }
  queue_exit(a.bwd_queue);
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
  a.class_cnt = ws->tile_class_cnt;
  a.class_list = ws->tile_class_list;
  a.tiles = ws->views.total_tiles;
  a.fwd_queue = TileQueue{ws->ctr + kCtrBlendFwdCursor, ws->ctr + kCtrBlendFwdExits};
  a.ctr = ws->ctr;
  a.cap_splats = ws->cap.max_splats;
  a.bwd_queue = TileQueue{ws->ctr + kCtrBlendBwdCursor, ws->ctr + kCtrBlendBwdExits};
  a.zero = GradZero{nullptr, 0, {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}, 0};
  a.sorted_splats = ws->dup_val[ws->dup_final];
  a.sp_tin = reinterpret_cast<const uint4*>(ws->sp_tin);
  a.sp_rgb_d = ws->sp_rgb_d;
  a.final_T = ws->final_T;
  a.n_contrib = ws->n_contrib;
  a.sp_grad = ws->sp_grad;
  a.pairs = reinterpret_cast<unsigned long long*>(ws->ctr + kCtrPairs);
  a.eval_fwd = reinterpret_cast<unsigned long long*>(ws->ctr + kCtrEvalFwd);
  a.eval_bwd = reinterpret_cast<unsigned long long*>(ws->ctr + kCtrEvalBwd);
  a.contrib = ws->contrib;
  a.contrib_words = ws->contrib_words;
  a.bg = nullptr;
  a.dL = nullptr;
  a.out = nullptr;
  return a;
}

// Resident CTAs per SM of a blend instantiation, queried once per process.
template <typename K>
int blend_blocks_per_sm(K kernel, int* cache) {
  if (*cache == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBandThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    *cache = per_sm;
  }
  return *cache;
}

cudaError_t launch_render_fwd(s3r_workspace* ws, const float* bg, float* out, cudaStream_t st) {
  BlendArgs a = make_args(ws);
  a.bg = bg;
  a.out = out;
  if (ws->views.total_tiles == 0) return cudaSuccess;
  cudaError_t e;
  if (ws->counting) {
    // pairs walked and evaluated (two adjacent 64-bit counters)
    if ((e = cudaMemsetAsync(a.pairs, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
  }
  // the contributor bits were cleared by the sort's tile ranges
  static thread_local int per_sm[2] = {0, 0};
  KernelTimer timer(ws, kKBlendFwd, st);
  if (ws->counting) {
    const int g = ws->num_sms * blend_blocks_per_sm(k_blend_fwd<true>, &per_sm[1]);
    k_blend_fwd<true><<<g, kBandThreads, 0, st>>>(ws->views, a);
  } else {
    const int g = ws->num_sms * blend_blocks_per_sm(k_blend_fwd<false>, &per_sm[0]);
    k_blend_fwd<false><<<g, kBandThreads, 0, st>>>(ws->views, a);
  }
  ws->sp_grad_clean = 1;
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(s3r_workspace* ws, const float* bg, const float* dL,
                              const s3r_grads* grads, cudaStream_t st) {
  BlendArgs a = make_args(ws);
  a.bg = bg;
  a.dL = dL;
  // the splat adjoints start at zero: cleared by the forward (chunks in its queue), or here
  // when a backward has used them since
  if (!ws->sp_grad_clean) {
    KernelTimer timer(ws, kKZeroGrads, st);
    k_zero_grads<<<ws->num_sms * 4, 256, 0, st>>>(reinterpret_cast<float4*>(ws->sp_grad), ws->ctr,
                                                  ws->cap.max_splats);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
  }
  ws->sp_grad_clean = 0;
  if (ws->grad_mode == S3R_GRAD_OVERWRITE && ws->n > 0 &&
      (grads->means || grads->log_scales || grads->quats || grads->opacity_logits || grads->sh)) {
    a.zero.kept_bits = ws->kept_bits;
    a.zero.n = ws->n;
    a.zero.g = *grads;
    a.zero.sh_floats = 3 * (ws->sh_degree + 1) * (ws->sh_degree + 1);
  }
  cudaError_t e;
  if (ws->counting && (e = cudaMemsetAsync(a.eval_bwd, 0, sizeof(unsigned long long), st)) != cudaSuccess)
    return e;
  static thread_local int per_sm[2] = {0, 0};
  KernelTimer timer(ws, kKBlendBwd, st);
  if (ws->counting) {
    const int g = ws->num_sms * blend_blocks_per_sm(k_blend_bwd<true>, &per_sm[1]);
    k_blend_bwd<true><<<g, kBandThreads, 0, st>>>(ws->views, a);
  } else {
    const int g = ws->num_sms * blend_blocks_per_sm(k_blend_bwd<false>, &per_sm[0]);
    k_blend_bwd<false><<<g, kBandThreads, 0, st>>>(ws->views, a);
  }
  return cudaGetLastError();
}

}  // namespace s3r
