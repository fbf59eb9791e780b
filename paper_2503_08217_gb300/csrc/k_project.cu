// Instance-specific projection of the selected Gaussians into every camera of
// the call (Sec. 3.3 "Instance-specific projection", Eq. 1), the frustum mask
// M_t with the point-life update of Eq. 5, the adaptive-LOD cull (Sec. 3.3
// "Adaptive LOD"), SH colour, and the compaction of the kept (Gaussian, view)
// pairs ("splats") into a dense, ordered array.
//
// Three kernels. The mask pass: one thread per selected Gaussian reads its 44
// geometry bytes once and tests every camera (a conservative pre-test, then
// the full projection for the candidates) through the composed matrices W_t
// W_{t,i2g} (written by the compaction's first CTAs; the static segment's
// staged in shared memory for the pre-tests, the others read through L1); it
// writes the frustum and keep masks, applies Eq. 5 and appends the kept
// Gaussians to a work list. The splat-offset scan: block scans over chunks of
// tiles plus the chunk prefix over the kept-view counts. The splat writer: per kept Gaussian,
// its kept views again, SH colour (the warp's SH rows staged through shared
// memory with coalesced 16-B loads) and the splat records.
#include "s3r_math.cuh"

namespace s3r {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct ProjArgs {
  const float* means;
  const float* log_scales;
  const float4* quats;
  const float* opac_logits;
  const float4* sh;            // [n, K*3/4] when K*3 % 4 == 0, else read as floats
  const float* sh_f;
  const int64_t* inst_off;
  int n_inst;
  const float4* pose_q;
  const float* pose_t;
  float t;
  float2* life;
  float lod;
  LodArgs L;               // Eq. 7 on the Gaussians below lod (mode S3R_LOD_STOCHASTIC)
  // workspace
  const uint32_t* selected;
  uint32_t* frustum_mask;
  uint32_t* keep_mask;
  uint32_t* splat_start;
  uint2* kept_list;
  uint32_t* kept_bits;      // selection bitmap from the compaction; unkept bits cleared here
  float4* sp_rgb_d;
  uint2* sp_rect;
  uint8_t* sp_view;
  uint4* sp_tin;            // [S][2] packed splat record (position, conic, opacity, extent)
  uint32_t* depth_key;
  uint32_t* hist;
  uint32_t* ctr;
  unsigned long long* lookback;
  int64_t cap_splats;
  const InstMat* mats;      // [n_views][n_inst+1], composed by the compaction
};

// Pass 1: every selected Gaussian against every camera. Writes the frustum
// and keep masks, applies Eq. 5 to the point life (on the frustum mask, before
// LOD) and appends Gaussians kept in at least one view to the work list.
// S3R_PROJECT_MASK_BLOCKS: six blocks per SM (40 registers, a small spill)
// measured 4 % faster than the compiler's 64 registers
#ifndef S3R_PROJECT_MASK_BLOCKS
#define S3R_PROJECT_MASK_BLOCKS 6   // build-time define the autotuner varies
#endif
static_assert(S3R_PROJECT_MASK_BLOCKS >= 1 && S3R_PROJECT_MASK_BLOCKS * kThreads <= 2048,
              "an SM holds at most 2048 threads");
__global__ void __launch_bounds__(kThreads, S3R_PROJECT_MASK_BLOCKS) k_project_mask(const __grid_constant__ ViewSet vs,
                                                           ProjArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InstMat* __restrict__ mats = a.mats;
  const int nk = a.n_inst + 1;
  uint32_t* s_off = reinterpret_cast<uint32_t*>(smem_raw);   // [n_inst+2]
  __shared__ uint32_t s_frustum;
  __shared__ uint32_t s_wcount[kWarps];
  // per-lane view indices differ: camera records are read from shared memory
  __shared__ ViewInfo s_views[S3R_MAX_VIEWS];
  // the static segment's matrix for every view, staged in shared memory for
  // the pre-tests (the instances' matrices, and the candidates' full
  // projections, read them through L1)
  __shared__ InstMat s_static[S3R_MAX_VIEWS];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(vs.v);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
    const int words = vs.n_views * (int)(sizeof(ViewInfo) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    constexpr int kMatWords = (int)(sizeof(InstMat) / 4);
    float* mdst = reinterpret_cast<float*>(s_static);
    for (int i = threadIdx.x; i < vs.n_views * kMatWords; i += blockDim.x)
      mdst[i] = reinterpret_cast<const float*>(mats + (i / kMatWords) * nk)[i % kMatWords];
  }
  for (int i = threadIdx.x; i < nk + 1; i += blockDim.x) s_off[i] = (uint32_t)a.inst_off[i];
  if (threadIdx.x == 0) s_frustum = 0;
  __syncthreads();
  const uint32_t n_sel = a.ctr[kCtrSelected];
  const uint32_t epoch = a.ctr[kCtrEpoch];
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  uint32_t nfr_local = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int warp = threadIdx.x >> 5;
  // whole blocks stay in the loop (block-wide append below)
  const int64_t span = ((int64_t)n_sel + kThreads - 1) / kThreads * kThreads;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < span; j += stride) {
    const bool active = j < (int64_t)n_sel;
    uint32_t fmask = 0, kmask = 0, gid = 0;
    if (active) {
      gid = a.selected[j];
      const int k = segment_of(s_off, a.n_inst, gid);
      const float mu[3] = {a.means[3 * (size_t)gid], a.means[3 * (size_t)gid + 1],
                           a.means[3 * (size_t)gid + 2]};
      const float s0 = __expf(a.log_scales[3 * (size_t)gid]);
      const float s1 = __expf(a.log_scales[3 * (size_t)gid + 1]);
      const float s2 = __expf(a.log_scales[3 * (size_t)gid + 2]);
      float R[9], RS[9];
      quat_to_rot(a.quats[gid], R);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        RS[3 * r] = R[3 * r] * s0; RS[3 * r + 1] = R[3 * r + 1] * s1; RS[3 * r + 2] = R[3 * r + 2] * s2;
      }
      // cheap conservative test for every view, the full projection only for
      // the candidates (each lane walks its own; the loop runs max-over-lanes times)
      const float smax = fmaxf(s0, fmaxf(s1, s2));
      uint32_t cand = 0;
      if (k == 0) {
        for (int v = 0; v < vs.n_views; ++v)
          if (may_touch_view(s_static[v], mu, smax * smax, s_views[v])) cand |= 1u << v;
      } else {
        for (int v = 0; v < vs.n_views; ++v)
          if (may_touch_view(mats[v * nk + k], mu, smax * smax, s_views[v])) cand |= 1u << v;
      }
      while (cand) {
        const int v = __ffs(cand) - 1;
        cand &= cand - 1;
        const Proj2D p = project_view(mats[v * nk + k], mu, RS, s_views[v]);
        if (p.infrustum) {
          fmask |= 1u << v;
          if (p.sigma >= a.lod ||
              (a.L.mode == S3R_LOD_STOCHASTIC && lod_keep(a.L, gid, (uint32_t)v, epoch, p.z)))
            kmask |= 1u << v;
        }
      }
      a.frustum_mask[j] = fmask;
      a.keep_mask[j] = kmask;
      // Eq. 5: point-life update on M_t (before LOD)
      if (fmask && a.life) {
        const float2 l = a.life[gid];
        const float2 nl = make_float2(fminf(l.x, a.t), fmaxf(l.y, a.t));
        if (nl.x != l.x || nl.y != l.y) a.life[gid] = nl;
      }
    }
    nfr_local += fmask ? 1u : 0u;
    // clear the bitmap bits of selected Gaussians kept in no view, one atomic
    // per run of lanes in the same word (a warp's ids ascend, so the runs are
    // contiguous; a segmented OR collects each run's bits at its first lane)
    {
      const bool drop = active && kmask == 0u;
      if (__any_sync(0xffffffffu, drop)) {
        const uint32_t word = active ? gid >> 5 : 0xffffffffu;
        uint32_t bits = drop ? 1u << (gid & 31u) : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_down_sync(0xffffffffu, bits, o);
          const uint32_t wy = __shfl_down_sync(0xffffffffu, word, o);
          if (lane + (uint32_t)o < 32u && wy == word) bits |= y;
        }
        const uint32_t wprev = __shfl_up_sync(0xffffffffu, word, 1);
        if (active && (lane == 0 || wprev != word) && bits) atomicAnd(a.kept_bits + word, ~bits);
      }
    }
    // append the kept Gaussians to the work list: one atomic per block
    // iteration (a per-warp atomic on one counter serialises in L2)
    const uint32_t kb = __ballot_sync(0xffffffffu, kmask != 0u);
    if (lane == 0) s_wcount[warp] = (uint32_t)__popc(kb);
    __syncthreads();
    if (warp == 0) {
      const uint32_t c = lane < kWarps ? s_wcount[lane] : 0u;
      uint32_t incl = c;
#pragma unroll
      for (int o = 1; o < kWarps; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, incl, kWarps - 1);
      uint32_t base = 0;
      if (lane == 0 && total) base = atomicAdd(a.ctr + kCtrKept, total);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (lane < kWarps) s_wcount[lane] = base + incl - c;
    }
    __syncthreads();
    if (kmask) a.kept_list[s_wcount[warp] + __popc(kb & lt)] = make_uint2((uint32_t)j, gid);
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nfr_local += __shfl_xor_sync(0xffffffffu, nfr_local, o);
  if (lane == 0 && nfr_local) atomicAdd(&s_frustum, nfr_local);
  __syncthreads();
  if (threadIdx.x == 0 && s_frustum) atomicAdd(a.ctr + kCtrFrustum, s_frustum);
}

// First splat of every selected Gaussian: an exclusive scan of the kept-view
// counts popc(keep_mask) in 4096-Gaussian tiles. A thread owns 16 consecutive
// masks (four 128-bit loads and stores). A CTA takes a chunk of consecutive
// tiles, scans each tile in the block, gets the chunk's global offset from
// the counts that all earlier chunks published (chunk_prefix), and then reads
// its masks again (from L2) to write the offsets.
constexpr int kScanItems = 16;
constexpr int kScanTile = kThreads * kScanItems;
constexpr int kScanChunkTiles = 16;   // tiles a CTA's shared memory holds the offsets of

__global__ void __launch_bounds__(kThreads) k_splat_scan(const uint32_t* __restrict__ keep_mask,
                                                         uint32_t* __restrict__ splat_start,
                                                         uint32_t* ctr,
                                                         unsigned long long* lookback) {
  __shared__ uint32_t s_ex[kScanChunkTiles][kThreads];   // thread's offset within the chunk
  __shared__ uint32_t s_tmp[kWarps];
  __shared__ uint32_t s_chunk;
  const uint32_t n_sel = ctr[kCtrSelected];
  const int64_t n_tiles = ((int64_t)n_sel + kScanTile - 1) / kScanTile;
  // one chunk per CTA of the grid where kScanChunkTiles tiles allow it (the
  // count is on the device, so every CTA derives the same chunk length)
  const int per = (int)max((int64_t)1, min((int64_t)kScanChunkTiles,
                                           (n_tiles + gridDim.x - 1) / (int64_t)gridDim.x));
  const int64_t n_chunks = (n_tiles + per - 1) / per;
  const uint32_t tag = stage_tag(ctr[kCtrEpoch], kStageProject);
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  auto load = [&](int64_t tile, uint32_t (&m)[kScanItems]) {
    const int64_t j0 = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
    if (j0 + kScanItems <= (int64_t)n_sel) {
      const uint4* p = reinterpret_cast<const uint4*>(keep_mask + j0);
#pragma unroll
      for (int q = 0; q < kScanItems / 4; ++q) {
        const uint4 v = __ldg(p + q);
        m[4 * q] = v.x; m[4 * q + 1] = v.y; m[4 * q + 2] = v.z; m[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kScanItems; ++i) m[i] = (j0 + i < (int64_t)n_sel) ? keep_mask[j0 + i] : 0u;
    }
  };
  auto run_of = [](const uint32_t (&m)[kScanItems]) {
    uint32_t run = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) run += (uint32_t)__popc(m[i]);
    return run;
  };
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(ctr + kCtrTileBase + kStageProject, 1u);
    __syncthreads();
    const int64_t chunk = s_chunk;
    if (chunk >= n_chunks) break;
    const int64_t t0 = chunk * per;
    const int nt = (int)min((int64_t)per, n_tiles - t0);
    // 1. per tile: the threads' kept-view counts, scanned over the block and
    //    carried over the chunk's tiles (the next tile's loads issued first)
    uint32_t m[kScanItems];
    load(t0, m);
    uint32_t carry = 0;
    for (int i = 0; i < nt; ++i) {
      const uint32_t run = run_of(m);
      if (i + 1 < nt) load(t0 + i + 1, m);
      uint32_t incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      if (lane == 31) s_tmp[warp] = incl;
      __syncthreads();
      uint32_t wbase = 0, tot = 0;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) {
        const uint32_t y = s_tmp[q];
        if (q < warp) wbase += y;
        tot += y;
      }
      s_ex[i][threadIdx.x] = carry + wbase + incl - run;
      carry += tot;
      __syncthreads();   // s_tmp is rewritten by the next tile
    }
    // 2. the chunk's count, published, and every earlier chunk's count
    if (threadIdx.x == 0) lookback_publish(lookback, 1, chunk, tag, 1u, carry);
    const uint32_t prefix = chunk_prefix<kWarps>(lookback, chunk, tag, ctr, s_tmp);
    if (threadIdx.x == 0 && chunk == n_chunks - 1) ctr[kCtrSplats] = prefix + carry;
    // 3. the offsets, from the masks read again
    load(t0, m);
    for (int i = 0; i < nt; ++i) {
      const int64_t j0 = (t0 + i) * kScanTile + (int64_t)threadIdx.x * kScanItems;
      uint32_t o[kScanItems];
      uint32_t off = prefix + s_ex[i][threadIdx.x];
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) {
        o[k] = off;
        off += (uint32_t)__popc(m[k]);
      }
      if (i + 1 < nt) load(t0 + i + 1, m);
      if (j0 + kScanItems <= (int64_t)n_sel) {
        uint4* p = reinterpret_cast<uint4*>(splat_start + j0);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) p[q] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
          if (j0 + k < (int64_t)n_sel) splat_start[j0 + k] = o[k];
      }
    }
    __syncthreads();   // s_chunk / s_ex reuse
  }
}

// Pass 2: the kept (Gaussian, view) pairs become splats: projection of the
// kept views, SH colour, the splat record and its depth-key digit histograms.
// A warp takes 32 work-list entries; their SH rows are staged through shared
// memory with coalesced loads (a lane per 16 B of the warp's rows) instead of
// 32 scattered rows per load instruction.

template <int DEG>
__global__ void __launch_bounds__(kThreads, 3) k_project_splats(const __grid_constant__ ViewSet vs,
                                                             ProjArgs a) {
  using St = ShStage<DEG>;
  constexpr int K = St::K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const InstMat* __restrict__ mats = a.mats;
  const int nk = a.n_inst + 1;
  float* s_sh = reinterpret_cast<float*>(smem_raw);                        // [warps][kWords]
  uint32_t* s_off = reinterpret_cast<uint32_t*>(s_sh + kWarps * St::kWords);  // [n_inst+2]
  __shared__ uint32_t s_hist[4][kRadix];
  // per-lane view indices differ: camera records are read from shared memory
  __shared__ ViewInfo s_views[S3R_MAX_VIEWS];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(vs.v);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
    const int words = vs.n_views * (int)(sizeof(ViewInfo) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  for (int i = threadIdx.x; i < nk + 1; i += blockDim.x) s_off[i] = (uint32_t)a.inst_off[i];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  float* my_sh = s_sh + warp * St::kWords;
  const uint32_t n_kept = a.ctr[kCtrKept];
  const uint32_t epoch = a.ctr[kCtrEpoch];
  bool overflow = false;
  for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32; base < (int64_t)n_kept;
       base += (int64_t)gridDim.x * kThreads) {
    const int64_t t = base + lane;
    const int n_here = (int)min((int64_t)32, (int64_t)n_kept - base);
    const bool valid = lane < (uint32_t)n_here;
    const uint2 e = valid ? a.kept_list[t] : make_uint2(0u, 0u);
    const uint32_t j = e.x, gid = e.y;
    stage_sh_rows<DEG>(my_sh, a.sh_f, gid, n_here, lane);
    __syncwarp();
    if (valid) {
      const uint32_t kmask = a.keep_mask[j];
      uint32_t s = a.splat_start[j];
      const int k = segment_of(s_off, a.n_inst, gid);
      const float mu[3] = {a.means[3 * (size_t)gid], a.means[3 * (size_t)gid + 1],
                           a.means[3 * (size_t)gid + 2]};
      const float s0 = __expf(a.log_scales[3 * (size_t)gid]);
      const float s1 = __expf(a.log_scales[3 * (size_t)gid + 1]);
      const float s2 = __expf(a.log_scales[3 * (size_t)gid + 2]);
      const float4 qv = a.quats[gid];
      const float opac = 1.f / (1.f + __expf(-a.opac_logits[gid]));
      float R[9], RS[9];
      quat_to_rot(qv, R);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        RS[3 * r] = R[3 * r] * s0; RS[3 * r + 1] = R[3 * r + 1] * s1; RS[3 * r + 2] = R[3 * r + 2] * s2;
      }
      const float* row_sh = my_sh + lane * St::kFloatPitch;
      uint32_t m = kmask;
      while (m) {
        const int v = __ffs(m) - 1;
        m &= m - 1;
        const InstMat& M = mats[v * nk + k];
        const ViewInfo& vi = s_views[v];
        Proj2D p = project_view(M, mu, RS, vi);
        // Eq. 7: a kept view below the LOD scale survived the drop draw and is
        // rendered at its noisy mean (no tiles if that leaves the frustum)
        float mv[3] = {mu[0], mu[1], mu[2]};
        const bool moved = a.L.mode == S3R_LOD_STOCHASTIC && p.sigma < a.lod;
        if (moved) {
          lod_noisy_mean(a.L, gid, (uint32_t)v, epoch, p.z, mu, mv);
          p = project_view(M, mv, RS, vi);
          if (!p.infrustum) p.x0 = p.y0 = p.x1 = p.y1 = 0;
        }
        float rp[3];
        rel_pos(M, mv, rp);
        const float inv = rsqrtf(rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2]);
        float Y[16];
        sh_basis<DEG>(rp[0] * inv, rp[1] * inv, rp[2] * inv, Y);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        if constexpr (St::kVec) {
          const float4* r4 = reinterpret_cast<const float4*>(row_sh);
#pragma unroll
          for (int qd = 0; qd < St::kRow; ++qd) {
            const float4 c4 = r4[qd];
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int ee = 0; ee < 4; ++ee) {
              const int f = 4 * qd + ee;
              rgb[f % 3] = fmaf(cv[ee], Y[f / 3], rgb[f % 3]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < K; ++i)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(row_sh[3 * i + ch], Y[i], rgb[ch]);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(rgb[ch], 0.f);
        if ((int64_t)s < a.cap_splats) {
          a.sp_rgb_d[s] = make_float4(rgb[0], rgb[1], rgb[2], p.z);
          a.sp_rect[s] = make_uint2((uint32_t)p.x0 | ((uint32_t)p.y0 << 16),
                                    (uint32_t)p.x1 | ((uint32_t)p.y1 << 16));
          a.sp_view[s] = (uint8_t)v | (moved ? kSplatMoved : (uint8_t)0);
          const bool fits = vi.gx <= kTinMaxGrid && vi.gy <= kTinMaxGrid;
          const uint32_t ext = (uint32_t)(p.x1 - p.x0) | ((uint32_t)(p.y1 - p.y0) << 13) |
                               ((uint32_t)v << 26) | (moved ? 0x80000000u : 0u);
          a.sp_tin[2 * (size_t)s] = make_uint4(__float_as_uint(p.u), __float_as_uint(p.v),
                                               __float_as_uint(p.ca), __float_as_uint(p.cb));
          a.sp_tin[2 * (size_t)s + 1] =
              make_uint4(__float_as_uint(p.cc), __float_as_uint(opac),
                         (uint32_t)p.x0 | ((uint32_t)p.y0 << 16), fits ? ext : kTinFallback);
          // a splat without tiles (an Eq. 7 splat moved out of the frustum)
          // sorts after every real one (+inf), so that no expansion chunk
          // meets it between splats that have pairs
          const bool tiled = p.x1 > p.x0 && p.y1 > p.y0;
          const uint32_t key = tiled ? __float_as_uint(p.z) : 0x7F800000u;
          a.depth_key[s] = key;
          atomicAdd(&s_hist[0][key & 0xffu], 1u);
          atomicAdd(&s_hist[1][(key >> 8) & 0xffu], 1u);
          atomicAdd(&s_hist[2][(key >> 16) & 0xffu], 1u);
          atomicAdd(&s_hist[3][key >> 24], 1u);
        } else {
          overflow = true;
        }
        ++s;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(a.hist + kHistDepth * kRadix + i, c);
  }
  if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicOr(a.ctr + kCtrStatus, kStatusCapacity);
}

template <typename F>
int occupancy(F fn, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

template <int DEG>
cudaError_t launch_deg(s3r_workspace* ws, const ProjArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * (ws->n_inst + 2) + 16;
  const size_t smem_splats = sizeof(float) * kWarps * ShStage<DEG>::kWords + smem;
  // occupancy is queried once (the first, eager call), so that a launch
  // inside CUDA-graph capture issues nothing but the kernels
  static thread_local int per_mask = 0, per_splats = 0, per_scan = 0;
  if (!per_mask) per_mask = occupancy(k_project_mask, smem);
  if (!per_splats) {
    cudaFuncSetAttribute(k_project_splats<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(float) * kWarps * ShStage<DEG>::kWords + 16 * 1024));
    per_splats = occupancy(k_project_splats<DEG>, smem_splats);
  }
  if (!per_scan) per_scan = occupancy(k_splat_scan, 0);
  {
    KernelTimer timer(ws, kKProject, st);
    k_project_mask<<<ws->num_sms * per_mask, kThreads, smem, st>>>(ws->views, a);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKSplatScan, st);
    k_splat_scan<<<(unsigned)scan_ctas((int64_t)ws->num_sms * per_scan), kThreads, 0, st>>>(a.keep_mask, a.splat_start, a.ctr,
                                                              a.lookback);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    KernelTimer timer(ws, kKProjectSplats, st);
    k_project_splats<DEG><<<ws->num_sms * per_splats, kThreads, smem_splats, st>>>(ws->views, a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                           float t, float* life, float lod, cudaStream_t st) {
  ProjArgs a;
  a.means = sc->means;
  a.log_scales = sc->log_scales;
  a.quats = reinterpret_cast<const float4*>(sc->quats);
  a.opac_logits = sc->opacity_logits;
  a.sh = reinterpret_cast<const float4*>(sc->sh);
  a.sh_f = sc->sh;
  a.inst_off = sc->inst_offsets;
  a.n_inst = sc->n_inst;
  a.pose_q = reinterpret_cast<const float4*>(poses ? poses->quat : nullptr);
  a.pose_t = poses ? poses->trans : nullptr;
  a.t = t;
  a.life = reinterpret_cast<float2*>(life);
  a.lod = lod;
  a.L.mode = ws->lod.mode;
  a.L.p_max = ws->lod.p_max;
  a.L.dist = ws->lod.distance;
  for (int i = 0; i < 3; ++i) a.L.off[i] = ws->lod.offset[i];
  a.L.key0 = (uint32_t)ws->lod.seed;
  a.L.key1 = (uint32_t)(ws->lod.seed >> 32);
  a.selected = ws->selected;
  a.frustum_mask = ws->frustum_mask;
  a.keep_mask = ws->keep_mask;
  a.splat_start = ws->splat_start;
  a.kept_list = ws->kept_list;
  a.kept_bits = ws->kept_bits;
  a.sp_rgb_d = ws->sp_rgb_d;
  a.sp_rect = ws->sp_rect;
  a.sp_view = ws->sp_view;
  a.sp_tin = reinterpret_cast<uint4*>(ws->sp_tin);
  a.depth_key = ws->depth_key[0];
  a.hist = ws->hist;
  a.ctr = ws->ctr;
  a.lookback = ws->lookback;
  a.cap_splats = ws->cap.max_splats;
  a.mats = reinterpret_cast<const InstMat*>(ws->mats);
  // the instance matrices were composed by the compaction's first CTAs
  switch (sc->sh_degree) {
    case 0: return launch_deg<0>(ws, a, st);
    case 1: return launch_deg<1>(ws, a, st);
    case 2: return launch_deg<2>(ws, a, st);
    default: return launch_deg<3>(ws, a, st);
  }
}

}  // namespace s3r
