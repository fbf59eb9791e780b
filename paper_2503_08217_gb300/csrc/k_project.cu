// Instance-specific projection of the selected Gaussians into every camera of
// the call (Sec. 3.3 "Instance-specific projection", Eq. 1), the frustum mask
// M_t with the point-life update of Eq. 5, the adaptive-LOD cull (Sec. 3.3
// "Adaptive LOD"), SH colour, and the compaction of the kept (Gaussian, view)
// pairs ("splats") into a dense, ordered array.
//
// One persistent CTA per SM slot. Each CTA first composes all instance
// matrices W_t W_{t,i2g} of all views into shared memory (a few hundred 3x4
// products), then loops over tiles of 256 selected Gaussians taken from an
// atomic counter. Per Gaussian (one thread) the 44 geometry bytes are read
// once for all views; pass 1 computes the frustum/keep masks, a block scan
// plus decoupled look-back gives the splat offsets, pass 2 recomputes the kept
// views, loads the SH coefficients (16-B vector loads) and writes the splats.
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
  // workspace
  const uint32_t* selected;
  uint32_t* frustum_mask;
  uint32_t* keep_mask;
  uint32_t* splat_start;
  uint32_t* kept_list;
  float2* sp_xy;
  float4* sp_conic_o;
  float4* sp_rgb_d;
  uint2* sp_rect;
  uint8_t* sp_view;
  uint32_t* depth_key;
  uint32_t* hist;
  uint32_t* ctr;
  unsigned long long* lookback;
  int64_t cap_splats;
  const InstMat* mats;      // [n_views][n_inst+1], from k_compose
  int32_t* tile_diff;       // per-tile pair counts as a difference array
};

// W_v * P_k for every view v and segment k (k = 0: identity pose), and the
// camera centre in the segment's frame, computed in FP64 once per call. One
// block per view, one thread per segment.
__global__ void k_compose(const __grid_constant__ ViewSet vs, const float4* __restrict__ pose_q,
                          const float* __restrict__ pose_t, int n_inst, InstMat* __restrict__ out) {
  const int v = blockIdx.x;
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
    m.pad[0] = m.pad[1] = 0.f;
    out[v * nk + k] = m;
  }
}

template <int DEG>
__global__ void __launch_bounds__(kThreads) k_project(const __grid_constant__ ViewSet vs, ProjArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // composed matrices are read through L1: a CTA's Gaussians are contiguous,
  // so they touch the matrices of very few instances
  const InstMat* __restrict__ mats = a.mats;
  const int nk = a.n_inst + 1;
  uint32_t* s_off = reinterpret_cast<uint32_t*>(smem_raw);   // [n_inst+2]
  __shared__ uint32_t s_hist[4][kRadix];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_tile, s_base, s_frustum;
  constexpr int K = sh_count(DEG);

  for (int i = threadIdx.x; i < nk + 1; i += blockDim.x) s_off[i] = (uint32_t)a.inst_off[i];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  if (threadIdx.x == 0) s_frustum = 0;
  __syncthreads();

  const uint32_t n_sel = a.ctr[kCtrSelected];
  const uint32_t tag = stage_tag(a.ctr[kCtrEpoch], kStageProject);
  const int64_t n_tiles = ((int64_t)n_sel + kThreads - 1) / kThreads;
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  bool overflow = false;

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr + kCtrTileBase + kStageProject, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= n_tiles) break;
    const int64_t j = tile * kThreads + threadIdx.x;
    const bool active = j < (int64_t)n_sel;

    // ---- load the Gaussian (geometry only)
    uint32_t gid = 0;
    int k = 0;
    float mu[3] = {0.f, 0.f, 0.f}, RS[9];
    if (active) {
      gid = a.selected[j];
      k = segment_of(s_off, a.n_inst, gid);
      mu[0] = a.means[3 * (size_t)gid];
      mu[1] = a.means[3 * (size_t)gid + 1];
      mu[2] = a.means[3 * (size_t)gid + 2];
      const float s0 = __expf(a.log_scales[3 * (size_t)gid]);
      const float s1 = __expf(a.log_scales[3 * (size_t)gid + 1]);
      const float s2 = __expf(a.log_scales[3 * (size_t)gid + 2]);
      float R[9];
      quat_to_rot(a.quats[gid], R);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        RS[3 * r] = R[3 * r] * s0; RS[3 * r + 1] = R[3 * r + 1] * s1; RS[3 * r + 2] = R[3 * r + 2] * s2;
      }
    }

    // ---- pass 1: frustum and keep masks
    uint32_t fmask = 0, kmask = 0;
    if (active) {
      for (int v = 0; v < vs.n_views; ++v) {
        const Proj2D p = project_view(mats[v * nk + k], mu, RS, vs.v[v]);
        if (p.infrustum) {
          fmask |= 1u << v;
          if (p.sigma >= a.lod) kmask |= 1u << v;
        }
      }
    }
    const uint32_t nkept = __popc(kmask);

    // ---- Eq. 5: point-life update on M_t (before LOD)
    if (fmask && a.life) {
      const float2 l = a.life[gid];
      const float2 nl = make_float2(fminf(l.x, a.t), fmaxf(l.y, a.t));
      if (nl.x != l.x || nl.y != l.y) a.life[gid] = nl;
    }

    // ---- block scan of kept-view counts, look-back for the splat base
    uint32_t incl = nkept;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    const uint32_t nfr = __popc(__ballot_sync(0xffffffffu, fmask != 0));
    if (lane == 31) s_warp[warp] = incl;
    if (lane == 0 && nfr) atomicAdd(&s_frustum, nfr);
    __syncthreads();
    if (warp == 0) {
      const uint32_t c = lane < kWarps ? s_warp[lane] : 0u;
      uint32_t wincl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wincl, o);
        if (lane >= (uint32_t)o) wincl += y;
      }
      const uint32_t total = __shfl_sync(0xffffffffu, wincl, 31);
      const uint32_t prefix = warp_lookback(a.lookback, tile, tag, total, a.ctr);
      if (lane < kWarps) s_warp[lane] = wincl - c;
      if (lane == 0) {
        s_base = prefix;
        if (tile == n_tiles - 1) a.ctr[kCtrSplats] = prefix + total;
      }
    }
    __syncthreads();
    uint32_t s = s_base + s_warp[warp] + incl - nkept;

    if (active) {
      a.frustum_mask[j] = fmask;
      a.keep_mask[j] = kmask;
      a.splat_start[j] = s;
    }
    // append the kept Gaussians to the backward's work list (one atomic per warp)
    {
      const uint32_t kb = __ballot_sync(0xffffffffu, kmask != 0u);
      uint32_t kbase = 0;
      if (lane == 0 && kb) kbase = atomicAdd(a.ctr + kCtrKept, (uint32_t)__popc(kb));
      kbase = __shfl_sync(0xffffffffu, kbase, 0);
      if (kmask) a.kept_list[kbase + __popc(kb & lt)] = (uint32_t)j;
    }

    // ---- pass 2: kept views -> splats
    if (kmask) {
      const float opac = 1.f / (1.f + __expf(-a.opac_logits[gid]));
      const float4* sh4 = a.sh + (size_t)gid * (K * 3 / 4);   // K*3 % 4 == 0 for K = 4, 16
      const float* sh1 = a.sh_f + (size_t)gid * K * 3;
      uint32_t m = kmask;
      while (m) {
        const int v = __ffs(m) - 1;
        m &= m - 1;
        const InstMat& M = mats[v * nk + k];
        const Proj2D p = project_view(M, mu, RS, vs.v[v]);
        float rp[3];
        rel_pos(M, mu, rp);
        float dx = rp[0], dy = rp[1], dz = rp[2];
        const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16];
        sh_basis<DEG>(dx, dy, dz, Y);
        float rgb[3] = {0.5f, 0.5f, 0.5f};
        if constexpr ((K * 3) % 4 == 0) {
          // 128-bit loads: coefficient 4q+e of the [K][3] row
#pragma unroll
          for (int qd = 0; qd < K * 3 / 4; ++qd) {
            const float4 c4 = __ldg(sh4 + qd);
            const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int f = 4 * qd + e;
              rgb[f % 3] = fmaf(cv[e], Y[f / 3], rgb[f % 3]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < K; ++i)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaf(__ldg(sh1 + 3 * i + ch), Y[i], rgb[ch]);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) rgb[ch] = fmaxf(rgb[ch], 0.f);
        if ((int64_t)s < a.cap_splats) {
          a.sp_xy[s] = make_float2(p.u, p.v);
          a.sp_conic_o[s] = make_float4(p.ca, p.cb, p.cc, opac);
          a.sp_rgb_d[s] = make_float4(rgb[0], rgb[1], rgb[2], p.z);
          a.sp_rect[s] = make_uint2((uint32_t)p.x0 | ((uint32_t)p.y0 << 16),
                                    (uint32_t)p.x1 | ((uint32_t)p.y1 << 16));
          a.sp_view[s] = (uint8_t)v;
          const uint32_t key = __float_as_uint(p.z);
          a.depth_key[s] = key;
          atomicAdd(&s_hist[0][key & 0xffu], 1u);
          atomicAdd(&s_hist[1][(key >> 8) & 0xffu], 1u);
          atomicAdd(&s_hist[2][(key >> 16) & 0xffu], 1u);
          atomicAdd(&s_hist[3][key >> 24], 1u);
          // pairs per tile: +1 / -1 at the ends of each covered tile row
          const int gx = vs.v[v].gx, w = p.x1 - p.x0;
          int32_t* row = a.tile_diff + vs.v[v].tile_base + p.y0 * gx + p.x0;
          for (int ty = p.y0; ty < p.y1; ++ty, row += gx) {
            atomicAdd(row, 1);
            atomicAdd(row + w, -1);
          }
        } else {
          overflow = true;
        }
        ++s;
      }
    }
    __syncthreads();
  }

  // ---- flush the CTA's digit histograms and counters
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(a.hist + kHistDepth * kRadix + i, c);
  }
  if (threadIdx.x == 0 && s_frustum) atomicAdd(a.ctr + kCtrFrustum, s_frustum);
  if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicOr(a.ctr + kCtrStatus, kStatusCapacity);
}

template <int DEG>
cudaError_t launch_deg(s3r_workspace* ws, const ProjArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * (ws->n_inst + 2) + 16;
  // attribute and occupancy are queried once per shared-memory size, so that a
  // launch inside CUDA-graph capture issues nothing but the kernel
  static thread_local size_t cached_smem = 0;
  static thread_local int cached_per_sm = 0;
  if (smem != cached_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_project<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project<DEG>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cached_smem = smem;
    cached_per_sm = per_sm;
  }
  const int per_sm = cached_per_sm;
  const int grid = ws->num_sms * per_sm;
  KernelTimer timer(ws, kKProject, st);
  k_project<DEG><<<grid, kThreads, smem, st>>>(ws->views, a);
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
  a.selected = ws->selected;
  a.frustum_mask = ws->frustum_mask;
  a.keep_mask = ws->keep_mask;
  a.splat_start = ws->splat_start;
  a.kept_list = ws->kept_list;
  a.sp_xy = ws->sp_xy;
  a.sp_conic_o = ws->sp_conic_o;
  a.sp_rgb_d = ws->sp_rgb_d;
  a.sp_rect = ws->sp_rect;
  a.sp_view = ws->sp_view;
  a.depth_key = ws->depth_key[0];
  a.hist = ws->hist;
  a.ctr = ws->ctr;
  a.lookback = ws->lookback;
  a.cap_splats = ws->cap.max_splats;
  a.mats = reinterpret_cast<const InstMat*>(ws->mats);
  a.tile_diff = ws->tile_diff;
  {
    cudaError_t e0 = cudaMemsetAsync(ws->tile_diff, 0, sizeof(int32_t) * ((size_t)ws->views.total_tiles + 1), st);
    if (e0 != cudaSuccess) return e0;
  }
  {
    KernelTimer timer(ws, kKCompose, st);
    k_compose<<<ws->n_views, 128, 0, st>>>(ws->views, a.pose_q, a.pose_t, sc->n_inst,
                                           reinterpret_cast<InstMat*>(ws->mats));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (sc->sh_degree) {
    case 0: return launch_deg<0>(ws, a, st);
    case 1: return launch_deg<1>(ws, a, st);
    case 2: return launch_deg<2>(ws, a, st);
    default: return launch_deg<3>(ws, a, st);
  }
}

}  // namespace s3r
