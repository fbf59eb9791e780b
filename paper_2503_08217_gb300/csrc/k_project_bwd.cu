// Backward of the instance-specific projection (Eq. 1 through the composed
// matrices W_t W_{t,i2g} of Sec. 3.3) and of the SH colour: from the per-splat
// 2D adjoints written by the blend backward to the Gaussian parameters and to
// every instance pose.
//
// One thread per kept Gaussian (a warp takes 32 consecutive entries of the
// forward's work list) walks its kept views (its splats are contiguous)
// twice: first the geometry (recomputing the forward intermediates of each
// view: position, covariance, opacity and pose adjoints), then the colour
// (SH and the view-direction term), accumulating the parameter adjoints in
// registers; the owning thread then adds them to the caller's buffers (no
// atomics: a Gaussian has one thread). The SH rows are
// read, and their adjoints added, through shared memory with coalesced
// accesses of the whole warp.
// Adjoints of the composed 3x4 matrices are summed per (view, instance) in
// shared memory and flushed once per CTA; the last CTA to finish then maps
// them to the pose: dP = V_rot^T dW, and through R(q) to (dq, dt).
#include "s3r_math.cuh"

namespace s3r {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct BwdArgs {
  const float* means;
  const float* log_scales;
  const float4* quats;
  const float* opac_logits;
  const float4* sh;
  const float* sh_f;
  const int64_t* inst_off;
  int n_inst;
  const float4* pose_q;
  const float* pose_t;
  const uint32_t* selected;
  const uint32_t* keep_mask;
  const uint2* kept_list;
  const uint32_t* splat_start;
  const float4* sp_grad;   // [S][3] float4
  const uint8_t* sp_view;  // view | kSplatMoved
  LodArgs L;
  int64_t cap_splats;
  uint32_t* ctr;
  float* pose_dM;          // [n_views][n_inst+1][12]
  s3r_grads g;
  const InstMat* mats;     // composed by the forward's compaction (same poses)
  int overwrite;           // S3R_GRAD_OVERWRITE: write the rows instead of adding to them
};

// dL/dP_k = V_rot^T dL/dW_{v,k} summed over views, then (q, t) of the pose,
// for instance k (1-based). dM is read past L1 (other CTAs summed it).
__device__ __forceinline__ void pose_chain_one(const ViewSet& vs, const float* dM, int n_inst, int k,
                                               const float4* __restrict__ pose_q, float* g_q,
                                               float* g_t, int overwrite) {
  const int nk = n_inst + 1;
  float dPr[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, dPt[3] = {0.f, 0.f, 0.f};
  for (int v = 0; v < vs.n_views; ++v) {
    const float* V = vs.v[v].V;
    const float* dp = dM + (v * nk + k) * 12;
    float d[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) d[i] = __ldcg(dp + i);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        dPr[3 * r + c] += V[r] * d[c] + V[4 + r] * d[4 + c] + V[8 + r] * d[8 + c];
      dPt[r] += V[r] * d[3] + V[4 + r] * d[7] + V[8 + r] * d[11];
    }
  }
  if (g_t) {
    float* p = g_t + 3 * (k - 1);
    for (int c = 0; c < 3; ++c) p[c] = overwrite ? dPt[c] : p[c] + dPt[c];
  }
  if (g_q) {
    const float4 gq = quat_backward(pose_q[k - 1], dPr);
    const float v[4] = {gq.x, gq.y, gq.z, gq.w};
    float* p = g_q + 4 * (k - 1);
    for (int c = 0; c < 4; ++c) p[c] = overwrite ? v[c] : p[c] + v[c];
  }
}

template <int DEG>
__global__ void __launch_bounds__(kThreads, 2) k_project_bwd(const __grid_constant__ ViewSet vs,
                                                          BwdArgs a) {
  using St = ShStage<DEG>;
  constexpr int K = St::K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nk = a.n_inst + 1;
  // the composed matrices are read through L1 (a CTA touches few instances);
  // shared memory holds each warp's SH rows, the per-(view, instance) matrix
  // adjoints and the camera records (per-lane view indices differ)
  const InstMat* __restrict__ mats = a.mats;
  float* s_sh = reinterpret_cast<float*>(smem_raw);                        // [warps][kWords]
  float* s_dM = s_sh + kWarps * St::kWords;                                // [views][nk][12]
  uint32_t* s_off = reinterpret_cast<uint32_t*>(s_dM + vs.n_views * nk * 12);
  __shared__ ViewInfo s_views[S3R_MAX_VIEWS];
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(vs.v);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_views);
    const int words = vs.n_views * (int)(sizeof(ViewInfo) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  for (int i = threadIdx.x; i < vs.n_views * nk * 12; i += blockDim.x) s_dM[i] = 0.f;
  for (int i = threadIdx.x; i < nk + 1; i += blockDim.x) s_off[i] = (uint32_t)a.inst_off[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  float* my_sh = s_sh + warp * St::kWords;
  float* row_sh = my_sh + lane * St::kFloatPitch;

  // only Gaussians kept in at least one view have adjoints; a warp takes 32
  // consecutive work-list entries
  const uint32_t n_kept = a.ctr[kCtrKept];
  const uint32_t epoch = a.ctr[kCtrEpoch];
  // software pipeline over the warp's batches: the next batch's work-list
  // entry is loaded one batch ahead, and a batch's mask, splat offset and
  // geometry loads are issued together with its SH staging
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32;
  uint2 kept_next = base + lane < (int64_t)n_kept ? a.kept_list[base + lane] : make_uint2(0u, 0u);
  for (; base < (int64_t)n_kept; base += stride) {
    const int n_here = (int)min((int64_t)32, (int64_t)n_kept - base);
    const bool valid = lane < (uint32_t)n_here;
    const uint2 kept = kept_next;
    kept_next = base + stride + lane < (int64_t)n_kept ? a.kept_list[base + stride + lane]
                                                       : make_uint2(0u, 0u);
    const uint32_t j = kept.x, gid = kept.y;
    uint32_t kmask = 0u, s0 = 0u;
    float mu[3] = {0.f, 0.f, 0.f}, ls[3] = {0.f, 0.f, 0.f}, ol = 0.f;
    float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
    if (valid) {
      kmask = a.keep_mask[j];
      s0 = a.splat_start[j];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        mu[c] = a.means[3 * (size_t)gid + c];
        ls[c] = a.log_scales[3 * (size_t)gid + c];
      }
      q = a.quats[gid];
      ol = a.opac_logits[gid];
    }
    stage_sh_rows<DEG>(my_sh, a.sh_f, gid, n_here, lane);
    __syncwarp();
    float g_sh[K * 3];
#pragma unroll
    for (int i = 0; i < K * 3; ++i) g_sh[i] = 0.f;
    if (kmask) {
    const int k = segment_of(s_off, a.n_inst, gid);
    uint32_t s = s0;

    const float sc[3] = {__expf(ls[0]), __expf(ls[1]), __expf(ls[2])};
    float R[9], RS[9];
    quat_to_rot(q, R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) RS[3 * r + c] = R[3 * r + c] * sc[c];
    const float opac = 1.f / (1.f + __expf(-ol));
    const volatile float* sh = row_sh;   // re-read per use: keeps 48 values out of registers

    float g_mu[3] = {0.f, 0.f, 0.f}, g_RS[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g_RS[i] = 0.f;
    float g_ol = 0.f;

    // Two passes over the kept views: the geometry (position, covariance and
    // opacity adjoints), then the colour (SH and the view-direction term).
    // The second pass recomputes the camera-relative position; the split
    // keeps the 48 SH adjoints out of the registers of the first pass, whose
    // chain is the longer one (fewer spills at the same occupancy).
    uint32_t m = kmask;
    while (m) {
      const int v = __ffs(m) - 1;
      m &= m - 1;
      const int64_t si = s++;
      if (si >= a.cap_splats) break;
      const float4 ga = a.sp_grad[3 * si], gb = a.sp_grad[3 * si + 1];
      // a splat without these adjoints (none of its pairs blended) adds
      // nothing here; skipping it also skips splats moved out of the frustum
      // by Eq. 7
      if (ga.x == 0.f && ga.y == 0.f && ga.z == 0.f && ga.w == 0.f && gb.x == 0.f && gb.y == 0.f)
        continue;
      const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb.x, gO = gb.y;
      const InstMat& M = mats[v * nk + k];
      const ViewInfo& vi = s_views[v];
      const float* A = M.m;   // rows at 0, 4, 8; translation at 3, 7, 11

      // ---- Eq. 7: a splat rendered at its noisy mean is differentiated there
      // (the drawn offset is a constant)
      float mv[3] = {mu[0], mu[1], mu[2]};
      if (a.sp_view[si] & kSplatMoved) {
        float rp0[3], x0, y0, z0;
        rel_pos(M, mu, rp0);
        cam_pos(M, rp0, x0, y0, z0);
        lod_noisy_mean(a.L, gid, (uint32_t)v, epoch, z0, mu, mv);
      }

      // ---- forward recompute (the same arithmetic as project_view)
      float rp[3], x, y, z;
      rel_pos(M, mv, rp);
      cam_pos(M, rp, x, y, z);
      float B[9];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          B[3 * r + c] = fmaf(A[4 * r], RS[c], fmaf(A[4 * r + 1], RS[3 + c], A[4 * r + 2] * RS[6 + c]));
      const float iz = rcp_fast(z);
      const float rx = x * iz, ry = y * iz;
      const bool clx = rx < -vi.limx || rx > vi.limx;
      const bool cly = ry < -vi.limy || ry > vi.limy;
      const float txr = fminf(vi.limx, fmaxf(-vi.limx, rx));
      const float tyr = fminf(vi.limy, fmaxf(-vi.limy, ry));
      const float j00 = vi.fx * iz, j02 = -vi.fx * txr * iz;
      const float j11 = vi.fy * iz, j12 = -vi.fy * tyr * iz;
      float C0[3], C1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C0[c] = fmaf(j00, B[c], j02 * B[6 + c]);
        C1[c] = fmaf(j11, B[3 + c], j12 * B[6 + c]);
      }
      const float sa = fmaf(C0[0], C0[0], fmaf(C0[1], C0[1], C0[2] * C0[2]));
      const float sb = fmaf(C0[0], C1[0], fmaf(C0[1], C1[1], C0[2] * C1[2]));
      const float scc = fmaf(C1[0], C1[0], fmaf(C1[1], C1[1], C1[2] * C1[2]));
      const float ad = sa + kDilation, cd = scc + kDilation;
      const float idet = rcp_fast(ad * cd - sb * sb);
      const float qa = cd * idet, qb = -sb * idet, qc = ad * idet;

      float dA[9], db[3], dp[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 9; ++i) dA[i] = 0.f;
      db[0] = db[1] = db[2] = 0.f;

      // ---- opacity = sigmoid(logit)
      g_ol += gO * opac * (1.f - opac);

      // ---- conic = inverse of the dilated 2D covariance
      const float hb = 0.5f * gB;
      const float m00 = qa * gA + qb * hb, m01 = qa * hb + qb * gC;
      const float m10 = qb * gA + qc * hb, m11 = qb * hb + qc * gC;
      const float g_a = -(m00 * qa + m01 * qb);
      const float g_b = -2.f * (m00 * qb + m01 * qc);
      const float g_c = -(m10 * qb + m11 * qc);
      // ---- Sigma2 = C C^T
      float dC0[3], dC1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dC0[c] = 2.f * g_a * C0[c] + g_b * C1[c];
        dC1[c] = 2.f * g_c * C1[c] + g_b * C0[c];
      }
      // ---- C = J B
      const float dj00 = dC0[0] * B[0] + dC0[1] * B[1] + dC0[2] * B[2];
      const float dj02 = dC0[0] * B[6] + dC0[1] * B[7] + dC0[2] * B[8];
      const float dj11 = dC1[0] * B[3] + dC1[1] * B[4] + dC1[2] * B[5];
      const float dj12 = dC1[0] * B[6] + dC1[1] * B[7] + dC1[2] * B[8];
      float dB[9];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dB[c] = j00 * dC0[c];
        dB[3 + c] = j11 * dC1[c];
        dB[6 + c] = j02 * dC0[c] + j12 * dC1[c];
      }
      // ---- B = A RS
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dA[3 * r + c] += dB[3 * r] * RS[3 * c] + dB[3 * r + 1] * RS[3 * c + 1] + dB[3 * r + 2] * RS[3 * c + 2];
          g_RS[3 * r + c] += A[r] * dB[c] + A[4 + r] * dB[3 + c] + A[8 + r] * dB[6 + c];
        }
      // ---- J(p), with the field-of-view clamp
      dp[2] -= (dj00 * j00 + dj11 * j11) * iz;
      if (!clx) {
        dp[0] -= dj02 * vi.fx * iz * iz;
        dp[2] -= 2.f * dj02 * j02 * iz;
      } else {
        dp[2] -= dj02 * j02 * iz;
      }
      if (!cly) {
        dp[1] -= dj12 * vi.fy * iz * iz;
        dp[2] -= 2.f * dj12 * j12 * iz;
      } else {
        dp[2] -= dj12 * j12 * iz;
      }
      // ---- (u, v) = (fx x/z + cx, fy y/z + cy)
      dp[0] += gu * vi.fx * iz;
      dp[1] += gv * vi.fy * iz;
      dp[2] -= (gu * vi.fx * rx + gv * vi.fy * ry) * iz;
      // ---- p = A mu + b
#pragma unroll
      for (int c = 0; c < 3; ++c) g_mu[c] += A[c] * dp[0] + A[4 + c] * dp[1] + A[8 + c] * dp[2];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        dA[3 * r] += dp[r] * mv[0]; dA[3 * r + 1] += dp[r] * mv[1]; dA[3 * r + 2] += dp[r] * mv[2];
        db[r] += dp[r];
      }
      if (k > 0) {
        float* dst = s_dM + (v * nk + k) * 12;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          atomicAdd(dst + 4 * r, dA[3 * r]);
          atomicAdd(dst + 4 * r + 1, dA[3 * r + 1]);
          atomicAdd(dst + 4 * r + 2, dA[3 * r + 2]);
          atomicAdd(dst + 4 * r + 3, db[r]);
        }
      }
    }

    // ---- RS = R diag(s), s = exp(log s), R = R(q/|q|)
    float dR[9], g_ls[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g_ls[c] = (R[c] * g_RS[c] + R[3 + c] * g_RS[3 + c] + R[6 + c] * g_RS[6 + c]) * sc[c];
#pragma unroll
      for (int r = 0; r < 3; ++r) dR[3 * r + c] = g_RS[3 * r + c] * sc[c];
    }
    const float4 g_q = quat_backward(q, dR);

    if (a.g.log_scales) {
      float* p = a.g.log_scales + 3 * (size_t)gid;
      if (a.overwrite) {
        p[0] = g_ls[0]; p[1] = g_ls[1]; p[2] = g_ls[2];
      } else {
        p[0] += g_ls[0]; p[1] += g_ls[1]; p[2] += g_ls[2];
      }
    }
    if (a.g.quats) {
      float4* p = reinterpret_cast<float4*>(a.g.quats) + gid;
      if (a.overwrite) {
        *p = g_q;
      } else {
        float4 o = *p;
        o.x += g_q.x; o.y += g_q.y; o.z += g_q.z; o.w += g_q.w;
        *p = o;
      }
    }
    if (a.g.opacity_logits) {
      if (a.overwrite) a.g.opacity_logits[gid] = g_ol;
      else a.g.opacity_logits[gid] += g_ol;
    }

    // ---- second pass: the colour of each kept view
    m = kmask;
    s = s0;
    while (m) {
      const int v = __ffs(m) - 1;
      m &= m - 1;
      const int64_t si = s++;
      if (si >= a.cap_splats) break;
      const float4 gb = a.sp_grad[3 * si + 1], gc = a.sp_grad[3 * si + 2];
      if (gb.z == 0.f && gb.w == 0.f && gc.x == 0.f) continue;   // no colour adjoint
      const float grgb[3] = {gb.z, gb.w, gc.x};
      const InstMat& M = mats[v * nk + k];
      const float* A = M.m;
      float mv[3] = {mu[0], mu[1], mu[2]};
      if (a.sp_view[si] & kSplatMoved) {
        float rp0[3], x0, y0, z0;
        rel_pos(M, mu, rp0);
        cam_pos(M, rp0, x0, y0, z0);
        lod_noisy_mean(a.L, gid, (uint32_t)v, epoch, z0, mu, mv);
      }
      float rp[3];
      rel_pos(M, mv, rp);
      float dA[9], db[3];
#pragma unroll
      for (int i = 0; i < 9; ++i) dA[i] = 0.f;
      db[0] = db[1] = db[2] = 0.f;
      // ---- colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5), dir from the camera centre
      {
        const float vx = rp[0], vy = rp[1], vz = rp[2];
        const float inv = rsqrtf(vx * vx + vy * vy + vz * vz);
        const float dx = vx * inv, dy = vy * inv, dz = vz * inv;
        float Y[16];
        sh_basis<DEG>(dx, dy, dz, Y);
        float graw[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          float acc = 0.5f;
#pragma unroll
          for (int i = 0; i < K; ++i) acc = fmaf(sh[3 * i + ch], Y[i], acc);
          graw[ch] = acc < 0.f ? 0.f : grgb[ch];
        }
        float wk[16];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          g_sh[3 * i] += Y[i] * graw[0];
          g_sh[3 * i + 1] += Y[i] * graw[1];
          g_sh[3 * i + 2] += Y[i] * graw[2];
          wk[i] = sh[3 * i] * graw[0] + sh[3 * i + 1] * graw[1] + sh[3 * i + 2] * graw[2];
        }
        if (DEG > 0) {
          float gd[3];
          sh_dir_grad<DEG>(dx, dy, dz, wk, gd);
          const float dd = gd[0] * dx + gd[1] * dy + gd[2] * dz;
          const float gv3[3] = {(gd[0] - dx * dd) * inv, (gd[1] - dy * dd) * inv,
                                (gd[2] - dz * dd) * inv};
          g_mu[0] += gv3[0]; g_mu[1] += gv3[1]; g_mu[2] += gv3[2];
          // camera centre c = -A^{-1} b with gc = -gv3: dA = (A gv3) c^T, db = A gv3
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const float t = A[4 * r] * gv3[0] + A[4 * r + 1] * gv3[1] + A[4 * r + 2] * gv3[2];
            dA[3 * r] += t * M.c[0]; dA[3 * r + 1] += t * M.c[1]; dA[3 * r + 2] += t * M.c[2];
            db[r] += t;
          }
        }
      }

      if (DEG > 0 && k > 0) {
        float* dst = s_dM + (v * nk + k) * 12;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          atomicAdd(dst + 4 * r, dA[3 * r]);
          atomicAdd(dst + 4 * r + 1, dA[3 * r + 1]);
          atomicAdd(dst + 4 * r + 2, dA[3 * r + 2]);
          atomicAdd(dst + 4 * r + 3, db[r]);
        }
      }
    }
    if (a.g.means) {
      float* p = a.g.means + 3 * (size_t)gid;
      if (a.overwrite) {
        p[0] = g_mu[0]; p[1] = g_mu[1]; p[2] = g_mu[2];
      } else {
        p[0] += g_mu[0]; p[1] += g_mu[1]; p[2] += g_mu[2];
      }
    }
    }
    // SH adjoints: each lane writes its row over its (consumed) SH row, then
    // the warp adds the rows to the caller's buffer with coalesced accesses
    __syncwarp();
    if (kmask) {
#pragma unroll
      for (int i = 0; i < K * 3; ++i) row_sh[i] = g_sh[i];
    }
    __syncwarp();
    if (a.g.sh) {
      const uint32_t live = __ballot_sync(0xffffffffu, kmask != 0u);
      if constexpr (St::kVec) {
        float4* dst = reinterpret_cast<float4*>(a.g.sh);
        const float4* src = reinterpret_cast<const float4*>(my_sh);
#pragma unroll
        for (int it = 0; it < St::kRow; ++it) {
          const int idx = it * 32 + (int)lane;
          const int g = idx / St::kRow, qd = idx - g * St::kRow;
          const uint32_t gg = __shfl_sync(0xffffffffu, gid, g);
          if ((live >> g) & 1u) {
            const float4 d = src[g * St::kPitch + qd];
            if (a.overwrite) {
              dst[(size_t)gg * St::kRow + qd] = d;
            } else {
              float4 o = dst[(size_t)gg * St::kRow + qd];
              o.x += d.x; o.y += d.y; o.z += d.z; o.w += d.w;
              dst[(size_t)gg * St::kRow + qd] = o;
            }
          }
        }
      } else {
#pragma unroll
        for (int it = 0; it < St::kRow; ++it) {
          const int idx = it * 32 + (int)lane;
          const int g = idx / St::kRow, qd = idx - g * St::kRow;
          const uint32_t gg = __shfl_sync(0xffffffffu, gid, g);
          if ((live >> g) & 1u) {
            float* q = a.g.sh + (size_t)gg * St::kRow + qd;
            *q = a.overwrite ? my_sh[g * St::kPitch + qd] : *q + my_sh[g * St::kPitch + qd];
          }
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < vs.n_views * nk * 12; i += blockDim.x) {
    const int k = (i / 12) % nk;
    if (k > 0 && s_dM[i] != 0.f) atomicAdd(a.pose_dM + i, s_dM[i]);
  }
  // the last CTA to finish maps the summed matrix adjoints to the poses, then
  // clears the sums for the next call (they start at zero with the workspace)
  if (a.n_inst > 0) {
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.ctr + kCtrProjBwdExits, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (a.g.inst_quat || a.g.inst_trans)
        for (int k = 1 + (int)threadIdx.x; k <= a.n_inst; k += blockDim.x)
          pose_chain_one(vs, a.pose_dM, a.n_inst, k, a.pose_q, a.g.inst_quat, a.g.inst_trans,
                         a.overwrite);
      __syncthreads();
      for (int i = threadIdx.x; i < vs.n_views * nk * 12; i += blockDim.x) __stcg(a.pose_dM + i, 0.f);
      if (threadIdx.x == 0) a.ctr[kCtrProjBwdExits] = 0u;
    }
  }
}

template <int DEG>
cudaError_t launch_deg(s3r_workspace* ws, const BwdArgs& a, cudaStream_t st) {
  const int nk = ws->n_inst + 1;
  const size_t smem = sizeof(float) * kWarps * ShStage<DEG>::kWords +
                      (size_t)ws->n_views * nk * 12 * sizeof(float) + sizeof(uint32_t) * (nk + 1) + 16;
  static thread_local size_t cached_smem = 0;
  static thread_local int cached_per_sm = 0;
  if (smem != cached_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_project_bwd<DEG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project_bwd<DEG>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    cached_smem = smem;
    cached_per_sm = per_sm;
  }
  const int per_sm = cached_per_sm;
  KernelTimer timer(ws, kKProjectBwd, st);
  k_project_bwd<DEG><<<ws->num_sms * per_sm, kThreads, smem, st>>>(ws->views, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_project_bwd(s3r_workspace* ws, const s3r_scene* sc, const s3r_poses* poses,
                               const s3r_grads* g, cudaStream_t st) {
  BwdArgs a;
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
  a.selected = ws->selected;
  a.keep_mask = ws->keep_mask;
  a.kept_list = ws->kept_list;
  a.splat_start = ws->splat_start;
  a.sp_grad = reinterpret_cast<const float4*>(ws->sp_grad);
  a.sp_view = ws->sp_view;
  a.L.mode = ws->lod.mode;
  a.L.p_max = ws->lod.p_max;
  a.L.dist = ws->lod.distance;
  for (int i = 0; i < 3; ++i) a.L.off[i] = ws->lod.offset[i];
  a.L.key0 = (uint32_t)ws->lod.seed;
  a.L.key1 = (uint32_t)(ws->lod.seed >> 32);
  a.cap_splats = ws->cap.max_splats;
  a.ctr = ws->ctr;
  a.pose_dM = ws->pose_dM;
  a.g = *g;
  a.mats = reinterpret_cast<const InstMat*>(ws->mats);
  a.overwrite = ws->grad_mode == S3R_GRAD_OVERWRITE ? 1 : 0;
  cudaError_t e = cudaSuccess;
  switch (sc->sh_degree) {
    case 0: e = launch_deg<0>(ws, a, st); break;
    case 1: e = launch_deg<1>(ws, a, st); break;
    case 2: e = launch_deg<2>(ws, a, st); break;
    default: e = launch_deg<3>(ws, a, st); break;
  }
  return e;
}

}  // namespace s3r
