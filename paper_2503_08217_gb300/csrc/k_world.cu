// The conventional pipeline of Fig. 1(a), the comparator that the
// instance-specific projection of Sec. 3.3 replaces: every step moves the
// Gaussians of each dynamic instance k to the world frame by the instance's
// pose (R_k = R(q_k/|q_k|), t_k):
//   mu_w = R_k mu + t_k,   q_w = (q_k/|q_k|) (x) (q/|q|)   (Hamilton product),
// and rotates their SH coefficients so that the world-frame view direction
// gives the colour the object-frame direction gives (band l: c'_l = D_l^T c_l
// with Y_l(R_k^T d) = D_l Y_l(d)); its backward maps the adjoints of the
// world-frame parameters back to the object frame and to the poses.
//
// D_l is the projection of the rotated basis on the basis,
//   (D_l)_ij = integral over the sphere of Y_li(R^T d) Y_lj(d) dd,
// evaluated exactly (the integrand is a polynomial of degree <= 6 on the
// sphere) with Lebedev's 26-point rule of degree 7: the 6 axis directions
// (weight 1/21), the 12 edge midpoints of the cube (weight 4/105) and its 8
// corners (weight 9/280), weights summing to 1, times 4 pi.
//
// Only the rows of dynamic Gaussians are read or written: static Gaussians
// do not move, so the caller copies their rows once. The backward works in
// place on the gradient buffers (the world-frame adjoints of the renderer's
// backward become the object-frame ones) and sums the pose terms per
// instance in the workspace before one thread per instance maps them to the
// pose quaternion and translation.
#include "s3r_math.cuh"

namespace s3r {
namespace {

constexpr int kWorldWarps = 2;
constexpr int kWorldThreads = 32 * kWorldWarps;   // Gaussians per chunk of a CTA
constexpr int kRotFloats = 9 + 25 + 49;      // D_1, D_2, D_3 row-major
constexpr int kWorldAcc = 9 + 3 + 4 + kRotFloats;   // dR, dt, dp, dD per instance
constexpr int kLocalInst = 4;                // instances whose matrices a CTA keeps in shared memory

// entries of D_1..D_deg
__host__ __device__ constexpr int rot_count(int deg) {
  return deg <= 0 ? 0 : (deg == 1 ? 9 : (deg == 2 ? 34 : 83));
}

__device__ __forceinline__ void lebedev26(int m, float d[3], float& w) {
  const float s2 = 0.70710678118654752f, s3 = 0.57735026918962576f;
  if (m < 6) {
    d[0] = d[1] = d[2] = 0.f;
    d[m >> 1] = (m & 1) ? -1.f : 1.f;
    w = 1.f / 21.f;
  } else if (m < 18) {
    const int e = m - 6, pair = e >> 2;            // axes (0,1), (0,2), (1,2)
    const int a = pair == 2 ? 1 : 0, b = pair == 0 ? 1 : 2;
    d[0] = d[1] = d[2] = 0.f;
    d[a] = (e & 1) ? -s2 : s2;
    d[b] = (e & 2) ? -s2 : s2;
    w = 4.f / 105.f;
  } else {
    const int e = m - 18;
    d[0] = (e & 1) ? -s3 : s3;
    d[1] = (e & 2) ? -s3 : s3;
    d[2] = (e & 4) ? -s3 : s3;
    w = 9.f / 280.f;
  }
}

// first basis function of band l, and the offset of D_l in the packed matrices
__host__ __device__ constexpr int band_start(int l) { return l * l; }
__host__ __device__ constexpr int rot_off(int l) { return l <= 1 ? 0 : (l == 2 ? 9 : 34); }

// D_1..D_3 of rotation R into D (kRotFloats), for bands 1..deg.
template <int DEG>
__device__ void sh_rotation(const float R[9], float* D) {
  for (int i = 0; i < kRotFloats; ++i) D[i] = 0.f;
  for (int m = 0; m < 26; ++m) {
    float d[3], w;
    lebedev26(m, d, w);
    const float u[3] = {R[0] * d[0] + R[3] * d[1] + R[6] * d[2], R[1] * d[0] + R[4] * d[1] + R[7] * d[2],
                        R[2] * d[0] + R[5] * d[1] + R[8] * d[2]};   // R^T d
    float Yu[16], Yd[16];
    sh_basis<DEG>(u[0], u[1], u[2], Yu);
    sh_basis<DEG>(d[0], d[1], d[2], Yd);
    const float s = 12.566370614359172f * w;
#pragma unroll
    for (int l = 1; l <= DEG; ++l) {
      const int n = 2 * l + 1, b = band_start(l);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) D[rot_off(l) + i * n + j] = fmaf(s * Yu[b + i], Yd[b + j], D[rot_off(l) + i * n + j]);
    }
  }
}

__device__ __forceinline__ int segment_of_gid(const int64_t* __restrict__ off, int n_inst, int64_t g) {
  int lo = 0, hi = n_inst + 1;   // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

struct WorldArgs {
  int64_t n;
  const float* means;
  const float4* quats;
  const float* sh;
  const int64_t* inst_off;
  int n_inst;
  const float4* pose_q;
  const float* pose_t;
  float* means_out;
  float4* quats_out;
  float* sh_out;        // null: SH not rotated
  // backward
  float* g_means;
  float4* g_quats;
  float* g_sh;
  float* acc;           // [n_inst + 1][kWorldAcc]
  float* g_pose_q;
  float* g_pose_t;
};

// The SH basis at the 26 Lebedev points, [26][16] (once per CTA).
template <int DEG>
__device__ void lebedev_basis(float* s_Yd) {
  constexpr int K = sh_count(DEG);
  for (int m = threadIdx.x; m < 26; m += blockDim.x) {
    float d[3], w, Y[16];
    lebedev26(m, d, w);
    sh_basis<DEG>(d[0], d[1], d[2], Y);
    for (int i = 0; i < K; ++i) s_Yd[m * 16 + i] = Y[i];
  }
}

// D_1..D_DEG of the instances k0 .. min(k1, k0 + kLocalInst - 1) that a
// chunk of Gaussians touches (usually one), into s_D [kLocalInst][kRotFloats]:
// first 4 pi w_m Y(R^T d_m) at the 26 points (one thread per point and
// instance), then one thread per matrix entry for its 26-term sum (the
// quadrature in the order of sh_rotation). Instances past kLocalInst compute
// theirs per Gaussian. Synchronises the CTA before returning.
template <int DEG>
__device__ void chunk_rotations(const WorldArgs& a, int k0, int k1, const float* s_Yd, float* s_Yu,
                                float* s_D) {
  constexpr int K = sh_count(DEG), E = rot_count(DEG);
  const int ns = min(k1 - k0 + 1, kLocalInst);
  for (int e = threadIdx.x; e < ns * 26; e += blockDim.x) {
    const int sl = e / 26, m = e - sl * 26;
    float R[9], d[3], w, Y[16];
    quat_to_rot(a.pose_q[k0 + sl - 1], R);
    lebedev26(m, d, w);
    sh_basis<DEG>(R[0] * d[0] + R[3] * d[1] + R[6] * d[2], R[1] * d[0] + R[4] * d[1] + R[7] * d[2],
                  R[2] * d[0] + R[5] * d[1] + R[8] * d[2], Y);
    const float sw = 12.566370614359172f * w;
    for (int i = 0; i < K; ++i) s_Yu[e * 16 + i] = sw * Y[i];
  }
  __syncthreads();
  constexpr int kE = E > 0 ? E : 1;   // degree 0 has no rotation entries (the loop runs 0 times)
  for (int e = threadIdx.x; e < ns * E; e += blockDim.x) {
    const int sl = e / kE, r = e - sl * kE;
    const int l = r < 9 ? 1 : (r < 34 ? 2 : 3);
    const int nb = 2 * l + 1, idx = r - rot_off(l), i = idx / nb, j = idx - i * nb, b = band_start(l);
    float acc = 0.f;
    for (int m = 0; m < 26; ++m) acc = fmaf(s_Yu[(sl * 26 + m) * 16 + b + i], s_Yd[m * 16 + b + j], acc);
    s_D[sl * kRotFloats + r] = acc;
  }
  __syncthreads();
}

// A lane's own staged SH row (kFloatPitch floats from `row`) to and from
// registers: as float4s where the rows are (conflict-free across a quarter
// warp with the odd float4 pitch), else as floats.
template <int DEG>
__device__ __forceinline__ void row_get(const float* row, float (&c)[3 * sh_count(DEG)]) {
  using St = ShStage<DEG>;
  if constexpr (St::kVec) {
#pragma unroll
    for (int q = 0; q < St::kRow; ++q) {
      const float4 v = reinterpret_cast<const float4*>(row)[q];
      c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 3 * sh_count(DEG); ++q) c[q] = row[q];
  }
}
template <int DEG>
__device__ __forceinline__ void row_put(float* row, const float (&c)[3 * sh_count(DEG)]) {
  using St = ShStage<DEG>;
  if constexpr (St::kVec) {
#pragma unroll
    for (int q = 0; q < St::kRow; ++q)
      reinterpret_cast<float4*>(row)[q] = make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < 3 * sh_count(DEG); ++q) row[q] = c[q];
  }
}

// Coalesced copy of n_here staged rows to the consecutive rows g0.. of `sh`
// (the inverse of stage_sh_rows for consecutive Gaussians).
template <int DEG>
__device__ __forceinline__ void unstage_sh_rows(float* __restrict__ sh, const float* stage, int64_t g0,
                                                int n_here, uint32_t lane) {
  using St = ShStage<DEG>;
  if constexpr (St::kVec) {
    float4* dst = reinterpret_cast<float4*>(sh) + g0 * St::kRow;
    const float4* src = reinterpret_cast<const float4*>(stage);
    for (int idx = (int)lane; idx < n_here * St::kRow; idx += 32) {
      const int g = idx / St::kRow, q = idx - g * St::kRow;
      dst[idx] = src[g * St::kPitch + q];
    }
  } else {
    float* dst = sh + g0 * St::kRow;
    for (int idx = (int)lane; idx < n_here * St::kRow; idx += 32) {
      const int g = idx / St::kRow, q = idx - g * St::kRow;
      dst[idx] = stage[g * St::kPitch + q];
    }
  }
}

// The CTA's contiguous range of 64-Gaussian chunks of the dynamic rows, so
// that consecutive chunks mostly share their instance's matrices.
struct ChunkRange {
  int64_t first, begin, end;
};
__device__ __forceinline__ ChunkRange chunk_range(const WorldArgs& a) {
  ChunkRange r;
  r.first = a.inst_off[1];
  const int64_t n_chunks = (a.n - r.first + kWorldThreads - 1) / kWorldThreads;
  const int64_t per = (n_chunks + gridDim.x - 1) / gridDim.x;
  r.begin = (int64_t)blockIdx.x * per;
  r.end = min(n_chunks, r.begin + per);
  return r;
}

template <int DEG>
__global__ void __launch_bounds__(kWorldThreads) k_to_world(WorldArgs a) {
  using St = ShStage<DEG>;
  constexpr int K = sh_count(DEG);
  __shared__ float s_D[kLocalInst * kRotFloats];
  __shared__ float s_Yd[26 * 16];
  __shared__ float s_Yu[kLocalInst * 26 * 16];
  __shared__ __align__(16) float s_rows[kWorldWarps * St::kWords];
  const ChunkRange cr = chunk_range(a);
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  float* rows = s_rows + warp * St::kWords;
  const bool rotate = DEG > 0 && a.sh_out;
  if (rotate) lebedev_basis<DEG>(s_Yd);   // read after chunk_rotations' first barrier
  int kc0 = -1, kc1 = -1;
  for (int64_t c = cr.begin; c < cr.end; ++c) {
    const int64_t base = cr.first + c * kWorldThreads;
    const int64_t g = base + threadIdx.x;
    const int k0 = segment_of_gid(a.inst_off, a.n_inst, base);
    const int k1 = segment_of_gid(a.inst_off, a.n_inst, min(a.n, base + kWorldThreads) - 1);
    if (rotate && (k0 != kc0 || k1 != kc1)) {   // block-uniform
      __syncthreads();   // the previous chunk's reads of s_D are done
      chunk_rotations<DEG>(a, k0, k1, s_Yd, s_Yu, s_D);
      kc0 = k0;
      kc1 = k1;
    }
    const bool live = g < a.n;
    const int k = live ? segment_of_gid(a.inst_off, a.n_inst, g) : k0;
    const float4 qp = a.pose_q[k - 1];
    float R[9];
    quat_to_rot(qp, R);
    if (live) {
      const float* t = a.pose_t + 3 * (k - 1);
      const float m0 = a.means[3 * g], m1 = a.means[3 * g + 1], m2 = a.means[3 * g + 2];
      a.means_out[3 * g] = fmaf(R[0], m0, fmaf(R[1], m1, fmaf(R[2], m2, t[0])));
      a.means_out[3 * g + 1] = fmaf(R[3], m0, fmaf(R[4], m1, fmaf(R[5], m2, t[1])));
      a.means_out[3 * g + 2] = fmaf(R[6], m0, fmaf(R[7], m1, fmaf(R[8], m2, t[2])));
      const float4 q = a.quats[g];
      const float iq = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const float w2 = q.x * iq, x2 = q.y * iq, y2 = q.z * iq, z2 = q.w * iq;
      const float ip = rsqrtf(qp.x * qp.x + qp.y * qp.y + qp.z * qp.z + qp.w * qp.w);
      const float w1 = qp.x * ip, x1 = qp.y * ip, y1 = qp.z * ip, z1 = qp.w * ip;
      a.quats_out[g] = make_float4(w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                                   w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                                   w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                                   w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2);
    }
    if (a.sh_out) {
      // the warp's rows through shared memory: coalesced in, rotated per
      // lane, coalesced out (c'_l = D_l^T c_l per channel; degree 0 as is)
      const int64_t wbase = base + warp * 32;
      const int n_here = (int)max((int64_t)0, min((int64_t)32, a.n - wbase));
      if (n_here > 0) {
        stage_sh_rows<DEG>(rows, a.sh, (uint32_t)(wbase + lane), n_here, lane);
        __syncwarp();
        if (DEG > 0 && live) {
          float cr_[3 * K], o[3 * K];
          float* row = rows + lane * St::kFloatPitch;
          row_get<DEG>(row, cr_);
          float Dl[kRotFloats];
          const float* D = s_D + (k - k0) * kRotFloats;
          if (k - k0 >= kLocalInst) {
            sh_rotation<DEG>(R, Dl);
            D = Dl;
          }
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) o[ch] = cr_[ch];
#pragma unroll
          for (int l = 1; l <= DEG; ++l) {
            const int nb = 2 * l + 1, b = band_start(l);
#pragma unroll
            for (int j = 0; j < nb; ++j)
#pragma unroll
              for (int ch = 0; ch < 3; ++ch) {
                float v = 0.f;
#pragma unroll
                for (int i = 0; i < nb; ++i) v = fmaf(D[rot_off(l) + i * nb + j], cr_[3 * (b + i) + ch], v);
                o[3 * (b + j) + ch] = v;
              }
          }
          row_put<DEG>(row, o);
        }
        __syncwarp();
        unstage_sh_rows<DEG>(a.sh_out, rows, wbase, n_here, lane);
        __syncwarp();   // the rows are restaged by the next chunk
      }
    }
  }
}

// Adjoint of the world transform for the dynamic rows, in place. Per
// Gaussian: dmu = R^T dmu_w; dq from q_w = p (x) q^ (dq^ = p* (x) dq_w, then
// through the normalisation); dc_l = D_l dc'_l. Per instance (summed): dR
// from the means and dD_l = sum c_l dc'_l^T, dt = sum dmu_w, dp = sum dq_w (x) q^*.
// The SH rows of the parameters and of the adjoints go through shared memory
// (coalesced); a warp's dD sums are taken over its staged rows, one matrix
// entry per lane, before one atomic per entry and instance.
template <int DEG>
__global__ void __launch_bounds__(kWorldThreads) k_to_world_bwd(WorldArgs a) {
  using St = ShStage<DEG>;
  constexpr int K = sh_count(DEG), E = rot_count(DEG);
  __shared__ float s_D[kLocalInst * kRotFloats];
  __shared__ float s_Yd[26 * 16];
  __shared__ float s_Yu[kLocalInst * 26 * 16];
  __shared__ __align__(16) float s_c[kWorldWarps * St::kWords];
  __shared__ __align__(16) float s_g[kWorldWarps * St::kWords];
  __shared__ float s_t[kWorldWarps][32][17];
  __shared__ int s_k[kWorldWarps][32];
  const ChunkRange cr = chunk_range(a);
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  float* crow = s_c + warp * St::kWords;
  float* grow = s_g + warp * St::kWords;
  const bool rotate = DEG > 0 && a.g_sh;
  if (rotate) lebedev_basis<DEG>(s_Yd);
  int kc0 = -1, kc1 = -1;
  for (int64_t c = cr.begin; c < cr.end; ++c) {
    const int64_t base = cr.first + c * kWorldThreads;
    const int64_t g = base + threadIdx.x;
    const int k0 = segment_of_gid(a.inst_off, a.n_inst, base);
    const int k1 = segment_of_gid(a.inst_off, a.n_inst, min(a.n, base + kWorldThreads) - 1);
    if (rotate && (k0 != kc0 || k1 != kc1)) {
      __syncthreads();
      chunk_rotations<DEG>(a, k0, k1, s_Yd, s_Yu, s_D);
      kc0 = k0;
      kc1 = k1;
    }
    // this Gaussian's terms of its instance's sums: dR (9), dt (3), dp (4)
    float t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = 0.f;
    const bool live = g < a.n;
    const int k = live ? segment_of_gid(a.inst_off, a.n_inst, g) : -1;
    const float4 qp = a.pose_q[(live ? k : k0) - 1];
    float R[9];
    quat_to_rot(qp, R);
    if (live && a.g_means) {
      float* gm = a.g_means + 3 * g;
      const float d0 = gm[0], d1 = gm[1], d2 = gm[2];
      const float m[3] = {a.means[3 * g], a.means[3 * g + 1], a.means[3 * g + 2]};
      gm[0] = R[0] * d0 + R[3] * d1 + R[6] * d2;
      gm[1] = R[1] * d0 + R[4] * d1 + R[7] * d2;
      gm[2] = R[2] * d0 + R[5] * d1 + R[8] * d2;
      const float dw[3] = {d0, d1, d2};
#pragma unroll
      for (int r = 0; r < 3; ++r) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) t[3 * r + cc] = dw[r] * m[cc];
        t[9 + r] = dw[r];
      }
    }
    if (live && a.g_quats) {
      const float4 q = a.quats[g];
      const float nq = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
      const float qw = q.x / nq, qx = q.y / nq, qy = q.z / nq, qz = q.w / nq;
      const float np = sqrtf(qp.x * qp.x + qp.y * qp.y + qp.z * qp.z + qp.w * qp.w);
      const float pw = qp.x / np, px = qp.y / np, py = qp.z / np, pz = qp.w / np;
      const float4 G = a.g_quats[g];
      // dq^ = p* (x) G, then through the normalisation of q
      const float aw = pw * G.x + px * G.y + py * G.z + pz * G.w;
      const float ax = pw * G.y - px * G.x - py * G.w + pz * G.z;
      const float ay = pw * G.z + px * G.w - py * G.x - pz * G.y;
      const float az = pw * G.w - px * G.z + py * G.y - pz * G.x;
      const float dot = aw * qw + ax * qx + ay * qy + az * qz;
      a.g_quats[g] = make_float4((aw - qw * dot) / nq, (ax - qx * dot) / nq, (ay - qy * dot) / nq,
                                 (az - qz * dot) / nq);
      // dp^ = G (x) q^*
      t[12] = G.x * qw + G.y * qx + G.z * qy + G.w * qz;
      t[13] = -G.x * qx + G.y * qw - G.z * qz + G.w * qy;
      t[14] = -G.x * qy + G.y * qz + G.z * qw - G.w * qx;
      t[15] = -G.x * qz - G.y * qy + G.z * qx + G.w * qw;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) s_t[warp][lane][i] = t[i];
    s_k[warp][lane] = k;
    const int64_t wbase = base + warp * 32;
    const int n_here = (int)max((int64_t)0, min((int64_t)32, a.n - wbase));
    __syncwarp();
    if (n_here > 0) {   // warp-uniform
      const int k_lo = s_k[warp][0], k_hi = s_k[warp][n_here - 1];
      if (rotate) {
        stage_sh_rows<DEG>(crow, a.sh, (uint32_t)(wbase + lane), n_here, lane);
        stage_sh_rows<DEG>(grow, a.g_sh, (uint32_t)(wbase + lane), n_here, lane);
        __syncwarp();
        // dD_l[i][j] = sum over the instance's Gaussians and channels of c_{b+i} dc'_{b+j}
        for (int kk = k_lo; kk <= k_hi; ++kk) {
          for (int e = (int)lane; e < E; e += 32) {
            const int l = e < 9 ? 1 : (e < 34 ? 2 : 3);
            const int nb = 2 * l + 1, idx = e - rot_off(l), i = idx / nb, j = idx - i * nb;
            const int ci = 3 * (band_start(l) + i), cj = 3 * (band_start(l) + j);
            float acc = 0.f;
            for (int g2 = 0; g2 < n_here; ++g2) {
              if (s_k[warp][g2] != kk) continue;
              const float* cg = crow + g2 * St::kFloatPitch;
              const float* gg = grow + g2 * St::kFloatPitch;
              acc = fmaf(cg[ci], gg[cj], fmaf(cg[ci + 1], gg[cj + 1], fmaf(cg[ci + 2], gg[cj + 2], acc)));
            }
            if (acc != 0.f) atomicAdd(a.acc + (size_t)kk * kWorldAcc + 16 + e, acc);
          }
        }
        __syncwarp();
        if (live) {
          float gw[3 * K], o[3 * K];
          float* row = grow + lane * St::kFloatPitch;
          row_get<DEG>(row, gw);
          float Dl[kRotFloats];
          const float* D = s_D + (k - k0) * kRotFloats;
          if (k - k0 >= kLocalInst) {
            sh_rotation<DEG>(R, Dl);
            D = Dl;
          }
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) o[ch] = gw[ch];
#pragma unroll
          for (int l = 1; l <= DEG; ++l) {
            const int nb = 2 * l + 1, b = band_start(l);
#pragma unroll
            for (int i = 0; i < nb; ++i)
#pragma unroll
              for (int ch = 0; ch < 3; ++ch) {
                float v = 0.f;
#pragma unroll
                for (int j = 0; j < nb; ++j) v = fmaf(D[rot_off(l) + i * nb + j], gw[3 * (b + j) + ch], v);
                o[3 * (b + i) + ch] = v;
              }
          }
          row_put<DEG>(row, o);
        }
        __syncwarp();
        unstage_sh_rows<DEG>(a.g_sh, grow, wbase, n_here, lane);
      }
      // dR, dt, dp: one lane per term, summed over the warp's Gaussians of each instance
      for (int kk = k_lo; kk <= k_hi; ++kk) {
        if (lane < 16) {
          float v = 0.f;
          for (int g2 = 0; g2 < n_here; ++g2)
            if (s_k[warp][g2] == kk) v += s_t[warp][g2][lane];
          if (v != 0.f) atomicAdd(a.acc + (size_t)kk * kWorldAcc + lane, v);
        }
      }
    }
    __syncwarp();   // s_t, s_k and the staged rows are rewritten by the next chunk
  }
}

// Per instance: the pose adjoints from the sums (written), then the sums cleared.
template <int DEG>
__global__ void k_world_pose(WorldArgs a) {
  const int k = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (k > a.n_inst) return;
  float* acc = a.acc + (size_t)k * kWorldAcc;
  float dR[9];
  for (int i = 0; i < 9; ++i) dR[i] = acc[i];
  const float4 qp = a.pose_q[k - 1];
  if (DEG > 0) {
    // dD -> dR through D_ij = 4 pi sum_m w_m Y_i(R^T d_m) Y_j(d_m): with
    // u_m = R^T d_m, dL/du_m = 4 pi w_m grad(sum_i W_i Y_i)(u_m), W_i = sum_j dD_ij Y_j(d_m)
    float R[9];
    quat_to_rot(qp, R);
    for (int m = 0; m < 26; ++m) {
      float d[3], w;
      lebedev26(m, d, w);
      const float u[3] = {R[0] * d[0] + R[3] * d[1] + R[6] * d[2],
                          R[1] * d[0] + R[4] * d[1] + R[7] * d[2],
                          R[2] * d[0] + R[5] * d[1] + R[8] * d[2]};
      float Yd[16], W[16];
      sh_basis<DEG>(d[0], d[1], d[2], Yd);
      W[0] = 0.f;
      for (int l = 1; l <= DEG; ++l) {
        const int nb = 2 * l + 1, b = band_start(l);
        for (int i = 0; i < nb; ++i) {
          float v = 0.f;
          for (int j = 0; j < nb; ++j) v = fmaf(acc[16 + rot_off(l) + i * nb + j], Yd[b + j], v);
          W[b + i] = v;
        }
      }
      for (int i = sh_count(DEG); i < 16; ++i) W[i] = 0.f;
      float gu[3];
      sh_dir_grad<DEG>(u[0], u[1], u[2], W, gu);
      const float s = 12.566370614359172f * w;
      // u_a = sum_b R_ba d_b
      for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) dR[3 * b + c] = fmaf(s * gu[c], d[b], dR[3 * b + c]);
    }
  }
  float4 gq = quat_backward(qp, dR);
  const float np = sqrtf(qp.x * qp.x + qp.y * qp.y + qp.z * qp.z + qp.w * qp.w);
  const float pw = qp.x / np, px = qp.y / np, py = qp.z / np, pz = qp.w / np;
  const float dp[4] = {acc[12], acc[13], acc[14], acc[15]};
  const float dot = dp[0] * pw + dp[1] * px + dp[2] * py + dp[3] * pz;
  gq.x += (dp[0] - pw * dot) / np;
  gq.y += (dp[1] - px * dot) / np;
  gq.z += (dp[2] - py * dot) / np;
  gq.w += (dp[3] - pz * dot) / np;
  if (a.g_pose_q) {
    float* o = a.g_pose_q + 4 * (k - 1);
    o[0] = gq.x; o[1] = gq.y; o[2] = gq.z; o[3] = gq.w;
  }
  if (a.g_pose_t) {
    float* o = a.g_pose_t + 3 * (k - 1);
    o[0] = acc[9]; o[1] = acc[10]; o[2] = acc[11];
  }
  for (int i = 0; i < kWorldAcc; ++i) acc[i] = 0.f;
}

}  // namespace

int world_acc_floats() { return kWorldAcc; }

namespace {
// CTAs of a world-transform launch: one resident wave (each CTA takes a
// contiguous range of chunks), fewer for a small scene. The occupancy of each
// kernel is queried once.
int64_t world_grid(const void* fn, int* cache, int64_t n_rows, int num_sms) {
  if (*cache == 0 &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(cache, fn, kWorldThreads, 0) != cudaSuccess || *cache < 1))
    *cache = 1;
  int64_t blocks = (n_rows + kWorldThreads - 1) / kWorldThreads;
  if (blocks > (int64_t)num_sms * *cache) blocks = (int64_t)num_sms * *cache;
  return blocks < 1 ? 1 : blocks;
}
}  // namespace

cudaError_t launch_to_world(const s3r_scene* sc, const s3r_poses* poses, float* means_out,
                            float* quats_out, float* sh_out, int64_t n_dynamic, int num_sms,
                            cudaStream_t st) {
  if (n_dynamic <= 0) return cudaSuccess;
  WorldArgs a = {};
  a.n = sc->n;
  a.means = sc->means;
  a.quats = reinterpret_cast<const float4*>(sc->quats);
  a.sh = sc->sh;
  a.inst_off = sc->inst_offsets;
  a.n_inst = sc->n_inst;
  a.pose_q = reinterpret_cast<const float4*>(poses->quat);
  a.pose_t = poses->trans;
  a.means_out = means_out;
  a.quats_out = reinterpret_cast<float4*>(quats_out);
  a.sh_out = sh_out;
  static thread_local int occ[4] = {0, 0, 0, 0};
  switch (sc->sh_degree) {
    case 0:
      k_to_world<0><<<(unsigned)world_grid((const void*)k_to_world<0>, &occ[0], n_dynamic, num_sms),
                      kWorldThreads, 0, st>>>(a);
      break;
    case 1:
      k_to_world<1><<<(unsigned)world_grid((const void*)k_to_world<1>, &occ[1], n_dynamic, num_sms),
                      kWorldThreads, 0, st>>>(a);
      break;
    case 2:
      k_to_world<2><<<(unsigned)world_grid((const void*)k_to_world<2>, &occ[2], n_dynamic, num_sms),
                      kWorldThreads, 0, st>>>(a);
      break;
    default:
      k_to_world<3><<<(unsigned)world_grid((const void*)k_to_world<3>, &occ[3], n_dynamic, num_sms),
                      kWorldThreads, 0, st>>>(a);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_world_bwd(const s3r_scene* sc, const s3r_poses* poses, const s3r_grads* g,
                                float* acc, int64_t n_dynamic, int num_sms, cudaStream_t st) {
  if (sc->n_inst <= 0) return cudaSuccess;
  WorldArgs a = {};
  a.n = sc->n;
  a.means = sc->means;
  a.quats = reinterpret_cast<const float4*>(sc->quats);
  a.sh = sc->sh;
  a.inst_off = sc->inst_offsets;
  a.n_inst = sc->n_inst;
  a.pose_q = reinterpret_cast<const float4*>(poses->quat);
  a.pose_t = poses->trans;
  a.g_means = g->means;
  a.g_quats = reinterpret_cast<float4*>(g->quats);
  a.g_sh = g->sh;
  a.acc = acc;
  a.g_pose_q = g->inst_quat;
  a.g_pose_t = g->inst_trans;
  const unsigned pose_blocks = (unsigned)((sc->n_inst + 127) / 128);
  static thread_local int occ[4] = {0, 0, 0, 0};
  switch (sc->sh_degree) {
    case 0:
      k_to_world_bwd<0><<<(unsigned)world_grid((const void*)k_to_world_bwd<0>, &occ[0], n_dynamic, num_sms),
                          kWorldThreads, 0, st>>>(a);
      k_world_pose<0><<<pose_blocks, 128, 0, st>>>(a);
      break;
    case 1:
      k_to_world_bwd<1><<<(unsigned)world_grid((const void*)k_to_world_bwd<1>, &occ[1], n_dynamic, num_sms),
                          kWorldThreads, 0, st>>>(a);
      k_world_pose<1><<<pose_blocks, 128, 0, st>>>(a);
      break;
    case 2:
      k_to_world_bwd<2><<<(unsigned)world_grid((const void*)k_to_world_bwd<2>, &occ[2], n_dynamic, num_sms),
                          kWorldThreads, 0, st>>>(a);
      k_world_pose<2><<<pose_blocks, 128, 0, st>>>(a);
      break;
    default:
      k_to_world_bwd<3><<<(unsigned)world_grid((const void*)k_to_world_bwd<3>, &occ[3], n_dynamic, num_sms),
                          kWorldThreads, 0, st>>>(a);
      k_world_pose<3><<<pose_blocks, 128, 0, st>>>(a);
      break;
  }
  return cudaGetLastError();
}

}  // namespace s3r
