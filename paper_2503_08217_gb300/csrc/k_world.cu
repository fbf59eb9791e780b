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

constexpr int kWorldThreads = 256;
constexpr int kRotFloats = 9 + 25 + 49;      // D_1, D_2, D_3 row-major
constexpr int kWorldAcc = 9 + 3 + 4 + kRotFloats;   // dR, dt, dp, dD per instance
constexpr int kLocalInst = 4;                // instances whose matrices a CTA keeps in shared memory

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

// The matrices of the instances that a CTA's chunk of Gaussians touches
// (usually one), in shared memory: [kLocalInst][kRotFloats]; instances past
// kLocalInst compute theirs per Gaussian.
template <int DEG>
__device__ void chunk_rotations(const WorldArgs& a, int k0, int k1, float* s_D) {
  for (int k = k0 + (int)threadIdx.x; k <= k1 && k - k0 < kLocalInst; k += blockDim.x) {
    float R[9];
    quat_to_rot(a.pose_q[k - 1], R);
    sh_rotation<DEG>(R, s_D + (k - k0) * kRotFloats);
  }
}

template <int DEG>
__global__ void __launch_bounds__(kWorldThreads) k_to_world(WorldArgs a) {
  constexpr int K = sh_count(DEG);
  __shared__ float s_D[kLocalInst * kRotFloats];
  const int64_t first = a.inst_off[1];
  for (int64_t base = first + (int64_t)blockIdx.x * kWorldThreads; base < a.n;
       base += (int64_t)gridDim.x * kWorldThreads) {
    const int64_t g = base + threadIdx.x;
    const int k0 = segment_of_gid(a.inst_off, a.n_inst, base);
    const int k1 = segment_of_gid(a.inst_off, a.n_inst, min(a.n, base + kWorldThreads) - 1);
    if (DEG > 0 && a.sh_out) chunk_rotations<DEG>(a, k0, k1, s_D);
    __syncthreads();
    if (g < a.n) {
      const int k = segment_of_gid(a.inst_off, a.n_inst, g);
      const float4 qp = a.pose_q[k - 1];
      float R[9];
      quat_to_rot(qp, R);
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
      if (a.sh_out) {
        const float* c = a.sh + (size_t)K * 3 * g;
        float* o = a.sh_out + (size_t)K * 3 * g;
        for (int ch = 0; ch < 3; ++ch) o[ch] = c[ch];          // degree 0 is rotation invariant
        if (DEG > 0) {
          float Dl[kRotFloats];
          const float* D = s_D + (k - k0) * kRotFloats;
          if (k - k0 >= kLocalInst) {
            sh_rotation<DEG>(R, Dl);
            D = Dl;
          }
#pragma unroll
          for (int l = 1; l <= DEG; ++l) {
            const int nb = 2 * l + 1, b = band_start(l);
            for (int j = 0; j < nb; ++j)
              for (int ch = 0; ch < 3; ++ch) {
                float v = 0.f;
                for (int i = 0; i < nb; ++i) v = fmaf(D[rot_off(l) + i * nb + j], c[3 * (b + i) + ch], v);
                o[3 * (b + j) + ch] = v;
              }
          }
        }
      }
    }
    __syncthreads();
  }
}

// Adjoint of the world transform for the dynamic rows, in place. Per
// Gaussian: dmu = R^T dmu_w; dq from q_w = p (x) q^ (dq^ = p* (x) dq_w, then
// through the normalisation); dc_l = D_l dc'_l. Per instance (summed): dR
// from the means and dD_l = sum c_l dc'_l^T, dt = sum dmu_w, dp = sum dq_w (x) q^*.
template <int DEG>
__global__ void __launch_bounds__(kWorldThreads) k_to_world_bwd(WorldArgs a) {
  constexpr int K = sh_count(DEG);
  constexpr int kUsed = 16 + (DEG >= 1 ? 9 : 0) + (DEG >= 2 ? 25 : 0) + (DEG >= 3 ? 49 : 0);
  __shared__ float s_D[kLocalInst * kRotFloats];
  const int64_t first = a.inst_off[1];
  const uint32_t lane = threadIdx.x & 31u;
  for (int64_t base = first + (int64_t)blockIdx.x * kWorldThreads; base < a.n;
       base += (int64_t)gridDim.x * kWorldThreads) {
    const int64_t g = base + threadIdx.x;
    const int k0 = segment_of_gid(a.inst_off, a.n_inst, base);
    const int k1 = segment_of_gid(a.inst_off, a.n_inst, min(a.n, base + kWorldThreads) - 1);
    if (DEG > 0 && a.g_sh) chunk_rotations<DEG>(a, k0, k1, s_D);
    __syncthreads();
    // this Gaussian's terms of its instance's sums: dR (9), dt (3), dp (4), dD
    float t[kUsed];
#pragma unroll
    for (int i = 0; i < kUsed; ++i) t[i] = 0.f;
    const bool live = g < a.n;
    const int k = live ? segment_of_gid(a.inst_off, a.n_inst, g) : k1;
    if (live) {
      const float4 qp = a.pose_q[k - 1];
      float R[9];
      quat_to_rot(qp, R);
      if (a.g_means) {
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
          for (int c = 0; c < 3; ++c) t[3 * r + c] = dw[r] * m[c];
          t[9 + r] = dw[r];
        }
      }
      if (a.g_quats) {
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
      if (DEG > 0 && a.g_sh) {
        float* gs = a.g_sh + (size_t)K * 3 * g;
        const float* c = a.sh + (size_t)K * 3 * g;
        float Dl[kRotFloats];
        const float* D = s_D + (k - k0) * kRotFloats;
        if (k - k0 >= kLocalInst) {
          sh_rotation<DEG>(R, Dl);
          D = Dl;
        }
#pragma unroll
        for (int l = 1; l <= DEG; ++l) {
          const int nb = 2 * l + 1, b = band_start(l);
          float gw[7][3];
          for (int j = 0; j < nb; ++j)
            for (int ch = 0; ch < 3; ++ch) gw[j][ch] = gs[3 * (b + j) + ch];
          for (int i = 0; i < nb; ++i) {
            for (int j = 0; j < nb; ++j)
              t[16 + rot_off(l) + i * nb + j] =
                  c[3 * (b + i)] * gw[j][0] + c[3 * (b + i) + 1] * gw[j][1] + c[3 * (b + i) + 2] * gw[j][2];
            for (int ch = 0; ch < 3; ++ch) {
              float v = 0.f;
              for (int j = 0; j < nb; ++j) v = fmaf(D[rot_off(l) + i * nb + j], gw[j][ch], v);
              gs[3 * (b + i) + ch] = v;
            }
          }
        }
      }
    }
    // sums over the warp where all its lanes belong to one instance (the
    // common case: instances are contiguous runs of thousands), else per lane
    const int k_lane0 = __shfl_sync(0xffffffffu, k, 0);
    const bool uniform = __all_sync(0xffffffffu, k == k_lane0);
    float* acc = a.acc + (size_t)k * kWorldAcc;
#pragma unroll
    for (int i = 0; i < kUsed; ++i) {
      if (uniform) {
        float v = t[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.f) atomicAdd(acc + i, v);
      } else if (live && t[i] != 0.f) {
        atomicAdd(acc + i, t[i]);
      }
    }
    __syncthreads();
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
  int64_t blocks = (n_dynamic + kWorldThreads - 1) / kWorldThreads;
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  switch (sc->sh_degree) {
    case 0: k_to_world<0><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a); break;
    case 1: k_to_world<1><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a); break;
    case 2: k_to_world<2><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a); break;
    default: k_to_world<3><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a); break;
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
  int64_t blocks = (n_dynamic + kWorldThreads - 1) / kWorldThreads;
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  if (blocks < 1) blocks = 1;
  const unsigned pose_blocks = (unsigned)((sc->n_inst + 127) / 128);
  switch (sc->sh_degree) {
    case 0:
      k_to_world_bwd<0><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a);
      k_world_pose<0><<<pose_blocks, 128, 0, st>>>(a);
      break;
    case 1:
      k_to_world_bwd<1><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a);
      k_world_pose<1><<<pose_blocks, 128, 0, st>>>(a);
      break;
    case 2:
      k_to_world_bwd<2><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a);
      k_world_pose<2><<<pose_blocks, 128, 0, st>>>(a);
      break;
    default:
      k_to_world_bwd<3><<<(unsigned)blocks, kWorldThreads, 0, st>>>(a);
      k_world_pose<3><<<pose_blocks, 128, 0, st>>>(a);
      break;
  }
  return cudaGetLastError();
}

}  // namespace s3r
