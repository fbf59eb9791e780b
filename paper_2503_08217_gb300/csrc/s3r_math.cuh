// FP32 device math of the instance-specific projection (Sec. 3.3 with Eq. 1)
// and of the SH colour, shared by the forward and backward projection
// kernels of libs3r.
#pragma once

#include "s3r_internal.cuh"

namespace s3r {

// Composed instance matrix W_{t,i} = W_t W_{t,i2g} (3x4, row-major, rows
// [A | b]) and the camera centre in the instance's frame, c = -A^{-1} b, as an
// unevaluated sum c_hi + c_lo of two floats. Both are computed in FP64 once per
// call (by the compaction's first CTAs). Camera-space positions are evaluated as
// A ((mu - c_hi) - c_lo): for Gaussians near the camera mu - c_hi is exact
// (Sterbenz), so positions far from the world origin do not lose their
// camera-relative precision the way A mu + b does.
struct __align__(16) InstMat {
  float m[12];
  float c[3];     // c_hi
  float c_lo[3];
  float a_frob2;  // squared Frobenius norm of A (bounds the splat radius, see may_touch_view)
  float pad;
};

// Single-instruction approximations (hardware reciprocal and square root,
// within a few ulp): the projection's decisions that they could move
// (near plane, rectangle edges, radius ceiling, LOD threshold) are compared
// with margins far wider than that, and the forward, the splat writer and the
// backward all call these same functions.
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_fast(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kDilation = 0.3f;
constexpr float kMinEig = 0.1f;

// Rotation of the unit quaternion q/|q| (w, x, y, z), row-major.
__device__ __forceinline__ void quat_to_rot(float4 q, float R[9]) {
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  const float xx = x * x, yy = y * y, zz = z * z;
  const float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
  R[0] = 1.f - 2.f * (yy + zz); R[1] = 2.f * (xy - wz); R[2] = 2.f * (xz + wy);
  R[3] = 2.f * (xy + wz); R[4] = 1.f - 2.f * (xx + zz); R[5] = 2.f * (yz - wx);
  R[6] = 2.f * (xz - wy); R[7] = 2.f * (yz + wx); R[8] = 1.f - 2.f * (xx + yy);
}

// Camera-relative position d = (mu - c_hi) - c_lo in the instance frame.
__device__ __forceinline__ void rel_pos(const InstMat& M, const float mu[3], float d[3]) {
  d[0] = (mu[0] - M.c[0]) - M.c_lo[0];
  d[1] = (mu[1] - M.c[1]) - M.c_lo[1];
  d[2] = (mu[2] - M.c[2]) - M.c_lo[2];
}

// Camera-space position p = A d.
__device__ __forceinline__ void cam_pos(const InstMat& M, const float d[3], float& x, float& y,
                                        float& z) {
  x = fmaf(M.m[0], d[0], fmaf(M.m[1], d[1], M.m[2] * d[2]));
  y = fmaf(M.m[4], d[0], fmaf(M.m[5], d[1], M.m[6] * d[2]));
  z = fmaf(M.m[8], d[0], fmaf(M.m[9], d[1], M.m[10] * d[2]));
}

// Segment (0 = static, k = instance k) of Gaussian `gid` from the offsets.
__device__ __forceinline__ int segment_of(const uint32_t* off, int n_inst, uint32_t gid) {
  int lo = 0, hi = n_inst + 1;  // off[lo] <= gid < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= gid) lo = mid; else hi = mid;
  }
  return lo;
}

// Result of projecting one Gaussian into one view.
struct Proj2D {
  float x, y, z;        // camera-space position
  float u, v;           // pixel position
  float ca, cb, cc;     // conic: power = -0.5 (ca dx^2 + cc dy^2) - cb dx dy
  float sigma;          // sqrt(largest eigenvalue) before dilation (LOD scale)
  float radius;
  int x0, y0, x1, y1;   // tile rectangle, half-open
  bool infrustum;
};

// Project a Gaussian with local mean mu and RS = R(q) diag(s) through the
// composed matrix M. Follows Eq. 1 with the 3DGS conventions: near plane,
// the 1.3x field-of-view clamp of the Jacobian, 0.3 px^2 dilation, 3-sigma
// radius and a 16x16-tile bounding rectangle.
__device__ __forceinline__ Proj2D project_view(const InstMat& M, const float mu[3],
                                               const float RS[9], const ViewInfo& vi) {
  Proj2D o;
  o.infrustum = false;
  o.u = o.v = o.ca = o.cb = o.cc = o.sigma = o.radius = 0.f;
  o.x0 = o.y0 = o.x1 = o.y1 = 0;
  float d[3];
  rel_pos(M, mu, d);
  cam_pos(M, d, o.x, o.y, o.z);
  if (!(o.z > vi.near_z)) return o;
  // B = A * RS (A = rotation part of M): camera-space covariance is B B^T
  float B[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      B[3 * r + c] = fmaf(M.m[4 * r], RS[c], fmaf(M.m[4 * r + 1], RS[3 + c], M.m[4 * r + 2] * RS[6 + c]));
  const float iz = rcp_fast(o.z);
  const float rx = o.x * iz, ry = o.y * iz;
  const float txr = fminf(vi.limx, fmaxf(-vi.limx, rx));
  const float tyr = fminf(vi.limy, fmaxf(-vi.limy, ry));
  const float j00 = vi.fx * iz, j02 = -vi.fx * txr * iz;
  const float j11 = vi.fy * iz, j12 = -vi.fy * tyr * iz;
  // C = J B (2x3); Sigma2 = C C^T
  float C0[3], C1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C0[c] = fmaf(j00, B[c], j02 * B[6 + c]);
    C1[c] = fmaf(j11, B[3 + c], j12 * B[6 + c]);
  }
  const float a = fmaf(C0[0], C0[0], fmaf(C0[1], C0[1], C0[2] * C0[2]));
  const float b = fmaf(C0[0], C1[0], fmaf(C0[1], C1[1], C0[2] * C1[2]));
  const float c = fmaf(C1[0], C1[0], fmaf(C1[1], C1[1], C1[2] * C1[2]));
  const float mid0 = 0.5f * (a + c);
  const float det0 = a * c - b * b;
  o.sigma = sqrt_fast(mid0 + sqrt_fast(fmaxf(0.f, mid0 * mid0 - det0)));
  const float ad = a + kDilation, cd = c + kDilation;
  const float det = ad * cd - b * b;
  if (!(det > 0.f)) return o;
  const float idet = rcp_fast(det);
  o.ca = cd * idet;
  o.cb = -b * idet;
  o.cc = ad * idet;
  const float mid = 0.5f * (ad + cd);
  const float lam = mid + sqrt_fast(fmaxf(kMinEig, mid * mid - det));
  o.radius = ceilf(3.f * sqrt_fast(lam));
  o.u = fmaf(vi.fx, rx, vi.cx);
  o.v = fmaf(vi.fy, ry, vi.cy);
  const float inv_tile = 1.f / kTile;
  o.x0 = (int)fminf((float)vi.gx, fmaxf(0.f, floorf((o.u - o.radius) * inv_tile)));
  o.x1 = (int)fminf((float)vi.gx, fmaxf(0.f, floorf((o.u + o.radius + (kTile - 1)) * inv_tile)));
  o.y0 = (int)fminf((float)vi.gy, fmaxf(0.f, floorf((o.v - o.radius) * inv_tile)));
  o.y1 = (int)fminf((float)vi.gy, fmaxf(0.f, floorf((o.v + o.radius + (kTile - 1)) * inv_tile)));
  o.infrustum = (o.x1 > o.x0) && (o.y1 > o.y0);
  return o;
}

// Conservative frustum pre-test: false only if project_view would find the
// tile rectangle empty (or the mean behind the near plane). The radius of
// project_view is ceil(3 sqrt(lam)) with lam <= trace of the dilated 2D
// covariance + sqrt(0.1) <= |J|_F^2 |A|_F^2 s_max^2 + 0.92 (|JB|_F <= |J|_F
// |B|_2, |A RS|_2 <= |A|_F s_max), and |J|_F^2 <= (fx^2 (1 + limx^2) +
// fy^2 (1 + limy^2)) / z^2 under the field-of-view clamp. The bound gets 1 %
// and 2 px of slack for the FP32 rounding of both computations.
__device__ __forceinline__ bool may_touch_view(const InstMat& M, const float mu[3], float smax2,
                                               const ViewInfo& vi) {
  float d[3], x, y, z;
  rel_pos(M, mu, d);
  cam_pos(M, d, x, y, z);
  if (!(z > vi.near_z)) return false;
  const float iz = rcp_fast(z);
  const float u = fmaf(vi.fx, x * iz, vi.cx), v = fmaf(vi.fy, y * iz, vi.cy);
  const float rb = fmaf(3.03f, sqrt_fast(fmaf(vi.jc * M.a_frob2 * smax2, iz * iz, 0.93f)), 3.f);
  return !(u + rb < 0.f || u - rb > (float)(vi.gx * kTile) || v + rb < 0.f ||
           v - rb > (float)(vi.gy * kTile));
}

// Real SH basis (orthonormal, Condon-Shortley sign) at a unit direction d,
// degrees 0..DEG. Band constants: sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!)
// times the usual factor 2 for m != 0, folded into one number per term.
template <int DEG>
__device__ __forceinline__ void sh_basis(float dx, float dy, float dz, float Y[16]) {
  Y[0] = 0.28209479177387814f;
  if (DEG >= 1) {
    const float k1 = 0.48860251190291992f;
    Y[1] = -k1 * dy;
    Y[2] = k1 * dz;
    Y[3] = -k1 * dx;
  }
  if (DEG >= 2) {
    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    Y[4] = 1.0925484305920792f * dx * dy;
    Y[5] = -1.0925484305920792f * dy * dz;
    Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * dx * dz;
    Y[8] = 0.54627421529603959f * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -0.59004358992664352f * dy * (3.f * xx - yy);
      Y[10] = 2.8906114426405538f * dx * dy * dz;
      Y[11] = -0.45704579946446572f * dy * (4.f * zz - xx - yy);
      Y[12] = 0.37317633259011546f * dz * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -0.45704579946446572f * dx * (4.f * zz - xx - yy);
      Y[14] = 1.4453057213202769f * dz * (xx - yy);
      Y[15] = -0.59004358992664352f * dx * (xx - 3.f * yy);
    }
  }
}

__host__ __device__ constexpr int sh_count(int deg) { return (deg + 1) * (deg + 1); }

// d/d(direction) of sum_k w_k Y_k(d) for the real SH basis of sh_basis<DEG>.
template <int DEG>
__device__ __forceinline__ void sh_dir_grad(float x, float y, float z, const float w[16],
                                            float g[3]) {
  g[0] = g[1] = g[2] = 0.f;
  if (DEG >= 1) {
    const float k1 = 0.48860251190291992f;
    g[1] -= k1 * w[1];
    g[2] += k1 * w[2];
    g[0] -= k1 * w[3];
  }
  if (DEG >= 2) {
    const float k2a = 1.0925484305920792f, k2c = 0.31539156525252005f, k2e = 0.54627421529603959f;
    g[0] += k2a * y * w[4];                    g[1] += k2a * x * w[4];
    g[1] -= k2a * z * w[5];                    g[2] -= k2a * y * w[5];
    g[0] -= 2.f * k2c * x * w[6];              g[1] -= 2.f * k2c * y * w[6];
    g[2] += 4.f * k2c * z * w[6];
    g[0] -= k2a * z * w[7];                    g[2] -= k2a * x * w[7];
    g[0] += 2.f * k2e * x * w[8];              g[1] -= 2.f * k2e * y * w[8];
    if (DEG >= 3) {
      const float k3a = 0.59004358992664352f, k3b = 2.8906114426405538f,
                  k3c = 0.45704579946446572f, k3d = 0.37317633259011546f,
                  k3e = 1.4453057213202769f;
      const float xx = x * x, yy = y * y, zz = z * z;
      g[0] -= 6.f * k3a * x * y * w[9];
      g[1] -= k3a * (3.f * xx - 3.f * yy) * w[9];
      g[0] += k3b * y * z * w[10]; g[1] += k3b * x * z * w[10]; g[2] += k3b * x * y * w[10];
      g[0] += 2.f * k3c * x * y * w[11];
      g[1] -= k3c * (4.f * zz - xx - 3.f * yy) * w[11];
      g[2] -= 8.f * k3c * y * z * w[11];
      g[0] -= 6.f * k3d * x * z * w[12];
      g[1] -= 6.f * k3d * y * z * w[12];
      g[2] += k3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      g[0] -= k3c * (4.f * zz - 3.f * xx - yy) * w[13];
      g[1] += 2.f * k3c * x * y * w[13];
      g[2] -= 8.f * k3c * x * z * w[13];
      g[0] += 2.f * k3e * x * z * w[14];
      g[1] -= 2.f * k3e * y * z * w[14];
      g[2] += k3e * (xx - yy) * w[14];
      g[0] -= k3a * (3.f * xx - 3.f * yy) * w[15];
      g[1] += 6.f * k3a * x * y * w[15];
    }
  }
}

// Adjoint of the raw quaternion q (w, x, y, z) given dL/dR for R(q/|q|).
__device__ __forceinline__ float4 quat_backward(float4 q, const float dR[9]) {
  const float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  const float inv = rsqrtf(n2);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  // partials of the nine entries of R w.r.t. the unit quaternion
  float gw = 2.f * (x * (dR[7] - dR[5]) + y * (dR[2] - dR[6]) + z * (dR[3] - dR[1]));
  float gx = 2.f * (y * (dR[1] + dR[3]) + z * (dR[2] + dR[6]) + w * (dR[7] - dR[5])) -
             4.f * x * (dR[4] + dR[8]);
  float gy = 2.f * (x * (dR[1] + dR[3]) + z * (dR[5] + dR[7]) + w * (dR[2] - dR[6])) -
             4.f * y * (dR[0] + dR[8]);
  float gz = 2.f * (x * (dR[2] + dR[6]) + y * (dR[5] + dR[7]) + w * (dR[3] - dR[1])) -
             4.f * z * (dR[0] + dR[4]);
  const float dot = gw * w + gx * x + gy * y + gz * z;
  return make_float4((gw - w * dot) * inv, (gx - x * dot) * inv, (gy - y * dot) * inv,
                     (gz - z * dot) * inv);
}


// ---- stochastic LOD (Eq. 7) ---------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC 2011): ten rounds of two
// 32x32 -> 64-bit products by fixed odd multipliers, high halves XORed with
// the other counter words and the round key, key bumped by two Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

struct LodArgs {
  int mode;            // S3R_LOD_THRESHOLD / S3R_LOD_STOCHASTIC
  float p_max, dist;
  float off[3];
  uint32_t key0, key1;
};

// Eq. 7 drop decision for a small in-frustum (Gaussian, view) at depth z:
// drop iff the top 24 bits of the first draw are below p * 2^24, p evaluated
// with rounded single-precision operations (no contraction) so that it is the
// same number on any IEEE host.
__device__ __forceinline__ bool lod_keep(const LodArgs& L, uint32_t gid, uint32_t view,
                                         uint32_t epoch, float z) {
  const uint4 a = philox4x32_10(make_uint4(gid, view, epoch, 0u), L.key0, L.key1);
  const float t = fminf(0.f, __fdiv_rn(__fsub_rn(z, L.dist), L.dist));
  const float p = __fadd_rn(L.p_max, __fmul_rn(__fsub_rn(L.p_max, 0.01f), t));
  return !((float)(a.x >> 8) < __fmul_rn(p, 16777216.f));
}

// Noisy mean of a surviving small Gaussian: offset * min(1, z / D) * n with
// n per-axis standard normals by Box-Muller on 24-bit uniforms in (0, 1] and
// [0, 1) from the remaining words of the two blocks.
__device__ __forceinline__ void lod_noisy_mean(const LodArgs& L, uint32_t gid, uint32_t view,
                                               uint32_t epoch, float z, const float mu[3],
                                               float out[3]) {
  const uint4 a = philox4x32_10(make_uint4(gid, view, epoch, 0u), L.key0, L.key1);
  const uint4 b = philox4x32_10(make_uint4(gid, view, epoch, 1u), L.key0, L.key1);
  const float k24 = 1.f / 16777216.f;
  const float u1 = (float)((a.y >> 8) + 1u) * k24, u2 = (float)(a.z >> 8) * k24;
  const float u3 = (float)((a.w >> 8) + 1u) * k24, u4 = (float)(b.x >> 8) * k24;
  const float r1 = sqrtf(-2.f * logf(u1)), r2 = sqrtf(-2.f * logf(u3));
  float s1, c1, s2, c2;
  sincospif(2.f * u2, &s1, &c1);
  sincospif(2.f * u4, &s2, &c2);
  const float sc = fminf(1.f, z / L.dist);
  out[0] = fmaf(L.off[0] * sc, r1 * c1, mu[0]);
  out[1] = fmaf(L.off[1] * sc, r1 * s1, mu[1]);
  out[2] = fmaf(L.off[2] * sc, r2 * c2, mu[2]);
}

constexpr uint8_t kSplatMoved = 0x80;   // splat view byte: rendered at its noisy mean

// Shared-memory staging of the SH rows of a warp's 32 Gaussians: K*3 floats
// per Gaussian, moved as float4s when K*3 is a multiple of 4 (degrees 1, 3),
// each row padded by one element so that lanes reading their own rows spread
// over the banks. kWords = floats per warp.
template <int DEG>
struct ShStage {
  static constexpr int K = sh_count(DEG);
  static constexpr bool kVec = (K * 3) % 4 == 0;
  static constexpr int kRow = kVec ? K * 3 / 4 : K * 3;   // float4s or floats per Gaussian
  static constexpr int kPitch = kRow + 1;
  static constexpr int kFloatPitch = kPitch * (kVec ? 4 : 1);
  static constexpr int kWords = 32 * kFloatPitch;
};

// Coalesced copy of the SH rows of the warp's Gaussians gid (lane g holds the
// id of row g; rows g >= n_here are skipped) into `stage`.
template <int DEG>
__device__ __forceinline__ void stage_sh_rows(float* stage, const float* __restrict__ sh,
                                              uint32_t gid, int n_here, uint32_t lane) {
  using St = ShStage<DEG>;
  if constexpr (St::kVec) {
    const float4* src = reinterpret_cast<const float4*>(sh);
    float4* dst = reinterpret_cast<float4*>(stage);
#pragma unroll
    for (int it = 0; it < St::kRow; ++it) {
      const int idx = it * 32 + (int)lane;
      const int g = idx / St::kRow, q = idx - g * St::kRow;
      const uint32_t gg = __shfl_sync(0xffffffffu, gid, g);
      if (g < n_here) dst[g * St::kPitch + q] = __ldg(src + (size_t)gg * St::kRow + q);
    }
  } else {
#pragma unroll
    for (int it = 0; it < St::kRow; ++it) {
      const int idx = it * 32 + (int)lane;
      const int g = idx / St::kRow, q = idx - g * St::kRow;
      const uint32_t gg = __shfl_sync(0xffffffffu, gid, g);
      if (g < n_here) stage[g * St::kPitch + q] = __ldg(sh + (size_t)gg * St::kRow + q);
    }
  }
}

}  // namespace s3r
