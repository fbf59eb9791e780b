// FP64 CPU oracle for the S3R-GS per-timestep render-and-backprop path.
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
// GPU path is checked against. Only the tests, the smoke check and the bench's
// CPU-baseline leg may load it; the product path never does. It shares no
// code, header, table or constant with the CUDA library.
//
// What it computes, in the paper's order (Sec. 3.3, "Streamlined
// Reconstruction Stage"):
//   1. temporal selection: keep Gaussians with v_s <= t <= v_e   (Sec. 3.3,
//      "Temporal separation"; FP32 comparison, the record is FP32);
//   2. instance-specific projection: one composed matrix M = W_t * W_{t,i2g}
//      per instance, no local-to-global pass (Sec. 3.3, "Instance-specific
//      projection"), then Eq. 1 (mu' = K W mu, Sigma' = J W Sigma W^T J^T);
//   3. the visible mask M_t from the view frustum, and the point-life update
//      of Eq. 5 (done on M_t, before LOD);
//   4. adaptive-LOD threshold cull (Sec. 3.3, "Adaptive LOD", deterministic
//      reading: cull iff the projected 2D scale is below r), or, when enabled,
//      the stochastic form of Eq. 7 on the Gaussians below r (depth-dependent
//      Bernoulli drop, noisy offset of the survivors), drawn from a
//      Philox4x32-10 counter-based generator;
//   5. SH colour and front-to-back alpha blending, Eq. 2;
//   6. Eq. 6 (visibility from point life) and the reset to "always visible";
//   7. the exact gradient of the rendered image w.r.t. every parameter and the
//      per-instance poses, derived by hand with the chain rule in FP64.
// Constants the paper leaves to 3DGS (near plane 0.2, the 1.3 x/z clamp, the
// 0.3 dilation, the 1/255 alpha floor, the 0.99 alpha cap, the 1e-4
// transmittance stop, the 3-sigma radius, 16x16 tiles, the +0.5 SH offset)
// are taken as definitions.
//
// All arithmetic is double; inputs arrive as float32 and are widened exactly.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int kTile = 16;
constexpr double kNear = 0.2;          // only used when a camera passes near <= 0
constexpr double kDilation = 0.3;
constexpr double kAlphaMin = 1.0 / 255.0;
constexpr double kAlphaMax = 0.99;
constexpr double kTStop = 1e-4;
constexpr double kClampFov = 1.3;

// ---------------------------------------------------------------- cameras
// A camera is passed as 19 doubles:
//   width, height, fx, fy, cx, cy, near, world_to_cam[12] (3x4 row-major).
struct Cam {
  int w, h;
  double fx, fy, cx, cy, near_z;
  double V[3][4];
};

Cam load_cam(const double* c) {
  Cam k;
  k.w = (int)c[0];
  k.h = (int)c[1];
  k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
  k.near_z = c[6] > 0 ? c[6] : kNear;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 4; ++q) k.V[r][q] = c[7 + 4 * r + q];
  return k;
}

// ---------------------------------------------------------------- rotations
// Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z).
void quat_rot(const double qin[4], double R[3][3], double qn[4], double* norm) {
  double n = std::sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
  if (qn) { qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z; }
  if (norm) *norm = n;
}

// Gradient w.r.t. the raw (unnormalised) quaternion, given dL/dR.
void quat_rot_backward(const double qin[4], const double dR[3][3], double dq[4]) {
  double R[3][3], qn[4], n;
  quat_rot(qin, R, qn, &n);
  double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
  double gw = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
  double gx = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2]
                   + z * dR[2][0] + w * dR[2][1] - 2 * x * dR[2][2]);
  double gy = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2]
                   - w * dR[2][0] + z * dR[2][1] - 2 * y * dR[2][2]);
  double gz = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1]
                   + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
  double g[4] = {gw, gx, gy, gz};
  double dot = g[0] * qn[0] + g[1] * qn[1] + g[2] * qn[2] + g[3] * qn[3];
  for (int i = 0; i < 4; ++i) dq[i] = (g[i] - qn[i] * dot) / n;
}

void inv3(const double A[3][3], double Ai[3][3]) {
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
             - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
             + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

// ---------------------------------------------------------------- SH basis
// Real spherical harmonics up to degree 3 on a unit direction (x, y, z), with
// the Condon-Shortley sign and orthonormal normalisation over the sphere.
const double kPi = 3.14159265358979323846;

void sh_basis(const double d[3], double Y[16], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  const double c0 = 0.5 / std::sqrt(kPi);
  const double c1 = std::sqrt(3.0 / (4.0 * kPi));
  const double c2a = std::sqrt(15.0 / (4.0 * kPi));
  const double c2c = std::sqrt(5.0 / (16.0 * kPi));
  const double c2e = std::sqrt(15.0 / (16.0 * kPi));
  const double c3a = std::sqrt(35.0 / (32.0 * kPi));
  const double c3b = std::sqrt(105.0 / (4.0 * kPi));
  const double c3c = std::sqrt(21.0 / (32.0 * kPi));
  const double c3d = std::sqrt(7.0 / (16.0 * kPi));
  const double c3e = std::sqrt(105.0 / (16.0 * kPi));
  const double xx = x * x, yy = y * y, zz = z * z;
  Y[0] = c0;
  Y[1] = -c1 * y;
  Y[2] = c1 * z;
  Y[3] = -c1 * x;
  Y[4] = c2a * x * y;
  Y[5] = -c2a * y * z;
  Y[6] = c2c * (2 * zz - xx - yy);
  Y[7] = -c2a * x * z;
  Y[8] = c2e * (xx - yy);
  Y[9] = -c3a * y * (3 * xx - yy);
  Y[10] = c3b * x * y * z;
  Y[11] = -c3c * y * (4 * zz - xx - yy);
  Y[12] = c3d * z * (2 * zz - 3 * xx - 3 * yy);
  Y[13] = -c3c * x * (4 * zz - xx - yy);
  Y[14] = c3e * z * (xx - yy);
  Y[15] = -c3a * x * (xx - 3 * yy);
  if (!dY) return;
  auto set = [&](int k, double gx, double gy, double gz) { dY[k][0] = gx; dY[k][1] = gy; dY[k][2] = gz; };
  set(0, 0, 0, 0);
  set(1, 0, -c1, 0);
  set(2, 0, 0, c1);
  set(3, -c1, 0, 0);
  set(4, c2a * y, c2a * x, 0);
  set(5, 0, -c2a * z, -c2a * y);
  set(6, -2 * c2c * x, -2 * c2c * y, 4 * c2c * z);
  set(7, -c2a * z, 0, -c2a * x);
  set(8, 2 * c2e * x, -2 * c2e * y, 0);
  set(9, -c3a * 6 * x * y, -c3a * (3 * xx - 3 * yy), 0);
  set(10, c3b * y * z, c3b * x * z, c3b * x * y);
  set(11, c3c * 2 * x * y, -c3c * (4 * zz - xx - 3 * yy), -c3c * 8 * y * z);
  set(12, -6 * c3d * x * z, -6 * c3d * y * z, c3d * (6 * zz - 3 * xx - 3 * yy));
  set(13, -c3c * (4 * zz - 3 * xx - yy), c3c * 2 * x * y, -c3c * 8 * x * z);
  set(14, 2 * c3e * x * z, -2 * c3e * y * z, c3e * (xx - yy));
  set(15, -c3a * (3 * xx - 3 * yy), c3a * 6 * x * y, 0);
}

// ------------------------------------------------------- counter-based RNG
// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As
// Easy as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplications by
// fixed odd multipliers, the high halves XORed with the other two counter
// words and the round key; the key is bumped by two Weyl constants between
// rounds.
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  const uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kW0;
      k1 += kW1;
    }
    const uint64_t p0 = (uint64_t)kM0 * c0, p1 = (uint64_t)kM1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Stochastic LOD of Eq. 7 (off unless set by orc_set_lod).
struct LodParams {
  int mode = 0;                 // 0: deterministic threshold cull, 1: Eq. 7 on the small ones
  float p_max = 0.f, dist = 1.f;
  double offset[3] = {0, 0, 0}; // [dx, dy, dz] of Eq. 7
  uint32_t key[2] = {0, 0};     // generator key (the seed)
  uint32_t epoch = 0;           // third counter word: which call
};
LodParams g_lod;

// ---------------------------------------------------------------- projection
// Everything the forward computes for one Gaussian in one view.
struct Proj {
  int infrustum;   // M_t bit: z > near, det > 0, non-empty tile rectangle
  int kept;        // infrustum and sigma_lod >= r
  int near_boundary;  // bits set when a decision lies within a tiny margin of its
                      // threshold: 1 near plane, 2 left, 4 right, 8 top, 16 bottom
                      // rect edge, 32 radius ceil, 64 LOD threshold, 128 Eq. 7 draw
  int offset;      // Eq. 7: projected at the noisy position (2D values below are there)
  double p[3];     // camera-space position
  double u, v;
  double conic[3]; // (A, B, C): power = -0.5 (A dx^2 + C dy^2) - B dx dy
  double opacity;
  double rgb[3];
  int rgb_clamped[3];
  double radius;
  int rect[4];     // x0, y0, x1, y1 in tiles, half-open
  double sigma_lod;
  // intermediates kept for the backward pass
  double s[3], R[3][3], qraw[4], S3[3][3], A[3][3], b[3], Sc[3][3], J[2][3];
  int clampx, clampy;
  double ratio_x, ratio_y;  // clamped x/z, y/z
  double S2[3];    // a, b, c of J Sc J^T (before dilation)
  double cam_c[3], vec[3], vnorm, dir[3];
};

// Composed instance matrix M = V * P, P = [R(q) | t] (local -> world).
void compose(const Cam& cam, const double* P /*3x4 or null = identity*/, double A[3][3], double b[3]) {
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += cam.V[r][k] * (P ? P[4 * k + c] : (k == c ? 1.0 : 0.0));
      A[r][c] = acc;
    }
    double acc = cam.V[r][3];
    for (int k = 0; k < 3; ++k) acc += cam.V[r][k] * (P ? P[4 * k + 3] : 0.0);
    b[r] = acc;
  }
}

void pose_matrix(const double* q, const double* t, double P[12]) {
  double qd[4] = {q[0], q[1], q[2], q[3]}, R[3][3];
  quat_rot(qd, R, nullptr, nullptr);
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) P[4 * r + c] = R[r][c];
    P[4 * r + 3] = t[r];
  }
}

bool near_int(double q, double tol) { return std::fabs(q - std::nearbyint(q)) < tol; }

// F (may be null = identity) is the rotation from the frame the SH
// coefficients live in to the frame of `mean`; the SH direction is F^T dir.
void project_core(const Cam& cam, const double A[3][3], const double b[3], const double mu[3],
                  const double log_scale[3], const double quat[4], double opac_logit,
                  const double* sh, int sh_deg, double lod_r, const double (*F)[3], Proj& o) {
  std::memset(&o, 0, sizeof(o));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) o.A[i][j] = A[i][j];
  for (int i = 0; i < 3; ++i) o.b[i] = b[i];
  for (int r = 0; r < 3; ++r) o.p[r] = A[r][0] * mu[0] + A[r][1] * mu[1] + A[r][2] * mu[2] + b[r];
  const double x = o.p[0], y = o.p[1], z = o.p[2];
  const double margin = 3e-6;
  if (std::fabs(z - cam.near_z) < margin * cam.near_z) o.near_boundary |= 1;
  if (!(z > cam.near_z)) return;

  // 3D covariance Sigma = R S S^T R^T
  for (int i = 0; i < 3; ++i) o.s[i] = std::exp(log_scale[i]);
  for (int i = 0; i < 4; ++i) o.qraw[i] = quat[i];
  quat_rot(o.qraw, o.R, nullptr, nullptr);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += o.R[i][k] * o.s[k] * o.s[k] * o.R[j][k];
      o.S3[i][j] = acc;
    }
  // camera-space covariance A Sigma A^T (the W Sigma W^T of Eq. 1)
  double T1[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += A[i][k] * o.S3[k][j];
      T1[i][j] = acc;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += T1[i][k] * A[j][k];
      o.Sc[i][j] = acc;
    }
  // Jacobian of the perspective map at p, with the x/z and y/z clamp
  const double limx = kClampFov * (0.5 * cam.w / cam.fx);
  const double limy = kClampFov * (0.5 * cam.h / cam.fy);
  const double rx = x / z, ry = y / z;
  o.clampx = (rx < -limx || rx > limx);
  o.clampy = (ry < -limy || ry > limy);
  o.ratio_x = std::min(limx, std::max(-limx, rx));
  o.ratio_y = std::min(limy, std::max(-limy, ry));
  const double tx = o.ratio_x * z, ty = o.ratio_y * z;
  o.J[0][0] = cam.fx / z; o.J[0][1] = 0; o.J[0][2] = -cam.fx * tx / (z * z);
  o.J[1][0] = 0; o.J[1][1] = cam.fy / z; o.J[1][2] = -cam.fy * ty / (z * z);
  double JS[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += o.J[i][k] * o.Sc[k][j];
      JS[i][j] = acc;
    }
  double S2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += JS[i][k] * o.J[j][k];
      S2[i][j] = acc;
    }
  const double a = S2[0][0], bb = S2[0][1], c = S2[1][1];
  o.S2[0] = a; o.S2[1] = bb; o.S2[2] = c;
  // 2D scale for LOD: largest standard deviation before dilation
  const double mid0 = 0.5 * (a + c), det0 = a * c - bb * bb;
  o.sigma_lod = std::sqrt(mid0 + std::sqrt(std::max(0.0, mid0 * mid0 - det0)));
  // dilated 2D covariance, conic, radius
  const double ad = a + kDilation, cd = c + kDilation;
  const double det = ad * cd - bb * bb;
  if (!(det > 0)) return;
  o.conic[0] = cd / det; o.conic[1] = -bb / det; o.conic[2] = ad / det;
  const double mid = 0.5 * (ad + cd);
  const double lam = mid + std::sqrt(std::max(0.1, mid * mid - det));
  const double r3 = 3.0 * std::sqrt(lam);
  o.radius = std::ceil(r3);
  if (near_int(r3, margin * r3)) o.near_boundary |= 32;
  o.u = cam.fx * x / z + cam.cx;
  o.v = cam.fy * y / z + cam.cy;
  const int gx = (cam.w + kTile - 1) / kTile, gy = (cam.h + kTile - 1) / kTile;
  auto edge = [&](double q, int g) {
    double f = std::floor(q);
    return (int)std::min((double)g, std::max(0.0, f));
  };
  const double qx0 = (o.u - o.radius) / kTile, qx1 = (o.u + o.radius + kTile - 1) / kTile;
  const double qy0 = (o.v - o.radius) / kTile, qy1 = (o.v + o.radius + kTile - 1) / kTile;
  const double tol_x = margin * (std::fabs(o.u) + o.radius + kTile) / kTile;
  const double tol_y = margin * (std::fabs(o.v) + o.radius + kTile) / kTile;
  if (near_int(qx0, tol_x)) o.near_boundary |= 2;
  if (near_int(qx1, tol_x)) o.near_boundary |= 4;
  if (near_int(qy0, tol_y)) o.near_boundary |= 8;
  if (near_int(qy1, tol_y)) o.near_boundary |= 16;
  o.rect[0] = edge(qx0, gx); o.rect[1] = edge(qy0, gy);
  o.rect[2] = edge(qx1, gx); o.rect[3] = edge(qy1, gy);
  if ((o.rect[2] - o.rect[0]) * (o.rect[3] - o.rect[1]) <= 0) return;
  o.infrustum = 1;
  if (lod_r > 0 && std::fabs(o.sigma_lod - lod_r) < margin * lod_r) o.near_boundary |= 64;
  o.kept = (o.sigma_lod >= lod_r);
  o.opacity = 1.0 / (1.0 + std::exp(-opac_logit));
  // colour: SH evaluated on the direction from the camera centre, expressed in
  // the Gaussian's own (instance) frame: c = -A^{-1} b
  double Ai[3][3];
  inv3(A, Ai);
  for (int r = 0; r < 3; ++r) o.cam_c[r] = -(Ai[r][0] * b[0] + Ai[r][1] * b[1] + Ai[r][2] * b[2]);
  for (int r = 0; r < 3; ++r) o.vec[r] = mu[r] - o.cam_c[r];
  o.vnorm = std::sqrt(o.vec[0] * o.vec[0] + o.vec[1] * o.vec[1] + o.vec[2] * o.vec[2]);
  for (int r = 0; r < 3; ++r) o.dir[r] = o.vec[r] / o.vnorm;
  double dsh[3] = {o.dir[0], o.dir[1], o.dir[2]};
  if (F)
    for (int r = 0; r < 3; ++r) dsh[r] = F[0][r] * o.dir[0] + F[1][r] * o.dir[1] + F[2][r] * o.dir[2];
  double Y[16];
  sh_basis(dsh, Y, nullptr);
  const int K = (sh_deg + 1) * (sh_deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0;
    for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * Y[k];
    acc += 0.5;
    o.rgb_clamped[ch] = acc < 0;
    o.rgb[ch] = acc < 0 ? 0.0 : acc;
  }
}

void project_one(const Cam& cam, const double A[3][3], const double b[3], const double* mean,
                 const double* log_scale, const double* quat, double opac_logit, const double* sh,
                 int sh_deg, double lod_r, Proj& o) {
  const double mu[3] = {mean[0], mean[1], mean[2]};
  const double ls[3] = {log_scale[0], log_scale[1], log_scale[2]};
  const double q[4] = {quat[0], quat[1], quat[2], quat[3]};
  project_core(cam, A, b, mu, ls, q, opac_logit, sh, sh_deg, lod_r, nullptr, o);
}

// Eq. 7 for one (Gaussian, view) that is in the frustum with a 2D scale below
// r. Reading of the garbled parts: p rises linearly from 0.01 at depth 0 to
// p_max at depth D and stays there; "Bernoulli(p) <= 0" keeps the Gaussian
// iff the draw is 0 (probability 1 - p); "normalize(d)" is min(1, d / D); the
// standard normal is drawn per axis. The draw is decided in FP32, as the GPU
// does: drop iff (a0 >> 8) < p * 2^24 with p evaluated in FP32 from the FP32
// depth. Normals by Box-Muller on (0, 1] x [0, 1) uniforms of 24 bits.
// Returns true if kept and writes the noisy mean.
bool lod_draw(int64_t gid, int view, double z, const double mu[3], double mu_out[3],
              int* near_bits) {
  const uint32_t ctr0[4] = {(uint32_t)gid, (uint32_t)view, g_lod.epoch, 0u};
  const uint32_t ctr1[4] = {(uint32_t)gid, (uint32_t)view, g_lod.epoch, 1u};
  uint32_t a[4], b[4];
  philox4x32_10(ctr0, g_lod.key, a);
  const float zf = (float)z;
  const float D = g_lod.dist;
  const float p = g_lod.p_max + (g_lod.p_max - 0.01f) * std::min(0.f, (zf - D) / D);
  const float thr = p * 16777216.f;
  const float u0 = (float)(a[0] >> 8);
  if (std::fabs((double)u0 - (double)thr) <= 8.0) *near_bits |= 128;
  if (u0 < thr) return false;
  philox4x32_10(ctr1, g_lod.key, b);
  const double two24 = 16777216.0;
  const double u1 = ((a[1] >> 8) + 1.0) / two24, u2 = (a[2] >> 8) / two24;
  const double u3 = ((a[3] >> 8) + 1.0) / two24, u4 = (b[0] >> 8) / two24;
  const double r1 = std::sqrt(-2.0 * std::log(u1)), r2 = std::sqrt(-2.0 * std::log(u3));
  const double n[3] = {r1 * std::cos(2 * kPi * u2), r1 * std::sin(2 * kPi * u2),
                       r2 * std::cos(2 * kPi * u4)};
  const double s = std::min(1.0, z / (double)D);
  for (int i = 0; i < 3; ++i) mu_out[i] = mu[i] + g_lod.offset[i] * n[i] * s;
  return true;
}

// The projection of one (Gaussian, view) as the path renders it: Eq. 1 at the
// mean; under the stochastic LOD a small Gaussian is dropped or re-projected
// at its noisy mean (then kept even if that leaves the frustum: it is a splat
// with no tiles). mu_used receives the mean the 2D values belong to.
void project_lod(const Cam& cam, const double A[3][3], const double b[3], int64_t gid, int view,
                 const double* mean, const double* log_scale, const double* quat,
                 double opac_logit, const double* sh, int sh_deg, double lod_r, Proj& o,
                 double mu_used[3]) {
  project_one(cam, A, b, mean, log_scale, quat, opac_logit, sh, sh_deg, lod_r, o);
  for (int i = 0; i < 3; ++i) mu_used[i] = mean[i];
  if (g_lod.mode != 1 || !o.infrustum || o.kept) return;
  int bits = o.near_boundary;
  double mu2[3];
  if (!lod_draw(gid, view, o.p[2], mean, mu2, &bits)) {
    o.near_boundary = bits;
    return;
  }
  Proj o2;
  project_one(cam, A, b, mu2, log_scale, quat, opac_logit, sh, sh_deg, 0.0, o2);
  if (!o2.infrustum) {
    for (int i = 0; i < 4; ++i) o2.rect[i] = 0;
  }
  o2.near_boundary |= bits;
  o2.infrustum = 1;   // M_t is the frustum test at the mean
  o2.kept = 1;
  o2.offset = 1;
  o2.sigma_lod = o.sigma_lod;
  o = o2;
  for (int i = 0; i < 3; ++i) mu_used[i] = mu2[i];
}

// Gradient of one projected Gaussian: from the 2D quantities back to the
// parameters and to the composed matrix [A | b].
struct ProjGrad {
  double mean[3], log_scale[3], quat[4], opac_logit;
  double sh[16][3];
  double dA[3][3], db[3];
};

void project_one_backward(const Cam& cam, const Proj& o, const double* mean, const double* sh,
                          int sh_deg, const double g_uv[2], const double g_conic[3],
                          double g_opac, const double g_rgb[3], ProjGrad& g) {
  std::memset(&g, 0, sizeof(g));
  const double mu[3] = {mean[0], mean[1], mean[2]};
  const double x = o.p[0], y = o.p[1], z = o.p[2];
  double dp[3] = {0, 0, 0};

  // opacity = sigmoid(logit)
  g.opac_logit = g_opac * o.opacity * (1.0 - o.opacity);

  // colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5)
  double Y[16], dY[16][3];
  sh_basis(o.dir, Y, dY);
  const int K = (sh_deg + 1) * (sh_deg + 1);
  double graw[3];
  for (int ch = 0; ch < 3; ++ch) graw[ch] = o.rgb_clamped[ch] ? 0.0 : g_rgb[ch];
  double gdir[3] = {0, 0, 0};
  for (int k = 0; k < K; ++k)
    for (int ch = 0; ch < 3; ++ch) {
      g.sh[k][ch] = Y[k] * graw[ch];
      for (int r = 0; r < 3; ++r) gdir[r] += sh[3 * k + ch] * graw[ch] * dY[k][r];
    }
  // dir = vec / |vec|, vec = mu - c
  double dd = gdir[0] * o.dir[0] + gdir[1] * o.dir[1] + gdir[2] * o.dir[2];
  double gvec[3];
  for (int r = 0; r < 3; ++r) gvec[r] = (gdir[r] - o.dir[r] * dd) / o.vnorm;
  for (int r = 0; r < 3; ++r) g.mean[r] += gvec[r];
  // c = -A^{-1} b  =>  dL/db = -A^{-T} gc,  dL/dA = -(A^{-T} gc) c^T, with gc = -gvec
  double Ai[3][3];
  inv3(o.A, Ai);
  double w[3];
  for (int r = 0; r < 3; ++r) w[r] = -(Ai[0][r] * (-gvec[0]) + Ai[1][r] * (-gvec[1]) + Ai[2][r] * (-gvec[2]));
  for (int r = 0; r < 3; ++r) {
    g.db[r] += w[r];
    for (int c = 0; c < 3; ++c) g.dA[r][c] += w[r] * o.cam_c[c];
  }

  // conic = inverse of the dilated 2D covariance X = [[a', b], [b, c']]
  const double Q[2][2] = {{o.conic[0], o.conic[1]}, {o.conic[1], o.conic[2]}};
  const double GQ[2][2] = {{g_conic[0], 0.5 * g_conic[1]}, {0.5 * g_conic[1], g_conic[2]}};
  double GX[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double acc = 0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) acc += Q[i][k] * GQ[k][l] * Q[l][j];
      GX[i][j] = -acc;
    }
  // the dilation adds a constant, so dL/dSigma2 = dL/dX (symmetric form)
  const double G2[2][2] = {{GX[0][0], GX[0][1]}, {GX[1][0], GX[1][1]}};
  // Sigma2 = J Sc J^T
  double dJ[2][3], dSc[3][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 3; ++l) acc += G2[i][k] * o.J[k][l] * o.Sc[l][j];
      dJ[i][j] = 2.0 * acc;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) acc += o.J[k][i] * G2[k][l] * o.J[l][j];
      dSc[i][j] = acc;
    }
  // Sc = A S3 A^T
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += dSc[i][k] * o.A[k][l] * o.S3[l][j];
      g.dA[i][j] += 2.0 * acc;
    }
  double dS3[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc += o.A[k][i] * dSc[k][l] * o.A[l][j];
      dS3[i][j] = acc;
    }
  // S3 = M M^T, M = R diag(s)
  double Mm[3][3], dM[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Mm[i][j] = o.R[i][j] * o.s[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += dS3[i][k] * Mm[k][j];
      dM[i][j] = 2.0 * acc;
    }
  double dR[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dR[i][j] = dM[i][j] * o.s[j];
  for (int j = 0; j < 3; ++j) {
    double ds = 0;
    for (int i = 0; i < 3; ++i) ds += o.R[i][j] * dM[i][j];
    g.log_scale[j] = ds * o.s[j];
  }
  quat_rot_backward(o.qraw, dR, g.quat);

  // J(p): J00 = fx/z, J11 = fy/z, J02 = -fx tx/z^2, J12 = -fy ty/z^2
  dp[2] += dJ[0][0] * (-cam.fx / (z * z)) + dJ[1][1] * (-cam.fy / (z * z));
  if (!o.clampx) {
    dp[0] += dJ[0][2] * (-cam.fx / (z * z));
    dp[2] += dJ[0][2] * (2.0 * cam.fx * x / (z * z * z));
  } else {
    dp[2] += dJ[0][2] * (cam.fx * o.ratio_x / (z * z));
  }
  if (!o.clampy) {
    dp[1] += dJ[1][2] * (-cam.fy / (z * z));
    dp[2] += dJ[1][2] * (2.0 * cam.fy * y / (z * z * z));
  } else {
    dp[2] += dJ[1][2] * (cam.fy * o.ratio_y / (z * z));
  }
  // (u, v) = (fx x/z + cx, fy y/z + cy)
  dp[0] += g_uv[0] * cam.fx / z;
  dp[1] += g_uv[1] * cam.fy / z;
  dp[2] += -g_uv[0] * cam.fx * x / (z * z) - g_uv[1] * cam.fy * y / (z * z);
  // p = A mu + b
  for (int c = 0; c < 3; ++c) g.mean[c] += o.A[0][c] * dp[0] + o.A[1][c] * dp[1] + o.A[2][c] * dp[2];
  for (int r = 0; r < 3; ++r) {
    g.db[r] += dp[r];
    for (int c = 0; c < 3; ++c) g.dA[r][c] += dp[r] * mu[c];
  }
}

int instance_of(const int64_t* off, int n_inst, int64_t gid) {
  // segment k covers [off[k], off[k+1]); segment 0 is static
  for (int k = 0; k <= n_inst; ++k)
    if (gid >= off[k] && gid < off[k + 1]) return k;
  return -1;
}

// ---------------------------------------------------------------- blending
// A splat is one kept (Gaussian, view) pair as the blend sees it.
struct SplatView {
  int n;
  const double *u, *v, *conic, *opac, *rgb;
  const float* depth32;
  const int64_t* order;   // tie-break among equal depths (ascending)
  const int32_t* rect;    // [n,4]
};

// Global front-to-back order: ascending FP32 depth, ties by `order`.
std::vector<int> depth_order(const SplatView& s) {
  std::vector<int> idx(s.n);
  for (int i = 0; i < s.n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (s.depth32[a] != s.depth32[b]) return s.depth32[a] < s.depth32[b];
    return s.order[a] < s.order[b];
  });
  return idx;
}

bool covers(const int32_t* r, int tx, int ty) { return tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]; }

// Margins within which a blend decision counts as "near its threshold".
// Tests that perturb inputs (finite differences) widen them.
double g_tol_alpha = 1e-6, g_tol_T = 1e-8, g_tol_power = 1e-9;

// Per-pixel record of what happened along the ordered list.
struct PixelTrace {
  std::vector<int> list;      // splats (indices) whose rect covers the tile, in order
  std::vector<int> contrib;   // positions in `list` that were blended
  std::vector<double> alpha, T, G;
  std::vector<int> capped;    // alpha hit the 0.99 cap
  double Tfinal;
  int n_contrib;              // 1 + position of the last blended splat, 0 if none
  int flag;                   // a decision within a tiny margin of its threshold
};

void blend_pixel(const SplatView& s, const std::vector<int>& list, double px, double py,
                 PixelTrace& tr) {
  tr.list = list;
  tr.contrib.clear(); tr.alpha.clear(); tr.T.clear(); tr.G.clear(); tr.capped.clear();
  tr.flag = 0;
  double T = 1.0;
  tr.n_contrib = 0;
  std::vector<char> active(list.size(), 0);
  bool done = false;
  for (size_t pos = 0; pos < list.size(); ++pos) {
    const int i = list[pos];
    const double dx = s.u[i] - px, dy = s.v[i] - py;
    const double A = s.conic[3 * i], B = s.conic[3 * i + 1], C = s.conic[3 * i + 2];
    const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
    if (!done && std::fabs(power) < g_tol_power) tr.flag = 1;
    if (power > 0) continue;
    const double G = std::exp(power);
    const double raw = s.opac[i] * G;
    const double alpha = std::min(kAlphaMax, raw);
    if (!done && std::fabs(raw - kAlphaMax) < g_tol_alpha) tr.flag = 1;
    if (!done && std::fabs(alpha - kAlphaMin) < g_tol_alpha) tr.flag = 1;
    if (alpha < kAlphaMin) continue;
    if (done) continue;
    active[pos] = 1;
    const double nextT = T * (1.0 - alpha);
    if (std::fabs(nextT - kTStop) < g_tol_T) tr.flag = 1;
    if (nextT < kTStop) { done = true; continue; }
    tr.contrib.push_back((int)pos);
    tr.alpha.push_back(alpha);
    tr.T.push_back(T);
    tr.G.push_back(G);
    tr.capped.push_back(raw > kAlphaMax);
    T = nextT;
    tr.n_contrib = (int)pos + 1;
  }
  tr.Tfinal = T;
  // two splats that both reach this pixel with nearly equal FP32 depths make
  // the blend order (and so the result) fragile under rounding
  for (size_t k = 1; k < active.size(); ++k) {
    if (!active[k - 1] || !active[k]) continue;
    float a = s.depth32[list[k - 1]], b = s.depth32[list[k]];
    if (std::fabs((double)b - (double)a) <= 4.0 * std::ldexp(1.0, std::ilogb(std::max(a, b)) - 23))
      tr.flag = 1;
  }
}

}  // namespace

// ============================================================== C interface
extern "C" {

// Temporal selection (Sec. 3.3, "Temporal separation"): ascending indices i
// with v_s[i] <= t <= v_e[i], compared in FP32. Returns the count.
int64_t orc_select(int64_t n, const float* vis, float t, int64_t* idx_out) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const float vs = vis[2 * i], ve = vis[2 * i + 1];
    if (vs <= t && t <= ve) idx_out[m++] = i;
  }
  return m;
}

// Point-life update, Eq. 5: where mask[i], l_s = min(l_s, t), l_e = max(l_e, t).
void orc_vis_record(int64_t n, const uint8_t* mask, float t, float* life) {
  for (int64_t i = 0; i < n; ++i)
    if (mask[i]) {
      life[2 * i] = std::min(life[2 * i], t);
      life[2 * i + 1] = std::max(life[2 * i + 1], t);
    }
}

// Visibility from point life, Eq. 6: v_s = l_s - 0.1, v_e = l_e + 0.1 (FP32).
void orc_vis_finalize(int64_t n, const float* life, float* vis) {
  const float m = 0.1f;
  for (int64_t i = 0; i < n; ++i) {
    vis[2 * i] = life[2 * i] - m;
    vis[2 * i + 1] = life[2 * i + 1] + m;
  }
}

// Reset to "visible at all times" (Sec. 3.3): v = (-1, 1), l = (1, -1).
void orc_vis_reset(int64_t n, float* life, float* vis) {
  for (int64_t i = 0; i < n; ++i) {
    vis[2 * i] = -1.0f; vis[2 * i + 1] = 1.0f;
    life[2 * i] = 1.0f; life[2 * i + 1] = -1.0f;
  }
}

// Number of doubles per projected record written by orc_project.
int orc_rec_width(void) { return 24; }

// Instance-specific projection of the selected Gaussians into one view.
// cam: 19 doubles (see Cam). Instance k >= 1 has pose (inst_q[k-1], inst_t[k-1]).
// rec[i*24 + ...]: 0 infrustum, 1 kept, 2 near_boundary, 3..5 p, 6 u, 7 v,
//   8..10 conic, 11 opacity, 12..14 rgb, 15 radius, 16..19 rect, 20 sigma_lod,
//   21 fl32(z), 22 instance, 23 gid.
void orc_project(int64_t n_sel, const int64_t* sel, const double* means, const double* log_scales,
                 const double* quats, const double* opac_logits, const double* sh, int sh_deg,
                 const int64_t* inst_off, int n_inst, const double* inst_q, const double* inst_t,
                 const double* cam_raw, double lod_r, int view, double* rec) {
  const Cam cam = load_cam(cam_raw);
  std::vector<double> As((n_inst + 1) * 9), bs((n_inst + 1) * 3);
  for (int k = 0; k <= n_inst; ++k) {
    double P[12], A[3][3], b[3];
    if (k > 0) pose_matrix(inst_q + 4 * (k - 1), inst_t + 3 * (k - 1), P);
    compose(cam, k > 0 ? P : nullptr, A, b);
    for (int i = 0; i < 9; ++i) As[9 * k + i] = A[i / 3][i % 3];
    for (int i = 0; i < 3; ++i) bs[3 * k + i] = b[i];
  }
  const int K = (sh_deg + 1) * (sh_deg + 1);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_sel; ++j) {
    const int64_t g = sel[j];
    const int k = instance_of(inst_off, n_inst, g);
    double A[3][3], b[3];
    for (int i = 0; i < 9; ++i) A[i / 3][i % 3] = As[9 * k + i];
    for (int i = 0; i < 3; ++i) b[i] = bs[3 * k + i];
    Proj o;
    double mu_used[3];
    project_lod(cam, A, b, g, view, means + 3 * g, log_scales + 3 * g, quats + 4 * g,
                opac_logits[g], sh + (size_t)K * 3 * g, sh_deg, lod_r, o, mu_used);
    double* r = rec + 24 * j;
    r[0] = o.infrustum; r[1] = o.kept; r[2] = o.near_boundary;
    r[3] = o.p[0]; r[4] = o.p[1]; r[5] = o.p[2];
    r[6] = o.u; r[7] = o.v;
    r[8] = o.conic[0]; r[9] = o.conic[1]; r[10] = o.conic[2];
    r[11] = o.opacity; r[12] = o.rgb[0]; r[13] = o.rgb[1]; r[14] = o.rgb[2];
    r[15] = o.radius;
    r[16] = o.rect[0]; r[17] = o.rect[1]; r[18] = o.rect[2]; r[19] = o.rect[3];
    r[20] = o.sigma_lod; r[21] = (double)(float)o.p[2]; r[22] = k; r[23] = (double)g;
  }
}

// The conventional path (Fig. 1(a)): transform each dynamic Gaussian to the
// world frame first (mu_w = P mu, q_w = q_P * q, so R_w = R_P R), then project
// it with the camera alone. Same record layout as orc_project. The SH
// direction is rotated back into the Gaussian's own frame (by R_P^T) so that
// colours are comparable with the instance-specific path.
void orc_project_conventional(int64_t n_sel, const int64_t* sel, const double* means,
                              const double* log_scales, const double* quats,
                              const double* opac_logits, const double* sh, int sh_deg,
                              const int64_t* inst_off, int n_inst, const double* inst_q,
                              const double* inst_t, const double* cam_raw, double lod_r,
                              double* rec) {
  const Cam cam = load_cam(cam_raw);
  const int K = (sh_deg + 1) * (sh_deg + 1);
  double V[3][3], Vt[3];
  compose(cam, nullptr, V, Vt);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_sel; ++j) {
    const int64_t g = sel[j];
    const int k = instance_of(inst_off, n_inst, g);
    double PR[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, Pt[3] = {0, 0, 0};
    double qp[4] = {1, 0, 0, 0};
    if (k > 0) {
      const double* q = inst_q + 4 * (k - 1);
      const double qin[4] = {q[0], q[1], q[2], q[3]};
      quat_rot(qin, PR, qp, nullptr);
      for (int r = 0; r < 3; ++r) Pt[r] = inst_t[3 * (k - 1) + r];
    }
    double mw[3];
    for (int r = 0; r < 3; ++r)
      mw[r] = PR[r][0] * means[3 * g] + PR[r][1] * means[3 * g + 1] + PR[r][2] * means[3 * g + 2] + Pt[r];
    // Hamilton product q_w = q_P * q/|q|
    const double* qf = quats + 4 * g;
    const double qn = std::sqrt(qf[0] * qf[0] + qf[1] * qf[1] + qf[2] * qf[2] + qf[3] * qf[3]);
    const double w2 = qf[0] / qn, x2 = qf[1] / qn, y2 = qf[2] / qn, z2 = qf[3] / qn;
    const double w1 = qp[0], x1 = qp[1], y1 = qp[2], z1 = qp[3];
    const double qw[4] = {w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                          w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2};
    const double ls[3] = {log_scales[3 * g], log_scales[3 * g + 1], log_scales[3 * g + 2]};
    Proj o;
    project_core(cam, V, Vt, mw, ls, qw, opac_logits[g], sh + (size_t)K * 3 * g, sh_deg, lod_r, PR, o);
    double* r = rec + 24 * j;
    r[0] = o.infrustum; r[1] = o.kept; r[2] = o.near_boundary;
    r[3] = o.p[0]; r[4] = o.p[1]; r[5] = o.p[2];
    r[6] = o.u; r[7] = o.v;
    r[8] = o.conic[0]; r[9] = o.conic[1]; r[10] = o.conic[2];
    r[11] = o.opacity; r[12] = o.rgb[0]; r[13] = o.rgb[1]; r[14] = o.rgb[2];
    r[15] = o.radius;
    r[16] = o.rect[0]; r[17] = o.rect[1]; r[18] = o.rect[2]; r[19] = o.rect[3];
    r[20] = o.sigma_lod; r[21] = (double)(float)o.p[2]; r[22] = k; r[23] = (double)g;
  }
}

// Alpha blending, Eq. 2, brute force and untiled: for every pixel, walk ALL
// splats in global front-to-back order and blend those whose tile rectangle
// contains the pixel's tile. Pixel (x, y) is sampled at (x + 0.5, y + 0.5).
// out_rgb is planar [3,H,W]; background bg[3] is composited with the final T.
void orc_render(int W, int H, int n, const double* u, const double* v, const double* conic,
                const double* opac, const double* rgb, const float* depth32, const int64_t* order,
                const int32_t* rect, const double* bg, double* out_rgb, double* out_T,
                int32_t* out_ncontrib, int32_t* out_flag) {
  SplatView s{n, u, v, conic, opac, rgb, depth32, order, rect};
  const std::vector<int> all = depth_order(s);
  const int gx = (W + kTile - 1) / kTile, gy = (H + kTile - 1) / kTile;
  // every pixel of a tile has the same list (the Gaussians whose rectangle
  // contains the tile, in global depth order): it is gathered once per tile
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < gx * gy; ++t) {
    const int tx = t % gx, ty = t / gx;
    PixelTrace tr;
    std::vector<int> list;
    for (int i : all)
      if (covers(rect + 4 * i, tx, ty)) list.push_back(i);
    for (int py = ty * kTile; py < std::min(H, (ty + 1) * kTile); ++py)
      for (int px = tx * kTile; px < std::min(W, (tx + 1) * kTile); ++px) {
        blend_pixel(s, list, px + 0.5, py + 0.5, tr);
        double C[3] = {0, 0, 0};
        for (size_t c = 0; c < tr.contrib.size(); ++c) {
          const int i = tr.list[tr.contrib[c]];
          for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * i + ch] * tr.alpha[c] * tr.T[c];
        }
        const size_t pix = (size_t)py * W + px;
        for (int ch = 0; ch < 3; ++ch) out_rgb[(size_t)ch * W * H + pix] = C[ch] + tr.Tfinal * bg[ch];
        out_T[pix] = tr.Tfinal;
        out_ncontrib[pix] = tr.n_contrib;
        out_flag[pix] = tr.flag;
      }
  }
}

// The tiled form of the same blend, written out the way a rasteriser does it:
// one key per (tile, splat) pair, key = (tile_base + tile id) << 32 | bits of
// the FP32 depth, a stable sort, then per-tile ranges. Returns the number of
// pairs; keys/vals must hold that many (query with keys == null first).
int64_t orc_tile_keys(int W, int H, int n, const float* depth32, const int32_t* rect,
                      int64_t tile_base, uint64_t* keys, int32_t* vals, int64_t* ranges /*[tiles,2]*/) {
  const int gx = (W + kTile - 1) / kTile, gy = (H + kTile - 1) / kTile;
  std::vector<std::pair<uint64_t, int32_t>> kv;
  for (int i = 0; i < n; ++i) {
    const int32_t* r = rect + 4 * i;
    uint32_t bits;
    std::memcpy(&bits, depth32 + i, 4);
    for (int ty = r[1]; ty < r[3]; ++ty)
      for (int tx = r[0]; tx < r[2]; ++tx) {
        const uint64_t tile = (uint64_t)(tile_base + (int64_t)ty * gx + tx);
        kv.push_back({(tile << 32) | bits, i});
      }
  }
  if (!keys) return (int64_t)kv.size();
  std::stable_sort(kv.begin(), kv.end(),
                   [](const std::pair<uint64_t, int32_t>& a, const std::pair<uint64_t, int32_t>& b) {
                     return a.first < b.first;
                   });
  for (size_t i = 0; i < kv.size(); ++i) { keys[i] = kv[i].first; vals[i] = kv[i].second; }
  if (ranges) {
    for (int64_t t = 0; t < (int64_t)gx * gy; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (size_t i = 0; i < kv.size(); ++i) {
      const int64_t t = (int64_t)(kv[i].first >> 32) - tile_base;
      if (i == 0 || (kv[i - 1].first >> 32) != (kv[i].first >> 32)) ranges[2 * t] = (int64_t)i;
      ranges[2 * t + 1] = (int64_t)i + 1;
    }
  }
  return (int64_t)kv.size();
}

void orc_render_tiled(int W, int H, int n, const double* u, const double* v, const double* conic,
                      const double* opac, const double* rgb, const float* depth32,
                      const int32_t* rect, const double* bg, double* out_rgb, double* out_T,
                      int32_t* out_ncontrib) {
  const int gx = (W + kTile - 1) / kTile, gy = (H + kTile - 1) / kTile;
  const int64_t m = orc_tile_keys(W, H, n, depth32, rect, 0, nullptr, nullptr, nullptr);
  std::vector<uint64_t> keys(m);
  std::vector<int32_t> vals(m);
  std::vector<int64_t> ranges(2 * (size_t)gx * gy);
  orc_tile_keys(W, H, n, depth32, rect, 0, keys.data(), vals.data(), ranges.data());
  std::vector<int64_t> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  SplatView s{n, u, v, conic, opac, rgb, depth32, order.data(), rect};
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < gx * gy; ++t) {
    std::vector<int> list;
    for (int64_t k = ranges[2 * t]; k < ranges[2 * t + 1]; ++k) list.push_back(vals[k]);
    PixelTrace tr;
    const int tx = t % gx, ty = t / gx;
    for (int py = ty * kTile; py < std::min(H, (ty + 1) * kTile); ++py)
      for (int px = tx * kTile; px < std::min(W, (tx + 1) * kTile); ++px) {
        blend_pixel(s, list, px + 0.5, py + 0.5, tr);
        double C[3] = {0, 0, 0};
        for (size_t c = 0; c < tr.contrib.size(); ++c) {
          const int i = tr.list[tr.contrib[c]];
          for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * i + ch] * tr.alpha[c] * tr.T[c];
        }
        const size_t pix = (size_t)py * W + px;
        for (int ch = 0; ch < 3; ++ch) out_rgb[(size_t)ch * W * H + pix] = C[ch] + tr.Tfinal * bg[ch];
        out_T[pix] = tr.Tfinal;
        out_ncontrib[pix] = tr.n_contrib;
      }
  }
}

// Gradient of sum(dL_dimg * image) w.r.t. each splat's (u, v), conic, opacity
// and rgb, for one view. Uses the stored contributor list of each pixel and
// the exact derivative of Eq. 2 (front-to-back products, back-to-front sums).
// Outputs are accumulated (+=). g_flag[pix] marks pixels with a decision near
// its threshold (the same events as orc_render).
void orc_render_backward(int W, int H, int n, const double* u, const double* v,
                         const double* conic, const double* opac, const double* rgb,
                         const float* depth32, const int64_t* order, const int32_t* rect,
                         const double* bg, const double* dL_dimg, double* g_uv, double* g_conic,
                         double* g_opac, double* g_rgb, int32_t* out_flag) {
  SplatView s{n, u, v, conic, opac, rgb, depth32, order, rect};
  const std::vector<int> all = depth_order(s);
  const int gx = (W + kTile - 1) / kTile, gy = (H + kTile - 1) / kTile;
  // per-tile lists (the same lists the untiled walk produces)
  std::vector<std::vector<int>> lists((size_t)gx * gy);
  for (int i : all)
    for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
      for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) lists[(size_t)ty * gx + tx].push_back(i);
#ifdef _OPENMP
  const int nt = omp_get_max_threads();
#else
  const int nt = 1;
#endif
  std::vector<std::vector<double>> acc(nt, std::vector<double>((size_t)n * 9, 0.0));
#pragma omp parallel for schedule(dynamic, 4)
  for (int py = 0; py < H; ++py) {
#ifdef _OPENMP
    std::vector<double>& a = acc[omp_get_thread_num()];
#else
    std::vector<double>& a = acc[0];
#endif
    PixelTrace tr;
    for (int px = 0; px < W; ++px) {
      const size_t pix = (size_t)py * W + px;
      blend_pixel(s, lists[(size_t)(py / kTile) * gx + px / kTile], px + 0.5, py + 0.5, tr);
      if (out_flag) out_flag[pix] = tr.flag;
      const double dC[3] = {dL_dimg[pix], dL_dimg[(size_t)W * H + pix], dL_dimg[2 * (size_t)W * H + pix]};
      const int m = (int)tr.contrib.size();
      // suffix[k] = sum_{i>k} c_i alpha_i T_i  (per channel)
      double suffix[3] = {0, 0, 0};
      for (int c = m - 1; c >= 0; --c) {
        const int i = tr.list[tr.contrib[c]];
        const double al = tr.alpha[c], T = tr.T[c];
        double dalpha = 0;
        for (int ch = 0; ch < 3; ++ch) {
          dalpha += dC[ch] * (rgb[3 * i + ch] * T - suffix[ch] / (1.0 - al) - tr.Tfinal * bg[ch] / (1.0 - al));
          a[9 * (size_t)i + 6 + ch] += al * T * dC[ch];
        }
        for (int ch = 0; ch < 3; ++ch) suffix[ch] += rgb[3 * i + ch] * al * T;
        if (tr.capped[c]) continue;  // alpha = 0.99 is constant there
        const double G = tr.G[c];
        a[9 * (size_t)i + 5] += G * dalpha;                   // d/d opacity
        const double dpow = opac[i] * dalpha * G;             // dL/dpower
        const double dx = u[i] - (px + 0.5), dy = v[i] - (py + 0.5);
        const double A = conic[3 * i], B = conic[3 * i + 1], C = conic[3 * i + 2];
        a[9 * (size_t)i + 0] += dpow * (-A * dx - B * dy);
        a[9 * (size_t)i + 1] += dpow * (-C * dy - B * dx);
        a[9 * (size_t)i + 2] += dpow * (-0.5 * dx * dx);
        a[9 * (size_t)i + 3] += dpow * (-dx * dy);
        a[9 * (size_t)i + 4] += dpow * (-0.5 * dy * dy);
      }
    }
  }
  for (int th = 0; th < nt; ++th)
    for (int i = 0; i < n; ++i) {
      const double* a = &acc[th][9 * (size_t)i];
      g_uv[2 * i] += a[0]; g_uv[2 * i + 1] += a[1];
      g_conic[3 * i] += a[2]; g_conic[3 * i + 1] += a[3]; g_conic[3 * i + 2] += a[4];
      g_opac[i] += a[5];
      g_rgb[3 * i] += a[6]; g_rgb[3 * i + 1] += a[7]; g_rgb[3 * i + 2] += a[8];
    }
}

// The same blend for a chosen set of pixels only: the tile lists are built
// just for the tiles those pixels lie in. For spot checks at full size.
void orc_render_pixels(int W, int H, int n, const double* u, const double* v, const double* conic,
                       const double* opac, const double* rgb, const float* depth32,
                       const int64_t* order, const int32_t* rect, const double* bg, int n_pix,
                       const int32_t* px, const int32_t* py, double* out_rgb /*[n_pix,3]*/,
                       double* out_T, int32_t* out_ncontrib, int32_t* out_flag) {
  SplatView s{n, u, v, conic, opac, rgb, depth32, order, rect};
  const std::vector<int> all = depth_order(s);
#pragma omp parallel for schedule(dynamic, 1)
  for (int q = 0; q < n_pix; ++q) {
    const int tx = px[q] / kTile, ty = py[q] / kTile;
    std::vector<int> list;
    for (int i : all)
      if (covers(rect + 4 * i, tx, ty)) list.push_back(i);
    PixelTrace tr;
    blend_pixel(s, list, px[q] + 0.5, py[q] + 0.5, tr);
    double C[3] = {0, 0, 0};
    for (size_t c = 0; c < tr.contrib.size(); ++c) {
      const int i = tr.list[tr.contrib[c]];
      for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * i + ch] * tr.alpha[c] * tr.T[c];
    }
    for (int ch = 0; ch < 3; ++ch) out_rgb[3 * q + ch] = C[ch] + tr.Tfinal * bg[ch];
    out_T[q] = tr.Tfinal;
    out_ncontrib[q] = tr.n_contrib;
    out_flag[q] = tr.flag;
  }
  (void)W; (void)H;
}

// Gradient of sum_q dL[q] . image(px[q], py[q]) w.r.t. the splats, for a
// chosen set of pixels (accumulated, same layout as orc_render_backward).
void orc_render_backward_pixels(int n, const double* u, const double* v, const double* conic,
                                const double* opac, const double* rgb, const float* depth32,
                                const int64_t* order, const int32_t* rect, const double* bg,
                                int n_pix, const int32_t* px, const int32_t* py,
                                const double* dL /*[n_pix,3]*/, double* g_uv, double* g_conic,
                                double* g_opac, double* g_rgb) {
  SplatView s{n, u, v, conic, opac, rgb, depth32, order, rect};
  const std::vector<int> all = depth_order(s);
  for (int q = 0; q < n_pix; ++q) {
    const int tx = px[q] / kTile, ty = py[q] / kTile;
    std::vector<int> list;
    for (int i : all)
      if (covers(rect + 4 * i, tx, ty)) list.push_back(i);
    PixelTrace tr;
    const double fx = px[q] + 0.5, fy = py[q] + 0.5;
    blend_pixel(s, list, fx, fy, tr);
    const double* dC = dL + 3 * q;
    const int m = (int)tr.contrib.size();
    double suffix[3] = {0, 0, 0};
    for (int c = m - 1; c >= 0; --c) {
      const int i = tr.list[tr.contrib[c]];
      const double al = tr.alpha[c], T = tr.T[c];
      double dalpha = 0;
      for (int ch = 0; ch < 3; ++ch) {
        dalpha += dC[ch] * (rgb[3 * i + ch] * T - suffix[ch] / (1.0 - al) - tr.Tfinal * bg[ch] / (1.0 - al));
        g_rgb[3 * i + ch] += al * T * dC[ch];
      }
      for (int ch = 0; ch < 3; ++ch) suffix[ch] += rgb[3 * i + ch] * al * T;
      if (tr.capped[c]) continue;
      const double G = tr.G[c];
      g_opac[i] += G * dalpha;
      const double dpow = opac[i] * dalpha * G;
      const double dx = u[i] - fx, dy = v[i] - fy;
      const double A = conic[3 * i], B = conic[3 * i + 1], C = conic[3 * i + 2];
      g_uv[2 * i] += dpow * (-A * dx - B * dy);
      g_uv[2 * i + 1] += dpow * (-C * dy - B * dx);
      g_conic[3 * i] += dpow * (-0.5 * dx * dx);
      g_conic[3 * i + 1] += dpow * (-dx * dy);
      g_conic[3 * i + 2] += dpow * (-0.5 * dy * dy);
    }
  }
}

// Projection backward for one view: from the splat gradients of the kept
// selected Gaussians (arrays indexed like `sel`, zero where not kept) to the
// parameter gradients (accumulated, full-size arrays indexed by gid), the
// composed-matrix gradient g_M[(n_inst+1),12] of this view, and the pose
// gradients g_inst_q[n_inst,4], g_inst_t[n_inst,3] (accumulated).
void orc_project_backward(int64_t n_sel, const int64_t* sel, const double* means,
                          const double* log_scales, const double* quats, const double* opac_logits,
                          const double* sh, int sh_deg, const int64_t* inst_off, int n_inst,
                          const double* inst_q, const double* inst_t, const double* cam_raw,
                          double lod_r, int view, const double* g_uv, const double* g_conic,
                          const double* g_opac, const double* g_rgb, double* g_means,
                          double* g_log_scales, double* g_quats, double* g_opac_logits,
                          double* g_sh, double* g_M, double* g_inst_q, double* g_inst_t) {
  const Cam cam = load_cam(cam_raw);
  const int K = (sh_deg + 1) * (sh_deg + 1);
  std::vector<double> As((n_inst + 1) * 9), bs((n_inst + 1) * 3), Ps((n_inst + 1) * 12);
  for (int k = 0; k <= n_inst; ++k) {
    double P[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0}, A[3][3], b[3];
    if (k > 0) pose_matrix(inst_q + 4 * (k - 1), inst_t + 3 * (k - 1), P);
    compose(cam, k > 0 ? P : nullptr, A, b);
    for (int i = 0; i < 9; ++i) As[9 * k + i] = A[i / 3][i % 3];
    for (int i = 0; i < 3; ++i) bs[3 * k + i] = b[i];
    for (int i = 0; i < 12; ++i) Ps[12 * k + i] = P[i];
  }
  std::vector<double> gM((size_t)(n_inst + 1) * 12, 0.0);
  for (int64_t j = 0; j < n_sel; ++j) {
    const int64_t g = sel[j];
    const int k = instance_of(inst_off, n_inst, g);
    double A[3][3], b[3];
    for (int i = 0; i < 9; ++i) A[i / 3][i % 3] = As[9 * k + i];
    for (int i = 0; i < 3; ++i) b[i] = bs[3 * k + i];
    Proj o;
    double mu_used[3];
    project_lod(cam, A, b, g, view, means + 3 * g, log_scales + 3 * g, quats + 4 * g,
                opac_logits[g], sh + (size_t)K * 3 * g, sh_deg, lod_r, o, mu_used);
    if (!o.kept) continue;
    // a splat re-projected outside the frustum has no tiles and no adjoint
    if (o.offset && (o.rect[2] - o.rect[0]) * (o.rect[3] - o.rect[1]) <= 0) continue;
    // the noisy offset is a drawn constant: the adjoint of the noisy mean is
    // that of the mean (no derivative through its depth-dependent scale)
    ProjGrad pg;
    project_one_backward(cam, o, mu_used, sh + (size_t)K * 3 * g, sh_deg, g_uv + 2 * j,
                         g_conic + 3 * j, g_opac[j], g_rgb + 3 * j, pg);
    for (int i = 0; i < 3; ++i) g_means[3 * g + i] += pg.mean[i];
    for (int i = 0; i < 3; ++i) g_log_scales[3 * g + i] += pg.log_scale[i];
    for (int i = 0; i < 4; ++i) g_quats[4 * g + i] += pg.quat[i];
    g_opac_logits[g] += pg.opac_logit;
    for (int kk = 0; kk < K; ++kk)
      for (int ch = 0; ch < 3; ++ch) g_sh[((size_t)g * K + kk) * 3 + ch] += pg.sh[kk][ch];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) gM[12 * k + 4 * r + c] += pg.dA[r][c];
      gM[12 * k + 4 * r + 3] += pg.db[r];
    }
  }
  for (size_t i = 0; i < gM.size(); ++i) g_M[i] += gM[i];
  // M = V P: dP_rot = V_rot^T dA, dP_t = V_rot^T db; then P_rot = R(q_inst)
  for (int k = 1; k <= n_inst; ++k) {
    double dPr[3][3], dPt[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int m = 0; m < 3; ++m) acc += cam.V[m][r] * gM[12 * k + 4 * m + c];
        dPr[r][c] = acc;
      }
      double acc = 0;
      for (int m = 0; m < 3; ++m) acc += cam.V[m][r] * gM[12 * k + 4 * m + 3];
      dPt[r] = acc;
    }
    const double* q = inst_q + 4 * (k - 1);
    double qd[4] = {q[0], q[1], q[2], q[3]}, dq[4];
    quat_rot_backward(qd, dPr, dq);
    for (int i = 0; i < 4; ++i) g_inst_q[4 * (k - 1) + i] += dq[i];
    for (int i = 0; i < 3; ++i) g_inst_t[3 * (k - 1) + i] += dPt[i];
  }
}

// Real SH basis values (and gradients, dY may be null) at a unit direction,
// exported so that tests can pin the basis by quadrature over the sphere.
void orc_sh_basis(const double* dir, double* Y, double* dY) {
  double d[3] = {dir[0], dir[1], dir[2]}, dYl[16][3];
  sh_basis(d, Y, dY ? dYl : nullptr);
  if (dY)
    for (int k = 0; k < 16; ++k)
      for (int r = 0; r < 3; ++r) dY[3 * k + r] = dYl[k][r];
}

// One Adam step (Kingma and Ba, "Adam: A Method for Stochastic
// Optimization", Algorithm 1), in the form PyTorch's Adam uses without weight
// decay: the first and second moment estimates are updated, bias-corrected by
// 1 - beta^step, and the parameter moves by lr * mhat / (sqrt(vhat) + eps).
// The paper reuses its baseline's optimiser and states none of this.
void orc_adam_step(int64_t n, double* p, const double* g, double* m, double* v, double lr,
                   double beta1, double beta2, double eps, int step) {
  const double bc1 = 1.0 - std::pow(beta1, step);
  const double bc2 = 1.0 - std::pow(beta2, step);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    const double mhat = m[i] / bc1;
    const double vhat = v[i] / bc2;
    p[i] -= lr * mhat / (std::sqrt(vhat) + eps);
  }
}

// Stochastic LOD of Eq. 7: mode 0 = deterministic threshold cull, 1 = Eq. 7
// on the Gaussians below r. key = the generator seed, epoch = the counter
// word that distinguishes calls.
void orc_set_lod(int mode, double p_max, double dist, double ox, double oy, double oz,
                 uint32_t key0, uint32_t key1, uint32_t epoch) {
  g_lod.mode = mode;
  g_lod.p_max = (float)p_max;
  g_lod.dist = (float)dist;
  g_lod.offset[0] = ox; g_lod.offset[1] = oy; g_lod.offset[2] = oz;
  g_lod.key[0] = key0; g_lod.key[1] = key1;
  g_lod.epoch = epoch;
}

// Philox4x32-10 of one counter under one key (for pinning the generator).
void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

void orc_set_margins(double alpha_tol, double T_tol, double power_tol) {
  g_tol_alpha = alpha_tol; g_tol_T = T_tol; g_tol_power = power_tol;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
