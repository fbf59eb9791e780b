// NeuralODE object poses (Sec. 3.2, Eqs. 3-4): the object state
// z(t) = [position, rotation vector] evolves as dz/dt = f(z, t, c), f a
// two-hidden-layer tanh perceptron of width 64 and c the object's instance
// embedding; z at the output times comes from classical fourth-order
// Runge-Kutta steps from z(t0) (`substeps` equal steps between consecutive
// output times), and the pose at each output time is the rotation exp(r) as
// a unit quaternion with the translation z[0:3] (the instance pose of
// Sec. 3.3, local -> world).
//
// One warp per instance, all instances in parallel; the time steps of an
// instance are sequential. Lane l holds hidden units l and l + 32. The
// weights sit in shared memory in the layouts the lanes read without bank
// conflicts (W1 and W2 transposed for the forward, W2 also row-major for the
// backward's W2^T product). The backward walks an instance's steps in
// reverse from the stored states, recomputes each step's four stages and
// accumulates the parameter adjoints in per-warp copies in shared memory,
// summed over the CTA's warps and added to the caller's buffer at the end.
#include "s3r_internal.cuh"

namespace s3r {
namespace {

constexpr int kH = S3R_ODE_HIDDEN;     // hidden width
constexpr int kMaxD = S3R_ODE_MAX_EMBED;
constexpr int kOdeWarps = 4;           // instances per CTA
static_assert(kH == 64, "lanes hold hidden units l and l + 32");

struct OdeLayout {
  int D, I;
  int64_t oW1, ob1, oW2, ob2, oW3, ob3, count;   // offsets in the flat parameter vector
};
__host__ __device__ inline OdeLayout ode_layout(int D) {
  OdeLayout L;
  L.D = D;
  L.I = 7 + D;
  L.oW1 = 0;
  L.ob1 = L.oW1 + (int64_t)kH * L.I;
  L.oW2 = L.ob1 + kH;
  L.ob2 = L.oW2 + (int64_t)kH * kH;
  L.oW3 = L.ob2 + kH;
  L.ob3 = L.oW3 + 6 * kH;
  L.count = L.ob3 + 6;
  return L;
}

// Shared weights: W1t [I][H] (W1t[i][u] = W1[u][i]), b1 [H], W2t [H][H]
// (W2t[j][u] = W2[u][j]), W2 [H][H], b2 [H], W3 [6][H], b3 [6].
struct SW {
  float* W1t;
  float* b1;
  float* W2t;
  float* W2;
  float* b2;
  float* W3;
  float* b3;
};
__host__ __device__ inline int sw_floats(int I) { return I * kH + kH + 2 * kH * kH + kH + 6 * kH + 6; }

__device__ SW load_weights(const float* __restrict__ p, const OdeLayout& L, float* smem) {
  SW w;
  w.W1t = smem;
  w.b1 = w.W1t + L.I * kH;
  w.W2t = w.b1 + kH;
  w.W2 = w.W2t + kH * kH;
  w.b2 = w.W2 + kH * kH;
  w.W3 = w.b2 + kH;
  w.b3 = w.W3 + 6 * kH;
  for (int e = threadIdx.x; e < kH * L.I; e += blockDim.x) {
    const int u = e / L.I, i = e - u * L.I;
    w.W1t[i * kH + u] = p[L.oW1 + e];
  }
  for (int e = threadIdx.x; e < kH * kH; e += blockDim.x) {
    const int u = e / kH, j = e - u * kH;
    const float v = p[L.oW2 + e];
    w.W2t[j * kH + u] = v;
    w.W2[e] = v;
  }
  for (int e = threadIdx.x; e < kH; e += blockDim.x) {
    w.b1[e] = p[L.ob1 + e];
    w.b2[e] = p[L.ob2 + e];
  }
  for (int e = threadIdx.x; e < 6 * kH; e += blockDim.x) w.W3[e] = p[L.oW3 + e];
  for (int e = threadIdx.x; e < 6; e += blockDim.x) w.b3[e] = p[L.ob3 + e];
  return w;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// f(z, t, c) (Eq. 3) for the warp's instance: `out` (6, the same in every
// lane) and the lane's hidden activations h1[2], h2[2] (units l, l + 32).
__device__ __forceinline__ void eval_f(const SW& w, int I, const float (&z)[6], float t,
                                       const float* c, int D, uint32_t lane, float (&out)[6],
                                       float (&h1)[2], float (&h2)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int u = (int)lane + 32 * q;
    float a = w.b1[u];
#pragma unroll
    for (int i = 0; i < 6; ++i) a = fmaf(w.W1t[i * kH + u], z[i], a);
    a = fmaf(w.W1t[6 * kH + u], t, a);
    for (int d = 0; d < D; ++d) a = fmaf(w.W1t[(7 + d) * kH + u], c[d], a);
    h1[q] = tanhf(a);
  }
  // four partial sums per output (inputs j = 4 i + p), so that the chain of
  // dependent FMAs is 16 long instead of 64: the products are latency-bound
  // (one warp per instance walks its steps in sequence)
  float a0[4] = {w.b2[lane], 0.f, 0.f, 0.f}, a1[4] = {w.b2[lane + 32], 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int i = 0; i < kH / 4; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = 4 * i + q;
      const float hj = __shfl_sync(0xffffffffu, h1[j >> 5], j & 31);
      a0[q] = fmaf(w.W2t[j * kH + lane], hj, a0[q]);
      a1[q] = fmaf(w.W2t[j * kH + lane + 32], hj, a1[q]);
    }
  }
  h2[0] = tanhf((a0[0] + a0[1]) + (a0[2] + a0[3]));
  h2[1] = tanhf((a1[0] + a1[1]) + (a1[2] + a1[3]));
#pragma unroll
  for (int o = 0; o < 6; ++o)
    out[o] = w.b3[o] + warp_sum(fmaf(w.W3[o * kH + lane], h2[0], w.W3[o * kH + lane + 32] * h2[1]));
}

// exp(r) as a unit quaternion (w, x, y, z); a series below |r| = 1e-4.
__device__ __forceinline__ float4 quat_from_rotvec(float rx, float ry, float rz) {
  const float th2 = rx * rx + ry * ry + rz * rz;
  float cw, s;
  if (th2 < 1e-8f) {
    cw = 1.f - th2 * 0.125f;
    s = 0.5f - th2 * (1.f / 48.f);
  } else {
    const float th = sqrtf(th2);
    float sn, cs;
    sincosf(0.5f * th, &sn, &cs);
    cw = cs;
    s = sn / th;
  }
  return make_float4(cw, s * rx, s * ry, s * rz);
}

// Adjoint of r for the adjoint g of quat_from_rotvec(r).
__device__ __forceinline__ void quat_from_rotvec_vjp(const float r[3], float4 g, float out[3]) {
  const float th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  const float gv[3] = {g.y, g.z, g.w};
  if (th2 < 1e-8f) {
    // w = 1 - th^2/8, v = (1/2 - th^2/48) r to second order
    const float dot = r[0] * gv[0] + r[1] * gv[1] + r[2] * gv[2];
    for (int i = 0; i < 3; ++i)
      out[i] = -0.25f * r[i] * g.x + (0.5f - th2 * (1.f / 48.f)) * gv[i] - (1.f / 24.f) * r[i] * dot;
    return;
  }
  const float th = sqrtf(th2);
  float sn, cs;
  sincosf(0.5f * th, &sn, &cs);
  const float s = sn / th;
  const float ds = (0.5f * cs * th - sn) / th2;   // d s / d th
  const float dot = r[0] * gv[0] + r[1] * gv[1] + r[2] * gv[2];
  for (int i = 0; i < 3; ++i)
    out[i] = -0.5f * s * r[i] * g.x + s * gv[i] + r[i] * (ds / th) * dot;
}

__device__ __forceinline__ void store6(float* dst, const float (&v)[6], uint32_t lane) {
  float x = v[0];
#pragma unroll
  for (int i = 1; i < 6; ++i) x = (int)lane == i ? v[i] : x;
  if (lane < 6) dst[lane] = x;
}

__device__ __forceinline__ void write_pose(const float (&z)[6], float* quat, float* trans,
                                           uint32_t lane) {
  if (lane == 0) {
    const float4 q = quat_from_rotvec(z[3], z[4], z[5]);
    *reinterpret_cast<float4*>(quat) = q;
    trans[0] = z[0];
    trans[1] = z[1];
    trans[2] = z[2];
  }
}

struct OdeArgs {
  const float* params;
  const float* embed;
  int D, n_inst, n_times, substeps;
  const float* times;
  const float* z0;          // forward
  float* states;            // [(n_times - 1) * substeps + 1][n_inst][6]
  float* quat;              // [n_times][n_inst][4]
  float* trans;             // [n_times][n_inst][3]
  const float* g_quat;      // backward
  const float* g_trans;
  float* g_params;
  float* g_embed;
  float* g_z0;
};

__global__ void __launch_bounds__(32 * kOdeWarps) k_ode_fwd(OdeArgs a) {
  extern __shared__ __align__(16) float smem[];
  const OdeLayout L = ode_layout(a.D);
  const SW w = load_weights(a.params, L, smem);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const int k = blockIdx.x * kOdeWarps + (int)(threadIdx.x >> 5);
  if (k >= a.n_inst) return;
  float c[kMaxD];
  for (int d = 0; d < a.D; ++d) c[d] = a.embed[(size_t)k * a.D + d];
  float z[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) z[i] = a.z0[6 * (size_t)k + i];
  const int K = a.n_inst;
  store6(a.states + 6 * (size_t)k, z, lane);
  write_pose(z, a.quat + 4 * (size_t)k, a.trans + 3 * (size_t)k, lane);
  int step = 0;
  for (int j = 0; j + 1 < a.n_times; ++j) {
    const float t0 = a.times[j];
    const float h = (a.times[j + 1] - t0) / (float)a.substeps;
    for (int s = 0; s < a.substeps; ++s) {
      const float t = t0 + (float)s * h;
      float k1[6], k2[6], k3[6], k4[6], u[6], h1[2], h2[2];
      eval_f(w, L.I, z, t, c, a.D, lane, k1, h1, h2);
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = fmaf(0.5f * h, k1[i], z[i]);
      eval_f(w, L.I, u, t + 0.5f * h, c, a.D, lane, k2, h1, h2);
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = fmaf(0.5f * h, k2[i], z[i]);
      eval_f(w, L.I, u, t + 0.5f * h, c, a.D, lane, k3, h1, h2);
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = fmaf(h, k3[i], z[i]);
      eval_f(w, L.I, u, t + h, c, a.D, lane, k4, h1, h2);
#pragma unroll
      for (int i = 0; i < 6; ++i)
        z[i] = fmaf(h * (1.f / 6.f), k1[i] + 2.f * k2[i] + 2.f * k3[i] + k4[i], z[i]);
      ++step;
      store6(a.states + 6 * ((size_t)step * K + k), z, lane);
    }
    write_pose(z, a.quat + 4 * ((size_t)(j + 1) * K + k), a.trans + 3 * ((size_t)(j + 1) * K + k),
               lane);
  }
}

// Per-warp adjoint accumulators in shared memory: dW1t [I][H], db1 [H],
// dW2t [H][H] (dW2t[j][u] = dW2[u][j]), db2 [H], dW3 [6][H], db3 [6].
__host__ __device__ inline int acc_floats(int I) { return I * kH + kH + kH * kH + kH + 6 * kH + 6; }
struct Acc {
  float* W1t;
  float* b1;
  float* W2t;
  float* b2;
  float* W3;
  float* b3;
};
__device__ __forceinline__ Acc acc_at(float* base, int I) {
  Acc g;
  g.W1t = base;
  g.b1 = g.W1t + I * kH;
  g.W2t = g.b1 + kH;
  g.b2 = g.W2t + kH * kH;
  g.W3 = g.b2 + kH;
  g.b3 = g.W3 + 6 * kH;
  return g;
}

// VJP of f at one stage: adds the parameter adjoints to the warp's
// accumulators and returns the adjoints of z (6) and c (D), uniform in lanes.
__device__ __forceinline__ void vjp_f(const SW& w, const Acc& g, int I, const float (&x6)[6], float t,
                                      const float* c, int D, const float (&h1)[2],
                                      const float (&h2)[2], const float (&yb)[6], uint32_t lane,
                                      float (&zb)[6], float* cb) {
  // layer 3: dW3 += yb h2^T, db3 += yb, hb2 = W3^T yb
  float hb2[2] = {0.f, 0.f};
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    g.W3[o * kH + lane] += yb[o] * h2[0];
    g.W3[o * kH + lane + 32] += yb[o] * h2[1];
    hb2[0] = fmaf(w.W3[o * kH + lane], yb[o], hb2[0]);
    hb2[1] = fmaf(w.W3[o * kH + lane + 32], yb[o], hb2[1]);
  }
  if (lane == 0)
#pragma unroll
    for (int o = 0; o < 6; ++o) g.b3[o] += yb[o];
  const float p2[2] = {hb2[0] * (1.f - h2[0] * h2[0]), hb2[1] * (1.f - h2[1] * h2[1])};
  g.b2[lane] += p2[0];
  g.b2[lane + 32] += p2[1];
  // dW2[u][j] += p2[u] h1[j] (lane owns rows u = l, l + 32); hb1[j] = sum_u W2[u][j] p2[u]
  // (lane owns columns j = l, l + 32)
  // (four partial sums per column, as in eval_f, to shorten the FMA chain)
  float hb1a[4] = {0.f, 0.f, 0.f, 0.f}, hb1b[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int i = 0; i < kH / 4; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = 4 * i + q;
      const float h1m = __shfl_sync(0xffffffffu, h1[m >> 5], m & 31);
      const float p2m = __shfl_sync(0xffffffffu, p2[m >> 5], m & 31);
      g.W2t[m * kH + lane] += p2[0] * h1m;
      g.W2t[m * kH + lane + 32] += p2[1] * h1m;
      hb1a[q] = fmaf(w.W2[m * kH + lane], p2m, hb1a[q]);
      hb1b[q] = fmaf(w.W2[m * kH + lane + 32], p2m, hb1b[q]);
    }
  }
  const float hb1[2] = {(hb1a[0] + hb1a[1]) + (hb1a[2] + hb1a[3]),
                        (hb1b[0] + hb1b[1]) + (hb1b[2] + hb1b[3])};
  const float p1[2] = {hb1[0] * (1.f - h1[0] * h1[0]), hb1[1] * (1.f - h1[1] * h1[1])};
  g.b1[lane] += p1[0];
  g.b1[lane + 32] += p1[1];
  // dW1[u][i] += p1[u] x[i]; xb[i] = sum_u W1[u][i] p1[u]
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    g.W1t[i * kH + lane] += p1[0] * x6[i];
    g.W1t[i * kH + lane + 32] += p1[1] * x6[i];
    zb[i] = warp_sum(fmaf(w.W1t[i * kH + lane], p1[0], w.W1t[i * kH + lane + 32] * p1[1]));
  }
  g.W1t[6 * kH + lane] += p1[0] * t;
  g.W1t[6 * kH + lane + 32] += p1[1] * t;
  for (int d = 0; d < D; ++d) {
    const int i = 7 + d;
    g.W1t[i * kH + lane] += p1[0] * c[d];
    g.W1t[i * kH + lane + 32] += p1[1] * c[d];
    cb[d] += warp_sum(fmaf(w.W1t[i * kH + lane], p1[0], w.W1t[i * kH + lane + 32] * p1[1]));
  }
}

__global__ void __launch_bounds__(32 * kOdeWarps) k_ode_bwd(OdeArgs a) {
  extern __shared__ __align__(16) float smem[];
  const OdeLayout L = ode_layout(a.D);
  const int I = L.I;
  const SW w = load_weights(a.params, L, smem);
  float* acc_base = smem + sw_floats(I);
  const int nacc = acc_floats(I);
  for (int e = threadIdx.x; e < kOdeWarps * nacc; e += blockDim.x) acc_base[e] = 0.f;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  const int k = blockIdx.x * kOdeWarps + warp;
  const Acc g = acc_at(acc_base + warp * nacc, I);
  if (k < a.n_inst) {
    const int K = a.n_inst;
    const int S = a.substeps;
    float c[kMaxD], cb[kMaxD];
    for (int d = 0; d < a.D; ++d) {
      c[d] = a.embed[(size_t)k * a.D + d];
      cb[d] = 0.f;
    }
    float ab[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int n_steps = (a.n_times - 1) * S;
    for (int i = n_steps; i >= 0; --i) {
      if (i % S == 0) {
        // this output time's pose adjoints enter the state's
        const int j = i / S;
        const float* zs = a.states + 6 * ((size_t)i * K + k);
        const float r[3] = {zs[3], zs[4], zs[5]};
        const float4 gq = *reinterpret_cast<const float4*>(a.g_quat + 4 * ((size_t)j * K + k));
        float gr[3];
        quat_from_rotvec_vjp(r, gq, gr);
        const float* gt = a.g_trans + 3 * ((size_t)j * K + k);
        ab[0] += gt[0];
        ab[1] += gt[1];
        ab[2] += gt[2];
        ab[3] += gr[0];
        ab[4] += gr[1];
        ab[5] += gr[2];
      }
      if (i == 0) break;
      const int jj = (i - 1) / S, s = (i - 1) - jj * S;
      const float t0 = a.times[jj];
      const float h = (a.times[jj + 1] - t0) / (float)S;
      const float t = t0 + (float)s * h;
      float z[6];
      const float* zs = a.states + 6 * ((size_t)(i - 1) * K + k);
#pragma unroll
      for (int q = 0; q < 6; ++q) z[q] = zs[q];
      // the step's four stages again, with their hidden activations
      float kk[6], u2[6], u3[6], u4[6];
      float h1a[2], h2a[2], h1b[2], h2b[2], h1c[2], h2c[2], h1d[2], h2d[2];
      eval_f(w, I, z, t, c, a.D, lane, kk, h1a, h2a);
#pragma unroll
      for (int q = 0; q < 6; ++q) u2[q] = fmaf(0.5f * h, kk[q], z[q]);
      eval_f(w, I, u2, t + 0.5f * h, c, a.D, lane, kk, h1b, h2b);
#pragma unroll
      for (int q = 0; q < 6; ++q) u3[q] = fmaf(0.5f * h, kk[q], z[q]);
      eval_f(w, I, u3, t + 0.5f * h, c, a.D, lane, kk, h1c, h2c);
#pragma unroll
      for (int q = 0; q < 6; ++q) u4[q] = fmaf(h, kk[q], z[q]);
      eval_f(w, I, u4, t + h, c, a.D, lane, kk, h1d, h2d);
      // z' = z + h/6 (k1 + 2 k2 + 2 k3 + k4), stages in reverse
      float zb[6], kb[6], xb[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        zb[q] = ab[q];
        kb[q] = h * (1.f / 6.f) * ab[q];
      }
      vjp_f(w, g, I, u4, t + h, c, a.D, h1d, h2d, kb, lane, xb, cb);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        zb[q] += xb[q];
        kb[q] = fmaf(h, xb[q], h * (1.f / 3.f) * ab[q]);
      }
      vjp_f(w, g, I, u3, t + 0.5f * h, c, a.D, h1c, h2c, kb, lane, xb, cb);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        zb[q] += xb[q];
        kb[q] = fmaf(0.5f * h, xb[q], h * (1.f / 3.f) * ab[q]);
      }
      vjp_f(w, g, I, u2, t + 0.5f * h, c, a.D, h1b, h2b, kb, lane, xb, cb);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        zb[q] += xb[q];
        kb[q] = fmaf(0.5f * h, xb[q], h * (1.f / 6.f) * ab[q]);
      }
      vjp_f(w, g, I, z, t, c, a.D, h1a, h2a, kb, lane, xb, cb);
#pragma unroll
      for (int q = 0; q < 6; ++q) ab[q] = zb[q] + xb[q];
    }
    if (lane == 0) {
      for (int q = 0; q < 6; ++q) a.g_z0[6 * (size_t)k + q] += ab[q];
      for (int d = 0; d < a.D; ++d) a.g_embed[(size_t)k * a.D + d] += cb[d];
    }
  }
  __syncthreads();
  // the CTA's sums of the warps' accumulators, added to the caller's buffer
  for (int e = threadIdx.x; e < nacc; e += blockDim.x) {
    float v = 0.f;
    for (int q = 0; q < kOdeWarps; ++q) v += acc_base[q * nacc + e];
    if (v == 0.f) continue;
    int64_t dst;
    if (e < I * kH) {                                   // dW1t[i][u] -> W1[u][i]
      const int i = e / kH, u = e - i * kH;
      dst = L.oW1 + (int64_t)u * I + i;
    } else if (e < I * kH + kH) {
      dst = L.ob1 + (e - I * kH);
    } else if (e < I * kH + kH + kH * kH) {             // dW2t[j][u] -> W2[u][j]
      const int r = e - (I * kH + kH);
      const int j = r / kH, u = r - j * kH;
      dst = L.oW2 + (int64_t)u * kH + j;
    } else if (e < I * kH + 2 * kH + kH * kH) {
      dst = L.ob2 + (e - (I * kH + kH + kH * kH));
    } else if (e < I * kH + 2 * kH + kH * kH + 6 * kH) {
      dst = L.oW3 + (e - (I * kH + 2 * kH + kH * kH));
    } else {
      dst = L.ob3 + (e - (I * kH + 2 * kH + kH * kH + 6 * kH));
    }
    atomicAdd(a.g_params + dst, v);
  }
}

}  // namespace

int64_t ode_param_count(int embed_dim) { return ode_layout(embed_dim).count; }

cudaError_t launch_ode_fwd(const s3r_ode_net* net, int n_inst, const float* z0, const float* times,
                           int n_times, int substeps, float* states, float* quat, float* trans,
                           cudaStream_t st) {
  OdeArgs a = {};
  a.params = net->params;
  a.embed = net->embed;
  a.D = net->embed_dim;
  a.n_inst = n_inst;
  a.n_times = n_times;
  a.substeps = substeps;
  a.times = times;
  a.z0 = z0;
  a.states = states;
  a.quat = quat;
  a.trans = trans;
  const size_t smem = sizeof(float) * (size_t)sw_floats(7 + a.D);
  cudaError_t e = cudaFuncSetAttribute(k_ode_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ode_fwd<<<(n_inst + kOdeWarps - 1) / kOdeWarps, 32 * kOdeWarps, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ode_bwd(const s3r_ode_net* net, int n_inst, const float* times, int n_times,
                           int substeps, const float* states, const float* g_quat,
                           const float* g_trans, float* g_params, float* g_embed, float* g_z0,
                           cudaStream_t st) {
  OdeArgs a = {};
  a.params = net->params;
  a.embed = net->embed;
  a.D = net->embed_dim;
  a.n_inst = n_inst;
  a.n_times = n_times;
  a.substeps = substeps;
  a.times = times;
  a.states = const_cast<float*>(states);
  a.g_quat = g_quat;
  a.g_trans = g_trans;
  a.g_params = g_params;
  a.g_embed = g_embed;
  a.g_z0 = g_z0;
  const int I = 7 + a.D;
  const size_t smem = sizeof(float) * ((size_t)sw_floats(I) + (size_t)kOdeWarps * acc_floats(I));
  cudaError_t e = cudaFuncSetAttribute(k_ode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ode_bwd<<<(n_inst + kOdeWarps - 1) / kOdeWarps, 32 * kOdeWarps, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s3r
