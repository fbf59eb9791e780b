// Host side of the C ABI declared in include/s3r.h: workspace allocation,
// argument validation, the per-call camera set, and the entry points that
// sequence the kernels. Everything here is asynchronous on the caller's
// stream except s3r_workspace_create/destroy, s3r_query_counts and
// s3r_sync_status.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>

#include "s3r_internal.cuh"

#ifndef S3R_ARCH
#define S3R_ARCH 0
#endif

using namespace s3r;

namespace {

thread_local std::string g_last_error;

s3r_status fail(s3r_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
s3r_status fail(s3r_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

s3r_status cuda_fail(cudaError_t e, const char* where) {
  return fail(S3R_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Sets the workspace's device current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
cudaError_t alloc(s3r_workspace* ws, T** p, int64_t count) {
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  ws->bytes += (int64_t)bytes;
  return cudaMalloc((void**)p, bytes);
}

const char* const kKernelNames[kKCount] = {
    "temporal_compact", "project", "splat_scan", "project_splats", "sort_depth_pass0", "sort_depth_pass1",
    "sort_depth_pass2", "sort_depth_pass3", "duplicate", "sort_tile_pass0", "sort_tile_pass1",
    "sort_tile_pass2", "sort_tile_pass3", "tile_ranges", "duplicate_expand", "blend_fwd",
    "zero_splat_grads", "blend_bwd", "project_bwd", "splat_tiles"};

void free_all(s3r_workspace* ws) {
  for (int i = 0; i < 2 * kKCount; ++i)
    if (ws->ev[i]) cudaEventDestroy(ws->ev[i]);
  void* ptrs[] = {ws->ctr, ws->hist, ws->lookback, ws->selected, ws->frustum_mask,
                  ws->keep_mask, ws->splat_start, ws->kept_list, ws->kept_bits, ws->sp_rgb_d,
                  ws->sp_rect, ws->sp_view, ws->sp_tin, ws->depth_key[0], ws->depth_key[1],
                  ws->depth_val[0], ws->depth_val[1], ws->dup_key[0], ws->dup_key[1],
                  ws->dup_val[0], ws->dup_val[1], ws->ranges, ws->final_T, ws->n_contrib,
                  ws->sp_grad, ws->pose_dM, ws->world_acc, ws->mats, ws->dup_excl, ws->dup_meta, ws->sp_tiles, ws->sp_region, ws->row_spans, ws->dup_chunk, ws->tile_class_cnt, ws->tile_class_list, ws->contrib};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// Dynamic shared memory the projection kernels need for n_views x segments.
size_t proj_smem_bytes(int n_views, int n_inst) {
  return (size_t)n_views * (n_inst + 1) * (80 + 48) + 4 * (size_t)(n_inst + 2) + 16;
}

s3r_status check_scene(const s3r_workspace* ws, const s3r_scene* sc) {
  if (!sc) return fail(S3R_ERR_INVALID, "scene is NULL");
  if (sc->n < 0 || sc->n > ws->cap.max_gaussians)
    return fail(S3R_ERR_INVALID, "scene n=%lld outside [0, %lld]", (long long)sc->n,
                (long long)ws->cap.max_gaussians);
  if (sc->n > 0xffffffffLL) return fail(S3R_ERR_INVALID, "scene n must be < 2^32");
  if (sc->sh_degree < 0 || sc->sh_degree > 3)
    return fail(S3R_ERR_INVALID, "sh_degree %d outside [0, 3]", sc->sh_degree);
  if (sc->n_inst < 0 || sc->n_inst > ws->cap.max_instances)
    return fail(S3R_ERR_INVALID, "n_inst %d outside [0, %d]", sc->n_inst, ws->cap.max_instances);
  if (!sc->inst_offsets) return fail(S3R_ERR_INVALID, "inst_offsets is NULL");
  if (sc->n > 0) {
    if (!sc->means || !sc->log_scales || !sc->quats || !sc->opacity_logits || !sc->sh)
      return fail(S3R_ERR_INVALID, "a scene array is NULL");
    if (!aligned(sc->means, 4) || !aligned(sc->log_scales, 4) || !aligned(sc->opacity_logits, 4))
      return fail(S3R_ERR_INVALID, "means/log_scales/opacity_logits must be 4-byte aligned");
    if (!aligned(sc->quats, 16) || !aligned(sc->sh, 16))
      return fail(S3R_ERR_INVALID, "quats and sh must be 16-byte aligned");
  }
  if (!aligned(sc->inst_offsets, 8)) return fail(S3R_ERR_INVALID, "inst_offsets must be 8-byte aligned");
  return S3R_OK;
}

s3r_status check_poses(const s3r_scene* sc, const s3r_poses* poses) {
  if (sc->n_inst == 0) return S3R_OK;
  if (!poses || !poses->quat || !poses->trans)
    return fail(S3R_ERR_INVALID, "poses are required when n_inst > 0");
  if (!aligned(poses->quat, 16) || !aligned(poses->trans, 4))
    return fail(S3R_ERR_INVALID, "pose quaternions must be 16-byte aligned");
  return S3R_OK;
}

}  // namespace

namespace s3r {
s3r_status set_last_error(s3r_status st, const char* msg) {
  g_last_error = msg;
  return st;
}

int sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}
}  // namespace s3r

extern "C" {

const char* s3r_last_error(void) { return g_last_error.c_str(); }
int32_t s3r_version(void) { return 10000; }
int32_t s3r_built_arch(void) { return S3R_ARCH; }

s3r_status s3r_workspace_create(const s3r_capacity* cap, int device, s3r_workspace** out) {
  if (!cap || !out) return fail(S3R_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (cap->max_gaussians < 1 || cap->max_splats < 1 || cap->max_duplicates < 1 ||
      cap->max_views < 1 || cap->max_views > S3R_MAX_VIEWS || cap->max_instances < 0 ||
      cap->max_tiles < 1 || cap->max_pixels < 1 || cap->max_rows < 0)
    return fail(S3R_ERR_INVALID, "capacities must be positive and max_views <= %d", S3R_MAX_VIEWS);
  if (cap->max_gaussians > 0xffffffffLL || cap->max_splats > 0xffffffffLL ||
      cap->max_duplicates > 0x7fffffffLL || cap->max_tiles > 0x7fffffffLL ||
      cap->max_pixels > 0x7fffffffLL)
    return fail(S3R_ERR_INVALID, "capacity beyond the 32-bit index range");
  DeviceGuard g(device);
  if (!g.ok) return fail(S3R_ERR_CUDA, "cannot select device %d", device);
  s3r_workspace* ws = new s3r_workspace();
  memset(ws, 0, sizeof(*ws));
  ws->lod = s3r_lod_params{S3R_LOD_THRESHOLD, 0.f, 1.f, {0.f, 0.f, 0.f}, 0u};
  ws->device = device;
  ws->cap = *cap;
  cudaError_t e = cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    delete ws;
    return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  const int64_t N = cap->max_gaussians, S = cap->max_splats, K = cap->max_duplicates;
  const int64_t sort_n = S > K ? S : K;
  int64_t lb = (sort_n + kSortTileKeys - 1) / kSortTileKeys * kRadix;
  const int64_t lb_scan = (N > S ? N : S) / 256 + 1;
  if (lb_scan > lb) lb = lb_scan;
  ws->lookback_words = lb + 1024;
  const int nk = cap->max_instances + 1;
#define S3R_ALLOC(ptr, count)                                   \
  if ((e = alloc(ws, &(ptr), (count))) != cudaSuccess) {        \
    free_all(ws);                                               \
    delete ws;                                                  \
    return cuda_fail(e, "cudaMalloc " #ptr);                    \
  }
  S3R_ALLOC(ws->ctr, kCtrCount);
  S3R_ALLOC(ws->hist, kHistCount * kRadix);
  S3R_ALLOC(ws->lookback, ws->lookback_words);
  S3R_ALLOC(ws->selected, N);
  S3R_ALLOC(ws->frustum_mask, N);
  S3R_ALLOC(ws->keep_mask, N);
  S3R_ALLOC(ws->splat_start, N);
  S3R_ALLOC(ws->kept_list, N);
  ws->kept_words = (N + 4095) / 4096 * 128;   // whole compaction tiles
  S3R_ALLOC(ws->kept_bits, ws->kept_words);
  S3R_ALLOC(ws->sp_rgb_d, S);
  S3R_ALLOC(ws->sp_rect, S);
  S3R_ALLOC(ws->sp_view, S);
  S3R_ALLOC(ws->sp_tin, 8 * S);
  S3R_ALLOC(ws->depth_key[0], S);
  S3R_ALLOC(ws->depth_key[1], S);
  S3R_ALLOC(ws->depth_val[0], S);
  S3R_ALLOC(ws->depth_val[1], S);
  S3R_ALLOC(ws->dup_key[0], K);
  S3R_ALLOC(ws->dup_key[1], K);
  S3R_ALLOC(ws->dup_val[0], K);
  S3R_ALLOC(ws->dup_val[1], K);
  S3R_ALLOC(ws->ranges, cap->max_tiles);
  S3R_ALLOC(ws->tile_class_cnt, 64);
  S3R_ALLOC(ws->tile_class_list, (int64_t)kTileClasses * cap->max_tiles);
  S3R_ALLOC(ws->final_T, cap->max_pixels);
  S3R_ALLOC(ws->n_contrib, cap->max_pixels);
  S3R_ALLOC(ws->sp_grad, 12 * S);
  S3R_ALLOC(ws->pose_dM, (int64_t)cap->max_views * nk * 12);
  S3R_ALLOC(ws->world_acc, (int64_t)nk * world_acc_floats());
  S3R_ALLOC(ws->mats, (int64_t)cap->max_views * nk * 20);
  S3R_ALLOC(ws->dup_excl, S + 1);
  S3R_ALLOC(ws->dup_meta, 8 * S);
  S3R_ALLOC(ws->sp_tiles, S);
  S3R_ALLOC(ws->sp_region, 8 * S);
  // about 2.5 rows per splat at 1 px LOD; past the table, rows are recomputed
  ws->rows_cap = std::min<int64_t>(cap->max_rows > 0 ? cap->max_rows : 4 * S, 0xfffffff0LL);
  S3R_ALLOC(ws->row_spans, ws->rows_cap);
  S3R_ALLOC(ws->dup_chunk, K / kDupChunkMin + 2);
  ws->contrib_words = K / 32 + 2;
  S3R_ALLOC(ws->contrib, 4 * ws->contrib_words);
#undef S3R_ALLOC
  for (int i = 0; i < 2 * kKCount; ++i) {
    if ((e = cudaEventCreate(&ws->ev[i])) != cudaSuccess) {
      free_all(ws);
      delete ws;
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  if ((e = cudaMemset(ws->ctr, 0, sizeof(uint32_t) * kCtrCount)) != cudaSuccess ||
      (e = cudaMemset(ws->pose_dM, 0, sizeof(float) * 12 * (size_t)cap->max_views * nk)) != cudaSuccess ||
      (e = cudaMemset(ws->world_acc, 0, sizeof(float) * (size_t)nk * world_acc_floats())) != cudaSuccess ||
      (e = cudaMemset(ws->lookback, 0, sizeof(unsigned long long) * ws->lookback_words)) !=
          cudaSuccess ||
      (e = cudaDeviceSynchronize()) != cudaSuccess) {
    free_all(ws);
    delete ws;
    return cuda_fail(e, "workspace initialisation");
  }
  *out = ws;
  return S3R_OK;
}

s3r_status s3r_workspace_destroy(s3r_workspace* ws) {
  if (!ws) return S3R_OK;
  DeviceGuard g(ws->device);
  free_all(ws);
  delete ws;
  return S3R_OK;
}

int64_t s3r_workspace_bytes(const s3r_workspace* ws) { return ws ? ws->bytes : 0; }

s3r_status s3r_project(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                       const s3r_camera* cams, int32_t n_views, float t,
                       const float* vis_window, float* point_life, float lod_threshold,
                       void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  s3r_status st = check_scene(ws, scene);
  if (st != S3R_OK) return st;
  if ((st = check_poses(scene, poses)) != S3R_OK) return st;
  if (!cams || n_views < 1 || n_views > ws->cap.max_views)
    return fail(S3R_ERR_INVALID, "n_views %d outside [1, %d]", n_views, ws->cap.max_views);
  if (scene->n > 0 && (!vis_window || !aligned(vis_window, 16)))
    return fail(S3R_ERR_INVALID, "vis_window must be a 16-byte aligned [n,2] array");
  if (point_life && !aligned(point_life, 8))
    return fail(S3R_ERR_INVALID, "point_life must be 8-byte aligned");
  if (!std::isfinite(t) || !std::isfinite(lod_threshold))
    return fail(S3R_ERR_INVALID, "t and lod_threshold must be finite");
  if (proj_smem_bytes(n_views, scene->n_inst) > 200 * 1024)
    return fail(S3R_ERR_INVALID, "n_views x (n_inst+1) = %d x %d exceeds the shared-memory budget",
                n_views, scene->n_inst + 1);
  ViewSet vs;
  memset(&vs, 0, sizeof(vs));
  int64_t tiles = 0, pixels = 0;
  for (int v = 0; v < n_views; ++v) {
    const s3r_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 65535 * kTile || c.height > 65535 * kTile ||
        !(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.cx) || !std::isfinite(c.cy))
      return fail(S3R_ERR_INVALID, "camera %d has invalid intrinsics or size", v);
    ViewInfo& vi = vs.v[v];
    vi.width = c.width;
    vi.height = c.height;
    vi.gx = (c.width + kTile - 1) / kTile;
    vi.gy = (c.height + kTile - 1) / kTile;
    vi.tile_base = (int32_t)tiles;
    vi.pix_base = (int32_t)pixels;
    vi.fx = c.fx; vi.fy = c.fy; vi.cx = c.cx; vi.cy = c.cy;
    vi.near_z = c.near_z > 0.f ? c.near_z : 0.2f;
    vi.limx = 1.3f * (0.5f * (float)c.width / c.fx);
    vi.limy = 1.3f * (0.5f * (float)c.height / c.fy);
    vi.jc = c.fx * c.fx * (1.f + vi.limx * vi.limx) + c.fy * c.fy * (1.f + vi.limy * vi.limy);
    for (int i = 0; i < 12; ++i) vi.V[i] = c.world_to_cam[i];
    tiles += (int64_t)vi.gx * vi.gy;
    pixels += (int64_t)c.width * c.height;
  }
  if (tiles > ws->cap.max_tiles || pixels > ws->cap.max_pixels)
    return fail(S3R_ERR_INVALID, "cameras need %lld tiles / %lld pixels, capacity %lld / %lld",
                (long long)tiles, (long long)pixels, (long long)ws->cap.max_tiles,
                (long long)ws->cap.max_pixels);
  vs.n_views = n_views;
  vs.total_tiles = (int32_t)tiles;
  vs.total_pixels = (int32_t)pixels;
  DeviceGuard g(ws->device);
  if (!g.ok) return fail(S3R_ERR_CUDA, "cannot select device %d", ws->device);
  ws->views = vs;
  ws->n_views = n_views;
  ws->n_inst = scene->n_inst;
  ws->sh_degree = scene->sh_degree;
  ws->n = scene->n;
  int bits = 0;
  while (bits < 32 && ((int64_t)1 << bits) < tiles) ++bits;
  ws->tile_passes = (bits + kRadixBits - 1) / kRadixBits;
  ws->stage_done = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = launch_compact(ws, scene, poses, vis_window, t, s)) != cudaSuccess)
    return cuda_fail(e, "temporal selection");
  if ((e = launch_project(ws, scene, poses, t, point_life, lod_threshold, s)) != cudaSuccess)
    return cuda_fail(e, "projection");
  ws->stage_done = 1;
  return S3R_OK;
}

s3r_status s3r_sort(s3r_workspace* ws, void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  if (ws->stage_done != 1)
    return fail(S3R_ERR_STATE, "s3r_sort must follow s3r_project (once per projection)");
  DeviceGuard g(ws->device);
  cudaError_t e = launch_sort(ws, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sort");
  ws->stage_done = 2;
  return S3R_OK;
}

s3r_status s3r_render_fwd(s3r_workspace* ws, const float* background, float* out_rgb,
                          void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  if (ws->stage_done < 2) return fail(S3R_ERR_STATE, "s3r_render_fwd needs s3r_sort first");
  if (!background || !out_rgb || !aligned(background, 4) || !aligned(out_rgb, 4))
    return fail(S3R_ERR_INVALID, "background and out_rgb must be non-NULL float arrays");
  DeviceGuard g(ws->device);
  cudaError_t e = launch_render_fwd(ws, background, out_rgb, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "render forward");
  ws->stage_done = 3;
  return S3R_OK;
}

s3r_status s3r_render_bwd(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                          const float* background, const float* dL_drgb,
                          const s3r_grads* grads, void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  if (ws->stage_done < 3) return fail(S3R_ERR_STATE, "s3r_render_bwd needs s3r_render_fwd first");
  s3r_status st = check_scene(ws, scene);
  if (st != S3R_OK) return st;
  if ((st = check_poses(scene, poses)) != S3R_OK) return st;
  if (scene->n != ws->n || scene->n_inst != ws->n_inst || scene->sh_degree != ws->sh_degree)
    return fail(S3R_ERR_INVALID, "the scene differs from the one of the forward pass");
  if (!background || !dL_drgb || !grads || !aligned(dL_drgb, 4))
    return fail(S3R_ERR_INVALID, "background, dL_drgb and grads must be non-NULL");
  if ((grads->quats && !aligned(grads->quats, 16)) || (grads->sh && !aligned(grads->sh, 16)))
    return fail(S3R_ERR_INVALID, "quaternion and SH gradients must be 16-byte aligned");
  DeviceGuard g(ws->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_render_bwd(ws, background, dL_drgb, grads, s);
  if (e != cudaSuccess) return cuda_fail(e, "render backward");
  e = launch_project_bwd(ws, scene, poses, grads, s);
  if (e != cudaSuccess) return cuda_fail(e, "projection backward");
  return S3R_OK;
}

s3r_status s3r_update_visibility(int64_t n, float t, const uint32_t* mask, float* point_life,
                                 float* vis_window, int32_t mode, void* stream) {
  if (n < 0) return fail(S3R_ERR_INVALID, "n < 0");
  if (mode != S3R_VIS_RECORD && mode != S3R_VIS_FINALIZE && mode != S3R_VIS_RESET)
    return fail(S3R_ERR_INVALID, "unknown mode %d", mode);
  if (n == 0) return S3R_OK;
  if (!point_life || !aligned(point_life, 8))
    return fail(S3R_ERR_INVALID, "point_life must be an 8-byte aligned [n,2] array");
  if (mode != S3R_VIS_RECORD && (!vis_window || !aligned(vis_window, 8)))
    return fail(S3R_ERR_INVALID, "vis_window must be an 8-byte aligned [n,2] array");
  if (mode == S3R_VIS_RECORD && (!mask || !aligned(mask, 4)))
    return fail(S3R_ERR_INVALID, "RECORD needs the M_t bitmask");
  if (!std::isfinite(t)) return fail(S3R_ERR_INVALID, "t must be finite");
  cudaError_t e = launch_visibility(n, t, mask, point_life, vis_window, mode, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "visibility update");
  return S3R_OK;
}

s3r_status s3r_set_timing(s3r_workspace* ws, int32_t enable) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  ws->timing = enable ? 1 : 0;
  return S3R_OK;
}

int32_t s3r_kernel_count(void) { return kKCount; }

const char* s3r_kernel_name(int32_t id) {
  return (id >= 0 && id < kKCount) ? kKernelNames[id] : nullptr;
}

s3r_status s3r_kernel_times(s3r_workspace* ws, float* ms, int32_t n) {
  if (!ws || !ms || n < 0) return fail(S3R_ERR_INVALID, "NULL argument");
  DeviceGuard g(ws->device);
  for (int i = 0; i < n; ++i) {
    ms[i] = -1.f;
    if (i >= kKCount || !ws->ev_used[i]) continue;
    float t = 0.f;
    cudaError_t e = cudaEventElapsedTime(&t, ws->ev[2 * i], ws->ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms[i] = t;
  }
  return S3R_OK;
}

s3r_status s3r_set_grad_mode(s3r_workspace* ws, int32_t mode) {
  if (!ws) return fail(S3R_ERR_INVALID, "NULL workspace");
  if (mode != S3R_GRAD_ACCUMULATE && mode != S3R_GRAD_OVERWRITE)
    return fail(S3R_ERR_INVALID, "gradient mode %d unknown", mode);
  ws->grad_mode = mode;
  return S3R_OK;
}

s3r_status s3r_set_counting(s3r_workspace* ws, int32_t enable) {
  if (!ws) return fail(S3R_ERR_INVALID, "NULL workspace");
  ws->counting = enable ? 1 : 0;
  return S3R_OK;
}

s3r_status s3r_check_wait_timeout(s3r_workspace* ws, int32_t max_polls, void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "NULL workspace");
  if (max_polls < 1 || max_polls > S3R_MAX_PROBE_POLLS)
    return fail(S3R_ERR_INVALID, "max_polls %d outside [1, %d]", (int)max_polls,
                S3R_MAX_PROBE_POLLS);
  DeviceGuard g(ws->device);
  const cudaError_t e = launch_wait_probe(ws, max_polls, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  return S3R_OK;
}

s3r_status s3r_set_lod(s3r_workspace* ws, const s3r_lod_params* params) {
  if (!ws) return fail(S3R_ERR_INVALID, "NULL workspace");
  if (!params) {
    ws->lod = s3r_lod_params{S3R_LOD_THRESHOLD, 0.f, 1.f, {0.f, 0.f, 0.f}, 0u};
    return S3R_OK;
  }
  if (params->mode != S3R_LOD_THRESHOLD && params->mode != S3R_LOD_STOCHASTIC)
    return fail(S3R_ERR_INVALID, "lod mode %d unknown", params->mode);
  if (params->mode == S3R_LOD_STOCHASTIC &&
      (!(params->p_max >= 0.f && params->p_max <= 1.f) || !(params->distance > 0.f) ||
       !std::isfinite(params->distance) || !std::isfinite(params->offset[0]) ||
       !std::isfinite(params->offset[1]) || !std::isfinite(params->offset[2])))
    return fail(S3R_ERR_INVALID, "stochastic LOD needs 0 <= p_max <= 1, distance > 0, finite offsets");
  ws->lod = *params;
  return S3R_OK;
}

s3r_status s3r_adam_step(const s3r_adam_tensor* tensors, int32_t count, float lr, float beta1,
                         float beta2, float eps, int32_t step, const uint32_t* gate,
                         void* stream) {
  if (!tensors || count < 0 || count > S3R_ADAM_MAX_TENSORS)
    return fail(S3R_ERR_INVALID, "adam: 0 <= count <= %d tensors required", S3R_ADAM_MAX_TENSORS);
  if (step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
      !std::isfinite(lr))
    return fail(S3R_ERR_INVALID, "adam: step >= 1, betas in [0, 1), eps > 0 required");
  if (gate && !aligned(gate, 4)) return fail(S3R_ERR_INVALID, "adam: gate must be a device uint32");
  for (int k = 0; k < count; ++k) {
    const s3r_adam_tensor& t = tensors[k];
    if (t.n < 0) return fail(S3R_ERR_INVALID, "adam: tensor %d has n < 0", k);
    if (t.n > 0 && (!t.param || !t.grad || !t.exp_avg || !t.exp_avg_sq || !aligned(t.param, 4) ||
                    !aligned(t.grad, 4) || !aligned(t.exp_avg, 4) || !aligned(t.exp_avg_sq, 4)))
      return fail(S3R_ERR_INVALID, "adam: tensor %d needs four float arrays", k);
  }
  const double bc1 = 1.0 - std::pow((double)beta1, step), bc2 = 1.0 - std::pow((double)beta2, step);
  cudaError_t e = launch_adam(tensors, count, lr, beta1, beta2, eps, (float)bc1, (float)bc2, gate,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "adam");
  return S3R_OK;
}

s3r_status s3r_to_world(const s3r_scene* scene, const s3r_poses* poses, float* means_out,
                        float* quats_out, float* sh_out, void* stream) {
  if (!scene) return fail(S3R_ERR_INVALID, "NULL scene");
  if (scene->n < 0 || scene->n > 0xffffffffLL) return fail(S3R_ERR_INVALID, "n outside [0, 2^32)");
  if (scene->n_inst < 0) return fail(S3R_ERR_INVALID, "n_inst < 0");
  if (scene->sh_degree < 0 || scene->sh_degree > 3)
    return fail(S3R_ERR_INVALID, "sh_degree %d outside [0, 3]", scene->sh_degree);
  if (!scene->inst_offsets || !aligned(scene->inst_offsets, 8))
    return fail(S3R_ERR_INVALID, "inst_offsets must be an 8-byte aligned array");
  if (scene->n == 0 || scene->n_inst == 0) return S3R_OK;
  if (!scene->means || !scene->quats || !means_out || !quats_out)
    return fail(S3R_ERR_INVALID, "means, quats and both outputs are required");
  if (!aligned(scene->means, 4) || !aligned(means_out, 4) || !aligned(scene->quats, 16) ||
      !aligned(quats_out, 16))
    return fail(S3R_ERR_INVALID, "means 4-byte and quaternions 16-byte aligned required");
  if (sh_out && (!scene->sh || !aligned(sh_out, 16) || !aligned(scene->sh, 16)))
    return fail(S3R_ERR_INVALID, "sh_out needs the scene's SH, both 16-byte aligned");
  s3r_status st = check_poses(scene, poses);
  if (st != S3R_OK) return st;
  cudaError_t e = launch_to_world(scene, poses, means_out, quats_out, sh_out, scene->n, sm_count(),
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "to_world");
  return S3R_OK;
}

s3r_status s3r_to_world_bwd(s3r_workspace* ws, const s3r_scene* scene, const s3r_poses* poses,
                            const s3r_grads* grads, void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "workspace is NULL");
  s3r_status st = check_scene(ws, scene);
  if (st != S3R_OK) return st;
  if ((st = check_poses(scene, poses)) != S3R_OK) return st;
  if (!grads) return fail(S3R_ERR_INVALID, "grads is NULL");
  if ((grads->quats && !aligned(grads->quats, 16)) || (grads->means && !aligned(grads->means, 4)) ||
      (grads->sh && !aligned(grads->sh, 16)))
    return fail(S3R_ERR_INVALID, "quaternion and SH gradients must be 16-byte aligned");
  if (scene->n == 0 || scene->n_inst == 0) return S3R_OK;
  DeviceGuard g(ws->device);
  cudaError_t e = launch_to_world_bwd(scene, poses, grads, ws->world_acc, scene->n, ws->num_sms,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "to_world backward");
  return S3R_OK;
}

s3r_status s3r_l1_loss(int64_t n, const float* pred, const float* target, float* dL_dpred,
                       float* loss_out, void* stream) {
  if (n < 0) return fail(S3R_ERR_INVALID, "n < 0");
  if (n == 0) return S3R_OK;
  if (!pred || !target || !dL_dpred || !loss_out || !aligned(pred, 4) || !aligned(target, 4) ||
      !aligned(dL_dpred, 4) || !aligned(loss_out, 4))
    return fail(S3R_ERR_INVALID, "pred, target, dL_dpred and loss_out must be float arrays");
  cudaError_t e = launch_l1_loss(n, pred, target, dL_dpred, loss_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "l1 loss");
  return S3R_OK;
}

int64_t s3r_ode_param_count(int32_t embed_dim) {
  if (embed_dim < 0 || embed_dim > S3R_ODE_MAX_EMBED) return -1;
  return ode_param_count(embed_dim);
}

static s3r_status check_ode(const s3r_ode_net* net, int32_t n_inst, const float* times,
                            int32_t n_times, int32_t substeps, const float* states) {
  if (!net || !net->params || net->embed_dim < 0 || net->embed_dim > S3R_ODE_MAX_EMBED ||
      (net->embed_dim > 0 && !net->embed))
    return fail(S3R_ERR_INVALID, "ode: params, and embed when embed_dim > 0, with embed_dim <= %d",
                S3R_ODE_MAX_EMBED);
  if (n_inst < 0 || n_times < 1 || substeps < 1 || !times || (n_inst > 0 && !states))
    return fail(S3R_ERR_INVALID, "ode: n_inst >= 0, n_times >= 1, substeps >= 1, times and states");
  if ((int64_t)(n_times - 1) * substeps + 1 > 0x7fffffffLL / 6 / (n_inst > 0 ? n_inst : 1))
    return fail(S3R_ERR_INVALID, "ode: trajectory too long");
  if (!aligned(net->params, 4) || !aligned(times, 4) || !aligned(states, 4))
    return fail(S3R_ERR_INVALID, "ode: float arrays required");
  return S3R_OK;
}

s3r_status s3r_ode_poses(const s3r_ode_net* net, int32_t n_inst, const float* z0,
                         const float* times, int32_t n_times, int32_t substeps, float* states,
                         float* quat, float* trans, void* stream) {
  s3r_status st = check_ode(net, n_inst, times, n_times, substeps, states);
  if (st != S3R_OK) return st;
  if (n_inst == 0) return S3R_OK;
  if (!z0 || !quat || !trans || !aligned(quat, 16) || !aligned(trans, 4) || !aligned(z0, 4))
    return fail(S3R_ERR_INVALID, "ode: z0, quat (16-byte aligned) and trans required");
  cudaError_t e = launch_ode_fwd(net, n_inst, z0, times, n_times, substeps, states, quat, trans,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ode forward");
  return S3R_OK;
}

s3r_status s3r_ode_poses_bwd(const s3r_ode_net* net, int32_t n_inst, const float* times,
                             int32_t n_times, int32_t substeps, const float* states,
                             const float* g_quat, const float* g_trans, float* g_params,
                             float* g_embed, float* g_z0, void* stream) {
  s3r_status st = check_ode(net, n_inst, times, n_times, substeps, states);
  if (st != S3R_OK) return st;
  if (n_inst == 0) return S3R_OK;
  if (!g_quat || !g_trans || !g_params || !g_z0 || (net->embed_dim > 0 && !g_embed) ||
      !aligned(g_quat, 16) || !aligned(g_trans, 4) || !aligned(g_params, 4) || !aligned(g_z0, 4))
    return fail(S3R_ERR_INVALID, "ode: the pose adjoints (quaternions 16-byte aligned) and the "
                                 "gradient buffers are required");
  cudaError_t e = launch_ode_bwd(net, n_inst, times, n_times, substeps, states, g_quat, g_trans,
                                 g_params, g_embed, g_z0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "ode backward");
  return S3R_OK;
}

s3r_status s3r_query_counts(s3r_workspace* ws, void* stream, s3r_counts* out) {
  if (!ws || !out) return fail(S3R_ERR_INVALID, "NULL argument");
  DeviceGuard g(ws->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  uint32_t h[kCtrCount];
  if ((e = cudaMemcpy(h, ws->ctr, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy counts");
  out->n_selected = h[kCtrSelected];
  out->n_splats = h[kCtrSplats];
  out->n_duplicates = h[kCtrDups];
  out->n_frustum = h[kCtrFrustum];
  out->n_blend_pairs = (int64_t)((uint64_t)h[kCtrPairs] | ((uint64_t)h[kCtrPairs + 1] << 32));
  out->epoch = h[kCtrEpoch];
  out->n_eval_fwd = (int64_t)((uint64_t)h[kCtrEvalFwd] | ((uint64_t)h[kCtrEvalFwd + 1] << 32));
  out->n_eval_bwd = (int64_t)((uint64_t)h[kCtrEvalBwd] | ((uint64_t)h[kCtrEvalBwd + 1] << 32));
  out->device_status = h[kCtrStatus];
  if (h[kCtrStatus] && (e = cudaMemset(ws->ctr + kCtrStatus, 0, sizeof(uint32_t))) != cudaSuccess)
    return cuda_fail(e, "cudaMemset status");
  return S3R_OK;
}

s3r_status s3r_set_epoch(s3r_workspace* ws, uint32_t epoch, void* stream) {
  if (!ws) return fail(S3R_ERR_INVALID, "NULL workspace");
  DeviceGuard g(ws->device);
  cudaStream_t s = (cudaStream_t)stream;
  // the counter also tags the look-back words: a jump could bring back the
  // tag of an earlier call, so every word is cleared with it
  cudaError_t e = cudaMemsetAsync(ws->lookback, 0, sizeof(unsigned long long) * ws->lookback_words, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync look-back words");
  if ((e = cudaMemcpyAsync(ws->ctr + kCtrEpoch, &epoch, sizeof(epoch), cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync epoch");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return S3R_OK;
}

const uint32_t* s3r_device_status(const s3r_workspace* ws) {
  return ws ? ws->ctr + kCtrStatus : nullptr;
}

s3r_status s3r_sync_status(s3r_workspace* ws, void* stream) {
  s3r_counts c = {};
  s3r_status st = s3r_query_counts(ws, stream, &c);
  if (st != S3R_OK) return st;
  if (c.device_status & kStatusTimeout)
    return fail(S3R_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (c.device_status & kStatusCapacity)
    return fail(S3R_ERR_CAPACITY,
                "capacity exceeded: %lld splats (max %lld), %lld duplicates (max %lld)",
                (long long)c.n_splats, (long long)ws->cap.max_splats, (long long)c.n_duplicates,
                (long long)ws->cap.max_duplicates);
  return S3R_OK;
}

const void* s3r_debug_buffer(const s3r_workspace* ws, const char* name) {
  if (!ws || !name) return nullptr;
  struct {
    const char* n;
    const void* p;
  } table[] = {
      {"selected", ws->selected},
      {"frustum_mask", ws->frustum_mask},
      {"keep_mask", ws->keep_mask},
      {"splat_start", ws->splat_start},
      {"splat_record", ws->sp_tin},
      {"splat_rgb_depth", ws->sp_rgb_d},
      {"splat_rect", ws->sp_rect},
      {"splat_view", ws->sp_view},
      {"sorted_splats", ws->dup_val[ws->dup_final]},
      {"sorted_tiles", ws->dup_key[ws->dup_final]},
      {"tile_ranges", ws->ranges},
      {"final_T", ws->final_T},
      {"n_contrib", ws->n_contrib},
      {"splat_grads", ws->sp_grad},
      {"pose_grad_matrix", ws->pose_dM},
      {"depth_sorted_splats", ws->depth_val[ws->depth_final]},
  };
  for (auto& e : table)
    if (strcmp(e.n, name) == 0) return e.p;
  return nullptr;
}

}  // extern "C"
