// vr_api.cu -- the C ABI of libvr (argument validation, state, memory, launches).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "vr_internal.h"
#include "vr_output.h"

namespace vr {

static thread_local char g_cuda_err[256] = "";

vr_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return VR_OK;
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
  return VR_ERR_CUDA;
}

vr_status ctx_alloc(vr_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 256;
  if (ctx->alloc) {
    *p = ctx->alloc(bytes, ctx->user);
    return *p ? VR_OK : VR_ERR_OUT_OF_MEMORY;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *p = nullptr;
    return VR_ERR_OUT_OF_MEMORY;
  }
  return cuda_status(e);
}

void ctx_free(vr_ctx* ctx, void* p) {
  if (!p) return;
  if (ctx->free_fn) ctx->free_fn(p, ctx->user);
  else cudaFree(p);
}

// Grow-only buffer: reallocates (without preserving contents) when `bytes` exceeds *cap.
vr_status ensure(vr_ctx* ctx, void** p, size_t* cap, size_t bytes) {
  if (*p && *cap >= bytes) return VR_OK;
  if (*p) {
    cudaDeviceSynchronize();  // the old buffer may still be read by queued work
    ctx_free(ctx, *p);
    *p = nullptr;
    *cap = 0;
  }
  const vr_status st = ctx_alloc(ctx, p, bytes);
  if (st == VR_OK) *cap = bytes;
  return st;
}

// Switches to the context's device for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); prev = -1; }
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static bool finite3(const float v[3]) {
  return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

static int dtype_bytes(vr_dtype t) {
  switch (t) {
    case VR_U8: return 1;
    case VR_U16: return 2;
    case VR_F16: return 2;
    case VR_F32: return 4;
  }
  return 0;
}

VolDev vol_dev(const vr_ctx* ctx) {
  VolDev V;
  V.data = ctx->vol;
  for (int a = 0; a < 3; ++a) {
    V.n[a] = ctx->n[a];
    V.nb[a] = ctx->nb[a];
  }
  V.px = ctx->px;
  V.py = ctx->py;
  V.pxy = ctx->px * ctx->py;
  V.value_max = ctx->value_max;
  V.vis = ctx->brick_vis;
  V.mvis = ctx->macro_vis;
  for (int a = 0; a < 3; ++a) V.nm[a] = ctx->nm[a];
  V.svis = ctx->super_vis;
  for (int a = 0; a < 3; ++a) V.ns[a] = ctx->ns[a];
  V.bounds = ctx->stats + 7;
  return V;
}

TfDev tf_dev(const vr_ctx* ctx) {
  TfDev t;
  t.tf = ctx->tf;
  t.n = ctx->ntf;
  t.scale = (float)(ctx->ntf - 1) / ctx->value_max;
  t.bounds = ctx->stats + 7;
  return t;
}

RenderDev render_dev_for(const int n[3], float value_max, const vr_render_params* p) {
  RenderDev r;
  r.step = p->step;
  r.ert = p->ert_threshold;
  r.skip = p->skip_empty ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    const float vhi = (float)(n[a] - 1);
    r.lo[a] = p->clip_lo[a] > 0.0f ? p->clip_lo[a] : 0.0f;
    r.hi[a] = p->clip_hi[a] < vhi ? p->clip_hi[a] : vhi;
  }
  r.gscale = op_scale(p->grad) / value_max;
  r.sh.ka = p->ka;
  r.sh.kd = p->kd;
  r.sh.ks = p->ks;
  r.sh.shininess = p->shininess;
  for (int a = 0; a < 3; ++a) r.sh.light[a] = p->light[a];
  r.sh.headlight = p->headlight ? 1 : 0;
  r.mult = nullptr;
  return r;
}

RenderDev render_dev(const vr_ctx* ctx, const vr_render_params* p) {
  return render_dev_for(ctx->n, ctx->value_max, p);
}

// Upper bound of the per-ray sample count K for the current box and step.
int max_samples(const vr_ctx* ctx, const vr_render_params* p) {
  const RenderDev r = render_dev(ctx, p);
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double e = (double)r.hi[a] - (double)r.lo[a];
    if (e > 0) d2 += e * e;
  }
  const double k = std::floor(std::sqrt(d2) / (double)p->step + 0.5) + 2.0;
  return k > 1.5e9 ? 1500000000 : (int)k;
}

// FP32 camera basis with every operation rounded on its own (this file is compiled with
// -ffp-contract=off for the host): fwd, right, up' and the screen half-extents.
bool camera_basis(const vr_camera* c, CamDev* b) {
  float f[3], r[3], u[3];
  for (int a = 0; a < 3; ++a) f[a] = c->target[a] - c->eye[a];
  float l = f[0] * f[0];
  l = l + f[1] * f[1];
  l = l + f[2] * f[2];
  l = std::sqrt(l);
  if (!(l > 0.0f) || !std::isfinite(l)) return false;
  for (int a = 0; a < 3; ++a) f[a] = f[a] / l;
  r[0] = f[1] * c->up[2] - f[2] * c->up[1];
  r[1] = f[2] * c->up[0] - f[0] * c->up[2];
  r[2] = f[0] * c->up[1] - f[1] * c->up[0];
  l = r[0] * r[0];
  l = l + r[1] * r[1];
  l = l + r[2] * r[2];
  l = std::sqrt(l);
  if (!(l > 0.0f) || !std::isfinite(l)) return false;
  for (int a = 0; a < 3; ++a) r[a] = r[a] / l;
  u[0] = r[1] * f[2] - r[2] * f[1];
  u[1] = r[2] * f[0] - r[0] * f[2];
  u[2] = r[0] * f[1] - r[1] * f[0];
  double half;
  if (c->ortho) half = (double)(c->ortho_height / 2.0f);
  else half = std::tan(((double)c->fov_y_deg * M_PI) / 360.0);
  for (int a = 0; a < 3; ++a) {
    b->eye[a] = c->eye[a];
    b->fwd[a] = f[a];
    b->right[a] = r[a];
    b->upv[a] = u[a];
  }
  b->ay = (float)half;
  b->ax = (float)((half * (double)c->width) / (double)c->height);
  b->ortho = c->ortho ? 1 : 0;
  b->width = c->width;
  b->height = c->height;
  return true;
}

vr_status check_params(const vr_render_params* p) {
  if (!p) return VR_ERR_INVALID_ARG;
  if (!(p->step > 0.0f) || !std::isfinite(p->step)) return VR_ERR_INVALID_ARG;
  if (p->grad < VR_GRAD_CENTRAL || p->grad > VR_GRAD_ZUCKER_HUMMEL) return VR_ERR_INVALID_ARG;
  if (!(p->ert_threshold > 0.0f) || std::isnan(p->ert_threshold)) return VR_ERR_INVALID_ARG;
  if (!(p->shininess >= 0.0f) || !std::isfinite(p->shininess)) return VR_ERR_INVALID_ARG;
  if (!std::isfinite(p->ka) || !std::isfinite(p->kd) || !std::isfinite(p->ks))
    return VR_ERR_INVALID_ARG;
  if (!finite3(p->light)) return VR_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (std::isnan(p->clip_lo[a]) || std::isnan(p->clip_hi[a])) return VR_ERR_INVALID_ARG;
  if (p->adaptive && (std::isnan(p->adapt_range2) || std::isnan(p->adapt_range4)))
    return VR_ERR_INVALID_ARG;
  if (p->march < VR_MARCH_AUTO || p->march > VR_MARCH_SLABS) return VR_ERR_INVALID_ARG;
  return VR_OK;
}

static vr_status refresh_visibility(vr_ctx* ctx, cudaStream_t s) {
  if (!ctx->has_volume || !ctx->has_tf) return VR_OK;
  const float scale = (float)(ctx->ntf - 1) / ctx->value_max;
  return cuda_status(
      launch_brick_visibility(ctx->brick_minmax, ctx->nb, ctx->tf_prefix, ctx->ntf, scale,
                              ctx->brick_vis, ctx->brick_list, ctx->macro_vis, ctx->nm, s,
                              ctx->super_vis, ctx->ns));
}

// Which march a plain render launches: from the visible-brick count the previous plain
// render's march saw (1: tiles, 2: list; a count of an earlier transfer function only costs
// speed, the image is the same either way), or 0 (decided on the device from the current
// count) while none has arrived for a volume of this brick grid.
static vr_status ensure_hint(vr_ctx* ctx) {
  if (ctx->vis_hint) return VR_OK;
  // mapped pinned host memory the march writes the count into (no copy joins the stream);
  // {-1, 0} until a march has written it
  void* h = nullptr;
  void* d = nullptr;
  vr_status st = cuda_status(cudaHostAlloc(&h, 2 * sizeof(int), cudaHostAllocMapped));
  if (st != VR_OK) return st;
  st = cuda_status(cudaHostGetDevicePointer(&d, h, 0));
  if (st != VR_OK) {
    cudaFreeHost(h);
    return st;
  }
  static_cast<int*>(h)[0] = -1;
  static_cast<int*>(h)[1] = 0;
  ctx->vis_hint = static_cast<volatile int*>(h);
  ctx->vis_hint_dev = static_cast<int*>(d);
  return VR_OK;
}

static int march_mode_hint(vr_ctx* ctx) {
  if (!ctx->vis_hint) return 0;
  const int count = ctx->vis_hint[0], nbricks = ctx->vis_hint[1];
  if (count < 0 || nbricks != ctx->nb[0] * ctx->nb[1] * ctx->nb[2]) return 0;
  return (long long)count * kListDenom < nbricks ? 2 : 1;
}

// Operator gradient records for the current volume, operator and (with skipping) the
// current brick visibility; recomputed only when one of them changed.
vr_status ensure_records(vr_ctx* ctx, const vr_render_params* p, cudaStream_t s) {
  const bool skip = p->skip_empty != 0;
  if (ctx->rec_valid && ctx->rec_vol_gen == ctx->vol_gen && ctx->rec_op == p->grad &&
      (ctx->rec_all || (skip && ctx->rec_tf_gen == ctx->tf_gen)))
    return VR_OK;
  const size_t nvox = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  void* r = ctx->rec;
  vr_status st = ensure(ctx, &r, &ctx->rec_cap, nvox * sizeof(float4));
  ctx->rec = static_cast<float4*>(r);  // ensure() may have released the old buffer
  if (st != VR_OK) {
    ctx->rec_valid = false;
    return st;
  }
  st = cuda_status(launch_records(vol_dev(ctx), (int)ctx->dtype, p->grad,
                                  skip ? ctx->brick_vis : nullptr,
                                  skip ? ctx->brick_list : nullptr, ctx->rec, s,
                                  reinterpret_cast<unsigned*>(ctx->stats + 8)));
  if (st != VR_OK) {
    ctx->rec_valid = false;
    return st;
  }
  ctx->rec_valid = true;
  ctx->rec_all = !skip;
  ctx->rec_vol_gen = ctx->vol_gen;
  ctx->rec_tf_gen = ctx->tf_gen;
  ctx->rec_op = p->grad;
  return VR_OK;
}

RecDev rec_dev(const vr_ctx* ctx) {
  RecDev R;
  R.rec = ctx->rec;
  for (int a = 0; a < 3; ++a) R.n[a] = ctx->n[a];
  R.sx = ctx->n[0] > 1 ? 1 : 0;
  R.sy = ctx->n[1] > 1 ? ctx->n[0] : 0;
  R.sz = ctx->n[2] > 1 ? ctx->n[0] * ctx->n[1] : 0;
  R.bounds = ctx->stats + 7;
  return R;
}

// Pixels whose rays can meet the sampling box [lo, hi]: the bounding rectangle of the
// box corners projected onto the image (the projection of a convex box in front of the
// camera is the convex hull of its projected corners), widened by two pixels for the FP32
// rounding of the ray set-up.  The full image when a corner lies near or behind the eye
// plane of a perspective camera; empty when the box is empty.
void screen_rect(const CamDev& c, const float lo[3], const float hi[3], int rect[4]) {
  const int W = c.width, H = c.height;
  rect[0] = 0;
  rect[1] = 0;
  rect[2] = W;
  rect[3] = H;
  for (int a = 0; a < 3; ++a)
    if (lo[a] > hi[a]) {
      rect[2] = rect[3] = 0;
      return;
    }
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int k = 0; k < 8; ++k) {
    const double P[3] = {(k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2]};
    double rel[3], u = 0.0, v = 0.0, z = 0.0;
    for (int a = 0; a < 3; ++a) rel[a] = P[a] - (double)c.eye[a];
    for (int a = 0; a < 3; ++a) {
      u += rel[a] * c.right[a];
      v += rel[a] * c.upv[a];
      z += rel[a] * c.fwd[a];
    }
    if (!c.ortho) {
      if (!(z > 1e-3)) return;  // near or behind the eye plane: no culling
      u /= z;
      v /= z;
    }
    const double sx = u / c.ax, sy = v / c.ay;
    const double x = (sx + 1.0) * 0.5 * W - 0.5, y = (1.0 - sy) * 0.5 * H - 0.5;
    if (!std::isfinite(x) || !std::isfinite(y)) return;
    xmin = std::min(xmin, x);
    xmax = std::max(xmax, x);
    ymin = std::min(ymin, y);
    ymax = std::max(ymax, y);
  }
  const double x0 = std::floor(xmin) - 2.0, x1 = std::ceil(xmax) + 3.0;
  const double y0 = std::floor(ymin) - 2.0, y1 = std::ceil(ymax) + 3.0;
  rect[0] = (int)std::min(std::max(x0, 0.0), (double)W);
  rect[2] = (int)std::min(std::max(x1, 0.0), (double)W);
  rect[1] = (int)std::min(std::max(y0, 0.0), (double)H);
  rect[3] = (int)std::min(std::max(y1, 0.0), (double)H);
  if (rect[2] <= rect[0] || rect[3] <= rect[1]) rect[0] = rect[1] = rect[2] = rect[3] = 0;
}

// Renders rows [row0, row1) of the image (row1 < 0: to the last row) into `out`, a band of
// (row1 - row0) rows.
static vr_status render_common(vr_ctx* ctx, const vr_render_params* p, float* out,
                               int* ck_kend, float* ck_T, int nslots, cudaStream_t s,
                               float* ck_Tend = nullptr, int row0 = 0, int row1 = -1,
                               const float* zwin = nullptr) {
  MarchLaunch L;
  L.V = vol_dev(ctx);
  L.R = rec_dev(ctx);  // refreshed below when the records are computed
  L.tf = tf_dev(ctx);
  L.cam = ctx->camdev;
  L.r = render_dev(ctx, p);
  L.dtype = (int)ctx->dtype;
  L.op = p->grad;
  L.out = reinterpret_cast<float4*>(out);
  L.stats = nullptr;
  L.tile_counter = reinterpret_cast<unsigned*>(ctx->stats + 4);
  L.ck_kend = ck_kend;
  L.ck_T = ck_T;
  L.ck_Tend = ck_Tend;
  L.nslots = nslots;
  L.row0 = row0;
  L.row1 = row1 < 0 ? L.cam.height : row1;
  L.rect[0] = 0;
  L.rect[1] = L.row0;
  L.rect[2] = L.cam.width;
  L.rect[3] = L.row1;
  if (!ck_kend) {
    // march only the tiles of the box's screen rectangle (within the band); the other
    // pixels are zero.  A checkpointed render marches every tile: its rays outside the
    // rectangle miss the box and record end index 0 without any memset (the adjoint skips
    // the rectangle's outside)
    screen_rect(L.cam, L.r.lo, L.r.hi, L.rect);
    L.rect[1] = std::max(L.rect[1], L.row0);
    L.rect[3] = std::min(L.rect[3], L.row1);
    if (L.rect[3] <= L.rect[1] || L.rect[2] <= L.rect[0])
      L.rect[0] = L.rect[1] = L.rect[2] = L.rect[3] = 0;
    if (L.rect[0] > 0 || L.rect[1] > L.row0 || L.rect[2] < L.cam.width || L.rect[3] < L.row1) {
      vr_status st = cuda_status(cudaMemsetAsync(
          out, 0, (size_t)L.cam.width * (L.row1 - L.row0) * sizeof(float4), s));
      if (st != VR_OK) return st;
    }
  }
  // a plain render marches in slabs (no record table) when asked to and the camera allows
  // it; the automatic choice is the record march, the faster one on every workload measured
  bool slab = false;
  if (!ck_kend && !p->adaptive && !zwin && p->march == VR_MARCH_SLABS) {
    vr_status st = ensure_hint(ctx);
    if (st != VR_OK) return st;
    L.hint = ctx->vis_hint_dev;
    L.vis_count = ctx->brick_list;  // [0]: visible bricks
    slab = slab_eligible(L);
  }
  if (!slab) {
    const vr_status rst = ensure_records(ctx, p, s);
    if (rst != VR_OK) return rst;
    L.R = rec_dev(ctx);
  }
  if (zwin) {
    L.zwin[0] = zwin[0];
    L.zwin[1] = zwin[1];
  }
  if (!slab && !zwin && !ck_kend && !p->adaptive && L.rect[2] > L.rect[0]) {
    // plain render: the rays of the rectangle's tiles are set up and listed first
    const size_t tiles = (size_t)((L.rect[2] + 3) / 4 - L.rect[0] / 4) *
                         (size_t)((L.rect[3] + 1) / 2 - L.rect[1] / 2);
    vr_status st = ensure(ctx, &ctx->ray_list, &ctx->ray_list_cap, 256 + tiles * 8 * sizeof(RayRec));
    if (st != VR_OK) return st;
    L.list_head = static_cast<int*>(ctx->ray_list);
    L.list = reinterpret_cast<RayRec*>(static_cast<char*>(ctx->ray_list) + 256);
    L.vis_count = ctx->brick_list;  // [0]: visible bricks
    st = ensure_hint(ctx);
    if (st != VR_OK) return st;
    L.hint = ctx->vis_hint_dev;
    L.mode = (p->skip_empty && L.V.mvis) ? march_mode_hint(ctx) : 1;
  }
  if (p->collect_stats) {
    vr_status st = cuda_status(cudaMemsetAsync(ctx->stats, 0, 4 * sizeof(unsigned long long), s));
    if (st != VR_OK) return st;
    L.stats = ctx->stats;
  }
  if (p->adaptive) {
    // sampling multiplier of every macro brick from its footprint's value range (§5.2)
    const int nmacro = ctx->nm[0] * ctx->nm[1] * ctx->nm[2];
    vr_status st = ensure(ctx, &ctx->adapt_mult, &ctx->adapt_mult_cap, (size_t)nmacro);
    if (st != VR_OK) return st;
    st = cuda_status(launch_macro_multiplier(ctx->brick_minmax, ctx->nb, ctx->nm, p->adapt_range2,
                                             p->adapt_range4,
                                             static_cast<uint8_t*>(ctx->adapt_mult), s));
    if (st != VR_OK) return st;
    L.r.mult = static_cast<const uint8_t*>(ctx->adapt_mult);
  }
  const vr_status st = cuda_status(zwin ? launch_march_zwin(L, s)
                                        : (slab ? launch_march_slab(L, s) : launch_march(L, s)));
  if (st == VR_OK && p->collect_stats) {
    ctx->stats_valid = true;
    ctx->stats_march = slab ? VR_MARCH_SLABS : VR_MARCH_RECORDS;
  }
  return st;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static void ckpt_layout(vr_ctx* ctx, const vr_render_params* p, int* nrays, int* nslots,
                        size_t* bytes) {
  *nrays = ctx->cam.width * ctx->cam.height;
  const int kmax = max_samples(ctx, p);
  *nslots = kmax > 1 ? (kmax - 1) / kCkptStride : 0;
  // per ray: end index, final transmittance, transmittance before every 32nd sample
  *bytes = 2 * align256((size_t)*nrays * 4) + (size_t)*nrays * 4 * (size_t)*nslots;
}

}  // namespace vr

namespace vr {

vr_status check_camera(const vr_camera* cam, CamDev* b) {
  if (!cam) return VR_ERR_INVALID_ARG;
  if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
    return VR_ERR_INVALID_ARG;
  if (!finite3(cam->eye) || !finite3(cam->target) || !finite3(cam->up)) return VR_ERR_INVALID_ARG;
  if (cam->ortho) {
    if (!(cam->ortho_height > 0.0f) || !std::isfinite(cam->ortho_height)) return VR_ERR_INVALID_ARG;
  } else {
    if (!(cam->fov_y_deg > 0.0f && cam->fov_y_deg < 180.0f)) return VR_ERR_INVALID_ARG;
  }
  return camera_basis(cam, b) ? VR_OK : VR_ERR_INVALID_ARG;
}
}  // namespace vr

using namespace vr;

extern "C" {

vr_status vr_create(vr_ctx** out, int device, vr_alloc_fn alloc, vr_free_fn free_fn, void* user) {
  if (!out) return VR_ERR_INVALID_ARG;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return VR_ERR_INVALID_ARG;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_status(e);
  if (device < 0 || device >= count) return VR_ERR_INVALID_ARG;
  vr_ctx* ctx = new (std::nothrow) vr_ctx();
  if (!ctx) return VR_ERR_OUT_OF_MEMORY;
  ctx->device = device;
  ctx->alloc = alloc;
  ctx->free_fn = free_fn;
  ctx->user = user;
  DeviceGuard g(device);
  if (!g.ok) {
    delete ctx;
    return cuda_status(cudaGetLastError());
  }
  void* st = nullptr;
  const vr_status s = ctx_alloc(ctx, &st, 16 * sizeof(unsigned long long));
  if (s != VR_OK) {
    delete ctx;
    return s;
  }
  ctx->stats = static_cast<unsigned long long*>(st);
  // counters and work queues start at zero (the bounds counter is never reset)
  const vr_status z = cuda_status(cudaMemset(ctx->stats, 0, 16 * sizeof(unsigned long long)));
  const vr_status zs = z == VR_OK ? cuda_status(cudaDeviceSynchronize()) : z;
  if (zs != VR_OK) {
    ctx_free(ctx, ctx->stats);
    delete ctx;
    return zs;
  }
  *out = ctx;
  return VR_OK;
}

void vr_destroy(vr_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  ctx_free(ctx, ctx->vol);
  ctx_free(ctx, ctx->brick_minmax);
  ctx_free(ctx, ctx->upload_staging);
  if (ctx->host_copy_done) cudaEventDestroy(ctx->host_copy_done);
  if (ctx->tf_stage_done) cudaEventDestroy(ctx->tf_stage_done);
  if (ctx->tf_host_stage) cudaFreeHost(ctx->tf_host_stage);
  if (ctx->vis_hint) cudaFreeHost(const_cast<int*>(ctx->vis_hint));
  ctx_free(ctx, ctx->tf);
  ctx_free(ctx, ctx->stats);
  ctx_free(ctx, ctx->out_staging);
  ctx_free(ctx, ctx->adj);
  ctx_free(ctx, ctx->tf_partial);
  ctx_free(ctx, ctx->batch_tab);
  ctx_free(ctx, ctx->surf_vis);
  ctx_free(ctx, ctx->adapt_mult);
  ctx_free(ctx, ctx->rec);
  ctx_free(ctx, ctx->ray_list);
  delete ctx;
}

// Record the end of a copy from a caller's host buffer on `s` (waited for before returning).
static vr_status mark_host_copy(vr_ctx* ctx, cudaStream_t s) {
  if (!ctx->host_copy_done) {
    const vr_status st =
        cuda_status(cudaEventCreateWithFlags(&ctx->host_copy_done, cudaEventDisableTiming));
    if (st != VR_OK) return st;
  }
  return cuda_status(cudaEventRecord(ctx->host_copy_done, s));
}

vr_status vr_upload_volume(vr_ctx* ctx, const void* voxels, vr_dtype dtype, int nx, int ny,
                           int nz, float value_max, void* stream) {
  TraceRange trace_("vr_upload_volume");
  if (!ctx || !voxels) return VR_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return VR_ERR_INVALID_ARG;
  if (!(value_max > 0.0f) || !std::isfinite(value_max)) return VR_ERR_INVALID_ARG;
  const int eb = dtype_bytes(dtype);
  if (eb == 0) return VR_ERR_UNSUPPORTED;
  if (!aligned_to(voxels, (size_t)eb)) return VR_ERR_INVALID_ARG;
  const long long nvox = (long long)nx * ny * nz;
  // x pitch: a multiple of 16 elements and at least nx + 8, so that the vector row loads
  // of the brick footprints (which start at padded x = 8 bx) stay inside each row
  const long long px = ((long long)nx + 8 + 15) / 16 * 16;
  const long long py = ny + kPadLo + kPadHi, pz = nz + kPadLo + kPadHi;
  if (nvox > 2147483647LL || px * py * pz > 2147483647LL) return VR_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const void* src = voxels;
  vr_status st;
  // until this upload completes the context holds no volume (a failed allocation below may
  // have released the previous one)
  ctx->has_volume = false;
  ctx->rec_valid = false;
  if (!is_device_pointer(voxels)) {
    st = ensure(ctx, &ctx->upload_staging, &ctx->upload_cap, (size_t)nvox * eb);
    if (st != VR_OK) return st;
    st = cuda_status(cudaMemcpyAsync(ctx->upload_staging, voxels, (size_t)nvox * eb,
                                     cudaMemcpyHostToDevice, s));
    if (st != VR_OK) return st;
    st = mark_host_copy(ctx, s);
    if (st != VR_OK) return st;
    src = ctx->upload_staging;
  }
  st = ensure(ctx, &ctx->vol, &ctx->vol_cap, (size_t)(px * py * pz) * eb);
  if (st != VR_OK) return st;
  const int nb[3] = {(nx + kBrick - 1) / kBrick, (ny + kBrick - 1) / kBrick,
                     (nz + kBrick - 1) / kBrick};
  const size_t nbricks = (size_t)nb[0] * nb[1] * nb[2];
  void* bt = ctx->brick_minmax;
  const int nm[3] = {(nb[0] + 3) >> kMacroShift, (nb[1] + 3) >> kMacroShift,
                     (nb[2] + 3) >> kMacroShift};
  const size_t nmacro = (size_t)nm[0] * nm[1] * nm[2];
  const int ns[3] = {(nm[0] + 3) >> kSuperShift, (nm[1] + 3) >> kSuperShift,
                     (nm[2] + 3) >> kSuperShift};
  const size_t nsuper = (size_t)ns[0] * ns[1] * ns[2];
  const size_t off_vis = align256(nbricks * sizeof(float2));
  const size_t off_list = off_vis + align256(nbricks);
  const size_t off_macro = off_list + align256((nbricks + 1) * sizeof(int));
  const size_t off_super = off_macro + align256(nmacro);
  st = ensure(ctx, &bt, &ctx->brick_cap, off_super + nsuper);
  ctx->brick_minmax = static_cast<float2*>(bt);
  if (st != VR_OK) {
    ctx->brick_vis = ctx->macro_vis = ctx->super_vis = nullptr;
    ctx->brick_list = nullptr;
    return st;
  }
  ctx->brick_vis = reinterpret_cast<uint8_t*>(static_cast<char*>(bt) + off_vis);
  ctx->brick_list = reinterpret_cast<int*>(static_cast<char*>(bt) + off_list);
  ctx->macro_vis = reinterpret_cast<uint8_t*>(static_cast<char*>(bt) + off_macro);
  ctx->super_vis = reinterpret_cast<uint8_t*>(static_cast<char*>(bt) + off_super);
  ctx->dtype = dtype;
  ctx->n[0] = nx; ctx->n[1] = ny; ctx->n[2] = nz;
  ctx->px = (int)px; ctx->py = (int)py; ctx->pz = (int)pz;
  for (int a = 0; a < 3; ++a) {
    ctx->nb[a] = nb[a];
    ctx->nm[a] = nm[a];
    ctx->ns[a] = ns[a];
  }
  ctx->value_max = value_max;
  st = cuda_status(launch_pad_volume(src, (int)dtype, ctx->n, ctx->vol, ctx->px, ctx->py,
                                     ctx->pz, s));
  if (st != VR_OK) return st;
  st = cuda_status(launch_brick_minmax(vol_dev(ctx), (int)dtype, ctx->brick_minmax, s));
  if (st != VR_OK) return st;
  if (!ctx->has_tf) {
    // no transfer function yet: everything visible until one is set
    st = cuda_status(cudaMemsetAsync(ctx->brick_vis, 1, nbricks, s));
    if (st != VR_OK) return st;
    st = cuda_status(cudaMemsetAsync(ctx->macro_vis, 1, nmacro, s));
    if (st != VR_OK) return st;
    st = cuda_status(cudaMemsetAsync(ctx->super_vis, 1, nsuper, s));
    if (st != VR_OK) return st;
  }
  ctx->has_volume = true;
  ++ctx->vol_gen;
  st = refresh_visibility(ctx, s);
  if (st != VR_OK) return st;
  if (!is_device_pointer(voxels)) {
    // keep the host buffer's contract ("read before the call returns"): wait for the
    // host-to-device copy only; the padding and brick kernels stay queued on the stream.
    st = cuda_status(cudaEventSynchronize(ctx->host_copy_done));
  }
  return st;
}

vr_status vr_set_transfer_function(vr_ctx* ctx, const float* rgba, int n, void* stream) {
  TraceRange trace_("vr_set_transfer_function");
  if (!ctx || !rgba || n < 2 || n > 65536) return VR_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ctx->has_tf = false;  // until this table is in place
  void* buf = ctx->tf;
  const size_t tfb = align256((size_t)n * sizeof(float4));
  vr_status st = ensure(ctx, &buf, &ctx->tf_cap, tfb + (size_t)(n + 1) * sizeof(int));
  ctx->tf = static_cast<float4*>(buf);
  if (st != VR_OK) {
    ctx->tf_prefix = nullptr;
    return st;
  }
  ctx->tf_prefix = reinterpret_cast<int*>(static_cast<char*>(buf) + tfb);
  const bool dev = is_device_pointer(rgba);
  const size_t bytes = (size_t)n * sizeof(float4);
  const void* src = rgba;
  if (!dev) {
    // a host table goes through the context's pinned staging: the caller's table is free as
    // soon as it is copied there, and the call need not wait for the stream to reach the
    // copy (behind, say, the upload of a volume); only the previous copy out of the staging
    // must have finished before it is overwritten
    if (ctx->tf_stage_done) {
      st = cuda_status(cudaEventSynchronize(ctx->tf_stage_done));
      if (st != VR_OK) return st;
    } else {
      st = cuda_status(cudaEventCreateWithFlags(&ctx->tf_stage_done, cudaEventDisableTiming));
      if (st != VR_OK) return st;
    }
    if (ctx->tf_host_stage_cap < bytes) {
      if (ctx->tf_host_stage) cudaFreeHost(ctx->tf_host_stage);
      ctx->tf_host_stage = nullptr;
      ctx->tf_host_stage_cap = 0;
      st = cuda_status(cudaHostAlloc(&ctx->tf_host_stage, bytes, cudaHostAllocDefault));
      if (st != VR_OK) {
        ctx->tf_host_stage = nullptr;
        return st;
      }
      ctx->tf_host_stage_cap = bytes;
    }
    std::memcpy(ctx->tf_host_stage, rgba, bytes);
    src = ctx->tf_host_stage;
  }
  st = cuda_status(cudaMemcpyAsync(ctx->tf, src, bytes,
                                   dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  if (st != VR_OK) return st;
  if (!dev) {
    st = cuda_status(cudaEventRecord(ctx->tf_stage_done, s));
    if (st != VR_OK) return st;
  }
  st = cuda_status(launch_tf_prefix(ctx->tf, n, ctx->tf_prefix, s));
  if (st != VR_OK) return st;
  ctx->ntf = n;
  ctx->has_tf = true;
  ++ctx->tf_gen;
  return refresh_visibility(ctx, s);
}


vr_status vr_set_camera(vr_ctx* ctx, const vr_camera* cam) {
  if (!ctx || !cam) return VR_ERR_INVALID_ARG;
  CamDev b;
  const vr_status st = check_camera(cam, &b);
  if (st != VR_OK) return st;
  ctx->cam = *cam;
  ctx->camdev = b;
  ctx->has_camera = true;
  return VR_OK;
}

vr_status vr_render(vr_ctx* ctx, const vr_render_params* params, float* out_rgba, void* stream) {
  TraceRange trace_("vr_render");
  if (!ctx || !out_rgba) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->cam.width * ctx->cam.height * sizeof(float4);
  float* dst = out_rgba;
  const bool host_out = !is_device_pointer(out_rgba);
  if (!host_out && !aligned_to(out_rgba, 16)) return VR_ERR_INVALID_ARG;
  if (host_out) {
    st = ensure(ctx, &ctx->out_staging, &ctx->out_cap, bytes);
    if (st != VR_OK) return st;
    dst = static_cast<float*>(ctx->out_staging);
  }
  st = render_common(ctx, params, dst, nullptr, nullptr, 0, s);
  if (st != VR_OK) return st;
  if (host_out)
    st = cuda_status(cudaMemcpyAsync(out_rgba, dst, bytes, cudaMemcpyDeviceToHost, s));
  return st;
}

vr_status vr_render_rgba8(vr_ctx* ctx, const vr_render_params* params, unsigned char* out_rgba8,
                          void* stream) {
  TraceRange trace_("vr_render_rgba8");
  if (!ctx || !out_rgba8) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t npix = (size_t)ctx->cam.width * ctx->cam.height;
  const size_t fbytes = npix * sizeof(float4), bbytes = npix * sizeof(uchar4);
  const bool host_out = !is_device_pointer(out_rgba8);
  if (!host_out && !aligned_to(out_rgba8, 4)) return VR_ERR_INVALID_ARG;
  // the FP32 image goes to the staging buffer, followed (for a host output) by its bytes
  st = ensure(ctx, &ctx->out_staging, &ctx->out_cap, fbytes + (host_out ? bbytes : 0));
  if (st != VR_OK) return st;
  float* f = static_cast<float*>(ctx->out_staging);
  st = render_common(ctx, params, f, nullptr, nullptr, 0, s);
  if (st != VR_OK) return st;
  uchar4* q = host_out ? reinterpret_cast<uchar4*>(static_cast<char*>(ctx->out_staging) + fbytes)
                       : reinterpret_cast<uchar4*>(out_rgba8);
  st = cuda_status(launch_quantize_rgba8(reinterpret_cast<const float4*>(f), q, npix, s));
  if (st != VR_OK) return st;
  if (host_out) st = cuda_status(cudaMemcpyAsync(out_rgba8, q, bbytes, cudaMemcpyDeviceToHost, s));
  return st;
}

vr_status vr_render_rows(vr_ctx* ctx, const vr_render_params* params, int row0, int row1,
                         float* out_rgba, void* stream) {
  TraceRange trace_("vr_render_rows");
  if (!ctx || !out_rgba) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  if (row0 < 0 || row1 <= row0 || row1 > ctx->cam.height) return VR_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->cam.width * (row1 - row0) * sizeof(float4);
  float* dst = out_rgba;
  const bool host_out = !is_device_pointer(out_rgba);
  if (!host_out && !aligned_to(out_rgba, 16)) return VR_ERR_INVALID_ARG;
  if (host_out) {
    st = ensure(ctx, &ctx->out_staging, &ctx->out_cap, bytes);
    if (st != VR_OK) return st;
    dst = static_cast<float*>(ctx->out_staging);
  }
  st = render_common(ctx, params, dst, nullptr, nullptr, 0, s, nullptr, row0, row1);
  if (st != VR_OK) return st;
  if (host_out)
    st = cuda_status(cudaMemcpyAsync(out_rgba, dst, bytes, cudaMemcpyDeviceToHost, s));
  return st;
}

vr_status vr_render_partial(vr_ctx* ctx, const vr_render_params* params, float z0, float z1,
                            float* out_rgba, void* stream) {
  TraceRange trace_("vr_render_partial");
  if (!ctx || !out_rgba) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->adaptive) return VR_ERR_UNSUPPORTED;  // partial images follow the regular grid
  if (std::isnan(z0) || std::isnan(z1) || !(z0 < z1)) return VR_ERR_INVALID_ARG;
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->cam.width * ctx->cam.height * sizeof(float4);
  float* dst = out_rgba;
  const bool host_out = !is_device_pointer(out_rgba);
  if (!host_out && !aligned_to(out_rgba, 16)) return VR_ERR_INVALID_ARG;
  if (host_out) {
    st = ensure(ctx, &ctx->out_staging, &ctx->out_cap, bytes);
    if (st != VR_OK) return st;
    dst = static_cast<float*>(ctx->out_staging);
  }
  const float zw[2] = {z0, z1};
  st = render_common(ctx, params, dst, nullptr, nullptr, 0, s, nullptr, 0, -1, zw);
  if (st != VR_OK) return st;
  if (host_out)
    st = cuda_status(cudaMemcpyAsync(out_rgba, dst, bytes, cudaMemcpyDeviceToHost, s));
  return st;
}

vr_status vr_checkpoint_bytes(vr_ctx* ctx, const vr_render_params* params, size_t* bytes) {
  if (!ctx || !bytes) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->adaptive) return VR_ERR_UNSUPPORTED;  // the adjoint marches the regular grid
  if (!ctx->has_volume || !ctx->has_camera) return VR_ERR_STATE;
  int nrays, nslots;
  ckpt_layout(ctx, params, &nrays, &nslots, bytes);
  return VR_OK;
}

vr_status vr_render_forward_train(vr_ctx* ctx, const vr_render_params* params, float* out_rgba,
                                  void* checkpoints, size_t checkpoint_bytes, void* stream) {
  TraceRange trace_("vr_render_forward_train");
  if (!ctx || !out_rgba || !checkpoints) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->adaptive) return VR_ERR_UNSUPPORTED;  // the adjoint marches the regular grid
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  if (((uintptr_t)checkpoints & 255) != 0) return VR_ERR_INVALID_ARG;
  int nrays, nslots;
  size_t need;
  ckpt_layout(ctx, params, &nrays, &nslots, &need);
  if (checkpoint_bytes < need) return VR_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  if (!is_device_pointer(out_rgba) || !is_device_pointer(checkpoints)) return VR_ERR_INVALID_ARG;
  if (!aligned_to(out_rgba, 16)) return VR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* kend = static_cast<int*>(checkpoints);
  float* Tend = reinterpret_cast<float*>(static_cast<char*>(checkpoints) + align256((size_t)nrays * 4));
  float* T = reinterpret_cast<float*>(static_cast<char*>(checkpoints) +
                                      2 * align256((size_t)nrays * 4));
  st = render_common(ctx, params, out_rgba, kend, T, nslots, s, Tend);
  if (st != VR_OK) return st;
  // remember what was recorded (replace an older record of the same buffer)
  int slot = -1;
  for (int i = 0; i < kMaxCkptRecords; ++i)
    if (ctx->ckpt[i].ptr == checkpoints) slot = i;
  if (slot < 0) {
    slot = ctx->ckpt_next;
    ctx->ckpt_next = (ctx->ckpt_next + 1) % kMaxCkptRecords;
  }
  CkptRecord& r = ctx->ckpt[slot];
  r.ptr = checkpoints;
  r.bytes = checkpoint_bytes;
  r.cam = ctx->cam;
  r.params = *params;
  r.vol_gen = ctx->vol_gen;
  r.tf_gen = ctx->tf_gen;
  r.nrays = nrays;
  r.nslots = nslots;
  return VR_OK;
}

vr_status vr_render_backward_views(vr_ctx* ctx, const vr_render_params* params, int nviews,
                                   const vr_camera* cams, const void* const* checkpoints,
                                   const float* const* grad_rgba, float* grad_volume,
                                   float* grad_tf, void* stream) {
  TraceRange trace_("vr_render_backward_views");
  if (!ctx || nviews < 1 || !cams || !checkpoints || !grad_rgba) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->adaptive) return VR_ERR_UNSUPPORTED;  // the adjoint marches the regular grid
  if (!ctx->has_volume || !ctx->has_tf) return VR_ERR_STATE;
  // validate every view before queuing any work
  const CkptRecord* recs[256];
  if (nviews > 256) return VR_ERR_INVALID_ARG;
  for (int v = 0; v < nviews; ++v) {
    if (!checkpoints[v] || !grad_rgba[v]) return VR_ERR_INVALID_ARG;
    const CkptRecord* rec = nullptr;
    for (int i = 0; i < kMaxCkptRecords; ++i)
      if (ctx->ckpt[i].ptr == checkpoints[v]) rec = &ctx->ckpt[i];
    if (!rec) return VR_ERR_STATE;
    if (rec->vol_gen != ctx->vol_gen || rec->tf_gen != ctx->tf_gen) return VR_ERR_STATE;
    if (std::memcmp(&rec->cam, &cams[v], sizeof(vr_camera)) != 0) return VR_ERR_STATE;
    vr_render_params a = rec->params, b = *params;
    a.collect_stats = b.collect_stats = 0;
    if (std::memcmp(&a, &b, sizeof(vr_render_params)) != 0) return VR_ERR_STATE;
    recs[v] = rec;
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  for (int v = 0; v < nviews; ++v)
    if (!is_device_pointer(grad_rgba[v]) || !aligned_to(grad_rgba[v], 16))
      return VR_ERR_INVALID_ARG;
  if (grad_volume && (!is_device_pointer(grad_volume) || !aligned_to(grad_volume, 4)))
    return VR_ERR_INVALID_ARG;
  if (grad_tf && (!is_device_pointer(grad_tf) || !aligned_to(grad_tf, 4)))
    return VR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nvox = (size_t)ctx->n[0] * ctx->n[1] * ctx->n[2];
  if (grad_volume) {
    void* adj = ctx->adj;
    st = ensure(ctx, &adj, &ctx->adj_cap, nvox * sizeof(float4));
    ctx->adj = static_cast<float4*>(adj);
    if (st != VR_OK) return st;
    st = cuda_status(cudaMemsetAsync(ctx->adj, 0, nvox * sizeof(float4), s));
    if (st != VR_OK) return st;
  }
  // transfer-function gradient: per-block partial sums, reduced once after all views
  const bool tf_partial = grad_tf && adjoint_tf_rows(ctx->ntf);
  const int ablocks = adjoint_grid(ctx->ntf);
  if (tf_partial) {
    const size_t pbytes = (size_t)ablocks * 4 * ctx->ntf * sizeof(float);
    void* pp = ctx->tf_partial;
    st = ensure(ctx, &pp, &ctx->tf_partial_cap, pbytes);
    ctx->tf_partial = static_cast<float*>(pp);
    if (st != VR_OK) return st;
    st = cuda_status(cudaMemsetAsync(ctx->tf_partial, 0, pbytes, s));
    if (st != VR_OK) return st;
  }
  // the adjoint visits every sample (no skipping): records are needed everywhere
  vr_render_params all = *params;
  all.skip_empty = 0;
  st = ensure_records(ctx, &all, s);
  if (st != VR_OK) return st;
  // the views' tiles form one work queue per launch of up to kAdjViews views
  AdjointLaunch L;
  L.V = vol_dev(ctx);
  L.R = rec_dev(ctx);
  L.tf = tf_dev(ctx);
  L.r = render_dev(ctx, params);
  L.dtype = (int)ctx->dtype;
  L.op = params->grad;
  L.tile_counter = reinterpret_cast<unsigned*>(ctx->stats + 5);
  L.adj = grad_volume ? ctx->adj : nullptr;
  L.grad_tf = grad_tf;
  L.tf_partial = tf_partial ? ctx->tf_partial : nullptr;
  for (int v = 0; v < nviews; ++v) {
    const CkptRecord* rec = recs[v];
    CamDev basis;
    st = check_camera(&cams[v], &basis);
    if (st != VR_OK) return st;
    const char* ck = static_cast<const char*>(checkpoints[v]);
    int rect[4];
    screen_rect(basis, L.r.lo, L.r.hi, rect);  // rays outside it recorded end index 0
    adjoint_add_view(L, basis, rect, reinterpret_cast<const int*>(ck),
                     reinterpret_cast<const float*>(ck + 2 * align256((size_t)rec->nrays * 4)),
                     reinterpret_cast<const float*>(ck + align256((size_t)rec->nrays * 4)),
                     reinterpret_cast<const float4*>(grad_rgba[v]));
    if (L.nviews == kAdjViews || v == nviews - 1) {
      st = cuda_status(launch_adjoint(L, s));
      if (st != VR_OK) return st;
      L.nviews = 0;
      L.tiles_total = 0;
    }
  }
  if (tf_partial) {
    st = cuda_status(launch_tf_partial_reduce(ctx->tf_partial, ablocks, 4 * ctx->ntf, grad_tf, s));
    if (st != VR_OK) return st;
  }
  if (grad_volume)
    st = cuda_status(launch_adjoint_volume(ctx->adj, ctx->n, params->grad, 1.0f / ctx->value_max,
                                           grad_volume, s));
  return st;
}

vr_status vr_render_backward(vr_ctx* ctx, const vr_render_params* params, const void* checkpoints,
                             const float* grad_rgba, float* grad_volume, float* grad_tf,
                             void* stream) {
  TraceRange trace_("vr_render_backward");
  if (!ctx || !checkpoints || !grad_rgba) return VR_ERR_INVALID_ARG;
  if (!ctx->has_camera) return VR_ERR_STATE;
  return vr_render_backward_views(ctx, params, 1, &ctx->cam, &checkpoints, &grad_rgba,
                                  grad_volume, grad_tf, stream);
}

vr_status vr_read_stats(vr_ctx* ctx, vr_stats* out, void* stream) {
  if (!ctx || !out) return VR_ERR_INVALID_ARG;
  if (!ctx->stats_valid) return VR_ERR_STATE;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  unsigned long long h[9];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  vr_status st = cuda_status(cudaMemcpyAsync(h, ctx->stats, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (st != VR_OK) return st;
  st = cuda_status(cudaStreamSynchronize(s));
  if (st != VR_OK) return st;
  if (h[8] & 1u) return VR_ERR_TIMEOUT;  // a records pass gave up waiting for a staged copy
  out->rays_hit = h[0];
  out->samples_plain = h[1];
  out->samples_visited = h[2];
  out->samples_shaded = h[3];
  out->march = (unsigned long long)ctx->stats_march;
  return VR_OK;
}

vr_status vr_screen_rect(const vr_camera* cam, const float lo[3], const float hi[3], int rect[4]) {
  if (!lo || !hi || !rect) return VR_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (std::isnan(lo[a]) || std::isnan(hi[a])) return VR_ERR_INVALID_ARG;
  CamDev c;
  const vr_status st = check_camera(cam, &c);
  if (st != VR_OK) return st;
  screen_rect(c, lo, hi, rect);
  return VR_OK;
}

vr_status vr_read_bounds_violations(vr_ctx* ctx, unsigned long long* count, void* stream) {
  if (!ctx || !count) return VR_ERR_INVALID_ARG;
  *count = 0;
#ifndef VR_DEBUG_BOUNDS
  (void)stream;
  return VR_ERR_UNSUPPORTED;
#else
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_status(cudaGetLastError());
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long h = 0;
  vr_status st = cuda_status(cudaMemcpyAsync(&h, ctx->stats + 7, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (st != VR_OK) return st;
  st = cuda_status(cudaStreamSynchronize(s));
  if (st == VR_OK) *count = h;
  return st;
#endif
}

const char* vr_status_string(vr_status s) {
  switch (s) {
    case VR_OK: return "ok";
    case VR_ERR_INVALID_ARG: return "invalid argument";
    case VR_ERR_OUT_OF_MEMORY: return "out of device memory";
    case VR_ERR_CUDA: return "CUDA error";
    case VR_ERR_UNSUPPORTED: return "unsupported";
    case VR_ERR_TIMEOUT: return "device-side wait timed out";
    case VR_ERR_STATE: return "invalid call order or state";
  }
  return "unknown status";
}

const char* vr_last_cuda_error(void) { return g_cuda_err; }

int vr_version(void) { return 100; }

}  // extern "C"
