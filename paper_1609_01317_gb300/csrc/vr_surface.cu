// vr_surface.cu -- first-hit surface rendering (§3.11) with hitpoint refinement (§5.1).
//
// The paper's own renderer shows surfaces only: a threshold window of voxel values marks
// solid matter, the ray advances in large steps until a sample falls inside the window, and
// the entry point is then searched backwards with ever smaller steps.  Here: coarse samples
// on the sample grid of the direct renderer, the first one inside the window ends the
// march, bisection between it and the previous sample refines the hit, and the hit is
// shaded once with the operator gradient and Phong.
//
// One thread per ray (the work per ray is a short march plus a few refinement samples, so
// there is nothing to share between lanes); persistent warps take 8 x 4 pixel tiles from an
// atomic counter.  Every FP32 operation that decides inside / outside is written as an
// explicit fused multiply-add or a separately rounded intrinsic, so the decisions do not
// depend on the compiler's contraction choices.  Coarse samples in bricks whose footprint
// value range misses the window are skipped (exact: a trilinear value lies within the range
// of its eight corners, all inside the footprint).
#include <cmath>
#include <cstring>

#include "vr_internal.h"

namespace vr {

struct SurfaceLaunch {
  VolDev V;   // padded volume; vis / mvis: bricks whose footprint can meet the window
  CamDev cam;
  float step, lo, hi;
  int refine;
  int skip;
  float rlo[3], rhi[3];  // sampling box
  float gscale;
  ShadeDev sh;
  float color[3];
  float4* out;
  float* depth;
  unsigned* counter;
  int rect[4];  // pixels whose tiles are marched; every other ray misses the sampling box
};

// No-hit output (0, 0, 0, 0) and depth +inf for every pixel, before a march restricted to
// the box's screen rectangle.
__global__ void k_surface_clear(float4* __restrict__ out, float* __restrict__ depth, int n) {
  const float inf = __int_as_float(0x7f800000);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    out[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (depth) depth[i] = inf;
  }
}

// Footprint range [min, max] meets the window, widened by a relative 1e-6 (FP32 lerps of
// non-integer voxel values may leave the corners' range by an ulp).
__global__ void k_surface_visibility(const float2* __restrict__ mm, int nbx, int nby, int nbricks,
                                     float lo, float hi, uint8_t* __restrict__ vis,
                                     uint8_t* __restrict__ mvis, int nmx, int nmy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbricks) return;
  const float2 m = mm[i];
  const float slo = fmaf(-1e-6f, fabsf(lo), lo) - 1e-30f;
  const float shi = fmaf(1e-6f, fabsf(hi), hi) + 1e-30f;
  const float mlo = fmaf(-1e-6f, fabsf(m.x), m.x), mhi = fmaf(1e-6f, fabsf(m.y), m.y);
  const bool v = mhi >= slo && mlo <= shi;
  vis[i] = v ? 1 : 0;
  if (v) {
    const int bx = i % nbx, by = (i / nbx) % nby, bz = i / (nbx * nby);
    mvis[(bx >> kMacroShift) + nmx * ((by >> kMacroShift) + nmy * (bz >> kMacroShift))] = 1;
  }
}

template <int VTYPE>
__device__ __forceinline__ bool inside_at(const SurfaceLaunch& L, const float o[3], const float d[3],
                                          float t) {
  float p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
  const float s = trilinear<VTYPE>(L.V, cell_of(L.V, p));
  return s >= L.lo && s <= L.hi;
}

// One ray of pixel (px, py): coarse march, refinement, shading.
template <int VTYPE, int OP>
__device__ __forceinline__ void surface_ray(const SurfaceLaunch& L, int px, int py) {
  const int ray = py * L.cam.width + px;
  float o[3], d[3], tn = 0.0f;
  int K = 0;
  ray_setup(L.cam, L.rlo, L.rhi, L.step, px, py, o, d, tn, K);
  const float inv_step = 1.0f / L.step;
  float inv_d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) inv_d[a] = d[a] != 0.0f ? 1.0f / d[a] : 0.0f;
  // coarse march to the first sample inside the window
  int k = 0;
  while (k < K) {
    const float t = fmaf((float)k + 0.5f, L.step, tn);
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
    if (L.skip) {
      int b[3];
      const int bi = brick_of(L.V, p, b);
      if (!__ldg(L.V.vis + VR_CHECK(L.V.bounds, bi, 0, L.V.nb[0] * L.V.nb[1] * L.V.nb[2] - 1))) {
        int shift = kBrickShift;
        const int m[3] = {b[0] >> kMacroShift, b[1] >> kMacroShift, b[2] >> kMacroShift};
        if (!__ldg(L.V.mvis + VR_CHECK(L.V.bounds, m[0] + L.V.nm[0] * (m[1] + L.V.nm[1] * m[2]),
                                       0, L.V.nm[0] * L.V.nm[1] * L.V.nm[2] - 1))) {
          b[0] = m[0];
          b[1] = m[1];
          b[2] = m[2];
          shift = kBrickShift + kMacroShift;
        }
        const int kn = region_exit_sample(b, shift, o, d, inv_d, tn, inv_step);
        k = kn > k ? kn : k + 1;
        continue;
      }
    }
    const float s = trilinear<VTYPE>(L.V, cell_of(L.V, p));
    if (s >= L.lo && s <= L.hi) break;
    ++k;
  }
  if (k >= K) {
    L.out[ray] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (L.depth) L.depth[ray] = __int_as_float(0x7f800000);
    return;
  }
  // refinement: bisection keeping ta outside and tb inside (§5.1)
  float t_hit;
  if (k == 0 && inside_at<VTYPE>(L, o, d, tn)) {
    t_hit = tn;
  } else {
    float ta = k == 0 ? tn : fmaf((float)k - 0.5f, L.step, tn);
    float tb = fmaf((float)k + 0.5f, L.step, tn);
    for (int r = 0; r < L.refine; ++r) {
      const float mid = __fmul_rn(0.5f, __fadd_rn(ta, tb));
      if (inside_at<VTYPE>(L, o, d, mid)) tb = mid;
      else ta = mid;
    }
    t_hit = __fmul_rn(0.5f, __fadd_rn(ta, tb));
  }
  // shading at the hit: operator gradient, normal turned to the viewer, Phong
  float p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) p[a] = fmaf(t_hit, d[a], o[a]);
  float s, g[3];
  value_and_gradient<VTYPE, OP>(L.V, cell_of(L.V, p), s, g);
  float gh[3] = {g[0] * L.gscale, g[1] * L.gscale, g[2] * L.gscale};
  // N = -gh/|gh| must satisfy N.d <= 0, i.e. gh.d >= 0
  if (gh[0] * d[0] + gh[1] * d[1] + gh[2] * d[2] < 0.0f) {
    gh[0] = -gh[0];
    gh[1] = -gh[1];
    gh[2] = -gh[2];
  }
  ShadeOut so;
  shade(L.sh, L.cam, d, p, gh, make_float4(L.color[0], L.color[1], L.color[2], 1.0f), so);
  L.out[ray] = make_float4(so.c[0], so.c[1], so.c[2], 1.0f);
  if (L.depth) L.depth[ray] = t_hit;
}

template <int VTYPE, int OP>
__global__ void __launch_bounds__(128) k_surface(const SurfaceLaunch L) {
  const int lane = threadIdx.x & 31;
  const int W = L.cam.width, H = L.cam.height;
  const int tx0 = L.rect[0] / 8, ty0 = L.rect[1] / 4;
  const int tiles_x = (L.rect[2] + 7) / 8 - tx0;
  const int tiles = tiles_x * ((L.rect[3] + 3) / 4 - ty0);
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(L.counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= tiles) break;
    const int px = (tx0 + tile % tiles_x) * 8 + (lane & 7);
    const int py = (ty0 + tile / tiles_x) * 4 + (lane >> 3);
    if (px < W && py < H) surface_ray<VTYPE, OP>(L, px, py);
    __syncwarp();
  }
}

static int surface_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 152) * 8;
}

template <int VTYPE>
static void launch_surface_op(const SurfaceLaunch& L, int op, cudaStream_t s) {
  const int blocks = surface_grid();
  switch (op) {
    case OP_CENTRAL: k_surface<VTYPE, OP_CENTRAL><<<blocks, 128, 0, s>>>(L); break;
    case OP_SOBEL: k_surface<VTYPE, OP_SOBEL><<<blocks, 128, 0, s>>>(L); break;
    default: k_surface<VTYPE, OP_ZH><<<blocks, 128, 0, s>>>(L);
  }
}

}  // namespace vr

using namespace vr;

namespace {

vr_status check_surface_params(const vr_surface_params* p) {
  if (!p) return VR_ERR_INVALID_ARG;
  if (!(p->step > 0.0f) || !std::isfinite(p->step)) return VR_ERR_INVALID_ARG;
  if (std::isnan(p->iso_lo) || std::isnan(p->iso_hi) || p->iso_lo > p->iso_hi)
    return VR_ERR_INVALID_ARG;
  if (p->refine < 0 || p->refine > 24) return VR_ERR_INVALID_ARG;
  if (p->grad < VR_GRAD_CENTRAL || p->grad > VR_GRAD_ZUCKER_HUMMEL) return VR_ERR_INVALID_ARG;
  if (!(p->shininess >= 0.0f) || !std::isfinite(p->shininess)) return VR_ERR_INVALID_ARG;
  if (!std::isfinite(p->ka) || !std::isfinite(p->kd) || !std::isfinite(p->ks))
    return VR_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(p->light[a]) || !std::isfinite(p->color[a])) return VR_ERR_INVALID_ARG;
    if (std::isnan(p->clip_lo[a]) || std::isnan(p->clip_hi[a])) return VR_ERR_INVALID_ARG;
  }
  return VR_OK;
}

}  // namespace

extern "C" vr_status vr_render_surface(vr_ctx* ctx, const vr_surface_params* params,
                                       float* out_rgba, float* out_depth, void* stream) {
  TraceRange trace_("vr_render_surface");
  if (!ctx || !out_rgba) return VR_ERR_INVALID_ARG;
  vr_status st = check_surface_params(params);
  if (st != VR_OK) return st;
  if (!ctx->has_volume || !ctx->has_camera) return VR_ERR_STATE;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, ctx->device};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t npix = (size_t)ctx->cam.width * ctx->cam.height;
  const bool host_rgba = !is_device_pointer(out_rgba);
  const bool host_depth = out_depth && !is_device_pointer(out_depth);
  if ((!host_rgba && !aligned_to(out_rgba, 16)) ||
      (out_depth && !host_depth && !aligned_to(out_depth, 4)))
    return VR_ERR_INVALID_ARG;
  // device staging for host outputs: image, then depth
  const size_t img_bytes = npix * sizeof(float4), depth_bytes = npix * sizeof(float);
  if (host_rgba || host_depth) {
    st = ensure(ctx, &ctx->out_staging, &ctx->out_cap, img_bytes + depth_bytes);
    if (st != VR_OK) return st;
  }
  float* dst = host_rgba ? static_cast<float*>(ctx->out_staging) : out_rgba;
  float* ddst = out_depth;
  if (host_depth)
    ddst = reinterpret_cast<float*>(static_cast<char*>(ctx->out_staging) + img_bytes);
  // brick and macro-brick visibility for the window
  const int nbricks = ctx->nb[0] * ctx->nb[1] * ctx->nb[2];
  const int nmacro = ctx->nm[0] * ctx->nm[1] * ctx->nm[2];
  st = ensure(ctx, &ctx->surf_vis, &ctx->surf_vis_cap, 256 + (size_t)nbricks + nmacro);
  if (st != VR_OK) return st;
  uint8_t* svis = static_cast<uint8_t*>(ctx->surf_vis);
  uint8_t* smvis = svis + nbricks;
  unsigned* counter = reinterpret_cast<unsigned*>(ctx->stats + 6);
  if (params->skip_empty) {
    st = cuda_status(cudaMemsetAsync(smvis, 0, nmacro, s));
    if (st != VR_OK) return st;
    k_surface_visibility<<<(nbricks + 255) / 256, 256, 0, s>>>(
        ctx->brick_minmax, ctx->nb[0], ctx->nb[1], nbricks, params->iso_lo, params->iso_hi, svis,
        smvis, ctx->nm[0], ctx->nm[1]);
    st = cuda_status(cudaGetLastError());
    if (st != VR_OK) return st;
  }
  SurfaceLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.V = vol_dev(ctx);
  L.V.vis = svis;
  L.V.mvis = smvis;
  L.cam = ctx->camdev;
  L.step = params->step;
  L.lo = params->iso_lo;
  L.hi = params->iso_hi;
  L.refine = params->refine;
  L.skip = params->skip_empty ? 1 : 0;
  for (int a = 0; a < 3; ++a) {
    const float vhi = (float)(ctx->n[a] - 1);
    L.rlo[a] = params->clip_lo[a] > 0.0f ? params->clip_lo[a] : 0.0f;
    L.rhi[a] = params->clip_hi[a] < vhi ? params->clip_hi[a] : vhi;
    L.sh.light[a] = params->light[a];
    L.color[a] = params->color[a];
  }
  L.gscale = op_scale(params->grad) / ctx->value_max;
  L.sh.ka = params->ka;
  L.sh.kd = params->kd;
  L.sh.ks = params->ks;
  L.sh.shininess = params->shininess;
  L.sh.headlight = params->headlight ? 1 : 0;
  L.out = reinterpret_cast<float4*>(dst);
  L.depth = ddst;
  L.counter = counter;
  st = cuda_status(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  if (st != VR_OK) return st;
  // march the tiles of the sampling box's screen rectangle; clear the rest first
  screen_rect(L.cam, L.rlo, L.rhi, L.rect);
  if (L.rect[0] > 0 || L.rect[1] > 0 || L.rect[2] < L.cam.width || L.rect[3] < L.cam.height) {
    k_surface_clear<<<surface_grid(), 256, 0, s>>>(L.out, L.depth, (int)npix);
    st = cuda_status(cudaGetLastError());
    if (st != VR_OK) return st;
  }
  switch (ctx->dtype) {
    case VR_U8: launch_surface_op<VT_U8>(L, params->grad, s); break;
    case VR_U16: launch_surface_op<VT_U16>(L, params->grad, s); break;
    case VR_F16: launch_surface_op<VT_F16>(L, params->grad, s); break;
    default: launch_surface_op<VT_F32>(L, params->grad, s);
  }
  st = cuda_status(cudaGetLastError());
  if (st != VR_OK) return st;
  if (host_rgba) st = cuda_status(cudaMemcpyAsync(out_rgba, dst, img_bytes, cudaMemcpyDeviceToHost, s));
  if (st == VR_OK && host_depth)
    st = cuda_status(cudaMemcpyAsync(out_depth, ddst, depth_bytes, cudaMemcpyDeviceToHost, s));
  return st;
}
