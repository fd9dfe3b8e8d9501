// vr_probe.cu -- the march's per-sample stages at caller-given points (testing aid).
//
// For each point p the kernel runs exactly the device functions the march runs for a sample
// at p: the cell and its 8 corner gradient records, the trilinear value (§3.4), the transfer
// function (§3.7), the operator gradient blended over the corners (§3.5) and Phong (§3.8)
// for the current camera's view of p, so each stage can be compared on its own with the
// definition it implements.
#include <cstring>

#include "vr_march.cuh"

namespace vr {
namespace {

constexpr int kProbeOut = 12;

__global__ void k_probe(const MarchLaunch L, const float* __restrict__ pos, int n,
                        float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  const Cell c = cell_of(L.V, p);
  Corners cr;
  corners_load(L.R, c, cr);
  const float4 bl = corners_blend(cr, c);
  const float s = bl.w;
  const TfSample ts = tf_lookup<false>(L.tf, s);
  const float g[3] = {bl.x, bl.y, bl.z};
  const float gh[3] = {g[0] * L.r.gscale, g[1] * L.r.gscale, g[2] * L.r.gscale};
  // the direction of the camera ray through p
  float d[3];
  if (L.cam.ortho) {
    for (int a = 0; a < 3; ++a) d[a] = L.cam.fwd[a];
  } else {
    float e[3];
    for (int a = 0; a < 3; ++a) e[a] = p[a] - L.cam.eye[a];
    const float il = rsqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    for (int a = 0; a < 3; ++a) d[a] = e[a] * il;
  }
  ShadeOut so;
  shade(L.r.sh, L.cam, d, p, gh, ts.rgba, so);
  float* o = out + (size_t)kProbeOut * i;
  o[0] = s / L.V.value_max;
  o[1] = ts.rgba.x;
  o[2] = ts.rgba.y;
  o[3] = ts.rgba.z;
  o[4] = ts.rgba.w;
  o[5] = gh[0];
  o[6] = gh[1];
  o[7] = gh[2];
  o[8] = so.c[0];
  o[9] = so.c[1];
  o[10] = so.c[2];
  o[11] = so.gl;
}

}  // namespace
}  // namespace vr

using namespace vr;

vr_status vr_probe_samples(vr_ctx* ctx, const vr_render_params* params, const float* pos, int n,
                           float* out, void* stream) {
  TraceRange trace_("vr_probe_samples");
  if (!ctx || !pos || !out || n < 0) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->adaptive) return VR_ERR_UNSUPPORTED;
  if (!ctx->has_volume || !ctx->has_tf || !ctx->has_camera) return VR_ERR_STATE;
  if (!is_device_pointer(pos) || !is_device_pointer(out)) return VR_ERR_INVALID_ARG;
  if (!aligned_to(pos, 4) || !aligned_to(out, 4)) return VR_ERR_INVALID_ARG;
  if (n == 0) return VR_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return VR_ERR_CUDA;
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, ctx->device};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // records of every brick (a probe point may lie in a brick the renderer would skip)
  vr_render_params all = *params;
  all.skip_empty = 0;
  st = ensure_records(ctx, &all, s);
  if (st != VR_OK) return st;
  MarchLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.V = vol_dev(ctx);
  L.R = rec_dev(ctx);
  L.tf = tf_dev(ctx);
  L.cam = ctx->camdev;
  L.r = render_dev(ctx, &all);
  k_probe<<<(n + 127) / 128, 128, 0, s>>>(L, pos, n, out);
  return cuda_status(cudaGetLastError());
}
