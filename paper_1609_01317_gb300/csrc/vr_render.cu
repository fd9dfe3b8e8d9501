// vr_render.cu -- the fused forward ray march (§3.10 steps 1-4 in one kernel).
//
// One thread per ray.  A warp covers an 8x4 pixel tile and a block of four warps a 16x8
// tile, so neighbouring lanes sample neighbouring voxels.  Per ray: ray setup against the
// clip box (§3.3, §3.6), then for k = 0..K-1 the sample at t_k = t_near + (k + 1/2) step:
// skip to the next brick if the current one has zero opacity for this transfer function
// (§5.3), else trilinear value (§3.4) -> transfer function (§3.7) -> if alpha != 0:
// operator gradient (§3.5), normal and Phong (§3.8) -> front-to-back Eq. 6 (§3.9); stop
// once 1 - T >= the termination threshold.
#include "vr_internal.h"

namespace vr {

constexpr int kTileW = 16, kTileH = 8, kThreads = 128;

__device__ __forceinline__ void pixel_of(int& px, int& py) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  px = blockIdx.x * kTileW + (w & 1) * 8 + (lane & 7);
  py = blockIdx.y * kTileH + (w >> 1) * 4 + (lane >> 3);
}

template <int VTYPE, int OP, bool CKPT>
__global__ void __launch_bounds__(kThreads) k_march(const MarchLaunch L) {
  int px, py;
  pixel_of(px, py);
  const int W = L.cam.width, H = L.cam.height;
  const bool active = px < W && py < H;
  const int ray = py * W + px;
  float o[3], d[3], tn = 0.0f;
  int K = 0;
  if (active) ray_setup(L.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
  unsigned visited = 0, shaded = 0;
  int k = 0;
  const float step = L.r.step;
  extern __shared__ float4 ring_mem[];
  Ring ring;
  ring.base = ring_mem + threadIdx.x;
  ring.stride = kThreads;
  ring.ci[0] = ring.ci[1] = ring.ci[2] = -0x40000000;
  while (k < K) {
    if (CKPT && k > 0 && (k & (kCkptStride - 1)) == 0)
      L.ck_T[(size_t)((k >> 5) - 1) * (W * H) + ray] = T;
    const float t = fmaf((float)k + 0.5f, step, tn);
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
    if (L.r.skip) {
      int b[3];
      const int bi = brick_of(L.V, p, b);
      if (!__ldg(L.V.vis + bi)) {
        int kn = brick_exit_sample(b, o, d, tn, step);
        if (kn <= k) kn = k + 1;
        if (CKPT) {
          const int stop = kn < K ? kn : K;
          for (int j = ((k >> 5) + 1) << 5; j < stop; j += kCkptStride)
            L.ck_T[(size_t)((j >> 5) - 1) * (W * H) + ray] = T;
        }
        k = kn;
        continue;
      }
    }
    ++visited;
    const Cell c = cell_of(L.V, p);
    ring_update<VTYPE>(ring, L.V, c);
    const ZWeights zw = z_weights(c.f[2], (c.ib[2] - 1) & 3);
    const float s = ring_value(ring, c, zw);
    const TfSample ts = tf_lookup(L.tf, s);
    const float alpha = ts.rgba.w;
    if (alpha != 0.0f) {
      ++shaded;
      float g[3];
      ring_gradient<OP>(ring, c, zw, g);
      const float gh[3] = {g[0] * L.r.gscale, g[1] * L.r.gscale, g[2] * L.r.gscale};
      ShadeOut so;
      shade(L.r.sh, L.cam, d, p, gh, ts.rgba, so);
      const float ta = T * alpha;
      C0 = fmaf(ta, so.c[0], C0);
      C1 = fmaf(ta, so.c[1], C1);
      C2 = fmaf(ta, so.c[2], C2);
      T = T * (1.0f - alpha);
    }
    ++k;
    if (1.0f - T >= L.r.ert) break;
  }
  const int kend = k < K ? k : K;
  if (active) {
    reinterpret_cast<float4*>(L.out)[ray] = make_float4(C0, C1, C2, 1.0f - T);
    if (CKPT) L.ck_kend[ray] = kend;
  }
  if (L.stats) {
    unsigned hit = (active && K > 0) ? 1u : 0u;
    unsigned plain = active ? (unsigned)kend : 0u;
    hit = __reduce_add_sync(0xffffffffu, hit);
    plain = __reduce_add_sync(0xffffffffu, plain);
    visited = __reduce_add_sync(0xffffffffu, visited);
    shaded = __reduce_add_sync(0xffffffffu, shaded);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(L.stats + 0, (unsigned long long)hit);
      atomicAdd(L.stats + 1, (unsigned long long)plain);
      atomicAdd(L.stats + 2, (unsigned long long)visited);
      atomicAdd(L.stats + 3, (unsigned long long)shaded);
    }
  }
}

template <int VTYPE, int OP>
static void launch_typed(const MarchLaunch& L, dim3 grid, cudaStream_t s) {
  const size_t smem = sizeof(float4) * 16 * kThreads;
  if (L.ck_kend) k_march<VTYPE, OP, true><<<grid, kThreads, smem, s>>>(L);
  else k_march<VTYPE, OP, false><<<grid, kThreads, smem, s>>>(L);
}

template <int VTYPE>
static void launch_op(const MarchLaunch& L, dim3 grid, cudaStream_t s) {
  switch (L.op) {
    case OP_CENTRAL: launch_typed<VTYPE, OP_CENTRAL>(L, grid, s); break;
    case OP_SOBEL: launch_typed<VTYPE, OP_SOBEL>(L, grid, s); break;
    default: launch_typed<VTYPE, OP_ZH>(L, grid, s);
  }
}

cudaError_t launch_march(const MarchLaunch& L, cudaStream_t s) {
  const dim3 grid((L.cam.width + kTileW - 1) / kTileW, (L.cam.height + kTileH - 1) / kTileH);
  switch (L.dtype) {
    case VT_U8: launch_op<VT_U8>(L, grid, s); break;
    case VT_U16: launch_op<VT_U16>(L, grid, s); break;
    case VT_F16: launch_op<VT_F16>(L, grid, s); break;
    default: launch_op<VT_F32>(L, grid, s);
  }
  return cudaGetLastError();
}

}  // namespace vr
