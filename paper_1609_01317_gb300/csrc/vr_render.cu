// vr_render.cu -- the fused forward ray march (§3.10 steps 1-4 in one kernel).
//
// Four lanes per ray (a quad, each lane one of four consecutive samples); a warp marches a
// 4x2 pixel tile, so neighbouring lanes sample neighbouring voxels.  The kernel is persistent: a grid that fills the GPU once, each warp
// taking the next tile from an atomic counter, so a warp that finishes a cheap tile (rays
// that miss or cross empty space) immediately takes another and the frame's cost, which
// is concentrated where rays cross the object, spreads over all SMs.  Per ray: ray setup against the
// clip box (§3.3, §3.6), then for k = 0..K-1 the sample at t_k = t_near + (k + 1/2) step:
// skip to the next brick if the current one has zero opacity for this transfer function
// (§5.3), else read the 8 corner records (operator gradient G and value V) of the sample's
// cell, interpolate V trilinearly (§3.4) -> transfer function (§3.7) -> if alpha != 0:
// blend G over the corners (= the operator of §3.5 evaluated at the sample), normalise,
// Phong (§3.8) -> front-to-back Eq. 6 (§3.9); stop once 1 - T >= the threshold.
#include "vr_march.cuh"

namespace vr {

constexpr int kThreads = 128;
constexpr int kTileW = 4, kTileH = 2;  // one warp's pixels (a quad of lanes per ray)

constexpr int kMaxSharedTf = 1024;  // tables up to this many entries are copied to shared memory

// TFS: the block copies the transfer function (n <= kMaxSharedTf entries) to shared memory.
// ADAPT: adaptive sampling with the per-brick multipliers L.r.mult.
template <bool CKPT, bool TFS, bool ADAPT = false>
__global__ void __launch_bounds__(kThreads, 7) k_march(const MarchLaunch L) {
  extern __shared__ float4 s_tf[];
  if constexpr (TFS) {
    for (int i = threadIdx.x; i < L.tf.n; i += kThreads) s_tf[i] = L.tf.tf[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int q = lane & 3, qd = lane >> 2;
  const unsigned qmask = 0xFu << (lane & ~3);
  const int W = L.cam.width, H = L.cam.height;
  // tiles covering the pixel rectangle L.rect (every ray outside it misses the box)
  const int tx0 = L.rect[0] / kTileW, ty0 = L.rect[1] / kTileH;
  const int tiles_x = (L.rect[2] + kTileW - 1) / kTileW - tx0;
  const int tiles = tiles_x * ((L.rect[3] + kTileH - 1) / kTileH - ty0);
  unsigned hit = 0, plain = 0, visited = 0, shaded = 0;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(L.tile_counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= tiles) break;
    const int px = (tx0 + tile % tiles_x) * kTileW + (qd & 3);
    const int py = (ty0 + tile / tiles_x) * kTileH + (qd >> 2);
    march_ray<CKPT, TFS, ADAPT>(L, px, py, px < W && py < H, q, qmask, hit, plain, visited,
                                shaded, s_tf);
    __syncwarp();
  }
  if (L.stats) {
    hit = __reduce_add_sync(0xffffffffu, hit);
    plain = __reduce_add_sync(0xffffffffu, plain);
    visited = __reduce_add_sync(0xffffffffu, visited);
    shaded = __reduce_add_sync(0xffffffffu, shaded);
    if (lane == 0) {
      atomicAdd(L.stats + 0, (unsigned long long)hit);
      atomicAdd(L.stats + 1, (unsigned long long)plain);
      atomicAdd(L.stats + 2, (unsigned long long)visited);
      atomicAdd(L.stats + 3, (unsigned long long)shaded);
    }
  }
}

// Blocks that keep every SM busy once (the kernel is persistent).
template <bool CKPT, bool TFS, bool ADAPT>
static int persistent_blocks(size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march<CKPT, TFS, ADAPT>, kThreads, smem);
  return (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
}

template <bool CKPT, bool ADAPT>
static void launch_march_k(const MarchLaunch& L, cudaStream_t s) {
  if (L.tf.n <= kMaxSharedTf) {
    const size_t smem = sizeof(float4) * (size_t)L.tf.n;
    k_march<CKPT, true, ADAPT><<<persistent_blocks<CKPT, true, ADAPT>(smem), kThreads, smem, s>>>(L);
  } else {
    k_march<CKPT, false, ADAPT><<<persistent_blocks<CKPT, false, ADAPT>(0), kThreads, 0, s>>>(L);
  }
}

cudaError_t launch_march(const MarchLaunch& L, cudaStream_t s) {
  // the tile counter starts at zero for every launch
  cudaError_t e = cudaMemsetAsync(L.tile_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (L.ck_kend) launch_march_k<true, false>(L, s);
  else if (L.r.mult) launch_march_k<false, true>(L, s);
  else launch_march_k<false, false>(L, s);
  return cudaGetLastError();
}

}  // namespace vr
