// vr_render.cu -- the fused forward ray march (§3.10 steps 1-4 in one kernel).
//
// Four lanes per ray (a quad, each lane one of four consecutive samples); a warp marches
// eight rays of neighbouring pixels, so neighbouring lanes sample neighbouring voxels.  The
// kernel is persistent: a grid that fills the GPU once, each warp taking its next rays from
// an atomic counter, so a warp that finishes cheap rays (rays that miss or cross empty space)
// immediately takes others and the frame's cost, which is concentrated where rays cross the
// object, spreads over all SMs.  Per ray: ray setup against the clip box (§3.3, §3.6), then
// for k = 0..K-1 the sample at t_k = t_near + (k + 1/2) step: skip to the next brick if the
// current one has zero opacity for this transfer function (§5.3), else read the 8 corner
// records (operator gradient G and value V) of the sample's cell, interpolate V trilinearly
// (§3.4) -> transfer function (§3.7) -> if alpha != 0: blend G over the corners (= the
// operator of §3.5 evaluated at the sample), normalise, Phong (§3.8) -> front-to-back Eq. 6
// (§3.9); stop once 1 - T >= the threshold.
//
// Two ways to hand rays to the warps, chosen on the device for every plain render:
//   tiles  the warp takes a 4 x 2 pixel tile of the box's screen rectangle and sets up its
//          rays itself (dense data: the set-up and the approach through empty space hide
//          under the latency of the march);
//   list   with few visible bricks (sparse data, §5.4), k_ray_list first sets up every ray
//          of the rectangle with one thread per ray, walks it past the transparent macro and
//          super bricks and lists only the rays that reach a visible one; the warps then take
//          eight listed rays at a time and start each at its first visible group.
// Both give the same image bit for bit: a ray's samples before its first visible macro
// brick have zero opacity, and groups stay aligned to multiples of four samples either way.
#include "vr_march.cuh"

namespace vr {

constexpr int kThreads = 128;
constexpr int kTileW = 4, kTileH = 2;  // one warp's pixels (a quad of lanes per ray)

constexpr int kMaxSharedTf = 1024;  // tables up to this many entries are copied to shared memory

__device__ __forceinline__ bool list_mode(const MarchLaunch& L) {
  if (!L.list || !L.vis_count || !L.r.skip || !L.V.mvis || L.mode == 1) return false;
  if (L.mode == 2) return true;
  const long long nbricks = (long long)L.V.nb[0] * L.V.nb[1] * L.V.nb[2];
  return (long long)__ldg(L.vis_count) * kListDenom < nbricks;
}

// The first thread of the grid passes the visible-brick count on to the host for the next
// render's choice of march (mapped pinned memory; a posted write under a long kernel).
__device__ __forceinline__ void write_hint(const MarchLaunch& L) {
  if (L.hint && L.vis_count && blockIdx.x == 0 && threadIdx.x == 0) {
    L.hint[0] = __ldg(L.vis_count);
    L.hint[1] = L.V.nb[0] * L.V.nb[1] * L.V.nb[2];
  }
}

__device__ __forceinline__ void add_stats(const MarchLaunch& L, unsigned hit, unsigned plain,
                                          unsigned visited, unsigned shaded) {
  const int lane = threadIdx.x & 31;
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

// The march of tiles.  TFS: the block copies the transfer function (n <= kMaxSharedTf
// entries) to shared memory.  ADAPT: adaptive sampling with the per-brick multipliers
// L.r.mult.  A plain render in list mode returns at once (k_march_list marches it).
template <bool CKPT, bool TFS, bool ADAPT = false, bool ZWIN = false>
__global__ void __launch_bounds__(kThreads, 8) k_march(const MarchLaunch L) {
  if constexpr (!CKPT && !ADAPT && !ZWIN) {
    write_hint(L);
    if (list_mode(L)) return;
  }
  extern __shared__ float4 s_tf[];
  if constexpr (TFS) {
    for (int i = threadIdx.x; i < L.tf.n; i += kThreads) s_tf[i] = L.tf.tf[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int q = lane & 3, qd = lane >> 2;
  const unsigned qmask = 0xFu << (lane & ~3);
  const int W = L.cam.width, H = L.cam.height;
  // work counter of this launch: in the list's head when a list buffer is given
  unsigned* counter = L.list ? reinterpret_cast<unsigned*>(L.list_head + 1) : L.tile_counter;
  unsigned hit = 0, plain = 0, visited = 0, shaded = 0;
  // tiles covering the pixel rectangle L.rect (every ray outside it misses the box)
  const int tx0 = L.rect[0] / kTileW, ty0 = L.rect[1] / kTileH;
  const int tiles_x = (L.rect[2] + kTileW - 1) / kTileW - tx0;
  const int tiles = tiles_x * ((L.rect[3] + kTileH - 1) / kTileH - ty0);
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= tiles) break;
    const int px = (tx0 + tile % tiles_x) * kTileW + (qd & 3);
    const int py = (ty0 + tile / tiles_x) * kTileH + (qd >> 2);
    march_ray<CKPT, TFS, ADAPT, ZWIN>(L, px, py, px < W && py < H && py >= L.row0 && py < L.row1,
                                      q, qmask, hit, plain, visited, shaded, s_tf);
    __syncwarp();
  }
  if (L.stats) add_stats(L, hit, plain, visited, shaded);
}

// The march of the listed rays of a plain render in list mode (returns at once otherwise):
// persistent, each warp takes the next 8 rays of the list (neighbouring pixels: the list
// keeps the tiles' order), a quad of lanes per ray, from each ray's first visible group.
template <bool TFS>
__global__ void __launch_bounds__(kThreads, 8) k_march_list(const MarchLaunch L) {
  write_hint(L);
  if (!list_mode(L)) return;
  extern __shared__ float4 s_tf[];
  if constexpr (TFS) {
    for (int i = threadIdx.x; i < L.tf.n; i += kThreads) s_tf[i] = L.tf.tf[i];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int q = lane & 3, qd = lane >> 2;
  const unsigned qmask = 0xFu << (lane & ~3);
  unsigned* counter = reinterpret_cast<unsigned*>(L.list_head + 1);
  const int n = L.list_head[0];
  unsigned hit = 0, plain = 0, visited = 0, shaded = 0;
  for (;;) {
    int base = 0;
    if (lane == 0) base = (int)atomicAdd(counter, 8u);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    const int idx = base + qd;
    const bool active = idx < n;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f}, tn = 0.0f;
    int K = 0, k0 = 0, px = 0, py = L.row0;
    if (active) {
      const RayRec* r = L.list + VR_CHECK(L.V.bounds, idx, 0, n - 1);
      const float4 a = __ldg(&r->o_tn), b = __ldg(&r->d_K);
      const int4 c = __ldg(&r->px_py_k0);
      o[0] = a.x; o[1] = a.y; o[2] = a.z; tn = a.w;
      d[0] = b.x; d[1] = b.y; d[2] = b.z; K = __float_as_int(b.w);
      px = c.x; py = c.y; k0 = c.z;
    }
    // no inner jump loop here: on sparse data a quad's runs of jumps are long and uneven, and
    // the quads that reached a visible group would wait for the longest run (measured slower)
    march_core<false, TFS, false, false, false>(L, o, d, tn, K, k0, px, py, active, q, qmask,
                                                hit, plain, visited, shaded, s_tf);
    __syncwarp();
  }
  if (L.stats) add_stats(L, hit, plain, visited, shaded);
}

// Ray set-up of a plain render in list mode, one thread per pixel of the rectangle's tiles
// (the same 4 x 2 tiles, in the same order, as the tile march): the slab test of §3.3 / §3.6,
// then the march's own rule for transparent regions (§5.3, §5.4) walked on one lane -- from
// the entry, while the sample lies in a transparent super brick or macro brick, jump to the
// first sample past it.  A ray that reaches a visible macro brick is appended to the list
// with the aligned group of that sample as its first group (every sample before it lies in
// transparent regions: zero opacity, so starting there changes no bit of the result); the
// pixel of any other ray is written as (0, 0, 0, 0), and with counting its samples are
// counted here.  Lanes append with one atomic per warp, in lane order, so the list keeps the
// tiles' order.  Outside list mode the kernel returns at once.
__global__ void __launch_bounds__(256) k_ray_list(const MarchLaunch L) {
  if (!list_mode(L)) return;
  const int lane = threadIdx.x & 31;
  const int W = L.cam.width, H = L.cam.height;
  const int tx0 = L.rect[0] / kTileW, ty0 = L.rect[1] / kTileH;
  const int tiles_x = (L.rect[2] + kTileW - 1) / kTileW - tx0;
  const int tiles = tiles_x * ((L.rect[3] + kTileH - 1) / kTileH - ty0);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int tile = t >> 3, slot = t & 7;
  const int px = (tx0 + tile % tiles_x) * kTileW + (slot & 3);
  const int py = (ty0 + tile / tiles_x) * kTileH + (slot >> 2);
  const bool active = tile < tiles && px < W && py < H && py >= L.row0 && py < L.row1;
  float o[3], d[3], tn = 0.0f;
  int K = 0;
  if (active) ray_setup(L.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
  int k = 0;
  if (K > 0) {
    const float step = L.r.step, inv_step = 1.0f / step;
    float inv_d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) inv_d[a] = d[a] != 0.0f ? 1.0f / d[a] : 0.0f;
    const int nmacro = L.V.nm[0] * L.V.nm[1] * L.V.nm[2];
    const int nsuper = L.V.ns[0] * L.V.ns[1] * L.V.ns[2];
    while (k < K) {
      const float tk = fmaf((float)k + 0.5f, step, tn);
      float p[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = fmaf(tk, d[a], o[a]);
      int b[3];
      brick_of(L.V, p, b);
      const int m[3] = {b[0] >> kMacroShift, b[1] >> kMacroShift, b[2] >> kMacroShift};
      const int u[3] = {m[0] >> kSuperShift, m[1] >> kSuperShift, m[2] >> kSuperShift};
      int kn;
      if (L.V.svis && !__ldg(L.V.svis + VR_CHECK(L.V.bounds, u[0] + L.V.ns[0] * (u[1] + L.V.ns[1] * u[2]),
                                                 0, nsuper - 1))) {
        kn = region_exit_sample(u, kBrickShift + kMacroShift + kSuperShift, o, d, inv_d, tn,
                                inv_step);
      } else {
        if (__ldg(L.V.mvis + VR_CHECK(L.V.bounds, m[0] + L.V.nm[0] * (m[1] + L.V.nm[1] * m[2]), 0,
                                      nmacro - 1)))
          break;
        kn = region_exit_sample(m, kBrickShift + kMacroShift, o, d, inv_d, tn, inv_step);
      }
      k = kn > k ? kn : k + 1;
    }
  }
  const bool listed = active && k < K;
  const unsigned m = __ballot_sync(0xffffffffu, listed);
  int base = 0;
  if (lane == 0 && m) base = atomicAdd(L.list_head, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (listed) {
    RayRec r;
    r.o_tn = make_float4(o[0], o[1], o[2], tn);
    r.d_K = make_float4(d[0], d[1], d[2], __int_as_float(K));
    r.px_py_k0 = make_int4(px, py, k & ~3, 0);
    L.list[base + __popc(m & ((1u << lane) - 1u))] = r;
  } else if (active) {
    reinterpret_cast<float4*>(L.out)[(size_t)(py - L.row0) * W + px] =
        make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  if (L.stats) {
    // rays that meet the box but no visible macro brick: every sample is a plain sample
    const unsigned hit = __reduce_add_sync(0xffffffffu, (active && !listed && K > 0) ? 1u : 0u);
    const unsigned plain = __reduce_add_sync(0xffffffffu, (active && !listed) ? (unsigned)K : 0u);
    if (lane == 0 && hit) {
      atomicAdd(L.stats + 0, (unsigned long long)hit);
      atomicAdd(L.stats + 1, (unsigned long long)plain);
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

template <bool TFS>
static int persistent_list_blocks(size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_list<TFS>, kThreads, smem);
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
  const bool plain = L.list && !L.ck_kend && !L.r.mult;
  // the work counter (and, for a plain render, the list's length) start at zero per launch
  cudaError_t e = plain ? cudaMemsetAsync(L.list_head, 0, 2 * sizeof(int), s)
                        : cudaMemsetAsync(L.tile_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (plain) {
    const long tiles = (long)((L.rect[2] + kTileW - 1) / kTileW - L.rect[0] / kTileW) *
                       ((L.rect[3] + kTileH - 1) / kTileH - L.rect[1] / kTileH);
    if (tiles <= 0) return cudaSuccess;  // every pixel was cleared: no ray meets the box
    if (L.mode != 1) {
      // list mode (L.mode 2), or decided on the device (L.mode 0): then k_ray_list and
      // k_march_list return at once outside list mode and the tile march inside it
      k_ray_list<<<(unsigned)((tiles * 8 + 255) / 256), 256, 0, s>>>(L);
      if (L.tf.n <= kMaxSharedTf) {
        const size_t smem = sizeof(float4) * (size_t)L.tf.n;
        k_march_list<true><<<persistent_list_blocks<true>(smem), kThreads, smem, s>>>(L);
      } else {
        k_march_list<false><<<persistent_list_blocks<false>(0), kThreads, 0, s>>>(L);
      }
      if (L.mode == 2) return cudaGetLastError();
    }
  }
  if (L.ck_kend) launch_march_k<true, false>(L, s);
  else if (L.r.mult) launch_march_k<false, true>(L, s);
  else launch_march_k<false, false>(L, s);
  return cudaGetLastError();
}

cudaError_t launch_march_zwin(const MarchLaunch& L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(L.tile_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (L.rect[2] <= L.rect[0] || L.rect[3] <= L.rect[1]) return cudaSuccess;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (L.tf.n <= kMaxSharedTf) {
    const size_t smem = sizeof(float4) * (size_t)L.tf.n;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march<false, true, false, true>, kThreads, smem);
    k_march<false, true, false, true><<<(sms > 0 ? sms : 152) * (per > 0 ? per : 1), kThreads, smem, s>>>(L);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march<false, false, false, true>, kThreads, 0);
    k_march<false, false, false, true><<<(sms > 0 ? sms : 152) * (per > 0 ? per : 1), kThreads, 0, s>>>(L);
  }
  return cudaGetLastError();
}

}  // namespace vr
