// vr_noalloc.cu -- vr_render_noalloc: a render that allocates no device memory.
//
// Some callers cannot allocate device memory at render time: a plug-in hosted by an
// application that owns the whole device memory pool and hands out only the buffers it
// manages, a real-time loop with a fixed memory budget that must not allocate per frame,
// or a process whose device memory is already reserved in full by another framework's
// caching allocator.  vr_render_noalloc serves them: the caller passes the volume, the
// transfer function and the output image (device memory it already owns), and the
// library's own scratch -- the per-brick min/max and visibility tables of empty-space
// skipping, the transfer-function prefix counts and the work counter of the persistent
// march -- lives in the file-scope array below, which every GPU that loads the library
// keeps until the process exits.
//
// The kernels are variants of the context path's: the volume is read in place with
// clamp-to-edge index arithmetic (no padded copy) and the operator gradient is evaluated
// from each sample's 4x4x4 neighbourhood (no gradient records), so the only scratch is the
// small tables above.
#include <mutex>

#include "vr_internal.h"

namespace vr {

constexpr int kNoAllocMaxBricks = 1 << 18;  // e.g. 512^3 voxels
constexpr int kNoAllocMaxTf = 4096;
constexpr size_t kNaCounterOff = 0;
constexpr size_t kNaMinMaxOff = 256;
constexpr size_t kNaVisOff = kNaMinMaxOff + sizeof(float2) * kNoAllocMaxBricks;
constexpr size_t kNaPrefixOff = kNaVisOff + kNoAllocMaxBricks;
constexpr size_t kNaBytes = kNaPrefixOff + sizeof(int) * (kNoAllocMaxTf + 1);

// The scratch of every vr_render_noalloc call on this device (about 2.3 MiB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch per device ordinal (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).
constexpr int kNaMaxDevices = 64;
static void* g_na_addr[kNaMaxDevices];
static std::mutex g_na_mutex;

static vr_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kNaMaxDevices) return VR_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_status(e);
    g_na_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_na_addr[dev]);
  return VR_OK;
}

// Unpadded volume read in place.
struct RawVol {
  const void* data;
  int n[3];
  int sy, sz;  // element strides of y and z
};

template <int VTYPE>
struct ClampedHood {
  const typename VoxelT<VTYPE>::T* v;
  int xs[4], ys[4], zs[4];  // clamped offsets of i0 - 1 .. i0 + 2 per axis
  __device__ __forceinline__ float operator()(int a, int b, int c) const {
    return ldv<VTYPE>(v, xs[a] + ys[b] + zs[c]);
  }
};

// Brick footprint min / max read from the unpadded volume (one warp per brick).
template <int VTYPE>
__global__ void k_na_minmax(const RawVol R, const int nb0, const int nb1, const int nbricks,
                            float2* __restrict__ mm) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nbricks) return;
  const int bx = warp % nb0, by = (warp / nb0) % nb1, bz = warp / (nb0 * nb1);
  const int b[3] = {bx, by, bz};
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = max((b[a] << kBrickShift) - 1, 0);
    hi[a] = min((b[a] << kBrickShift) + kBrick + 1, R.n[a] - 1);
  }
  const int ey = hi[1] - lo[1] + 1, nrows = ey * (hi[2] - lo[2] + 1);
  const auto* v = static_cast<const typename VoxelT<VTYPE>::T*>(R.data);
  float vmin = __int_as_float(0x7f800000), vmax = -vmin;
  for (int r = lane; r < nrows; r += 32) {
    const int y = lo[1] + r % ey, z = lo[2] + r / ey;
    const int row = y * R.sy + z * R.sz;
    for (int x = lo[0]; x <= hi[0]; ++x) {
      const float val = ldv<VTYPE>(v, row + x);
      vmin = fminf(vmin, val);
      vmax = fmaxf(vmax, val);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  if (lane == 0) mm[warp] = make_float2(vmin, vmax);
}

struct NaLaunch {
  RawVol R;
  VolDev V;  // brick grid and visibility (no voxel data)
  TfDev tf;
  CamDev cam;
  RenderDev r;
  float4* out;
  unsigned* counter;
};

// Persistent march, one thread per ray, warps take 8x4 pixel tiles from the counter.
template <int VTYPE, int OP>
__global__ void __launch_bounds__(128) k_na_march(const NaLaunch L) {
  const int lane = threadIdx.x & 31;
  const int W = L.cam.width, H = L.cam.height;
  const int tiles_x = (W + 7) / 8;
  const int tiles = tiles_x * ((H + 3) / 4);
  const auto* v = static_cast<const typename VoxelT<VTYPE>::T*>(L.R.data);
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(L.counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= tiles) break;
    const int px = (tile % tiles_x) * 8 + (lane & 7);
    const int py = (tile / tiles_x) * 4 + (lane >> 3);
    const bool active = px < W && py < H;
    float o[3], d[3], tn = 0.0f;
    int K = 0;
    if (active) ray_setup(L.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
    int k = 0;
    while (k < K) {
      const float t = fmaf((float)k + 0.5f, L.r.step, tn);
      float p[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
      if (L.r.skip) {
        int b[3];
        const int bi = brick_of(L.V, p, b);
        if (!__ldg(L.V.vis + bi)) {
          const int kn = brick_exit_sample(b, o, d, tn, L.r.step);
          k = kn > k ? kn : k + 1;
          continue;
        }
      }
      ClampedHood<VTYPE> nb;
      nb.v = v;
      float f[3];
      int i0[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int i = (int)floorf(p[a]);
        const int top = L.R.n[a] > 1 ? L.R.n[a] - 2 : 0;
        i = i < 0 ? 0 : (i > top ? top : i);
        i0[a] = i;
        f[a] = p[a] - (float)i;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        nb.xs[j] = min(max(i0[0] - 1 + j, 0), L.R.n[0] - 1);
        nb.ys[j] = min(max(i0[1] - 1 + j, 0), L.R.n[1] - 1) * L.R.sy;
        nb.zs[j] = min(max(i0[2] - 1 + j, 0), L.R.n[2] - 1) * L.R.sz;
      }
      const float x00 = lerpf(nb(1, 1, 1), nb(2, 1, 1), f[0]);
      const float x10 = lerpf(nb(1, 2, 1), nb(2, 2, 1), f[0]);
      const float x01 = lerpf(nb(1, 1, 2), nb(2, 1, 2), f[0]);
      const float x11 = lerpf(nb(1, 2, 2), nb(2, 2, 2), f[0]);
      const float s = lerpf(lerpf(x00, x10, f[1]), lerpf(x01, x11, f[1]), f[2]);
      const TfSample ts = tf_lookup(L.tf, s);
      const float alpha = ts.rgba.w;
      if (alpha != 0.0f) {
        float sv, g[3];
        contract_neighbourhood<OP>(nb, f, sv, g);
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
    if (active) L.out[py * W + px] = make_float4(C0, C1, C2, 1.0f - T);
    __syncwarp();
  }
}

template <int VTYPE>
static void na_launch_op(const NaLaunch& L, int op, int blocks, cudaStream_t s) {
  switch (op) {
    case OP_CENTRAL: k_na_march<VTYPE, OP_CENTRAL><<<blocks, 128, 0, s>>>(L); break;
    case OP_SOBEL: k_na_march<VTYPE, OP_SOBEL><<<blocks, 128, 0, s>>>(L); break;
    default: k_na_march<VTYPE, OP_ZH><<<blocks, 128, 0, s>>>(L);
  }
}

}  // namespace vr

using namespace vr;

extern "C" vr_status vr_render_noalloc(const void* voxels, vr_dtype dtype, int nx, int ny, int nz,
                                       float value_max, const float* tf_rgba, int ntf,
                                       const vr_camera* cam, const vr_render_params* params,
                                       float* out_rgba, void* stream) {
  TraceRange trace_("vr_render_noalloc");
  if (!voxels || !tf_rgba || !out_rgba) return VR_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return VR_ERR_INVALID_ARG;
  if (!(value_max > 0.0f) || !(value_max < 3.0e38f)) return VR_ERR_INVALID_ARG;
  if (dtype != VR_U8 && dtype != VR_U16 && dtype != VR_F16 && dtype != VR_F32)
    return VR_ERR_UNSUPPORTED;
  // the kernels read the table and write the image as float4 and read voxels as elements
  const size_t esz = dtype == VR_U8 ? 1 : (dtype == VR_F32 ? 4 : 2);
  if (!aligned_to(voxels, esz) || !aligned_to(tf_rgba, 16) || !aligned_to(out_rgba, 16))
    return VR_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz > 2147483647LL) return VR_ERR_INVALID_ARG;
  const int nb[3] = {(nx + kBrick - 1) / kBrick, (ny + kBrick - 1) / kBrick,
                     (nz + kBrick - 1) / kBrick};
  const long long nbricks = (long long)nb[0] * nb[1] * nb[2];
  if (nbricks > kNoAllocMaxBricks) return VR_ERR_INVALID_ARG;  // volume beyond the scratch
  if (ntf < 2 || ntf > kNoAllocMaxTf) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->collect_stats || params->adaptive) return VR_ERR_UNSUPPORTED;
  CamDev basis;
  st = check_camera(cam, &basis);
  if (st != VR_OK) return st;
  if (!is_device_pointer(voxels) || !is_device_pointer(tf_rgba) || !is_device_pointer(out_rgba))
    return VR_ERR_INVALID_ARG;
  int dev = 0;
  st = cuda_status(cudaGetDevice(&dev));
  if (st != VR_OK) return st;
  unsigned char* scratch = nullptr;
  st = noalloc_scratch(dev, &scratch);
  if (st != VR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  float2* mm = reinterpret_cast<float2*>(scratch + kNaMinMaxOff);
  uint8_t* vis = scratch + kNaVisOff;
  int* prefix = reinterpret_cast<int*>(scratch + kNaPrefixOff);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaCounterOff);

  RawVol R;
  R.data = voxels;
  R.n[0] = nx; R.n[1] = ny; R.n[2] = nz;
  R.sy = nx;
  R.sz = nx * ny;
  const int nbr = (int)nbricks;
  const int mm_blocks = (nbr * 32 + 255) / 256;
  switch (dtype) {
    case VR_U8: k_na_minmax<VT_U8><<<mm_blocks, 256, 0, s>>>(R, nb[0], nb[1], nbr, mm); break;
    case VR_U16: k_na_minmax<VT_U16><<<mm_blocks, 256, 0, s>>>(R, nb[0], nb[1], nbr, mm); break;
    case VR_F16: k_na_minmax<VT_F16><<<mm_blocks, 256, 0, s>>>(R, nb[0], nb[1], nbr, mm); break;
    default: k_na_minmax<VT_F32><<<mm_blocks, 256, 0, s>>>(R, nb[0], nb[1], nbr, mm);
  }
  st = cuda_status(cudaGetLastError());
  if (st != VR_OK) return st;
  const float4* tf = reinterpret_cast<const float4*>(tf_rgba);
  st = cuda_status(launch_tf_prefix(tf, ntf, prefix, s));
  if (st != VR_OK) return st;
  const float scale = (float)(ntf - 1) / value_max;
  st = cuda_status(launch_brick_visibility(mm, nb, prefix, ntf, scale, vis, nullptr, nullptr, nullptr, s));
  if (st != VR_OK) return st;
  st = cuda_status(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  if (st != VR_OK) return st;

  NaLaunch L;
  L.R = R;
  L.V.data = nullptr;
  for (int a = 0; a < 3; ++a) {
    L.V.n[a] = R.n[a];
    L.V.nb[a] = nb[a];
  }
  L.V.px = L.V.py = L.V.pxy = 0;
  L.V.value_max = value_max;
  L.V.vis = vis;
  L.V.mvis = nullptr;
  L.V.nm[0] = L.V.nm[1] = L.V.nm[2] = 0;
  L.tf.tf = tf;
  L.tf.n = ntf;
  L.tf.scale = scale;
  L.cam = basis;
  L.r = render_dev_for(R.n, value_max, params);
  L.out = reinterpret_cast<float4*>(out_rgba);
  L.counter = counter;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 4;
  switch (dtype) {
    case VR_U8: na_launch_op<VT_U8>(L, params->grad, blocks, s); break;
    case VR_U16: na_launch_op<VT_U16>(L, params->grad, blocks, s); break;
    case VR_F16: na_launch_op<VT_F16>(L, params->grad, blocks, s); break;
    default: na_launch_op<VT_F32>(L, params->grad, blocks, s);
  }
  return cuda_status(cudaGetLastError());
}
