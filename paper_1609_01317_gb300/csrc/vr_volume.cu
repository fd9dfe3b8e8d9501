// vr_volume.cu -- volume upload kernels: clamp-to-edge padded copy, per-brick min/max
// footprints and per-brick visibility for empty-space skipping (§5.3, §5.4).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "vr_internal.h"
#include "vr_records.cuh"

namespace vr {

// ---------------------------------------------------------------- padded copy
// dst element (x, y, z), x in [0, px), holds src(clamp(x-1), clamp(y-1), clamp(z-1)):
// the clamp-to-edge extension the gradient taps read beyond the volume (§3.6: gradients
// use voxels before the ray start).  One warp per destination row; each lane writes 8
// consecutive elements with one vector store (px is a multiple of 16 elements).
template <typename T, typename V>
__global__ void k_pad(const T* __restrict__ src, int nx, int ny, int nz, T* __restrict__ dst,
                      int px, int py, int pz) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int rows = py * pz;
  if (warp >= rows) return;
  const int y = warp % py, z = warp / py;
  int sy = y - kPadLo, sz = z - kPadLo;
  sy = sy < 0 ? 0 : (sy >= ny ? ny - 1 : sy);
  sz = sz < 0 ? 0 : (sz >= nz ? nz - 1 : sz);
  const T* srow = src + ((size_t)sz * ny + sy) * nx;
  T* drow = dst + (size_t)warp * px;
  constexpr int kPer = 8;
  static_assert(sizeof(V) * (kPer * sizeof(T) / sizeof(V)) == kPer * sizeof(T), "vector");
  for (int x0 = lane * kPer; x0 < px; x0 += 32 * kPer) {
    union {
      T e[kPer];
      V v[kPer * sizeof(T) / sizeof(V)];
    } u;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      int sx = x0 + j - kPadLo;
      sx = sx < 0 ? 0 : (sx >= nx ? nx - 1 : sx);
      u.e[j] = srow[sx];
    }
#pragma unroll
    for (int j = 0; j < (int)(kPer * sizeof(T) / sizeof(V)); ++j)
      reinterpret_cast<V*>(drow + x0)[j] = u.v[j];
  }
}

cudaError_t launch_pad_volume(const void* src, int dtype, const int n[3], void* dst, int px,
                              int py, int pz, cudaStream_t s) {
  const long rows = (long)py * pz;
  const int threads = 256;
  const int blocks = (int)((rows * 32 + threads - 1) / threads);
  switch (dtype) {
    case VT_U8:
      k_pad<uint8_t, uint2><<<blocks, threads, 0, s>>>((const uint8_t*)src, n[0], n[1], n[2],
                                                       (uint8_t*)dst, px, py, pz);
      break;
    case VT_U16:
    case VT_F16:
      k_pad<uint16_t, uint4><<<blocks, threads, 0, s>>>((const uint16_t*)src, n[0], n[1], n[2],
                                                        (uint16_t*)dst, px, py, pz);
      break;
    default:
      k_pad<float, uint4><<<blocks, threads, 0, s>>>((const float*)src, n[0], n[1], n[2],
                                                     (float*)dst, px, py, pz);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------- brick min / max
// Brick (bx, by, bz) covers voxels [8b, 8b+8) per axis.  Its footprint is
// [8b - 1, 8b + 9] (clipped to the volume): every sample whose position lies within one
// voxel of the brick box interpolates only voxels from it.
//
// One block per row of bricks (by, bz); its warps stream the padded rows of the row's
// y / z footprint.  In padded coordinates (padded = voxel + 1) the x footprint of brick bx
// is [8 bx, 8 bx + 10]; every padded element holds the clamp-to-edge value of a voxel
// inside the clipped footprint or an edge voxel the clipped footprint contains, so the
// x range needs no clipping.  Lane l takes the bricks 2l and 2l + 1 of a 64-brick segment:
// one aligned 16-element vector (padded [16l', 16l' + 16), l' the brick pair) plus three
// more elements for the second brick.  Rows in y and z are clipped to the volume.
template <int VTYPE>
__device__ __forceinline__ void load16(const typename VoxelT<VTYPE>::T* p, float e[16]) {
  if constexpr (VTYPE == VT_U8) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) e[j] = (float)((w[j >> 2] >> (8 * (j & 3))) & 0xffu);
  } else if constexpr (VTYPE == VT_U16 || VTYPE == VT_F16) {
    const uint4 a = *reinterpret_cast<const uint4*>(p);
    const uint4 b = *(reinterpret_cast<const uint4*>(p) + 1);
    const unsigned w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const unsigned short h = (unsigned short)((w[j >> 1] >> (16 * (j & 1))) & 0xffffu);
      if constexpr (VTYPE == VT_U16) e[j] = (float)h;
      else e[j] = __half2float(__ushort_as_half(h));
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 a = *(reinterpret_cast<const float4*>(p) + k);
      e[4 * k] = a.x; e[4 * k + 1] = a.y; e[4 * k + 2] = a.z; e[4 * k + 3] = a.w;
    }
  }
}

constexpr int kMinmaxWarps = 8;

template <int VTYPE>
__global__ void __launch_bounds__(32 * kMinmaxWarps) k_brick_minmax(const VolDev V, float2* __restrict__ mm) {
  __shared__ float2 red[kMinmaxWarps][64];
  const int by = blockIdx.x, bz = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nbx = V.nb[0];
  const int ylo = max((by << kBrickShift) - 1, 0), yhi = min((by << kBrickShift) + kBrick + 1, V.n[1] - 1);
  const int zlo = max((bz << kBrickShift) - 1, 0), zhi = min((bz << kBrickShift) + kBrick + 1, V.n[2] - 1);
  const int ey = yhi - ylo + 1, nrows = ey * (zhi - zlo + 1);
  const auto* v = static_cast<const typename VoxelT<VTYPE>::T*>(V.data);
  const float inf = __int_as_float(0x7f800000);
  for (int seg = 0; seg < nbx; seg += 64) {
    const int b0 = seg + 2 * lane;
    const bool has0 = b0 < nbx, has1 = b0 + 1 < nbx;
    float mn0 = inf, mx0 = -inf, mn1 = inf, mx1 = -inf;
    for (int r = warp; r < nrows && has0; r += kMinmaxWarps) {
      const int y = ylo + r % ey, z = zlo + r / ey;
      const auto* row = v + (size_t)V.px * (y + kPadLo) + (size_t)V.pxy * (z + kPadLo);
      float e[16];
      load16<VTYPE>(row + (b0 << kBrickShift), e);
#pragma unroll
      for (int j = 0; j <= 10; ++j) {
        mn0 = fminf(mn0, e[j]);
        mx0 = fmaxf(mx0, e[j]);
      }
      if (has1) {
#pragma unroll
        for (int j = 8; j < 16; ++j) {
          mn1 = fminf(mn1, e[j]);
          mx1 = fmaxf(mx1, e[j]);
        }
#pragma unroll
        for (int j = 16; j <= 18; ++j) {
          const float x = ldv<VTYPE>(row, (b0 << kBrickShift) + j);
          mn1 = fminf(mn1, x);
          mx1 = fmaxf(mx1, x);
        }
      }
    }
    red[warp][2 * lane] = make_float2(mn0, mx0);
    red[warp][2 * lane + 1] = make_float2(mn1, mx1);
    __syncthreads();
    if (threadIdx.x < 64 && seg + (int)threadIdx.x < nbx) {
      float2 m = red[0][threadIdx.x];
#pragma unroll
      for (int w = 1; w < kMinmaxWarps; ++w) {
        const float2 o = red[w][threadIdx.x];
        m.x = fminf(m.x, o.x);
        m.y = fmaxf(m.y, o.y);
      }
      mm[(size_t)(bz * V.nb[1] + by) * nbx + seg + threadIdx.x] = m;
    }
    __syncthreads();
  }
}

cudaError_t launch_brick_minmax(const VolDev& V, int dtype, float2* mm, cudaStream_t s) {
  const dim3 grid(V.nb[1], V.nb[2]);
  const int threads = 32 * kMinmaxWarps;
  switch (dtype) {
    case VT_U8: k_brick_minmax<VT_U8><<<grid, threads, 0, s>>>(V, mm); break;
    case VT_U16: k_brick_minmax<VT_U16><<<grid, threads, 0, s>>>(V, mm); break;
    case VT_F16: k_brick_minmax<VT_F16><<<grid, threads, 0, s>>>(V, mm); break;
    default: k_brick_minmax<VT_F32><<<grid, threads, 0, s>>>(V, mm);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ TF prefix counts
// prefix[i] = number of entries j < i with alpha != 0 (prefix has n + 1 entries).
// One block: each thread counts a contiguous chunk, then a shared-memory scan.
__global__ void k_tf_prefix(const float4* __restrict__ tf, int n, int* __restrict__ prefix) {
  __shared__ int part[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int chunk = (n + nt - 1) / nt;
  const int i0 = t * chunk, i1 = min(i0 + chunk, n);
  int c = 0;
  for (int i = i0; i < i1; ++i) c += (tf[i].w != 0.0f);
  part[t] = c;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const int add = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  int run = part[t] - c;  // exclusive prefix of this chunk
  for (int i = i0; i < i1; ++i) {
    prefix[i] = run;
    run += (tf[i].w != 0.0f);
  }
  if (t == nt - 1) prefix[n] = part[t];
}

cudaError_t launch_tf_prefix(const float4* tf, int n, int* prefix, cudaStream_t s) {
  k_tf_prefix<<<1, 1024, 0, s>>>(tf, n, prefix);
  return cudaGetLastError();
}

// ------------------------------------------------------------ brick visibility
// A brick is invisible when every table entry a sample in it can touch has alpha == 0.
// A macro brick (4 x 4 x 4 bricks) is visible when any of its bricks is: a ray may leave a
// transparent macro brick at its exit in one step (the bricks' footprints, and so their
// union, extend one voxel beyond it).
// The table coordinate is computed with the same FP32 expression as the march
// (u = raw * scale, clamped), widened by one entry below and two above so that a one-ulp
// excursion of an interpolated value cannot reach an unchecked entry.
__global__ void k_brick_visibility(const float2* __restrict__ mm, int nbx, int nby, int nbricks,
                                   const int* __restrict__ prefix, int ntf, float scale,
                                   uint8_t* __restrict__ vis, int* __restrict__ list,
                                   uint8_t* __restrict__ mvis, int nmx, int nmy,
                                   uint8_t* __restrict__ svis, int nsx, int nsy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool visible = false;
  if (i < nbricks) {
    const float2 m = mm[i];
    const float top = (float)(ntf - 1);
    const float ulo = fminf(fmaxf(m.x * scale, 0.0f), top);
    const float uhi = fminf(fmaxf(m.y * scale, 0.0f), top);
    const int jlo = max((int)ulo - 1, 0);
    const int jhi = min((int)uhi + 2, ntf - 1);
    visible = (prefix[jhi + 1] - prefix[jlo]) > 0;
    vis[i] = visible ? 1 : 0;
    if (visible && mvis) {
      // the macro brick holding this brick is visible (every writer stores the same 1)
      const int bx = i % nbx, by = (i / nbx) % nby, bz = i / (nbx * nby);
      mvis[(bx >> kMacroShift) + nmx * ((by >> kMacroShift) + nmy * (bz >> kMacroShift))] = 1;
      if (svis) {
        constexpr int sh = kMacroShift + kSuperShift;
        svis[(bx >> sh) + nsx * ((by >> sh) + nsy * (bz >> sh))] = 1;
      }
    }
  }
  if (list) {
    // one atomic per warp for its visible bricks
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, visible);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(list, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (visible) list[1 + base + __popc(m & ((1u << lane) - 1u))] = i;
  }
}

cudaError_t launch_brick_visibility(const float2* mm, const int nb[3], const int* prefix,
                                    int ntf, float scale, uint8_t* vis, int* list,
                                    uint8_t* mvis, const int nm[3], cudaStream_t s,
                                    uint8_t* svis, const int* ns) {
  const int nbricks = nb[0] * nb[1] * nb[2];
  const int threads = 256;
  if (list) {
    const cudaError_t e = cudaMemsetAsync(list, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  if (!mvis) svis = nullptr;
  if (mvis) {
    // the macro flags, and the super flags that follow them in the same allocation
    const size_t bytes = svis ? (size_t)(svis - mvis) + (size_t)ns[0] * ns[1] * ns[2]
                              : (size_t)nm[0] * nm[1] * nm[2];
    const cudaError_t e = cudaMemsetAsync(mvis, 0, bytes, s);
    if (e != cudaSuccess) return e;
  }
  k_brick_visibility<<<(nbricks + threads - 1) / threads, threads, 0, s>>>(
      mm, nb[0], nb[1], nbricks, prefix, ntf, scale, vis, list, mvis, mvis ? nm[0] : 0,
      mvis ? nm[1] : 0, svis, svis ? ns[0] : 0, svis ? ns[1] : 0);
  return cudaGetLastError();
}

// ------------------------------------------------------ adaptive-sampling multipliers
// §5.2: detail-poor regions are sampled more coarsely.  The regions are the macro bricks
// (4 x 4 x 4 bricks, 32^3 voxels); a macro brick's footprint [32m - 1, 32m + 33] is the union
// of its bricks' footprints, so its value range comes from their min / max.
__global__ void k_macro_multiplier(const float2* __restrict__ mm, int nbx, int nby, int nbz,
                                   int nmx, int nmy, int nmz, float r2, float r4,
                                   uint8_t* __restrict__ mult) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nmx * nmy * nmz) return;
  const int mx = i % nmx, my = (i / nmx) % nmy, mz = i / (nmx * nmy);
  float lo = __int_as_float(0x7f800000), hi = -lo;
  for (int z = mz << kMacroShift; z < min((mz + 1) << kMacroShift, nbz); ++z)
    for (int y = my << kMacroShift; y < min((my + 1) << kMacroShift, nby); ++y)
      for (int x = mx << kMacroShift; x < min((mx + 1) << kMacroShift, nbx); ++x) {
        const float2 m = mm[x + nbx * (y + nby * z)];
        lo = fminf(lo, m.x);
        hi = fmaxf(hi, m.y);
      }
  const float range = hi - lo;
  uint8_t k = 1;
  if (r4 >= 0.0f && range <= r4) k = 4;
  else if (r2 >= 0.0f && range <= r2) k = 2;
  mult[i] = k;
}

cudaError_t launch_macro_multiplier(const float2* mm, const int nb[3], const int nm[3], float r2,
                                    float r4, uint8_t* mult, cudaStream_t s) {
  const int n = nm[0] * nm[1] * nm[2];
  k_macro_multiplier<<<(n + 127) / 128, 128, 0, s>>>(mm, nb[0], nb[1], nb[2], nm[0], nm[1], nm[2],
                                                     r2, r4, mult);
  return cudaGetLastError();
}

}  // namespace vr

namespace vr {

// ------------------------------------------------------ operator gradient records
// rec[v] = (G_x, G_y, G_z, V) at every voxel v a sample can use as a cell corner, where
// G is the integer-grid operator of §3.5 (Eq. 3, Eq. 4, Zucker-Hummel) applied to the
// clamp-to-edge volume: G_a(v) = sum_o W^a_o E(v + o), unscaled, in raw value units.
// Because every tap of a sample shares the sample's fractional weights, the operator
// gradient at any point p equals the trilinear blend of G over p's cell corners, so the
// march reads 8 records per sample instead of evaluating the taps.
//
// A brick needs the records of voxels [8b, 8b+8]^3 (its cells' corners); with skipping
// on, only visible bricks are visited.  Each voxel is written by the brick whose core
// [8b, 8b+8)^3 holds it when that brick is computed, else by the computed brick whose
// upper face it lies on (several such bricks write the same value).  Per brick the 11^3
// clamp-to-edge neighbourhood [8b-1, 8b+9]^3 is staged in shared memory, then the (x, y)
// columns of records are streamed along z (see k_records).
// Padded row (y0 - 1 + j, z0 - 1 + k) of brick (x0, y0, z0) from padded x = x0, i.e. voxels
// x0 - 1 .. x0 + 14, as one aligned 16-element vector of raw words (row pitches are
// multiples of 16 elements and x0 of 8; the vector ends inside the row); rows beyond n are
// clamped to n (inside the padded border, where E is the edge value).
template <int VTYPE>
struct RawRow {
  static constexpr int kWords = 16 * (int)sizeof(typename VoxelT<VTYPE>::T) / 4;
  uint32_t w[kWords];
};

template <int VTYPE>
__device__ __forceinline__ void load_raw_row(RawRow<VTYPE>& r, const VolDev& V, int x0, int y0,
                                             int z0, int j, int k) {
  using T = typename VoxelT<VTYPE>::T;
  const int Y = min(y0 - 1 + j, V.n[1]), Z = min(z0 - 1 + k, V.n[2]);
  const T* row = static_cast<const T*>(V.data) +
                 VR_CHECK(V.bounds, (size_t)V.px * (Y + kPadLo) + (size_t)V.pxy * (Z + kPadLo) + x0,
                          0, padded_elems(V) - 16);
  if constexpr (sizeof(T) == 1) {
    const uint2 a0 = __ldg(reinterpret_cast<const uint2*>(row));
    const uint2 a1 = __ldg(reinterpret_cast<const uint2*>(row) + 1);
    r.w[0] = a0.x; r.w[1] = a0.y; r.w[2] = a1.x; r.w[3] = a1.y;
  } else {
#pragma unroll
    for (int q = 0; q < RawRow<VTYPE>::kWords / 4; ++q) {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(row) + q);
      r.w[4 * q] = a.x; r.w[4 * q + 1] = a.y; r.w[4 * q + 2] = a.z; r.w[4 * q + 3] = a.w;
    }
  }
}

// Voxels x0 - 1 .. x0 + 10 of a raw row into tile[k][j][0..11].
template <int VTYPE>
__device__ __forceinline__ void store_row(float (*tile)[11][12], const RawRow<VTYPE>& r, int j,
                                          int k) {
  float e[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    if constexpr (VTYPE == VT_U8) {
      e[i] = (float)((r.w[i >> 2] >> (8 * (i & 3))) & 0xffu);
    } else if constexpr (VTYPE == VT_U16 || VTYPE == VT_F16) {
      const unsigned short h = (unsigned short)((r.w[i >> 1] >> (16 * (i & 1))) & 0xffffu);
      if constexpr (VTYPE == VT_F16) e[i] = __half2float(__ushort_as_half(h));
      else e[i] = (float)h;
    } else {
      e[i] = __uint_as_float(r.w[i]);
    }
  }
  float4* dst = reinterpret_cast<float4*>(&tile[k][j][0]);
  dst[0] = make_float4(e[0], e[1], e[2], e[3]);
  dst[1] = make_float4(e[4], e[5], e[6], e[7]);
  dst[2] = make_float4(e[8], e[9], e[10], e[11]);
}

// Persistent blocks of 64 threads take bricks in grid stride (from `list` when given).  Work
// items: 32 threads for the 8 x 8 core columns as pairs (x offsets 2p, 2p + 1), 4 for the
// pairs of the upper y face (row 8) and 9 for the upper x face column (x offset 8, rows
// 0..8); each streams its column(s) along z with rolling plane sums.
template <int VTYPE, int OP>
__global__ void __launch_bounds__(64) k_records(const VolDev V, const uint8_t* __restrict__ need,
                                                const int* __restrict__ list,
                                                float4* __restrict__ rec) {
  __shared__ __align__(16) float tile[11][11][12];  // [z][y][x], x padded to 12
  const int t = threadIdx.x;
  const int nbx = V.nb[0], nby = V.nb[1];
  const int nbricks = nbx * nby * V.nb[2];
  const int nx = V.n[0], ny = V.n[1], nz = V.n[2];
  int u = 0, w = 0, ncol = 0;  // first column, row, columns of this thread (0: idle)
  if (t < 32) {
    u = 2 * (t & 3);
    w = t >> 2;
    ncol = 2;
  } else if (t < 36) {
    u = 2 * (t - 32);
    w = kBrick;
    ncol = 2;
  } else if (t < 45) {
    u = kBrick;
    w = t - 36;
    ncol = 1;
  }
  const int nwork = list ? list[0] : nbricks;
  const size_t zstride = (size_t)nx * ny;
  // rows t and t + 64 of the 121 rows of a brick's neighbourhood; the next brick's rows are
  // loaded into registers while the current brick is computed
  const int j0 = t % 11, k0 = t / 11, j1 = (t + 64) % 11, k1 = (t + 64) / 11;
  const bool has1 = t + 64 < 121;
  RawRow<VTYPE> ra, rb;
  auto load_rows = [&](int item) {
    const int b = list ? list[1 + item] : item;
    const int x0 = (b % nbx) << kBrickShift, y0 = ((b / nbx) % nby) << kBrickShift,
              z0 = (b / (nbx * nby)) << kBrickShift;
    load_raw_row<VTYPE>(ra, V, x0, y0, z0, j0, k0);
    if (has1) load_raw_row<VTYPE>(rb, V, x0, y0, z0, j1, k1);
  };
  if ((int)blockIdx.x < nwork) load_rows(blockIdx.x);
  for (int item = blockIdx.x; item < nwork; item += gridDim.x) {
    const int bid = list ? list[1 + item] : item;
    const int bx = bid % nbx, by = (bid / nbx) % nby, bz = bid / (nbx * nby);
    const int x0 = bx << kBrickShift, y0 = by << kBrickShift, z0 = bz << kBrickShift;
    store_row<VTYPE>(tile, ra, j0, k0);
    if (has1) store_row<VTYPE>(tile, rb, j1, k1);
    __syncthreads();
    if (item + (int)gridDim.x < nwork) load_rows(item + gridDim.x);
    const int x = x0 + u, y = y0 + w;
    if (ncol && x < nx && y < ny) {
      // which of this item's records to write: the core always; a face voxel when the brick
      // that owns it is not computed
      const int ox = u == kBrick, oy = w == kBrick;
      bool wr_lo = true, wr_top = false;
      if (need) {
        if (ox | oy) wr_lo = !need[(bx + ox) + nbx * ((by + oy) + nby * bz)];
        if (z0 + kBrick < nz) wr_top = !need[(bx + ox) + nbx * ((by + oy) + nby * (bz + 1))];
      } else {
        wr_lo = !(ox | oy);
      }
      const int qn = min(kBrick + 1, nz - z0);
      const size_t obase = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z0);
      const long long olast = (long long)nx * ny * nz - 1;
      float4* out = rec + obase;
      if (wr_lo || (wr_top && qn > kBrick)) {
        if (ncol == 2) {
          const bool two = x + 1 < nx;
          PlaneSums A[3], B[3];
          plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[0], u, w, A[0], B[0]);
          plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[1], u, w, A[1], B[1]);
#pragma unroll
          for (int q = 0; q <= kBrick; ++q) {
            if (q < qn) {
              plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[q + 2], u, w, A[(q + 2) % 3], B[(q + 2) % 3]);
              if (q < kBrick ? wr_lo : wr_top) {
                out[VR_CHECK(V.bounds, q * zstride, -(long long)obase, olast - (long long)obase)] =
                    record_of<OP>(A[q % 3], A[(q + 1) % 3], A[(q + 2) % 3]);
                if (two)
                  out[VR_CHECK(V.bounds, q * zstride + 1, -(long long)obase, olast - (long long)obase)] =
                      record_of<OP>(B[q % 3], B[(q + 1) % 3], B[(q + 2) % 3]);
              }
            }
          }
        } else {
          PlaneSums ps[3];
          ps[0] = plane_sums<OP>(tile[0], u, w);
          ps[1] = plane_sums<OP>(tile[1], u, w);
#pragma unroll
          for (int q = 0; q <= kBrick; ++q) {
            if (q < qn) {
              ps[(q + 2) % 3] = plane_sums<OP>(tile[q + 2], u, w);
              if (q < kBrick ? wr_lo : wr_top)
                out[VR_CHECK(V.bounds, q * zstride, -(long long)obase, olast - (long long)obase)] =
                    record_of<OP>(ps[q % 3], ps[(q + 1) % 3], ps[(q + 2) % 3]);
            }
          }
        }
      }
    }
    __syncthreads();  // the tile is restaged for the next brick
  }
}

// ------------------------------------------------ records with TMA-staged neighbourhoods
// The same records, with each brick's clamp-to-edge neighbourhood brought into shared memory
// by the tensor memory accelerator: a 3-D tiled copy (cp.async.bulk.tensor) of the padded
// volume's box [x0, x0 + BX) x [8by, 8by + 11) x [8bz, 8bz + 11) (padded coordinates; the
// padded index of voxel 8b - 1 is 8b, so x0 = 8bx keeps the copy's start on a 16-byte
// boundary for 2- and 4-byte voxels, and x0 = 16 (bx / 2) for 1-byte voxels, which then
// copy 32 columns) completes on an mbarrier.  Two raw stages are in flight: the copy of the
// brick after next is issued as soon as a stage has been converted into the float tile, so
// the march of loads overlaps the computation.  Rows beyond the padded array read as zero;
// they only feed records of voxels outside the volume, which are not written.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier for at most about a second of SM clock.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > 2000000000ll) return false;
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

template <int VTYPE>
struct TmaBox {
  using T = typename VoxelT<VTYPE>::T;
  static constexpr int BX = sizeof(T) == 1 ? 32 : 16;  // columns per copied row
  static constexpr int BYTES = 11 * 11 * BX * (int)sizeof(T);
  static constexpr int STAGE = (BYTES + 127) / 128 * 128;
};

template <int VTYPE, int OP>
__global__ void __launch_bounds__(64) k_records_tma(const VolDev V, const uint8_t* __restrict__ need,
                                                    const int* __restrict__ list,
                                                    float4* __restrict__ rec,
                                                    const __grid_constant__ CUtensorMap tmap,
                                                    unsigned* __restrict__ err) {
  using T = typename VoxelT<VTYPE>::T;
  using B = TmaBox<VTYPE>;
  __shared__ __align__(128) unsigned char raw[2][B::STAGE];
  __shared__ __align__(16) float tile[11][11][12];  // [z][y][x], x padded to 12
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_all;
  const int t = threadIdx.x;
  const int nbx = V.nb[0], nby = V.nb[1];
  const int nbricks = nbx * nby * V.nb[2];
  const int nx = V.n[0], ny = V.n[1], nz = V.n[2];
  int u = 0, w = 0, ncol = 0;  // first column, row, columns of this thread (0: idle)
  if (t < 32) {
    u = 2 * (t & 3);
    w = t >> 2;
    ncol = 2;
  } else if (t < 36) {
    u = 2 * (t - 32);
    w = kBrick;
    ncol = 2;
  } else if (t < 45) {
    u = kBrick;
    w = t - 36;
    ncol = 1;
  }
  const int nwork = list ? list[0] : nbricks;
  const size_t zstride = (size_t)nx * ny;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_all = 0;
  }
  __syncthreads();
  auto issue = [&](int item, int s) {  // thread 0: the copy of item's neighbourhood
    const int b = list ? list[1 + item] : item;
    const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    const int x0 = sizeof(T) == 1 ? 16 * (bx >> 1) : 8 * bx;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], B::BYTES);
    tma_load_3d(raw[s], &tmap, &bar[s], x0, 8 * by, 8 * bz);
  };
  const int first = blockIdx.x;
  if (t == 0) {
    if (first < nwork) issue(first, 0);
    if (first + (int)gridDim.x < nwork) issue(first + gridDim.x, 1);
  }
  int it = 0;
  for (int item = first; item < nwork; item += gridDim.x, ++it) {
    const int s = it & 1;
    if (t == 0 && !mbar_wait_bounded(&bar[s], (unsigned)(it >> 1) & 1u)) {
      abort_all = 1;
      atomicOr(err, 1u);
      // the other stage's copy may be in flight: wait for it (bounded) before leaving
      if (item + (int)gridDim.x < nwork) mbar_wait_bounded(&bar[s ^ 1], (unsigned)((it + 1) >> 1) & 1u);
    }
    __syncthreads();
    if (abort_all) return;
    const int bid = list ? list[1 + item] : item;
    const int bx = bid % nbx, by = (bid / nbx) % nby, bz = bid / (nbx * nby);
    const int x0 = bx << kBrickShift, y0 = by << kBrickShift, z0 = bz << kBrickShift;
    // raw stage -> float tile: rows t and t + 64 of the 121, columns x0 - 1 .. x0 + 10
    {
      const T* src = reinterpret_cast<const T*>(raw[s]);
      const int xoff = sizeof(T) == 1 ? 8 * (bx & 1) : 0;
      for (int r = t; r < 121; r += 64) {
        const T* row = src + r * B::BX + xoff;
        float e[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) e[i] = to_float<VTYPE>(row[i]);
        float4* dst = reinterpret_cast<float4*>(&tile[r / 11][r % 11][0]);
        dst[0] = make_float4(e[0], e[1], e[2], e[3]);
        dst[1] = make_float4(e[4], e[5], e[6], e[7]);
        dst[2] = make_float4(e[8], e[9], e[10], e[11]);
      }
    }
    __syncthreads();
    if (t == 0 && item + 2 * (int)gridDim.x < nwork) issue(item + 2 * gridDim.x, s);
    const int x = x0 + u, y = y0 + w;
    if (ncol && x < nx && y < ny) {
      const int ox = u == kBrick, oy = w == kBrick;
      bool wr_lo = true, wr_top = false;
      if (need) {
        if (ox | oy) wr_lo = !need[(bx + ox) + nbx * ((by + oy) + nby * bz)];
        if (z0 + kBrick < nz) wr_top = !need[(bx + ox) + nbx * ((by + oy) + nby * (bz + 1))];
      } else {
        wr_lo = !(ox | oy);
      }
      const int qn = min(kBrick + 1, nz - z0);
      const size_t obase = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z0);
      const long long olast = (long long)nx * ny * nz - 1;
      float4* out = rec + obase;
      if (wr_lo || (wr_top && qn > kBrick)) {
        if (ncol == 2) {
          const bool two = x + 1 < nx;
          PlaneSums A[3], Bs[3];
          plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[0], u, w, A[0], Bs[0]);
          plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[1], u, w, A[1], Bs[1]);
#pragma unroll
          for (int q = 0; q <= kBrick; ++q) {
            if (q < qn) {
              plane_sums2<OP, VTYPE == VT_U8 || VTYPE == VT_U16>(tile[q + 2], u, w, A[(q + 2) % 3], Bs[(q + 2) % 3]);
              if (q < kBrick ? wr_lo : wr_top) {
                out[VR_CHECK(V.bounds, q * zstride, -(long long)obase, olast - (long long)obase)] =
                    record_of<OP>(A[q % 3], A[(q + 1) % 3], A[(q + 2) % 3]);
                if (two)
                  out[VR_CHECK(V.bounds, q * zstride + 1, -(long long)obase, olast - (long long)obase)] =
                      record_of<OP>(Bs[q % 3], Bs[(q + 1) % 3], Bs[(q + 2) % 3]);
              }
            }
          }
        } else {
          PlaneSums ps[3];
          ps[0] = plane_sums<OP>(tile[0], u, w);
          ps[1] = plane_sums<OP>(tile[1], u, w);
#pragma unroll
          for (int q = 0; q <= kBrick; ++q) {
            if (q < qn) {
              ps[(q + 2) % 3] = plane_sums<OP>(tile[q + 2], u, w);
              if (q < kBrick ? wr_lo : wr_top)
                out[VR_CHECK(V.bounds, q * zstride, -(long long)obase, olast - (long long)obase)] =
                    record_of<OP>(ps[q % 3], ps[(q + 1) % 3], ps[(q + 2) % 3]);
            }
          }
        }
      }
    }
    __syncthreads();  // the tile is rewritten for the next brick
  }
}

// cuTensorMapEncodeTiled from the driver the runtime uses (null when unavailable).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// The tensor map of the padded volume for the records' neighbourhood copies.
template <int VTYPE>
static bool records_tensor_map(const VolDev& V, CUtensorMap* map) {
  using T = typename VoxelT<VTYPE>::T;
  const auto encode = tensor_map_encoder();
  if (!encode) return false;
  const CUtensorMapDataType dt = sizeof(T) == 1   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t dims[3] = {(cuuint64_t)V.px, (cuuint64_t)V.py,
                              (cuuint64_t)(V.n[2] + kPadLo + kPadHi)};
  const cuuint64_t strides[2] = {(cuuint64_t)V.px * sizeof(T), (cuuint64_t)V.pxy * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)TmaBox<VTYPE>::BX, 11, 11};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, dt, 3, const_cast<void*>(V.data), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int VTYPE, int OP>
static void launch_records_k(const VolDev& V, const uint8_t* need, const int* list, float4* rec,
                             unsigned* err, cudaStream_t s) {
  // persistent grid: the current device's SMs x resident blocks
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nbricks = V.nb[0] * V.nb[1] * V.nb[2];
  CUtensorMap map;
  if (err && records_tensor_map<VTYPE>(V, &map)) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_records_tma<VTYPE, OP>, 64, 0);
    const int grid = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
    k_records_tma<VTYPE, OP><<<min(grid, nbricks), 64, 0, s>>>(V, need, list, rec, map, err);
    return;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_records<VTYPE, OP>, 64, 0);
  const int grid = (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
  k_records<VTYPE, OP><<<min(grid, nbricks), 64, 0, s>>>(V, need, list, rec);
}

template <int VTYPE>
static void launch_records_op(const VolDev& V, int op, const uint8_t* need, const int* list,
                              float4* rec, unsigned* err, cudaStream_t s) {
  switch (op) {
    case OP_CENTRAL: launch_records_k<VTYPE, OP_CENTRAL>(V, need, list, rec, err, s); break;
    case OP_SOBEL: launch_records_k<VTYPE, OP_SOBEL>(V, need, list, rec, err, s); break;
    default: launch_records_k<VTYPE, OP_ZH>(V, need, list, rec, err, s);
  }
}

cudaError_t launch_records(const VolDev& V, int dtype, int op, const uint8_t* need,
                           const int* list, float4* rec, cudaStream_t s, unsigned* err) {
  switch (dtype) {
    case VT_U8: launch_records_op<VT_U8>(V, op, need, list, rec, err, s); break;
    case VT_U16: launch_records_op<VT_U16>(V, op, need, list, rec, err, s); break;
    case VT_F16: launch_records_op<VT_F16>(V, op, need, list, rec, err, s); break;
    default: launch_records_op<VT_F32>(V, op, need, list, rec, err, s);
  }
  return cudaGetLastError();
}

}  // namespace vr
