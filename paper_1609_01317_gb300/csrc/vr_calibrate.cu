// vr_calibrate.cu -- measured ceilings for the march's roofline (no part of rendering).
//
// The march is neither a dense contraction nor HBM-bound: its ceiling is either the FP32
// pipes or the rate at which the SMs gather and interpolate the eight corner records of a
// sample.  vr_measure_peaks times three microbenchmarks on the device:
//   - FP32 fused multiply-adds on independent chains at full occupancy;
//   - the gather-and-interpolate core of the march (cell, 8 float4 corner records, the
//     trilinear value and gradient blend) with the march's own access pattern: quads of
//     lanes on consecutive samples (step 0.5) of 8 neighbouring rays (4 x 2 pixels,
//     1.09 voxels apart, the pixel footprint of the 1080p CT frame) in a table resident in L2;
//   - the same core at uniformly random cells of a table resident in L1 (16^3 records);
//   - the plain 8-voxel gather of a sample's cell in 16-bit voxels with its trilinear blend
//     (the per-sample footprint of the method itself, before any precomputation), at
//     uniformly random cells of an L1-resident 32^3 volume and in the march's coherent
//     pattern over an L2-resident 256^3 volume.
// Each is the best of `repeats` timed launches (CUDA events, private stream).
#include "vr_march.cuh"

namespace vr {
namespace {

constexpr int kFmaChains = 8;
constexpr int kCoherentN = 128;  // coherent-gather table: 128^3 float4 = 32 MiB
constexpr int kRandomN = 16;     // random-gather table: 16^3 float4 = 64 KiB
constexpr int kGroupsPerTask = 16;
constexpr int kVoxRandomN = 32;    // random u16 gathers: 32^3 voxels = 64 KiB
constexpr int kVoxCoherentN = 256; // coherent u16 gathers: 256^3 voxels = 32 MiB

__global__ void __launch_bounds__(256) k_peak_fma(float* out, int iters, float a, float b) {
  float x[kFmaChains];
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) x[i] = (float)(threadIdx.x & 63) * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int i = 0; i < kFmaChains; ++i) x[i] = fmaf(x[i], a, b);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < kFmaChains; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 32-bit integer mixing (the finaliser of MurmurHash3).
__device__ __forceinline__ unsigned mix32(unsigned h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ float unit(unsigned h) { return (float)(h >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ Cell table_cell(const float p[3], int n) {
  Cell c;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int i = (int)floorf(p[a]);
    i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
    c.ib[a] = i;
    c.f[a] = p[a] - (float)i;
  }
  c.base = 0;
  return c;
}

__device__ __forceinline__ float gather_core(const RecDev& R, const float p[3], int n) {
  const Cell c = table_cell(p, n);
  Corners cr;
  corners_load(R, c, cr);
  const float4 bl = corners_blend(cr, c);
  return bl.w + bl.x + bl.y + bl.z;
}

// Warp task: 8 rays (4 x 2 pixels) x 64 samples, four lanes per ray on consecutive samples.
__global__ void __launch_bounds__(128) k_peak_gather_coherent(const RecDev R, int ntasks,
                                                              float* out) {
  const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  float acc = 0.0f;
  for (int task = warp; task < ntasks; task += nwarps) {
    const unsigned h = mix32((unsigned)task * 0x9e3779b9u + 1u);
    float d[3] = {2.0f * unit(mix32(h ^ 0x68bc21ebu)) - 1.0f, 2.0f * unit(mix32(h ^ 0x02e5be93u)) - 1.0f,
                  2.0f * unit(mix32(h ^ 0x967a889bu)) - 1.0f};
    float dl = rsqrtf(fmaxf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], 1e-6f));
    if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < 1e-6f) d[0] = 1.0f, dl = 1.0f;
    for (int a = 0; a < 3; ++a) d[a] *= dl;
    // tile basis: u = normalize(d x up), v = u x d (up = z, or x when d is nearly along z)
    const float up[3] = {fabsf(d[2]) > 0.9f ? 1.0f : 0.0f, 0.0f, fabsf(d[2]) > 0.9f ? 0.0f : 1.0f};
    float u[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
    const float ul = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) u[a] *= ul;
    const float v[3] = {u[1] * d[2] - u[2] * d[1], u[2] * d[0] - u[0] * d[2], u[0] * d[1] - u[1] * d[0]};
    const float du = ((float)(r & 3) - 1.5f) * 1.09f, dv = ((float)(r >> 2) - 0.5f) * 1.09f;
    float o[3];
    // start inside [40, 88]^3: 32 voxels of travel and the tile stay inside the table
    o[0] = 40.0f + 48.0f * unit(mix32(h ^ 0x1b873593u)) + du * u[0] + dv * v[0];
    o[1] = 40.0f + 48.0f * unit(mix32(h ^ 0xcc9e2d51u)) + du * u[1] + dv * v[1];
    o[2] = 40.0f + 48.0f * unit(mix32(h ^ 0xe6546b64u)) + du * u[2] + dv * v[2];
    for (int j = 0; j < kGroupsPerTask; ++j) {
      const float t = ((float)(4 * j + q) + 0.5f) * 0.5f;
      const float p[3] = {fmaf(t, d[0], o[0]), fmaf(t, d[1], o[1]), fmaf(t, d[2], o[2])};
      acc += gather_core(R, p, kCoherentN);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Same core at uniformly random cells of a 16^3 table (16 samples per lane per task).
__global__ void __launch_bounds__(128) k_peak_gather_random(const RecDev R, int ntasks,
                                                            float* out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  float acc = 0.0f;
  const float span = (float)(kRandomN - 1);
  for (int task = warp; task < ntasks; task += nwarps) {
    unsigned h = mix32((unsigned)task * 0x9e3779b9u + (unsigned)lane * 0x85ebca6bu + 7u);
    for (int j = 0; j < kGroupsPerTask; ++j) {
      h = mix32(h + 0x6b43a9b5u);
      const unsigned h1 = mix32(h ^ 0x1b873593u), h2 = mix32(h ^ 0xcc9e2d51u);
      const float p[3] = {span * unit(h), span * unit(h1), span * unit(h2)};
      acc += gather_core(R, p, kRandomN);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Trilinear value of the cell of p in an n^3 volume of 16-bit voxels (8 voxel loads, lerps
// along x, then y, then z).
__device__ __forceinline__ float gather_u16(const uint16_t* __restrict__ v, const float p[3], int n) {
  const Cell c = table_cell(p, n);
  const int b = c.ib[0] + n * (c.ib[1] + n * c.ib[2]);
  const int sy = n, sz = n * n;
  const float c000 = __ldg(v + b), c100 = __ldg(v + b + 1);
  const float c010 = __ldg(v + b + sy), c110 = __ldg(v + b + sy + 1);
  const float c001 = __ldg(v + b + sz), c101 = __ldg(v + b + sz + 1);
  const float c011 = __ldg(v + b + sy + sz), c111 = __ldg(v + b + sy + sz + 1);
  const float x00 = lerpf(c000, c100, c.f[0]), x10 = lerpf(c010, c110, c.f[0]);
  const float x01 = lerpf(c001, c101, c.f[0]), x11 = lerpf(c011, c111, c.f[0]);
  return lerpf(lerpf(x00, x10, c.f[1]), lerpf(x01, x11, c.f[1]), c.f[2]);
}

// u16 gathers at uniformly random cells (16 samples per lane per task).
__global__ void __launch_bounds__(128) k_peak_gather_u16_random(const uint16_t* v, int ntasks,
                                                                float* out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  float acc = 0.0f;
  const float span = (float)(kVoxRandomN - 1);
  for (int task = warp; task < ntasks; task += nwarps) {
    unsigned h = mix32((unsigned)task * 0x9e3779b9u + (unsigned)lane * 0x85ebca6bu + 11u);
    for (int j = 0; j < kGroupsPerTask; ++j) {
      h = mix32(h + 0x6b43a9b5u);
      const unsigned h1 = mix32(h ^ 0x1b873593u), h2 = mix32(h ^ 0xcc9e2d51u);
      const float p[3] = {span * unit(h), span * unit(h1), span * unit(h2)};
      acc += gather_u16(v, p, kVoxRandomN);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// u16 gathers in the march's pattern: 8 rays of a 4 x 2 tile 1.09 voxels apart, four lanes
// per ray on consecutive samples (step 0.5), random directions and starts.
__global__ void __launch_bounds__(128) k_peak_gather_u16_coherent(const uint16_t* v, int ntasks,
                                                                  float* out) {
  const int lane = threadIdx.x & 31, r = lane >> 2, q = lane & 3;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  float acc = 0.0f;
  for (int task = warp; task < ntasks; task += nwarps) {
    const unsigned h = mix32((unsigned)task * 0x9e3779b9u + 3u);
    float d[3] = {2.0f * unit(mix32(h ^ 0x68bc21ebu)) - 1.0f, 2.0f * unit(mix32(h ^ 0x02e5be93u)) - 1.0f,
                  2.0f * unit(mix32(h ^ 0x967a889bu)) - 1.0f};
    const float n2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (n2 < 1e-6f) d[0] = 1.0f, d[1] = d[2] = 0.0f;
    const float dl = rsqrtf(fmaxf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2], 1e-6f));
    for (int a = 0; a < 3; ++a) d[a] *= dl;
    const float up[3] = {fabsf(d[2]) > 0.9f ? 1.0f : 0.0f, 0.0f, fabsf(d[2]) > 0.9f ? 0.0f : 1.0f};
    float u[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
    const float ul = rsqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) u[a] *= ul;
    const float w[3] = {u[1] * d[2] - u[2] * d[1], u[2] * d[0] - u[0] * d[2], u[0] * d[1] - u[1] * d[0]};
    const float du = ((float)(r & 3) - 1.5f) * 1.09f, dv = ((float)(r >> 2) - 0.5f) * 1.09f;
    float o[3];
    // start inside [64, 192]^3: 32 voxels of travel and the tile stay inside the volume
    for (int a = 0; a < 3; ++a)
      o[a] = 64.0f + 128.0f * unit(mix32(h ^ (0x1b873593u + 0x3c6ef372u * (unsigned)a))) +
             du * u[a] + dv * w[a];
    for (int j = 0; j < kGroupsPerTask; ++j) {
      const float t = ((float)(4 * j + q) + 0.5f) * 0.5f;
      const float p[3] = {fmaf(t, d[0], o[0]), fmaf(t, d[1], o[1]), fmaf(t, d[2], o[2])};
      acc += gather_u16(v, p, kVoxCoherentN);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void k_fill_u16(uint16_t* v, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    v[i] = (uint16_t)((i * 2654435761u) >> 20);
}

__global__ void k_fill_table(float4* t, int n3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    const float v = (float)(i % 4093) * (1.0f / 4093.0f);
    t[i] = make_float4(v - 0.5f, 0.25f - v, v * v, 4095.0f * v);
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace
}  // namespace vr

using namespace vr;

vr_status vr_measure_peaks(int device, int repeats, vr_peaks* out) {
  TraceRange trace_("vr_measure_peaks");
  if (!out || repeats < 1 || repeats > 1000) return VR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? VR_ERR_INVALID_ARG : VR_ERR_CUDA;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return VR_ERR_CUDA;
  int sms = 0, per_fma = 0, per_g1 = 0, per_g2 = 0, per_g3 = 0, per_g4 = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_fma, k_peak_fma, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_g1, k_peak_gather_coherent, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_g2, k_peak_gather_random, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_g3, k_peak_gather_u16_random, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_g4, k_peak_gather_u16_coherent, 128, 0);
  sms = sms > 0 ? sms : 1;
  const int g_fma = sms * (per_fma > 0 ? per_fma : 1);
  const int g1 = sms * (per_g1 > 0 ? per_g1 : 1), g2 = sms * (per_g2 > 0 ? per_g2 : 1);
  const int g3 = sms * (per_g3 > 0 ? per_g3 : 1), g4 = sms * (per_g4 > 0 ? per_g4 : 1);
  const size_t nv_r = (size_t)kVoxRandomN * kVoxRandomN * kVoxRandomN;
  const size_t nv_c = (size_t)kVoxCoherentN * kVoxCoherentN * kVoxCoherentN;
  const size_t nc3 = (size_t)kCoherentN * kCoherentN * kCoherentN, nr3 = (size_t)kRandomN * kRandomN * kRandomN;
  // one float per thread of the largest launch
  size_t nsink = (size_t)g_fma * 256;
  if ((size_t)g1 * 128 > nsink) nsink = (size_t)g1 * 128;
  if ((size_t)g2 * 128 > nsink) nsink = (size_t)g2 * 128;
  if ((size_t)g3 * 128 > nsink) nsink = (size_t)g3 * 128;
  if ((size_t)g4 * 128 > nsink) nsink = (size_t)g4 * 128;
  float4* table = nullptr;
  uint16_t* vox = nullptr;  // [nv_c] coherent volume, then [nv_r] random volume
  float* sink = nullptr;
  cudaStream_t s = nullptr;
  vr_status st = VR_OK;
  if (cudaMalloc(&table, (nc3 + nr3) * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&vox, (nv_c + nv_r) * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&sink, nsink * sizeof(float)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = VR_ERR_OUT_OF_MEMORY;
  }
  double best[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (st == VR_OK) {
    Timer tm;
    k_fill_table<<<sms * 4, 256, 0, s>>>(table, (int)(nc3 + nr3));
    k_fill_u16<<<sms * 4, 256, 0, s>>>(vox, (long)(nv_c + nv_r));
    RecDev Rc;
    Rc.rec = table;
    Rc.n[0] = Rc.n[1] = Rc.n[2] = kCoherentN;
    Rc.sx = 1;
    Rc.sy = kCoherentN;
    Rc.sz = kCoherentN * kCoherentN;
    RecDev Rr;
    Rr.rec = table + nc3;
    Rr.n[0] = Rr.n[1] = Rr.n[2] = kRandomN;
    Rr.sx = 1;
    Rr.sy = kRandomN;
    Rr.sz = kRandomN * kRandomN;
    const int fma_iters = 20000;  // x 4 unrolled x 8 chains
    const int tasks_c = sms * 2048, tasks_r = sms * 2048;
    const double fma_flops = (double)g_fma * 256 * fma_iters * 4 * kFmaChains * 2;
    const double samples_c = (double)tasks_c * 32 * kGroupsPerTask;
    const double samples_r = (double)tasks_r * 32 * kGroupsPerTask;
    for (int rep = 0; rep < repeats + 1 && st == VR_OK; ++rep) {  // launch 0 warms up
      float ms[5] = {0, 0, 0, 0, 0};
      for (int kind = 0; kind < 5; ++kind) {
        cudaEventRecord(tm.a, s);
        if (kind == 0) k_peak_fma<<<g_fma, 256, 0, s>>>(sink, fma_iters, 0.9999999f, 1e-7f);
        else if (kind == 1) k_peak_gather_coherent<<<g1, 128, 0, s>>>(Rc, tasks_c, sink);
        else if (kind == 2) k_peak_gather_random<<<g2, 128, 0, s>>>(Rr, tasks_r, sink);
        else if (kind == 3) k_peak_gather_u16_random<<<g3, 128, 0, s>>>(vox + nv_c, tasks_r, sink);
        else k_peak_gather_u16_coherent<<<g4, 128, 0, s>>>(vox, tasks_c, sink);
        cudaEventRecord(tm.b, s);
        if (cudaEventSynchronize(tm.b) != cudaSuccess) {
          st = VR_ERR_CUDA;
          break;
        }
        cudaEventElapsedTime(&ms[kind], tm.a, tm.b);
      }
      if (st != VR_OK || rep == 0) continue;
      const double rate[5] = {fma_flops / (ms[0] * 1e-3) / 1e12, samples_c / (ms[1] * 1e-3) / 1e9,
                              samples_r / (ms[2] * 1e-3) / 1e9, samples_r / (ms[3] * 1e-3) / 1e9,
                              samples_c / (ms[4] * 1e-3) / 1e9};
      for (int i = 0; i < 5; ++i)
        if (ms[i] > 0.0f && rate[i] > best[i]) best[i] = rate[i];
    }
    if (st == VR_OK && cudaGetLastError() != cudaSuccess) st = VR_ERR_CUDA;
  }
  if (s) cudaStreamDestroy(s);
  if (table) cudaFree(table);
  if (vox) cudaFree(vox);
  if (sink) cudaFree(sink);
  cudaSetDevice(prev);
  if (st != VR_OK) return st;
  out->fma_tflops = best[0];
  out->gather_coherent_gsps = best[1];
  out->gather_random_gsps = best[2];
  out->gather_u16_random_gsps = best[3];
  out->gather_u16_coherent_gsps = best[4];
  return VR_OK;
}
