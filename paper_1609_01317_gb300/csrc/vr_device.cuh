// vr_device.cuh -- device-side building blocks of the ray march (sm_103a).
//
// Every function here is one step of the method in "Volume Raycasting mit OpenCL"
// (Kopal 2011), §3.10: ray setup against the bounding box (§3.3, §3.6), trilinear
// sampling (§3.4, Eq. 2), transfer-function lookup (§3.7), gradient operators (§3.5,
// Eq. 3, Eq. 4), point-light Phong shading (§3.8, Listing 3) and front-to-back
// compositing (§3.9, Eq. 6).
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace vr {

constexpr int kBrick = 8;       // brick edge in voxels (empty-space skipping, §5.3)
constexpr int kBrickShift = 3;
constexpr int kMacroShift = 2;  // a macro brick is 4 x 4 x 4 bricks (32^3 voxels)
constexpr int kSuperShift = 2;  // a super brick is 4 x 4 x 4 macro bricks (128^3 voxels)
constexpr int kCkptStride = 32; // samples per adjoint checkpoint segment
constexpr int kPadLo = 1;       // clamp-to-edge border below each axis
constexpr int kPadHi = 2;       // ... and above (covers the 4^3 stencil of the last cell)

enum Op { OP_CENTRAL = 0, OP_SOBEL = 1, OP_ZH = 2 };
enum VType { VT_U8 = 0, VT_U16 = 1, VT_F16 = 2, VT_F32 = 3 };

// Camera basis, computed on the host in FP32 with separately rounded operations.
struct CamDev {
  float eye[3], fwd[3], right[3], upv[3];
  float ax, ay;
  int ortho, width, height;
};

// Padded volume: element (x, y, z), x,y,z in [-1, n+1], at
// (x + 1) + px * ((y + 1) + py * (z + 1)).
struct VolDev {
  const void* data;
  int n[3];
  int px, pxy;       // x pitch and slice pitch of the padded array, in elements
  int py;            // padded rows per slice
  float value_max;   // raw -> [0,1]
  int nb[3];         // bricks per axis
  const uint8_t* vis;  // per-brick visibility (1 = some sample may be non-transparent)
  const uint8_t* mvis;  // per-macro-brick visibility (OR over its bricks), or null
  int nm[3];            // macro bricks per axis
  const uint8_t* svis = nullptr;  // per-super-brick visibility (OR over its macro bricks), or
  int ns[3] = {0, 0, 0};          // null; super bricks per axis
  unsigned long long* bounds = nullptr;  // out-of-range index counter (bounds-checked builds)
};

// Gradient records over the unpadded grid: rec[x + nx*(y + ny*z)] = (G_x, G_y, G_z, V).
// sx, sy, sz: element strides to the +1 neighbour (0 along an axis of size 1, where the
// clamp-to-edge neighbour is the voxel itself).
struct RecDev {
  const float4* rec;
  int n[3];
  int sx, sy, sz;
  unsigned long long* bounds = nullptr;  // out-of-range index counter (bounds-checked builds)
};

struct TfDev {
  const float4* tf;
  int n;
  float scale;  // (n - 1) / value_max: raw value -> table coordinate
  unsigned long long* bounds = nullptr;  // out-of-range index counter (bounds-checked builds)
};

// ------------------------------------------------------------ bounds checks
// A build with -DVR_DEBUG_BOUNDS tests the gather and scatter indices of the kernels against
// their buffers before use: an index outside [lo, hi] is counted in *counter (the context's
// statistics slot 7, read by vr_read_bounds_violations) and clamped into the range, so the
// access itself stays in bounds.  Regular builds compile the checks away.
#ifdef VR_DEBUG_BOUNDS
__device__ __forceinline__ long long vr_check(unsigned long long* counter, long long i,
                                              long long lo, long long hi) {
  if (i >= lo && i <= hi) return i;
  if (counter) atomicAdd(counter, 1ull);
  return i < lo ? lo : hi;
}
#define VR_CHECK(counter, i, lo, hi) \
  vr_check((counter), (long long)(i), (long long)(lo), (long long)(hi))
#else
#define VR_CHECK(counter, i, lo, hi) (i)
#endif

// Elements of the padded volume.
__device__ __forceinline__ long long padded_elems(const VolDev& V) {
  return (long long)V.pxy * (V.n[2] + kPadLo + kPadHi);
}

// Largest record index offset of a cell's corners (+x, +y and +z neighbours).
__device__ __forceinline__ long long corner_span(const RecDev& R) { return R.sx + R.sy + R.sz; }

struct ShadeDev {
  float ka, kd, ks, shininess;
  float light[3];
  int headlight;
};

struct RenderDev {
  float step;
  float ert;          // stop once 1 - T >= ert
  int skip;           // empty-space skipping on/off
  float lo[3], hi[3]; // sampling box: clip box intersected with [0, n-1]^3
  float gscale;       // gradient operator scale / value_max
  ShadeDev sh;
  const uint8_t* mult;  // per-macro-brick sampling multiplier (adaptive sampling, §5.2), or null
};

// ----------------------------------------------------------------------- voxel fetch
template <int VTYPE> struct VoxelT;
template <> struct VoxelT<VT_U8> { using T = uint8_t; };
template <> struct VoxelT<VT_U16> { using T = uint16_t; };
template <> struct VoxelT<VT_F16> { using T = __half; };
template <> struct VoxelT<VT_F32> { using T = float; };

template <int VTYPE>
__device__ __forceinline__ float to_float(typename VoxelT<VTYPE>::T x) {
  if constexpr (VTYPE == VT_F16) {
    return __half2float(x);
  } else {
    return static_cast<float>(x);
  }
}

template <int VTYPE>
__device__ __forceinline__ float ldv(const typename VoxelT<VTYPE>::T* __restrict__ v, int off) {
  if constexpr (VTYPE == VT_F16) {
    return __half2float(__ldg(v + off));
  } else {
    return static_cast<float>(__ldg(v + off));
  }
}

// --------------------------------------------------------------- ray setup (§3.3)
// FP32 with every operation rounded on its own (no contraction), so that the integer
// sample count K is the same on every IEEE-754 implementation of this convention.
__device__ __forceinline__ float dot_rn(const float a[3], const float b[3]) {
  float r = __fmul_rn(a[0], b[0]);
  r = __fadd_rn(r, __fmul_rn(a[1], b[1]));
  return __fadd_rn(r, __fmul_rn(a[2], b[2]));
}

// Returns true on a hit; K receives the sample count (midpoint rule), tn the entry.
__device__ __forceinline__ bool ray_setup(const CamDev& c, const float lo[3], const float hi[3],
                                          float step, int px, int py, float o[3], float d[3],
                                          float& tn, int& K) {
  const float sx = __fsub_rn(__fdiv_rn((float)(2 * px + 1), (float)c.width), 1.0f);
  const float sy = __fsub_rn(1.0f, __fdiv_rn((float)(2 * py + 1), (float)c.height));
  const float u = __fmul_rn(sx, c.ax), v = __fmul_rn(sy, c.ay);
  if (c.ortho) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      o[a] = __fadd_rn(__fadd_rn(c.eye[a], __fmul_rn(u, c.right[a])), __fmul_rn(v, c.upv[a]));
      d[a] = c.fwd[a];
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      d[a] = __fadd_rn(__fadd_rn(c.fwd[a], __fmul_rn(u, c.right[a])), __fmul_rn(v, c.upv[a]));
      o[a] = c.eye[a];
    }
    const float l = __fsqrt_rn(dot_rn(d, d));
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = __fdiv_rn(d[a], l);
  }
  float t0 = 0.0f, t1 = __int_as_float(0x7f800000);  // entry clamped to t >= 0
  tn = 0.0f;
  K = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (lo[a] > hi[a]) return false;
    if (d[a] == 0.0f) {
      if (o[a] < lo[a] || o[a] > hi[a]) return false;
    } else {
      const float ta = __fdiv_rn(__fsub_rn(lo[a], o[a]), d[a]);
      const float tb = __fdiv_rn(__fsub_rn(hi[a], o[a]), d[a]);
      const float tmin = ta < tb ? ta : tb, tmax = ta < tb ? tb : ta;
      if (tmin > t0) t0 = tmin;
      if (tmax < t1) t1 = tmax;
    }
  }
  tn = t0;
  if (!(t1 >= t0)) return false;
  const float kf = floorf(__fadd_rn(__fdiv_rn(__fsub_rn(t1, t0), step), 0.5f));
  K = kf > 0.0f ? (int)kf : 0;
  return true;
}

// ------------------------------------------------------------------ cell (§3.4)
struct Cell {
  int base;          // padded offset of voxel (ix, iy, iz)
  float f[3];        // fractional position inside the cell
  int ib[3];         // integer cell coordinates
};

__device__ __forceinline__ Cell cell_of(const VolDev& V, const float p[3]) {
  Cell c;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int i = (int)floorf(p[a]);
    const int top = V.n[a] > 1 ? V.n[a] - 2 : 0;
    i = i < 0 ? 0 : (i > top ? top : i);
    c.ib[a] = i;
    c.f[a] = p[a] - (float)i;
  }
  c.base = (c.ib[0] + kPadLo) + V.px * (c.ib[1] + kPadLo) + V.pxy * (c.ib[2] + kPadLo);
  return c;
}

// lerp written as a + f (b - a): for integer voxels b - a is exact, so the result
// stays inside [min(a,b), max(a,b)] (the empty-space test relies on this).
__device__ __forceinline__ float lerpf(float a, float b, float f) { return fmaf(f, b - a, a); }

// Trilinear interpolation in raw units: lerps along x, then y, then z.
template <int VTYPE>
__device__ __forceinline__ float trilinear(const VolDev& V, const Cell& c) {
  const auto* v = static_cast<const typename VoxelT<VTYPE>::T*>(V.data);
  const int px = V.px, pxy = V.pxy;
  const int b = (int)VR_CHECK(V.bounds, c.base, 0, padded_elems(V) - 1 - (pxy + px + 1));
  const float c000 = ldv<VTYPE>(v, b), c100 = ldv<VTYPE>(v, b + 1);
  const float c010 = ldv<VTYPE>(v, b + px), c110 = ldv<VTYPE>(v, b + px + 1);
  const float c001 = ldv<VTYPE>(v, b + pxy), c101 = ldv<VTYPE>(v, b + pxy + 1);
  const float c011 = ldv<VTYPE>(v, b + pxy + px), c111 = ldv<VTYPE>(v, b + pxy + px + 1);
  const float x00 = lerpf(c000, c100, c.f[0]), x10 = lerpf(c010, c110, c.f[0]);
  const float x01 = lerpf(c001, c101, c.f[0]), x11 = lerpf(c011, c111, c.f[0]);
  const float y0 = lerpf(x00, x10, c.f[1]), y1 = lerpf(x01, x11, c.f[1]);
  return lerpf(y0, y1, c.f[2]);
}

// ------------------------------------------------------------ transfer function
struct TfSample {
  float4 rgba;
  int i;     // lower entry
  float w;   // weight of entry i + 1
  bool inside;  // u was not clamped (slope is defined)
};

// §3.7 lookup table read with linear interpolation between entries.  `table` is tf.tf or a
// copy of it in shared memory (SHARED: plain loads, which the compiler issues as shared
// loads when the pointer comes from a __shared__ array).
template <bool SHARED = false>
__device__ __forceinline__ TfSample tf_lookup(const TfDev& tf, float s_raw,
                                              const float4* table = nullptr) {
  TfSample r;
  float u = s_raw * tf.scale;
  const float top = (float)(tf.n - 1);
  r.inside = (u >= 0.0f) && (u <= top);
  u = fminf(fmaxf(u, 0.0f), top);
  int i = (int)u;
  if (i > tf.n - 2) i = tf.n - 2;
  i = (int)VR_CHECK(tf.bounds, i, 0, tf.n - 2);
  r.i = i;
  r.w = u - (float)i;
  float4 a, b;
  if constexpr (SHARED) {
    a = table[i];
    b = table[i + 1];
  } else {
    a = __ldg(tf.tf + i);
    b = __ldg(tf.tf + i + 1);
  }
  r.rgba.x = lerpf(a.x, b.x, r.w);
  r.rgba.y = lerpf(a.y, b.y, r.w);
  r.rgba.z = lerpf(a.z, b.z, r.w);
  r.rgba.w = lerpf(a.w, b.w, r.w);
  return r;
}

// ------------------------------------------------------------- gradient (§3.5)
// The operators are linear and all taps of a sample share its fractional weights, so
// the gradient at p equals the trilinear blend of the integer-grid operator evaluated at
// the eight corners of p's cell.  With clamp-to-edge addressing that blend needs the
// 4x4x4 voxel neighbourhood N[a][b][c] = E(i0 + (a-1, b-1, c-1)); it is contracted one
// axis at a time with three 4-tap kernels per axis:
//   T = [0, 1-f, f, 0]         (plain interpolation)
//   U = [1-f, f, 1-f, f]       (the +-1 cross taps blended over the two corners)
//   D = [-(1-f), -f, 1-f, f]   (the +-1 difference along the component's own axis)
// An operator with plane weights W[b][c] = w0 d(b)d(c) + w1 (d(b)o(c) + o(b)d(c)) +
// w2 o(b)o(c) (d = centre tap, o = the two outer taps) then gives, e.g. for x,
//   g_x = D_x . (w0 T_yT_z + w1 (T_yU_z + U_yT_z) + w2 U_yU_z) . N.
// Sobel3D (Eq. 4): w = (6, 3, 1).  Zucker-Hummel: w = (1, 1/sqrt2, 1/sqrt3).
__device__ __forceinline__ float kT(float x0, float x1, float x2, float x3, float f) {
  (void)x0; (void)x3;
  return fmaf(f, x2 - x1, x1);
}
__device__ __forceinline__ float kU(float x0, float x1, float x2, float x3, float f) {
  const float a = x0 + x2, b = x1 + x3;
  return fmaf(f, b - a, a);
}
__device__ __forceinline__ float kD(float x0, float x1, float x2, float x3, float f) {
  const float p = x2 - x0, q = x3 - x1;
  return fmaf(f, q - p, p);
}

// Value (raw units) and unscaled operator gradient from the 4^3 neighbourhood, read
// through nb(a, b, c) = N[a][b][c] = E(i0 + (a-1, b-1, c-1)).
template <int OP, typename Hood>
__device__ __forceinline__ void contract_neighbourhood(const Hood& nb, const float f[3], float& s,
                                                       float g[3]) {
  const float fx = f[0], fy = f[1], fz = f[2];
  if constexpr (OP == OP_CENTRAL) {
    // Eq. 3 blended over the cell: only the cross-shaped 32-voxel subset is needed.
    // zt[a][b] = T_z-contraction for b in {1,2}; all a.
    float zt_x[4][2], zt_y[2][4], zd[2][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 1; b <= 2; ++b) {
        zt_x[a][b - 1] = kT(0.f, nb(a, b, 1), nb(a, b, 2), 0.f, fz);
      }
#pragma unroll
    for (int a = 1; a <= 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (b == 1 || b == 2) {
          zt_y[a - 1][b] = zt_x[a][b - 1];
        } else {
          zt_y[a - 1][b] = kT(0.f, nb(a, b, 1), nb(a, b, 2), 0.f, fz);
        }
      }
#pragma unroll
    for (int a = 1; a <= 2; ++a)
#pragma unroll
      for (int b = 1; b <= 2; ++b) {
        zd[a - 1][b - 1] = kD(nb(a, b, 0), nb(a, b, 1), nb(a, b, 2), nb(a, b, 3), fz);
      }
    // x: D_x over a of (T_y over b of zt)
    float yt[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) yt[a] = fmaf(fy, zt_x[a][1] - zt_x[a][0], zt_x[a][0]);
    s = kT(yt[0], yt[1], yt[2], yt[3], fx);
    g[0] = kD(yt[0], yt[1], yt[2], yt[3], fx);
    float yd[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) yd[a] = kD(zt_y[a][0], zt_y[a][1], zt_y[a][2], zt_y[a][3], fy);
    g[1] = fmaf(fx, yd[1] - yd[0], yd[0]);
    const float z0 = fmaf(fy, zd[0][1] - zd[0][0], zd[0][0]);
    const float z1 = fmaf(fy, zd[1][1] - zd[1][0], zd[1][0]);
    g[2] = fmaf(fx, z1 - z0, z0);
  } else {
    constexpr float w0 = (OP == OP_SOBEL) ? 6.0f : 1.0f;
    constexpr float w1 = (OP == OP_SOBEL) ? 3.0f : 0.70710678118654752f;
    constexpr float w2 = (OP == OP_SOBEL) ? 1.0f : 0.57735026918962576f;
    float Zt[4][4], Zu[4][4], Zd[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const float n0 = nb(a, b, 0), n1 = nb(a, b, 1), n2 = nb(a, b, 2), n3 = nb(a, b, 3);
        Zt[a][b] = kT(n0, n1, n2, n3, fz);
        Zu[a][b] = kU(n0, n1, n2, n3, fz);
        Zd[a][b] = kD(n0, n1, n2, n3, fz);
      }
    float ytt[4], yut[4], ydt[4], ytu[4], yuu[4], ydu[4], ytd[4], yud[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ytt[a] = kT(Zt[a][0], Zt[a][1], Zt[a][2], Zt[a][3], fy);
      yut[a] = kU(Zt[a][0], Zt[a][1], Zt[a][2], Zt[a][3], fy);
      ydt[a] = kD(Zt[a][0], Zt[a][1], Zt[a][2], Zt[a][3], fy);
      ytu[a] = kT(Zu[a][0], Zu[a][1], Zu[a][2], Zu[a][3], fy);
      yuu[a] = kU(Zu[a][0], Zu[a][1], Zu[a][2], Zu[a][3], fy);
      ydu[a] = kD(Zu[a][0], Zu[a][1], Zu[a][2], Zu[a][3], fy);
      ytd[a] = kT(Zd[a][0], Zd[a][1], Zd[a][2], Zd[a][3], fy);
      yud[a] = kU(Zd[a][0], Zd[a][1], Zd[a][2], Zd[a][3], fy);
    }
    s = kT(ytt[0], ytt[1], ytt[2], ytt[3], fx);
    float ex[4], ey0[4], ey1[4], ez0[4], ez1[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ex[a] = w0 * ytt[a] + w1 * (ytu[a] + yut[a]) + w2 * yuu[a];
      ey0[a] = w0 * ydt[a] + w1 * ydu[a];
      ey1[a] = w1 * ydt[a] + w2 * ydu[a];
      ez0[a] = w0 * ytd[a] + w1 * yud[a];
      ez1[a] = w1 * ytd[a] + w2 * yud[a];
    }
    g[0] = kD(ex[0], ex[1], ex[2], ex[3], fx);
    g[1] = kT(ey0[0], ey0[1], ey0[2], ey0[3], fx) + kU(ey1[0], ey1[1], ey1[2], ey1[3], fx);
    g[2] = kT(ez0[0], ez0[1], ez0[2], ez0[3], fx) + kU(ez1[0], ez1[1], ez1[2], ez1[3], fx);
  }
}

// Neighbourhood of a cell in the padded volume (no clamping needed).
template <int VTYPE>
struct PaddedHood {
  const typename VoxelT<VTYPE>::T* v;
  int b0, px, pxy;  // b0: padded offset of N[0][0][0]
  __device__ __forceinline__ float operator()(int a, int b, int c) const {
    return ldv<VTYPE>(v, b0 + a + b * px + c * pxy);
  }
};

template <int VTYPE, int OP>
__device__ __forceinline__ void value_and_gradient(const VolDev& V, const Cell& c, float& s,
                                                   float g[3]) {
  // the 4 x 4 x 4 neighbourhood spans offsets 0 .. 3 (1 + px + pxy) from its first voxel
  const int b0 = (int)VR_CHECK(V.bounds, c.base - 1 - V.px - V.pxy, 0,
                               padded_elems(V) - 1 - 3 * (1 + V.px + V.pxy));
  PaddedHood<VTYPE> nb{static_cast<const typename VoxelT<VTYPE>::T*>(V.data), b0, V.px, V.pxy};
  contract_neighbourhood<OP>(nb, c.f, s, g);
}

// Scale of each operator: 1 / (2 * sum of one side's weights).
__host__ __device__ constexpr float op_scale(int op) {
  return op == OP_CENTRAL ? 0.5f
       : op == OP_SOBEL   ? (1.0f / 44.0f)
                          : (float)(1.0 / (2.0 * (1.0 + 4.0 / 1.4142135623730951 +
                                                  4.0 / 1.7320508075688772)));
}

// --------------------------------------------------------------------- shading
struct ShadeOut {
  float c[3];
  float N[3], L[3], V[3];
  float nl, rv, gl;  // N.L, R.V, |g_hat|
};

// Outward normal N = -g/|g| (zero below 1e-6), point light and Phong (§3.8).
__device__ __forceinline__ void shade(const ShadeDev& sh, const CamDev& cam, const float d[3],
                                      const float p[3], const float gh[3], const float4& rgba,
                                      ShadeOut& r) {
  const float g2 = gh[0] * gh[0] + gh[1] * gh[1] + gh[2] * gh[2];
  r.gl = sqrtf(g2);
  if (g2 > 1e-12f) {
    const float inv = -rsqrtf(g2);
    r.N[0] = gh[0] * inv; r.N[1] = gh[1] * inv; r.N[2] = gh[2] * inv;
  } else {
    r.N[0] = r.N[1] = r.N[2] = 0.0f;
  }
  float lp[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) lp[a] = (sh.headlight ? cam.eye[a] : sh.light[a]) - p[a];
  const float il = rsqrtf(lp[0] * lp[0] + lp[1] * lp[1] + lp[2] * lp[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) r.L[a] = lp[a] * il;
  if (cam.ortho) {
#pragma unroll
    for (int a = 0; a < 3; ++a) r.V[a] = -d[a];
  } else if (sh.headlight) {
#pragma unroll
    for (int a = 0; a < 3; ++a) r.V[a] = r.L[a];
  } else {
    float e[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) e[a] = cam.eye[a] - p[a];
    const float ie = rsqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) r.V[a] = e[a] * ie;
  }
  const float nl = r.N[0] * r.L[0] + r.N[1] * r.L[1] + r.N[2] * r.L[2];
  r.nl = nl;
  const float diff = fmaxf(nl, 0.0f);
  float spec = 0.0f;
  r.rv = 0.0f;
  if (nl > 0.0f) {
    const float nv = r.N[0] * r.V[0] + r.N[1] * r.V[1] + r.N[2] * r.V[2];
    const float lv = r.L[0] * r.V[0] + r.L[1] * r.V[1] + r.L[2] * r.V[2];
    const float rv = 2.0f * nl * nv - lv;  // R.V with R = 2 (N.L) N - L
    r.rv = rv;
    if (rv > 0.0f) spec = __powf(rv, sh.shininess);
  }
  const float k = fmaf(sh.kd, diff, sh.ka);
  r.c[0] = fmaf(rgba.x, k, sh.ks * spec);
  r.c[1] = fmaf(rgba.y, k, sh.ks * spec);
  r.c[2] = fmaf(rgba.z, k, sh.ks * spec);
}

// Index of the macro brick holding brick b.
__device__ __forceinline__ int macro_of(const VolDev& V, const int b[3]) {
  return (b[0] >> kMacroShift) + V.nm[0] * ((b[1] >> kMacroShift) + V.nm[1] * (b[2] >> kMacroShift));
}

// Index of the brick containing p (clamped to the brick grid).
__device__ __forceinline__ int brick_of(const VolDev& V, const float p[3], int b[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int i = ((int)floorf(p[a])) >> kBrickShift;
    b[a] = i < 0 ? 0 : (i >= V.nb[a] ? V.nb[a] - 1 : i);
  }
  return b[0] + V.nb[0] * (b[1] + V.nb[1] * b[2]);
}

// First sample index whose t lies at or beyond the exit of the axis-aligned region
// [c << shift, (c + 1) << shift) (a brick for shift 3, a macro brick for shift 5), with the
// ray's reciprocal direction and step precomputed.  Rounding of t is harmless: every brick's
// footprint covers one voxel around it, so samples just past the exit are still transparent.
__device__ __forceinline__ int region_exit_sample(const int c[3], int shift, const float o[3],
                                                  const float d[3], const float inv_d[3],
                                                  float tn, float inv_step) {
  float te = __int_as_float(0x7f800000);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] > 0.0f) te = fminf(te, ((float)((c[a] + 1) << shift) - o[a]) * inv_d[a]);
    else if (d[a] < 0.0f) te = fminf(te, ((float)(c[a] << shift) - o[a]) * inv_d[a]);
  }
  const float kf = ceilf(fmaf(te - tn, inv_step, -0.5f));
  return kf > 2.0e9f ? 2000000000 : (int)kf;
}

// First sample index whose t lies at or beyond the exit of brick b (§5.3 skipping; the
// brick footprint tables cover one voxel around the brick, so rounding of t is harmless).
__device__ __forceinline__ int brick_exit_sample(const int b[3], const float o[3],
                                                 const float d[3], float tn, float step) {
  float te = __int_as_float(0x7f800000);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] > 0.0f) te = fminf(te, ((float)((b[a] + 1) << kBrickShift) - o[a]) / d[a]);
    else if (d[a] < 0.0f) te = fminf(te, ((float)(b[a] << kBrickShift) - o[a]) / d[a]);
  }
  const float kf = ceilf((te - tn) / step - 0.5f);
  return kf > 2.0e9f ? 2000000000 : (int)kf;
}

}  // namespace vr
