// vr_records.cuh -- the gradient record of a voxel (§3.5): the operator gradient G on the
// integer grid and the voxel's value, assembled from sums over the z planes of its 3x3x3
// clamp-to-edge neighbourhood.  Shared by the records pass (every visible brick, written to
// global memory) and the slab march (the region a ray tile crosses, in shared memory): both
// produce the same bits for the same voxel.
#pragma once

#include "vr_internal.h"

namespace vr {

// Sums of one z plane of a voxel's 3x3x3 neighbourhood (pl[y][x], the voxel at [w+1][u+1])
// from which the operators of §3.5 are assembled.  Every 3x3x3 operator here weights a tap
// by its class only: centre w0, edge w1, corner w2 of the 3x3 mask across the component's
// axis.  With d_x(b) the difference along x in row b of the plane, and likewise d_y(a):
//   ax = d_x(0), bx = d_x(-1) + d_x(+1), ay = d_y(0), by = d_y(-1) + d_y(+1),
//   q  = the plane weighted by the mask (for the z component), c = the voxel's own value.
// G_x = w0 ax(z) + w1 (bx(z) + ax(z-1) + ax(z+1)) + w2 (bx(z-1) + bx(z+1)), G_y likewise,
// G_z = q(z+1) - q(z-1); central differences use ax, ay and c only.  Every way of computing
// the sums below adds the same terms in the same order (or, for integer voxels, in an order
// whose every partial sum is exact), so a voxel's record does not depend on which kernel, or
// which of its code paths, produced it.
struct PlaneSums {
  float ax, bx, ay, by, q, c;
};

template <int OP>
struct OpWeights {
  static constexpr float w0 = (OP == OP_SOBEL) ? 6.0f : 1.0f;
  static constexpr float w1 = (OP == OP_SOBEL) ? 3.0f : 0.70710678118654752f;
  static constexpr float w2 = (OP == OP_SOBEL) ? 1.0f : 0.57735026918962576f;
};

// Plane sums from the 3x3 patch p[b][a] (row b, column a; the voxel at p[1][1]).
template <int OP>
__device__ __forceinline__ PlaneSums plane_sums_of(const float p[3][3]) {
  PlaneSums r;
  r.ax = p[1][2] - p[1][0];
  r.ay = p[2][1] - p[0][1];
  r.c = p[1][1];
  if constexpr (OP == OP_CENTRAL) {
    r.bx = r.by = r.q = 0.0f;
  } else {
    constexpr float w0 = OpWeights<OP>::w0, w1 = OpWeights<OP>::w1, w2 = OpWeights<OP>::w2;
    r.bx = (p[0][2] - p[0][0]) + (p[2][2] - p[2][0]);
    r.by = (p[2][0] - p[0][0]) + (p[2][2] - p[0][2]);
    r.q = fmaf(w0, p[1][1], fmaf(w1, (p[0][1] + p[2][1]) + (p[1][0] + p[1][2]),
                                 w2 * ((p[0][0] + p[0][2]) + (p[2][0] + p[2][2]))));
  }
  return r;
}

// Plane sums of the voxel at column u + 1, row w + 1 of a plane stored with row pitch `pitch`.
template <int OP>
__device__ __forceinline__ PlaneSums plane_sums_at(const float* pl, int pitch, int u, int w) {
  float p[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) p[b][a] = pl[(w + b) * pitch + u + a];
  return plane_sums_of<OP>(p);
}

template <int OP>
__device__ __forceinline__ PlaneSums plane_sums(const float (*pl)[12], int u, int w) {
  return plane_sums_at<OP>(&pl[0][0], 12, u, w);
}

// Plane sums of two neighbouring voxels (tile columns u + 1 and u + 2, rows w .. w + 2) from
// one 3 x 4 patch read with 64-bit shared loads (u even).  INTEGER: the voxels are integers
// (8- or 16-bit storage), so every partial sum below is exact in FP32 and the two voxels may
// share the patch's sums along y -- the result equals plane_sums_of bit for bit; otherwise
// each voxel's sums are formed as plane_sums_of forms them.
template <int OP, bool INTEGER = false>
__device__ __forceinline__ void plane_sums2(const float (*pl)[12], int u, int w, PlaneSums& A,
                                            PlaneSums& B) {
  float p[3][4];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const float2 lo = *reinterpret_cast<const float2*>(&pl[w + b][u]);
    const float2 hi = *reinterpret_cast<const float2*>(&pl[w + b][u + 2]);
    p[b][0] = lo.x;
    p[b][1] = lo.y;
    p[b][2] = hi.x;
    p[b][3] = hi.y;
  }
  if constexpr (INTEGER && OP != OP_CENTRAL) {
    constexpr float w0 = OpWeights<OP>::w0, w1 = OpWeights<OP>::w1, w2 = OpWeights<OP>::w2;
    float dy[4], sy[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      dy[c] = p[2][c] - p[0][c];
      sy[c] = p[0][c] + p[2][c];
    }
    A.ax = p[1][2] - p[1][0];
    B.ax = p[1][3] - p[1][1];
    A.c = p[1][1];
    B.c = p[1][2];
    A.ay = dy[1];
    B.ay = dy[2];
    A.bx = sy[2] - sy[0];
    B.bx = sy[3] - sy[1];
    A.by = dy[0] + dy[2];
    B.by = dy[1] + dy[3];
    A.q = fmaf(w0, p[1][1], fmaf(w1, sy[1] + (p[1][0] + p[1][2]), w2 * (sy[0] + sy[2])));
    B.q = fmaf(w0, p[1][2], fmaf(w1, sy[2] + (p[1][1] + p[1][3]), w2 * (sy[1] + sy[3])));
  } else {
    float pa[3][3], pb[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pa[b][a] = p[b][a];
        pb[b][a] = p[b][a + 1];
      }
    A = plane_sums_of<OP>(pa);
    B = plane_sums_of<OP>(pb);
  }
}

// The record (G_x, G_y, G_z, value) of a voxel from the plane sums below, at and above it.
template <int OP>
__device__ __forceinline__ float4 record_of(const PlaneSums& lo, const PlaneSums& md,
                                            const PlaneSums& hi) {
  if constexpr (OP == OP_CENTRAL) {
    return make_float4(md.ax, md.ay, hi.c - lo.c, md.c);
  } else {
    constexpr float w0 = OpWeights<OP>::w0, w1 = OpWeights<OP>::w1, w2 = OpWeights<OP>::w2;
    return make_float4(fmaf(w0, md.ax, fmaf(w1, md.bx + (lo.ax + hi.ax), w2 * (lo.bx + hi.bx))),
                       fmaf(w0, md.ay, fmaf(w1, md.by + (lo.ay + hi.ay), w2 * (lo.by + hi.by))),
                       hi.q - lo.q, md.c);
  }
}

// Raw voxel -> float, as the records are computed.
template <int VTYPE>
__device__ __forceinline__ float raw_to_float(typename VoxelT<VTYPE>::T v) {
  if constexpr (VTYPE == VT_F16) return __half2float(v);
  else return (float)v;
}

}  // namespace vr
