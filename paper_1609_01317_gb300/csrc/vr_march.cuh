// vr_march.cuh -- the per-ray march shared by the single-frame and batched kernels.
//
// Four lanes (a quad) march one ray: lane q evaluates sample k + q of every group of four
// consecutive samples and every lane composites the group in sample order (§3.9, Eq. 6).
// The sample's value and operator gradient come from the 8 gradient records of its cell
// (§3.4, §3.5), then the transfer function (§3.7) and Phong (§3.8).
#pragma once

#include "vr_internal.h"

namespace vr {

// brick_of and cell_of of the device header, from ip = floor(p) computed once per sample
// (the brick test and the cell share it).
__device__ __forceinline__ int brick_of_floor(const VolDev& V, const int ip[3], int b[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int i = ip[a] >> kBrickShift;
    b[a] = i < 0 ? 0 : (i >= V.nb[a] ? V.nb[a] - 1 : i);
  }
  return b[0] + V.nb[0] * (b[1] + V.nb[1] * b[2]);
}

__device__ __forceinline__ Cell cell_of_floor(const VolDev& V, const float p[3], const int ip[3]) {
  Cell c;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int top = V.n[a] > 1 ? V.n[a] - 2 : 0;
    const int i = ip[a] < 0 ? 0 : (ip[a] > top ? top : ip[a]);
    c.ib[a] = i;
    c.f[a] = p[a] - (float)i;
  }
  c.base = (c.ib[0] + kPadLo) + V.px * (c.ib[1] + kPadLo) + V.pxy * (c.ib[2] + kPadLo);
  return c;
}

// The 8 corner records of a cell.
struct Corners {
  float4 r[8];  // index bit 0: +x, bit 1: +y, bit 2: +z
};

// Record indices fit in 32 bits: the upload refuses volumes of 2^31 voxels or more.
__device__ __forceinline__ void corners_load(const RecDev& R, const Cell& c, Corners& k) {
  const int base = (int)VR_CHECK(
      R.bounds, c.ib[0] + R.n[0] * (c.ib[1] + R.n[1] * c.ib[2]), 0,
      (long long)R.n[0] * R.n[1] * R.n[2] - 1 - corner_span(R));
  const float4* __restrict__ p = R.rec;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    k.r[i] = __ldg(p + (base + ((i & 1) ? R.sx : 0) + ((i & 2) ? R.sy : 0) + ((i & 4) ? R.sz : 0)));
}

// lerpf on two channels at once: one packed FP32 subtraction and one packed fused
// multiply-add (sm_100 and later), each channel rounded exactly as lerpf rounds it.
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float2 f) {
  return __ffma2_rn(f, __fadd2_rn(b, make_float2(-a.x, -a.y)), a);
}

// Trilinear interpolation (§3.4) of all four channels of the corner records at the sample:
// (G_x, G_y, G_z, V), lerps along x, then y, then z, two channels per packed instruction.
// The value channel takes the same seven lerps, in the same order, as the adjoint's
// recomputation of the forward (record_value), so both see the same opacities bit for bit.
// The gradient is blended before the transfer function says whether the sample is shaded:
// that frees the 32 registers of the corners early and lets the march run 8 blocks of 128
// threads per SM (measured faster than blending only shaded samples at 7 blocks).
__device__ __forceinline__ float4 corners_blend(const Corners& k, const Cell& c) {
  const float2 fx = make_float2(c.f[0], c.f[0]), fy = make_float2(c.f[1], c.f[1]),
               fz = make_float2(c.f[2], c.f[2]);
  float2 lo[4], hi[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float4 a = k.r[2 * i], b = k.r[2 * i + 1];
    lo[i] = lerp2(make_float2(a.x, a.y), make_float2(b.x, b.y), fx);
    hi[i] = lerp2(make_float2(a.z, a.w), make_float2(b.z, b.w), fx);
  }
  const float2 l0 = lerp2(lo[0], lo[1], fy), h0 = lerp2(hi[0], hi[1], fy);
  const float2 l1 = lerp2(lo[2], lo[3], fy), h1 = lerp2(hi[2], hi[3], fy);
  const float2 l = lerp2(l0, l1, fz), h = lerp2(h0, h1, fz);
  return make_float4(l.x, l.y, h.x, h.y);
}

// March one ray with a quad: lane q evaluates sample k + q of every group of four
// consecutive samples (value, transfer function and, if alpha != 0, gradient and Phong),
// then every lane composites the group front to back in sample order; the first sample
// after which 1 - T reaches the threshold ends the ray (later samples of the group are
// dropped, and counted as not marched).  A group whose samples
// all lie in invisible bricks jumps to the furthest of their brick exits: every sample in
// between lies in one of those bricks (each lane's interval starts at its own sample and the
// starts are consecutive), so nothing visible is skipped.
// TFS: the transfer function is read from s_tf, a copy in shared memory.
// ADAPT: adaptive sampling (§5.2): sample k is taken iff k mod m == 0, m in {1, 2, 4} the
// multiplier of its macro brick (L.r.mult), with opacity 1 - (1 - a)^m.  A group whose span of
// 4 m samples lies in one macro brick of multiplier m (its first and last samples share it;
// the macro index is monotone along the ray) takes samples k, k + m, k + 2m, k + 3m; any
// other group takes the next 1-4 consecutive samples up to a multiple of 4 (so the following
// group starts aligned to every multiplier) and drops the samples off their region's grid.
// march_core: the march of a ray whose set-up (o, d, tn, K) is given, from sample k0 (a
// multiple of 4; every sample before it lies in a transparent macro brick, so it contributes
// nothing).
// ZWIN: only the samples whose z lies in [L.zwin[0], L.zwin[1]) are composited (a partial
// image of one z-slab of the volume, on the whole box's sampling grid); the others count as
// transparent.
// JLOOP: a quad's run of consecutive jumps is taken in an inner loop of its own, so that a
// quad crossing empty space holds the other quads of its warp for its jumps only, not for a
// whole march iteration per jump; without it every jump ends the iteration.  The sequence of
// groups, and so the image, is the same either way.  The inner loop ends: every jump moves k
// on by at least 4 samples or to K (the progress rule of the jump, below).  Measured on GB300:
// faster for the tile march on the dense CT frame, slower for the list march on sparse data
// and for adaptive sampling (off for both).
template <bool CKPT, bool TFS = false, bool ADAPT = false, bool ZWIN = false, bool JLOOP = !ADAPT>
__device__ __forceinline__ void march_core(const MarchLaunch& L, const float o[3],
                                           const float d[3], float tn, int K, int k0, int px,
                                           int py, bool active, int q, unsigned qmask,
                                           unsigned& hit, unsigned& plain, unsigned& visited,
                                           unsigned& shaded, const float4* s_tf) {
  static_assert(!(CKPT && ADAPT), "the adjoint's checkpoints follow the regular grid");
  static_assert(!(ZWIN && (CKPT || ADAPT)), "partial images come from the plain march");
  const int W = L.cam.width, H = L.cam.height;
  const int ray = py * W + px;
  const int qbase = (threadIdx.x & 31) & ~3;
  float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, T = 1.0f;
  int k = k0;
  const float step = L.r.step;
  const float inv_step = 1.0f / step;
  float inv_d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) inv_d[a] = d[a] != 0.0f ? 1.0f / d[a] : 0.0f;
  while (k < K) {
    int stride, span, ks, kn, w;  // samples between the quad's lanes; samples the group covers
    float p[3];
    int ip[3];
    bool live, vis;
    bool jumped = false;  // without JLOOP: this iteration's group jumped
    for (;;) {
      stride = 1;
      span = 4;
      if constexpr (ADAPT) {
        float p0[3];
        const float t0 = fmaf((float)k + 0.5f, step, tn);
#pragma unroll
        for (int a = 0; a < 3; ++a) p0[a] = fmaf(t0, d[a], o[a]);
        int b0[3];
        brick_of(L.V, p0, b0);
        const int mi0 = macro_of(L.V, b0);
        const int m0 = __ldg(L.r.mult + VR_CHECK(L.V.bounds, mi0, 0, L.V.nm[0] * L.V.nm[1] * L.V.nm[2] - 1));
        if (m0 > 1 && (k & (m0 - 1)) == 0) {
          const int kl = min(k + 4 * m0 - 1, K - 1);
          float pl[3];
          const float tl = fmaf((float)kl + 0.5f, step, tn);
#pragma unroll
          for (int a = 0; a < 3; ++a) pl[a] = fmaf(tl, d[a], o[a]);
          int bl[3];
          brick_of(L.V, pl, bl);
          if (macro_of(L.V, bl) == mi0) {
            stride = m0;
            span = 4 * m0;
          }
        }
        if (stride == 1) span = 4 - (k & 3);
      }
      ks = k + q * stride;
      const float t = fmaf((float)ks + 0.5f, step, tn);
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
#pragma unroll
      for (int a = 0; a < 3; ++a) ip[a] = (int)floorf(p[a]);  // shared by brick and cell
      live = q * stride < span && ks < K;
      if constexpr (ZWIN) live = live && p[2] >= L.zwin[0] && p[2] < L.zwin[1];
      vis = live;
      kn = ks < K ? k + span : K;  // a lane past the group's span bounds the jump by it
      w = stride;                  // samples this lane's sample stands for
      if constexpr (ADAPT) {
        if (live && stride == 1) {
          int bm[3];
          brick_of(L.V, p, bm);
          w = __ldg(L.r.mult + VR_CHECK(L.V.bounds, macro_of(L.V, bm), 0,
                                        L.V.nm[0] * L.V.nm[1] * L.V.nm[2] - 1));
        }
      }
      if (L.r.skip && live) {
        int b[3];
        const int bi = brick_of_floor(L.V, ip, b);
        if (!__ldg(L.V.vis + VR_CHECK(L.V.bounds, bi, 0, L.V.nb[0] * L.V.nb[1] * L.V.nb[2] - 1))) {
          // transparent brick: leave it, or its whole macro brick when that is transparent too
          vis = false;
          int shift = kBrickShift;
          if (L.V.mvis) {
            const int m[3] = {b[0] >> kMacroShift, b[1] >> kMacroShift, b[2] >> kMacroShift};
            if (!__ldg(L.V.mvis + VR_CHECK(L.V.bounds, m[0] + L.V.nm[0] * (m[1] + L.V.nm[1] * m[2]),
                                           0, L.V.nm[0] * L.V.nm[1] * L.V.nm[2] - 1))) {
              b[0] = m[0];
              b[1] = m[1];
              b[2] = m[2];
              shift = kBrickShift + kMacroShift;
              if (L.V.svis) {
                const int u[3] = {m[0] >> kSuperShift, m[1] >> kSuperShift, m[2] >> kSuperShift};
                if (!__ldg(L.V.svis + VR_CHECK(L.V.bounds, u[0] + L.V.ns[0] * (u[1] + L.V.ns[1] * u[2]),
                                               0, L.V.ns[0] * L.V.ns[1] * L.V.ns[2] - 1))) {
                  b[0] = u[0];
                  b[1] = u[1];
                  b[2] = u[2];
                  shift = kBrickShift + kMacroShift + kSuperShift;
                }
              }
            }
          }
          kn = region_exit_sample(b, shift, o, d, inv_d, tn, inv_step);
          if (kn <= ks) kn = ks + 1;
        }
      }
      // a live lane in a visible brick keeps the group; otherwise the group jumps
      if (((__ballot_sync(qmask, vis) >> qbase) & 0xFu) != 0u) break;
      {
        // the whole group lies in empty bricks: jump
        kn = max(kn, __shfl_xor_sync(qmask, kn, 1));
        kn = max(kn, __shfl_xor_sync(qmask, kn, 2));
        if (CKPT && q == 0) {
          const int stop = kn < K ? kn : K;
          for (int j = ((k + kCkptStride - 1) >> 5) << 5; j < stop; j += kCkptStride)
            if (j > 0) L.ck_T[(size_t)((j >> 5) - 1) * (W * H) + ray] = T;
        }
        // Without adaptive sampling groups stay aligned to multiples of four, so that lane q
        // always holds the samples k = q (mod 4); the samples of the new group before kn lie
        // in the bricks just left (transparent: they contribute nothing).  Progress: if every
        // lane was live, lane 3's exit makes kn >= k + 4, so kn rounded down is still >= k + 4;
        // otherwise a lane past K set kn = K and the ray ends here (no rounding).
        k = (ADAPT || kn >= K) ? kn : (kn & ~3);
      }
      if (!JLOOP) {
        jumped = true;
        break;
      }
      if (k >= K) break;
    }
    if (k >= K) break;
    if (jumped) continue;
    float alpha = 0.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
    if constexpr (ADAPT) {
      if (stride == 1 && (ks & (w - 1)) != 0) vis = false;  // off its brick's coarser grid
    }
    if (vis) {
      ++visited;
      const Cell c = cell_of_floor(L.V, p, ip);
      Corners cr;
      corners_load(L.R, c, cr);
      const float4 bl = corners_blend(cr, c);
      const float s = bl.w;
      const TfSample ts = tf_lookup<TFS>(L.tf, s, s_tf);
      alpha = ts.rgba.w;
      if constexpr (ADAPT) {
        if (w > 1) {  // the sample stands for w samples: 1 - (1 - a)^w, w in {2, 4}
          const float om = 1.0f - alpha, om2 = om * om;
          alpha = 1.0f - (w == 2 ? om2 : om2 * om2);
        }
      }
      if (alpha != 0.0f) {
        ++shaded;
        const float gh[3] = {bl.x * L.r.gscale, bl.y * L.r.gscale, bl.z * L.r.gscale};
        ShadeOut so;
        shade(L.r.sh, L.cam, d, p, gh, ts.rgba, so);
        c0 = so.c[0];
        c1 = so.c[1];
        c2 = so.c[2];
      }
    }
    // Composite the group in sample order with the recurrence of Eq. 6.  T runs through
    // the group's samples in order on every lane (the same FP32 operations as a
    // one-sample-at-a-time march).  Without adaptive sampling each lane adds only its own
    // sample's term T_before * alpha * c to a partial colour, and the four partial colours
    // are summed once at the end of the ray: groups are aligned to multiples of four (also
    // after a jump), so lane q sums the samples k = q (mod 4) whether or not transparent
    // bricks are skipped, and a zero alpha adds an exact zero -- skipping never changes a
    // bit of the result.  With adaptive sampling the groups follow the regions, and every
    // lane sums all terms in sample order.  A zero alpha leaves C and T bit-identical (its
    // colour is zero and 1 - 0 is exact), so it needs no branch.
    bool stop = false;
    int used = 0;
    if constexpr (ADAPT) {
      float a4[4], c4[4][3];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a4[j] = __shfl_sync(qmask, alpha, j, 4);
        c4[j][0] = __shfl_sync(qmask, c0, j, 4);
        c4[j][1] = __shfl_sync(qmask, c1, j, 4);
        c4[j][2] = __shfl_sync(qmask, c2, j, 4);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!stop && j * stride < span && k + j * stride < K) {
          const float aj = a4[j];
          const float ta = T * aj;
          C0 = fmaf(ta, c4[j][0], C0);
          C1 = fmaf(ta, c4[j][1], C1);
          C2 = fmaf(ta, c4[j][2], C2);
          T = T * (1.0f - aj);
          used = j * stride + 1;
          if (1.0f - T >= L.r.ert) stop = true;
        }
      }
    } else {
      float a4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a4[j] = __shfl_sync(qmask, alpha, j, 4);
      float Tq = 0.0f;  // transmittance before this lane's sample (0: not composited)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (!stop && j < span && k + j < K) {
          if (CKPT && q == 0 && k + j > 0 && ((k + j) & (kCkptStride - 1)) == 0)
            L.ck_T[(size_t)(((k + j) >> 5) - 1) * (W * H) + ray] = T;
          if (j == q) Tq = T;
          T = T * (1.0f - a4[j]);
          used = j + 1;
          if (1.0f - T >= L.r.ert) stop = true;
        }
      }
      const float ta = Tq * alpha;
      C0 = fmaf(ta, c0, C0);
      C1 = fmaf(ta, c1, C1);
      C2 = fmaf(ta, c2, C2);
    }
    k += stop ? used : span;
    if (stop) break;
  }
  const int kend = k < K ? k : K;
  if constexpr (!ADAPT) {
    // the quad's partial colours, summed in a fixed order: (C_0 + C_1) + (C_2 + C_3)
    C0 += __shfl_xor_sync(qmask, C0, 1);
    C1 += __shfl_xor_sync(qmask, C1, 1);
    C2 += __shfl_xor_sync(qmask, C2, 1);
    C0 += __shfl_xor_sync(qmask, C0, 2);
    C1 += __shfl_xor_sync(qmask, C1, 2);
    C2 += __shfl_xor_sync(qmask, C2, 2);
  }
  if (active && q == 0) {
    reinterpret_cast<float4*>(L.out)[(size_t)(py - L.row0) * W + px] =
        make_float4(C0, C1, C2, 1.0f - T);
    if (CKPT) {
      L.ck_kend[ray] = kend;
      L.ck_Tend[ray] = T;
    }
    hit += K > 0 ? 1u : 0u;
    plain += (unsigned)kend;
  }
}

// The march of pixel (px, py): ray set-up (§3.3, §3.6), then march_core from sample 0.
template <bool CKPT, bool TFS = false, bool ADAPT = false, bool ZWIN = false>
__device__ __forceinline__ void march_ray(const MarchLaunch& L, int px, int py, bool active,
                                          int q, unsigned qmask, unsigned& hit, unsigned& plain,
                                          unsigned& visited, unsigned& shaded,
                                          const float4* s_tf = nullptr) {
  float o[3], d[3], tn = 0.0f;
  int K = 0;
  if (active) ray_setup(L.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
  int k0 = 0;
  if constexpr (ZWIN) {
    // march only the groups around the samples inside the z window (one sample of margin on
    // either side: the exact test is each sample's own position)
    if (K > 0) {
      if (d[2] != 0.0f) {
        const float ta = (L.zwin[0] - o[2]) / d[2], tb = (L.zwin[1] - o[2]) / d[2];
        const float inv_step = 1.0f / L.r.step;
        const float kf0 = floorf(fmaf(fminf(ta, tb) - tn, inv_step, -0.5f)) - 1.0f;
        const float kf1 = ceilf(fmaf(fmaxf(ta, tb) - tn, inv_step, -0.5f)) + 2.0f;
        k0 = !(kf0 > 0.0f) ? 0 : (kf0 >= (float)K ? K : ((int)kf0 & ~3));
        if (kf1 < (float)K) K = kf1 > 0.0f ? (int)kf1 : 0;
        if (k0 > K) k0 = K & ~3;
      } else if (!(o[2] >= L.zwin[0] && o[2] < L.zwin[1])) {
        K = 0;
      }
    }
  }
  march_core<CKPT, TFS, ADAPT, ZWIN>(L, o, d, tn, K, k0, px, py, active, q, qmask, hit, plain,
                                     visited, shaded, s_tf);
}

}  // namespace vr
