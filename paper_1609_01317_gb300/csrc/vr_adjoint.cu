// vr_adjoint.cu -- reverse-mode differentiation of the ray march.
//
// The forward pass (vr_render_forward_train) stores, per ray, the index of the last
// sample it composited and the transmittance T before every 32nd sample.  The adjoint
// walks each ray back to front one 32-sample segment at a time: it recomputes the
// segment's transmittances from the stored T (value + transfer function only), then
// visits the samples in reverse order, recomputing each sample in full from the gradient
// records (value, operator gradient, normal, Phong) and applying the chain rule of Eq. 6
// (§3.9):
//   C = sum_k T_k a_k c_k,  T_{k+1} = T_k (1 - a_k),  A = 1 - T_end
//   dL/da_k = T_k (g.c_k - Tadj_{k+1}),  dL/dc_k = T_k a_k g,
//   Tadj_k  = a_k g.c_k + (1 - a_k) Tadj_{k+1},  Tadj_end = -dL/dA,
// with g = dL/dRGB.  Gradients flow through Phong (§3.8), the normalisation of the
// operator gradient, the transfer-function interpolation (§3.7) and the trilinear blend
// (§3.4).  Because the operator gradient at p is the trilinear blend of the integer-grid
// operator G at the cell corners, the kernel scatters (dL/ds, dL/dG) to the 8 corners
// with one vector atomic each; a second, dense pass applies the transposed operator
// stencil (with the clamp-to-edge folding) to turn dL/dG into dL/dV.
#include <algorithm>

#include "vr_internal.h"

namespace vr {

constexpr int kThreads = 128;
constexpr int kMaxTfRows = 4096;  // per-block partial rows of the TF gradient up to this many entries
constexpr int kMaxSharedTf = 1024;  // the block copies transfer functions up to this size to shared memory
constexpr int kQuadTileW = 4, kQuadTileH = 2;  // pixels per warp (a quad of lanes per ray)

// Corner records of a cell and the trilinear weights of the sample in it.
struct AdjCell {
  size_t base;  // record index of the cell's (0,0,0) corner
  float f[3];
};

__device__ __forceinline__ AdjCell adj_cell(const VolDev& V, const float p[3]) {
  AdjCell a;
  int ib[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int c = (int)floorf(p[i]);
    const int top = V.n[i] > 1 ? V.n[i] - 2 : 0;
    c = c < 0 ? 0 : (c > top ? top : c);
    ib[i] = c;
    a.f[i] = p[i] - (float)c;
  }
  a.base = (size_t)ib[0] + (size_t)V.n[0] * ((size_t)ib[1] + (size_t)V.n[1] * ib[2]);
  // corners reach +1 along every axis longer than one voxel
  a.base = (size_t)VR_CHECK(V.bounds, a.base, 0,
                            (long long)V.n[0] * V.n[1] * V.n[2] - 1 -
                                ((V.n[0] > 1) + (V.n[1] > 1) * (long long)V.n[0] +
                                 (V.n[2] > 1) * (long long)V.n[0] * V.n[1]));
  return a;
}

__device__ __forceinline__ size_t corner_index(const RecDev& R, size_t base, int i) {
  return base + ((i & 1) ? R.sx : 0) + ((i & 2) ? R.sy : 0) + ((i & 4) ? R.sz : 0);
}

__device__ __forceinline__ float corner_weight(const float f[3], int i) {
  return ((i & 1) ? f[0] : 1.0f - f[0]) * ((i & 2) ? f[1] : 1.0f - f[1]) *
         ((i & 4) ? f[2] : 1.0f - f[2]);
}

// Trilinear value from the records' V channel (lerps along x, y, z as in the forward).
__device__ __forceinline__ float record_value(const RecDev& R, const AdjCell& c, float4 r[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = __ldg(R.rec + corner_index(R, c.base, i));
  const float x00 = lerpf(r[0].w, r[1].w, c.f[0]), x10 = lerpf(r[2].w, r[3].w, c.f[0]);
  const float x01 = lerpf(r[4].w, r[5].w, c.f[0]), x11 = lerpf(r[6].w, r[7].w, c.f[0]);
  return lerpf(lerpf(x00, x10, c.f[1]), lerpf(x01, x11, c.f[1]), c.f[2]);
}

// §3.7 lookup with linear interpolation between entries (the forward's tf_lookup), also
// returning the difference of the two entries read: the slope of the table in u.
template <bool SMEM>
__device__ __forceinline__ TfSample tf_lookup_slope(const TfDev& tf, const float4* s_tf,
                                                    float s_raw, float4& dab) {
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
  if constexpr (SMEM) {
    a = s_tf[i];
    b = s_tf[i + 1];
  } else {
    a = __ldg(tf.tf + i);
    b = __ldg(tf.tf + i + 1);
  }
  r.rgba.x = lerpf(a.x, b.x, r.w);
  r.rgba.y = lerpf(a.y, b.y, r.w);
  r.rgba.z = lerpf(a.z, b.z, r.w);
  r.rgba.w = lerpf(a.w, b.w, r.w);
  dab = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
  return r;
}

__device__ __forceinline__ void flush_tf(float* dst, int i, const float lo[4], const float hi[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (lo[q] != 0.0f) atomicAdd(dst + 4 * i + q, lo[q]);
    if (hi[q] != 0.0f) atomicAdd(dst + 4 * (i + 1) + q, hi[q]);
  }
}

// Transmittance before sample kg, recomputed forward from the checkpoint of its
// 32-sample segment (used when dividing back through a group would lose precision).
__device__ __noinline__ float recompute_T(const AdjointLaunch& L, const float* ck_T, int nrays,
                                          const float o[3], const float d[3], float tn, int kg,
                                          int ray) {
  const int s0 = (kg >> 5) << 5;
  float T = s0 == 0 ? 1.0f : ck_T[(size_t)((s0 >> 5) - 1) * nrays + ray];
  for (int j = s0; j < kg; ++j) {
    const float t = fmaf((float)j + 0.5f, L.r.step, tn);
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
    float4 r[8];
    const float al = tf_lookup(L.tf, record_value(L.R, adj_cell(L.V, p), r)).rgba.w;
    if (al != 0.0f) T = T * (1.0f - al);
  }
  return T;
}


// Adds a finished run of the transfer-function gradient (lo to entry i, hi to entry i + 1)
// to the block's row of the partial sums with two vector reductions.
__device__ __forceinline__ void flush_tf_row(float* row, int i, const float lo[4], const float hi[4]) {
  float4* e = reinterpret_cast<float4*>(row) + i;
  if (lo[0] != 0.0f || lo[1] != 0.0f || lo[2] != 0.0f || lo[3] != 0.0f)
    atomicAdd(e, make_float4(lo[0], lo[1], lo[2], lo[3]));
  if (hi[0] != 0.0f || hi[1] != 0.0f || hi[2] != 0.0f || hi[3] != 0.0f)
    atomicAdd(e + 1, make_float4(hi[0], hi[1], hi[2], hi[3]));
}

// Four lanes per ray: lane q takes sample kg + q of every group of four, groups visited from
// the last to the first.  Per group: the transmittances before each sample come from the
// transmittance after the group divided by the product of (1 - alpha) over it (exactly
// re-anchored at every 32-sample checkpoint), and the adjoint of the transmittance follows
// from a suffix scan of the affine maps Tadj -> alpha g.c + (1 - alpha) Tadj.  The group loop
// runs the same number of times on every lane of the warp (quads whose ray is done idle).
template <bool SMEM>
__global__ void __launch_bounds__(kThreads) k_adjoint(const __grid_constant__ AdjointLaunch L) {
  // SMEM: the block reads the transfer function from its copy in shared memory
  extern __shared__ float4 s_tf[];
  if constexpr (SMEM) {
    for (int i = threadIdx.x; i < L.tf.n; i += kThreads) s_tf[i] = __ldg(L.tf.tf + i);
    __syncthreads();
  }
  // TF contributions: summed in registers per run of samples that read the same pair of
  // entries; a finished run goes to this block's row of the partial sums in global memory
  // (vector reductions, no contention between blocks), or, without a partial-sum buffer,
  // straight to grad_tf with scalar atomics.
  const int tid = threadIdx.x;
  const int lane = tid & 31, q = lane & 3, qd = lane >> 2;
  float* tf_row = L.tf_partial ? L.tf_partial + (size_t)blockIdx.x * 4 * L.tf.n : nullptr;
  const unsigned qmask = 0xFu << (lane & ~3);
  const float step = L.r.step;
  const float gs = L.r.gscale;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(L.tile_counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= L.tiles_total) break;
    // the view of this tile: the last one whose first tile is <= tile
    int lo = 0, hi = L.nviews;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (L.view[mid].tile0 <= tile) lo = mid;
      else hi = mid;
    }
    const AdjView& vw = L.view[lo];
    const int local = tile - vw.tile0;
    const int W = vw.cam.width, H = vw.cam.height;
    const int nrays = W * H;
    const int px = (vw.tx0 + local % vw.tiles_x) * kQuadTileW + (qd & 3);
    const int py = (vw.ty0 + local / vw.tiles_x) * kQuadTileH + (qd >> 2);
    const bool active = px < W && py < H;
    const int ray = py * W + px;
    float o[3], d[3], tn = 0.0f;
    int K = 0, kend = 0;
    if (active) {
      ray_setup(vw.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
      kend = min(max(vw.ck_kend[ray], 0), K);
    }
    float4 gr = make_float4(0.f, 0.f, 0.f, 0.f);
    float Tcur = 1.0f;
    if (kend > 0) {
      gr = __ldg(vw.grad_rgba + ray);
      Tcur = vw.ck_Tend[ray];
    }
    float Tadj = -gr.w;
    const int ng = kend > 0 ? ((kend - 1) >> 2) + 1 : 0;  // groups of this quad's ray
    const int maxg = (int)__reduce_max_sync(0xffffffffu, (unsigned)ng);
    int tf_run = -1;
    float tf_lo[4] = {0.f, 0.f, 0.f, 0.f}, tf_hi[4] = {0.f, 0.f, 0.f, 0.f};
    for (int it = 0; it < maxg; ++it) {
      bool contrib = false;
      int ci = 0;
      float cw = 0.0f;
      float drgba[4] = {0.f, 0.f, 0.f, 0.f};
      if (it < ng) {
        const int kg = (ng - 1 - it) << 2;
        const int k = kg + q;
        const bool live = k < kend;
        float alpha = 0.0f, gc = 0.0f;
        float p[3];
        AdjCell c;
        float4 r[8];
        TfSample ts;
        float4 dab;  // tf[i + 1] - tf[i] of the sample's entries
        ShadeOut so;
        float gh[3] = {0.f, 0.f, 0.f};
        float sv[4] = {0.f, 0.f, 0.f, 0.f};  // (dL/ds, dL/dG) of this sample
        bool scat = false;
        if (live) {
          const float t = fmaf((float)k + 0.5f, step, tn);
#pragma unroll
          for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
          c = adj_cell(L.V, p);
          ts = tf_lookup_slope<SMEM>(L.tf, s_tf, record_value(L.R, c, r), dab);
          float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float wci = corner_weight(c.f, i);
            g[0] = fmaf(wci, r[i].x, g[0]);
            g[1] = fmaf(wci, r[i].y, g[1]);
            g[2] = fmaf(wci, r[i].z, g[2]);
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) gh[a] = g[a] * gs;
          shade(L.r.sh, vw.cam, d, p, gh, ts.rgba, so);
          alpha = ts.rgba.w;
          gc = gr.x * so.c[0] + gr.y * so.c[1] + gr.z * so.c[2];
        }
        // transmittances: exclusive / inclusive prefix products of (1 - alpha) over the group
        const float om = 1.0f - alpha;
        float P = om;
        float u = __shfl_up_sync(qmask, P, 1, 4);
        if (q >= 1) P *= u;
        u = __shfl_up_sync(qmask, P, 2, 4);
        if (q >= 2) P *= u;
        float E = __shfl_up_sync(qmask, P, 1, 4);
        if (q == 0) E = 1.0f;
        const float prod = __shfl_sync(qmask, P, 3, 4);
        float Tb;
        if (kg == 0) Tb = 1.0f;
        else if ((kg & (kCkptStride - 1)) == 0) Tb = vw.ck_T[(size_t)((kg >> 5) - 1) * nrays + ray];
        else if (prod > 1e-4f) Tb = Tcur / prod;
        else Tb = recompute_T(L, vw.ck_T, nrays, o, d, tn, kg, ray);
        const float Tk = Tb * E;
        // adjoint of T: suffix scan of x -> A + B x over the group
        float A = alpha * gc, B = om;
        float An = __shfl_down_sync(qmask, A, 1, 4), Bn = __shfl_down_sync(qmask, B, 1, 4);
        if (q <= 2) {
          A = fmaf(B, An, A);
          B = B * Bn;
        }
        An = __shfl_down_sync(qmask, A, 2, 4);
        Bn = __shfl_down_sync(qmask, B, 2, 4);
        if (q <= 1) {
          A = fmaf(B, An, A);
          B = B * Bn;
        }
        float Ae = __shfl_down_sync(qmask, A, 1, 4), Be = __shfl_down_sync(qmask, B, 1, 4);
        if (q == 3) {
          Ae = 0.0f;
          Be = 1.0f;
        }
        const float Tadj_next = fmaf(Be, Tadj, Ae);  // adjoint of T after this lane's sample
        const float A0 = __shfl_sync(qmask, A, 0, 4), B0 = __shfl_sync(qmask, B, 0, 4);
        if (live) {
          const float dalpha = Tk * (gc - Tadj_next);
          const float ta = Tk * alpha;
          const float dc[3] = {ta * gr.x, ta * gr.y, ta * gr.z};
          // Phong backward: c = rgb (ka + kd diff) + ks spec
          const float diff = fmaxf(so.nl, 0.0f);
          const float kk = fmaf(L.r.sh.kd, diff, L.r.sh.ka);
          drgba[0] = dc[0] * kk;
          drgba[1] = dc[1] * kk;
          drgba[2] = dc[2] * kk;
          drgba[3] = dalpha;
          float dN[3] = {0.f, 0.f, 0.f};
          if (so.nl > 0.0f) {
            const float d_diff = L.r.sh.kd * (dc[0] * ts.rgba.x + dc[1] * ts.rgba.y + dc[2] * ts.rgba.z);
#pragma unroll
            for (int a = 0; a < 3; ++a) dN[a] = d_diff * so.L[a];
            if (so.rv > 0.0f && L.r.sh.shininess != 0.0f) {
              const float d_spec = L.r.sh.ks * (dc[0] + dc[1] + dc[2]);
              const float dx = d_spec * L.r.sh.shininess * __powf(so.rv, L.r.sh.shininess - 1.0f);
              const float nv = so.N[0] * so.V[0] + so.N[1] * so.V[1] + so.N[2] * so.V[2];
#pragma unroll
              for (int a = 0; a < 3; ++a) dN[a] += dx * 2.0f * (nv * so.L[a] + so.nl * so.V[a]);
            }
          }
          // normal backward: N = -g_hat / |g_hat|, then to the unscaled operator gradient
          float dg[3] = {0.f, 0.f, 0.f};
          if (so.gl * so.gl > 1e-12f && so.gl > 0.0f) {
            const float il = 1.0f / so.gl;
            const float nh[3] = {gh[0] * il, gh[1] * il, gh[2] * il};
            const float dn = dN[0] * nh[0] + dN[1] * nh[1] + dN[2] * nh[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) dg[a] = -(dN[a] - dn * nh[a]) * il * gs;
          }
          // transfer-function backward: the slope to the value here, the entries below
          float ds = 0.0f;
          if (ts.inside) {
            ds = (drgba[0] * dab.x + drgba[1] * dab.y + drgba[2] * dab.z + drgba[3] * dab.w) *
                 L.tf.scale;
          }
          contrib = L.grad_tf != nullptr;
          ci = ts.i;
          cw = ts.w;
          sv[0] = ds;
          sv[1] = dg[0];
          sv[2] = dg[1];
          sv[3] = dg[2];
          scat = L.adj && (ds != 0.0f || dg[0] != 0.0f || dg[1] != 0.0f || dg[2] != 0.0f);
        }
        // scatter (dL/dV direct, dL/dG) to the cell corners; two neighbouring samples of
        // the ray (lanes q, q ^ 1) in the same cell are scattered together by the even lane
        {
          const unsigned cb_lo = scat ? (unsigned)c.base : 0xffffffffu;
          const unsigned cb_hi = scat ? (unsigned)(c.base >> 32) : 0xffffffffu;
          const unsigned pb_lo = __shfl_xor_sync(qmask, cb_lo, 1, 4);
          const unsigned pb_hi = __shfl_xor_sync(qmask, cb_hi, 1, 4);
          const bool pscat = __shfl_xor_sync(qmask, (int)scat, 1, 4) != 0;
          float pf[3], pv[4];
#pragma unroll
          for (int a = 0; a < 3; ++a) pf[a] = __shfl_xor_sync(qmask, scat ? c.f[a] : 0.0f, 1, 4);
#pragma unroll
          for (int a = 0; a < 4; ++a) pv[a] = __shfl_xor_sync(qmask, sv[a], 1, 4);
          const bool same = scat && pscat && pb_lo == cb_lo && pb_hi == cb_hi;
          if (scat && !(same && (q & 1))) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float wci = corner_weight(c.f, i);
              float4 v = make_float4(wci * sv[0], wci * sv[1], wci * sv[2], wci * sv[3]);
              if (same) {
                const float wpi = corner_weight(pf, i);
                v.x = fmaf(wpi, pv[0], v.x);
                v.y = fmaf(wpi, pv[1], v.y);
                v.z = fmaf(wpi, pv[2], v.z);
                v.w = fmaf(wpi, pv[3], v.w);
              }
              atomicAdd(L.adj + corner_index(L.R, c.base, i), v);
            }
          }
        }
        Tcur = Tb;
        Tadj = fmaf(B0, Tadj, A0);
      }
      if (contrib) {
        if (ci != tf_run) {
          if (tf_run >= 0) {
            if (tf_row) flush_tf_row(tf_row, tf_run, tf_lo, tf_hi);
            else flush_tf(L.grad_tf, tf_run, tf_lo, tf_hi);
          }
          tf_run = ci;
#pragma unroll
          for (int j = 0; j < 4; ++j) tf_lo[j] = tf_hi[j] = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          tf_lo[j] = fmaf(1.0f - cw, drgba[j], tf_lo[j]);
          tf_hi[j] = fmaf(cw, drgba[j], tf_hi[j]);
        }
      }
    }
    if (tf_run >= 0) {
      if (tf_row) flush_tf_row(tf_row, tf_run, tf_lo, tf_hi);
      else flush_tf(L.grad_tf, tf_run, tf_lo, tf_hi);
    }
  }
}

// grad_tf[e] += sum over blocks b of partial[b][e].  A block takes 32 entries: its 8 warps
// sum the rows b = w, w + 8, ... in order (coalesced across the entries), then warp 0 adds
// the 8 partial sums in order -- the same summation order on every run.
__global__ void __launch_bounds__(256) k_tf_partial_reduce(const float* __restrict__ partial,
                                                           int blocks, int n4,
                                                           float* __restrict__ grad_tf) {
  __shared__ float part[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  float v = 0.0f;
  if (e < n4)
    for (int b = w; b < blocks; b += 8) v += partial[(size_t)b * n4 + e];
  part[w][lane] = v;
  __syncthreads();
  if (w == 0 && e < n4) {
    float sum = part[0][lane];
#pragma unroll
    for (int j = 1; j < 8; ++j) sum += part[j][lane];
    grad_tf[e] += sum;
  }
}

cudaError_t launch_tf_partial_reduce(const float* partial, int blocks, int n4, float* grad_tf,
                                     cudaStream_t s) {
  k_tf_partial_reduce<<<(n4 + 31) / 32, 256, 0, s>>>(partial, blocks, n4, grad_tf);
  return cudaGetLastError();
}

bool adjoint_tf_rows(int ntf) { return ntf <= kMaxTfRows; }

static bool tf_shared(int ntf) { return ntf <= kMaxSharedTf; }

int adjoint_grid(int ntf) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (tf_shared(ntf))
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adjoint<true>, kThreads,
                                                  (size_t)ntf * sizeof(float4));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adjoint<false>, kThreads, 0);
  return (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
}

void adjoint_add_view(AdjointLaunch& L, const CamDev& cam, const int rect[4], const int* ck_kend,
                      const float* ck_T, const float* ck_Tend, const float4* grad_rgba) {
  AdjView& v = L.view[L.nviews++];
  v.cam = cam;
  v.ck_kend = ck_kend;
  v.ck_T = ck_T;
  v.ck_Tend = ck_Tend;
  v.grad_rgba = grad_rgba;
  const int rx1 = std::min(rect[2], cam.width), ry1 = std::min(rect[3], cam.height);
  v.tx0 = rect[0] / kQuadTileW;
  v.ty0 = rect[1] / kQuadTileH;
  v.tiles_x = (rx1 + kQuadTileW - 1) / kQuadTileW - v.tx0;
  const int tiles = rx1 > rect[0] && ry1 > rect[1]
                        ? v.tiles_x * ((ry1 + kQuadTileH - 1) / kQuadTileH - v.ty0) : 0;
  v.tile0 = L.tiles_total;
  L.tiles_total += tiles;
}

cudaError_t launch_adjoint(const AdjointLaunch& L, cudaStream_t s) {
  if (L.tiles_total == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(L.tile_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (tf_shared(L.tf.n))
    k_adjoint<true><<<adjoint_grid(L.tf.n), kThreads, (size_t)L.tf.n * sizeof(float4), s>>>(L);
  else
    k_adjoint<false><<<adjoint_grid(L.tf.n), kThreads, 0, s>>>(L);
  return cudaGetLastError();
}

// ------------------------------------------------------- transposed operator stencil
// G_a(j) = sum_o W^a_o E(j + o) over the integer grid j in [0, n-1]^3, E(m) = V(clamp(m)).
// Hence dL/dV(v) = adj(v).x + sum over m with clamp(m) = v, over the taps o of every
// component a, of W^a_o * adj(m - o).(1 + a) for m - o inside the grid.
template <int OP>
__device__ __forceinline__ float tap_weight(int along, int b, int c) {
  // weight of the tap (+1 along the component axis, b, c on the two others)
  if constexpr (OP == OP_CENTRAL) {
    return (b == 0 && c == 0) ? 1.0f : 0.0f;
  } else if constexpr (OP == OP_SOBEL) {
    const float wb = b == 0 ? 2.0f : 1.0f, wc = c == 0 ? 2.0f : 1.0f;
    // [[1,3,1],[3,6,3],[1,3,1]]
    return (b == 0 && c == 0) ? 6.0f : (wb * wc == 2.0f ? 3.0f : 1.0f);
  } else {
    const int r2 = b * b + c * c;
    return r2 == 0 ? 1.0f : (r2 == 1 ? 0.70710678118654752f : 0.57735026918962576f);
  }
  (void)along;
}

// acc += the transposed taps that reach m's operator from the grid points j = m - o (CHECK:
// skip j outside the grid; without it every j must lie inside).
template <int OP, bool CHECK>
__device__ __forceinline__ float add_transposed_taps(const float4* __restrict__ adj, const int m[3],
                                                     int nx, int ny, int nz, float acc) {
#pragma unroll
  for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        // signed weights of the three components' taps at offset (ox, oy, oz): the x
        // component's tap has ox = +-1 and (b, c) = (oy, oz), and so on; offsets where all
        // three vanish (every one but the six axis neighbours for central differences) are
        // dropped when the loops unroll
        const float wx = ox != 0 ? (float)ox * tap_weight<OP>(0, oy, oz) : 0.0f;
        const float wy = oy != 0 ? (float)oy * tap_weight<OP>(1, oz, ox) : 0.0f;
        const float wz = oz != 0 ? (float)oz * tap_weight<OP>(2, ox, oy) : 0.0f;
        if (wx == 0.0f && wy == 0.0f && wz == 0.0f) continue;
        const int j[3] = {m[0] - ox, m[1] - oy, m[2] - oz};
        if (CHECK && (j[0] < 0 || j[0] >= nx || j[1] < 0 || j[1] >= ny || j[2] < 0 || j[2] >= nz))
          continue;
        const float4 aj = __ldg(adj + (j[0] + nx * (j[1] + ny * j[2])));
        if (wx != 0.0f) acc += wx * aj.y;
        if (wy != 0.0f) acc += wy * aj.z;
        if (wz != 0.0f) acc += wz * aj.w;
      }
  return acc;
}

template <int OP>
__global__ void __launch_bounds__(256) k_adjoint_volume(const float4* __restrict__ adj, int nx,
                                                        int ny, int nz, float* __restrict__ gvol) {
  // the grid holds fewer than 2^31 voxels (checked at upload)
  const int nvox = nx * ny * nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const int v[3] = {i % nx, (i / nx) % ny, i / (nx * ny)};
  float acc = __ldg(&adj[i].x);
  if (v[0] > 0 && v[0] < nx - 1 && v[1] > 0 && v[1] < ny - 1 && v[2] > 0 && v[2] < nz - 1) {
    // inside: only m = v clamps onto v, and all of its taps' grid points exist
    gvol[i] += add_transposed_taps<OP, false>(adj, v, nx, ny, nz, acc);
    return;
  }
  // candidate m per axis: v itself (bit 0), and the border cells that clamp onto v: -1 when
  // v = 0 (bit 1), n when v = n - 1 (bit 2)
  const unsigned mkx = 1u | (v[0] == 0 ? 2u : 0u) | (v[0] == nx - 1 ? 4u : 0u);
  const unsigned mky = 1u | (v[1] == 0 ? 2u : 0u) | (v[1] == ny - 1 ? 4u : 0u);
  const unsigned mkz = 1u | (v[2] == 0 ? 2u : 0u) | (v[2] == nz - 1 ? 4u : 0u);
#pragma unroll 1
  for (int iz = 0; iz < 3; ++iz)
#pragma unroll 1
    for (int iy = 0; iy < 3; ++iy)
#pragma unroll 1
      for (int ix = 0; ix < 3; ++ix) {
        if (!((mkx >> ix) & (mky >> iy) & (mkz >> iz) & 1u)) continue;
        const int m[3] = {v[0] + (ix == 0 ? 0 : (ix == 1 ? -1 : 1)),
                          v[1] + (iy == 0 ? 0 : (iy == 1 ? -1 : 1)),
                          v[2] + (iz == 0 ? 0 : (iz == 1 ? -1 : 1))};
        acc = add_transposed_taps<OP, true>(adj, m, nx, ny, nz, acc);
      }
  gvol[i] += acc;
}

cudaError_t launch_adjoint_volume(const float4* adj, const int n[3], int op, float inv_vmax,
                                  float* grad_volume, cudaStream_t s) {
  (void)inv_vmax;
  const long nvox = (long)n[0] * n[1] * n[2];
  const int threads = 256;
  const int blocks = (int)((nvox + threads - 1) / threads);
  switch (op) {
    case OP_CENTRAL: k_adjoint_volume<OP_CENTRAL><<<blocks, threads, 0, s>>>(adj, n[0], n[1], n[2], grad_volume); break;
    case OP_SOBEL: k_adjoint_volume<OP_SOBEL><<<blocks, threads, 0, s>>>(adj, n[0], n[1], n[2], grad_volume); break;
    default: k_adjoint_volume<OP_ZH><<<blocks, threads, 0, s>>>(adj, n[0], n[1], n[2], grad_volume);
  }
  return cudaGetLastError();
}

}  // namespace vr
