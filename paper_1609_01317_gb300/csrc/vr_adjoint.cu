// vr_adjoint.cu -- reverse-mode differentiation of the ray march.
//
// The forward pass (vr_render_forward_train) stores, per ray, the index of the last
// sample it composited and the transmittance T before every 32nd sample.  The adjoint
// walks each ray back to front one 32-sample segment at a time: it recomputes the
// segment's transmittances from the stored T (cheap: value + transfer function only),
// then visits the samples in reverse order, recomputing each sample in full (value,
// gradient, normal, Phong) and applying the chain rule of Eq. 6 (§3.9):
//   C = sum_k T_k a_k c_k,  T_{k+1} = T_k (1 - a_k),  A = 1 - T_end
//   dL/da_k = T_k (g.c_k - Tadj_{k+1}),  dL/dc_k = T_k a_k g,
//   Tadj_k  = a_k g.c_k + (1 - a_k) Tadj_{k+1},  Tadj_end = -dL/dA,
// with g = dL/dRGB.  Gradients flow through Phong (§3.8), the normalisation of the
// operator gradient, the transfer-function interpolation (§3.7) and the trilinear blend
// (§3.4).  Because the operator gradient at p is the trilinear blend of the integer-grid
// operator G at the cell corners, the kernel scatters (dL/ds, dL/dG) to the 8 corners
// with one vector atomic each; a second, dense pass applies the transposed operator
// stencil (with the clamp-to-edge folding) to turn dL/dG into dL/dV.
#include "vr_internal.h"

namespace vr {

constexpr int kTileW = 16, kTileH = 8, kThreads = 128;
constexpr int kMaxSharedTf = 1024;  // tables up to this size accumulate in shared memory

template <int VTYPE>
__device__ __forceinline__ float alpha_at(const VolDev& V, const TfDev& tf, const float o[3],
                                          const float d[3], float tn, float step, int k) {
  const float t = fmaf((float)k + 0.5f, step, tn);
  float p[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
  const Cell c = cell_of(V, p);
  return tf_lookup(tf, trilinear<VTYPE>(V, c)).rgba.w;
}

template <int VTYPE, int OP>
__global__ void __launch_bounds__(kThreads) k_adjoint(const AdjointLaunch L) {
  extern __shared__ float smem[];
  float* Ts = smem;                               // [kCkptStride][kThreads]
  float* hist = smem + kCkptStride * kThreads;    // [ntf][4] when shared
  const bool shared_tf = L.grad_tf && L.tf.n <= kMaxSharedTf;
  const int tid = threadIdx.x;
  if (shared_tf)
    for (int i = tid; i < 4 * L.tf.n; i += kThreads) hist[i] = 0.0f;
  __syncthreads();

  const int lane = tid & 31, w = tid >> 5;
  const int px = blockIdx.x * kTileW + (w & 1) * 8 + (lane & 7);
  const int py = blockIdx.y * kTileH + (w >> 1) * 4 + (lane >> 3);
  const int W = L.cam.width, H = L.cam.height;
  const bool active = px < W && py < H;
  const int ray = py * W + px;
  const int nrays = W * H;
  float o[3], d[3], tn = 0.0f;
  int K = 0, kend = 0;
  if (active) {
    ray_setup(L.cam, L.r.lo, L.r.hi, L.r.step, px, py, o, d, tn, K);
    kend = min(max(L.ck_kend[ray], 0), K);
  }
  float4 gr = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active && kend > 0) gr = __ldg(L.grad_rgba + ray);
  const float step = L.r.step;
  float Tadj = -gr.w;
  const auto* vox = static_cast<const typename VoxelT<VTYPE>::T*>(L.V.data);
  (void)vox;
  const int nseg = (kend + kCkptStride - 1) / kCkptStride;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * kCkptStride;
    const int k1 = min(k0 + kCkptStride, kend);
    float T = seg == 0 ? 1.0f : L.ck_T[(size_t)(seg - 1) * nrays + ray];
    for (int k = k0; k < k1; ++k) {
      Ts[(k - k0) * kThreads + tid] = T;
      const float a = alpha_at<VTYPE>(L.V, L.tf, o, d, tn, step, k);
      if (a != 0.0f) T = T * (1.0f - a);
    }
    for (int k = k1 - 1; k >= k0; --k) {
      const float Tk = Ts[(k - k0) * kThreads + tid];
      const float t = fmaf((float)k + 0.5f, step, tn);
      float p[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
      const Cell c = cell_of(L.V, p);
      float s, g[3];
      value_and_gradient<VTYPE, OP>(L.V, c, s, g);
      const TfSample ts = tf_lookup(L.tf, trilinear<VTYPE>(L.V, c));
      const float gs = L.r.gscale;
      const float gh[3] = {g[0] * gs, g[1] * gs, g[2] * gs};
      ShadeOut so;
      shade(L.r.sh, L.cam, d, p, gh, ts.rgba, so);
      const float alpha = ts.rgba.w;
      const float gc = gr.x * so.c[0] + gr.y * so.c[1] + gr.z * so.c[2];
      const float dalpha = Tk * (gc - Tadj);
      const float ta = Tk * alpha;
      const float dc[3] = {ta * gr.x, ta * gr.y, ta * gr.z};
      Tadj = fmaf(alpha, gc, (1.0f - alpha) * Tadj);
      // Phong backward: c = rgb (ka + kd diff) + ks spec
      const float diff = fmaxf(so.nl, 0.0f);
      const float kk = fmaf(L.r.sh.kd, diff, L.r.sh.ka);
      float drgba[4] = {dc[0] * kk, dc[1] * kk, dc[2] * kk, dalpha};
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
      // normal backward: N = -g_hat / |g_hat|
      float dg[3] = {0.f, 0.f, 0.f};
      if (so.gl * so.gl > 1e-12f && so.gl > 0.0f) {
        const float il = 1.0f / so.gl;
        const float nh[3] = {gh[0] * il, gh[1] * il, gh[2] * il};
        const float dn = dN[0] * nh[0] + dN[1] * nh[1] + dN[2] * nh[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) dg[a] = -(dN[a] - dn * nh[a]) * il * gs;  // -> raw units
      }
      // transfer-function backward
      float ds = 0.0f;
      if (L.grad_tf || L.adj) {
        const int i = ts.i;
        const float wt = ts.w;
        if (ts.inside) {
          const float4 ta4 = __ldg(L.tf.tf + i), tb4 = __ldg(L.tf.tf + i + 1);
          ds = (drgba[0] * (tb4.x - ta4.x) + drgba[1] * (tb4.y - ta4.y) +
                drgba[2] * (tb4.z - ta4.z) + drgba[3] * (tb4.w - ta4.w)) * L.tf.scale;
        }
        if (L.grad_tf) {
          float* dst = shared_tf ? hist : L.grad_tf;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float v0 = (1.0f - wt) * drgba[q], v1 = wt * drgba[q];
            if (v0 != 0.0f) atomicAdd(dst + 4 * i + q, v0);
            if (v1 != 0.0f) atomicAdd(dst + 4 * (i + 1) + q, v1);
          }
        }
      }
      // scatter (dL/ds, dL/dG) to the cell corners
      if (L.adj && (ds != 0.0f || dg[0] != 0.0f || dg[1] != 0.0f || dg[2] != 0.0f)) {
        const int nx = L.V.n[0], ny = L.V.n[1], nz = L.V.n[2];
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const float wx = (cc & 1) ? c.f[0] : 1.0f - c.f[0];
          const float wy = (cc & 2) ? c.f[1] : 1.0f - c.f[1];
          const float wz = (cc & 4) ? c.f[2] : 1.0f - c.f[2];
          const float wc = wx * wy * wz;
          const int x = min(c.ib[0] + (cc & 1), nx - 1);
          const int y = min(c.ib[1] + ((cc >> 1) & 1), ny - 1);
          const int z = min(c.ib[2] + ((cc >> 2) & 1), nz - 1);
          atomicAdd(L.adj + ((size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z)),
                    make_float4(wc * ds, wc * dg[0], wc * dg[1], wc * dg[2]));
        }
      }
    }
  }
  if (shared_tf) {
    __syncthreads();
    for (int i = tid; i < 4 * L.tf.n; i += kThreads) {
      const float v = hist[i];
      if (v != 0.0f) atomicAdd(L.grad_tf + i, v);
    }
  }
}

template <int VTYPE, int OP>
static void launch_adj_typed(const AdjointLaunch& L, dim3 grid, size_t smem, cudaStream_t s) {
  k_adjoint<VTYPE, OP><<<grid, kThreads, smem, s>>>(L);
}

template <int VTYPE>
static void launch_adj_op(const AdjointLaunch& L, dim3 grid, size_t smem, cudaStream_t s) {
  switch (L.op) {
    case OP_CENTRAL: launch_adj_typed<VTYPE, OP_CENTRAL>(L, grid, smem, s); break;
    case OP_SOBEL: launch_adj_typed<VTYPE, OP_SOBEL>(L, grid, smem, s); break;
    default: launch_adj_typed<VTYPE, OP_ZH>(L, grid, smem, s);
  }
}

cudaError_t launch_adjoint(const AdjointLaunch& L, cudaStream_t s) {
  const dim3 grid((L.cam.width + kTileW - 1) / kTileW, (L.cam.height + kTileH - 1) / kTileH);
  size_t smem = sizeof(float) * kCkptStride * kThreads;
  if (L.grad_tf && L.tf.n <= kMaxSharedTf) smem += sizeof(float) * 4 * L.tf.n;
  switch (L.dtype) {
    case VT_U8: launch_adj_op<VT_U8>(L, grid, smem, s); break;
    case VT_U16: launch_adj_op<VT_U16>(L, grid, smem, s); break;
    case VT_F16: launch_adj_op<VT_F16>(L, grid, smem, s); break;
    default: launch_adj_op<VT_F32>(L, grid, smem, s);
  }
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

template <int OP>
__global__ void k_adjoint_volume(const float4* __restrict__ adj, int nx, int ny, int nz,
                                 float* __restrict__ gvol) {
  const long nvox = (long)nx * ny * nz;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nvox) return;
  const int v[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / ((long)nx * ny))};
  const int n[3] = {nx, ny, nz};
  float acc = __ldg(&adj[i].x);
  // candidate m per axis: v itself, and the border cells that clamp onto v
  int mlist[3][3], mcnt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mcnt[a] = 0;
    mlist[a][mcnt[a]++] = v[a];
    if (v[a] == 0) mlist[a][mcnt[a]++] = -1;
    if (v[a] == n[a] - 1) mlist[a][mcnt[a]++] = n[a];
  }
  for (int iz = 0; iz < mcnt[2]; ++iz)
    for (int iy = 0; iy < mcnt[1]; ++iy)
      for (int ix = 0; ix < mcnt[0]; ++ix) {
        const int m[3] = {mlist[0][ix], mlist[1][iy], mlist[2][iz]};
#pragma unroll
        for (int oz = -1; oz <= 1; ++oz)
#pragma unroll
          for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
              if (ox == 0 && oy == 0 && oz == 0) continue;
              const int j[3] = {m[0] - ox, m[1] - oy, m[2] - oz};
              if (j[0] < 0 || j[0] >= nx || j[1] < 0 || j[1] >= ny || j[2] < 0 || j[2] >= nz)
                continue;
              const float4 aj = __ldg(adj + ((long)j[0] + (long)nx * ((long)j[1] + (long)ny * j[2])));
              // x component: tap offset (ox, oy, oz) with ox = +-1, (b, c) = (oy, oz)
              if (ox != 0) acc += (float)ox * tap_weight<OP>(0, oy, oz) * aj.y;
              if (oy != 0) acc += (float)oy * tap_weight<OP>(1, oz, ox) * aj.z;
              if (oz != 0) acc += (float)oz * tap_weight<OP>(2, ox, oy) * aj.w;
            }
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
