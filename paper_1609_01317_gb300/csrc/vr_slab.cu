// vr_slab.cu -- the plain march with the bricks each ray tile crosses staged in shared memory
// (VR_MARCH_SLABS; the record march stays the default, being faster on every workload
// measured).
//
// A block of 256 threads marches a 16 x 16 pixel tile of the box's screen rectangle, one ray
// per thread.  The rays of a tile are nearly parallel, so they advance together along the
// axis a on which every one of them moves fastest (all with the same sign): the block walks
// the volume front to back in slabs along a -- 2^Ds cells of a fixed grid (Ds set per launch
// from how far apart the rays are), or the single next cell where the coarse slab's region
// would not fit in shared memory.  Per slab:
//   0. each ray first jumps over transparent bricks, macro bricks and super bricks on its own
//      (§5.3, §5.4; the samples passed over have zero opacity);
//   1. one block reduction of packed keys finds the nearest slab any ray is still in and the
//      cell range the rays' samples cover there (per ray: its next sample and one past its
//      analytic exit of the slab, one cell of margin), for both slab sizes at once;
//   2. the bricks of that region are looked up: when none is visible, the rays only step
//      their sample index through the slab;
//   3. otherwise the clamp-to-edge raw voxels of the region plus one voxel around it are
//      staged in shared memory (every thread issuing several loads before storing them), and
//      the gradient record of every voxel of the region -- the operator gradient G and the
//      value, §3.5 -- is computed there with the records pass's arithmetic (vr_records.cuh);
//   4. every ray marches its samples in the slab exactly as the tile march does: the sample
//      at t_k = t_near + (k + 1/2) step, skipped when its brick is transparent, else the 8
//      corner records of its cell (now from shared memory), trilinear value (§3.4),
//      transfer function (§3.7), gradient blend and Phong (§3.8) when alpha != 0, and the
//      compositing of Eq. 6 with the same four partial colours (sample k adds to partial
//      k mod 4, summed (C_0 + C_1) + (C_2 + C_3) at the end) and the same termination rule,
//      so the image equals the tile march's bit for bit.
// No global record table is read or written: the volume is read once per slab region, and
// the per-frame records pass is not needed.  A sample whose cell falls outside the staged
// region (a region too large for shared memory, or rays of mixed direction) reads its corner
// records from the padded volume directly (slow, same bits).
#include <algorithm>
#include <cmath>

#include "vr_march.cuh"
#include "vr_records.cuh"

namespace vr {

constexpr int kSlabThreads = 256;
constexpr int kSlabTileW = 16, kSlabTileH = 16;  // one ray per thread
constexpr int kSlabMaxRec = 2944;   // records staged per slab (float4)
constexpr int kSlabMaxRaw = 4800;   // raw voxels staged per slab (float)
constexpr int kSlabMaxBricks = 128; // brick flags of a region
constexpr int kSlabMaxTf = 1024;    // the transfer function is copied to shared memory
constexpr int kKeyMax = 0x7fffffff;

struct SlabSmem {
  float4 rec[kSlabMaxRec];
  float raw[kSlabMaxRaw];
  unsigned char bvis[kSlabMaxBricks];
  int red[2][8];   // packed-key reductions, double-buffered across slabs
  int ax[6];       // per axis: min |d| (float bits), sign flags
  int tile;
};

// The record of voxel (x, y, z) straight from the padded volume, from its 3x3x3
// clamp-to-edge neighbourhood, assembled as the records pass does.
template <int VTYPE, int OP>
__device__ __forceinline__ float4 record_from_volume(const VolDev& V, int x, int y, int z) {
  using Vox = typename VoxelT<VTYPE>::T;
  const Vox* vol = static_cast<const Vox*>(V.data);
  PlaneSums ps[3];
#pragma unroll
  for (int dz = 0; dz < 3; ++dz) {
    float p[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long e = (long long)(x - 1 + a + kPadLo) + (long long)V.px * (y - 1 + b + kPadLo) +
                            (long long)V.pxy * (z - 1 + dz + kPadLo);
        p[b][a] = raw_to_float<VTYPE>(vol[VR_CHECK(V.bounds, e, 0, padded_elems(V) - 1)]);
      }
    ps[dz] = plane_sums_of<OP>(p);
  }
  return record_of<OP>(ps[0], ps[1], ps[2]);
}

template <typename V>
__device__ __forceinline__ V pick3(const V v[3], int a) {
  return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]);
}

__device__ __forceinline__ int clamp_cell(float v, int top) {
  const int i = (int)floorf(v);
  return i < 0 ? 0 : (i > top ? top : i);
}

// Block-wide minimum of eight packed keys (warp minimum, then shared atomics).
__device__ __forceinline__ void block_min8(int* red, const int v[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = __reduce_min_sync(0xffffffffu, v[i]);
    if ((threadIdx.x & 31) == 0 && m != kKeyMax) atomicMin(red + i, m);
  }
}

// Alpha and shaded colour (alpha, r, g, b) of the sample at p in cell c with corner
// records cr: trilinear value (§3.4), transfer function (§3.7), and when alpha != 0 the
// blended operator gradient and Phong (§3.8) -- the tile march's arithmetic.
__device__ __forceinline__ float4 sample_colour(const MarchLaunch& L, const float4* s_tf,
                                                const Corners& cr, const Cell& c,
                                                const float p[3], const float d[3]) {
  const float4 bl = corners_blend(cr, c);
  const TfSample ts = tf_lookup<true>(L.tf, bl.w, s_tf);
  float4 out = make_float4(ts.rgba.w, 0.0f, 0.0f, 0.0f);
  if (ts.rgba.w != 0.0f) {
    const float gh[3] = {bl.x * L.r.gscale, bl.y * L.r.gscale, bl.z * L.r.gscale};
    ShadeOut so;
    shade(L.r.sh, L.cam, d, p, gh, ts.rgba, so);
    out.y = so.c[0];
    out.z = so.c[1];
    out.w = so.c[2];
  }
  return out;
}

template <int VTYPE, int OP>
__global__ void __launch_bounds__(kSlabThreads, 3) k_march_slab(const __grid_constant__ MarchLaunch L, int Ds) {
  using Vox = typename VoxelT<VTYPE>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s_tf = reinterpret_cast<float4*>(smem_raw);
  SlabSmem& S = *reinterpret_cast<SlabSmem*>(smem_raw + sizeof(float4) * L.tf.n);
  const int tid = threadIdx.x;
  for (int i = tid; i < L.tf.n; i += kSlabThreads) s_tf[i] = L.tf.tf[i];
  if (L.hint && L.vis_count && blockIdx.x == 0 && tid == 0) {
    // the visible-brick count, for the host's choice of march for the next render
    L.hint[0] = __ldg(L.vis_count);
    L.hint[1] = L.V.nb[0] * L.V.nb[1] * L.V.nb[2];
  }
  const int W = L.cam.width;
  const int n0 = L.V.n[0], n1 = L.V.n[1], n2 = L.V.n[2];
  const int top[3] = {n0 > 1 ? n0 - 2 : 0, n1 > 1 ? n1 - 2 : 0, n2 > 1 ? n2 - 2 : 0};
  const int tx0 = L.rect[0] / kSlabTileW, ty0 = L.rect[1] / kSlabTileH;
  const int tiles_x = (L.rect[2] + kSlabTileW - 1) / kSlabTileW - tx0;
  const int tiles = tiles_x * ((L.rect[3] + kSlabTileH - 1) / kSlabTileH - ty0);
  const float step = L.r.step;
  unsigned hit = 0, plain = 0, visited = 0, shaded = 0;
  for (;;) {
    __syncthreads();  // every thread is done with the previous tile's shared state
    if (tid == 0) S.tile = (int)atomicAdd(L.tile_counter, 1u);
    if (tid < 3) S.ax[tid] = kKeyMax;
    if (tid >= 3 && tid < 6) S.ax[tid] = 0;
    if (tid < 16) (&S.red[0][0])[tid] = kKeyMax;
    __syncthreads();
    const int tile = S.tile;
    if (tile >= tiles) break;
    const int px = (tx0 + tile % tiles_x) * kSlabTileW + (tid % kSlabTileW);
    const int py = (ty0 + tile / tiles_x) * kSlabTileH + (tid / kSlabTileW);
    const bool active = px < W && px >= L.rect[0] && px < L.rect[2] && py >= L.rect[1] &&
                        py < L.rect[3];
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f}, tn = 0.0f;
    int K = 0;
    if (active) ray_setup(L.cam, L.r.lo, L.r.hi, step, px, py, o, d, tn, K);
    // slab axis: the largest smallest |d_a| over the tile's rays among the axes along which
    // no two rays move in opposite directions
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int m = __reduce_min_sync(0xffffffffu, K > 0 ? __float_as_int(fabsf(d[a])) : kKeyMax);
      const unsigned sg = __reduce_or_sync(0xffffffffu, K > 0 ? (d[a] > 0.0f ? 1u : (d[a] < 0.0f ? 2u : 3u)) : 0u);
      if ((tid & 31) == 0) {
        if (m != kKeyMax) atomicMin(&S.ax[a], m);
        if (sg) atomicOr(&S.ax[3 + a], (int)sg);
      }
    }
    __syncthreads();
    int ax = -1;
    float best = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int sg = S.ax[3 + a];
      const float m = S.ax[a] == kKeyMax ? 0.0f : __int_as_float(S.ax[a]);
      if ((sg == 1 || sg == 2) && m > best) {
        best = m;
        ax = a;
      }
    }
    const bool fwd = ax >= 0 && S.ax[3 + ax] == 1;  // cells along the axis increase
    // per-axis values of the slab axis a and the two others (b, c), picked without indexing
    // register arrays by a run-time axis
    const int bax = ax == 0 ? 1 : 0, cax = ax == 2 ? 1 : 2;
    const int na = pick3(top, ax), nb_ = pick3(top, bax), nc_ = pick3(top, cax);
    const float oa = pick3(o, ax), ob = pick3(o, bax), oc = pick3(o, cax);
    const float da = pick3(d, ax), db = pick3(d, bax), dc = pick3(d, cax);
    const float inv_da = (ax >= 0 && K > 0) ? 1.0f / da : 0.0f;
    const float inv_step = 1.0f / step;

    float T = 1.0f;
    float C[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) C[j][0] = C[j][1] = C[j][2] = 0.0f;
    int k = 0;
    bool live = K > 0;
    int buf = 0;
    for (;;) {
      // --- 0. each ray leaves transparent space on its own (§5.3, §5.4): past a transparent
      // brick, or the transparent macro or super brick around it, with the tile march's
      // exit rule.  Every sample passed over has zero opacity, so it would change neither T
      // nor a partial colour.
      if (live && L.r.skip) {
        float inv_d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) inv_d[a] = d[a] != 0.0f ? 1.0f / d[a] : 0.0f;
        while (k < K) {
          const float t = fmaf((float)k + 0.5f, step, tn);
          float p[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
          int b[3];
          const int bi = brick_of(L.V, p, b);
          if (__ldg(L.V.vis + VR_CHECK(L.V.bounds, bi, 0, L.V.nb[0] * L.V.nb[1] * L.V.nb[2] - 1)))
            break;
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
          const int kn = region_exit_sample(b, shift, o, d, inv_d, tn, inv_step);
          k = kn > k ? kn : k + 1;
        }
        if (k >= K) live = false;
      }
      // --- 1. the next slab and the cells its rays' samples cover, for the coarse slab
      // (2^Ds cells of the fixed grid along the axis) and for the single next cell; the
      // keys pack the slab (nearest first) above a cell bound, so one minimum gives both
      int key[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) key[i] = kKeyMax;
      int ca = 0;
      if (live && ax >= 0) {
        const float t = fmaf((float)k + 0.5f, step, tn);
        ca = clamp_cell(fmaf(t, da, oa), na);
        const int pb = clamp_cell(fmaf(t, db, ob), nb_), pc = clamp_cell(fmaf(t, dc, oc), nc_);
#pragma unroll
        for (int lvl = 0; lvl < 2; ++lvl) {
          const int shl = lvl == 0 ? Ds : 0;
          const int js = ca >> shl;
          // one sample past the slab's analytic exit (or the ray's last sample)
          const int edge = fwd ? (js + 1) << shl : js << shl;
          int kl = K - 1;
          if (fwd ? edge <= na : edge > 0) {
            const float te = ((float)edge - oa) * inv_da;
            const float kf = ceilf(fmaf(te - tn, inv_step, -0.5f));
            if (kf < (float)(K - 1)) kl = kf < (float)k ? k : (int)kf;
            kl = min(kl + 1, K - 1);
          }
          const float tl = fmaf((float)kl + 0.5f, step, tn);
          const int lb = clamp_cell(fmaf(tl, db, ob), nb_), lc = clamp_cell(fmaf(tl, dc, oc), nc_);
          const int jkey = (fwd ? js : (0x7ffe - js)) << 16;
          key[4 * lvl + 0] = jkey | max(min(pb, lb) - 1, 0);
          key[4 * lvl + 1] = jkey | (0xffff - min(max(pb, lb) + 1, nb_));
          key[4 * lvl + 2] = jkey | max(min(pc, lc) - 1, 0);
          key[4 * lvl + 3] = jkey | (0xffff - min(max(pc, lc) + 1, nc_));
        }
      } else if (live) {
        key[0] = 0;  // mixed directions: no slabs, every sample reads the volume
      }
      block_min8(S.red[buf], key);
      __syncthreads();
      int red[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) red[i] = S.red[buf][i];
      if (tid < 8) S.red[buf ^ 1][tid] = kKeyMax;  // for the next slab (read after a barrier)
      buf ^= 1;
      if (red[0] == kKeyMax) break;  // every ray of the tile has ended
      // region of the slab: cells lo..hi per axis, records of voxels lo..hi+1; the coarse
      // slab when its records fit in shared memory, else the next cell alone (then staged
      // only if that fits)
      int la = 0, ha = -1, lb = 0, hb = -1, lc = 0, hc = -1;
      int jslab = -1, sh = 0;
      bool staged = false;
      if (ax >= 0) {
#pragma unroll
        for (int lvl = 0; lvl < 2; ++lvl) {
          const int shl = lvl == 0 ? Ds : 0;
          const int jkey = red[4 * lvl] >> 16;
          const int js = fwd ? jkey : 0x7ffe - jkey;
          const int l0 = js << shl, h0 = min(((js + 1) << shl) - 1, na);
          const int l1 = red[4 * lvl] & 0xffff, h1 = 0xffff - (red[4 * lvl + 1] & 0xffff);
          const int l2 = red[4 * lvl + 2] & 0xffff, h2 = 0xffff - (red[4 * lvl + 3] & 0xffff);
          const int nr = (h0 - l0 + 2) * (h1 - l1 + 2) * (h2 - l2 + 2);
          const int nw = (h0 - l0 + 4) * (h1 - l1 + 4) * (h2 - l2 + 4);
          const bool fits = nr <= kSlabMaxRec && nw <= kSlabMaxRaw;
          if (jslab < 0 && (fits || lvl == 1)) {
            staged = fits;
            jslab = js;
            sh = shl;
            la = l0; ha = h0; lb = l1; hb = h1; lc = l2; hc = h2;
          }
        }
      }
      int lo[3], hi[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        lo[a] = a == ax ? la : (a == bax ? lb : lc);
        hi[a] = a == ax ? ha : (a == bax ? hb : hc);
      }
      // --- 2. bricks of the region (§5.3)
      int bl[3], bn[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        bl[a] = min(lo[a] >> kBrickShift, L.V.nb[a] - 1);
        bn[a] = min((hi[a] + 1) >> kBrickShift, L.V.nb[a] - 1) - bl[a] + 1;
      }
      const bool flags = staged && bn[0] * bn[1] * bn[2] <= kSlabMaxBricks;
      bool any = true;
      if (staged && L.r.skip) {
        int v = 0;
        if (flags && tid < bn[0] * bn[1] * bn[2]) {
          const int bx = bl[0] + tid % bn[0], by = bl[1] + (tid / bn[0]) % bn[1],
                    bz = bl[2] + tid / (bn[0] * bn[1]);
          v = __ldg(L.V.vis + VR_CHECK(L.V.bounds, bx + L.V.nb[0] * (by + L.V.nb[1] * bz), 0,
                                       L.V.nb[0] * L.V.nb[1] * L.V.nb[2] - 1));
          S.bvis[tid] = (unsigned char)v;
        }
        any = __syncthreads_or(v) != 0 || !flags;
      }
      // --- 3. stage the raw region and compute its records
      const int rx = hi[0] - lo[0] + 2, ry = hi[1] - lo[1] + 2, rz = hi[2] - lo[2] + 2;
      if (staged && any) {
        const int qx = rx + 2, qy = ry + 2, qz = rz + 2;
        const Vox* vol = static_cast<const Vox*>(L.V.data);
        // every thread issues up to four loads before storing them (latency)
        const int nw = qx * qy * qz, qxy = qx * qy;
        const long long base = (long long)(lo[0] - 1 + kPadLo) + (long long)L.V.px * (lo[1] - 1 + kPadLo) +
                               (long long)L.V.pxy * (lo[2] - 1 + kPadLo);
        for (int i0 = tid; i0 < nw; i0 += 4 * kSlabThreads) {
          Vox v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int i = i0 + j * kSlabThreads;
            if (i < nw) {
              const int z = i / qxy, r = i - z * qxy, y = r / qx, x = r - y * qx;
              v[j] = vol[VR_CHECK(L.V.bounds, base + x + (long long)L.V.px * y + (long long)L.V.pxy * z,
                                  0, padded_elems(L.V) - 1)];
            }
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int i = i0 + j * kSlabThreads;
            if (i < nw) S.raw[i] = raw_to_float<VTYPE>(v[j]);
          }
        }
        __syncthreads();
        const int nrec = rx * ry * rz;
        for (int i = tid; i < nrec; i += kSlabThreads) {
          const int x = i % rx, y = (i / rx) % ry, z = i / (rx * ry);
          const float* pl = S.raw + (z * qy + y) * qx + x;  // raw (x-1, y-1, z-1)
          const PlaneSums s0 = plane_sums_at<OP>(pl, qx, 0, 0);
          const PlaneSums s1 = plane_sums_at<OP>(pl + qx * qy, qx, 0, 0);
          const PlaneSums s2 = plane_sums_at<OP>(pl + 2 * qx * qy, qx, 0, 0);
          S.rec[i] = record_of<OP>(s0, s1, s2);
        }
        __syncthreads();
      }
      // --- 4. the rays' samples in the slab
      if (live && (ax < 0 || (ca >> sh) == jslab)) {
        while (k < K) {
          const float t = fmaf((float)k + 0.5f, step, tn);
          float p[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) p[a] = fmaf(t, d[a], o[a]);
          const Cell c = cell_of(L.V, p);
          if (ax >= 0 && (pick3(c.ib, ax) >> sh) != jslab) break;  // past the slab
          bool vis = any;
          if (vis && L.r.skip) {
            int bb[3];
            const int bi = brick_of(L.V, p, bb);
            const int lx = bb[0] - bl[0], ly = bb[1] - bl[1], lz = bb[2] - bl[2];
            if (flags && lx >= 0 && lx < bn[0] && ly >= 0 && ly < bn[1] && lz >= 0 && lz < bn[2])
              vis = S.bvis[lx + bn[0] * (ly + bn[1] * lz)] != 0;
            else
              vis = __ldg(L.V.vis + VR_CHECK(L.V.bounds, bi, 0,
                                             L.V.nb[0] * L.V.nb[1] * L.V.nb[2] - 1)) != 0;
          }
          float alpha = 0.0f, c0 = 0.0f, c1 = 0.0f, c2 = 0.0f;
          if (vis) {
            ++visited;
            const int lx = c.ib[0] - lo[0], ly = c.ib[1] - lo[1], lz = c.ib[2] - lo[2];
            float4 ac;
            if (staged && lx >= 0 && lx <= hi[0] - lo[0] && ly >= 0 && ly <= hi[1] - lo[1] &&
                lz >= 0 && lz <= hi[2] - lo[2]) {
              const float4* r = S.rec + lx + rx * (ly + ry * lz);
              const int sy = rx, sz = rx * ry;
              Corners cr;
              cr.r[0] = r[0];
              cr.r[1] = r[1];
              cr.r[2] = r[sy];
              cr.r[3] = r[sy + 1];
              cr.r[4] = r[sz];
              cr.r[5] = r[sz + 1];
              cr.r[6] = r[sz + sy];
              cr.r[7] = r[sz + sy + 1];
              ac = sample_colour(L, s_tf, cr, c, p, d);
            } else {
              // outside the staged region: the corner records from the padded volume (slow;
              // the same bits)
              Corners cv;
#pragma unroll 1
              for (int i = 0; i < 8; ++i)
                cv.r[i] = record_from_volume<VTYPE, OP>(L.V, c.ib[0] + (i & 1),
                                                        c.ib[1] + ((i >> 1) & 1),
                                                        c.ib[2] + ((i >> 2) & 1));
              ac = sample_colour(L, s_tf, cv, c, p, d);
            }
            alpha = ac.x;
            c0 = ac.y;
            c1 = ac.z;
            c2 = ac.w;
            if (alpha != 0.0f) ++shaded;
          }
          // Eq. 6, as the tile march composites: T in sample order, the colour term of sample
          // k into partial k mod 4 (a zero alpha changes neither)
          if (alpha != 0.0f) {
            const float ta = T * alpha;
            const int q = k & 3;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (j == q) {
                C[j][0] = fmaf(ta, c0, C[j][0]);
                C[j][1] = fmaf(ta, c1, C[j][1]);
                C[j][2] = fmaf(ta, c2, C[j][2]);
              }
            }
            T = T * (1.0f - alpha);
          }
          ++k;
          if (1.0f - T >= L.r.ert) {
            live = false;
            break;
          }
        }
        if (k >= K) live = false;
      }
      __syncthreads();  // the staged region is replaced by the next slab's
    }
    if (active) {
      const float r0 = (C[0][0] + C[1][0]) + (C[2][0] + C[3][0]);
      const float r1 = (C[0][1] + C[1][1]) + (C[2][1] + C[3][1]);
      const float r2 = (C[0][2] + C[1][2]) + (C[2][2] + C[3][2]);
      reinterpret_cast<float4*>(L.out)[(size_t)(py - L.row0) * W + px] =
          make_float4(r0, r1, r2, 1.0f - T);
      hit += K > 0 ? 1u : 0u;
      plain += (unsigned)(k < K ? k : K);
    }
  }
  if (L.stats) {
    const int lane = tid & 31;
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

// ---------------------------------------------------------------------------- launch
static int slab_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 152;
}

template <int VTYPE, int OP>
static cudaError_t launch_slab_k(const MarchLaunch& L, int Ds, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (size_t)L.tf.n + sizeof(SlabSmem);
  static bool attr = false;  // shared memory beyond 48 KiB, set once for the largest table
  if (!attr) {
    const size_t most = sizeof(float4) * (size_t)kSlabMaxTf + sizeof(SlabSmem);
    const cudaError_t e = cudaFuncSetAttribute(
        k_march_slab<VTYPE, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int per = 0;  // resident blocks per SM with this table
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_slab<VTYPE, OP>, kSlabThreads, smem);
  if (e != cudaSuccess) return e;
  if (per < 1) per = 1;
  k_march_slab<VTYPE, OP><<<slab_sms() * per, kSlabThreads, smem, s>>>(L, Ds);
  return cudaGetLastError();
}

template <int VTYPE>
static cudaError_t launch_slab_op(const MarchLaunch& L, int Ds, cudaStream_t s) {
  switch (L.op) {
    case OP_CENTRAL: return launch_slab_k<VTYPE, OP_CENTRAL>(L, Ds, s);
    case OP_SOBEL: return launch_slab_k<VTYPE, OP_SOBEL>(L, Ds, s);
    default: return launch_slab_k<VTYPE, OP_ZH>(L, Ds, s);
  }
}

// Cells per coarse slab (log2): the deepest slab whose region for a tile of rays spread
// `spread` voxels apart fits the staged records (the width: the tile's rays, the drift of a
// ray across the slab -- at most one cell per cell along the slab axis -- and the margins).
static int slab_shift(float spread) {
  for (int sh = 3; sh > 0; --sh) {
    const float w = (kSlabTileW - 1) * spread + (float)(1 << sh) + 4.0f;
    if ((float)((1 << sh) + 1) * w * w <= (float)kSlabMaxRec) return sh;
  }
  return 0;
}

// Largest distance between neighbouring rays inside the sampling box, in voxels.
static float ray_spread(const MarchLaunch& L) {
  const CamDev& c = L.cam;
  if (c.ortho) return 2.0f * std::max(c.ax / (float)c.width, c.ay / (float)c.height);
  float far = 0.0f;
  for (int i = 0; i < 8; ++i) {
    const float q[3] = {(i & 1) ? L.r.hi[0] : L.r.lo[0], (i & 2) ? L.r.hi[1] : L.r.lo[1],
                        (i & 4) ? L.r.hi[2] : L.r.lo[2]};
    const float dx = q[0] - c.eye[0], dy = q[1] - c.eye[1], dz = q[2] - c.eye[2];
    far = std::max(far, std::sqrt(dx * dx + dy * dy + dz * dz));
  }
  return 2.0f * far * std::max(c.ax / (float)c.width, c.ay / (float)c.height);
}

bool slab_eligible(const MarchLaunch& L) {
  if (L.ck_kend || L.r.mult || L.tf.n > kSlabMaxTf) return false;
  for (int a = 0; a < 3; ++a)
    if (L.V.n[a] >= 32768) return false;
  // one-cell slabs must fit too (else the tile march, whose gathers do not care)
  const float w = (kSlabTileW - 1) * ray_spread(L) + 5.0f;
  return 2.0f * w * w <= (float)kSlabMaxRec;
}

cudaError_t launch_march_slab(const MarchLaunch& L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(L.tile_counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  if (L.rect[2] <= L.rect[0] || L.rect[3] <= L.rect[1]) return cudaSuccess;
  const int Ds = slab_shift(ray_spread(L));
  switch (L.dtype) {
    case VT_U8: return launch_slab_op<VT_U8>(L, Ds, s);
    case VT_U16: return launch_slab_op<VT_U16>(L, Ds, s);
    case VT_F16: return launch_slab_op<VT_F16>(L, Ds, s);
    default: return launch_slab_op<VT_F32>(L, Ds, s);
  }
}

}  // namespace vr
