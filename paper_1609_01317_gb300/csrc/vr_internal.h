// vr_internal.h -- host-side context and launcher declarations of libvr.
#pragma once

#include <cmath>

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/vr.h"
#include "vr_device.cuh"

#include <nvtx3/nvToolsExt.h>

namespace vr {

// An NVTX range around one entry point, so that a profiler's timeline shows which library
// call launched which kernels (header-only NVTX; no cost without an attached tool).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};


// One forward pass that wrote adjoint checkpoints (remembered to validate the backward).
struct CkptRecord {
  const void* ptr = nullptr;
  size_t bytes = 0;
  vr_camera cam{};
  vr_render_params params{};
  uint64_t vol_gen = 0, tf_gen = 0;
  int nrays = 0, nslots = 0;
};

constexpr int kMaxCkptRecords = 128;

}  // namespace vr

struct vr_ctx {
  int device = 0;
  vr_alloc_fn alloc = nullptr;
  vr_free_fn free_fn = nullptr;
  void* user = nullptr;

  // volume (padded copy with clamp-to-edge border) and brick tables
  bool has_volume = false;
  vr_dtype dtype = VR_U8;
  int n[3] = {0, 0, 0};
  float value_max = 1.0f;
  void* vol = nullptr;
  size_t vol_cap = 0;
  int px = 0, py = 0, pz = 0;  // padded extents
  int nb[3] = {0, 0, 0};
  float2* brick_minmax = nullptr;
  uint8_t* brick_vis = nullptr;
  int* brick_list = nullptr;  // [0]: count of visible bricks, then their indices
  uint8_t* macro_vis = nullptr;  // per macro brick (4^3 bricks): OR of the bricks' visibility
  int nm[3] = {0, 0, 0};
  uint8_t* super_vis = nullptr;  // per super brick (4^3 macro bricks): OR of their visibility
  int ns[3] = {0, 0, 0};
  size_t brick_cap = 0;
  void* upload_staging = nullptr;
  cudaEvent_t host_copy_done = nullptr;  // end of the last copy from a caller's host buffer
  // pinned staging of a host transfer function, and the end of the last copy out of it
  void* tf_host_stage = nullptr;
  size_t tf_host_stage_cap = 0;
  cudaEvent_t tf_stage_done = nullptr;
  size_t upload_cap = 0;

  // transfer function
  bool has_tf = false;
  int ntf = 0;
  float4* tf = nullptr;
  size_t tf_cap = 0;
  int* tf_prefix = nullptr;  // number of entries with alpha != 0 below each index
  uint64_t vol_gen = 0, tf_gen = 0;

  // camera
  bool has_camera = false;
  vr_camera cam{};
  vr::CamDev camdev{};

  // statistics: [0..3] counters, then the tile counters of the march [4], the adjoint [5]
  // and the surface renderer [6], the bounds-violation counter [7] and the records pass's
  // timeout word [8] (16 slots)
  unsigned long long* stats = nullptr;
  bool stats_valid = false;
  int stats_march = 0;  // VR_MARCH_RECORDS / VR_MARCH_SLABS of the render the counters are from

  // output staging for host destinations
  void* out_staging = nullptr;
  size_t out_cap = 0;

  // adjoint scratch: per voxel (dL/ds, dL/dG) at the cell corners, float4
  float4* adj = nullptr;
  size_t adj_cap = 0;
  // per-block partial sums of the transfer-function gradient, [blocks][4 * ntf]
  float* tf_partial = nullptr;
  size_t tf_partial_cap = 0;

  // per-macro-brick sampling multipliers of an adaptive render
  void* adapt_mult = nullptr;
  size_t adapt_mult_cap = 0;

  // brick and macro-brick visibility for a surface render's threshold window
  void* surf_vis = nullptr;
  size_t surf_vis_cap = 0;

  // tables of one-shot batched renders issued with this context first (vr_render_batch)
  void* batch_tab = nullptr;
  size_t batch_tab_cap = 0;

  // rays of a plain render that reach a visible macro brick ([0]: count, [1]: work counter,
  // records from byte 256 on)
  void* ray_list = nullptr;
  size_t ray_list_cap = 0;
  // the visible-brick count seen by the latest plain render's march, written by the march
  // into mapped pinned host memory: {count, bricks} (a hint for choosing the next render's
  // march; read without waiting)
  volatile int* vis_hint = nullptr;
  int* vis_hint_dev = nullptr;  // the same memory as the device sees it

  // operator gradient records (G, V) per voxel and what they were computed for
  float4* rec = nullptr;
  size_t rec_cap = 0;
  bool rec_valid = false, rec_all = false;
  uint64_t rec_vol_gen = 0, rec_tf_gen = 0;
  int rec_op = -1;

  vr::CkptRecord ckpt[vr::kMaxCkptRecords];
  int ckpt_next = 0;
};

namespace vr {

// allocation through the context's allocator
vr_status ctx_alloc(vr_ctx* ctx, void** p, size_t bytes);
void ctx_free(vr_ctx* ctx, void* p);
vr_status ensure(vr_ctx* ctx, void** p, size_t* cap, size_t bytes);
vr_status cuda_status(cudaError_t e);

// argument checks and host-side set-up shared by the entry points
vr_status check_params(const vr_render_params* p);
vr_status check_camera(const vr_camera* cam, CamDev* basis);
bool camera_basis(const vr_camera* c, CamDev* b);
bool is_device_pointer(const void* p);
// whether p is a multiple of `bytes` (a power of two): device buffers the kernels access as
// float4 (images, image gradients, a transfer function read in place) need 16, other float
// buffers 4, voxel arrays their element size
inline bool aligned_to(const void* p, size_t bytes) {
  return (reinterpret_cast<uintptr_t>(p) & (bytes - 1)) == 0;
}

// device descriptors
VolDev vol_dev(const vr_ctx* ctx);
RenderDev render_dev_for(const int n[3], float value_max, const vr_render_params* p);
RecDev rec_dev(const vr_ctx* ctx);
// gradient records of the context's volume for `p` (recomputed on `s` when stale)
vr_status ensure_records(vr_ctx* ctx, const vr_render_params* p, cudaStream_t s);
TfDev tf_dev(const vr_ctx* ctx);
RenderDev render_dev(const vr_ctx* ctx, const vr_render_params* p);
int max_samples(const vr_ctx* ctx, const vr_render_params* p);

// launchers (return the first CUDA error, if any)
cudaError_t launch_pad_volume(const void* src, int dtype, const int n[3], void* dst, int px,
                              int py, int pz, cudaStream_t s);
cudaError_t launch_brick_minmax(const VolDev& V, int dtype, float2* mm, cudaStream_t s);
cudaError_t launch_tf_prefix(const float4* tf, int n, int* prefix, cudaStream_t s);
// vis[b] for every brick; when `list` is non-null, its visible bricks' indices are written
// after list[0] (= their count, order unspecified); when `mvis` is non-null, mvis[m] = OR of
// vis over the bricks of macro brick m (grid nm), and when `svis` is non-null too, svis[u] =
// OR over the macro bricks of super brick u (grid ns; svis must follow mvis in the same
// allocation: both are cleared by one memset)
cudaError_t launch_brick_visibility(const float2* mm, const int nb[3], const int* prefix,
                                    int ntf, float scale, uint8_t* vis, int* list,
                                    uint8_t* mvis, const int nm[3], cudaStream_t s,
                                    uint8_t* svis = nullptr, const int* ns = nullptr);
// mult[m] = 4 if the footprint range max - min of macro brick m is <= r4 (r4 >= 0), else 2
// if <= r2 (r2 >= 0), else 1
cudaError_t launch_macro_multiplier(const float2* mm, const int nb[3], const int nm[3], float r2,
                                    float r4, uint8_t* mult, cudaStream_t s);
// records of the bricks in `list` (as built by launch_brick_visibility, `need` its vis
// array), or of every brick when `list` is null; with `err` (a device word) the bricks'
// neighbourhoods are staged by TMA copies, and a copy that does not complete within about a
// second sets *err |= 1 and ends the launch (the records are then incomplete)
cudaError_t launch_records(const VolDev& V, int dtype, int op, const uint8_t* need,
                           const int* list, float4* rec, cudaStream_t s, unsigned* err = nullptr);

// A plain render takes the ray list when fewer than one brick in kListDenom is visible for
// the current transfer function (the count k_brick_visibility leaves in the brick list).
// Measured on GB300: 1.4 % visible (vessel tree, 3840 x 2160) -> the list march is 1.28x
// faster than the tile march; 32 % visible (CT phantom, 1920 x 1080) -> 2 % slower.
constexpr long long kListDenom = 10;

// A ray of a plain render after its set-up: origin and entry distance, direction and sample
// count, pixel and the first sample the march needs (a multiple of 4; the samples before it
// lie in transparent macro bricks).
struct RayRec {
  float4 o_tn;    // o.x, o.y, o.z, t_near
  float4 d_K;     // d.x, d.y, d.z, K (int bits)
  int4 px_py_k0;  // px, py, k0, unused
};

struct MarchLaunch {
  VolDev V;
  RecDev R;
  TfDev tf;
  CamDev cam;
  RenderDev r;
  int dtype, op;
  float4* out;
  unsigned long long* stats;  // NULL: no counting
  unsigned* tile_counter;     // work counter of the persistent launch (zeroed per launch)
  int rect[4];                // pixels [rect[0], rect[2]) x [rect[1], rect[3]) whose tiles the
                              // launch marches; every ray outside misses the sampling box
                              // and its pixel is zeroed beforehand
  int* ck_kend;               // NULL: no checkpoints
  float* ck_T;                // transmittance before every 32nd sample, [slot][ray]
  float* ck_Tend;             // transmittance after the last sample, [ray]
  int nslots;
  // rows [row0, row1) of the image are marched and pixel (px, py) is written to
  // out[(py - row0) * width + px] (a band of the frame; the whole frame by default)
  int row0 = 0, row1 = 1 << 30;
  // plain renders (no checkpoints, regular grid): when few bricks are visible, a ray set-up
  // kernel lists the rays that reach a visible macro brick and the march takes them from the
  // list (null, or many visible bricks: the march sets up every ray of its tiles itself)
  RayRec* list = nullptr;
  int* list_head = nullptr;  // [0]: rays listed, [1]: the march's work counter (zeroed per launch)
  const int* vis_count = nullptr;  // visible bricks of the current transfer function (device)
  int mode = 0;  // 0: list mode decided on the device from vis_count; 1: tiles; 2: list
  int* hint = nullptr;  // host-mapped {count, bricks}: written by the march for the next render
  // partial images (sort-last): only samples with z in [zwin[0], zwin[1]) are composited
  float zwin[2] = {-HUGE_VALF, HUGE_VALF};
};
cudaError_t launch_march(const MarchLaunch& L, cudaStream_t s);
// The plain tile march restricted to the samples in L.zwin (records must be current).
cudaError_t launch_march_zwin(const MarchLaunch& L, cudaStream_t s);
// The slab march (no record table): whether it can render L (a plain render whose rays lie
// close enough together), and its launch.
bool slab_eligible(const MarchLaunch& L);
cudaError_t launch_march_slab(const MarchLaunch& L, cudaStream_t s);
// Pixel rectangle [rect[0], rect[2]) x [rect[1], rect[3]) outside which every ray of camera c
// misses the box [lo, hi] (the full image when that cannot be shown, empty for an empty box).
void screen_rect(const CamDev& c, const float lo[3], const float hi[3], int rect[4]);

// One view of an adjoint launch: its camera, the checkpoints its forward recorded, the
// gradient of its image, and the tiles of its work in the launch's queue.
struct AdjView {
  CamDev cam;
  const int* ck_kend;
  const float* ck_T;
  const float* ck_Tend;
  const float4* grad_rgba;
  // the warp tiles of the pixel rectangle [rect[0], rect[2]) x [rect[1], rect[3]) (every ray
  // outside it misses the sampling box: its recorded end index is 0): tiles_x per row from
  // tile (tx0, ty0), numbered from tile0 in the launch's queue
  int tx0, ty0, tiles_x, tile0;
};
// views per adjoint launch (the descriptors travel in the launch's parameters)
constexpr int kAdjViews = 16;

struct AdjointLaunch {
  VolDev V;
  RecDev R;
  TfDev tf;
  RenderDev r;
  int dtype, op;
  unsigned* tile_counter;  // work counter of the persistent launch (zeroed per launch)
  float4* adj;     // per voxel corner accumulators (dL/ds, dL/dG) over the unpadded grid
  float* grad_tf;  // n x 4, accumulated
  // when non-null: [adjoint_grid(n)][4 n] per-block sums of the TF gradient, added to with
  // vector reductions; grad_tf then receives them through launch_tf_partial_reduce instead
  // of from the kernel
  float* tf_partial;
  // the queue: the tiles of view[0], then those of view[1], ...
  int nviews = 0, tiles_total = 0;
  AdjView view[kAdjViews];
};
static_assert(sizeof(AdjointLaunch) <= 4096, "adjoint launch parameters exceed 4 KiB");
// Appends a view to L's queue: the tiles of the rectangle rect of its image.
void adjoint_add_view(AdjointLaunch& L, const CamDev& cam, const int rect[4], const int* ck_kend,
                      const float* ck_T, const float* ck_Tend, const float4* grad_rgba);
// whether the TF gradient goes through per-block partial rows for a table of ntf entries,
// and the persistent grid the adjoint launches for it
bool adjoint_tf_rows(int ntf);
int adjoint_grid(int ntf);
cudaError_t launch_adjoint(const AdjointLaunch& L, cudaStream_t s);
// grad_tf[e] += sum over blocks b of partial[b][e], e < n4, in block order
cudaError_t launch_tf_partial_reduce(const float* partial, int blocks, int n4, float* grad_tf,
                                     cudaStream_t s);
cudaError_t launch_adjoint_volume(const float4* adj, const int n[3], int op, float inv_vmax,
                                  float* grad_volume, cudaStream_t s);

}  // namespace vr
