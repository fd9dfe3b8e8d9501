// vr_batch.cu -- many renders (cameras over volumes of uneven sizes) in one persistent
// launch, captured once into a CUDA graph and replayed.
//
// The work queue is the concatenation of every render's warp tiles: warps take global tile
// indices from one atomic counter, find their render by binary search over the tiles'
// prefix sums and march the tile with that render's descriptor (the same per-ray march as a
// single render, §3.10).  Rays are independent (§2.2: each ray is computed separately), so
// cheap renders (small volumes, rays that miss) and expensive ones share the SMs without
// any per-render launch or tail.  The descriptors refer to each context's gradient records,
// so volumes of different voxel types mix in one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vr_march.cuh"

namespace vr {

struct BatchLaunch {
  const MarchLaunch* items;  // [n] per-render descriptors (device)
  const int* prefix;         // [n + 1] first warp tile of each render
  int nitems;
  int tiles_total;
  unsigned* counter;
  int tw, th;                // quads per warp tile along x and y (tw * th == 8)
};

// 1024 threads per SM at every block size, i.e. 64 registers a thread: 32 warps per SM, as the
// single-frame march (measured faster than the 80 registers the march takes uncapped).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_march_batch(const BatchLaunch B) {
  const int lane = threadIdx.x & 31;
  const int q = lane & 3, qd = lane >> 2;
  const unsigned qmask = 0xFu << (lane & ~3);
  unsigned hit = 0, plain = 0, visited = 0, shaded = 0;
  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(B.counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= B.tiles_total) break;
    // render of this tile: the last prefix entry <= tile
    int lo = 0, hi = B.nitems;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(B.prefix + mid) <= tile) lo = mid;
      else hi = mid;
    }
    const MarchLaunch& L = B.items[lo];
    const int local = tile - __ldg(B.prefix + lo);
    const int W = L.cam.width, H = L.cam.height;
    const int tiles_x = (W + B.tw - 1) / B.tw;
    const int x0 = (local % tiles_x) * B.tw, y0 = (local / tiles_x) * B.th;
    const int px = x0 + (qd % B.tw);
    const int py = y0 + (qd / B.tw);
    if (x0 + B.tw <= L.rect[0] || x0 >= L.rect[2] || y0 + B.th <= L.rect[1] || y0 >= L.rect[3]) {
      // the whole tile lies outside the box's screen rectangle: its rays miss the box
      if (q == 0 && px < W && py < H) L.out[py * W + px] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      continue;
    }
    march_ray<false>(L, px, py, px < W && py < H, q, qmask, hit, plain, visited, shaded);
    __syncwarp();
  }
}

}  // namespace vr

using namespace vr;

struct vr_batch {
  vr_ctx* owner = nullptr;  // allocator of the device tables
  std::vector<vr_ctx*> ctxs;
  std::vector<uint64_t> vol_gen, tf_gen;
  std::vector<const float4*> rec;  // each context's records buffer at creation
  vr_render_params params{};
  std::vector<MarchLaunch> host_items;
  MarchLaunch* items = nullptr;
  int* prefix = nullptr;
  unsigned* counter = nullptr;
  size_t items_cap = 0, prefix_cap = 0, counter_cap = 0;
  int n = 0, tiles_total = 0;
  int threads = 128, tw = 4, th = 2;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

namespace {

void batch_release_graph(vr_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

int batch_blocks(int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (threads) {
    case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_batch<64>, 64, 0); break;
    case 256: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_batch<256>, 256, 0); break;
    default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_march_batch<128>, 128, 0);
  }
  return (sms > 0 ? sms : 152) * (per > 0 ? per : 1);
}

cudaError_t batch_enqueue(vr_batch* b, int blocks, cudaStream_t s) {
  BatchLaunch B;
  B.items = b->items;
  B.prefix = b->prefix;
  B.nitems = b->n;
  B.tiles_total = b->tiles_total;
  B.counter = b->counter;
  B.tw = b->tw;
  B.th = b->th;
  cudaError_t e = cudaMemsetAsync(b->counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  switch (b->threads) {
    case 64: k_march_batch<64><<<blocks, 64, 0, s>>>(B); break;
    case 256: k_march_batch<256><<<blocks, 256, 0, s>>>(B); break;
    default: k_march_batch<128><<<blocks, 128, 0, s>>>(B);
  }
  return cudaGetLastError();
}

// Tile prefix sums for the current warp-tile shape, uploaded, and the graph rebuilt.
vr_status batch_layout(vr_batch* b) {
  std::vector<int> pre(b->n + 1, 0);
  for (int i = 0; i < b->n; ++i) {
    const CamDev& c = b->host_items[i].cam;
    const long long t = (long long)((c.width + b->tw - 1) / b->tw) * ((c.height + b->th - 1) / b->th);
    const long long next = (long long)pre[i] + t;
    if (next > 2000000000LL) return VR_ERR_INVALID_ARG;
    pre[i + 1] = (int)next;
  }
  b->tiles_total = pre[b->n];
  vr_status st = cuda_status(cudaMemcpyAsync(b->prefix, pre.data(), sizeof(int) * (b->n + 1),
                                             cudaMemcpyHostToDevice, b->capture));
  if (st != VR_OK) return st;
  st = cuda_status(cudaStreamSynchronize(b->capture));
  if (st != VR_OK) return st;
  batch_release_graph(b);
  const int blocks = batch_blocks(b->threads);
  st = cuda_status(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
  if (st != VR_OK) return st;
  const cudaError_t e = batch_enqueue(b, blocks, b->capture);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_status(e);
  }
  if (e2 != cudaSuccess) return cuda_status(e2);
  b->graph = g;
  return cuda_status(cudaGraphInstantiate(&b->exec, g, 0));
}

bool batch_state_current(const vr_batch* b) {
  for (size_t i = 0; i < b->ctxs.size(); ++i)
    if (b->ctxs[i]->vol_gen != b->vol_gen[i] || b->ctxs[i]->tf_gen != b->tf_gen[i]) return false;
  return true;
}

// Records may have been recomputed for other parameters since the batch was built (a
// render with another operator): bring them back for the batch's parameters on `s`.
vr_status batch_records(vr_batch* b, cudaStream_t s) {
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const vr_status st = ensure_records(b->ctxs[i], &b->params, s);
    if (st != VR_OK) return st;
    if (b->ctxs[i]->rec != b->rec[i]) return VR_ERR_STATE;  // reallocated: rebuild the batch
  }
  return VR_OK;
}

}  // namespace

extern "C" {

vr_status vr_batch_create(vr_batch** out, vr_ctx* const* ctxs, int nctx, const vr_camera* cams,
                          const int* ctx_of_cam, int ncams, const vr_render_params* params,
                          float* const* outs, void* stream) {
  if (!out) return VR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctxs || nctx < 1 || !cams || !ctx_of_cam || ncams < 1 || !outs) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->collect_stats || params->adaptive) return VR_ERR_UNSUPPORTED;
  for (int i = 0; i < nctx; ++i) {
    if (!ctxs[i]) return VR_ERR_INVALID_ARG;
    if (!ctxs[i]->has_volume || !ctxs[i]->has_tf) return VR_ERR_STATE;
    if (ctxs[i]->device != ctxs[0]->device) return VR_ERR_UNSUPPORTED;
  }
  std::vector<CamDev> basis(ncams);
  for (int i = 0; i < ncams; ++i) {
    if (ctx_of_cam[i] < 0 || ctx_of_cam[i] >= nctx || !outs[i]) return VR_ERR_INVALID_ARG;
    st = check_camera(&cams[i], &basis[i]);
    if (st != VR_OK) return st;
  }
  const int dev = ctxs[0]->device;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, dev};
  for (int i = 0; i < ncams; ++i)
    if (!is_device_pointer(outs[i]) || !aligned_to(outs[i], 16)) return VR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // gradient records of every volume (computed on `stream` if out of date)
  for (int i = 0; i < nctx; ++i) {
    st = ensure_records(ctxs[i], params, s);
    if (st != VR_OK) return st;
  }
  st = cuda_status(cudaStreamSynchronize(s));
  if (st != VR_OK) return st;
  vr_batch* b = new (std::nothrow) vr_batch();
  if (!b) return VR_ERR_OUT_OF_MEMORY;
  b->owner = ctxs[0];
  b->device = dev;
  b->n = ncams;
  b->params = *params;
  b->ctxs.assign(ctxs, ctxs + nctx);
  for (int i = 0; i < nctx; ++i) {
    b->vol_gen.push_back(ctxs[i]->vol_gen);
    b->tf_gen.push_back(ctxs[i]->tf_gen);
    b->rec.push_back(ctxs[i]->rec);
  }
  b->host_items.resize(ncams);
  for (int i = 0; i < ncams; ++i) {
    vr_ctx* c = ctxs[ctx_of_cam[i]];
    MarchLaunch& L = b->host_items[i];
    std::memset(&L, 0, sizeof(L));
    L.V = vol_dev(c);
    L.R = rec_dev(c);
    L.tf = tf_dev(c);
    L.cam = basis[i];
    L.r = render_dev(c, params);
    L.dtype = (int)c->dtype;
    L.op = params->grad;
    L.out = reinterpret_cast<float4*>(outs[i]);
    screen_rect(L.cam, L.r.lo, L.r.hi, L.rect);
  }
  void* p = nullptr;
  st = ensure(b->owner, &p, &b->items_cap, sizeof(MarchLaunch) * ncams);
  b->items = static_cast<MarchLaunch*>(p);
  if (st == VR_OK) {
    p = nullptr;
    st = ensure(b->owner, &p, &b->prefix_cap, sizeof(int) * (ncams + 1));
    b->prefix = static_cast<int*>(p);
  }
  if (st == VR_OK) {
    p = nullptr;
    st = ensure(b->owner, &p, &b->counter_cap, 256);
    b->counter = static_cast<unsigned*>(p);
  }
  if (st == VR_OK) st = cuda_status(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking));
  if (st == VR_OK)
    st = cuda_status(cudaMemcpyAsync(b->items, b->host_items.data(), sizeof(MarchLaunch) * ncams,
                                     cudaMemcpyHostToDevice, b->capture));
  if (st == VR_OK) st = batch_layout(b);
  if (st != VR_OK) {
    vr_batch_destroy(b);
    return st;
  }
  *out = b;
  return VR_OK;
}

vr_status vr_batch_run(vr_batch* b, void* stream) {
  TraceRange trace_("vr_batch_run");
  if (!b) return VR_ERR_INVALID_ARG;
  if (!batch_state_current(b)) return VR_ERR_STATE;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  vr_status st = batch_records(b, static_cast<cudaStream_t>(stream));
  if (st == VR_OK) st = cuda_status(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return st;
}

vr_status vr_batch_autotune(vr_batch* b, void* stream, int* chosen) {
  TraceRange trace_("vr_batch_autotune");
  if (!b) return VR_ERR_INVALID_ARG;
  if (!batch_state_current(b)) return VR_ERR_STATE;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  vr_status st0 = batch_records(b, s);
  if (st0 != VR_OK) {
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return st0;
  }
  const int threads_opts[3] = {64, 128, 256};
  const int tw_opts[3] = {4, 2, 8};
  float best = 3.4e38f;
  int best_t = b->threads, best_w = b->tw;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vr_status st = cuda_status(cudaEventCreate(&e0));
  if (st == VR_OK) st = cuda_status(cudaEventCreate(&e1));
  for (int ti = 0; ti < 3 && st == VR_OK; ++ti)
    for (int wi = 0; wi < 3 && st == VR_OK; ++wi) {
      b->threads = threads_opts[ti];
      b->tw = tw_opts[wi];
      b->th = 8 / b->tw;
      st = batch_layout(b);
      if (st != VR_OK) break;
      float t_best = 3.4e38f;
      for (int rep = 0; rep < 3 && st == VR_OK; ++rep) {
        st = cuda_status(cudaEventRecord(e0, s));
        if (st == VR_OK) st = cuda_status(cudaGraphLaunch(b->exec, s));
        if (st == VR_OK) st = cuda_status(cudaEventRecord(e1, s));
        if (st == VR_OK) st = cuda_status(cudaEventSynchronize(e1));
        float ms = 0.0f;
        if (st == VR_OK) st = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) t_best = std::min(t_best, ms);  // first run warms up
      }
      if (t_best < best) {
        best = t_best;
        best_t = b->threads;
        best_w = b->tw;
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->threads = best_t;
  b->tw = best_w;
  b->th = 8 / best_w;
  if (st == VR_OK) st = batch_layout(b);
  if (chosen) {
    chosen[0] = b->threads;
    chosen[1] = b->tw;
    chosen[2] = b->th;
  }
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return st;
}

vr_status vr_render_batch(vr_ctx* const* vols, const vr_camera* cams, const int* vol_of_cam,
                          int n, const vr_render_params* params, float* const* outs,
                          void* stream) {
  TraceRange trace_("vr_render_batch");
  if (!vols || !cams || !vol_of_cam || n < 1 || !outs) return VR_ERR_INVALID_ARG;
  vr_status st = check_params(params);
  if (st != VR_OK) return st;
  if (params->collect_stats || params->adaptive) return VR_ERR_UNSUPPORTED;
  int nvol = 0;
  for (int i = 0; i < n; ++i) {
    if (vol_of_cam[i] < 0 || !outs[i]) return VR_ERR_INVALID_ARG;
    nvol = std::max(nvol, vol_of_cam[i] + 1);
  }
  for (int i = 0; i < nvol; ++i) {
    if (!vols[i]) return VR_ERR_INVALID_ARG;
    if (!vols[i]->has_volume || !vols[i]->has_tf) return VR_ERR_STATE;
    if (vols[i]->device != vols[0]->device) return VR_ERR_UNSUPPORTED;
  }
  std::vector<MarchLaunch> items(n);
  for (int i = 0; i < n; ++i) {
    CamDev basis;
    st = check_camera(&cams[i], &basis);
    if (st != VR_OK) return st;
    std::memset(&items[i], 0, sizeof(MarchLaunch));
    items[i].cam = basis;
  }
  vr_ctx* owner = vols[0];
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != owner->device) cudaSetDevice(owner->device);
  struct Restore {
    int p, d;
    ~Restore() {
      if (p >= 0 && p != d) cudaSetDevice(p);
    }
  } restore{prev, owner->device};
  for (int i = 0; i < n; ++i)
    if (!is_device_pointer(outs[i]) || !aligned_to(outs[i], 16)) return VR_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < nvol; ++i) {
    st = ensure_records(vols[i], params, s);
    if (st != VR_OK) return st;
  }
  // descriptors and tile prefix sums, copied into the owner's table buffer on `stream`
  constexpr int tw = 4, th = 2;
  std::vector<int> pre(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    vr_ctx* c = vols[vol_of_cam[i]];
    MarchLaunch& L = items[i];
    L.V = vol_dev(c);
    L.R = rec_dev(c);
    L.tf = tf_dev(c);
    L.r = render_dev(c, params);
    L.dtype = (int)c->dtype;
    L.op = params->grad;
    L.out = reinterpret_cast<float4*>(outs[i]);
    screen_rect(L.cam, L.r.lo, L.r.hi, L.rect);
    const long long t = (long long)((L.cam.width + tw - 1) / tw) * ((L.cam.height + th - 1) / th);
    if ((long long)pre[i] + t > 2000000000LL) return VR_ERR_INVALID_ARG;
    pre[i + 1] = pre[i] + (int)t;
  }
  const size_t items_bytes = (sizeof(MarchLaunch) * n + 255) / 256 * 256;
  const size_t prefix_bytes = (sizeof(int) * (n + 1) + 255) / 256 * 256;
  st = ensure(owner, &owner->batch_tab, &owner->batch_tab_cap, items_bytes + prefix_bytes + 256);
  if (st != VR_OK) return st;
  char* tab = static_cast<char*>(owner->batch_tab);
  st = cuda_status(cudaMemcpyAsync(tab, items.data(), sizeof(MarchLaunch) * n,
                                   cudaMemcpyHostToDevice, s));
  if (st == VR_OK)
    st = cuda_status(cudaMemcpyAsync(tab + items_bytes, pre.data(), sizeof(int) * (n + 1),
                                     cudaMemcpyHostToDevice, s));
  if (st != VR_OK) return st;
  BatchLaunch B;
  B.items = reinterpret_cast<const MarchLaunch*>(tab);
  B.prefix = reinterpret_cast<const int*>(tab + items_bytes);
  B.nitems = n;
  B.tiles_total = pre[n];
  B.counter = reinterpret_cast<unsigned*>(tab + items_bytes + prefix_bytes);
  B.tw = tw;
  B.th = th;
  st = cuda_status(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), s));
  if (st != VR_OK) return st;
  k_march_batch<128><<<batch_blocks(128), 128, 0, s>>>(B);
  return cuda_status(cudaGetLastError());
}

void vr_batch_destroy(vr_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  batch_release_graph(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->owner) {
    ctx_free(b->owner, b->items);
    ctx_free(b->owner, b->prefix);
    ctx_free(b->owner, b->counter);
  }
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
