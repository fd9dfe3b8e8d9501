// vr_output.h -- the 8-bit image of a render (vr_render_rgba8).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace vr {

// out[i] = the four channels of in[i], each round(255 * clamp(c, 0, 1)) (FP32 product, round
// to nearest even; NaN gives 0), for i < n.  in and out are device memory aligned to 16 and
// 4 bytes.
cudaError_t launch_quantize_rgba8(const float4* in, uchar4* out, size_t n, cudaStream_t s);

}  // namespace vr
