// vr_output.cu -- the 8-bit image of a render: each RGBA channel of the FP32 image (the
// premultiplied colour and the opacity 1 - T of §3.9, Eq. 6) quantised to a byte.
#include "vr_output.h"

namespace vr {

__device__ __forceinline__ unsigned char quantize8(float c) {
  // __saturatef clamps to [0, 1] and maps NaN to 0; the product is rounded in FP32, then to
  // the nearest integer (ties to even)
  return (unsigned char)__float2uint_rn(__saturatef(c) * 255.0f);
}

// One thread per pixel: a 16-byte load and a 4-byte store.
__global__ void __launch_bounds__(256) k_quantize_rgba8(const float4* __restrict__ in,
                                                        uchar4* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 c = __ldg(in + i);
  out[i] = make_uchar4(quantize8(c.x), quantize8(c.y), quantize8(c.z), quantize8(c.w));
}

cudaError_t launch_quantize_rgba8(const float4* in, uchar4* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int threads = 256;
  const size_t blocks = (n + threads - 1) / threads;
  k_quantize_rgba8<<<(unsigned)blocks, threads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace vr
