// Read-bandwidth probe for the benchmark's rooflines.  A measurement helper,
// not part of the traversal and not part of the library's C ABI: it is
// built into its own small library (libtmprobe.so), which only the
// benchmark loads.  Every thread streams 64 bytes per iteration with
// L1-bypassing 16-byte loads over a caller buffer, so a buffer that fits in
// L2 measures the L2 read bandwidth, one larger than L2 the HBM read
// bandwidth.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(256)
read_probe_kernel(const int4 *__restrict__ p, int64_t n16, int32_t *__restrict__ sink) {
    int acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const int4 a = __ldcg(p + i), b = __ldcg(p + i + stride);
        const int4 c = __ldcg(p + i + 2 * stride), d = __ldcg(p + i + 3 * stride);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n16; i += stride) {
        const int4 a = __ldcg(p + i);
        acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    if (acc == 0x5EED5EED) sink[0] = acc;  // keeps the loads; a match is harmless
}

}  // namespace

// Reads `bytes` (a multiple of 16) of DEVICE memory at buf (16-byte aligned)
// `reps` times on `stream`, one kernel per pass; *sink (DEVICE int32) may
// receive a checksum.  Returns 0, 1 for a bad argument, or 2 when a CUDA
// call failed.
extern "C" int tm_bench_read_probe(const void *buf, int64_t bytes, int reps, int32_t *sink,
                                   void *stream) {
    if (!buf || !sink || bytes <= 0 || (bytes & 15) || (((uintptr_t)buf) & 15u) || reps < 1)
        return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 2;
    const int64_t n16 = bytes / 16;
    int64_t grid = (int64_t)sms * 8;
    const int64_t need = (n16 + 255) / 256;
    if (grid > need) grid = need;
    for (int r = 0; r < reps; ++r)
        read_probe_kernel<<<(int)grid, 256, 0, (cudaStream_t)stream>>>(
            static_cast<const int4 *>(buf), n16, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
