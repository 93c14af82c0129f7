// Bandwidth probe for roofline reporting: a read-only pass over a buffer that stays resident in L2.
//
// The screened lists are shared by every walker and stay in the 129 MB L2 while the local energy
// runs, so its list traffic is bounded by L2 bandwidth, not HBM.  This kernel measures that bound
// the same way the kernel reads the lists: 16-byte loads through L2 (bypassing L1), every CTA
// reading the whole buffer `reps` times after a first pass has brought it into L2.
#include "common.cuh"

namespace {

__device__ unsigned long long g_probe_sink;

__global__ void __launch_bounds__(512) k_l2_read(const uint4 *__restrict__ buf, size_t n16, int reps) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n16; i += 4 * stride) {   // four loads in flight per thread
            const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const uint4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = __ldcg(buf + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(&g_probe_sink, 1ull);   // keeps the loads; practically never taken
}

}  // namespace

extern "C" vmc_status vmc_probe_l2_read(vmc_ctx *ctx, const void *d_buf, size_t bytes, int reps) {
    if (!ctx) return VMC_ERR_ARG;
    if (!d_buf || bytes < 16 || reps < 1 || ((uintptr_t)d_buf & 15))
        return set_err(ctx, VMC_ERR_ARG, "buffer must be 16-byte aligned and at least 16 bytes; reps >= 1");
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(ctx, e, "vmc_probe_l2_read");
    k_l2_read<<<4 * nsm, 512, 0, ctx->stream>>>((const uint4 *)d_buf, bytes / 16, reps);
    ctx->launches += 1;
    return cuda_check(ctx, cudaGetLastError(), "k_l2_read");
}
