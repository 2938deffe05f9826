// Bandwidth probe for a roofline denominator that no vendor figure gives: the
// L2 read bandwidth of this GPU.  The traversal kernels read a tree that stays
// resident in L2 (a 200k-face mesh is ~40 MB of the 126 MB L2), so their bytes
// are bounded by L2, not HBM, bandwidth.  The probe reads a caller buffer small
// enough to stay in L2 several times over with L2-only loads (ld.global.cg:
// no L1 allocation) from a grid of a few blocks per SM, eight independent
// 16-byte loads in flight per thread, and folds the words into one value per
// thread so nothing is optimised away.
#include "common.cuh"

namespace meshgs {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;

__global__ void __launch_bounds__(kProbeThreads)
k_l2_read(const uint4 *__restrict__ buf, int64_t n16, int passes, unsigned int *__restrict__ sink) {
    const int64_t stride = (int64_t)gridDim.x * kProbeThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kProbeThreads + threadIdx.x;
    unsigned int acc = 0u;
    for (int p = 0; p < passes; ++p) {
        int64_t i = t0;
        for (; i + (kProbeUnroll - 1) * stride < n16; i += kProbeUnroll * stride) {
            uint4 v[kProbeUnroll];
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) v[u] = __ldcg(buf + i + u * stride);
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; i < n16; i += stride) {
            uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    sink[t0] = acc;
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

size_t mesh_probe_sink_bytes(void) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 0;
    return (size_t)sms * 4 * kProbeThreads * sizeof(unsigned int);
}

mesh_status mesh_probe_l2_read(const void *d_buf, size_t bytes, int passes, void *d_sink,
                               size_t sink_bytes, void *stream) {
    if (!d_buf || !d_sink || passes < 1 || bytes < 16 || (bytes & 15u) || ((uintptr_t)d_buf & 15u))
        return MESH_ERR_INVALID_ARG;
    size_t need = mesh_probe_sink_bytes();
    if (need == 0) return MESH_ERR_CUDA;
    if (sink_bytes < need) return MESH_ERR_WORKSPACE;
    unsigned int grid = (unsigned int)(need / (kProbeThreads * sizeof(unsigned int)));
    k_l2_read<<<grid, kProbeThreads, 0, (cudaStream_t)stream>>>(
        (const uint4 *)d_buf, (int64_t)(bytes / 16), passes, (unsigned int *)d_sink);
    count_launch();
    return check_launch();
}

}  // extern "C"
