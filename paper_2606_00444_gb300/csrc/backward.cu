// Gradients of the point-to-mesh squared distance and of barycentric
// interpolation, used for the differentiable form of the update (fitting a
// fixed-topology template to a varying-topology target through Chamfer).
//
// With the nearest face and its weights held fixed (envelope theorem; the
// closest point c = sum_j b_j v_j is optimal, so its own variation drops
// out): d(d^2)/dq = 2 (q - c), d(d^2)/dv_j = -2 b_j (q - c).
#include "common.cuh"

namespace meshgs {

__global__ void k_closest_point_backward(const int4 *__restrict__ faces,
                                         const float4 *__restrict__ verts, int nF,
                                         const float *__restrict__ Q, int64_t nQ,
                                         const int *__restrict__ face,
                                         const float *__restrict__ bary,
                                         const float *__restrict__ g, float *__restrict__ gQ,
                                         float *gV, unsigned int *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nQ) return;
    int f = face[i];
    float gi = g[i];
    if (f < 0 || gi == 0.0f) {
        if (gQ) { gQ[3 * i] = 0.0f; gQ[3 * i + 1] = 0.0f; gQ[3 * i + 2] = 0.0f; }
        return;
    }
    if (f >= nF) {
        atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE);
        if (gQ) { gQ[3 * i] = 0.0f; gQ[3 * i + 1] = 0.0f; gQ[3 * i + 2] = 0.0f; }
        return;
    }
    int4 fv = faces[f];
    float4 a = verts[fv.x], b = verts[fv.y], c = verts[fv.z];
    float u = bary[3 * i], v = bary[3 * i + 1], w = bary[3 * i + 2];
    float rx = 2.0f * gi * (Q[3 * i] - (u * a.x + v * b.x + w * c.x));
    float ry = 2.0f * gi * (Q[3 * i + 1] - (u * a.y + v * b.y + w * c.y));
    float rz = 2.0f * gi * (Q[3 * i + 2] - (u * a.z + v * b.z + w * c.z));
    if (gQ) { gQ[3 * i] = rx; gQ[3 * i + 1] = ry; gQ[3 * i + 2] = rz; }
    if (gV) {
        int vv[3] = {fv.x, fv.y, fv.z};
        float bb[3] = {u, v, w};
        for (int j = 0; j < 3; ++j) {
            if (bb[j] == 0.0f) continue;
            float *p = gV + 3 * (size_t)vv[j];
            atomicAdd(p, -bb[j] * rx);
            atomicAdd(p + 1, -bb[j] * ry);
            atomicAdd(p + 2, -bb[j] * rz);
        }
    }
}

__global__ void k_interpolate_backward(const int4 *__restrict__ faces, int nF,
                                       const int *__restrict__ face,
                                       const float *__restrict__ bary, int64_t n,
                                       const float *__restrict__ gP, float *gV,
                                       unsigned int *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = face[i];
    if ((unsigned)f >= (unsigned)nF) { atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE); return; }
    int4 fv = faces[f];
    float gx = gP[3 * i], gy = gP[3 * i + 1], gz = gP[3 * i + 2];
    int vv[3] = {fv.x, fv.y, fv.z};
    for (int j = 0; j < 3; ++j) {
        float bj = bary[3 * i + j];
        if (bj == 0.0f) continue;
        float *p = gV + 3 * (size_t)vv[j];
        atomicAdd(p, bj * gx);
        atomicAdd(p + 1, bj * gy);
        atomicAdd(p + 2, bj * gz);
    }
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

mesh_status mesh_closest_point_backward(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                                        const int32_t *d_face, const float *d_bary,
                                        const float *d_g, float *d_gQ, float *d_gV,
                                        void *stream) {
    if (!bvh || nQ < 0 || (nQ > 0 && (!d_Q || !d_face || !d_bary || !d_g)))
        return MESH_ERR_INVALID_ARG;
    if (nQ == 0 || (!d_gQ && !d_gV)) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_closest_point_backward<<<grid_for(nQ, 256), 256, 0, s>>>(
        bvh->faces(), bvh->verts(), (int)bvh->L.n_faces, d_Q, nQ, d_face, d_bary, d_g, d_gQ, d_gV,
        &bvh->hdr()->status);
    count_launch();
    return check_launch();
}

mesh_status mesh_interpolate_backward(const mesh_bvh *bvh, const int32_t *d_face,
                                      const float *d_bary, int64_t n, const float *d_gP,
                                      float *d_gV, void *stream) {
    if (!bvh || n < 0 || (n > 0 && (!d_face || !d_bary || !d_gP || !d_gV)))
        return MESH_ERR_INVALID_ARG;
    if (n == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_interpolate_backward<<<grid_for(n, 256), 256, 0, s>>>(bvh->faces(), (int)bvh->L.n_faces,
                                                            d_face, d_bary, n, d_gP, d_gV,
                                                            &bvh->hdr()->status);
    count_launch();
    return check_launch();
}

mesh_status mesh_bvh_status(mesh_bvh *bvh, uint32_t *bits, uint32_t *n_degenerate, void *stream) {
    if (!bvh) return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int h[2] = {0u, 0u};
    if (cudaMemcpyAsync(h, &bvh->hdr()->status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MESH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MESH_ERR_CUDA;
    if (cudaMemsetAsync(&bvh->hdr()->status, 0, sizeof(h), s) != cudaSuccess) return MESH_ERR_CUDA;
    if (bits) *bits = h[0];
    if (n_degenerate) *n_degenerate = h[1];
    return (h[0] & ~(unsigned)MESH_DEV_DEGENERATE) ? MESH_ERR_DEVICE : MESH_OK;
}

const char *mesh_status_string(mesh_status st) {
    switch (st) {
        case MESH_OK: return "ok";
        case MESH_ERR_INVALID_ARG: return "invalid argument";
        case MESH_ERR_CUDA: return "CUDA error";
        case MESH_ERR_WORKSPACE: return "storage or workspace too small or misaligned";
        case MESH_ERR_DEVICE: return "device-side error bits set";
    }
    return "unknown status";
}

}  // extern "C"
