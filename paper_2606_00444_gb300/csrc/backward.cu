// Gradients of the point-to-mesh squared distance, of the Chamfer distance and
// of barycentric interpolation, used for the differentiable form of the update (fitting a
// fixed-topology template to a varying-topology target through Chamfer).
//
// With the nearest face and its weights held fixed (envelope theorem; the
// closest point c = sum_j b_j v_j is optimal, so its own variation drops
// out): d(d^2)/dq = 2 (q - c), d(d^2)/dv_j = -2 b_j (q - c).
#include "common.cuh"

namespace meshgs {

// One query's share: dL/dq written to gq (when not NULL), -b_j dL/dq added to
// the face's vertices in gV (when not NULL).  gi = dL/d(dist2) of the query.
__device__ __forceinline__ void point_backward(const int4 *__restrict__ faces,
                                               const float4 *__restrict__ verts, int nF,
                                               const float *__restrict__ q, int f,
                                               const float *__restrict__ bary, float gi,
                                               float *__restrict__ gq, float *gV,
                                               unsigned int *status) {
    if (f < 0 || gi == 0.0f) {
        if (gq) { gq[0] = 0.0f; gq[1] = 0.0f; gq[2] = 0.0f; }
        return;
    }
    if (f >= nF) {
        atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE);
        if (gq) { gq[0] = 0.0f; gq[1] = 0.0f; gq[2] = 0.0f; }
        return;
    }
    int4 fv = faces[f];
    float4 a = verts[fv.x], b = verts[fv.y], c = verts[fv.z];
    float u = bary[0], v = bary[1], w = bary[2];
    float rx = 2.0f * gi * (q[0] - (u * a.x + v * b.x + w * c.x));
    float ry = 2.0f * gi * (q[1] - (u * a.y + v * b.y + w * c.y));
    float rz = 2.0f * gi * (q[2] - (u * a.z + v * b.z + w * c.z));
    if (gq) { gq[0] = rx; gq[1] = ry; gq[2] = rz; }
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

__global__ void k_closest_point_backward(const int4 *__restrict__ faces,
                                         const float4 *__restrict__ verts, int nF,
                                         const float *__restrict__ Q, int64_t nQ,
                                         const int *__restrict__ face,
                                         const float *__restrict__ bary,
                                         const float *__restrict__ g, float *__restrict__ gQ,
                                         float *gV, unsigned int *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nQ) return;
    point_backward(faces, verts, nF, Q + 3 * i, face[i], bary + 3 * i, g[i], gQ ? gQ + 3 * i : nullptr,
                   gV, status);
}

// Reverse mode of the Chamfer distance (Sec. 4.2): out[0] = mean over SA of
// d(a, B)^2 and out[1] = mean over SB of d(b, A)^2, so every sample of SA
// carries dL/d(dist2) = g[0] / |SA| and every sample of SB g[1] / |SB|.  One
// launch: blocks [0, nbA) take SA against mesh B (gradients into gSA and
// gVB), the rest SB against mesh A (gSB, gVA).  g is read on the device, so
// the call needs no host synchronisation.
struct ChamferGradSide {
    const int4 *faces;
    const float4 *verts;
    int nF;
    const float *S;
    int64_t n;
    const int *face;
    const float *bary;
    float *gS, *gV;
    unsigned int *status;
};

__global__ void k_chamfer_backward(ChamferGradSide A2B, ChamferGradSide B2A, unsigned int nbA,
                                   const double *__restrict__ g) {
    const bool first = blockIdx.x < nbA;
    const ChamferGradSide &C = first ? A2B : B2A;
    int64_t i = (int64_t)(first ? blockIdx.x : blockIdx.x - nbA) * blockDim.x + threadIdx.x;
    if (i >= C.n) return;
    float gi = (float)(g[first ? 0 : 1] / (double)C.n);
    point_backward(C.faces, C.verts, C.nF, C.S + 3 * i, C.face[i], C.bary + 3 * i, gi,
                   C.gS ? C.gS + 3 * i : nullptr, C.gV, C.status);
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

mesh_status mesh_chamfer_backward(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                                  const mesh_bvh *B, const float *d_SB, int64_t nSB,
                                  const double *d_g, const int32_t *d_faceA, const float *d_baryA,
                                  const int32_t *d_faceB, const float *d_baryB, float *d_gSA,
                                  float *d_gVA, float *d_gSB, float *d_gVB, void *stream) {
    if (!A || !B || !d_g || nSA < 0 || nSB < 0 ||
        (nSA > 0 && (!d_SA || !d_faceA || !d_baryA)) || (nSB > 0 && (!d_SB || !d_faceB || !d_baryB)))
        return MESH_ERR_INVALID_ARG;
    const bool wantA = nSA > 0 && (d_gSA || d_gVB), wantB = nSB > 0 && (d_gSB || d_gVA);
    if (!wantA && !wantB) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    unsigned int nbA = wantA ? grid_for(nSA, block) : 0u, nbB = wantB ? grid_for(nSB, block) : 0u;
    ChamferGradSide a2b{B->faces(), B->verts(), (int)B->L.n_faces, d_SA, wantA ? nSA : 0, d_faceA, d_baryA,
                        d_gSA, d_gVB, &B->hdr()->status};
    ChamferGradSide b2a{A->faces(), A->verts(), (int)A->L.n_faces, d_SB, wantB ? nSB : 0, d_faceB, d_baryB,
                        d_gSB, d_gVA, &A->hdr()->status};
    k_chamfer_backward<<<nbA + nbB, block, 0, s>>>(a2b, b2a, nbA, d_g);
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
    return (h[0] & ~(unsigned)(MESH_DEV_DEGENERATE | MESH_DEV_DEEP_TREE)) ? MESH_ERR_DEVICE : MESH_OK;
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
