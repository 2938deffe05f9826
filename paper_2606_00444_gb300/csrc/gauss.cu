// Face-bound Gaussians of the rendering representation (Sec. 3.2).  The paper
// anchors Gaussians to mesh faces (Sec. 2, Sec. 3.1) but prints no formula;
// the face frame used here is: e1 along edge v0->v1, n the unit face normal,
// e2 = n x e1; centre = barycentric anchor plus a normal offset; rotation =
// quaternion of [e1 e2 n]; scale from the edge length and the altitude.
// One thread per Gaussian; face and vertex reads are float4 / int4 gathers
// from the BVH's vertex buffer and face table (shared with the collision side).
#include <math.h>

#include "common.cuh"
#include "gauss_math.cuh"

namespace meshgs {

// Gaussians per thread: each thread issues the loads of all of them (index,
// face, three vertices, weights) before computing any, so their dependent
// load chains overlap instead of waiting one after the other.  Gaussian k of
// thread t in block b is b * kBindBlock * kBindPer + k * kBindBlock + t, so
// every load and store stays coalesced across a warp.
constexpr int kBindBlock = 256;
constexpr int kBindPer = 2;

__global__ void __launch_bounds__(kBindBlock)
k_bind_gaussians(const int4 *__restrict__ faces, const float4 *__restrict__ verts, int nF,
                 const int *__restrict__ gface, const float *__restrict__ gbary,
                 const float *__restrict__ goff, int64_t nG, float *__restrict__ mu,
                 float *__restrict__ quat, float *__restrict__ scale, Header *hdr) {
    const int64_t base = (int64_t)blockIdx.x * (kBindBlock * kBindPer) + threadIdx.x;
    int f[kBindPer];
#pragma unroll
    for (int k = 0; k < kBindPer; ++k) {
        int64_t g = base + (int64_t)k * kBindBlock;
        f[k] = g < nG ? __ldg(gface + g) : -1;
    }
    float4 va[kBindPer], vb[kBindPer], vc[kBindPer];
    float w[kBindPer][4];
#pragma unroll
    for (int k = 0; k < kBindPer; ++k) {
        int64_t g = base + (int64_t)k * kBindBlock;
        int4 fv = (unsigned)f[k] < (unsigned)nF ? __ldg(faces + f[k]) : make_int4(0, 0, 0, 0);
        va[k] = __ldg(verts + fv.x);
        vb[k] = __ldg(verts + fv.y);
        vc[k] = __ldg(verts + fv.z);
        bool in = g < nG;
        w[k][0] = in ? __ldg(gbary + 3 * g) : 0.0f;
        w[k][1] = in ? __ldg(gbary + 3 * g + 1) : 0.0f;
        w[k][2] = in ? __ldg(gbary + 3 * g + 2) : 0.0f;
        w[k][3] = in && goff ? __ldg(goff + g) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < kBindPer; ++k) {
        int64_t g = base + (int64_t)k * kBindBlock;
        if (g >= nG) break;
        if ((unsigned)f[k] >= (unsigned)nF) { bind_invalid(g, mu, quat, scale, &hdr->status); continue; }
        bind_corners(v3(va[k]), v3(vb[k]), v3(vc[k]), w[k][0], w[k][1], w[k][2], w[k][3], g, mu, quat,
                     scale, &hdr->status, &hdr->n_degenerate);
    }
}

// Batched form: Gaussian g of scene s (gauss_off), face id local to s.  Grid-
// stride loop over all Gaussians of all scenes.
__global__ void k_batch_bind_gaussians(const int4 *__restrict__ faces, const float4 *__restrict__ verts,
                                       const int *__restrict__ face_off,
                                       const int *__restrict__ gauss_off, int nscenes,
                                       const int *__restrict__ gface,
                                       const float *__restrict__ gbary,
                                       const float *__restrict__ goff, int64_t nG,
                                       float *__restrict__ mu, float *__restrict__ quat,
                                       float *__restrict__ scale, BatchStatus *st) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nG;
         g += (int64_t)gridDim.x * blockDim.x) {
        int sc = segment_of(gauss_off, nscenes, g);
        int fb = __ldg(face_off + sc), ns = __ldg(face_off + sc + 1) - fb;
        int f = gface[g];
        if ((unsigned)f >= (unsigned)ns) { bind_invalid(g, mu, quat, scale, &st->status); continue; }
        bind_one(faces[fb + f], verts, gbary[3 * g], gbary[3 * g + 1], gbary[3 * g + 2],
                 goff ? goff[g] : 0.0f, g, mu, quat, scale, &st->status, &st->n_degenerate);
    }
}

__device__ __forceinline__ void add_grad(float *gV, int v, V3 g) {
    atomicAdd(gV + 3 * (size_t)v, g.x);
    atomicAdd(gV + 3 * (size_t)v + 1, g.y);
    atomicAdd(gV + 3 * (size_t)v + 2, g.z);
}

// VJP of the normalisation y = x / |x|: (g - y (y . g)) / |x|.
__device__ __forceinline__ V3 vjp_unit(V3 y, float len, V3 g) { return (g - y * dot(y, g)) * (1.0f / len); }

// Reverse mode of k_bind_gaussians with respect to the three face vertices.
__global__ void k_bind_gaussians_backward(const int4 *__restrict__ faces,
                                          const float4 *__restrict__ verts, int nF,
                                          const int *__restrict__ gface,
                                          const float *__restrict__ gbary,
                                          const float *__restrict__ goff, int64_t nG,
                                          const float *__restrict__ gmu,
                                          const float *__restrict__ gquat,
                                          const float *__restrict__ gscale, float *gV,
                                          Header *hdr) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nG) return;
    int f = gface[g];
    if ((unsigned)f >= (unsigned)nF) { set_status(hdr, MESH_DEV_INDEX_RANGE); return; }
    int4 fv = faces[f];
    V3 a = v3(verts[fv.x]), b = v3(verts[fv.y]), c = v3(verts[fv.z]);
    float b0 = gbary[3 * g], b1 = gbary[3 * g + 1], b2 = gbary[3 * g + 2];
    V3 Gmu = gmu ? V3{gmu[3 * g], gmu[3 * g + 1], gmu[3 * g + 2]} : V3{0.0f, 0.0f, 0.0f};
    V3 g0 = Gmu * b0, g1 = Gmu * b1, g2 = Gmu * b2;
    Frame F = face_frame(a, b, c);
    if (!F.degenerate) {
        float off = goff ? goff[g] : 0.0f;
        float R[3][3], raw[4], p;
        frame_matrix(F, R);
        int br = quat_raw(R, raw, p);
        float sg = quat_sign(raw);
        float G[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (gquat)
            for (int k = 0; k < 4; ++k) G[k] = sg * gquat[4 * g + k];
        float dR[3][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
        // raw[k] (k != pivot) = off_k / (4 p); raw[pivot] = p = sqrt(S) / 2
        float Gp = G[br];
        for (int k = 0; k < 4; ++k) {
            if (k == br) continue;
            float coef = G[k] / (4.0f * p);
            Gp -= G[k] * raw[k] / p;        // d raw_k / d p = -off_k / (4 p^2) = -raw_k / p
            int lo = min(br, k), hi = max(br, k);
            if (lo == 0 && hi == 1) { dR[2][1] += coef; dR[1][2] -= coef; }
            else if (lo == 0 && hi == 2) { dR[0][2] += coef; dR[2][0] -= coef; }
            else if (lo == 0 && hi == 3) { dR[1][0] += coef; dR[0][1] -= coef; }
            else if (lo == 1 && hi == 2) { dR[0][1] += coef; dR[1][0] += coef; }
            else if (lo == 1 && hi == 3) { dR[0][2] += coef; dR[2][0] += coef; }
            else { dR[1][2] += coef; dR[2][1] += coef; }
        }
        float gS = Gp / (8.0f * p);         // p = sqrt(S)/2  ->  dp/dS = 1/(8p)
        const float sgn[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        for (int d = 0; d < 3; ++d) dR[d][d] += gS * sgn[br][d];
        V3 ge1{dR[0][0], dR[1][0], dR[2][0]};
        V3 ge2{dR[0][1], dR[1][1], dR[2][1]};
        V3 gn{dR[0][2], dR[1][2], dR[2][2]};
        gn = gn + Gmu * off;
        float Gs0 = gscale ? gscale[3 * g] : 0.0f, Gs1 = gscale ? gscale[3 * g + 1] : 0.0f;
        float Gs2 = gscale ? gscale[3 * g + 2] : 0.0f;
        float gl = kRho * Gs0 + kEpsS * kRho * 0.5f * Gs2;
        float gh = kRho * Gs1 + kEpsS * kRho * 0.5f * Gs2;
        gl -= gh * F.an / (F.l * F.l);      // h = an / l
        float gan = gh / F.l;
        gn = gn + cross(F.e1, ge2);         // e2 = n x e1
        ge1 = ge1 + cross(ge2, F.n);
        V3 gnu = vjp_unit(F.n, F.an, gn) + F.nu * (gan / F.an);
        V3 ge = vjp_unit(F.e1, F.l, ge1) + F.e * (gl / F.l);
        ge = ge + cross(F.f, gnu);          // nu = e x f
        V3 gf = cross(gnu, F.e);
        g1 = g1 + ge;
        g2 = g2 + gf;
        g0 = g0 - (ge + gf);
    }
    add_grad(gV, fv.x, g0);
    add_grad(gV, fv.y, g1);
    add_grad(gV, fv.z, g2);
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

mesh_status mesh_bind_gaussians(const mesh_bvh *bvh, const int32_t *d_gface, const float *d_gbary,
                                const float *d_goff, int64_t nG, float *d_mu, float *d_quat,
                                float *d_scale, void *stream) {
    if (!bvh || nG < 0 || (nG > 0 && (!d_gface || !d_gbary || !d_mu || !d_quat || !d_scale)))
        return MESH_ERR_INVALID_ARG;
    if (nG == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_bind_gaussians<<<grid_for((nG + kBindPer - 1) / kBindPer, kBindBlock), kBindBlock, 0, s>>>(
        bvh->faces(), bvh->verts(), (int)bvh->L.n_faces, d_gface, d_gbary, d_goff, nG, d_mu, d_quat,
        d_scale, bvh->hdr());
    count_launch();
    return check_launch();
}

mesh_status mesh_batch_bind_gaussians(mesh_batch *batch, const int32_t *d_gface,
                                      const int32_t *d_gauss_off, const float *d_gbary,
                                      const float *d_goff, int64_t nG, float *d_mu,
                                      float *d_quat, float *d_scale, void *stream) {
    if (!batch || nG < 0 ||
        (nG > 0 && (!d_gface || !d_gauss_off || !d_gbary || !d_mu || !d_quat || !d_scale)))
        return MESH_ERR_INVALID_ARG;
    if (nG == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    int64_t want = (nG + 255) / 256;
    unsigned int grid = (unsigned int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    k_batch_bind_gaussians<<<grid, 256, 0, s>>>(batch->faces(), batch->verts(), batch->face_off(),
                                                d_gauss_off, (int)batch->L.n_scenes, d_gface, d_gbary,
                                                d_goff, nG, d_mu, d_quat, d_scale, batch->st());
    count_launch();
    return check_launch();
}

mesh_status mesh_bind_gaussians_backward(const mesh_bvh *bvh, const int32_t *d_gface,
                                         const float *d_gbary, const float *d_goff, int64_t nG,
                                         const float *d_gmu, const float *d_gquat,
                                         const float *d_gscale, float *d_gV, void *stream) {
    if (!bvh || nG < 0 || (nG > 0 && (!d_gface || !d_gbary || !d_gV))) return MESH_ERR_INVALID_ARG;
    if (nG == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_bind_gaussians_backward<<<grid_for(nG, 256), 256, 0, s>>>(
        bvh->faces(), bvh->verts(), (int)bvh->L.n_faces, d_gface, d_gbary, d_goff, nG, d_gmu,
        d_gquat, d_gscale, d_gV, bvh->hdr());
    count_launch();
    return check_launch();
}

}  // extern "C"
