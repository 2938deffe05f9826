// Signed distance for contact (inside negative): the sign of (q - c) . N at
// the nearest point c, N the angle-weighted pseudo-normal of the feature c
// lies on (Baerentzen & Aanaes 2005) -- the face's unit normal in a face
// interior, the sum of the two faces' unit normals on an edge, the sum over
// the faces around a vertex of the unit normal times the face's angle there.
// Used for penetration depth on the physics side (the contact queries of
// Sec. 3.4 with a sign).  Needs a closed, consistently counter-clockwise
// (outward) manifold mesh; an edge with one face uses that face's normal.
//
// Face adjacency (the face across each edge) depends on the topology only and
// is built on the first call after a build: every half-edge is entered in an
// open-addressing table keyed by its two vertex ids (atomic compare-and-swap;
// probes bounded by the table size), then each half-edge reads its partner.
// The face normals depend on the vertices and are recomputed on every call;
// a vertex's pseudo-normal is summed where a query needs it, in ascending face
// id, so the signed distance is the same run to run.
#include <math.h>

#include "common.cuh"

namespace meshgs {

constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long edge_key(int x, int y) {
    unsigned lo = (unsigned)min(x, y), hi = (unsigned)max(x, y);
    return ((unsigned long long)lo << 32) | hi;
}

// 64-bit finaliser of MurmurHash3 (public domain), as the table's hash.
__device__ __forceinline__ unsigned hash64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return (unsigned)k;
}

__device__ __forceinline__ void half_edge(const int4 *__restrict__ faces, int he, int &x, int &y) {
    int4 fv = faces[he / 3];
    int v[3] = {fv.x, fv.y, fv.z};
    int k = he % 3;
    x = v[(k + 1) % 3];
    y = v[(k + 2) % 3];
}

__global__ void k_adj_insert(const int4 *__restrict__ faces, int nF, unsigned long long *keys, int *own,
                             int *oth, unsigned mask, Header *hdr) {
    int he = blockIdx.x * blockDim.x + threadIdx.x;
    if (he >= 3 * nF) return;
    int x, y;
    half_edge(faces, he, x, y);
    if (x == y) return;
    unsigned long long key = edge_key(x, y);
    unsigned h = hash64(key) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
        unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
        if (prev == kEmptyKey) { own[h] = he; return; }
        if (prev == key) {
            if (atomicCAS(&oth[h], -1, he) != -1) set_status(hdr, MESH_DEV_NONMANIFOLD);
            return;
        }
        h = (h + 1) & mask;
    }
}

__global__ void k_adj_resolve(const int4 *__restrict__ faces, int nF, const unsigned long long *__restrict__ keys,
                              const int *__restrict__ own, const int *__restrict__ oth, unsigned mask,
                              int *__restrict__ adj) {
    int he = blockIdx.x * blockDim.x + threadIdx.x;
    if (he >= 3 * nF) return;
    int x, y;
    half_edge(faces, he, x, y);
    int partner = -1;
    if (x != y) {
        unsigned long long key = edge_key(x, y);
        unsigned h = hash64(key) & mask;
        for (unsigned probe = 0; probe <= mask; ++probe) {
            unsigned long long kk = keys[h];
            if (kk == key) { int o = own[h]; partner = (o == he) ? oth[h] : o; break; }
            if (kk == kEmptyKey) break;
            h = (h + 1) & mask;
        }
    }
    adj[he] = partner >= 0 ? partner / 3 : -1;
}

// Unit face normals (the vertex pseudo-normals are summed where a query needs
// one, over the vertex's faces in ascending id: query.cu).
__global__ void k_face_normals(const int4 *__restrict__ faces, const float4 *__restrict__ verts, int nF,
                               float4 *__restrict__ fnorm) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    int4 fv = faces[f];
    int id[3] = {fv.x, fv.y, fv.z};
    float3 p[3];
    for (int j = 0; j < 3; ++j) { float4 t = verts[id[j]]; p[j] = make_float3(t.x, t.y, t.z); }
    float ex = p[1].x - p[0].x, ey = p[1].y - p[0].y, ez = p[1].z - p[0].z;
    float gx = p[2].x - p[0].x, gy = p[2].y - p[0].y, gz = p[2].z - p[0].z;
    float nx = ey * gz - ez * gy, ny = ez * gx - ex * gz, nz = ex * gy - ey * gx;
    float l = sqrtf(nx * nx + ny * ny + nz * nz);
    float s = l > 0.0f ? 1.0f / l : 0.0f;
    nx *= s; ny *= s; nz *= s;
    fnorm[f] = make_float4(nx, ny, nz, 0.0f);
}

struct AdjTable {
    unsigned long long *keys;
    int *own, *oth;
    unsigned slots;
    size_t bytes;
};

static AdjTable adj_table(void *ws, int64_t nF) {
    unsigned slots = 1;
    while ((int64_t)slots < 6 * (nF > 0 ? nF : 1)) slots <<= 1;
    AdjTable t;
    t.slots = slots;
    char *b = (char *)ws;
    t.keys = (unsigned long long *)b;
    t.own = (int *)(b + align_up(8 * (size_t)slots, 256));
    t.oth = (int *)(b + align_up(8 * (size_t)slots, 256) + align_up(4 * (size_t)slots, 256));
    t.bytes = align_up(8 * (size_t)slots, 256) + 2 * align_up(4 * (size_t)slots, 256);
    return t;
}

// In query.cu: NearestSurface plus the pseudo-normal sign.
mesh_status launch_signed_query(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                                int32_t *d_face, float *d_bary, float *d_point, float *d_sdist,
                                cudaStream_t s);

}  // namespace meshgs

using namespace meshgs;

extern "C" {

size_t mesh_signed_workspace_bytes(int64_t nF) {
    if (nF < 0 || nF > ((int64_t)1 << 28)) return 0;
    return adj_table(nullptr, nF).bytes;
}

mesh_status mesh_signed_distance(mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist, void *d_ws,
                                 size_t ws_bytes, int32_t *d_face, float *d_bary, float *d_point,
                                 float *d_sdist, void *stream) {
    if (!bvh || nQ < 0 || (nQ > 0 && (!d_Q || !d_sdist)) || !(max_dist >= 0.0f)) return MESH_ERR_INVALID_ARG;
    int n = (int)bvh->L.n_faces;
    if (n > (1 << 28)) return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0 && !bvh->adj_ready) {
        AdjTable t = adj_table(d_ws, n);
        if (!d_ws || ws_bytes < t.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
        cudaMemsetAsync(t.keys, 0xff, 8 * (size_t)t.slots, s);
        cudaMemsetAsync(t.oth, 0xff, 4 * (size_t)t.slots, s);
        k_adj_insert<<<grid_for(3 * (int64_t)n, 256), 256, 0, s>>>(bvh->faces(), n, t.keys, t.own, t.oth,
                                                                  t.slots - 1, bvh->hdr());
        k_adj_resolve<<<grid_for(3 * (int64_t)n, 256), 256, 0, s>>>(bvh->faces(), n, t.keys, t.own, t.oth,
                                                                   t.slots - 1, bvh->adj());
        count_launch(2);
        bvh->adj_ready = true;
    }
    if (n > 0) {
        k_face_normals<<<grid_for(n, 256), 256, 0, s>>>(bvh->faces(), bvh->verts(), n, bvh->fnorm());
        count_launch();
    }
    if (nQ == 0) return check_launch();
    return launch_signed_query(bvh, d_Q, nQ, max_dist, d_face, d_bary, d_point, d_sdist, s);
}

}  // extern "C"
