// Face-bound Gaussian arithmetic (Sec. 3.2) shared by the rebind kernel and
// the refit pass that rebinds in place: the face frame (e1 along edge
// v0->v1, n the unit face normal, e2 = n x e1), the quaternion of [e1 e2 n]
// and the scale rule.  The paper anchors Gaussians to faces but prints no
// formula; these are the readings used throughout.
#pragma once

#include <math.h>

#include "common.cuh"

namespace meshgs {

constexpr float kRho = 1.0f / 3.0f;
constexpr float kEpsS = 1e-2f;

struct V3 {
    float x, y, z;
};
// Every product and sum is rounded on its own (no contraction into fused
// multiply-adds, whose choice of operands the compiler may make differently in
// different kernels): a face's frame and a Gaussian's centre come out the
// same, bit for bit, in every kernel that computes them.
__device__ __forceinline__ V3 v3(float4 a) { return V3{a.x, a.y, a.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) {
    return V3{__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z)};
}
__device__ __forceinline__ V3 operator-(V3 a, V3 b) {
    return V3{__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)};
}
__device__ __forceinline__ V3 operator*(V3 a, float s) {
    return V3{__fmul_rn(a.x, s), __fmul_rn(a.y, s), __fmul_rn(a.z, s)};
}
__device__ __forceinline__ float dot(V3 a, V3 b) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return V3{__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)), __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
              __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x))};
}

// Zero area: the float32 cross product decides when it is clearly non-zero
// (above its rounding bound); otherwise it is recomputed in float64, where
// products of float32 inputs are exact, so the answer is the exact one.
__device__ __forceinline__ bool zero_area(V3 e, V3 f, V3 nu) {
    float an2 = dot(nu, nu);
    if (an2 > 1e-10f * dot(e, e) * dot(f, f)) return false;
    double ex = e.x, ey = e.y, ez = e.z, fx = f.x, fy = f.y, fz = f.z;
    return (ey * fz - ez * fy) == 0.0 && (ez * fx - ex * fz) == 0.0 && (ex * fy - ey * fx) == 0.0;
}

struct Frame {
    V3 e, f, nu, e1, n, e2;
    float l, an;
    bool degenerate;
};

__device__ __forceinline__ Frame face_frame(V3 a, V3 b, V3 c) {
    Frame F;
    F.e = b - a;
    F.f = c - a;
    F.nu = cross(F.e, F.f);
    float l2 = dot(F.e, F.e);
    F.degenerate = (l2 == 0.0f) || zero_area(F.e, F.f, F.nu);
    if (F.degenerate) return F;
    F.l = sqrtf(l2);
    F.an = sqrtf(dot(F.nu, F.nu));
    F.e1 = F.e * (1.0f / F.l);
    F.n = F.nu * (1.0f / F.an);
    F.e2 = cross(F.n, F.e1);
    return F;
}

// Rotation-matrix -> quaternion by the largest of (trace, R00, R11, R22)
// (Shepperd 1978).  R columns are (e1, e2, n).  raw = (w, x, y, z) before the
// sign is fixed; returns the branch.
__device__ __forceinline__ int quat_raw(const float R[3][3], float raw[4], float &p) {
    float tr = R[0][0] + R[1][1] + R[2][2];
    int br;
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) br = 0;
    else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) br = 1;
    else if (R[1][1] >= R[2][2]) br = 2;
    else br = 3;
    if (br == 0) {
        p = 0.5f * sqrtf(1.0f + tr);
        float k = 0.25f / p;
        raw[0] = p; raw[1] = (R[2][1] - R[1][2]) * k; raw[2] = (R[0][2] - R[2][0]) * k;
        raw[3] = (R[1][0] - R[0][1]) * k;
    } else if (br == 1) {
        p = 0.5f * sqrtf(1.0f + R[0][0] - R[1][1] - R[2][2]);
        float k = 0.25f / p;
        raw[1] = p; raw[0] = (R[2][1] - R[1][2]) * k; raw[2] = (R[0][1] + R[1][0]) * k;
        raw[3] = (R[0][2] + R[2][0]) * k;
    } else if (br == 2) {
        p = 0.5f * sqrtf(1.0f - R[0][0] + R[1][1] - R[2][2]);
        float k = 0.25f / p;
        raw[2] = p; raw[0] = (R[0][2] - R[2][0]) * k; raw[1] = (R[0][1] + R[1][0]) * k;
        raw[3] = (R[1][2] + R[2][1]) * k;
    } else {
        p = 0.5f * sqrtf(1.0f - R[0][0] - R[1][1] + R[2][2]);
        float k = 0.25f / p;
        raw[3] = p; raw[0] = (R[1][0] - R[0][1]) * k; raw[1] = (R[0][2] + R[2][0]) * k;
        raw[2] = (R[1][2] + R[2][1]) * k;
    }
    return br;
}

// Sign that makes w > 0 (or, at w == 0, the first non-zero of x, y, z > 0).
__device__ __forceinline__ float quat_sign(const float raw[4]) {
    if (raw[0] != 0.0f) return raw[0] < 0.0f ? -1.0f : 1.0f;
    for (int k = 1; k < 4; ++k)
        if (raw[k] != 0.0f) return raw[k] < 0.0f ? -1.0f : 1.0f;
    return 1.0f;
}

__device__ __forceinline__ void frame_matrix(const Frame &F, float R[3][3]) {
    R[0][0] = F.e1.x; R[0][1] = F.e2.x; R[0][2] = F.n.x;
    R[1][0] = F.e1.y; R[1][1] = F.e2.y; R[1][2] = F.n.y;
    R[2][0] = F.e1.z; R[2][1] = F.e2.z; R[2][2] = F.n.z;
}

// The part of a binding that depends on the face alone: its unit normal, the
// rotation (w, x, y, z) of [e1 e2 n] and the scale; a degenerate face gets the
// identity rotation and zero scale.
struct FaceBind {
    V3 n;
    float q[4], s[3];
    bool degenerate;
};

__device__ __forceinline__ FaceBind face_bind(V3 a, V3 b, V3 c) {
    FaceBind B;
    Frame F = face_frame(a, b, c);
    B.degenerate = F.degenerate;
    B.n = F.degenerate ? V3{0.0f, 0.0f, 0.0f} : F.n;
    B.q[0] = 1.0f; B.q[1] = B.q[2] = B.q[3] = 0.0f;
    B.s[0] = B.s[1] = B.s[2] = 0.0f;
    if (!F.degenerate) {
        float R[3][3], p;
        frame_matrix(F, R);
        quat_raw(R, B.q, p);
        float sg = quat_sign(B.q);
        for (int k = 0; k < 4; ++k) B.q[k] *= sg;
        float h = F.an / F.l;
        B.s[0] = kRho * F.l;
        B.s[1] = kRho * h;
        B.s[2] = kEpsS * kRho * (F.l + h) * 0.5f;
    }
    return B;
}

// The part that depends on the Gaussian: its centre, at weights (b0, b1, b2)
// and offset `off` along the normal (no offset on a degenerate face).
__device__ __forceinline__ V3 gaussian_centre(V3 a, V3 b, V3 c, V3 n, bool degenerate, float b0, float b1,
                                              float b2, float off) {
    V3 m = a * b0 + b * b1 + c * b2;
    if (!degenerate) m = m + n * off;
    return m;
}

// Writes Gaussian g (centre m, the face's rotation and scale); a degenerate
// face is counted and flagged.
__device__ __forceinline__ void put_gaussian(int64_t g, V3 m, const float q[4], const float s[3], bool degenerate,
                                             float *__restrict__ mu, float *__restrict__ quat,
                                             float *__restrict__ scale, unsigned int *status,
                                             unsigned int *n_degenerate) {
    if (degenerate) {
        atomicAdd(n_degenerate, 1u);
        atomicOr(status, (unsigned)MESH_DEV_DEGENERATE);
    }
    mu[3 * g] = m.x; mu[3 * g + 1] = m.y; mu[3 * g + 2] = m.z;
    quat[4 * g] = q[0]; quat[4 * g + 1] = q[1]; quat[4 * g + 2] = q[2]; quat[4 * g + 3] = q[3];
    scale[3 * g] = s[0]; scale[3 * g + 1] = s[1]; scale[3 * g + 2] = s[2];
}

// Gaussian g on the face with corners (a, b, c), weights (b0, b1, b2), normal
// offset off: centre, rotation and scale written at index g.
__device__ __forceinline__ void bind_corners(V3 a, V3 b, V3 c, float b0, float b1, float b2, float off,
                                             int64_t g, float *__restrict__ mu, float *__restrict__ quat,
                                             float *__restrict__ scale, unsigned int *status,
                                             unsigned int *n_degenerate) {
    FaceBind B = face_bind(a, b, c);
    put_gaussian(g, gaussian_centre(a, b, c, B.n, B.degenerate, b0, b1, b2, off), B.q, B.s, B.degenerate, mu,
                 quat, scale, status, n_degenerate);
}

__device__ __forceinline__ void bind_one(int4 fv, const float4 *__restrict__ verts, float b0, float b1,
                                         float b2, float off, int64_t g, float *__restrict__ mu,
                                         float *__restrict__ quat, float *__restrict__ scale,
                                         unsigned int *status, unsigned int *n_degenerate) {
    bind_corners(v3(verts[fv.x]), v3(verts[fv.y]), v3(verts[fv.z]), b0, b1, b2, off, g, mu, quat, scale,
                 status, n_degenerate);
}

__device__ __forceinline__ void bind_invalid(int64_t g, float *mu, float *quat, float *scale,
                                             unsigned int *status) {
    atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE);
    mu[3 * g] = mu[3 * g + 1] = mu[3 * g + 2] = 0.0f;
    quat[4 * g] = 1.0f; quat[4 * g + 1] = quat[4 * g + 2] = quat[4 * g + 3] = 0.0f;
    scale[3 * g] = scale[3 * g + 1] = scale[3 * g + 2] = 0.0f;
}


}  // namespace meshgs
