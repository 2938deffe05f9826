// NearestSurface queries (Eq. 1 / Eq. 2, Sec. 3.3) and the Chamfer distance
// of Sec. 4.2, by traversal of the LBVH built in lbvh.cu.
//
// One thread per query.  A node record holds both children's boxes, so a
// visit is one 64-byte read that tests two boxes.  Leaf children (single
// faces) are tested on the spot; of two surviving internal children the
// nearer is entered and the farther pushed, with its box distance, on a
// per-thread stack kept in shared memory ([depth][thread], conflict free)
// that spills to a small local array.  Boxes are pruned against the tie
// window of the nearest distance found so far, widened by the float32 error
// bound of a computed distance, so no face whose computed distance could fall
// inside the final window is ever skipped.  The nearest face is the lowest id
// within that final window (see Best), the same for every tree, traversal
// order and warm start: a function of the query and the mesh alone.
#include <climits>
#include <math.h>

#include <mutex>

#include "common.cuh"

namespace meshgs {

constexpr int kQueryBlock = 128;
constexpr int kQueryMinBlocks = 8;    // 8 x 128 threads per SM: at most 64 registers
constexpr int kStackShared = 24;      // entries per thread in shared memory
constexpr int kStackTotal = kMaxTreeDepth;   // every tree is at most this deep: the Karras tree by
                                             // its bound (30 key bits + log2 nF + 1), the
                                             // agglomerative one by the build's depth check

__device__ __forceinline__ float box_d2(float3 q, float4 lo, float4 hi) {
    float dx = fmaxf(fmaxf(lo.x - q.x, q.x - hi.x), 0.0f);
    float dy = fmaxf(fmaxf(lo.y - q.y, q.y - hi.y), 0.0f);
    float dz = fmaxf(fmaxf(lo.z - q.z, q.z - hi.z), 0.0f);
    return dx * dx + dy * dy + dz * dz;
}

// MinMaxDist of Roussopoulos, Kelley & Vincent (1995) for a tight AABB: every
// face of the box touches the geometry inside it, so some primitive in the box
// lies within this distance of q.  It bounds the nearest distance from above
// before any triangle is tested and orders children whose boxes both contain q.
__device__ __forceinline__ float box_minmax_d2(float3 q, float4 lo, float4 hi) {
    float mx = 0.5f * (lo.x + hi.x), my = 0.5f * (lo.y + hi.y), mz = 0.5f * (lo.z + hi.z);
    float nx = q.x - (q.x <= mx ? lo.x : hi.x), fx = q.x - (q.x >= mx ? lo.x : hi.x);
    float ny = q.y - (q.y <= my ? lo.y : hi.y), fy = q.y - (q.y >= my ? lo.y : hi.y);
    float nz = q.z - (q.z <= mz ? lo.z : hi.z), fz = q.z - (q.z >= mz ? lo.z : hi.z);
    float f2x = fx * fx, f2y = fy * fy, f2z = fz * fz;
    float S = f2x + f2y + f2z;
    return fminf(fminf(S - f2x + nx * nx, S - f2y + ny * ny), S - f2z + nz * nz);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }

// Closest point of segment xy to p: parameter t in [0, 1] and squared distance.
// The residual is formed from p - x (small when p is near the segment), never
// from absolute coordinates, so its rounding scales with the segment length.
__device__ __forceinline__ float seg_d2(float3 p, float3 x, float3 y, float &t) {
    float3 d = sub3(y, x), xp = sub3(p, x);
    float L = dot3(d, d);
    t = 0.0f;
    if (L > 0.0f) t = fminf(fmaxf(dot3(xp, d) / L, 0.0f), 1.0f);
    float3 r = make_float3(xp.x - t * d.x, xp.y - t * d.y, xp.z - t * d.z);
    return dot3(r, r);
}

// Closest point on triangle abc to p (Ericson, Real-Time Collision Detection
// 5.1.5: Voronoi regions of vertices, edges, face).  Faces flagged as exactly
// zero-area at build / refit use the nearest of their three edges instead.
// Returns the squared distance and the barycentric weights (u, v, w).  The
// residual p - closest point is assembled from the vertex-relative vectors
// (p - a, b - a, ...), so float32 rounding is relative to the triangle's size,
// not to the magnitude of the coordinates.
__device__ __forceinline__ float tri_closest(float3 p, float3 a, float3 b, float3 c, bool degenerate,
                                             float &u, float &v, float &w) {
    if (degenerate) {
        float t0, t1, t2;
        float s0 = seg_d2(p, a, b, t0), s1 = seg_d2(p, b, c, t1), s2 = seg_d2(p, c, a, t2);
        if (s0 <= s1 && s0 <= s2) { u = 1.0f - t0; v = t0; w = 0.0f; return s0; }
        if (s1 <= s2) { u = 0.0f; v = 1.0f - t1; w = t1; return s1; }
        u = t2; v = 0.0f; w = 1.0f - t2;
        return s2;
    }
    float3 ab = sub3(b, a), ac = sub3(c, a);
    float3 ap = sub3(p, a);
    float d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0f && d2 <= 0.0f) { u = 1.0f; v = 0.0f; w = 0.0f; return dot3(ap, ap); }
    float3 bp = sub3(p, b);
    float d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0f && d4 <= d3) { u = 0.0f; v = 1.0f; w = 0.0f; return dot3(bp, bp); }
    float vc = d1 * d4 - d3 * d2;
    float3 r;
    if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
        float t = d1 / (d1 - d3);
        u = 1.0f - t; v = t; w = 0.0f;
        r = make_float3(ap.x - t * ab.x, ap.y - t * ab.y, ap.z - t * ab.z);
    } else {
        float3 cp = sub3(p, c);
        float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
        if (d6 >= 0.0f && d5 <= d6) { u = 0.0f; v = 0.0f; w = 1.0f; return dot3(cp, cp); }
        float vb = d5 * d2 - d1 * d6;
        if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
            float t = d2 / (d2 - d6);
            u = 1.0f - t; v = 0.0f; w = t;
            r = make_float3(ap.x - t * ac.x, ap.y - t * ac.y, ap.z - t * ac.z);
        } else {
            float va = d3 * d6 - d5 * d4;
            if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {
                float t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
                u = 0.0f; v = 1.0f - t; w = t;
                float3 bc = sub3(c, b);
                r = make_float3(bp.x - t * bc.x, bp.y - t * bc.y, bp.z - t * bc.z);
            } else {
                float s = 1.0f / (va + vb + vc);
                v = vb * s;
                w = vc * s;
                u = 1.0f - v - w;
                r = make_float3(ap.x - (ab.x * v + ac.x * w), ap.y - (ab.y * v + ac.y * w),
                                ap.z - (ab.z * v + ac.z * w));
            }
        }
    }
    return dot3(r, r);
}

// The same region test in float64, used only to recompute the weights of the
// winning face when float32 would lose them: a query far from the face relative
// to its shortest edge (weight error grows like eps32 * d / edge) or a sliver.
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 dof(float3 a) { return D3{a.x, a.y, a.z}; }

__device__ __noinline__ void tri_weights_f64(float3 pf, float3 af, float3 bf, float3 cf,
                                             bool degenerate, float &u, float &v, float &w) {
    D3 p = dof(pf), a = dof(af), b = dof(bf), c = dof(cf);
    double U, V, W;
    if (degenerate) {
        D3 P[3] = {a, b, c};
        double best = 1e300, bt = 0.0;
        int be = 0;
        for (int e = 0; e < 3; ++e) {
            D3 x = P[e], d = dsub(P[(e + 1) % 3], x), xp = dsub(p, x);
            double L = ddot(d, d), t = 0.0;
            if (L > 0.0) t = fmin(fmax(ddot(xp, d) / L, 0.0), 1.0);
            D3 r = D3{xp.x - t * d.x, xp.y - t * d.y, xp.z - t * d.z};
            double s = ddot(r, r);
            if (s < best) { best = s; bt = t; be = e; }
        }
        if (be == 0) { U = 1.0 - bt; V = bt; W = 0.0; }
        else if (be == 1) { U = 0.0; V = 1.0 - bt; W = bt; }
        else { U = bt; V = 0.0; W = 1.0 - bt; }
    } else {
        D3 ab = dsub(b, a), ac = dsub(c, a), ap = dsub(p, a), bp = dsub(p, b), cp = dsub(p, c);
        double d1 = ddot(ab, ap), d2 = ddot(ac, ap), d3 = ddot(ab, bp), d4 = ddot(ac, bp);
        double d5 = ddot(ab, cp), d6 = ddot(ac, cp);
        double vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
        if (d1 <= 0.0 && d2 <= 0.0) { U = 1.0; V = 0.0; W = 0.0; }
        else if (d3 >= 0.0 && d4 <= d3) { U = 0.0; V = 1.0; W = 0.0; }
        else if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) { double t = d1 / (d1 - d3); U = 1.0 - t; V = t; W = 0.0; }
        else if (d6 >= 0.0 && d5 <= d6) { U = 0.0; V = 0.0; W = 1.0; }
        else if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) { double t = d2 / (d2 - d6); U = 1.0 - t; V = 0.0; W = t; }
        else if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
            double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
            U = 0.0; V = 1.0 - t; W = t;
        } else {
            double s = 1.0 / (va + vb + vc);
            V = vb * s; W = vc * s; U = 1.0 - V - W;
        }
    }
    u = (float)U; v = (float)V; w = (float)W;
}

// True when float32 weights of this face would be too coarse for the query.
// Their error grows like ~8 eps32 d / l_min (measured), so beyond 12 shortest
// edges it could approach 1e-5; slivers (altitude < 5% of the longest edge)
// are ill-conditioned at any distance.  Float64 is slow on this part, so the
// threshold keeps the float64 path off near-surface queries entirely.
__device__ __forceinline__ bool weights_need_f64(float3 a, float3 b, float3 c, float d2) {
    float3 ab = sub3(b, a), ac = sub3(c, a), bc = sub3(c, b);
    float l0 = dot3(ab, ab), l1 = dot3(ac, ac), l2 = dot3(bc, bc);
    float lmin = fminf(l0, fminf(l1, l2)), lmax = fmaxf(l0, fmaxf(l1, l2));
    float3 n = make_float3(ab.y * ac.z - ab.z * ac.y, ab.z * ac.x - ab.x * ac.z, ab.x * ac.y - ab.y * ac.x);
    return d2 > 144.0f * lmin || dot3(n, n) < 2.5e-3f * lmax * lmax;
}

struct Hit {
    int leaf;      // -1: nothing within the cutoff
    int face;
    float d2;
};

// Float32 error bound of a computed point-triangle or point-box distance for a
// query q on a mesh whose coordinates are at most vmax in magnitude.  Every
// difference such as q - a is below 2 s in magnitude, s = max(|q|_inf, vmax),
// and the residual assembled from such differences (and the box distance)
// carries at most about 30 eps32 s of rounding; 2^-18 s = 64 eps32 s covers
// it with a margin.  Pruning widened by this bound never skips a face whose
// computed distance lies inside the tie window, whatever the tree.
constexpr float kSlackScale = 0x1p-18f;

struct Traversal {
    const float4 *__restrict__ nodes;
    const float4 *__restrict__ tris;
    int n;
    float tau;     // absolute floor of the tie window (1e-12 of the box diagonal)
    float vmax;    // largest coordinate magnitude of the mesh box
    bool mmd;      // use MinMaxDist bounds (unbounded queries; a cutoff is tighter)
    const float4 *__restrict__ wide;   // the 4-wide records (traversal variant 13)
};

__device__ __forceinline__ float query_slack(const Traversal &T, float3 q) {
    return kSlackScale * fmaxf(fmaxf(fabsf(q.x), fabsf(q.y)), fmaxf(fabsf(q.z), T.vmax));
}

// The two thresholds of a nearest squared distance m: w2, the tie window (a
// face with d2 <= w2 counts as equally near), and p2, the pruning radius (the
// window widened by the float32 bound `slack`, so a box whose computed
// distance exceeds p2 holds no face whose computed distance is within w2).
__device__ __forceinline__ void windows(float m, float tau, float slack, float &w2, float &p2) {
    float r = sqrtf(m) * (1.0f + kTieRel) + tau;
    w2 = r * r;
    r += slack;
    p2 = r * r;
}

// Pruning radius implied by an upper bound u2 on the nearest squared distance
// (a MinMaxDist): some face lies within sqrt(u2) in exact arithmetic, so the
// final nearest computed distance is at most sqrt(u2) + slack; u2 itself is
// widened by 4e-5 relative for its own rounding.
__device__ __forceinline__ float bound_window2(float u2, float tau, float slack) {
    float r = (sqrtf(u2 * 1.00004f) + slack) * (1.0f + kTieRel) + tau + slack;
    return r * r;
}

// Pruning radius before any hit: the cutoff itself, widened the same way
// (faces just past the cutoff can still fall in the tie window of a hit).
__device__ __forceinline__ float cutoff_window2(float maxd2, float tau, float slack) {
    if (isinf(maxd2)) return INFINITY;
    float r = sqrtf(maxd2) * (1.0f + kTieRel) + tau + slack;
    return r * r;
}

// Candidate bookkeeping of the tie rule.  dmin is the nearest squared
// distance seen; the kept face (leaf `leaf`, its face id read back from the
// packed triangle when a tie needs it) is the lowest id among the faces seen
// within the window of dmin -- as long as every face seen inside the current
// window, other than the kept one, has a higher id.  `other` is the least
// squared distance of the faces seen and not kept; when the kept face leaves
// the shrinking window while `other` is still inside it, one of those faces
// may have the lowest id, and `other` is set to -1: the query is resolved at
// the end by one search with the final window fixed (resolve_ties).  The
// answer is therefore the lowest id within the final window, whatever the
// order in which faces were met.  Five registers, as the search carries them
// through every node visit.
struct Best {
    int leaf;
    float d2, dmin, thr, other;
};

__device__ __forceinline__ int face_of(const Traversal &T, int leaf) {
    return __float_as_int(ldg4(T.tris + 3 * (size_t)leaf).w);
}

__device__ __forceinline__ Best make_best(const Traversal &T, float3 q, float maxd2) {
    return Best{-1, INFINITY, INFINITY, cutoff_window2(maxd2, T.tau, query_slack(T, q)), INFINITY};
}

__device__ __forceinline__ void consider(const Traversal &T, Best &B, float3 q, int leaf, int face,
                                         float d2, float maxd2) {
    float nmin = fminf(B.dmin, d2);
    if (nmin > maxd2) {                       // no hit yet and this face is past the cutoff:
        B.other = fminf(B.other, d2);         // noted only (it may fall in a later hit's window)
        return;
    }
    float w2, p2;
    windows(nmin, T.tau, query_slack(T, q), w2, p2);
    if (d2 <= w2) {
        if (B.leaf >= 0 && B.d2 <= w2) {      // the kept face stays inside the window: a tie
            if (leaf != B.leaf) {
                if (face < face_of(T, B.leaf)) {
                    B.other = fminf(B.other, B.d2);
                    B.leaf = leaf; B.d2 = d2;
                } else {
                    B.other = fminf(B.other, d2);
                }
            }
        } else {                              // first hit, or the kept face left the window
            if (B.other <= w2) B.other = -1.0f;
            B.leaf = leaf; B.d2 = d2;
        }
    }
    B.dmin = nmin;
    B.thr = fminf(B.thr, p2);
}

__device__ __forceinline__ void test_leaf(const Traversal &T, Best &B, int leaf, float3 q,
                                          float maxd2) {
    const float4 *t = T.tris + 3 * (size_t)leaf;
    float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
    float u, v, w;
    float d2 = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
    consider(T, B, q, leaf, __float_as_int(a.w), d2, maxd2);
}

// The faces of a leaf link: first = -link - 1, cnt from the record's hi.w (1
// without leaf collapse).  The first face's box is the link's box when cnt is
// 1; the others are tested against their own box first (computed from the
// corners just loaded), so a face far outside the window costs no region test.
// kRange = false (a tree without leaf collapse) compiles to the single face
// alone: the leaf-range loop costs the one-thread searches ~10 % even when
// every count is 1, so the kernels come in both forms and the host picks the
// plain one for leaf size 1.
template <bool kRange>
__device__ __forceinline__ void test_range(const Traversal &T, Best &B, int first, int cnt, float3 q,
                                           float maxd2) {
    if constexpr (!kRange) {
        test_leaf(T, B, first, q, maxd2);
        return;
    }
    // one call site of the region test; the per-face box test only runs for a
    // real range
#pragma unroll 1
    for (int k = 0; k < cnt; ++k) {
        const float4 *t = T.tris + 3 * (size_t)(first + k);
        float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
        if (cnt > 1) {
            float4 lo = make_float4(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                                    fminf(fminf(a.z, b.z), c.z), 0.0f);
            float4 hi = make_float4(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                                    fmaxf(fmaxf(a.z, b.z), c.z), 0.0f);
            if (box_d2(q, lo, hi) > B.thr) continue;
        }
        float u, v, w;
        float d2 = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
        consider(T, B, q, first + k, __float_as_int(a.w), d2, maxd2);
    }
}

__device__ __forceinline__ int link_count(float4 hi) { return __float_as_int(hi.w); }

// The tie rule with the window fixed: one depth-first search that visits every
// box within the pruning radius of B.dmin and keeps the lowest face id whose
// distance lies within its window.  Run only for the rare queries whose online
// bookkeeping could not decide (three or more faces within about 2e-6 of one
// another, met in an order that moved the window past the kept one).
__device__ __noinline__ void resolve_ties(const Traversal &T, Best &B, float3 q,
                                          unsigned int *status) {
    float w2, p2;
    windows(B.dmin, T.tau, query_slack(T, q), w2, p2);
    int bl = -1, bf = 0x7fffffff;
    float bd = INFINITY;
    auto test = [&](int leaf) {
        const float4 *t = T.tris + 3 * (size_t)leaf;
        float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
        float u, v, w;
        float d2 = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
        int f = __float_as_int(a.w);
        if (d2 <= w2 && f < bf) { bl = leaf; bf = f; bd = d2; }
    };
    if (T.n == 1) {
        test(0);
    } else if (T.n > 1) {
        int stk[kStackTotal];
        int sp = 0, node = 0;
        while (true) {
            const float4 *r = T.nodes + 4 * (size_t)node;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            bool il = box_d2(q, l0, l1) <= p2, ir = box_d2(q, r0, r1) <= p2;
            if (il && cl < 0)
                for (int k = 0; k < link_count(l1); ++k) test(-cl - 1 + k);
            if (ir && cr < 0)
                for (int k = 0; k < link_count(r1); ++k) test(-cr - 1 + k);
            bool gl = il && cl >= 0, gr = ir && cr >= 0;
            if (gl && gr) {
                if (sp < kStackTotal) stk[sp++] = cr;
                else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                node = cl;
                continue;
            }
            if (gl) { node = cl; continue; }
            if (gr) { node = cr; continue; }
            if (sp == 0) break;
            node = stk[--sp];
        }
    }
    if (bl >= 0) { B.leaf = bl; B.d2 = bd; }
    B.other = INFINITY;
}

__device__ __forceinline__ Hit finish(const Traversal &T, Best &B, float3 q, unsigned int *status) {
    if (B.other < 0.0f) resolve_ties(T, B, q, status);
    return Hit{B.leaf, B.leaf >= 0 ? face_of(T, B.leaf) : 0x7fffffff, B.d2};
}

// kSmem: stack entries per thread kept in shared memory (the rest spill to a
// local array; 0 = all local, leaving the SM's L1 to the node cache).
// kOneSite: leaf children are gathered and tested at one call site (the nearer
// first) instead of one site per child, so lanes testing a left and a right
// leaf in the same step run the same instructions together.
struct Counts {
    int visits, tests;
};

// hint_leaf >= 0: a leaf tested before the traversal (a warm start, e.g. the
// previous frame's nearest face); its distance bounds the search from the
// first node on.  Every leaf within the final tie window is still reached and
// the tie rule does not depend on the order, so the answer is the same as
// without the hint; only the work changes.
template <int kBlockT, int kSmem = kStackShared, bool kOneSite = false, bool kCount = false,
          bool kRange = false>
__device__ __forceinline__ Hit nearest(const Traversal &T, float3 q, float maxd2,
                                       int2 (*stk)[kBlockT], unsigned int *status,
                                       Counts *cnt = nullptr, int hint_leaf = -1) {
    Best B = make_best(T, q, maxd2);
    if (hint_leaf >= 0) test_leaf(T, B, hint_leaf, q, maxd2);
    if (T.n == 1) {
        if constexpr (kCount) cnt->tests++;
        test_leaf(T, B, 0, q, maxd2);
    } else if (T.n > 1) {
        int2 spill[kStackTotal - kSmem];
        int sp = 0;
        int node = 0;
        const int tid = threadIdx.x;
        while (true) {
            const float4 *r = T.nodes + 4 * (size_t)node;
            if constexpr (kCount) cnt->visits++;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            float ml = 0.0f, mr = 0.0f;
            if (T.mmd) {
                ml = box_minmax_d2(q, l0, l1);
                mr = box_minmax_d2(q, r0, r1);
                B.thr = fminf(B.thr, bound_window2(fminf(ml, mr), T.tau, query_slack(T, q)));
            }
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            if constexpr (kCount)
                cnt->tests += (cl < 0 && dl <= B.thr ? link_count(l1) : 0) +
                              (cr < 0 && dr <= B.thr ? link_count(r1) : 0);
            if constexpr (kOneSite) {
                bool tl = cl < 0 && dl <= B.thr, tr = cr < 0 && dr <= B.thr;
                int la = tl ? -cl - 1 : -cr - 1, lb = -cr - 1;
                int na = tl ? link_count(l1) : link_count(r1), nb = link_count(r1);
                bool two = tl && tr;
                if (two && dr < dl) { int t = la; la = lb; lb = t; t = na; na = nb; nb = t; }
#pragma unroll 1
                for (int k = 0; k < 2; ++k) {
                    if (k == 0 ? !(tl || tr) : !two) break;
                    test_range<kRange>(T, B, k == 0 ? la : lb, k == 0 ? na : nb, q, maxd2);
                }
            } else {
                if (cl < 0 && dl <= B.thr) test_range<kRange>(T, B, -cl - 1, link_count(l1), q, maxd2);
                if (cr < 0 && dr <= B.thr) test_range<kRange>(T, B, -cr - 1, link_count(r1), q, maxd2);
            }
            bool gl = cl >= 0 && dl <= B.thr;
            bool gr = cr >= 0 && dr <= B.thr;
            if (gl && gr) {
                bool lfirst = dl < dr || (dl == dr && ml <= mr);
                int2 e = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
                if (sp < kSmem) stk[sp][tid] = e;
                else if (sp < kStackTotal) spill[sp - kSmem] = e;
                else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                if (sp < kStackTotal) ++sp;
                node = lfirst ? cl : cr;
                continue;
            }
            if (gl) { node = cl; continue; }
            if (gr) { node = cr; continue; }
            bool found = false;
            while (sp > 0) {
                --sp;
                int2 e = sp < kSmem ? stk[sp][tid] : spill[sp - kSmem];
                if (__int_as_float(e.y) <= B.thr) { node = e.x; found = true; break; }
            }
            if (!found) break;
        }
    }
    return finish(T, B, q, status);
}

// Depth-first over the 4-wide records (variant 13): each visit tests up to four
// boxes -- the node's children, an internal child replaced by its own two --
// so a search takes about half the visits of the binary one, each reading one
// 128-byte record.  Leaf slots are tested first (they may shrink the window),
// then the internal slots still within it are ordered by box distance: the
// nearest is entered, the others pushed farthest first.  The pruning, the
// candidate bookkeeping and the tie rule are those of nearest(), so the answer
// is the same, bit for bit.  cnt->visits counts 4-wide records.
constexpr int kWideStack = 3 * kStackTotal / 2 + 2;   // up to 3 pushes per record, half the depth
constexpr int kWideEmpty = INT_MIN;

__device__ __forceinline__ void wide_swap(float &da, int &ca, float &db, int &cb) {
    if (db < da) {
        float t = da; da = db; db = t;
        int u = ca; ca = cb; cb = u;
    }
}

template <int kBlockT, int kSmem, bool kCount, bool kRange, bool kMmd>
__device__ __forceinline__ Hit nearest_wide_t(const Traversal &T, float3 q, float maxd2,
                                              int2 (*stk)[kBlockT], unsigned int *status, Counts *cnt,
                                              int hint_leaf) {
    Best B = make_best(T, q, maxd2);
    if (hint_leaf >= 0) test_leaf(T, B, hint_leaf, q, maxd2);
    if (T.n == 1) {
        if constexpr (kCount) cnt->tests++;
        test_leaf(T, B, 0, q, maxd2);
    } else if (T.n > 1) {
        const float4 *__restrict__ W = T.wide;
        int2 spill[kWideStack - kSmem];
        int sp = 0;
        int node = 0;
        const int tid = threadIdx.x % kBlockT;
        while (true) {
            const float4 *r = W + 8 * (size_t)node;
            if constexpr (kCount) cnt->visits++;
            const float4 lo0 = ldg4(r), hi0 = ldg4(r + 1), lo1 = ldg4(r + 2), hi1 = ldg4(r + 3), lo2 = ldg4(r + 4),
                         hi2 = ldg4(r + 5), lo3 = ldg4(r + 6), hi3 = ldg4(r + 7);
            float d0 = box_d2(q, lo0, hi0), d1 = box_d2(q, lo1, hi1), d2 = box_d2(q, lo2, hi2),
                  d3 = box_d2(q, lo3, hi3);
            int c0 = __float_as_int(lo0.w), c1 = __float_as_int(lo1.w), c2 = __float_as_int(lo2.w),
                c3 = __float_as_int(lo3.w);
            if constexpr (kMmd) {
                float u = INFINITY;
                if (c0 != kWideEmpty) u = fminf(u, box_minmax_d2(q, lo0, hi0));
                if (c1 != kWideEmpty) u = fminf(u, box_minmax_d2(q, lo1, hi1));
                if (c2 != kWideEmpty) u = fminf(u, box_minmax_d2(q, lo2, hi2));
                if (c3 != kWideEmpty) u = fminf(u, box_minmax_d2(q, lo3, hi3));
                B.thr = fminf(B.thr, bound_window2(u, T.tau, query_slack(T, q)));
            }
            // leaf slots (the face count of a leaf link is read only with leaf collapse)
            auto leaf = [&](int c, float d, float hw) {
                if (c < 0 && c != kWideEmpty && d <= B.thr) {
                    const int m = kRange ? __float_as_int(hw) : 1;
                    if constexpr (kCount) cnt->tests += m;
                    test_range<kRange>(T, B, -c - 1, m, q, maxd2);
                }
            };
            leaf(c0, d0, hi0.w);
            leaf(c1, d1, hi1.w);
            leaf(c2, d2, hi2.w);
            leaf(c3, d3, hi3.w);
            float k0 = (c0 >= 0 && d0 <= B.thr) ? d0 : INFINITY;
            float k1 = (c1 >= 0 && d1 <= B.thr) ? d1 : INFINITY;
            float k2 = (c2 >= 0 && d2 <= B.thr) ? d2 : INFINITY;
            float k3 = (c3 >= 0 && d3 <= B.thr) ? d3 : INFINITY;
            const int nin = (k0 < INFINITY) + (k1 < INFINITY) + (k2 < INFINITY) + (k3 < INFINITY);
            if (nin > 0) {
                wide_swap(k0, c0, k1, c1);
                wide_swap(k2, c2, k3, c3);
                wide_swap(k0, c0, k2, c2);
                wide_swap(k1, c1, k3, c3);
                wide_swap(k1, c1, k2, c2);
                auto push = [&](int c, float k) {
                    const int2 e = make_int2(c, __float_as_int(k));
                    if (sp < kSmem) stk[sp][tid] = e;
                    else if (sp < kWideStack) spill[sp - kSmem] = e;
                    else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                    if (sp < kWideStack) ++sp;
                };
                if (nin > 3) push(c3, k3);
                if (nin > 2) push(c2, k2);
                if (nin > 1) push(c1, k1);
                node = c0;
                continue;
            }
            bool found = false;
            while (sp > 0) {
                --sp;
                int2 e = sp < kSmem ? stk[sp][tid] : spill[sp - kSmem];
                if (__int_as_float(e.y) <= B.thr) { node = e.x; found = true; break; }
            }
            if (!found) break;
        }
    }
    return finish(T, B, q, status);
}

// (the MinMaxDist form, for unbounded queries, is a separate loop: the bounded
// one keeps the register budget of the search alone)
template <int kBlockT, int kSmem = 8, bool kCount = false, bool kRange = false>
__device__ __forceinline__ Hit nearest_wide(const Traversal &T, float3 q, float maxd2,
                                            int2 (*stk)[kBlockT], unsigned int *status,
                                            Counts *cnt = nullptr, int hint_leaf = -1) {
    if (T.mmd) return nearest_wide_t<kBlockT, kSmem, kCount, kRange, true>(T, q, maxd2, stk, status, cnt, hint_leaf);
    return nearest_wide_t<kBlockT, kSmem, kCount, kRange, false>(T, q, maxd2, stk, status, cnt, hint_leaf);
}

// The 4-wide records from the node records, one thread per (internal node,
// side): the record's half for that side is the child's own node record when the
// child is internal (its two children as two slots), else the node's slot for the
// leaf link and an empty slot -- a copy of 64 bytes.
__global__ void k_wide_update(const float4 *__restrict__ nodes, int nint, float4 *__restrict__ wide) {
    pdl_wait();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (int)(t >> 1), s = (int)(t & 1);
    if (n >= nint) return;
    const float4 a = __ldg(nodes + 4 * (size_t)n + 2 * s), b = __ldg(nodes + 4 * (size_t)n + 2 * s + 1);
    const int link = __float_as_int(a.w);
    float4 *w = wide + 8 * (size_t)n + 4 * s;
    if (link < 0) {
        w[0] = a;
        w[1] = b;
        w[2] = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(kWideEmpty));
        w[3] = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(0));
    } else {
        const float4 *c = nodes + 4 * (size_t)link;
        w[0] = __ldg(c);
        w[1] = __ldg(c + 1);
        w[2] = __ldg(c + 2);
        w[3] = __ldg(c + 3);
    }
}

// One thread per query, "while-while" form: internal nodes are traversed
// while leaf children are only queued (up to kLeafQueue); the queued leaves
// are tested when every lane still traversing has one queued (or its queue is
// full, or it is done).  Leaf tests then run with the warp mostly converged
// instead of in almost every step.  Same answers as nearest().
constexpr int kLeafQueue = 4;

template <int kBlockT>
__device__ __forceinline__ Hit nearest_ww(const Traversal &T, float3 q, float maxd2,
                                          int2 (*stk)[kBlockT], unsigned int *status) {
    Best B = make_best(T, q, maxd2);
    if (T.n == 1) {
        test_leaf(T, B, 0, q, maxd2);
        return Hit{B.leaf, B.leaf >= 0 ? face_of(T, B.leaf) : 0x7fffffff, B.d2};
    }
    if (T.n < 1) return Hit{-1, 0x7fffffff, INFINITY};
    int2 spill[kStackTotal - kStackShared];
    const int tid = threadIdx.x;
    int sp = 0, node = 0;
    bool done = false;
    int2 lq[kLeafQueue];                         // (first face, count) of each queued leaf link
    int nq = 0;
    while (true) {
        while (!done && nq + 2 <= kLeafQueue) {
            if (nq > 0 && __all_sync(__activemask(), nq > 0)) break;
            const float4 *r = T.nodes + 4 * (size_t)node;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            float ml = 0.0f, mr = 0.0f;
            if (T.mmd) {
                ml = box_minmax_d2(q, l0, l1);
                mr = box_minmax_d2(q, r0, r1);
                B.thr = fminf(B.thr, bound_window2(fminf(ml, mr), T.tau, query_slack(T, q)));
            }
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            if (cl < 0 && dl <= B.thr) lq[nq++] = make_int2(-cl - 1, link_count(l1));
            if (cr < 0 && dr <= B.thr) lq[nq++] = make_int2(-cr - 1, link_count(r1));
            bool gol = cl >= 0 && dl <= B.thr, gor = cr >= 0 && dr <= B.thr;
            if (gol && gor) {
                bool lfirst = dl < dr || (dl == dr && ml <= mr);
                int2 e = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
                if (sp < kStackShared) stk[sp][tid] = e;
                else if (sp < kStackTotal) spill[sp - kStackShared] = e;
                else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                if (sp < kStackTotal) ++sp;
                node = lfirst ? cl : cr;
                continue;
            }
            if (gol) { node = cl; continue; }
            if (gor) { node = cr; continue; }
            done = true;
            while (sp > 0) {
                --sp;
                int2 e = sp < kStackShared ? stk[sp][tid] : spill[sp - kStackShared];
                if (__int_as_float(e.y) <= B.thr) { node = e.x; done = false; break; }
            }
        }
        for (int k = 0; k < nq; ++k) test_range<false>(T, B, lq[k].x, lq[k].y, q, maxd2);
        nq = 0;
        if (done) break;
    }
    return finish(T, B, q, status);
}

// Depth-first search of the subtree under `start` by one thread with a
// local stack (the tree depth bounds it, so kStackTotal entries suffice),
// continuing the candidate state B.  Used by a cooperative group when its
// shared stack is nearly full.
template <bool kRange>
__device__ __noinline__ void dfs_private(const Traversal &T, Best &B, int start, float3 q,
                                         float maxd2, unsigned int *status) {
    int2 stk[kStackTotal];
    int sp = 0, node = start;
    while (true) {
        const float4 *r = T.nodes + 4 * (size_t)node;
        float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
        float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
        float ml = 0.0f, mr = 0.0f;
        if (T.mmd) {
            ml = box_minmax_d2(q, l0, l1);
            mr = box_minmax_d2(q, r0, r1);
            B.thr = fminf(B.thr, bound_window2(fminf(ml, mr), T.tau, query_slack(T, q)));
        }
        int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
        if (cl < 0 && dl <= B.thr) test_range<kRange>(T, B, -cl - 1, link_count(l1), q, maxd2);
        if (cr < 0 && dr <= B.thr) test_range<kRange>(T, B, -cr - 1, link_count(r1), q, maxd2);
        bool gl = cl >= 0 && dl <= B.thr, gr = cr >= 0 && dr <= B.thr;
        if (gl && gr) {
            bool lfirst = dl < dr || (dl == dr && ml <= mr);
            if (sp < kStackTotal) stk[sp++] = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
            else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
            node = lfirst ? cl : cr;
            continue;
        }
        if (gl) { node = cl; continue; }
        if (gr) { node = cr; continue; }
        bool found = false;
        while (sp > 0) {
            int2 e = stk[--sp];
            if (__int_as_float(e.y) <= B.thr) { node = e.x; found = true; break; }
        }
        if (!found) return;
    }
}

// ---------------------------------------------------------------------------
// Warp-cooperative NearestSurface: G lanes (an aligned group of a warp) share
// one query.  Each step the group pops up to G entries of its shared stack,
// every lane visits one node (testing its two child boxes and any leaf
// children), the group merges the leaf candidates under the tie rule with
// shuffles, and the surviving children are pushed back (each lane's nearer
// child above its farther one, lane 0's above lane 1's).  This keeps the GPU
// busy when there are too few queries for one thread each.  When the shared
// stack is nearly full each lane instead finishes its popped subtree alone
// (dfs_private), so no entry is ever dropped.  All collectives run on the full
// warp every step; groups that are done simply take nothing.
// ---------------------------------------------------------------------------
// shared-memory stack entries per group: room for one full step (2G pushes)
// above the near-full mark, plus a working depth
template <int G> __host__ __device__ constexpr int group_cap() { return 4 * G + 64; }

template <int G> __device__ __forceinline__ float grp_min(float x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
template <int G> __device__ __forceinline__ int grp_min(int x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
template <int G> __device__ __forceinline__ int grp_sum(int x) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
template <int G> __device__ __forceinline__ int grp_incl_scan(int x, int gl) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o, G);
        if (gl >= o) x += y;
    }
    return x;
}

// steps (when not NULL): the number of group steps this query took (its cost).
template <int G, bool kRange = false>
__device__ Hit nearest_group(const Traversal &T, float3 q, float maxd2, bool valid, int2 *stk,
                             unsigned int *status, int hint_leaf = -1, int *steps = nullptr) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    // The group's candidate state: the bookkeeping of consider(), identical in
    // every lane of the group (all updates come from group-wide reductions),
    // with the kept face's id in sface.  S.other here is only the undecided
    // flag (-1); the least distance of the faces not kept is accumulated per
    // lane (acc) and tested with one vote when it matters.
    Best S = make_best(T, q, maxd2);
    int sface = 0x7fffffff;
    float acc = INFINITY;
    int sp = 0;
    if (valid && T.n == 1) {
        test_leaf(T, S, 0, q, maxd2);
        if (S.leaf >= 0) sface = face_of(T, S.leaf);
    } else if (valid && T.n > 1) {
        // Greedy dive (every lane of the group on the same path): the nearer
        // child down to a leaf gives the parallel phase a tight window from
        // the start, so the shared stack stays small.  A warm-start face gives
        // that window without the dive (one serial step per tree level, with
        // every lane on the same node).
        int node = hint_leaf >= 0 ? -1 : 0;
        if (node < 0) test_leaf(T, S, hint_leaf, q, maxd2);
        while (node >= 0) {
            const float4 *r = T.nodes + 4 * (size_t)node;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            float ml = 0.0f, mr = 0.0f;
            if (T.mmd) { ml = box_minmax_d2(q, l0, l1); mr = box_minmax_d2(q, r0, r1); }
            bool lfirst = dl < dr || (dl == dr && ml <= mr);
            int c = lfirst ? __float_as_int(l0.w) : __float_as_int(r0.w);
            if (c >= 0) { node = c; continue; }
            test_range<kRange>(T, S, -c - 1, link_count(lfirst ? l1 : r1), q, maxd2);
            break;
        }
        if (S.leaf >= 0) sface = face_of(T, S.leaf);
        acc = S.other;                               // faces met and not kept
        S.other = S.other < 0.0f ? -1.0f : INFINITY;
        if (gl == 0) stk[0] = make_int2(0, __float_as_int(0.0f));
        sp = 1;
    }
    __syncwarp();
    int nsteps = 0;
    while (__any_sync(0xffffffffu, sp > 0)) {
        const bool near_full = sp > group_cap<G>() - 2 * G;
        const int take = min(G, sp);
        nsteps += take > 0;
        bool act = gl < take;
        int2 e = make_int2(0, 0);
        if (act) e = stk[sp - 1 - gl];
        __syncwarp();
        sp -= take;
        act = act && __int_as_float(e.y) <= S.thr;
        float c0 = INFINITY, c1 = INFINITY;
        int f0 = 0x7fffffff, f1 = 0x7fffffff, lf0 = -1, lf1 = -1;
        int npush = 0;
        float lane_ub = INFINITY, pother = INFINITY;
        bool lane_undecided = false;
        int2 p_far = make_int2(0, 0), p_near = make_int2(0, 0);
        if (act && !near_full) {
            const float4 *r = T.nodes + 4 * (size_t)e.x;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            float ml = 0.0f, mr = 0.0f;
            if (T.mmd) {
                ml = box_minmax_d2(q, l0, l1);
                mr = box_minmax_d2(q, r0, r1);
                lane_ub = fminf(ml, mr);
            }
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            bool tl = cl < 0 && dl <= S.thr, tr = cr < 0 && dr <= S.thr;
            if (kRange && ((tl && link_count(l1) > 1) || (tr && link_count(r1) > 1))) {
                // leaf ranges: the lane keeps its own candidate under the tie rule and
                // notes the faces it did not keep
                Best P = S;
                P.leaf = -1; P.d2 = INFINITY; P.other = INFINITY;
                if (tl) test_range<kRange>(T, P, -cl - 1, link_count(l1), q, maxd2);
                if (tr) test_range<kRange>(T, P, -cr - 1, link_count(r1), q, maxd2);
                if (P.leaf >= 0) { c0 = P.d2; f0 = face_of(T, P.leaf); lf0 = P.leaf; }
                pother = P.other;
                lane_undecided = P.other < 0.0f;
            } else {
                // single faces: each goes to the merge as a candidate
                float u, v, w;
                if (tl) {
                    lf0 = -cl - 1;
                    const float4 *t = T.tris + 3 * (size_t)lf0;
                    float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
                    c0 = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
                    f0 = __float_as_int(a.w);
                }
                if (tr) {
                    lf1 = -cr - 1;
                    const float4 *t = T.tris + 3 * (size_t)lf1;
                    float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
                    c1 = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
                    f1 = __float_as_int(a.w);
                }
            }
            bool gol = cl >= 0 && dl <= S.thr, gor = cr >= 0 && dr <= S.thr;
            if (gol && gor) {
                bool lfirst = dl < dr || (dl == dr && ml <= mr);
                p_near = make_int2(lfirst ? cl : cr, __float_as_int(lfirst ? dl : dr));
                p_far = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
                npush = 2;
            } else if (gol) {
                p_near = make_int2(cl, __float_as_int(dl));
                npush = 1;
            } else if (gor) {
                p_near = make_int2(cr, __float_as_int(dr));
                npush = 1;
            }
        } else if (act) {
            Best P = S;                          // the group's window and bounds, no kept face
            P.leaf = -1; P.d2 = INFINITY; P.other = INFINITY;
            dfs_private<kRange>(T, P, e.x, q, maxd2, status);
            if (P.leaf >= 0) { c0 = P.d2; f0 = face_of(T, P.leaf); lf0 = P.leaf; }
            pother = P.other;
            lane_undecided = P.other < 0.0f;
        }
        // Merge the step's candidates into S (consider() for a set of faces at
        // once).  Every reduction runs on the full warp, outside any branch.
        float m = grp_min<G>(fminf(c0, c1));
        float ub = grp_min<G>(lane_ub);
        float nmin = fminf(S.dmin, m);
        const bool hit = nmin <= maxd2;
        float w2 = -1.0f, p2 = INFINITY;
        if (hit) windows(nmin, T.tau, query_slack(T, q), w2, p2);
        int fc = min(c0 <= w2 ? f0 : 0x7fffffff, c1 <= w2 ? f1 : 0x7fffffff);
        int fmin = grp_min<G>(fc);
        bool mine = fmin != 0x7fffffff && fc == fmin;
        unsigned bal = __ballot_sync(0xffffffffu, mine) & gmask;
        int src = bal ? (__ffs(bal) - 1) & (G - 1) : 0;
        float md2 = (c0 <= w2 && f0 == fmin) ? c0 : c1;
        int mlf = (c0 <= w2 && f0 == fmin) ? lf0 : lf1;
        float sd2 = __shfl_sync(0xffffffffu, md2, src, G);
        int slf = __shfl_sync(0xffffffffu, mlf, src, G);
        const bool stays = S.leaf >= 0 && S.d2 <= w2;          // the kept face is still inside
        const int kept = (stays && sface <= fmin) ? sface : fmin;
        // undecided when a lane's own search was, or when the kept face leaves the
        // window while a face met earlier and not kept is still inside it
        bool undecided = (__ballot_sync(0xffffffffu, lane_undecided || (hit && !stays && acc <= w2)) &
                          gmask) != 0u;
        if (undecided) S.other = -1.0f;
        acc = fminf(acc, pother);              // faces of this step not kept: higher ids than kept
        if (f0 != kept) acc = fminf(acc, c0);
        if (f1 != kept) acc = fminf(acc, c1);
        if (hit) {
            if (kept != sface) {
                if (stays) acc = fminf(acc, S.d2);
                S.leaf = slf; sface = fmin; S.d2 = sd2;
            }
            S.dmin = nmin;
            S.thr = fminf(S.thr, p2);
        }
        S.thr = fminf(S.thr, bound_window2(ub, T.tau, query_slack(T, q)));
        // push surviving children: lane G-1's lowest, lane 0's on top
        int total = grp_sum<G>(npush);
        int above = total - grp_incl_scan<G>(npush, gl);
        if (npush == 2) { stk[sp + above] = p_far; stk[sp + above + 1] = p_near; }
        else if (npush == 1) { stk[sp + above] = p_near; }
        sp += total;
        __syncwarp();
    }
    // only the group's first lane writes the result, so only it resolves
    if (valid && gl == 0 && S.other < 0.0f) {
        resolve_ties(T, S, q, status);
        sface = S.leaf >= 0 ? face_of(T, S.leaf) : 0x7fffffff;
    }
    if (steps) *steps = nsteps;
    return Hit{S.leaf, sface, S.d2};
}

// Per-mesh constants of the tie rule from the mesh box: the window's absolute
// floor (1e-12 of the box diagonal) and the largest coordinate magnitude.
__device__ __forceinline__ void set_scale(Traversal &T, float4 lo, float4 hi) {
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    T.tau = kTieAbs * sqrtf(dx * dx + dy * dy + dz * dz);
    T.vmax = fmaxf(fmaxf(fmaxf(fabsf(lo.x), fabsf(hi.x)), fmaxf(fabsf(lo.y), fabsf(hi.y))),
                   fmaxf(fabsf(lo.z), fabsf(hi.z)));
    if (!(T.vmax < INFINITY)) T.vmax = 0.0f;   // empty mesh: an inverted (infinite) box
}
__device__ __forceinline__ void set_scale(Traversal &T, const Header *hdr) {
    set_scale(T, hdr->root_lo, hdr->root_hi);
}

// The weights and closest point of a hit on leaf `leaf` (squared distance d2),
// recomputed from the packed triangle.
__device__ __forceinline__ void write_weights(const Traversal &T, int leaf, float d2, float3 q, int64_t i,
                                              float *bary, float *point) {
    const float4 *t = T.tris + 3 * (size_t)leaf;
    float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
    float u, v, w;
    tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
    if (weights_need_f64(xyz(a), xyz(b), xyz(c), d2))
        tri_weights_f64(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
    if (bary) { bary[3 * i] = u; bary[3 * i + 1] = v; bary[3 * i + 2] = w; }
    if (point) {
        point[3 * i] = u * a.x + v * b.x + w * c.x;
        point[3 * i + 1] = u * a.y + v * b.y + w * c.y;
        point[3 * i + 2] = u * a.z + v * b.z + w * c.z;
    }
}

// The weights of the contact step, after its search (which writes face and
// distance only): one thread per query, so the recomputation of a hit's weights
// no longer holds a search warp until its last lane is done.  Same values as
// write_hit.
__global__ void __launch_bounds__(256)
k_hit_weights(Traversal T, const float *__restrict__ Q, int64_t nQ, const int *__restrict__ face,
              const float *__restrict__ dist2, const int *__restrict__ iperm, float *bary, float *point) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nQ) return;
    const int f = face[i];
    if (f < 0) {
        if (bary) { bary[3 * i] = 0.0f; bary[3 * i + 1] = 0.0f; bary[3 * i + 2] = 0.0f; }
        if (point) { point[3 * i] = 0.0f; point[3 * i + 1] = 0.0f; point[3 * i + 2] = 0.0f; }
        return;
    }
    const float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);
    write_weights(T, __ldg(iperm + f), dist2[i], q, i, bary, point);
}

// Writes the outputs of one query (recomputing the weights of the winning face).
__device__ __forceinline__ void write_hit(const Traversal &T, const Hit &h, float3 q, int64_t i,
                                          int *face, float *bary, float *point, float *dist2) {
    if (h.leaf < 0) {
        if (face) face[i] = -1;
        if (dist2) dist2[i] = INFINITY;
        if (bary) { bary[3 * i] = 0.0f; bary[3 * i + 1] = 0.0f; bary[3 * i + 2] = 0.0f; }
        if (point) { point[3 * i] = 0.0f; point[3 * i + 1] = 0.0f; point[3 * i + 2] = 0.0f; }
        return;
    }
    if (face) face[i] = h.face;
    if (dist2) dist2[i] = h.d2;
    if (bary || point) write_weights(T, h.leaf, h.d2, q, i, bary, point);
}

// kMode: 0 depth-first, 1 while-while, 2 depth-first with one leaf-test site,
// 3 depth-first over the 4-wide records.
// kMinBlocks: resident blocks per SM the register budget must allow
// (8 -> 64 registers, 9 -> 56, 12 -> 40, 16 -> 32; fewer registers, more warps
// to hide latency, more spilling).
// Work class of a query from its node visits, heaviest first (the contact step
// orders the next step's queries by it): 0: 48 or more, 1: 24-47, 2: 12-23, 3: fewer.
__device__ __forceinline__ unsigned int work_class(int visits) {
    return visits >= 48 ? 0u : visits >= 24 ? 1u : visits >= 12 ? 2u : 3u;
}

// kRecord: also count the node visits of each query and store its work class
// in cls[i] (the contact step).
// kBlock: threads per block (128, or 64 / 32 with the same register budget: the
// same warps per SM in finer blocks, so a block whose warps finish early frees
// its slot sooner -- the searches of one block end at very different times).
template <int kSmem, int kMode, int kMinBlocks = kQueryMinBlocks, bool kRecord = false,
          int kBlock = kQueryBlock, bool kRange = false>
__global__ void __launch_bounds__(kBlock, kMinBlocks * kQueryBlock / kBlock)
k_closest_point(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                const float *__restrict__ Q, int64_t nQ, float maxd2, int *face, float *bary,
                float *point, float *dist2, const int *hint, const int *__restrict__ iperm,
                const int *__restrict__ order = nullptr, unsigned int *__restrict__ cls = nullptr) {
    __shared__ int2 stk[kSmem > 0 ? kSmem : 1][kBlock];
    pdl_wait();
    int64_t k = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (k >= nQ) return;
    const int64_t i = order ? (int64_t)order[k] : k;       // order: a permutation of the queries
    set_scale(T, hdr);
    float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);
    int hint_leaf = -1;
    if (hint) {                                   // may alias face: read before the write below
        int hf = hint[i];
        if (hf >= 0 && hf < T.n) hint_leaf = __ldg(iperm + hf);
    }
    Hit h;
    if constexpr (kRecord) {
        static_assert(kMode != 1, "the recording form uses the depth-first traversal");
        Counts c{0, 0};
        if constexpr (kMode == 3) {          // a 4-wide record counts as two binary visits
            h = nearest_wide<kBlock, kSmem, true, kRange>(T, q, maxd2, stk, status, &c, hint_leaf);
            cls[i] = work_class(2 * c.visits);
        } else {
            h = nearest<kBlock, kSmem, kMode == 2, true, kRange>(T, q, maxd2, stk, status, &c, hint_leaf);
            cls[i] = work_class(c.visits);
        }
    } else if constexpr (kMode == 1) {
        static_assert(!kRange, "the while-while form has no leaf-range instantiation");
        h = nearest_ww<kBlock>(T, q, maxd2, stk, status);
    } else if constexpr (kMode == 3) {
        h = nearest_wide<kBlock, kSmem, false, kRange>(T, q, maxd2, stk, status, nullptr, hint_leaf);
    } else {
        h = nearest<kBlock, kSmem, kMode == 2, false, kRange>(T, q, maxd2, stk, status, nullptr, hint_leaf);
    }
    write_hit(T, h, q, i, face, bary, point, dist2);
}

// Warp-packet traversal: the 32 queries of a warp (consecutive, so nearby
// when the caller keeps them in Morton order) share one depth-first node
// sequence.  Each lane tests the node's two child boxes against its own query
// and bound; a child is entered when any lane needs it, nearer-first by a
// vote of the lanes, and the other child is deferred on a per-warp stack of
// (parent, side) entries.  A deferred child is re-tested against the lanes'
// bounds when it is popped (bounds only shrink), so a lane sees every leaf
// its own traversal would.  Node loads are warp-uniform (one broadcast per
// record) and all control flow outside the leaf tests is warp-uniform: the
// warp runs the union of its queries' traversals with every lane active,
// instead of each lane's traversal with most lanes idle.  Same answers as the
// depth-first kernels.
// hint_leaf >= 0 warm-starts the lane as in nearest(); visits (when not NULL)
// counts the nodes whose children this lane needed (its share of the work).
template <bool kRange>
__device__ __forceinline__ Hit nearest_packet(const Traversal &T, float3 q, float maxd2, bool valid,
                                              int *wstk, unsigned int *status, int hint_leaf = -1,
                                              int *visits = nullptr) {
    const unsigned int kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    Best B = make_best(T, q, maxd2);
    if (!valid) B.thr = -1.0f;                   // a lane past the end prunes everything
    if (valid && hint_leaf >= 0) test_leaf(T, B, hint_leaf, q, maxd2);
    if (T.n == 1) {
        if (valid) test_leaf(T, B, 0, q, maxd2);
        return Hit{B.leaf, B.leaf >= 0 ? face_of(T, B.leaf) : 0x7fffffff, B.d2};
    }
    if (T.n < 1) return Hit{-1, 0x7fffffff, INFINITY};
    int sp = 0, node = 0;
    while (true) {
        const float4 *r = T.nodes + 4 * (size_t)node;
        float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
        float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
        if (T.mmd && valid)
            B.thr = fminf(B.thr, bound_window2(fminf(box_minmax_d2(q, l0, l1), box_minmax_d2(q, r0, r1)),
                                               T.tau, query_slack(T, q)));
        int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
        bool wl = dl <= B.thr, wr = dr <= B.thr;
        if (visits) *visits += (wl || wr);
        unsigned int bl = __ballot_sync(kFull, wl), br = __ballot_sync(kFull, wr);
        if (cl < 0 && wl) test_range<kRange>(T, B, -cl - 1, link_count(l1), q, maxd2);
        if (cr < 0 && wr) test_range<kRange>(T, B, -cr - 1, link_count(r1), q, maxd2);
        bool gl = cl >= 0 && bl != 0u, gr = cr >= 0 && br != 0u;
        if (gl && gr) {
            unsigned int pl = __ballot_sync(kFull, wl && (!wr || dl <= dr));
            bool lfirst = 2 * __popc(pl) >= __popc(bl | br);
            if (sp < kStackTotal) {
                if (lane == 0) wstk[sp] = 2 * node + (lfirst ? 1 : 0);
                ++sp;
            } else if (lane == 0) {
                atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
            }
            node = lfirst ? cl : cr;
            continue;
        }
        if (gl) { node = cl; continue; }
        if (gr) { node = cr; continue; }
        bool found = false;
        __syncwarp();
        while (sp > 0) {
            --sp;
            int e = wstk[sp];
            const float4 *pr = T.nodes + 4 * (size_t)(e >> 1) + 2 * (e & 1);
            float4 lo = ldg4(pr), hi = ldg4(pr + 1);
            if (__any_sync(kFull, box_d2(q, lo, hi) <= B.thr)) {
                node = __float_as_int(lo.w);
                found = true;
                break;
            }
        }
        __syncwarp();
        if (!found) break;
    }
    return finish(T, B, q, status);
}

// hint / iperm: warm start as k_closest_point.  order: the queries' order (a
// permutation; NULL = as stored).  kRecord: also store each query's work class
// in cls (the contact step).
template <bool kRecord = false, bool kRange = false>
__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_closest_point_packet(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                       const float *__restrict__ Q, int64_t nQ, float maxd2, int *face, float *bary,
                       float *point, float *dist2, const int *hint, const int *__restrict__ iperm,
                       const int *__restrict__ order = nullptr, unsigned int *__restrict__ cls = nullptr) {
    __shared__ int wstk[kQueryBlock / 32][kStackTotal];
    pdl_wait();
    const int64_t w0 = (int64_t)blockIdx.x * kQueryBlock + (threadIdx.x & ~31);
    if (w0 >= nQ) return;                                  // whole warp past the end
    const int64_t k = w0 + (threadIdx.x & 31);
    const bool valid = k < nQ;
    const int64_t i = valid && order ? (int64_t)order[k] : k;
    set_scale(T, hdr);
    float3 q = valid ? make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]) : make_float3(0.0f, 0.0f, 0.0f);
    int hint_leaf = -1;
    if (valid && hint) {                          // may alias face: read before the write below
        int hf = hint[i];
        if (hf >= 0 && hf < T.n) hint_leaf = __ldg(iperm + hf);
    }
    int visits = 0;
    Hit h = nearest_packet<kRange>(T, q, maxd2, valid, wstk[threadIdx.x >> 5], status, hint_leaf,
                                   kRecord ? &visits : nullptr);
    if (valid) {
        write_hit(T, h, q, i, face, bary, point, dist2);
        if constexpr (kRecord) cls[i] = work_class(visits);
    }
}

// k-NN weighted surface projection: the NearestSurface of temporal tracking
// (Sec. 3.3, Strategy 1, Eq. 1).  The paper names the method without k or
// weights; here: the k faces nearest to the query (ties by the lower face
// id), each giving its closest point p_j at distance d_j, blended with
// weights 1 / max(d_j, 1e-6 x box diagonal); optionally mixed with an anchor
// point, (1 - a) v' + a anchor (the periodic re-anchoring to the template).
// One thread per query; the k best (distance, face) are kept sorted in
// registers by a fixed compare-and-swap cascade, and a node is pruned when
// its box is farther than the current k-th distance (with 1e-5 relative
// slack, so equal-distance faces with lower ids are still reached).
constexpr int kKnnMax = 8;

__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_knn_project(Traversal T, const Header *__restrict__ hdr, const float *Q, int64_t nQ, int k,
              const float *anchor, float anchor_w, float *point, int *face_out, float *d2_out,
              unsigned int *status) {
    int64_t i = (int64_t)blockIdx.x * kQueryBlock + threadIdx.x;
    if (i >= nQ) return;
    const float4 rlo = hdr->root_lo, rhi = hdr->root_hi;
    const float dx = rhi.x - rlo.x, dy = rhi.y - rlo.y, dz = rhi.z - rlo.z;
    const float delta = 1e-6f * sqrtf(dx * dx + dy * dy + dz * dz);
    const float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);   // may alias point
    float bd[kKnnMax];
    int bf[kKnnMax], bl[kKnnMax];
#pragma unroll
    for (int j = 0; j < kKnnMax; ++j) { bd[j] = INFINITY; bf[j] = 0x7fffffff; bl[j] = -1; }
    float thr = INFINITY;
    int cnt = 0;
    auto consider_leaf = [&](int leaf) {
        const float4 *t = T.tris + 3 * (size_t)leaf;
        float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
        float u, v, w;
        float cd = tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
        int cf = __float_as_int(a.w), cl = leaf;
#pragma unroll
        for (int j = 0; j < kKnnMax; ++j) {
            if (j < k && (cd < bd[j] || (cd == bd[j] && cf < bf[j]))) {
                float td = bd[j]; bd[j] = cd; cd = td;
                int tf = bf[j]; bf[j] = cf; cf = tf;
                int tl = bl[j]; bl[j] = cl; cl = tl;
            }
        }
        if (cnt < k) ++cnt;
#pragma unroll
        for (int j = 0; j < kKnnMax; ++j)
            if (j == k - 1) thr = bd[j];
    };
    if (T.n == 1) {
        consider_leaf(0);
    } else if (T.n > 1) {
        int2 stk[kStackTotal];
        int sp = 0, node = 0;
        while (true) {
            const float4 *r = T.nodes + 4 * (size_t)node;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float lim = thr * 1.00001f;
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            if (cl < 0 && dl <= lim) {
                for (int m = 0; m < link_count(l1); ++m) consider_leaf(-cl - 1 + m);
                lim = thr * 1.00001f;
            }
            if (cr < 0 && dr <= lim) {
                for (int m = 0; m < link_count(r1); ++m) consider_leaf(-cr - 1 + m);
                lim = thr * 1.00001f;
            }
            bool gl = cl >= 0 && dl <= lim, gr = cr >= 0 && dr <= lim;
            if (gl && gr) {
                bool lfirst = dl <= dr;
                if (sp < kStackTotal) stk[sp++] = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
                else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                node = lfirst ? cl : cr;
                continue;
            }
            if (gl) { node = cl; continue; }
            if (gr) { node = cr; continue; }
            bool found = false;
            while (sp > 0) {
                int2 e = stk[--sp];
                if (__int_as_float(e.y) <= thr * 1.00001f) { node = e.x; found = true; break; }
            }
            if (!found) break;
        }
    }
    float sw = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
    for (int j = 0; j < kKnnMax; ++j) {
        if (j < cnt) {
            const float4 *t = T.tris + 3 * (size_t)bl[j];
            float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
            float u, v, w;
            tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
            float wt = 1.0f / fmaxf(sqrtf(bd[j]), delta);
            sw += wt;
            ax += wt * (u * a.x + v * b.x + w * c.x);
            ay += wt * (u * a.y + v * b.y + w * c.y);
            az += wt * (u * a.z + v * b.z + w * c.z);
        }
        if (j < k) {
            if (face_out) face_out[i * k + j] = j < cnt ? bf[j] : -1;
            if (d2_out) d2_out[i * k + j] = j < cnt ? bd[j] : INFINITY;
        }
    }
    float px = cnt > 0 ? ax / sw : q.x, py = cnt > 0 ? ay / sw : q.y, pz = cnt > 0 ? az / sw : q.z;
    if (anchor) {
        px = (1.0f - anchor_w) * px + anchor_w * anchor[3 * i];
        py = (1.0f - anchor_w) * py + anchor_w * anchor[3 * i + 1];
        pz = (1.0f - anchor_w) * pz + anchor_w * anchor[3 * i + 2];
    }
    point[3 * i] = px;
    point[3 * i + 1] = py;
    point[3 * i + 2] = pz;
}

// Angle-weighted pseudo-normal of vertex vid (Baerentzen & Aanaes 2005): the
// sum over the faces around it of the unit face normal times the face's angle
// at the vertex.  The ring is found from face f through the face adjacency
// (for a consistently oriented mesh, crossing the edge that follows the vertex
// in each face turns one way round it; an open ring is also walked the other
// way from f), up to kMaxRing faces, and summed in ascending face id, so the
// result is the same whichever face the walk starts from and run to run.  A
// ring larger than kMaxRing (or one the adjacency cannot close) sets
// MESH_DEV_NONMANIFOLD and sums the faces found.
constexpr int kMaxRing = 32;

__device__ __forceinline__ int slot_of(int4 fv, int vid) {
    return fv.x == vid ? 0 : (fv.y == vid ? 1 : (fv.z == vid ? 2 : -1));
}

__device__ __forceinline__ float4 vertex_pseudo_normal(const int4 *__restrict__ faces, const int *__restrict__ adj,
                                                    const float4 *__restrict__ verts,
                                                    const float4 *__restrict__ fnorm, int f, int vid,
                                                    unsigned int *status) {
    int ring[kMaxRing];
    int nr = 0;
    bool full = false;
    int g = f;
    while (true) {                                   // one way round
        ring[nr++] = g;
        int k = slot_of(faces[g], vid);
        int h = k < 0 ? -1 : adj[3 * g + (k + 2) % 3];
        if (h == f) break;
        if (h < 0) break;
        if (nr == kMaxRing) { full = true; break; }
        g = h;
    }
    if (!full && nr < kMaxRing) {                     // open ring: the other way from f
        int k0 = slot_of(faces[f], vid);
        int h = k0 < 0 ? -1 : adj[3 * f + (k0 + 1) % 3];
        bool closed = false;
        for (int i = 0; i < nr; ++i) closed |= ring[i] == h;
        while (h >= 0 && !closed) {
            if (nr == kMaxRing) { full = true; break; }
            ring[nr++] = h;
            int k = slot_of(faces[h], vid);
            int nh = k < 0 ? -1 : adj[3 * h + (k + 1) % 3];
            for (int i = 0; i < nr; ++i) closed |= ring[i] == nh;
            h = nh;
        }
    }
    if (full) atomicOr(status, (unsigned)MESH_DEV_NONMANIFOLD);
    float nx = 0.0f, ny = 0.0f, nz = 0.0f;
    int last = -1;
    for (int done = 0; done < nr; ++done) {          // ascending face id (distinct ids)
        int pick = 0x7fffffff;
        for (int i = 0; i < nr; ++i)
            if (ring[i] > last && ring[i] < pick) pick = ring[i];
        if (pick == 0x7fffffff) break;
        last = pick;
        int4 fv = faces[pick];
        int k = slot_of(fv, vid);
        if (k < 0) continue;
        int id[3] = {fv.x, fv.y, fv.z};
        float4 p = verts[id[k]], a = verts[id[(k + 1) % 3]], b = verts[id[(k + 2) % 3]];
        float ax = a.x - p.x, ay = a.y - p.y, az = a.z - p.z;
        float bx = b.x - p.x, by = b.y - p.y, bz = b.z - p.z;
        float la = sqrtf(ax * ax + ay * ay + az * az), lb = sqrtf(bx * bx + by * by + bz * bz);
        if (la == 0.0f || lb == 0.0f) continue;
        float cs = fminf(1.0f, fmaxf(-1.0f, (ax * bx + ay * by + az * bz) / (la * lb)));
        float ang = acosf(cs);
        float4 n = fnorm[pick];
        nx += ang * n.x; ny += ang * n.y; nz += ang * n.z;
    }
    return make_float4(nx, ny, nz, 0.0f);
}

// NearestSurface plus the sign of (q - c) . N, N the pseudo-normal of the
// feature the nearest point lies on: face interior (no zero weight), edge
// opposite vertex k (weight k zero), vertex (two zero weights).
// 8 shared stack entries per thread (the contact queries' best one-thread form).
constexpr int kSignedStack = 8;

template <bool kRange>
__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_signed_distance(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                  const float *__restrict__ Q, int64_t nQ, float maxd2, const int4 *__restrict__ faces,
                  const int *__restrict__ adj, const float4 *__restrict__ fnorm,
                  const float4 *__restrict__ verts, int *face, float *bary, float *point, float *sdist) {
    __shared__ int2 stk[kSignedStack][kQueryBlock];
    int64_t i = (int64_t)blockIdx.x * kQueryBlock + threadIdx.x;
    if (i >= nQ) return;
    set_scale(T, hdr);
    float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);
    Hit h = nearest<kQueryBlock, kSignedStack, false, false, kRange>(T, q, maxd2, stk, status);
    write_hit(T, h, q, i, face, bary, point, nullptr);
    if (h.leaf < 0) { sdist[i] = INFINITY; return; }
    const float4 *t = T.tris + 3 * (size_t)h.leaf;
    float4 a = ldg4(t), b = ldg4(t + 1), c = ldg4(t + 2);
    float u, v, w;
    tri_closest(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
    if (weights_need_f64(xyz(a), xyz(b), xyz(c), h.d2))
        tri_weights_f64(q, xyz(a), xyz(b), xyz(c), b.w != 0.0f, u, v, w);
    int f = h.face;
    int zeros = (u == 0.0f) + (v == 0.0f) + (w == 0.0f);
    float4 N;
    if (zeros == 0) {
        N = fnorm[f];
    } else if (zeros == 1) {
        int k = u == 0.0f ? 0 : (v == 0.0f ? 1 : 2);
        N = fnorm[f];
        int g = adj[3 * f + k];
        if (g >= 0) { float4 m = fnorm[g]; N.x += m.x; N.y += m.y; N.z += m.z; }
    } else {
        int4 fv = faces[f];
        int vid = u != 0.0f ? fv.x : (v != 0.0f ? fv.y : fv.z);
        N = vertex_pseudo_normal(faces, adj, verts, fnorm, f, vid, status);
    }
    float cx = u * a.x + v * b.x + w * c.x, cy = u * a.y + v * b.y + w * c.y, cz = u * a.z + v * b.z + w * c.z;
    float dn = (q.x - cx) * N.x + (q.y - cy) * N.y + (q.z - cz) * N.z;
    sdist[i] = (dn >= 0.0f ? 1.0f : -1.0f) * sqrtf(h.d2);
}

mesh_status launch_signed_query(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                                int32_t *d_face, float *d_bary, float *d_point, float *d_sdist,
                                cudaStream_t s);

// Persistent depth-first traversal with dynamic fetch (Aila & Laine 2009):
// a fixed grid of warps; each lane works through a stream of queries, one
// node visit per step, and when at least kRefill lanes of the warp are idle
// the warp takes that many new query indices from a global counter.  Lanes no
// longer wait for the slowest query of their warp (contact queries near the
// surface need ~6x the visits of those far from it).  Same answers as the
// depth-first kernels.
// The counter lives in the mesh header (zeroed before each launch), so
// concurrent calls on one handle must not overlap.
constexpr int kRefill = 8;

template <int kSmem>
__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_closest_point_persistent(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                           const float *__restrict__ Q, int64_t nQ, float maxd2, int *face,
                           float *bary, float *point, float *dist2, unsigned int *work) {
    __shared__ int2 stk[kSmem > 0 ? kSmem : 1][kQueryBlock];
    int2 spill[kStackTotal - kSmem];
    const int lane = threadIdx.x & 31, tid = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    set_scale(T, hdr);
    int64_t qi = -1;
    float3 q = make_float3(0.f, 0.f, 0.f);
    Best B = make_best(T, q, maxd2);
    int node = 0, sp = 0;
    bool exhausted = false;
    while (true) {
        bool fin = false;
        unsigned idle = __ballot_sync(0xffffffffu, qi < 0);
        if (!exhausted && (__popc(idle) >= kRefill || idle == 0xffffffffu)) {
            unsigned int base = 0, want = __popc(idle);
            if (lane == 0) base = atomicAdd(work, want);
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((int64_t)base + want >= nQ) exhausted = true;
            if (qi < 0) {
                int64_t cand = (int64_t)base + __popc(idle & lt);
                if (cand < nQ) {
                    qi = cand;
                    q = make_float3(Q[3 * qi], Q[3 * qi + 1], Q[3 * qi + 2]);
                    B = make_best(T, q, maxd2);
                    node = 0;
                    sp = 0;
                    if (T.n <= 1) {                      // no internal node to visit
                        if (T.n == 1) test_leaf(T, B, 0, q, maxd2);
                        fin = true;
                    }
                }
            }
        }
        // every lane reaches this vote each iteration (a full-warp collective
        // must never sit on a path only some lanes take)
        const bool all_idle = __all_sync(0xffffffffu, qi < 0);
        if (all_idle && exhausted) break;
        if (qi < 0) continue;
        if (!fin) {                                      // one node visit
            const float4 *r = T.nodes + 4 * (size_t)node;
            float4 l0 = ldg4(r), l1 = ldg4(r + 1), r0 = ldg4(r + 2), r1 = ldg4(r + 3);
            float dl = box_d2(q, l0, l1), dr = box_d2(q, r0, r1);
            float ml = 0.0f, mr = 0.0f;
            if (T.mmd) {
                ml = box_minmax_d2(q, l0, l1);
                mr = box_minmax_d2(q, r0, r1);
                B.thr = fminf(B.thr, bound_window2(fminf(ml, mr), T.tau, query_slack(T, q)));
            }
            int cl = __float_as_int(l0.w), cr = __float_as_int(r0.w);
            if (cl < 0 && dl <= B.thr) test_range<false>(T, B, -cl - 1, link_count(l1), q, maxd2);
            if (cr < 0 && dr <= B.thr) test_range<false>(T, B, -cr - 1, link_count(r1), q, maxd2);
            bool gol = cl >= 0 && dl <= B.thr, gor = cr >= 0 && dr <= B.thr;
            if (gol && gor) {
                bool lfirst = dl < dr || (dl == dr && ml <= mr);
                int2 e = make_int2(lfirst ? cr : cl, __float_as_int(lfirst ? dr : dl));
                if (sp < kSmem) stk[sp][tid] = e;
                else if (sp < kStackTotal) spill[sp - kSmem] = e;
                else atomicOr(status, (unsigned)MESH_DEV_STACK_OVERFLOW);
                if (sp < kStackTotal) ++sp;
                node = lfirst ? cl : cr;
            } else if (gol) {
                node = cl;
            } else if (gor) {
                node = cr;
            } else {
                fin = true;
                while (sp > 0) {
                    --sp;
                    int2 e = sp < kSmem ? stk[sp][tid] : spill[sp - kSmem];
                    if (__int_as_float(e.y) <= B.thr) { node = e.x; fin = false; break; }
                }
            }
        }
        if (fin) {
            write_hit(T, finish(T, B, q, status), q, qi, face, bary, point, dist2);
            qi = -1;
        }
    }
}

// Counting form of the one-thread depth-first traversal (same visiting order
// as variants 0, 2 and 3): node visits, triangle tests and hits, summed over
// all queries.  Separate instantiation; the timed kernels carry no counters.
// kWide: the traversal over the 4-wide records (its visits count records).
template <bool kRange, bool kWide = false>
__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_closest_point_count(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                      const float *__restrict__ Q, int64_t nQ, float maxd2,
                      unsigned long long *counts) {
    __shared__ int2 stk[kStackShared][kQueryBlock];
    int64_t i = (int64_t)blockIdx.x * kQueryBlock + threadIdx.x;
    Counts c{0, 0};
    int hit = 0;
    if (i < nQ) {
        set_scale(T, hdr);
        float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);
        Hit h;
        if constexpr (kWide)
            h = nearest_wide<kQueryBlock, kStackShared, true, kRange>(T, q, maxd2, stk, status, &c);
        else
            h = nearest<kQueryBlock, kStackShared, false, true, kRange>(T, q, maxd2, stk, status, &c);
        hit = h.leaf >= 0;
    }
    unsigned long long v = c.visits, t = c.tests, k = hit;
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
        k += __shfl_xor_sync(0xffffffffu, k, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, v);
        atomicAdd(counts + 1, t);
        atomicAdd(counts + 2, k);
    }
}

template <int G, bool kRange = false>
__global__ void __launch_bounds__(kQueryBlock)
k_closest_point_group(Traversal T, const Header *__restrict__ hdr, unsigned int *status,
                      const float *__restrict__ Q, int64_t nQ, float maxd2, int *face, float *bary,
                      float *point, float *dist2, const int *hint, const int *__restrict__ iperm) {
    __shared__ int2 gstk[kQueryBlock / G][group_cap<G>()];
    int64_t i = ((int64_t)blockIdx.x * kQueryBlock + threadIdx.x) / G;
    bool valid = i < nQ;
    set_scale(T, hdr);
    float3 q = valid ? make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]) : make_float3(0.f, 0.f, 0.f);
    int hint_leaf = -1;
    if (valid && hint) {                          // every lane of the group reads it before any write
        int hf = hint[i];
        if (hf >= 0 && hf < T.n) hint_leaf = __ldg(iperm + hf);
    }
    Hit h = nearest_group<G, kRange>(T, q, maxd2, valid, gstk[threadIdx.x / G], status, hint_leaf);
    if (valid && (threadIdx.x & (G - 1)) == 0) write_hit(T, h, q, i, face, bary, point, dist2);
}

// Batched NearestSurface: one persistent launch for the queries of every
// scene.  Each warp takes the next 32 queries from a counter, each thread
// finds its query's scene (binary search of the offsets) and traverses that
// scene's tree; face ids are returned scene-local.
__global__ void __launch_bounds__(kQueryBlock, kQueryMinBlocks)
k_batch_closest_point(const float4 *__restrict__ nodes, const float4 *__restrict__ tris,
                      const float4 *__restrict__ scene_box, const int *__restrict__ face_off,
                      const int *__restrict__ query_off, int nscenes, const float *__restrict__ Q,
                      int64_t nQ, float maxd2, bool mmd, int *face, float *bary, float *point,
                      float *dist2, unsigned int *status, unsigned int *work) {
    __shared__ int2 stk[kStackShared][kQueryBlock];
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned int base = 0;
        if (lane == 0) base = atomicAdd(work, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((int64_t)base >= nQ) break;
        int64_t i = (int64_t)base + lane;
        if (i < nQ) {
            int sc = segment_of(query_off, nscenes, i);
            int fb = __ldg(face_off + sc), ns = __ldg(face_off + sc + 1) - fb;
            Traversal T{nodes + 4 * (size_t)fb, tris + 3 * (size_t)fb, ns, 0.0f, 0.0f, mmd};
            set_scale(T, scene_box[2 * sc], scene_box[2 * sc + 1]);
            float3 q = make_float3(Q[3 * i], Q[3 * i + 1], Q[3 * i + 2]);
            Hit h = nearest<kQueryBlock>(T, q, maxd2, stk, status);
            if (h.leaf >= 0) h.face -= fb;
            write_hit(T, h, q, i, face, bary, point, dist2);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Chamfer (Sec. 4.2): both directions in one launch (blocks [0, nbA) query SA
// against B, the rest SB against A).  Each block sums its squared distances in
// float64 with a fixed reduction tree and stores the partial; the last block
// to finish (ticket counter) adds the partials in a fixed order, writes the
// two means and resets the counter, so the result is bit-reproducible.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_d(double x, double *s) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s[w] = x;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s[k];
    __syncthreads();
    return t;
}

struct ChamferSide {
    Traversal T;
    const Header *hdr;
    const float *S;
    int64_t n;
    int *face;
    float *bary, *dist2;
    const int *hint = nullptr;     // warm start: a face id per sample (-1 = none), may alias face
    const int *iperm = nullptr;    // face -> leaf of the mesh searched
    // The ordered form (mesh_chamfer_step): slot k runs sample order[k] - base,
    // and each sample's sort key -- key_side | (127 - its cost, at least 0),
    // heaviest first -- goes to key[sample] for the next call's order.
    const int *order = nullptr;
    int base = 0;
    unsigned int *key = nullptr;
    unsigned int key_side = 0;
};

// Sort key of a Chamfer sample from its cost (node visits / 8 with one lane,
// group steps with several): lower keys first, so the heaviest run first.
__device__ __forceinline__ unsigned int chamfer_key(unsigned int side, int cost) {
    return side | (unsigned int)(127 - min(127, cost));
}

template <int G, bool kRange = false>
__global__ void __launch_bounds__(kQueryBlock, G == 1 ? kQueryMinBlocks : 1)
k_chamfer(ChamferSide A2B, ChamferSide B2A, unsigned int nbA, unsigned int *status,
          double *partial, unsigned int *ticket, double *out) {
    constexpr int kStk = G == 1 ? kStackShared * kQueryBlock : (kQueryBlock / G) * group_cap<G>();
    __shared__ int2 stk_mem[kStk];
    __shared__ double s_red[kQueryBlock / 32];
    __shared__ bool s_last;
    pdl_wait();
    bool first = blockIdx.x < nbA;
    ChamferSide &C = first ? A2B : B2A;
    int64_t i = ((int64_t)(first ? blockIdx.x : blockIdx.x - nbA) * kQueryBlock + threadIdx.x) / G;
    double d2 = 0.0;
    Traversal T = C.T;
    set_scale(T, C.hdr);
    bool valid = i < C.n;
    if (valid && C.order) i = (int64_t)C.order[i] - C.base;   // a permutation of this side's samples
    float3 q = valid ? make_float3(C.S[3 * i], C.S[3 * i + 1], C.S[3 * i + 2])
                     : make_float3(0.f, 0.f, 0.f);
    int hint_leaf = -1;
    if (valid && C.hint) {
        int hf = C.hint[i];
        if (hf >= 0 && hf < T.n) hint_leaf = __ldg(C.iperm + hf);
    }
    if constexpr (G == 1) {
        if (valid) {
            auto stk = reinterpret_cast<int2 (*)[kQueryBlock]>(stk_mem);
            Hit h;
            if (C.key) {
                Counts c{0, 0};
                h = nearest<kQueryBlock, kStackShared, false, true, kRange>(T, q, INFINITY, stk, status, &c,
                                                                            hint_leaf);
                C.key[i] = chamfer_key(C.key_side, c.visits >> 3);
            } else {
                h = nearest<kQueryBlock, kStackShared, false, false, kRange>(T, q, INFINITY, stk, status, nullptr,
                                                                             hint_leaf);
            }
            write_hit(T, h, q, i, C.face, C.bary, nullptr, C.dist2);
            d2 = h.leaf >= 0 ? (double)h.d2 : 0.0;
        }
    } else {
        int steps = 0;
        Hit h = nearest_group<G, kRange>(T, q, INFINITY, valid, stk_mem + (threadIdx.x / G) * group_cap<G>(),
                                         status, hint_leaf, C.key ? &steps : nullptr);
        if (valid && (threadIdx.x & (G - 1)) == 0) {
            write_hit(T, h, q, i, C.face, C.bary, nullptr, C.dist2);
            d2 = h.leaf >= 0 ? (double)h.d2 : 0.0;
            if (C.key) C.key[i] = chamfer_key(C.key_side, steps);
        }
    }
    double s = block_sum_d(d2, s_red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // fixed-order final sums: thread k adds partials k, k + blockDim, ... of each side
    double a = 0.0, b = 0.0;
    for (unsigned int k = threadIdx.x; k < nbA; k += blockDim.x) a += __ldcg(partial + k);
    for (unsigned int k = nbA + threadIdx.x; k < gridDim.x; k += blockDim.x) b += __ldcg(partial + k);
    a = block_sum_d(a, s_red);
    b = block_sum_d(b, s_red);
    if (threadIdx.x == 0) {
        out[0] = A2B.n > 0 ? a / (double)A2B.n : 0.0;
        out[1] = B2A.n > 0 ? b / (double)B2A.n : 0.0;
        *ticket = 0u;
    }
}

__global__ void k_interpolate(const int4 *__restrict__ faces, const float4 *__restrict__ verts,
                              int nF, const int *__restrict__ face, const float *__restrict__ bary,
                              int64_t n, float *__restrict__ out, unsigned int *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int f = face[i];
    if ((unsigned)f >= (unsigned)nF) {
        atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE);
        out[3 * i] = out[3 * i + 1] = out[3 * i + 2] = 0.0f;
        return;
    }
    int4 fv = faces[f];
    float4 a = verts[fv.x], b = verts[fv.y], c = verts[fv.z];
    float u = bary[3 * i], v = bary[3 * i + 1], w = bary[3 * i + 2];
    out[3 * i] = u * a.x + v * b.x + w * c.x;
    out[3 * i + 1] = u * a.y + v * b.y + w * c.y;
    out[3 * i + 2] = u * a.z + v * b.z + w * c.z;
}

static Traversal traversal_of(const mesh_bvh *b, bool mmd = true) {
    return Traversal{b->nodes(), b->tris(), (int)b->L.n_faces, 0.0f, 0.0f, mmd, b->wide()};
}

// The 4-wide records written from the node records: by every build or refit of a
// handle whose traversal is variant 13 (so a captured refit carries the update),
// and otherwise by the first variant-13 query after the records went stale
// (host-side flag; the update runs on that query's stream, ahead of it).
static void ensure_wide(const mesh_bvh *b, cudaStream_t s) {
    if (!b->wide_valid) wide_refresh(b, s, false);
}

}  // namespace meshgs

void meshgs::wide_refresh(const mesh_bvh *b, cudaStream_t s, bool pdl) {
    const int nint = (int)b->L.n_faces - 1;
    if (nint > 0) {
        launch_ex(pdl, k_wide_update, grid_for(2 * (int64_t)nint, 256), 256, 0, s, (const float4 *)b->nodes(), nint,
                  b->wide());
        count_launch();
    }
    b->wide_valid = true;
}

namespace meshgs {

static size_t chamfer_blocks(int64_t n, int G = 1) {
    return (size_t)((n * G + kQueryBlock - 1) / kQueryBlock);
}

// Lanes per query: one thread per query when there are enough queries to fill
// the GPU (two resident blocks of threads per SM), otherwise the smallest power
// of two G <= 32 that does.  (An explicit override can come from
// mesh_set_query_group.)
// The one-thread searches' weights in their own launch after the search (k_hit_weights).
constexpr bool kContactSplitWeights = true;

static int g_group_override = 0;
static int g_traversal = 0;          // one-thread traversal variant, see mesh_set_traversal

bool wide_wanted(const mesh_bvh *b) {
    return (b->cfg_variant >= 0 ? b->cfg_variant : g_traversal) == 13 && b->cfg_lanes <= 1;
}
static int pick_group(int64_t nQ) {
    if (g_group_override > 0) return g_group_override;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    int64_t target = (int64_t)sms * 2048;
    if (nQ >= target || nQ <= 0) return 1;
    int G = 1;
    while (G < 32 && nQ * G < target) G <<= 1;
    return G;
}


mesh_status launch_signed_query(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                                int32_t *d_face, float *d_bary, float *d_point, float *d_sdist,
                                cudaStream_t s) {
    float maxd2 = isinf(max_dist) ? INFINITY : max_dist * max_dist;
    Header *h = bvh->hdr();
    auto kern = bvh->leaf_size > 1 ? k_signed_distance<true> : k_signed_distance<false>;
    kern<<<grid_for(nQ, kQueryBlock), kQueryBlock, 0, s>>>(
        traversal_of(bvh, isinf(max_dist)), h, &h->status, d_Q, nQ, maxd2, bvh->faces(), bvh->adj(),
        bvh->fnorm(), bvh->verts(), d_face, d_bary, d_point, d_sdist);
    count_launch();
    return check_launch();
}

// The launch of mesh_closest_point_hinted for a tree with (R) or without leaf
// collapse.  With leaf collapse only the main forms exist -- the depth-first
// variants 0, 2, 3 (any block size), the warp packets (12) and the cooperative
// groups; the other one-thread variants run as variant 0.
template <bool R>
static void launch_closest_point(Traversal T, Header *h, const float *d_Q, int64_t nQ, float maxd2,
                                 int32_t *d_face, float *d_bary, float *d_point, float *d_dist2,
                                 const int32_t *d_hint, const int *iperm, int G, int variant, int blk,
                                 cudaStream_t s) {
    if (R && !(variant == 0 || variant == 2 || variant == 3 || variant == 12 || variant == 13)) variant = 0;
    unsigned int grid = grid_for(nQ * G, kQueryBlock);
    if (G == 1 && blk != kQueryBlock && (variant == 0 || variant == 2 || variant == 3 || variant == 13)) {
        unsigned int gb = grid_for(nQ, blk);
#define MESH_CPB(SM, M, B) k_closest_point<SM, M, kQueryMinBlocks, false, B, R><<<gb, B, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, d_hint, iperm)
        if (blk == 32) {
            if (variant == 2) MESH_CPB(8, 0, 32); else if (variant == 3) MESH_CPB(0, 0, 32);
            else if (variant == 13) MESH_CPB(8, 3, 32); else MESH_CPB(kStackShared, 0, 32);
        } else {
            if (variant == 2) MESH_CPB(8, 0, 64); else if (variant == 3) MESH_CPB(0, 0, 64);
            else if (variant == 13) MESH_CPB(8, 3, 64); else MESH_CPB(kStackShared, 0, 64);
        }
#undef MESH_CPB
        return;
    }
    switch (G) {
        case 1:
#define MESH_CP_ARGS <<<grid, kQueryBlock, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, d_hint, iperm)
            switch (variant) {
                case 2: k_closest_point<8, 0, kQueryMinBlocks, false, kQueryBlock, R> MESH_CP_ARGS; break;
                case 13: k_closest_point<8, 3, kQueryMinBlocks, false, kQueryBlock, R> MESH_CP_ARGS; break;
                case 3: k_closest_point<0, 0, kQueryMinBlocks, false, kQueryBlock, R> MESH_CP_ARGS; break;
                case 12: k_closest_point_packet<false, R><<<grid, kQueryBlock, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, d_hint, iperm); break;
                default:
                    if constexpr (!R) {
                        switch (variant) {
                            case 1: k_closest_point<kStackShared, 1> MESH_CP_ARGS; break;
                            case 4: k_closest_point<kStackShared, 2> MESH_CP_ARGS; break;
                            case 5: k_closest_point<0, 2> MESH_CP_ARGS; break;
                            case 6: k_closest_point<8, 0, 9> MESH_CP_ARGS; break;
                            case 7: k_closest_point<0, 0, 9> MESH_CP_ARGS; break;
                            case 8: k_closest_point<0, 0, 16> MESH_CP_ARGS; break;
                            case 9: k_closest_point<0, 2, 12> MESH_CP_ARGS; break;
                            case 10:
                            case 11: {
                                static int sms = 0;
                                if (sms == 0) {
                                    int dv = 0;
                                    if (cudaGetDevice(&dv) != cudaSuccess ||
                                        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dv) != cudaSuccess || sms <= 0)
                                        sms = 152;
                                }
                                unsigned int *work = &h->pad[0];
                                cudaMemsetAsync(work, 0, sizeof(unsigned int), s);
                                unsigned int pg = (unsigned int)((int64_t)sms * kQueryMinBlocks < (int64_t)grid ? sms * kQueryMinBlocks : grid);
                                if (variant == 10)
                                    k_closest_point_persistent<8><<<pg, kQueryBlock, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, work);
                                else
                                    k_closest_point_persistent<0><<<pg, kQueryBlock, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, work);
                                break;
                            }
                            default: k_closest_point<kStackShared, 0> MESH_CP_ARGS; break;
                        }
                    } else {
                        k_closest_point<kStackShared, 0, kQueryMinBlocks, false, kQueryBlock, R> MESH_CP_ARGS;
                    }
                    break;
            }
#undef MESH_CP_ARGS
            break;
#define MESH_CPG(g) k_closest_point_group<g, R><<<grid, kQueryBlock, 0, s>>>(T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2, d_hint, iperm)
        case 2: MESH_CPG(2); break;
        case 4: MESH_CPG(4); break;
        case 8: MESH_CPG(8); break;
        case 16: MESH_CPG(16); break;
        default: MESH_CPG(32); break;
#undef MESH_CPG
    }
}

// The ordered, recording launch of mesh_contact for a tree with (R) or without
// leaf collapse (with it, the one-thread variants other than 0, 2, 3 run as 0).
template <bool R>
static void launch_contact(Traversal T, Header *h, const float *d_Q, int64_t nQ, float maxd2, int32_t *d_face,
                           float *d_bary, float *d_point, float *d_dist2, const int *iperm, const int *order,
                           unsigned int *cls, int variant, int blk, cudaStream_t s) {
    if (R && !(variant == 0 || variant == 2 || variant == 3 || variant == 12 || variant == 13)) variant = 0;
    unsigned int grid = grid_for(nQ, kQueryBlock);
    // every form runs right after the sort of the classes: launched as its dependent
    auto go = [&](auto kern, unsigned int g, unsigned int b) {
        pdl_launch(kern, g, b, 0, s, T, h, &h->status, d_Q, nQ, maxd2, d_face, d_bary, d_point, d_dist2,
                   d_face, iperm, order, cls);
    };
    if (variant == 12) {
        go(k_closest_point_packet<true, R>, grid, kQueryBlock);
        return;
    }
    if (blk != kQueryBlock && (variant == 0 || variant == 2 || variant == 3 || variant == 13)) {
        unsigned int gb = grid_for(nQ, blk);
        if (blk == 32) {
            if (variant == 2) go(k_closest_point<8, 0, kQueryMinBlocks, true, 32, R>, gb, 32);
            else if (variant == 3) go(k_closest_point<0, 0, kQueryMinBlocks, true, 32, R>, gb, 32);
            else if (variant == 13) go(k_closest_point<8, 3, kQueryMinBlocks, true, 32, R>, gb, 32);
            else go(k_closest_point<kStackShared, 0, kQueryMinBlocks, true, 32, R>, gb, 32);
        } else {
            if (variant == 2) go(k_closest_point<8, 0, kQueryMinBlocks, true, 64, R>, gb, 64);
            else if (variant == 3) go(k_closest_point<0, 0, kQueryMinBlocks, true, 64, R>, gb, 64);
            else if (variant == 13) go(k_closest_point<8, 3, kQueryMinBlocks, true, 64, R>, gb, 64);
            else go(k_closest_point<kStackShared, 0, kQueryMinBlocks, true, 64, R>, gb, 64);
        }
        return;
    }
    switch (variant) {
        case 2: go(k_closest_point<8, 0, kQueryMinBlocks, true, kQueryBlock, R>, grid, kQueryBlock); break;
        case 13: go(k_closest_point<8, 3, kQueryMinBlocks, true, kQueryBlock, R>, grid, kQueryBlock); break;
        case 3: go(k_closest_point<0, 0, kQueryMinBlocks, true, kQueryBlock, R>, grid, kQueryBlock); break;
        default:
            if constexpr (!R) {
                switch (variant) {
                    case 4: go(k_closest_point<kStackShared, 2, kQueryMinBlocks, true>, grid, kQueryBlock); break;
                    case 5: go(k_closest_point<0, 2, kQueryMinBlocks, true>, grid, kQueryBlock); break;
                    case 6: go(k_closest_point<8, 0, 9, true>, grid, kQueryBlock); break;
                    case 7: go(k_closest_point<0, 0, 9, true>, grid, kQueryBlock); break;
                    case 8: go(k_closest_point<0, 0, 16, true>, grid, kQueryBlock); break;
                    case 9: go(k_closest_point<0, 2, 12, true>, grid, kQueryBlock); break;
                    default: go(k_closest_point<kStackShared, 0, kQueryMinBlocks, true>, grid, kQueryBlock); break;
                }
            } else {
                go(k_closest_point<kStackShared, 0, kQueryMinBlocks, true, kQueryBlock, R>, grid, kQueryBlock);
            }
            break;
    }
}

// The Chamfer launch: G lanes per sample, with (range) or without leaf collapse.
// pdl: launched as the dependent of the kernel before it (the sort of mesh_chamfer_step).
template <bool R>
static void launch_chamfer_r(int G, unsigned grid, const ChamferSide &a2b, const ChamferSide &b2a, unsigned nbA,
                             unsigned *st, double *partial, unsigned *ticket, double *out, cudaStream_t s,
                             bool pdl) {
    auto go = [&](auto kern) {
        if (pdl) pdl_launch(kern, grid, kQueryBlock, 0, s, a2b, b2a, nbA, st, partial, ticket, out);
        else kern<<<grid, kQueryBlock, 0, s>>>(a2b, b2a, nbA, st, partial, ticket, out);
    };
    switch (G) {
        case 1: go(k_chamfer<1, R>); break;
        case 2: go(k_chamfer<2, R>); break;
        case 4: go(k_chamfer<4, R>); break;
        case 8: go(k_chamfer<8, R>); break;
        case 16: go(k_chamfer<16, R>); break;
        default: go(k_chamfer<32, R>); break;
    }
}
static void launch_chamfer(int G, bool range, unsigned grid, const ChamferSide &a2b, const ChamferSide &b2a,
                           unsigned nbA, unsigned *st, double *partial, unsigned *ticket, double *out,
                           cudaStream_t s, bool pdl = false) {
    if (range) launch_chamfer_r<true>(G, grid, a2b, b2a, nbA, st, partial, ticket, out, s, pdl);
    else launch_chamfer_r<false>(G, grid, a2b, b2a, nbA, st, partial, ticket, out, s, pdl);
}

// The Chamfer of a sequence of frames (mesh_chamfer_step): each side's samples
// run warm-started from the previous call's faces and in the order of the
// previous call's costs, heaviest first, so that the samples sharing a block
// end together and the long searches do not trail the launch.  The keys of
// both sides are sorted together by one stable 8-bit pass (side in bit 7, so
// the order is side-major); k_chamfer_keys first sets every key's side bit,
// so a fresh or stale workspace gives a valid, if worse, order.
// It also zeroes the Chamfer kernel's last-block ticket (that kernel runs after it).
__global__ void k_chamfer_keys(unsigned int *__restrict__ key, int nA, int n, unsigned int *__restrict__ ticket) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *ticket = 0u;
    if (c < n) key[c] = (c < nA ? 0u : 128u) | (key[c] & 127u);
}

struct ChamferStepWs {
    char *base;                    // mesh_chamfer's workspace (partials, ticket)
    unsigned int *key, *key_sorted;
    int *order;
    void *sort_ws;
    size_t bytes;
};

static ChamferStepWs chamfer_step_ws(void *ws, int64_t nSA, int64_t nSB) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    int64_t m = nSA + nSB > 0 ? nSA + nSB : 1;
    size_t oB = take(mesh_chamfer_workspace_bytes(nSA, nSB)), oK = take(4 * m), oS = take(4 * m),
           oO = take(4 * m), oW = take(sort_pairs_ws_bytes(m));
    char *b = (char *)ws;
    return ChamferStepWs{b + oB, (unsigned int *)(b + oK), (unsigned int *)(b + oS), (int *)(b + oO), b + oW,
                         off};
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

mesh_status mesh_closest_point(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                               int32_t *d_face, float *d_bary, float *d_point, float *d_dist2,
                               void *stream) {
    return mesh_closest_point_hinted(bvh, d_Q, nQ, max_dist, nullptr, d_face, d_bary, d_point, d_dist2,
                                     stream);
}

mesh_status mesh_closest_point_hinted(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                                      const int32_t *d_hint, int32_t *d_face, float *d_bary,
                                      float *d_point, float *d_dist2, void *stream) {
    if (!bvh || nQ < 0 || (nQ > 0 && !d_Q) || !(max_dist >= 0.0f)) return MESH_ERR_INVALID_ARG;
    if (nQ == 0) return MESH_OK;
    const int *iperm = bvh->iperm();
    float maxd2 = isinf(max_dist) ? INFINITY : max_dist * max_dist;
    cudaStream_t s = (cudaStream_t)stream;
    int G = bvh->cfg_lanes > 0 ? bvh->cfg_lanes : pick_group(nQ);
    int variant = bvh->cfg_variant >= 0 ? bvh->cfg_variant : g_traversal;
    if (variant >= 10 && variant <= 12 && nQ >= ((int64_t)1 << 31)) variant = 0;   // 32-bit work counter
    if (G == 1 && variant == 13) ensure_wide(bvh, s);
    Traversal T = traversal_of(bvh, isinf(max_dist));
    // the one-thread depth-first searches write face and distance; the weights and
    // closest points follow in one thread per query (as in the contact step)
    const int rv = (bvh->leaf_size > 1 && !(variant == 0 || variant == 2 || variant == 3 || variant == 13))
                       ? 0 : variant;
    const bool split = kContactSplitWeights && G == 1 && d_face && d_dist2 && (d_bary || d_point) &&
                       !(rv == 1 || (rv >= 10 && rv <= 12));
    float *sb = split ? nullptr : d_bary, *sp = split ? nullptr : d_point;
    if (bvh->leaf_size > 1)
        launch_closest_point<true>(T, bvh->hdr(), d_Q, nQ, maxd2, d_face, sb, sp, d_dist2, d_hint,
                                   iperm, G, variant, bvh->cfg_block, s);
    else
        launch_closest_point<false>(T, bvh->hdr(), d_Q, nQ, maxd2, d_face, sb, sp, d_dist2, d_hint,
                                    iperm, G, variant, bvh->cfg_block, s);
    count_launch();
    if (split) {
        pdl_launch(k_hit_weights, grid_for(nQ, 256), 256, 0, s, T, d_Q, nQ, (const int *)d_face,
                   (const float *)d_dist2, iperm, d_bary, d_point);
        count_launch();
    }
    return check_launch();
}

// Contact queries of a physics step: warm-started by the previous step's faces
// and run in the order of the previous step's work classes (heaviest first,
// each class in the given order), so that a warp holds queries of similar
// depth -- near the surface (deep searches), near misses, or far away (short
// ones) -- instead of a mix that runs as long as its slowest lane.  The
// classes (their low two bits) are ordered by a stable counting sort in two
// launches: each tile of queries counts its classes, then each tile scatters
// its query indices from the counts of the tiles before it.  Any class bits
// give a valid permutation, so a workspace whose classes are stale or garbage
// only gives a worse order.
constexpr int kClassTile = 2048, kClassThreads = 256;

__global__ void __launch_bounds__(kClassThreads)
k_class_count(const unsigned int *__restrict__ cls, int n, int4 *__restrict__ counts) {
    __shared__ int s_cnt[4];
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kClassTile, lane = threadIdx.x & 31;
    int c[4] = {0, 0, 0, 0};
#pragma unroll
    for (int r = 0; r < kClassTile / kClassThreads; ++r) {
        int i = base + r * kClassThreads + threadIdx.x;
        unsigned int k = i < n ? (cls[i] & 3u) : 4u;
#pragma unroll
        for (int q = 0; q < 4; ++q) c[q] += __popc(__ballot_sync(0xffffffffu, k == (unsigned)q));
    }
    if (lane < 4) atomicAdd(&s_cnt[lane], c[lane]);
    __syncthreads();
    if (threadIdx.x == 0) counts[blockIdx.x] = make_int4(s_cnt[0], s_cnt[1], s_cnt[2], s_cnt[3]);
}

__global__ void __launch_bounds__(kClassThreads)
k_class_scatter(const unsigned int *__restrict__ cls, int n, const int4 *__restrict__ counts, int tiles,
                int *__restrict__ order) {
    constexpr int kWarps = kClassThreads / 32;
    __shared__ int s_red[kWarps][8];
    __shared__ int s_run[4];
    __shared__ int s_off[kWarps][4];
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // every class's total and this tile's prefix, from the tiles' counts
    int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int t = threadIdx.x; t < tiles; t += kClassThreads) {
        int4 c = counts[t];
        v[0] += c.x; v[1] += c.y; v[2] += c.z; v[3] += c.w;
        if (t < (int)blockIdx.x) { v[4] += c.x; v[5] += c.y; v[6] += c.z; v[7] += c.w; }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < 8; ++q) s_red[wid][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot[4] = {0, 0, 0, 0}, pre[4] = {0, 0, 0, 0};
        for (int w = 0; w < kWarps; ++w)
            for (int q = 0; q < 4; ++q) { tot[q] += s_red[w][q]; pre[q] += s_red[w][4 + q]; }
        int run = 0;
        for (int q = 0; q < 4; ++q) { s_run[q] = run + pre[q]; run += tot[q]; }
    }
    __syncthreads();
    const int base = blockIdx.x * kClassTile;
    const unsigned int lt = (1u << lane) - 1u;
    for (int r = 0; r < kClassTile / kClassThreads; ++r) {
        int i = base + r * kClassThreads + threadIdx.x;
        unsigned int k = i < n ? (cls[i] & 3u) : 4u;
        unsigned int mine = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            unsigned int b = __ballot_sync(0xffffffffu, k == (unsigned)q);
            if (lane == 0) s_off[wid][q] = __popc(b);
            if (k == (unsigned)q) mine = b;
        }
        __syncthreads();
        if (threadIdx.x < 4) {                         // warp offsets within the round, per class
            int q = threadIdx.x, run = s_run[q];
            for (int w = 0; w < kWarps; ++w) { int c = s_off[w][q]; s_off[w][q] = run; run += c; }
            s_run[q] = run;
        }
        __syncthreads();
        if (k < 4u) order[s_off[wid][k] + __popc(mine & lt)] = i;
        __syncthreads();
    }
}

struct ContactWs {
    unsigned int *cls;
    int *order;
    int4 *counts;
    float *d2;             // the distances, when the caller does not take them
    size_t bytes;
};

static ContactWs contact_ws(void *ws, int64_t n) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    int64_t m = n > 0 ? n : 1;
    size_t oC = take(4 * m), oO = take(4 * m), oT = take(16 * ((m + kClassTile - 1) / kClassTile)),
           oD = take(4 * m);
    char *b = (char *)ws;
    return ContactWs{(unsigned int *)(b + oC), (int *)(b + oO), (int4 *)(b + oT), (float *)(b + oD), off};
}


mesh_status mesh_knn_project(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, int k,
                             const float *d_anchor, float anchor_weight, float *d_point,
                             int32_t *d_face, float *d_dist2, void *stream) {
    if (!bvh || nQ < 0 || k < 1 || k > kKnnMax || !(anchor_weight >= 0.0f && anchor_weight <= 1.0f))
        return MESH_ERR_INVALID_ARG;
    if (nQ == 0) return MESH_OK;
    if (!d_Q || !d_point) return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Header *h = bvh->hdr();
    k_knn_project<<<grid_for(nQ, kQueryBlock), kQueryBlock, 0, s>>>(
        traversal_of(bvh, false), h, d_Q, nQ, k, d_anchor, anchor_weight, d_point, d_face, d_dist2,
        &h->status);
    count_launch();
    return check_launch();
}


size_t mesh_contact_workspace_bytes(int64_t nQ) {
    if (nQ < 0 || nQ > INT32_MAX) return 0;
    return contact_ws(nullptr, nQ).bytes;
}

mesh_status mesh_contact(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist, int32_t *d_face,
                         float *d_bary, float *d_point, float *d_dist2, void *d_ws, size_t ws_bytes,
                         void *stream) {
    if (!bvh || nQ < 0 || nQ > INT32_MAX || (nQ > 0 && (!d_Q || !d_face)) || !(max_dist >= 0.0f))
        return MESH_ERR_INVALID_ARG;
    if (nQ == 0) return MESH_OK;
    ContactWs w = contact_ws(d_ws, nQ);
    if (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    int variant = bvh->cfg_variant >= 0 ? bvh->cfg_variant : g_traversal;
    if (bvh->leaf_size > 1 && !(variant == 0 || variant == 2 || variant == 3 || variant == 12 || variant == 13))
        variant = 0;
    if (variant == 1 || (variant >= 10 && variant <= 11) || (bvh->cfg_lanes > 1))
        return mesh_closest_point_hinted(bvh, d_Q, nQ, max_dist, d_face, d_face, d_bary, d_point, d_dist2,
                                         stream);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)nQ;
    const int tiles = (n + kClassTile - 1) / kClassTile;
    if (variant == 13) ensure_wide(bvh, s);
    // the call's first kernel is a plain launch (ordered after whatever the caller
    // put on the stream); the two after it are its programmatic dependents
    k_class_count<<<tiles, kClassThreads, 0, s>>>(w.cls, n, w.counts);
    pdl_launch(k_class_scatter, tiles, kClassThreads, 0, s, w.cls, n, w.counts, tiles, w.order);
    count_launch(2);
    float maxd2 = isinf(max_dist) ? INFINITY : max_dist * max_dist;
    Traversal T = traversal_of(bvh, isinf(max_dist));
    Header *h = bvh->hdr();
    const int *iperm = bvh->iperm();
    // the search writes face and distance; the weights follow in one thread per query
    const bool split = kContactSplitWeights && variant != 12 && (d_bary || d_point);
    float *sb = split ? nullptr : d_bary, *sp = split ? nullptr : d_point;
    float *sd = split && !d_dist2 ? w.d2 : d_dist2;
    if (bvh->leaf_size > 1)
        launch_contact<true>(T, h, d_Q, nQ, maxd2, d_face, sb, sp, sd, iperm, w.order, w.cls, variant,
                             bvh->cfg_block, s);
    else
        launch_contact<false>(T, h, d_Q, nQ, maxd2, d_face, sb, sp, sd, iperm, w.order, w.cls, variant,
                              bvh->cfg_block, s);
    count_launch();
    if (split) {
        pdl_launch(k_hit_weights, grid_for(nQ, 256), 256, 0, s, T, d_Q, nQ, (const int *)d_face, (const float *)sd,
                   iperm, d_bary, d_point);
        count_launch();
    }
    return check_launch();
}


size_t mesh_chamfer_workspace_bytes(int64_t nSA, int64_t nSB) {
    if (nSA < 0 || nSB < 0) return 0;
    return align_up(8 * (chamfer_blocks(nSA, 32) + chamfer_blocks(nSB, 32) + 1), 256) + 256;
}

mesh_status mesh_chamfer(const mesh_bvh *A, const float *d_SA, int64_t nSA, const mesh_bvh *B,
                         const float *d_SB, int64_t nSB, void *d_ws, size_t ws_bytes,
                         double *d_out, int32_t *d_faceA, float *d_baryA, float *d_dist2A,
                         int32_t *d_faceB, float *d_baryB, float *d_dist2B, void *stream) {
    return mesh_chamfer_hinted(A, d_SA, nSA, B, d_SB, nSB, d_ws, ws_bytes, d_out, nullptr, nullptr,
                               d_faceA, d_baryA, d_dist2A, d_faceB, d_baryB, d_dist2B, stream);
}

mesh_status mesh_chamfer_hinted(const mesh_bvh *A, const float *d_SA, int64_t nSA, const mesh_bvh *B,
                                const float *d_SB, int64_t nSB, void *d_ws, size_t ws_bytes,
                                double *d_out, const int32_t *d_hintA, const int32_t *d_hintB,
                                int32_t *d_faceA, float *d_baryA, float *d_dist2A,
                                int32_t *d_faceB, float *d_baryB, float *d_dist2B, void *stream) {
    if (!A || !B || !d_out || nSA < 0 || nSB < 0 || (nSA > 0 && !d_SA) || (nSB > 0 && !d_SB))
        return MESH_ERR_INVALID_ARG;
    size_t need = mesh_chamfer_workspace_bytes(nSA, nSB);
    if (!d_ws || ws_bytes < need || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int G = pick_group(nSA + nSB);
    size_t nbA = chamfer_blocks(nSA, G), nbB = chamfer_blocks(nSB, G);
    double *partial = (double *)d_ws;
    unsigned int *ticket = (unsigned int *)((char *)d_ws + need - 256);
    if (nbA + nbB == 0) {
        cudaMemsetAsync(d_out, 0, 2 * sizeof(double), s);
        return check_launch();
    }
    cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
    ChamferSide a2b{traversal_of(B), B->hdr(), d_SA, nSA, d_faceA, d_baryA, d_dist2A, d_hintA, B->iperm()};
    ChamferSide b2a{traversal_of(A), A->hdr(), d_SB, nSB, d_faceB, d_baryB, d_dist2B, d_hintB, A->iperm()};
    unsigned grid = (unsigned)(nbA + nbB);
    unsigned *st = &A->hdr()->status;
    launch_chamfer(G, A->leaf_size > 1 || B->leaf_size > 1, grid, a2b, b2a, (unsigned)nbA, st, partial, ticket,
                   d_out, s);
    count_launch();
    return check_launch();
}

size_t mesh_chamfer_step_workspace_bytes(int64_t nSA, int64_t nSB) {
    if (nSA < 0 || nSB < 0 || nSA + nSB > INT32_MAX) return 0;
    return chamfer_step_ws(nullptr, nSA, nSB).bytes;
}

mesh_status mesh_chamfer_step(const mesh_bvh *A, const float *d_SA, int64_t nSA, const mesh_bvh *B,
                              const float *d_SB, int64_t nSB, void *d_ws, size_t ws_bytes, double *d_out,
                              int32_t *d_faceA, float *d_baryA, float *d_dist2A, int32_t *d_faceB,
                              float *d_baryB, float *d_dist2B, void *stream) {
    if (!A || !B || !d_out || nSA < 0 || nSB < 0 || nSA + nSB > INT32_MAX || (nSA > 0 && (!d_SA || !d_faceA)) ||
        (nSB > 0 && (!d_SB || !d_faceB)))
        return MESH_ERR_INVALID_ARG;
    ChamferStepWs w = chamfer_step_ws(d_ws, nSA, nSB);
    if (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = mesh_chamfer_workspace_bytes(nSA, nSB);
    int G = pick_group(nSA + nSB);
    size_t nbA = chamfer_blocks(nSA, G), nbB = chamfer_blocks(nSB, G);
    double *partial = (double *)w.base;
    unsigned int *ticket = (unsigned int *)(w.base + need - 256);
    if (nbA + nbB == 0) {
        cudaMemsetAsync(d_out, 0, 2 * sizeof(double), s);
        return check_launch();
    }
    const int n = (int)(nSA + nSB);
    k_chamfer_keys<<<grid_for(n, 256), 256, 0, s>>>(w.key, (int)nSA, n, ticket);
    count_launch();
    sort_pairs_u32(w.sort_ws, n, 8, w.key, nullptr, w.key_sorted, w.order, s);
    ChamferSide a2b{traversal_of(B), B->hdr(), d_SA, nSA, d_faceA, d_baryA, d_dist2A, d_faceA, B->iperm(),
                    w.order, 0, w.key, 0u};
    ChamferSide b2a{traversal_of(A), A->hdr(), d_SB, nSB, d_faceB, d_baryB, d_dist2B, d_faceB, A->iperm(),
                    w.order + nSA, (int)nSA, w.key + nSA, 128u};
    unsigned grid = (unsigned)(nbA + nbB);
    unsigned *st = &A->hdr()->status;
    launch_chamfer(G, A->leaf_size > 1 || B->leaf_size > 1, grid, a2b, b2a, (unsigned)nbA, st, partial, ticket,
                   d_out, s, true);
    count_launch();
    return check_launch();
}

mesh_status mesh_batch_closest_point(mesh_batch *batch, const float *d_Q,
                                     const int32_t *d_query_off, int64_t nQ, float max_dist,
                                     int32_t *d_face, float *d_bary, float *d_point,
                                     float *d_dist2, void *stream) {
    if (!batch || nQ < 0 || nQ > 0xffff0000LL || (nQ > 0 && (!d_Q || !d_query_off)) ||
        !(max_dist >= 0.0f))
        return MESH_ERR_INVALID_ARG;
    if (nQ == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 152;
    }
    float maxd2 = isinf(max_dist) ? INFINITY : max_dist * max_dist;
    unsigned int *work = &batch->st()->work;
    cudaMemsetAsync(work, 0, sizeof(unsigned int), s);
    int64_t want = (nQ + kQueryBlock - 1) / kQueryBlock;
    unsigned int grid = (unsigned int)(want < (int64_t)sms * kQueryMinBlocks ? want : (int64_t)sms * kQueryMinBlocks);
    k_batch_closest_point<<<grid, kQueryBlock, 0, s>>>(
        batch->nodes(), batch->tris(), batch->scene_box(), batch->face_off(), d_query_off,
        (int)batch->L.n_scenes, d_Q, nQ, maxd2, isinf(max_dist), d_face, d_bary, d_point, d_dist2,
        &batch->st()->status, work);
    count_launch();
    return check_launch();
}

mesh_status mesh_closest_point_stats(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                                     float max_dist, unsigned long long *d_counts, void *stream) {
    if (!bvh || !d_counts || nQ < 0 || (nQ > 0 && !d_Q) || !(max_dist >= 0.0f))
        return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemsetAsync(d_counts, 0, 3 * sizeof(unsigned long long), s);
    if (nQ == 0) return check_launch();
    float maxd2 = isinf(max_dist) ? INFINITY : max_dist * max_dist;
    const int variant = bvh->cfg_variant >= 0 ? bvh->cfg_variant : g_traversal;
    const bool wide = variant == 13 && bvh->cfg_lanes <= 1;   // the 4-wide records' visits
    if (wide) ensure_wide(bvh, s);
    (bvh->leaf_size > 1 ? (wide ? k_closest_point_count<true, true> : k_closest_point_count<true>)
                        : (wide ? k_closest_point_count<false, true> : k_closest_point_count<false>))
        <<<grid_for(nQ, kQueryBlock), kQueryBlock, 0, s>>>(
        traversal_of(bvh, isinf(max_dist)), bvh->hdr(), &bvh->hdr()->status, d_Q, nQ, maxd2,
        d_counts);
    count_launch();
    return check_launch();
}

mesh_status mesh_set_query_group(int lanes) {
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != 16 &&
        lanes != 32)
        return MESH_ERR_INVALID_ARG;
    g_group_override = lanes;
    return MESH_OK;
}

mesh_status mesh_bvh_set_query_config(mesh_bvh *bvh, int lanes, int variant) {
    if (!bvh) return MESH_ERR_INVALID_ARG;
    if (lanes != -1 && lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 &&
        lanes != 16 && lanes != 32)
        return MESH_ERR_INVALID_ARG;
    if (variant < -1 || variant > 13) return MESH_ERR_INVALID_ARG;
    bvh->cfg_lanes = lanes;
    bvh->cfg_variant = variant;
    return MESH_OK;
}

mesh_status mesh_bvh_set_query_block(mesh_bvh *bvh, int threads) {
    if (!bvh || (threads != 0 && threads != 32 && threads != 64 && threads != 128))
        return MESH_ERR_INVALID_ARG;
    bvh->cfg_block = threads == 0 ? kQueryBlock : threads;
    return MESH_OK;
}

mesh_status mesh_set_traversal(int variant) {
    if (variant < 0 || variant > 13) return MESH_ERR_INVALID_ARG;
    g_traversal = variant;
    return MESH_OK;
}

mesh_status mesh_interpolate(const mesh_bvh *bvh, const int32_t *d_face, const float *d_bary,
                             int64_t n, float *d_out, void *stream) {
    if (!bvh || n < 0 || (n > 0 && (!d_face || !d_bary || !d_out))) return MESH_ERR_INVALID_ARG;
    if (n == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_interpolate<<<grid_for(n, 256), 256, 0, s>>>(bvh->faces(), bvh->verts(), (int)bvh->L.n_faces,
                                                   d_face, d_bary, n, d_out, &bvh->hdr()->status);
    count_launch();
    return check_launch();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Chamfer without caller workspace.
//
// Some callers cannot allocate device memory at all -- a physics or renderer
// plugin whose host application owns every device allocation, or code that
// runs while another framework is capturing the stream into a CUDA graph and
// forbids allocation -- so they cannot hand mesh_chamfer a workspace.  This
// entry point runs the same Chamfer kernel, with the lanes per sample
// mesh_chamfer would pick (fewer when that many blocks would not fit), with its
// scratch (per-block float64 partial sums and the last-block ticket) in a fixed
// file-scope device array instead.  Every GPU that loads the library holds that
// array until exit.  The array's device address is looked up once per device
// and kept; a cudaDeviceReset invalidates it, so no call may follow a reset in
// the same process.
// ---------------------------------------------------------------------------
namespace meshgs {

constexpr int kNoAllocMaxBlocks = 16384;   // partial sums: 16384 x 8 B = 128 KB
static __device__ __align__(256) double g_chamfer_scratch[kNoAllocMaxBlocks + 32];

constexpr int kMaxDevices = 64;
static double *g_scratch_ptr[kMaxDevices];          // device address per device ordinal
static std::mutex g_scratch_mu;

// Device address of g_chamfer_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, never a device address).
static mesh_status scratch_address(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MESH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_chamfer_scratch) != cudaSuccess || !p) return MESH_ERR_CUDA;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return MESH_OK;
}

}  // namespace meshgs

extern "C" mesh_status mesh_chamfer_noalloc(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                                            const mesh_bvh *B, const float *d_SB, int64_t nSB,
                                            double *d_out, int32_t *d_faceA, float *d_baryA,
                                            float *d_dist2A, int32_t *d_faceB, float *d_baryB,
                                            float *d_dist2B, void *stream) {
    using namespace meshgs;
    if (!A || !B || !d_out || nSA < 0 || nSB < 0 || (nSA > 0 && !d_SA) || (nSB > 0 && !d_SB))
        return MESH_ERR_INVALID_ARG;
    // the lanes per sample mesh_chamfer would use, fewer if its blocks exceed the array
    int G = pick_group(nSA + nSB);
    while (G > 1 && chamfer_blocks(nSA, G) + chamfer_blocks(nSB, G) > (size_t)kNoAllocMaxBlocks) G >>= 1;
    size_t nbA = chamfer_blocks(nSA, G), nbB = chamfer_blocks(nSB, G);
    if (nbA + nbB > (size_t)kNoAllocMaxBlocks) return MESH_ERR_WORKSPACE;
    double *scratch = nullptr;
    mesh_status st = scratch_address(&scratch);
    if (st != MESH_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (nbA + nbB == 0) {
        cudaMemsetAsync(d_out, 0, 2 * sizeof(double), s);
        return check_launch();
    }
    unsigned int *ticket = (unsigned int *)(scratch + kNoAllocMaxBlocks);
    cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
    ChamferSide a2b{traversal_of(B), B->hdr(), d_SA, nSA, d_faceA, d_baryA, d_dist2A};
    ChamferSide b2a{traversal_of(A), A->hdr(), d_SB, nSB, d_faceB, d_baryB, d_dist2B};
    unsigned grid = (unsigned)(nbA + nbB), nb = (unsigned)nbA;
    unsigned *st_ = &A->hdr()->status;
    launch_chamfer(G, A->leaf_size > 1 || B->leaf_size > 1, grid, a2b, b2a, nb, st_, scratch, ticket, d_out, s);
    count_launch();
    return check_launch();
}
