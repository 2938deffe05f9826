/*
 * Reference oracle for the per-frame dynamic-mesh update -- TEST
 * INFRASTRUCTURE ONLY.  Plain, slow, serial C (the *_omp forms run the same
 * per-query arithmetic over the host's cores, for timing and for large
 * samples; results are identical).  It shares no code, header or
 * constant with the CUDA library; only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.
 *
 * Everything is float64 except the Morton-key step and the merge cost of the
 * agglomerative build, whose recipes are defined in float32 (see orc_morton,
 * orc_ploc); this file must be compiled with -ffp-contract=off so that no
 * fused multiply-add changes a rounding.
 *
 * What the paper fixes and what is our reading:
 *   - NearestSurface(v, M) of Eq. 1 / Eq. 2 (Sec. 3.3): the exact closest
 *     point of v on the triangle mesh M, returned with its barycentric
 *     weights ("barycentric interpolation for sub-face accuracy", Eq. 2).
 *     The k-NN weighting Sec. 3.3 mentions for Eq. 1 is not used (reading).
 *   - Acceleration structure built once from F0, holding indices only
 *     (Sec. 3.4, Initialization): the paper gives no construction; here a
 *     linear BVH whose leaves are sorted faces (Karras 2012), and for a mesh
 *     built once and refit, an agglomerative tree over the same leaves
 *     (PLOC, Meister & Bittner 2018; orc_ploc).
 *   - Collision-structure rebuild of the varying-topology baseline (Sec. 4.1).
 *   - Gaussians bound to faces (Sec. 2, Sec. 3.1): the paper gives no
 *     formula; the face-frame reading is ours (orc_bind_gaussians).
 *   - Chamfer distance on surface samples (Sec. 4.2); squared, mean per
 *     direction, point-to-mesh (reading).
 *
 * Pins for every function live in tests/test_oracle_*.py (closed forms,
 * invariants, brute force, central differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TIE_REL 1e-6      /* ties: lowest face id within 1e-6 relative distance */
#define ORC_TIE_ABS 1e-12     /* absolute floor, times the mesh bounding-box diagonal */

/* ------------------------------------------------------------------ */
/* small float64 vector helpers                                        */
/* ------------------------------------------------------------------ */
typedef struct { double x, y, z; } d3;

static d3 mk(double x, double y, double z) { d3 r = {x, y, z}; return r; }
static d3 ld3(const double *p) { return mk(p[0], p[1], p[2]); }
static d3 sub(d3 a, d3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static d3 add(d3 a, d3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static d3 scl(d3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static d3 cross(d3 a, d3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double norm(d3 a) { return sqrt(dot(a, a)); }

/* ------------------------------------------------------------------ */
/* Closest point on one triangle (Ericson, Real-Time Collision          */
/* Detection, 5.1.5: classify p into the Voronoi regions of the         */
/* vertices, edges and face of abc).                                   */
/* ------------------------------------------------------------------ */
static double seg_closest(d3 p, d3 x, d3 y, double *t_out) {
    d3 xy = sub(y, x);
    double L2 = dot(xy, xy);
    double t = 0.0;
    if (L2 > 0.0) {
        t = dot(sub(p, x), xy) / L2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    d3 c = add(x, scl(xy, t));
    d3 d = sub(p, c);
    *t_out = t;
    return dot(d, d);
}

/* Returns the squared distance; bary = (u, v, w) with point = u a + v b + w c. */
double orc_point_triangle(const double *P, const double *A, const double *B,
                          const double *C, double *bary, double *point) {
    d3 p = mk(P[0], P[1], P[2]), a = mk(A[0], A[1], A[2]);
    d3 b = mk(B[0], B[1], B[2]), c = mk(C[0], C[1], C[2]);
    double u, v, w;
    d3 ab = sub(b, a), ac = sub(c, a);
    d3 n = cross(ab, ac);
    if (n.x == 0.0 && n.y == 0.0 && n.z == 0.0) {
        /* Zero-area triangle (reading): nearest of its three edges, first wins. */
        double t0, t1, t2;
        double s0 = seg_closest(p, a, b, &t0);
        double s1 = seg_closest(p, b, c, &t1);
        double s2 = seg_closest(p, c, a, &t2);
        if (s0 <= s1 && s0 <= s2) { u = 1.0 - t0; v = t0; w = 0.0; }
        else if (s1 <= s2)       { u = 0.0; v = 1.0 - t1; w = t1; }
        else                     { u = t2; v = 0.0; w = 1.0 - t2; }
    } else {
        d3 ap = sub(p, a);
        double d1 = dot(ab, ap), d2 = dot(ac, ap);
        d3 bp = sub(p, b);
        double d3_ = dot(ab, bp), d4 = dot(ac, bp);
        d3 cp = sub(p, c);
        double d5 = dot(ab, cp), d6 = dot(ac, cp);
        double vc = d1 * d4 - d3_ * d2;
        double vb = d5 * d2 - d1 * d6;
        double va = d3_ * d6 - d5 * d4;
        if (d1 <= 0.0 && d2 <= 0.0) {                 /* vertex a */
            u = 1.0; v = 0.0; w = 0.0;
        } else if (d3_ >= 0.0 && d4 <= d3_) {          /* vertex b */
            u = 0.0; v = 1.0; w = 0.0;
        } else if (vc <= 0.0 && d1 >= 0.0 && d3_ <= 0.0) {   /* edge ab */
            double t = d1 / (d1 - d3_);
            u = 1.0 - t; v = t; w = 0.0;
        } else if (d6 >= 0.0 && d5 <= d6) {           /* vertex c */
            u = 0.0; v = 0.0; w = 1.0;
        } else if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {   /* edge ac */
            double t = d2 / (d2 - d6);
            u = 1.0 - t; v = 0.0; w = t;
        } else if (va <= 0.0 && (d4 - d3_) >= 0.0 && (d5 - d6) >= 0.0) {  /* edge bc */
            double t = (d4 - d3_) / ((d4 - d3_) + (d5 - d6));
            u = 0.0; v = 1.0 - t; w = t;
        } else {                                        /* face interior */
            double s = 1.0 / (va + vb + vc);
            v = vb * s;
            w = vc * s;
            u = 1.0 - v - w;
        }
    }
    d3 q = add(add(scl(a, u), scl(b, v)), scl(c, w));
    d3 d = sub(p, q);
    bary[0] = u; bary[1] = v; bary[2] = w;
    point[0] = q.x; point[1] = q.y; point[2] = q.z;
    return dot(d, d);
}

/* ------------------------------------------------------------------ */
/* NearestSurface over a whole mesh (Eq. 1, Eq. 2): brute force over     */
/* every face.  Ties: the lowest face id among faces whose distance is  */
/* within d* (1 + 1e-6) + 1e-12 diag, d* the exact minimum.  A query     */
/* whose d* exceeds max_dist gets face -1, d2 = +inf, zero bary/point.  */
/* ------------------------------------------------------------------ */
double orc_mesh_diag(const double *V, const int32_t *F, int64_t nF) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t f = 0; f < nF; ++f)
        for (int k = 0; k < 3; ++k) {
            const double *v = V + 3 * (int64_t)F[3 * f + k];
            for (int c = 0; c < 3; ++c) {
                if (v[c] < lo[c]) lo[c] = v[c];
                if (v[c] > hi[c]) hi[c] = v[c];
            }
        }
    if (nF == 0) return 0.0;
    return sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                (hi[2] - lo[2]) * (hi[2] - lo[2]));
}

/* One query p of the brute force: every face's distance into dist[nF] (and
 * into d2_row when not NULL), then the tie rule and the cutoff. */
static void closest_one(const double *V, const int32_t *F, int64_t nF, const double *p,
                        double max_dist, double tau, double *dist, double *d2_row,
                        int32_t *face, double *bary, double *point, double *d2) {
    double best = INFINITY;
    for (int64_t f = 0; f < nF; ++f) {
        double A[3], B[3], C[3], bb[3], pp[3];
        for (int c = 0; c < 3; ++c) {
            A[c] = V[3 * (int64_t)F[3 * f] + c];
            B[c] = V[3 * (int64_t)F[3 * f + 1] + c];
            C[c] = V[3 * (int64_t)F[3 * f + 2] + c];
        }
        dist[f] = orc_point_triangle(p, A, B, C, bb, pp);
        if (d2_row) d2_row[f] = dist[f];
        if (dist[f] < best) best = dist[f];
    }
    int32_t pick = -1;
    if (nF > 0 && sqrt(best) <= max_dist) {
        double lim = sqrt(best) * (1.0 + ORC_TIE_REL) + tau;
        for (int64_t f = 0; f < nF; ++f)
            if (sqrt(dist[f]) <= lim) { pick = (int32_t)f; break; }
    }
    *face = pick;
    if (pick < 0) {
        *d2 = INFINITY;
        for (int c = 0; c < 3; ++c) { bary[c] = 0.0; point[c] = 0.0; }
    } else {
        double A[3], B[3], C[3];
        for (int c = 0; c < 3; ++c) {
            A[c] = V[3 * (int64_t)F[3 * pick] + c];
            B[c] = V[3 * (int64_t)F[3 * pick + 1] + c];
            C[c] = V[3 * (int64_t)F[3 * pick + 2] + c];
        }
        *d2 = orc_point_triangle(p, A, B, C, bary, point);
    }
}

void orc_closest_point_mesh(const double *V, const int32_t *F, int64_t nF,
                            const double *Q, int64_t nQ, double max_dist,
                            int32_t *face, double *bary, double *point, double *d2,
                            double *d2_all /* nullable: [nQ * nF] every face's distance^2 */) {
    double tau = ORC_TIE_ABS * orc_mesh_diag(V, F, nF);
    double *dist = (double *)malloc(sizeof(double) * (size_t)(nF > 0 ? nF : 1));
    for (int64_t q = 0; q < nQ; ++q)
        closest_one(V, F, nF, Q + 3 * q, max_dist, tau, dist, d2_all ? d2_all + q * nF : NULL,
                    face + q, bary + 3 * q, point + 3 * q, d2 + q);
    free(dist);
}

/* ------------------------------------------------------------------ */
/* The same brute force with the queries spread over the host's cores   */
/* (OpenMP; serial when built without it).  Each query runs exactly the */
/* serial function's arithmetic, so the results are identical; it exists */
/* to time the CPU baseline on every core and to check large samples.    */
/* ------------------------------------------------------------------ */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_closest_point_mesh_omp(const double *V, const int32_t *F, int64_t nF, const double *Q,
                                int64_t nQ, double max_dist, int32_t *face, double *bary,
                                double *point, double *d2) {
    double tau = ORC_TIE_ABS * orc_mesh_diag(V, F, nF);
#pragma omp parallel
    {
        double *dist = (double *)malloc(sizeof(double) * (size_t)(nF > 0 ? nF : 1));
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < nQ; ++q)
            closest_one(V, F, nF, Q + 3 * q, max_dist, tau, dist, NULL, face + q, bary + 3 * q,
                        point + 3 * q, d2 + q);
        free(dist);
    }
}

/* ------------------------------------------------------------------ */
/* Morton keys of face centroids (Sec. 3.4 builds the structure from     */
/* F0; Sec. 4.1 rebuilds it per frame).  The paper defines no key, so    */
/* the recipe is ours and fixed in float32 round-to-nearest:             */
/*   s_f   = (v0 + v1) + v2                       (centroid times 3)     */
/*   lo,hi = componentwise min / max of s_f over all faces               */
/*   inv   = 1 / (hi - lo)   (0 where hi == lo)                          */
/*   t     = (s - lo) * inv                                              */
/*   q     = clamp(floor(t * 1024), 0, 1023)                             */
/*   key   = bits of qx, qy, qz interleaved, x most significant (30 bits)*/
/* ------------------------------------------------------------------ */
static uint32_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz) {
    uint32_t key = 0;
    for (int bit = 9; bit >= 0; --bit) {
        key = (key << 1) | ((qx >> bit) & 1u);
        key = (key << 1) | ((qy >> bit) & 1u);
        key = (key << 1) | ((qz >> bit) & 1u);
    }
    return key;
}

void orc_morton(const float *V, const int32_t *F, int64_t nF, uint32_t *keys) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float *s = (float *)malloc(sizeof(float) * 3 * (size_t)(nF > 0 ? nF : 1));
    for (int64_t f = 0; f < nF; ++f) {
        const float *a = V + 3 * (int64_t)F[3 * f];
        const float *b = V + 3 * (int64_t)F[3 * f + 1];
        const float *c = V + 3 * (int64_t)F[3 * f + 2];
        for (int k = 0; k < 3; ++k) {
            volatile float ab = a[k] + b[k];
            float v = ab + c[k];
            s[3 * f + k] = v;
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    }
    float inv[3];
    for (int k = 0; k < 3; ++k) {
        float ext = hi[k] - lo[k];
        inv[k] = (ext > 0.0f) ? 1.0f / ext : 0.0f;
    }
    for (int64_t f = 0; f < nF; ++f) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            volatile float d = s[3 * f + k] - lo[k];
            volatile float t = d * inv[k];
            float x = floorf(t * 1024.0f);
            int qi = (int)x;
            if (qi < 0) qi = 0;
            if (qi > 1023) qi = 1023;
            q[k] = (uint32_t)qi;
        }
        keys[f] = interleave3(q[0], q[1], q[2]);
    }
    free(s);
}

/* ------------------------------------------------------------------ */
/* Sort (key, face id) pairs ascending, lexicographically; equal keys    */
/* therefore keep ascending face id (a stable sort of the keys).         */
/* ------------------------------------------------------------------ */
typedef struct { uint32_t key; int32_t id; } kv;

static int kv_cmp(const void *x, const void *y) {
    const kv *a = (const kv *)x, *b = (const kv *)y;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

void orc_sort_pairs(const uint32_t *keys, int64_t n, uint32_t *sorted_keys, int32_t *perm) {
    kv *t = (kv *)malloc(sizeof(kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { t[i].key = keys[i]; t[i].id = (int32_t)i; }
    qsort(t, (size_t)n, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < n; ++i) { sorted_keys[i] = t[i].key; perm[i] = t[i].id; }
    free(t);
}

/* ------------------------------------------------------------------ */
/* Binary radix tree over sorted keys (Karras 2012), built serially      */
/* top-down.  Keys are augmented with their sorted position, so          */
/* delta(i, j) = common-prefix length of (key_i, i) and (key_j, j).      */
/* A node over [first, last] splits after gamma, the last position whose */
/* augmented key shares more than delta(first, last) leading bits with   */
/* position first (found by a linear scan).  Node numbering follows      */
/* Karras: the root is internal node 0; a child range [first, gamma] is  */
/* internal node gamma, a child range [gamma+1, last] is internal node   */
/* gamma+1, and a one-element range is leaf gamma / gamma+1.             */
/* Child encoding: internal c >= 0, leaf j as -(j+1).                    */
/* parent[] has 2n-1 entries: internal nodes first, then leaves.         */
/* ------------------------------------------------------------------ */
static int clz32(uint32_t x) {
    int n = 0;
    if (x == 0) return 32;
    while (!(x & 0x80000000u)) { x <<= 1; ++n; }
    return n;
}

static int orc_delta(const uint32_t *k, int64_t i, int64_t j) {
    if (k[i] != k[j]) return clz32(k[i] ^ k[j]);
    return 32 + clz32((uint32_t)i ^ (uint32_t)j);
}

void orc_karras(const uint32_t *k, int64_t n, int32_t *left, int32_t *right, int32_t *parent,
                int32_t *range_first, int32_t *range_last) {
    if (n <= 0) return;
    for (int64_t i = 0; i < 2 * n - 1; ++i) parent[i] = -1;
    if (n == 1) return;
    int64_t *stk = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)n);
    int64_t sp = 0;
    stk[sp++] = 0; stk[sp++] = 0; stk[sp++] = n - 1;
    while (sp > 0) {
        int64_t last = stk[--sp], first = stk[--sp], node = stk[--sp];
        range_first[node] = (int32_t)first;
        range_last[node] = (int32_t)last;
        int dn = orc_delta(k, first, last);
        int64_t gamma = first;
        for (int64_t j = first; j < last; ++j)
            if (orc_delta(k, first, j) > dn) gamma = j;
        if (gamma == first) {
            left[node] = -(int32_t)(gamma + 1);
            parent[(n - 1) + gamma] = (int32_t)node;
        } else {
            left[node] = (int32_t)gamma;
            parent[gamma] = (int32_t)node;
            stk[sp++] = gamma; stk[sp++] = first; stk[sp++] = gamma;
        }
        if (gamma + 1 == last) {
            right[node] = -(int32_t)(gamma + 2);
            parent[(n - 1) + gamma + 1] = (int32_t)node;
        } else {
            right[node] = (int32_t)(gamma + 1);
            parent[gamma + 1] = (int32_t)node;
            stk[sp++] = gamma + 1; stk[sp++] = gamma + 1; stk[sp++] = last;
        }
    }
    free(stk);
}

/* ------------------------------------------------------------------ */
/* Agglomerative tree for a mesh whose topology is fixed (built once):  */
/* parallel locally-ordered clustering, PLOC (Meister & Bittner 2018),  */
/* written as its iterations, serially.  Clusters start as the leaves   */
/* in Morton order, each with its face's box.  One iteration:           */
/*   1. every cluster i picks, among clusters i-R..i+R (not i), the one */
/*      whose union box with its own has the least surface area        */
/*      (float32, (dx dy + dy dz) + dz dx, no fused multiply-add; ties  */
/*      to the lower index);                                            */
/*   2. every mutual pair (nn[nn[i]] == i) merges into a new node, left */
/*      child the lower position, which takes that position; the other  */
/*      cluster is removed (new nodes numbered in position order);      */
/*   3. the clusters are compacted in order.                            */
/* An iteration without a mutual pair (impossible for finite boxes,     */
/* since the least-cost pair with the lowest indices is mutual) merges  */
/* positions 0 and 1.  The tree is then laid out like orc_karras's:     */
/* leaves in in-order, internal node numbered by the end of its range   */
/* not shared with its sibling (root 0, a left child by its last leaf,  */
/* a right child by its first), which is a bijection for any binary     */
/* tree over in-order leaves.                                           */
/* leaf_box: [n][6] float boxes of the leaves in Morton order.          */
/* order[p]: Morton position of the leaf at in-order position p.        */
/* left/right/parent/first/last as orc_karras (children: internal k,    */
/* leaf p as -(p+1); parent: internal nodes then leaves, -1 at root).   */
/* ------------------------------------------------------------------ */
static float ploc_area(const float *b) {
    float dx = b[3] - b[0], dy = b[4] - b[1], dz = b[5] - b[2];
    return (dx * dy + dy * dz) + dz * dx;
}

static void ploc_union(const float *a, const float *b, float *out) {
    for (int c = 0; c < 3; ++c) {
        out[c] = a[c] < b[c] ? a[c] : b[c];
        out[3 + c] = a[3 + c] > b[3 + c] ? a[3 + c] : b[3 + c];
    }
}

void orc_ploc(const float *leaf_box, int64_t n, int radius, int32_t *order, int32_t *left,
              int32_t *right, int32_t *parent, int32_t *first, int32_t *last) {
    if (n <= 0) return;
    for (int64_t i = 0; i < 2 * n - 1; ++i) parent[i] = -1;
    if (n == 1) { order[0] = 0; return; }
    int64_t m = n, made = 0;
    int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nn = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    float *cb = (float *)malloc(sizeof(float) * 6 * (size_t)n);
    int32_t *cl_l = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int32_t *cl_r = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n - 1));
    int32_t *kid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n - 1));
    for (int64_t j = 0; j < n; ++j) {
        cl[j] = -(int32_t)(j + 1);
        memcpy(cb + 6 * j, leaf_box + 6 * j, 6 * sizeof(float));
    }
    while (m > 1) {
        for (int64_t i = 0; i < m; ++i) {                        /* 1. nearest neighbour */
            float best = INFINITY, u[6];
            int64_t bj = -1;
            for (int64_t j = i - radius; j <= i + radius; ++j) {
                if (j < 0 || j >= m || j == i) continue;
                ploc_union(cb + 6 * i, cb + 6 * j, u);
                float a = ploc_area(u);
                if (bj < 0 || a < best) { best = a; bj = j; }
            }
            nn[i] = (int32_t)bj;
        }
        int64_t merges = 0;
        for (int64_t i = 0; i < m; ++i) merges += nn[nn[i]] == i && i < nn[i];
        if (merges == 0) { nn[0] = 1; nn[1] = 0; }
        int64_t w = 0;
        for (int64_t i = 0; i < m; ++i) {                        /* 2. merge, 3. compact */
            int64_t j = nn[i];
            int mutual = nn[j] == i;
            if (mutual && i > j) continue;
            if (mutual) {
                int64_t c = made++;
                int32_t a = cl[i], b = cl[j];
                cl_l[c] = a;
                cl_r[c] = b;
                cnt[c] = (a < 0 ? 1 : cnt[a]) + (b < 0 ? 1 : cnt[b]);
                float u[6];
                ploc_union(cb + 6 * i, cb + 6 * j, u);
                cl[w] = (int32_t)c;
                memcpy(cb + 6 * w, u, sizeof u);
            } else {
                cl[w] = cl[i];
                memmove(cb + 6 * w, cb + 6 * i, 6 * sizeof(float));
            }
            ++w;
        }
        m = w;
    }
    /* layout: parents were made after their children, so walk back */
    int64_t root = cl[0];
    pos[root] = 0;
    kid[root] = 0;
    for (int64_t c = made - 1; c >= 0; --c) {
        int32_t k = kid[c], p = pos[c];
        first[k] = p;
        last[k] = p + cnt[c] - 1;
        int32_t a = cl_l[c], b = cl_r[c];
        int32_t ca = a < 0 ? 1 : cnt[a];
        if (a < 0) {
            order[p] = -a - 1;
            left[k] = -(p + 1);
            parent[(n - 1) + p] = k;
        } else {
            pos[a] = p;
            kid[a] = p + ca - 1;
            left[k] = kid[a];
            parent[kid[a]] = k;
        }
        int32_t rp = p + ca;
        if (b < 0) {
            order[rp] = -b - 1;
            right[k] = -(rp + 1);
            parent[(n - 1) + rp] = k;
        } else {
            pos[b] = rp;
            kid[b] = rp;
            right[k] = rp;
            parent[rp] = k;
        }
    }
    free(cl); free(nn); free(cb); free(cl_l); free(cl_r); free(cnt); free(pos); free(kid);
}

/* ------------------------------------------------------------------ */
/* Leaf collapse with leaf size L (the scope's reading c6: a subtree    */
/* whose range holds at most L faces becomes one leaf over that range). */
/* The tree itself is unchanged; every child link of an internal node   */
/* is rewritten: a leaf j stays (-(j+1), 1); an internal child c whose  */
/* range [first[c], last[c]] holds at most L faces becomes the range    */
/* leaf (-(first[c]+1), last[c] - first[c] + 1); any other internal     */
/* child stays (c, c).  A search from the root then meets each face     */
/* once, inside the topmost subtree of at most L faces that holds it.   */
/* link[i][0..1] = left link, count; link[i][2..3] = right link, count. */
/* ------------------------------------------------------------------ */
static void collapse_one(int32_t c, const int32_t *first, const int32_t *last, int L, int32_t *out) {
    if (c < 0) { out[0] = c; out[1] = 1; return; }
    int32_t len = last[c] - first[c] + 1;
    if (len <= L) { out[0] = -(first[c] + 1); out[1] = len; }
    else { out[0] = c; out[1] = c; }
}

void orc_collapse(const int32_t *left, const int32_t *right, const int32_t *first,
                  const int32_t *last, int64_t n, int L, int32_t *link) {
    for (int64_t i = 0; i + 1 < n; ++i) {
        collapse_one(left[i], first, last, L, link + 4 * i);
        collapse_one(right[i], first, last, L, link + 4 * i + 2);
    }
}

/* ------------------------------------------------------------------ */
/* Node bounding boxes: for every node, the componentwise min / max of  */
/* the vertices of all faces in its sorted range, taken directly over   */
/* the range (not as a union of child boxes).  Exact in float32.        */
/* boxes: [2n-1][6] = (lo.xyz, hi.xyz), internal nodes then leaves.     */
/* A refit is the same function called with the new vertex buffer.      */
/* ------------------------------------------------------------------ */
static void range_box(const float *V, const int32_t *F, const int32_t *perm,
                      int64_t first, int64_t last, float *out) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = first; j <= last; ++j) {
        int64_t f = perm[j];
        for (int k = 0; k < 3; ++k) {
            const float *v = V + 3 * (int64_t)F[3 * f + k];
            for (int c = 0; c < 3; ++c) {
                if (v[c] < lo[c]) lo[c] = v[c];
                if (v[c] > hi[c]) hi[c] = v[c];
            }
        }
    }
    for (int c = 0; c < 3; ++c) { out[c] = lo[c]; out[3 + c] = hi[c]; }
}

void orc_node_boxes(const float *V, const int32_t *F, const int32_t *perm, int64_t n,
                    const int32_t *range_first, const int32_t *range_last, float *boxes) {
    for (int64_t i = 0; i + 1 < n; ++i)
        range_box(V, F, perm, range_first[i], range_last[i], boxes + 6 * i);
    for (int64_t j = 0; j < n; ++j)
        range_box(V, F, perm, j, j, boxes + 6 * (n - 1 + j));
}

/* ------------------------------------------------------------------ */
/* Gaussian binding to a face frame (reading; the paper says only that  */
/* Gaussians are anchored to mesh faces, Sec. 2 and Sec. 3.1).          */
/* For face (v0, v1, v2), barycentric anchor b and normal offset delta: */
/*   e1 = (v1 - v0)/|v1 - v0|,  n = (v1-v0) x (v2-v0) / |...|,  e2 = n x e1 */
/*   R  = [e1 e2 n] (columns),  mu = sum_j b_j v_j + delta n            */
/*   q  = unit quaternion (w, x, y, z) of R, Shepperd's largest-pivot    */
/*        branch, sign fixed so w > 0 (w == 0: first nonzero of x,y,z > 0) */
/*   l  = |v1 - v0|, h = |(v1-v0) x (v2-v0)| / l (altitude onto v0v1)    */
/*   s  = (l/3, h/3, 0.01 (l + h)/6)                                     */
/* A face with l == 0 or zero area is degenerate: mu from b alone,      */
/* q = (1, 0, 0, 0), s = 0, flag 1.                                      */
/* ------------------------------------------------------------------ */
#define ORC_RHO (1.0 / 3.0)
#define ORC_EPS_S 1e-2

static void orc_quat_from_R(const double R[3][3], double q[4]) {
    double tr = R[0][0] + R[1][1] + R[2][2];
    double w, x, y, z;
    int br;
    if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) br = 0;
    else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) br = 1;
    else if (R[1][1] >= R[2][2]) br = 2;
    else br = 3;
    if (br == 0) {
        w = 0.5 * sqrt(1.0 + tr);
        double f = 0.25 / w;
        x = (R[2][1] - R[1][2]) * f; y = (R[0][2] - R[2][0]) * f; z = (R[1][0] - R[0][1]) * f;
    } else if (br == 1) {
        x = 0.5 * sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]);
        double f = 0.25 / x;
        w = (R[2][1] - R[1][2]) * f; y = (R[0][1] + R[1][0]) * f; z = (R[0][2] + R[2][0]) * f;
    } else if (br == 2) {
        y = 0.5 * sqrt(1.0 - R[0][0] + R[1][1] - R[2][2]);
        double f = 0.25 / y;
        w = (R[0][2] - R[2][0]) * f; x = (R[0][1] + R[1][0]) * f; z = (R[1][2] + R[2][1]) * f;
    } else {
        z = 0.5 * sqrt(1.0 - R[0][0] - R[1][1] + R[2][2]);
        double f = 0.25 / z;
        w = (R[1][0] - R[0][1]) * f; x = (R[0][2] + R[2][0]) * f; y = (R[1][2] + R[2][1]) * f;
    }
    int neg = 0;
    if (w < 0.0) neg = 1;
    else if (w == 0.0) {
        if (x != 0.0) neg = x < 0.0;
        else if (y != 0.0) neg = y < 0.0;
        else neg = z < 0.0;
    }
    double sg = neg ? -1.0 : 1.0;
    q[0] = sg * w; q[1] = sg * x; q[2] = sg * y; q[3] = sg * z;
}

/* One Gaussian g of orc_bind_gaussians; returns 1 when its face is degenerate. */
static int bind_one(const double *V, const int32_t *F, const int32_t *gface, const double *gbary,
                    const double *goff, int64_t g, double *mu, double *quat, double *scale,
                    int32_t *flags) {
    int64_t f = gface[g];
    d3 v0 = ld3(V + 3 * (int64_t)F[3 * f]);
    d3 v1 = ld3(V + 3 * (int64_t)F[3 * f + 1]);
    d3 v2 = ld3(V + 3 * (int64_t)F[3 * f + 2]);
    double b0 = gbary[3 * g], b1 = gbary[3 * g + 1], b2 = gbary[3 * g + 2];
    double off = goff ? goff[g] : 0.0;
    d3 m = add(add(scl(v0, b0), scl(v1, b1)), scl(v2, b2));
    d3 e = sub(v1, v0);
    d3 nu = cross(e, sub(v2, v0));
    double l = norm(e), an = norm(nu);
    if (l == 0.0 || an == 0.0) {
        flags[g] = 1;
        mu[3 * g] = m.x; mu[3 * g + 1] = m.y; mu[3 * g + 2] = m.z;
        quat[4 * g] = 1.0; quat[4 * g + 1] = quat[4 * g + 2] = quat[4 * g + 3] = 0.0;
        scale[3 * g] = scale[3 * g + 1] = scale[3 * g + 2] = 0.0;
        return 1;
    }
    flags[g] = 0;
    d3 e1 = scl(e, 1.0 / l);
    d3 n = scl(nu, 1.0 / an);
    d3 e2 = cross(n, e1);
    double R[3][3] = {{e1.x, e2.x, n.x}, {e1.y, e2.y, n.y}, {e1.z, e2.z, n.z}};
    m = add(m, scl(n, off));
    mu[3 * g] = m.x; mu[3 * g + 1] = m.y; mu[3 * g + 2] = m.z;
    orc_quat_from_R(R, quat + 4 * g);
    double h = an / l;
    scale[3 * g] = ORC_RHO * l;
    scale[3 * g + 1] = ORC_RHO * h;
    scale[3 * g + 2] = ORC_EPS_S * ORC_RHO * (l + h) * 0.5;
    return 0;
}

int64_t orc_bind_gaussians(const double *V, const int32_t *F, const int32_t *gface,
                           const double *gbary, const double *goff /* nullable */, int64_t nG,
                           double *mu, double *quat, double *scale, int32_t *flags) {
    int64_t ndeg = 0;
    for (int64_t g = 0; g < nG; ++g) ndeg += bind_one(V, F, gface, gbary, goff, g, mu, quat, scale, flags);
    return ndeg;
}

/* orc_bind_gaussians over the host's cores (identical results). */
int64_t orc_bind_gaussians_omp(const double *V, const int32_t *F, const int32_t *gface,
                               const double *gbary, const double *goff, int64_t nG, double *mu,
                               double *quat, double *scale, int32_t *flags) {
    int64_t ndeg = 0;
#pragma omp parallel for schedule(static) reduction(+ : ndeg)
    for (int64_t g = 0; g < nG; ++g) ndeg += bind_one(V, F, gface, gbary, goff, g, mu, quat, scale, flags);
    return ndeg;
}

/* ------------------------------------------------------------------ */
/* Chamfer distance between two meshes on surface samples (Sec. 4.2):   */
/*   out[0] = mean over a in SA of d(a, mesh B)^2                       */
/*   out[1] = mean over b in SB of d(b, mesh A)^2                       */
/* (the symmetric CD is out[0] + out[1]).  Sums in float64, in order.   */
/* ------------------------------------------------------------------ */
void orc_chamfer(const double *VA, const int32_t *FA, int64_t nFA, const double *SA, int64_t nSA,
                 const double *VB, const int32_t *FB, int64_t nFB, const double *SB, int64_t nSB,
                 double *out, double *dA, double *dB) {
    int32_t *fc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nSA > nSB ? nSA : nSB) + 4);
    double *bb = (double *)malloc(sizeof(double) * 3 * (size_t)(nSA > nSB ? nSA : nSB) + 32);
    double *pp = (double *)malloc(sizeof(double) * 3 * (size_t)(nSA > nSB ? nSA : nSB) + 32);
    orc_closest_point_mesh(VB, FB, nFB, SA, nSA, INFINITY, fc, bb, pp, dA, NULL);
    orc_closest_point_mesh(VA, FA, nFA, SB, nSB, INFINITY, fc, bb, pp, dB, NULL);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = 0; i < nSA; ++i) s0 += dA[i];
    for (int64_t i = 0; i < nSB; ++i) s1 += dB[i];
    out[0] = nSA > 0 ? s0 / (double)nSA : 0.0;
    out[1] = nSB > 0 ? s1 / (double)nSB : 0.0;
    free(fc); free(bb); free(pp);
}

/* orc_chamfer with the two brute-force passes over the host's cores; the sums
 * stay serial and in order, so the result is identical. */
void orc_chamfer_omp(const double *VA, const int32_t *FA, int64_t nFA, const double *SA, int64_t nSA,
                     const double *VB, const int32_t *FB, int64_t nFB, const double *SB, int64_t nSB,
                     double *out, double *dA, double *dB) {
    int64_t m = nSA > nSB ? nSA : nSB;
    int32_t *fc = (int32_t *)malloc(sizeof(int32_t) * (size_t)m + 4);
    double *bb = (double *)malloc(sizeof(double) * 3 * (size_t)m + 32);
    double *pp = (double *)malloc(sizeof(double) * 3 * (size_t)m + 32);
    orc_closest_point_mesh_omp(VB, FB, nFB, SA, nSA, INFINITY, fc, bb, pp, dA);
    orc_closest_point_mesh_omp(VA, FA, nFA, SB, nSB, INFINITY, fc, bb, pp, dB);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = 0; i < nSA; ++i) s0 += dA[i];
    for (int64_t i = 0; i < nSB; ++i) s1 += dB[i];
    out[0] = nSA > 0 ? s0 / (double)nSA : 0.0;
    out[1] = nSB > 0 ? s1 / (double)nSB : 0.0;
    free(fc); free(bb); free(pp);
}

/* ------------------------------------------------------------------ */
/* Gradients (extension of the method: differentiating the update).    */
/* Point-to-mesh, with the nearest face and its barycentrics held fixed */
/* (envelope theorem; valid away from region boundaries and ties):      */
/*   d(d^2)/dq   =  2 (q - c)                                           */
/*   d(d^2)/dv_j = -2 b_j (q - c)   for the nearest face's vertex j      */
/* g is dL/d(d^2) per query; gQ [nQ,3], gV [nV,3] are accumulated into. */
/* ------------------------------------------------------------------ */
void orc_closest_point_backward(const double *V, const int32_t *F, const double *Q, int64_t nQ,
                                const int32_t *face, const double *bary, const double *g,
                                double *gQ, double *gV) {
    for (int64_t q = 0; q < nQ; ++q) {
        int64_t f = face[q];
        if (f < 0) continue;
        d3 p = ld3(Q + 3 * q);
        d3 c = mk(0, 0, 0);
        for (int j = 0; j < 3; ++j)
            c = add(c, scl(ld3(V + 3 * (int64_t)F[3 * f + j]), bary[3 * q + j]));
        d3 r = scl(sub(p, c), 2.0 * g[q]);
        gQ[3 * q] += r.x; gQ[3 * q + 1] += r.y; gQ[3 * q + 2] += r.z;
        for (int j = 0; j < 3; ++j) {
            int64_t v = F[3 * f + j];
            double bj = bary[3 * q + j];
            gV[3 * v] -= bj * r.x; gV[3 * v + 1] -= bj * r.y; gV[3 * v + 2] -= bj * r.z;
        }
    }
}

/* Samples placed by barycentric weights on a mesh: p = sum_j b_j v_j.  */
void orc_interpolate(const double *V, const int32_t *F, const int32_t *face, const double *bary,
                     int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) {
        d3 c = mk(0, 0, 0);
        for (int j = 0; j < 3; ++j)
            c = add(c, scl(ld3(V + 3 * (int64_t)F[3 * face[i] + j]), bary[3 * i + j]));
        out[3 * i] = c.x; out[3 * i + 1] = c.y; out[3 * i + 2] = c.z;
    }
}

/* d p / d v_j = b_j I: scatter dL/dp into dL/dV. */
void orc_interpolate_backward(const int32_t *F, const int32_t *face, const double *bary,
                              int64_t n, const double *gP, double *gV) {
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < 3; ++j) {
            int64_t v = F[3 * face[i] + j];
            double bj = bary[3 * i + j];
            for (int c = 0; c < 3; ++c) gV[3 * v + c] += bj * gP[3 * i + c];
        }
}

/* ------------------------------------------------------------------ */
/* Reverse-mode derivative of orc_bind_gaussians with respect to the    */
/* vertex positions.  Inputs dL/dmu [G,3], dL/dq [G,4], dL/ds [G,3];    */
/* dL/dV [V,3] is accumulated into.  Each step of the forward formula   */
/* is undone in reverse order; the quaternion step uses the same        */
/* Shepperd branch and sign the forward pass took.  Degenerate faces    */
/* contribute only through mu = sum_j b_j v_j.                          */
/* ------------------------------------------------------------------ */
static d3 vjp_normalize(d3 x, double len, d3 g) {
    /* y = x/len, len = |x|: dL/dx = (g - y (y . g)) / len */
    d3 y = scl(x, 1.0 / len);
    return scl(sub(g, scl(y, dot(y, g))), 1.0 / len);
}

void orc_bind_gaussians_backward(const double *V, const int32_t *F, const int32_t *gface,
                                 const double *gbary, const double *goff, int64_t nG,
                                 const double *gmu, const double *gq, const double *gs,
                                 double *gV) {
    for (int64_t g = 0; g < nG; ++g) {
        int64_t f = gface[g];
        int64_t iv[3] = {F[3 * f], F[3 * f + 1], F[3 * f + 2]};
        d3 v0 = ld3(V + 3 * iv[0]), v1 = ld3(V + 3 * iv[1]), v2 = ld3(V + 3 * iv[2]);
        double b[3] = {gbary[3 * g], gbary[3 * g + 1], gbary[3 * g + 2]};
        double off = goff ? goff[g] : 0.0;
        d3 Gmu = mk(gmu[3 * g], gmu[3 * g + 1], gmu[3 * g + 2]);
        d3 gv[3];
        for (int j = 0; j < 3; ++j) gv[j] = scl(Gmu, b[j]);
        d3 e = sub(v1, v0), e2v = sub(v2, v0);
        d3 nu = cross(e, e2v);
        double l = norm(e), an = norm(nu);
        if (!(l == 0.0 || an == 0.0)) {
            d3 e1 = scl(e, 1.0 / l), n = scl(nu, 1.0 / an), e2 = cross(n, e1);
            double R[3][3] = {{e1.x, e2.x, n.x}, {e1.y, e2.y, n.y}, {e1.z, e2.z, n.z}};
            /* quaternion -> dL/dR through the branch the forward pass used */
            double q[4];
            double tr = R[0][0] + R[1][1] + R[2][2];
            int br;
            if (tr >= R[0][0] && tr >= R[1][1] && tr >= R[2][2]) br = 0;
            else if (R[0][0] >= R[1][1] && R[0][0] >= R[2][2]) br = 1;
            else if (R[1][1] >= R[2][2]) br = 2;
            else br = 3;
            orc_quat_from_R(R, q);
            /* the forward output is sg * (w, x, y, z) of the branch; recover sg */
            double raw[4];
            double Gq[4] = {gq[4 * g], gq[4 * g + 1], gq[4 * g + 2], gq[4 * g + 3]};
            double dR[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            {
                double p, fct;
                /* raw branch values */
                if (br == 0) {
                    p = 0.5 * sqrt(1.0 + tr); fct = 0.25 / p;
                    raw[0] = p; raw[1] = (R[2][1] - R[1][2]) * fct;
                    raw[2] = (R[0][2] - R[2][0]) * fct; raw[3] = (R[1][0] - R[0][1]) * fct;
                } else if (br == 1) {
                    p = 0.5 * sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]); fct = 0.25 / p;
                    raw[1] = p; raw[0] = (R[2][1] - R[1][2]) * fct;
                    raw[2] = (R[0][1] + R[1][0]) * fct; raw[3] = (R[0][2] + R[2][0]) * fct;
                } else if (br == 2) {
                    p = 0.5 * sqrt(1.0 - R[0][0] + R[1][1] - R[2][2]); fct = 0.25 / p;
                    raw[2] = p; raw[0] = (R[0][2] - R[2][0]) * fct;
                    raw[1] = (R[0][1] + R[1][0]) * fct; raw[3] = (R[1][2] + R[2][1]) * fct;
                } else {
                    p = 0.5 * sqrt(1.0 - R[0][0] - R[1][1] + R[2][2]); fct = 0.25 / p;
                    raw[3] = p; raw[0] = (R[1][0] - R[0][1]) * fct;
                    raw[1] = (R[0][2] + R[2][0]) * fct; raw[2] = (R[1][2] + R[2][1]) * fct;
                }
                double sg = 1.0;
                for (int k = 0; k < 4; ++k)
                    if (raw[k] != 0.0) { sg = (q[k] == raw[k]) ? 1.0 : -1.0; break; }
                double G[4];
                for (int k = 0; k < 4; ++k) G[k] = sg * Gq[k];
                /* pivot index of the branch in (w, x, y, z) order, and the
                   3 off-diagonal combinations for the other components */
                int piv = br;               /* 0:w 1:x 2:y 3:z */
                /* off[k] = linear combination of R entries that equals 4 p raw[k] */
                /* d raw[k] = d(off_k)/(4p) - off_k/(4p^2) dp ;  p = 0.5 sqrt(S), dp = dS/(8p) */
                double Gp = G[piv];
                /* contributions of the three non-pivot components */
                for (int k = 0; k < 4; ++k) {
                    if (k == piv) continue;
                    double gk = G[k];
                    double off_k = raw[k] * 4.0 * p;
                    /* d raw_k / d off_k = 1/(4p); d raw_k / d p = -off_k / (4 p^2) */
                    double coef = gk / (4.0 * p);
                    Gp += -gk * off_k / (4.0 * p * p);
                    int a = piv, bb = k;
                    if (a > bb) { int t = a; a = bb; bb = t; }
                    /* pairs: (w,x): R21-R12  (w,y): R02-R20  (w,z): R10-R01
                              (x,y): R01+R10  (x,z): R02+R20  (y,z): R12+R21 */
                    if (a == 0 && bb == 1) { dR[2][1] += coef; dR[1][2] -= coef; }
                    else if (a == 0 && bb == 2) { dR[0][2] += coef; dR[2][0] -= coef; }
                    else if (a == 0 && bb == 3) { dR[1][0] += coef; dR[0][1] -= coef; }
                    else if (a == 1 && bb == 2) { dR[0][1] += coef; dR[1][0] += coef; }
                    else if (a == 1 && bb == 3) { dR[0][2] += coef; dR[2][0] += coef; }
                    else { dR[1][2] += coef; dR[2][1] += coef; }
                }
                /* p = 0.5 sqrt(S): dp/dS = 1/(8p); S = 1 + s0 R00 + s1 R11 + s2 R22 */
                double gS = Gp / (8.0 * p);
                double sgn[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
                for (int d = 0; d < 3; ++d) dR[d][d] += gS * sgn[br][d];
            }
            /* R columns: e1, e2, n */
            d3 ge1 = mk(dR[0][0], dR[1][0], dR[2][0]);
            d3 ge2 = mk(dR[0][1], dR[1][1], dR[2][1]);
            d3 gn = mk(dR[0][2], dR[1][2], dR[2][2]);
            gn = add(gn, scl(Gmu, off));
            /* scale: s0 = rho l, s1 = rho h, s2 = eps rho (l + h)/2, h = an / l */
            double gl = ORC_RHO * gs[3 * g] + ORC_EPS_S * ORC_RHO * 0.5 * gs[3 * g + 2];
            double gh = ORC_RHO * gs[3 * g + 1] + ORC_EPS_S * ORC_RHO * 0.5 * gs[3 * g + 2];
            gl += gh * (-an / (l * l));
            double gan = gh / l;
            /* e2 = n x e1 */
            gn = add(gn, cross(e1, ge2));          /* d(n x e1)/dn^T g = e1 x g */
            ge1 = add(ge1, cross(ge2, n));         /* d(n x e1)/de1^T g = g x n */
            /* n = nu / an, an = |nu| */
            d3 gnu = add(vjp_normalize(nu, an, gn), scl(nu, gan / an));
            /* e1 = e / l, l = |e| */
            d3 ge = add(vjp_normalize(e, l, ge1), scl(e, gl / l));
            /* nu = e x f, f = v2 - v0 */
            ge = add(ge, cross(e2v, gnu));         /* d(e x f)/de^T g = f x g */
            d3 gf = cross(gnu, e);                 /* d(e x f)/df^T g = g x e */
            gv[1] = add(gv[1], ge);
            gv[2] = add(gv[2], gf);
            gv[0] = sub(gv[0], add(ge, gf));
        }
        for (int j = 0; j < 3; ++j) {
            gV[3 * iv[j]] += gv[j].x; gV[3 * iv[j] + 1] += gv[j].y; gV[3 * iv[j] + 2] += gv[j].z;
        }
    }
}

/* ------------------------------------------------------------------ */
/* k-NN weighted surface projection: the NearestSurface of temporal      */
/* tracking (Sec. 3.3, Strategy 1, Eq. 1).  The paper names the method   */
/* but gives neither k nor the weights; the reading used here:           */
/*   the k faces nearest to v (ties: the lower face id), each giving its */
/*   closest point p_j at distance d_j, blended with inverse-distance    */
/*   weights w_j = 1 / max(d_j, delta), delta = 1e-6 times the mesh      */
/*   bounding-box diagonal:  v' = sum w_j p_j / sum w_j.                 */
/* With fewer than k faces, all of them.  Optionally the result is       */
/* blended with an anchor point: v'' = (1 - a) v' + a anchor (the        */
/* periodic re-anchoring to the template projection).                    */
/* ------------------------------------------------------------------ */
#define ORC_KNN_DELTA 1e-6
#define ORC_KNN_MAX 16

void orc_knn_project(const double *V, const int32_t *F, int64_t nF, const double *Q, int64_t nQ,
                     int k, const double *anchor /* nullable */, double anchor_w,
                     double *point, int32_t *face /* [nQ*k], -1 past nF */, double *d2 /* [nQ*k] */) {
    double delta = ORC_KNN_DELTA * orc_mesh_diag(V, F, nF);
    if (k > ORC_KNN_MAX) k = ORC_KNN_MAX;
    for (int64_t q = 0; q < nQ; ++q) {
        double p[3] = {Q[3 * q], Q[3 * q + 1], Q[3 * q + 2]};
        double bd[ORC_KNN_MAX];
        int32_t bf[ORC_KNN_MAX];
        int cnt = 0;
        for (int64_t f = 0; f < nF; ++f) {
            double A[3], B[3], C[3], bb[3], pp[3];
            for (int c = 0; c < 3; ++c) {
                A[c] = V[3 * (int64_t)F[3 * f] + c];
                B[c] = V[3 * (int64_t)F[3 * f + 1] + c];
                C[c] = V[3 * (int64_t)F[3 * f + 2] + c];
            }
            double d = orc_point_triangle(p, A, B, C, bb, pp);
            /* keep the k smallest (d, f); faces come in increasing id, so an
               equal distance never displaces an earlier face */
            if (cnt == k && !(d < bd[k - 1])) continue;
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && d < bd[pos - 1]) {
                bd[pos] = bd[pos - 1];
                bf[pos] = bf[pos - 1];
                --pos;
            }
            bd[pos] = d;
            bf[pos] = (int32_t)f;
            if (cnt < k) ++cnt;
        }
        double sw = 0.0, acc[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < cnt; ++j) {
            double A[3], B[3], C[3], bb[3], pp[3];
            int32_t f = bf[j];
            for (int c = 0; c < 3; ++c) {
                A[c] = V[3 * (int64_t)F[3 * f] + c];
                B[c] = V[3 * (int64_t)F[3 * f + 1] + c];
                C[c] = V[3 * (int64_t)F[3 * f + 2] + c];
            }
            orc_point_triangle(p, A, B, C, bb, pp);
            double dj = sqrt(bd[j]);
            double w = 1.0 / (dj > delta ? dj : delta);
            sw += w;
            for (int c = 0; c < 3; ++c) acc[c] += w * pp[c];
        }
        for (int c = 0; c < 3; ++c) {
            double v = cnt > 0 ? acc[c] / sw : p[c];
            if (anchor) v = (1.0 - anchor_w) * v + anchor_w * anchor[3 * q + c];
            point[3 * q + c] = v;
        }
        for (int j = 0; j < k; ++j) {
            if (face) face[q * k + j] = j < cnt ? bf[j] : -1;
            if (d2) d2[q * k + j] = j < cnt ? bd[j] : INFINITY;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Signed distance for contact (inside negative), by angle-weighted      */
/* pseudo-normals (Baerentzen & Aanaes 2005): the nearest point c of the */
/* NearestSurface query lies in a face interior, on an edge or at a      */
/* vertex (one / two barycentric weights exactly zero); its normal is    */
/* the face's unit normal, the sum of the two unit normals of the faces  */
/* sharing the edge, or the sum over the faces around the vertex of the  */
/* unit normal times the face's angle there.  sign = sign((q - c) . N),  */
/* + when zero.  Assumes a closed, consistently outward-oriented         */
/* (counter-clockwise) manifold mesh; an edge with one face uses that    */
/* face's normal alone.                                                  */
/* ------------------------------------------------------------------ */
static d3 vtx(const double *V, int32_t i) { return ld3(V + 3 * (int64_t)i); }

static d3 face_unit_normal(const double *V, const int32_t *F, int64_t f) {
    d3 a = vtx(V, F[3 * f]), b = vtx(V, F[3 * f + 1]), c = vtx(V, F[3 * f + 2]);
    d3 n = cross(sub(b, a), sub(c, a));
    double l = norm(n);
    return l > 0.0 ? scl(n, 1.0 / l) : mk(0.0, 0.0, 0.0);
}

void orc_signed_distance(const double *V, const int32_t *F, int64_t nF, const double *Q, int64_t nQ,
                         double *sd, int32_t *face) {
    double *bary = (double *)malloc(sizeof(double) * 3 * (size_t)(nQ > 0 ? nQ : 1));
    double *point = (double *)malloc(sizeof(double) * 3 * (size_t)(nQ > 0 ? nQ : 1));
    double *d2 = (double *)malloc(sizeof(double) * (size_t)(nQ > 0 ? nQ : 1));
    orc_closest_point_mesh(V, F, nF, Q, nQ, INFINITY, face, bary, point, d2, NULL);
    for (int64_t q = 0; q < nQ; ++q) {
        int32_t f = face[q];
        if (f < 0) { sd[q] = INFINITY; continue; }
        const double *b = bary + 3 * q;
        int zeros = (b[0] == 0.0) + (b[1] == 0.0) + (b[2] == 0.0);
        d3 N = mk(0.0, 0.0, 0.0);
        if (zeros == 0) {
            N = face_unit_normal(V, F, f);
        } else if (zeros == 1) {
            /* the edge opposite the zero weight */
            int k = b[0] == 0.0 ? 0 : (b[1] == 0.0 ? 1 : 2);
            int32_t x = F[3 * f + (k + 1) % 3], y = F[3 * f + (k + 2) % 3];
            N = face_unit_normal(V, F, f);
            for (int64_t g = 0; g < nF; ++g) {
                if (g == f) continue;
                int hx = 0, hy = 0;
                for (int j = 0; j < 3; ++j) { hx |= F[3 * g + j] == x; hy |= F[3 * g + j] == y; }
                if (hx && hy) { N = add(N, face_unit_normal(V, F, g)); break; }
            }
        } else {
            int k = b[0] != 0.0 ? 0 : (b[1] != 0.0 ? 1 : 2);
            int32_t v = F[3 * f + k];
            for (int64_t g = 0; g < nF; ++g) {
                for (int j = 0; j < 3; ++j) {
                    if (F[3 * g + j] != v) continue;
                    d3 p0 = vtx(V, v), p1 = vtx(V, F[3 * g + (j + 1) % 3]), p2 = vtx(V, F[3 * g + (j + 2) % 3]);
                    d3 e1 = sub(p1, p0), e2 = sub(p2, p0);
                    double l1 = norm(e1), l2 = norm(e2);
                    if (l1 == 0.0 || l2 == 0.0) continue;
                    double cs = dot(e1, e2) / (l1 * l2);
                    if (cs > 1.0) cs = 1.0;
                    if (cs < -1.0) cs = -1.0;
                    N = add(N, scl(face_unit_normal(V, F, g), acos(cs)));
                }
            }
        }
        d3 r = sub(ld3(Q + 3 * q), ld3(point + 3 * q));
        double s = dot(r, N) >= 0.0 ? 1.0 : -1.0;
        sd[q] = s * sqrt(d2[q]);
    }
    free(bary);
    free(point);
    free(d2);
}

/* ------------------------------------------------------------------ */
/* Gaussian splatting render of the face-bound Gaussians (Sec. 3.2's     */
/* R_render; the forward equations of 3D Gaussian splatting, Kerbl et    */
/* al. 2023).  Camera: x_c = Rc x + tc, pixel (u, v) = (fx x_c/z_c + cx, */
/* fy y_c/z_c + cy); a pixel (px, py) samples the point (px, py).        */
/* Per Gaussian: Sigma = M M^T, M = R(q) diag(s); Sigma_c = Rc Sigma     */
/* Rc^T; Sigma_2 = J Sigma_c J^T + 0.3 I with the projection's Jacobian  */
/* J; conic = Sigma_2^-1; radius r = ceil(3 sqrt(lambda_max)); tiles of  */
/* 16 x 16 pixels: [floor((u - r)/16), floor((u + r + 15)/16)) clamped   */
/* to the grid, likewise in y.  z_c <= near, det <= 0 or no tile: culled.*/
/* A pixel blends, front to back by z_c (ties: lower index), the        */
/* Gaussians whose tile range holds its tile:                            */
/*   p = -0.5 (a dx^2 + c dy^2) - b dx dy, d = (u - px, v - py);         */
/*   skip if p > 0; alpha = min(0.99, o e^p); skip if alpha < 1/255;     */
/*   stop if T (1 - alpha) < 1e-4; else C += color alpha T,              */
/*   T *= 1 - alpha.  Result C + T background; T is returned too.        */
/* ------------------------------------------------------------------ */
typedef struct { double u, v, ca, cb, cc, z; int r, x0, x1, y0, y1, ok, flags, fx0, fx1, fy0, fy1, tie; } orc_splat;

/* Flags the pixels of tiles [tx0, tx1) x [ty0, ty1), clamped to the image,  */
/* where the Gaussian o (opacity op) would contribute: alpha within the      */
/* margin of the 1/255 floor or above it.                                    */
static void gs_flag_tiles(unsigned char *fragile, int W, int H, int tx0, int tx1, int ty0, int ty1,
                          const orc_splat *o, double op, double margin) {
    int x0 = tx0 * 16, x1 = tx1 * 16, y0 = ty0 * 16, y1 = ty1 * 16;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W) x1 = W;
    if (y1 > H) y1 = H;
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            double dx = o->u - x, dy = o->v - y;
            double p = -0.5 * (o->ca * dx * dx + o->cc * dy * dy) - o->cb * dx * dy;
            if (fmin(0.99, op * exp(p)) >= (1.0 - margin) / 255.0) fragile[(int64_t)y * W + x] = 1;
        }
}


static const orc_splat *g_sp_sort;
static int cmp_splat(const void *x, const void *y) {
    int i = *(const int *)x, j = *(const int *)y;
    double a = g_sp_sort[i].z, b = g_sp_sort[j].z;
    if (a < b) return -1;
    if (a > b) return 1;
    return (i > j) - (i < j);
}

static void gs_render_impl(const double *mu, const double *quat, const double *scale, const double *opac,
                           const double *color, int64_t n, const double *Rc, const double *tc, double fx,
                           double fy, double cx, double cy, int W, int H, double near_z, const double *bg,
                           double *image, double *trans, double margin, unsigned char *fragile) {
    orc_splat *sp = (orc_splat *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_splat));
    int *order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int gx = (W + 15) / 16, gy = (H + 15) / 16;
    int whole = 0;               /* a cull or a determinant test within reach: every pixel */
    for (int64_t g = 0; g < n; ++g) {
        const double *m = mu + 3 * g, *q = quat + 4 * g, *s = scale + 3 * g;
        double xc[3];
        for (int r = 0; r < 3; ++r) xc[r] = Rc[3 * r] * m[0] + Rc[3 * r + 1] * m[1] + Rc[3 * r + 2] * m[2] + tc[r];
        orc_splat *o = sp + g;
        o->z = xc[2];
        if (fragile && fabs(xc[2] - near_z) <= 1e-5 * fmax(1.0, fmax(fabs(near_z), fabs(xc[2])))) whole = 1;
        if (!(xc[2] > near_z)) continue;
        double w = q[0], x = q[1], y = q[2], z = q[3];
        double qn = sqrt(w * w + x * x + y * y + z * z);
        w /= qn; x /= qn; y /= qn; z /= qn;
        double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                          {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                          {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double M[3][3], S[3][3], T1[3][3], Sc[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                S[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) S[i][j] += M[i][k] * M[j][k];
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                T1[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) T1[i][j] += Rc[3 * i + k] * S[k][j];
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                Sc[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) Sc[i][j] += T1[i][k] * Rc[3 * j + k];
            }
        double iz = 1.0 / xc[2];
        double J[2][3] = {{fx * iz, 0.0, -fx * xc[0] * iz * iz}, {0.0, fy * iz, -fy * xc[1] * iz * iz}};
        double JS[2][3], C2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                JS[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) JS[i][j] += J[i][k] * Sc[k][j];
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                C2[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) C2[i][j] += JS[i][k] * J[j][k];
            }
        double a = C2[0][0] + 0.3, b = C2[0][1], c = C2[1][1] + 0.3;
        double det = a * c - b * b;
        if (fragile && fabs(det) <= 1e-4 * (fabs(a * c) + b * b)) whole = 1;
        if (!(det > 0.0)) continue;
        double mid = 0.5 * (a + c);
        double lam = mid + sqrt(fmax(0.1, mid * mid - det));
        int r = (int)ceil(3.0 * sqrt(lam));
        double u = fx * xc[0] * iz + cx, v = fy * xc[1] * iz + cy;
        int x0 = (int)((u - r) / 16.0), x1 = (int)((u + r + 15) / 16.0);
        int y0 = (int)((v - r) / 16.0), y1 = (int)((v + r + 15) / 16.0);
        if (fragile) {
            /* the radius and the four tile bounds, each within float32 reach of a step */
            double rr = 3.0 * sqrt(lam), mpx = 2e-5 * fmax(64.0, fmax(fabs(u), fabs(v)));
            double bx0 = (u - r) / 16.0, bx1 = (u + r + 15) / 16.0, by0 = (v - r) / 16.0, by1 = (v + r + 15) / 16.0;
            o->flags = (fabs(rr - nearbyint(rr)) <= 1e-5 * fmax(1.0, rr) ? 1 : 0) |
                       (fabs(bx0 - nearbyint(bx0)) <= mpx / 16.0 ? 2 : 0) |
                       (fabs(bx1 - nearbyint(bx1)) <= mpx / 16.0 ? 4 : 0) |
                       (fabs(by0 - nearbyint(by0)) <= mpx / 16.0 ? 8 : 0) |
                       (fabs(by1 - nearbyint(by1)) <= mpx / 16.0 ? 16 : 0);
            /* the unclamped tile bounds and the footprint, for the strips flagged below */
            o->fx0 = x0; o->fx1 = x1; o->fy0 = y0; o->fy1 = y1;
            o->u = u; o->v = v; o->ca = c / det; o->cb = -b / det; o->cc = a / det; o->r = r;
        }
        x0 = x0 < 0 ? 0 : (x0 > gx ? gx : x0); x1 = x1 < 0 ? 0 : (x1 > gx ? gx : x1);
        y0 = y0 < 0 ? 0 : (y0 > gy ? gy : y0); y1 = y1 < 0 ? 0 : (y1 > gy ? gy : y1);
        if ((x1 - x0) * (y1 - y0) == 0) continue;
        o->u = u; o->v = v; o->ca = c / det; o->cb = -b / det; o->cc = a / det;
        o->r = r; o->x0 = x0; o->x1 = x1; o->y0 = y0; o->y1 = y1; o->ok = 1;
    }
    int m = 0;
    for (int64_t g = 0; g < n; ++g) if (sp[g].ok) order[m++] = (int)g;
    g_sp_sort = sp;
    qsort(order, (size_t)m, sizeof(int), cmp_splat);
    if (fragile) {
        memset(fragile, whole ? 1 : 0, (size_t)W * (size_t)H);
        /* depth order: runs of neighbours in the sorted order within float32 reach of    */
        /* each other share a tie group (the sorted position of the run's first)          */
        for (int k = 0; k < m; ++k) sp[order[k]].tie = -1;
        for (int k = 0; k + 1 < m; ++k) {
            double za = sp[order[k]].z, zb = sp[order[k + 1]].z;
            if (zb - za <= 1e-6 * fmax(1.0, fmax(fabs(za), fabs(zb)))) {
                if (sp[order[k]].tie < 0) sp[order[k]].tie = k;
                sp[order[k + 1]].tie = sp[order[k]].tie;
            }
        }
        /* a radius or tile bound near a step: the one tile column or row each such step    */
        /* adds or drops (a bound near integer k moves between k - 1 and k, so column k - 1 */
        /* is in or out; a radius step moves every bound by the r -> r +- 1 change)          */
        for (int64_t g = 0; g < n; ++g) {        /* culled for no tile too: a step may add one */
            const orc_splat *o = sp + g;
            int f = o->flags;
            if (!(f & 31)) continue;
            int r = o->r;
            int c0lo = o->fx0, c0hi = o->fx0, c1lo = o->fx1, c1hi = o->fx1;
            int r0lo = o->fy0, r0hi = o->fy0, r1lo = o->fy1, r1hi = o->fy1;
            for (int dr = -1; dr <= 1; dr += 2) {
                if (!(f & 1)) break;
                int rr = r + dr;
                int a0 = (int)((o->u - rr) / 16.0), a1 = (int)((o->u + rr + 15) / 16.0);
                int b0 = (int)((o->v - rr) / 16.0), b1 = (int)((o->v + rr + 15) / 16.0);
                c0lo = a0 < c0lo ? a0 : c0lo; c0hi = a0 > c0hi ? a0 : c0hi;
                c1lo = a1 < c1lo ? a1 : c1lo; c1hi = a1 > c1hi ? a1 : c1hi;
                r0lo = b0 < r0lo ? b0 : r0lo; r0hi = b0 > r0hi ? b0 : r0hi;
                r1lo = b1 < r1lo ? b1 : r1lo; r1hi = b1 > r1hi ? b1 : r1hi;
            }
            if (f & 2) { int k = (int)nearbyint((o->u - r) / 16.0); c0lo = c0lo < k - 1 ? c0lo : k - 1; c0hi = c0hi > k ? c0hi : k; }
            if (f & 4) { int k = (int)nearbyint((o->u + r + 15) / 16.0); c1lo = c1lo < k - 1 ? c1lo : k - 1; c1hi = c1hi > k ? c1hi : k; }
            if (f & 8) { int k = (int)nearbyint((o->v - r) / 16.0); r0lo = r0lo < k - 1 ? r0lo : k - 1; r0hi = r0hi > k ? r0hi : k; }
            if (f & 16) { int k = (int)nearbyint((o->v + r + 15) / 16.0); r1lo = r1lo < k - 1 ? r1lo : k - 1; r1hi = r1hi > k ? r1hi : k; }
            /* the columns [c0lo, c0hi) and [c1lo, c1hi), the rows [r0lo, r0hi) and [r1lo, r1hi) */
            int ylo = r0lo, yhi = r1hi, xlo = c0lo, xhi = c1hi;
            gs_flag_tiles(fragile, W, H, c0lo, c0hi, ylo, yhi, o, opac[g], margin);
            gs_flag_tiles(fragile, W, H, c1lo, c1hi, ylo, yhi, o, opac[g], margin);
            gs_flag_tiles(fragile, W, H, xlo, xhi, r0lo, r0hi, o, opac[g], margin);
            gs_flag_tiles(fragile, W, H, xlo, xhi, r1lo, r1hi, o, opac[g], margin);
        }
    }
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int tx = px / 16, ty = py / 16;
            double T = 1.0, C[3] = {0.0, 0.0, 0.0};
            int last_tie = -1;                  /* tie group of the last contributor */
            double tre = 0.0;                   /* relative error bound of a float32 T so far */
            for (int k = 0; k < m; ++k) {
                const orc_splat *o = sp + order[k];
                if (tx < o->x0 || tx >= o->x1 || ty < o->y0 || ty >= o->y1) continue;
                double dx = o->u - px, dy = o->v - py;
                double p = -0.5 * (o->ca * dx * dx + o->cc * dy * dy) - o->cb * dx * dy;
                if (p > 0.0) continue;
                double raw = opac[order[k]] * exp(p);
                double alpha = fmin(0.99, raw);
                double tt = T * (1.0 - alpha);
                if (fragile) {
                    /* two members of one tie group reach the pixel: their order may swap */
                    int tie_pair = 0, near_stop = 0;
                    if (alpha >= 1.0 / 255.0) {
                        tie_pair = o->tie >= 0 && o->tie == last_tie;
                        last_tie = o->tie;
                        /* T (1 - alpha) carries every earlier alpha's relative error, each
                         * amplified by alpha / (1 - alpha), and one rounding per step */
                        tre += margin * alpha / (1.0 - alpha) + 0x1p-23;
                        near_stop = fabs(tt - 1e-4) <= tre * tt;
                    }
                    if (fabs(raw - 0.99) <= margin * 0.99 || fabs(alpha - 1.0 / 255.0) <= margin / 255.0 ||
                        near_stop || tie_pair)
                        fragile[(int64_t)py * W + px] = 1;
                }
                if (alpha < 1.0 / 255.0) continue;
                if (tt < 1e-4) {
                    /* the stop falls on a member of a tie group: another member may come   */
                    /* first in float32 order and the stop land elsewhere                    */
                    if (fragile && o->tie >= 0) fragile[(int64_t)py * W + px] = 1;
                    break;
                }
                for (int ch = 0; ch < 3; ++ch) C[ch] += color[3 * (int64_t)order[k] + ch] * alpha * T;
                T = tt;
            }
            for (int ch = 0; ch < 3; ++ch) image[3 * ((int64_t)py * W + px) + ch] = C[ch] + T * bg[ch];
            trans[(int64_t)py * W + px] = T;
        }
    free(sp);
    free(order);
}

void orc_gs_render(const double *mu, const double *quat, const double *scale, const double *opac,
                   const double *color, int64_t n, const double *Rc, const double *tc, double fx,
                   double fy, double cx, double cy, int W, int H, double near_z, const double *bg,
                   double *image /* [H][W][3] */, double *trans /* [H][W] */) {
    gs_render_impl(mu, quat, scale, opac, color, n, Rc, tc, fx, fy, cx, cy, W, H, near_z, bg, image, trans, 0.0,
                   NULL);
}

/* orc_gs_render with parity flags (test infrastructure: which pixels a float32 */
/* implementation of the same equations may legitimately render differently).   */
/* fragile[py][px] = 1 where a discrete decision of the forward that reaches the */
/* pixel lies, in float64, within float32 reach of its threshold: the cull at    */
/* near_z or det > 0 (every pixel), the 3-sigma radius's ceil or a tile-square   */
/* bound's truncation (the pixels of the tile strips it may add or drop that the */
/* Gaussian reaches), the depth order of neighbours closer than 1e-6 relative    */
/* (two of them reach the pixel, or the transmittance stop falls on one), and the*/
/* per-pixel 0.99 cap and 1/255 floor (relative margin `margin`, the bound of a */
/* float32 alpha's relative error) and 1e-4 transmittance stop (within the     */
/* transmittance's own error bound: the sum over the alphas before it of        */
/* margin x alpha / (1 - alpha), plus 2^-23 a step).  The image and            */
/* transmittance are orc_gs_render's, bit for bit.                               */
void orc_gs_render_flags(const double *mu, const double *quat, const double *scale, const double *opac,
                         const double *color, int64_t n, const double *Rc, const double *tc, double fx,
                         double fy, double cx, double cy, int W, int H, double near_z, const double *bg,
                         double margin, double *image, double *trans, unsigned char *fragile) {
    gs_render_impl(mu, quat, scale, opac, color, n, Rc, tc, fx, fy, cx, cy, W, H, near_z, bg, image, trans, margin,
                   fragile);
}
