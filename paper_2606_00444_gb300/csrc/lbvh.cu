// LBVH construction and refit over a triangle mesh.
//
// The paper builds its collision structure once from the template faces and
// afterwards only replaces the vertex buffer (Sec. 3.4); the varying-topology
// baseline rebuilds it every frame (Sec. 4.1).  The paper gives no
// construction, so the build here is a linear BVH: 30-bit Morton keys of face
// centroids, a stable LSD radix sort, Karras's (2012) binary radix tree, and
// boxes computed bottom-up.  The refit reuses the tree and recomputes boxes.
#include <atomic>
#include <cstdlib>
#include <cstring>

#include <climits>
#include <utility>
#include <vector>

#include "common.cuh"
#include "gauss_math.cuh"

namespace meshgs {

static std::atomic<unsigned long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n); }

mesh_status check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MESH_OK : MESH_ERR_CUDA;
}

constexpr int kBlock = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per sort tile
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kRadix = 256;
constexpr int kScanThreads = 256;     // one block per digit; also scans the 256 digit totals
static_assert(kSortThreads == kRadix, "one thread per digit in the sort kernels");

// ---------------------------------------------------------------------------
// Float <-> order-preserving unsigned encoding, so box extremes can be reduced
// with integer atomics (exact: min / max need no rounding).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------------------
// a1: vertex-buffer update, [nV][3] -> float4 [nV] (w = 0).
// Optionally (re)initialises the 6-word centroid box used by the Morton step.
// ---------------------------------------------------------------------------
__global__ void k_copy_verts(const float *__restrict__ V3, int nV, float4 *__restrict__ V4,
                             unsigned int *__restrict__ cbox) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (cbox && i < 6) cbox[i] = (i < 3) ? 0xffffffffu : 0u;
    if (i >= nV) return;
    const float *p = V3 + 3 * (size_t)i;
    V4[i] = make_float4(p[0], p[1], p[2], 0.0f);
}

// ---------------------------------------------------------------------------
// Face table repack [nF][3] -> int4 (v0, v1, v2, 0) with index validation, and
// the centroid sum s = (v0 + v1) + v2 in float32 round-to-nearest (the Morton
// recipe uses the sum, not the mean: the normalisation absorbs the factor 3).
// The per-block min / max of s goes to the centroid box by ordered atomics.
// ---------------------------------------------------------------------------
__global__ void k_faces_centroids(const int *__restrict__ F3, int nF, int nV,
                                  const float4 *__restrict__ V4, int4 *__restrict__ F4,
                                  float4 *__restrict__ cent, unsigned int *__restrict__ cbox,
                                  Header *__restrict__ hdr) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (f < nF) {
        const int *p = F3 + 3 * (size_t)f;
        int i0 = p[0], i1 = p[1], i2 = p[2];
        bool bad = (unsigned)i0 >= (unsigned)nV || (unsigned)i1 >= (unsigned)nV ||
                   (unsigned)i2 >= (unsigned)nV;
        if (bad) {
            set_status(hdr, MESH_DEV_INDEX_RANGE);
            if ((unsigned)i0 >= (unsigned)nV) i0 = 0;
            if ((unsigned)i1 >= (unsigned)nV) i1 = 0;
            if ((unsigned)i2 >= (unsigned)nV) i2 = 0;
        }
        F4[f] = make_int4(i0, i1, i2, 0);
        float4 a = V4[i0], b = V4[i1], c = V4[i2];
        float s0 = __fadd_rn(__fadd_rn(a.x, b.x), c.x);
        float s1 = __fadd_rn(__fadd_rn(a.y, b.y), c.y);
        float s2 = __fadd_rn(__fadd_rn(a.z, b.z), c.z);
        cent[f] = make_float4(s0, s1, s2, 0.0f);
        lo[0] = hi[0] = s0;
        lo[1] = hi[1] = s1;
        lo[2] = hi[2] = s2;
    }
    // warp then block reduction of the 6 extremes
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    __shared__ float s_lo[3][kBlock / 32], s_hi[3][kBlock / 32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) { s_lo[k][w] = lo[k]; s_hi[k][w] = hi[k]; }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        float l = s_lo[k][0], h = s_hi[k][0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            l = fminf(l, s_lo[k][i]);
            h = fmaxf(h, s_hi[k][i]);
        }
        if (l <= h) {
            atomicMin(&cbox[k], f2ord(l));
            atomicMax(&cbox[3 + k], f2ord(h));
        }
    }
}

// Sort keys for points: a point p is keyed as the zero-area face (p, p, p),
// i.e. s = (p + p) + p in float32 round-to-nearest, so points and faces share
// one Morton recipe.
__global__ void k_points_centroids(const float *__restrict__ P, int n, float4 *__restrict__ cent,
                                   unsigned int *__restrict__ cbox) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < n) {
        const float *p = P + 3 * (size_t)i;
        float s0 = __fadd_rn(__fadd_rn(p[0], p[0]), p[0]);
        float s1 = __fadd_rn(__fadd_rn(p[1], p[1]), p[1]);
        float s2 = __fadd_rn(__fadd_rn(p[2], p[2]), p[2]);
        cent[i] = make_float4(s0, s1, s2, 0.0f);
        lo[0] = hi[0] = s0;
        lo[1] = hi[1] = s1;
        lo[2] = hi[2] = s2;
    }
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    __shared__ float s_lo[3][kBlock / 32], s_hi[3][kBlock / 32];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) { s_lo[k][w] = lo[k]; s_hi[k][w] = hi[k]; }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        float l = s_lo[k][0], h = s_hi[k][0];
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
            l = fminf(l, s_lo[k][j]);
            h = fmaxf(h, s_hi[k][j]);
        }
        if (l <= h) {
            atomicMin(&cbox[k], f2ord(l));
            atomicMax(&cbox[3 + k], f2ord(h));
        }
    }
}

__global__ void k_init_box(unsigned int *cbox) {
    if (threadIdx.x < 6) cbox[threadIdx.x] = (threadIdx.x < 3) ? 0xffffffffu : 0u;
}

// Bit i of v (10 bits) moved to bit 3i.
__device__ __forceinline__ unsigned int spread3(unsigned int v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// ---------------------------------------------------------------------------
// a2: 30-bit Morton key per face.  t = (s - lo) * (1 / (hi - lo)) per axis,
// q = clamp(floor(t * 1024), 0, 1023), bits interleaved x-major.  Every
// float operation is an explicit round-to-nearest intrinsic so no FMA
// contraction can change a key.
// ---------------------------------------------------------------------------
__global__ void k_morton(const float4 *__restrict__ cent, int nF,
                         const unsigned int *__restrict__ cbox, unsigned int *__restrict__ keys,
                         int *__restrict__ vals) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    float lo[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = ord2f(cbox[k]);
        float ext = __fsub_rn(ord2f(cbox[3 + k]), lo[k]);
        inv[k] = ext > 0.0f ? __fdiv_rn(1.0f, ext) : 0.0f;
    }
    float4 s = cent[f];
    float sv[3] = {s.x, s.y, s.z};
    unsigned int q[3];
    for (int k = 0; k < 3; ++k) {
        float t = __fmul_rn(__fsub_rn(sv[k], lo[k]), inv[k]);
        float x = floorf(__fmul_rn(t, 1024.0f));
        int qi = (int)x;
        qi = qi < 0 ? 0 : (qi > 1023 ? 1023 : qi);
        q[k] = (unsigned int)qi;
    }
    keys[f] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    vals[f] = f;
}

// ---------------------------------------------------------------------------
// a3: stable LSD radix sort of (key, face id), 8 bits per pass, reduce-then-
// scan (three kernels per pass, no inter-block waiting of any kind).
//   upsweep:   per-tile digit histogram, stored digit-major hist[d * T + t]
//   scan:      one block, exclusive scan of hist in that order, which makes
//              hist[d * T + t] the global output offset of digit d in tile t
//   downsweep: stable in-tile ranking (warp match_any + per-warp counters),
//              scatter through shared memory, coalesced write-out.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
k_sort_upsweep(const unsigned int *__restrict__ keys, int n, int shift,
               unsigned int *__restrict__ hist, int T, unsigned int *__restrict__ ticket) {
    __shared__ unsigned int h[kRadix];
    pdl_wait();
    pdl_trigger();
    h[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0u;   // the scan's ticket (it runs after this kernel)
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int idx = base + r * kSortThreads + threadIdx.x;
        bool valid = idx < n;
        unsigned int d = valid ? (keys[idx] >> shift) & 0xffu : 0x100u;
        unsigned int peers = __match_any_sync(0xffffffffu, d);
        if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&h[d], (unsigned)__popc(peers));
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * T + blockIdx.x] = h[threadIdx.x];
}

__device__ __forceinline__ unsigned int warp_incl_scan(unsigned int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of the per-thread values of one block (blockDim a multiple of 32,
// at most 1024 threads).  Returns the exclusive prefix; *total gets the sum.
__device__ unsigned int block_excl_scan(unsigned int x, unsigned int *s_warp, unsigned int *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned int inc = warp_incl_scan(x, lane);
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned int v = lane < nw ? s_warp[lane] : 0u;
        unsigned int vi = warp_incl_scan(v, lane);
        if (lane < nw) s_warp[lane] = vi - v;
        if (lane == 31) s_warp[32] = vi;
    }
    __syncthreads();
    unsigned int r = s_warp[w] + inc - x;
    if (total) *total = s_warp[32];
    __syncthreads();
    return r;
}

// Offsets for one pass, by one block per digit d: an exclusive scan of the
// digit's per-tile counts hist[d * T + t] (in place, tile offsets within the
// digit), and the digit's total.  The last block to finish (ticket counter;
// nobody waits) turns the 256 totals into exclusive digit bases and resets the
// ticket.  The output position of digit d in tile t is base[d] + hist[d*T+t].
__global__ void __launch_bounds__(kScanThreads)
k_sort_scan(unsigned int *__restrict__ hist, int T, unsigned int *__restrict__ dsum,
            unsigned int *__restrict__ base, unsigned int *__restrict__ ticket) {
    __shared__ unsigned int s_warp[33];
    __shared__ bool s_last;
    pdl_wait();
    pdl_trigger();
    unsigned int *h = hist + (size_t)blockIdx.x * T;
    unsigned int carry = 0;
    const int chunk = kScanThreads * 4;
    for (int b0 = 0; b0 < T; b0 += chunk) {
        int i0 = b0 + 4 * threadIdx.x;
        unsigned int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (i0 + k < T) ? h[i0 + k] : 0u;
        unsigned int tot;
        unsigned int run = carry + block_excl_scan(v[0] + v[1] + v[2] + v[3], s_warp, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < T) h[i0 + k] = run;
            run += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        dsum[blockIdx.x] = carry;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned int x = threadIdx.x < kRadix ? __ldcg(dsum + threadIdx.x) : 0u;
    unsigned int ex = block_excl_scan(x, s_warp, nullptr);
    if (threadIdx.x < kRadix) base[threadIdx.x] = ex;
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_downsweep(const unsigned int *__restrict__ kin, const int *__restrict__ vin,
                 unsigned int *__restrict__ kout, int *__restrict__ vout, int n, int shift,
                 const unsigned int *__restrict__ hist, int T,
                 const unsigned int *__restrict__ dbase) {
    __shared__ unsigned int s_keys[kSortTile];
    __shared__ int s_vals[kSortTile];
    __shared__ unsigned int s_wcnt[kSortWarps][kRadix];
    __shared__ unsigned int s_dstart[kRadix];
    __shared__ unsigned int s_goff[kRadix];
    __shared__ unsigned int s_warp[33];
    pdl_wait();
    pdl_trigger();
    int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
    unsigned int key[kSortItems], rank[kSortItems];
    int val[kSortItems];
    unsigned int lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int idx = base + w * (32 * kSortItems) + r * 32 + lane;
        bool valid = idx < n;
        key[r] = valid ? kin[idx] : 0u;
        val[r] = valid ? (vin ? vin[idx] : idx) : 0;      // vin NULL: the values are the indices
        unsigned int d = valid ? (key[r] >> shift) & 0xffu : 0x100u;
        unsigned int peers = __match_any_sync(0xffffffffu, d);
        unsigned int before = valid ? s_wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt_mask) == 0u) s_wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = valid ? before + __popc(peers & lt_mask) : 0xffffffffu;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then exclusive scan over digits
    unsigned int run = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
        unsigned int c = s_wcnt[ww][tid];
        s_wcnt[ww][tid] = run;
        run += c;
    }
    unsigned int start = block_excl_scan(run, s_warp, nullptr);
    s_dstart[tid] = start;
    s_goff[tid] = dbase[tid] + hist[(size_t)tid * T + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (rank[r] != 0xffffffffu) {
            unsigned int d = (key[r] >> shift) & 0xffu;
            unsigned int pos = s_dstart[d] + s_wcnt[w][d] + rank[r];
            s_keys[pos] = key[r];
            s_vals[pos] = val[r];
        }
    }
    __syncthreads();
    int nvalid = min(kSortTile, n - base);
    for (int i = tid; i < nvalid; i += kSortThreads) {
        unsigned int k = s_keys[i];
        unsigned int d = (k >> shift) & 0xffu;
        unsigned int g = s_goff[d] + (unsigned)i - s_dstart[d];
        kout[g] = k;
        vout[g] = s_vals[i];
    }
}

// ---------------------------------------------------------------------------
// a4: Karras (2012) hierarchy, one thread per internal node i in [0, n-2].
// delta(i, j) = common-prefix length of the keys augmented with their sorted
// position; -1 outside [0, n).  The node's range has i at one end; its
// direction, far end and split are found by exponential + binary search.
// Children go to the node record's .w slots; parent[] gets 2*i + side.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int kdelta(const unsigned int *__restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned int a = k[i], b = k[j];
    return a != b ? __clz(a ^ b) : 32 + __clz((unsigned)i ^ (unsigned)j);
}

// Children of internal node i of the tree over keys[0, n) (Karras 2012).
__device__ __forceinline__ void karras_children(const unsigned int *__restrict__ keys, int n, int i,
                                                int &left, int &right, int &far_end) {
    int d = (kdelta(keys, n, i, i + 1) - kdelta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = kdelta(keys, n, i, i - d);
    int lmax = 2;
    while (kdelta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (kdelta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = kdelta(keys, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (kdelta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    left = (lo == gamma) ? -(gamma + 1) : gamma;
    right = (hi == gamma + 1) ? -(gamma + 2) : gamma + 1;
    far_end = j;
}

// Child links of internal node i: lo.w = the child (internal c >= 0, leaf j as
// -(j+1)), hi.w = the number of faces of a leaf link (1 here) or c again.
__device__ __forceinline__ void write_children(float4 *__restrict__ nodes, int i, int left, int right) {
    float *rec = reinterpret_cast<float *>(nodes + 4 * (size_t)i);
    rec[3] = __int_as_float(left);
    rec[7] = __int_as_float(left < 0 ? 1 : left);
    rec[11] = __int_as_float(right);
    rec[15] = __int_as_float(right < 0 ? 1 : right);
}

__global__ void k_karras(const unsigned int *__restrict__ keys, int n, float4 *__restrict__ nodes,
                         int *__restrict__ parent, int *__restrict__ rend) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int left, right, far_end;
    karras_children(keys, n, i, left, right, far_end);
    rend[i] = far_end;
    write_children(nodes, i, left, right);
    parent[left >= 0 ? left : (n - 1) + (-left - 1)] = 2 * i;
    parent[right >= 0 ? right : (n - 1) + (-right - 1)] = 2 * i + 1;
    if (i == 0) parent[0] = -1;
}

// Exact zero-area test: the products of float32 coordinate differences are
// exact in float64 (each difference of two float32 values of similar
// magnitude has at most 25 significant bits), so the cross product is zero
// here exactly when it is zero in exact arithmetic.  A float32 evaluation
// first settles the common case: a component whose magnitude exceeds 2^-21
// of |p1| + |p2| (the two products it is the difference of) is nonzero in
// exact arithmetic too -- the rounding of the differences, the products and
// the subtraction moves it by at most about 4 * 2^-24 of that sum -- so the
// float64 pipe is used only for (nearly) degenerate triangles.
__device__ __forceinline__ bool clearly_nonzero(float p1, float p2) {
    float s = fabsf(p1) + fabsf(p2);
    return s > 1e-30f && s < 1e30f && fabsf(p1 - p2) > 0x1p-21f * s;
}

__device__ __forceinline__ bool exactly_degenerate(float4 a, float4 b, float4 c) {
    float fux = b.x - a.x, fuy = b.y - a.y, fuz = b.z - a.z;
    float fvx = c.x - a.x, fvy = c.y - a.y, fvz = c.z - a.z;
    if (clearly_nonzero(fuy * fvz, fuz * fvy) || clearly_nonzero(fuz * fvx, fux * fvz) ||
        clearly_nonzero(fux * fvy, fuy * fvx))
        return false;
    double ux = (double)b.x - a.x, uy = (double)b.y - a.y, uz = (double)b.z - a.z;
    double vx = (double)c.x - a.x, vy = (double)c.y - a.y, vz = (double)c.z - a.z;
    return (uy * vz - uz * vy) == 0.0 && (uz * vx - ux * vz) == 0.0 && (ux * vy - uy * vx) == 0.0;
}

// ---------------------------------------------------------------------------
// a5 (build and refit): bottom-up boxes in two kernels, without a climb.
//
// The box of an internal node is the union of the leaf boxes over its leaf
// range [a, b] (Karras's nodes cover contiguous ranges of the sorted leaves),
// so the boxes need no bottom-up dependency chain at all: they are range
// queries.  One block per kRefitBlock consecutive leaves:
//   * builds a sparse table of its leaf boxes in shared memory (level k holds
//     the union over [i, i + 2^k)), one level per round and one barrier per
//     level, reading consecutive entries (no bank conflicts);
//   * answers every internal node whose range lies inside the block (such a
//     node's index is one end of its range, so it is in the block's index
//     range) from two entries of level floor(log2(b - a + 1)) as soon as that
//     level exists;
//   * writes the prefix and suffix unions of its leaves and its own box.
// Every leaf and node writes its box into its parent's record half, so the
// records need no second pass.  The nodes whose ranges cross a block boundary
// -- a few per boundary -- are listed per block; the second kernel answers
// each of them with one warp: suffix union in the first block, prefix union
// in the last, and the boxes of the blocks between.  No atomics, no fences,
// no spin, and the result does not depend on thread timing.  When the caller
// passes new vertices, the first kernel also repacks them (a1) and gathers
// the triangles from the caller's buffer.
// ---------------------------------------------------------------------------
constexpr int kRefitBlock = 512;
constexpr int kRefitLevels = 9;                           // log2(kRefitBlock)

__device__ __forceinline__ bool crosses_block(int i, int j) {
    return (min(i, j) / kRefitBlock) != (max(i, j) / kRefitBlock);
}

__device__ __forceinline__ float4 box_min(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.0f);
}
__device__ __forceinline__ float4 box_max(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), 0.0f);
}

// Corners of face fv from the caller's [nV][3] buffer (V3) or the repacked one.
__device__ __forceinline__ void load_tri(const float *__restrict__ V3, const float4 *__restrict__ V4,
                                         int4 fv, float4 &a, float4 &b, float4 &c) {
    if (V3) {
        const float *pa = V3 + 3 * (size_t)fv.x, *pb = V3 + 3 * (size_t)fv.y, *pc = V3 + 3 * (size_t)fv.z;
        a = make_float4(pa[0], pa[1], pa[2], 0.0f);
        b = make_float4(pb[0], pb[1], pb[2], 0.0f);
        c = make_float4(pc[0], pc[1], pc[2], 0.0f);
    } else {
        a = V4[fv.x]; b = V4[fv.y]; c = V4[fv.z];
    }
}

// Writes box (lo, hi) of a child into its parent's record half, or into the
// header when it is the root (parent link pe < 0), with the child's link:
// `link` in lo.w (internal c >= 0, or -(first+1) for a leaf range) and `cnt`
// in hi.w (the range's face count, or c again for an internal child).
__device__ __forceinline__ void put_box(float4 *__restrict__ nodes, Header *__restrict__ hdr, int pe,
                                        int link, int cnt, float4 lo, float4 hi) {
    if (pe < 0) {
        hdr->root_lo = make_float4(lo.x, lo.y, lo.z, 0.0f);
        hdr->root_hi = make_float4(hi.x, hi.y, hi.z, 0.0f);
        return;
    }
    float4 *rec = nodes + 4 * (size_t)(pe >> 1) + 2 * (pe & 1);
    rec[0] = make_float4(lo.x, lo.y, lo.z, __int_as_float(link));
    rec[1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(cnt));
}

// Leaf collapse (leaf size L): internal node j over leaves [ra, rb] is linked
// from its parent as the leaf range (-(ra+1), rb - ra + 1) when it holds at
// most L faces, otherwise as itself.  A search then tests the faces of the
// topmost subtree of at most L faces in one loop instead of visiting its nodes
// (which are still refit: unreachable, and cheap to keep exact).
__device__ __forceinline__ void node_link(int j, int ra, int rb, int L, int &link, int &cnt) {
    int len = rb - ra + 1;
    if (len <= L) { link = -(ra + 1); cnt = len; }
    else { link = j; cnt = j; }
}

// Box of six floats in shared memory, structure of arrays ([6][kRefitBlock]).
struct SBox {
    float *f;
    __device__ float4 lo(int i) const { return make_float4(f[i], f[kRefitBlock + i], f[2 * kRefitBlock + i], 0.0f); }
    __device__ float4 hi(int i) const {
        return make_float4(f[3 * kRefitBlock + i], f[4 * kRefitBlock + i], f[5 * kRefitBlock + i], 0.0f);
    }
    __device__ void put(int i, float4 l, float4 h) const {
        f[i] = l.x; f[kRefitBlock + i] = l.y; f[2 * kRefitBlock + i] = l.z;
        f[3 * kRefitBlock + i] = h.x; f[4 * kRefitBlock + i] = h.y; f[5 * kRefitBlock + i] = h.z;
    }
};

// Face-bound Gaussians rebound in the refit pass (mesh_refit_bind): the
// Gaussians of face f are gstart[f] .. gstart[f + 1] - 1; gstart == NULL: none.
struct Rebind {
    const int *gstart;
    const float *gbary, *goff;
    int64_t nG;
    float *mu, *quat, *scale;
};

// Per-leaf record of the rebind, in shared memory after the table rounds
// ([kBindFloats][kRefitBlock]): corners a, b, c, unit normal, rotation, scale,
// degenerate flag.
constexpr int kBindFloats = 20;

constexpr size_t kRefitLocalSmem = 12 * kRefitBlock * sizeof(float)      // two table levels
                                   + 64 * sizeof(int);                    // crossing-list scan
constexpr size_t kRefitBindSmem = kBindFloats * kRefitBlock * sizeof(float)   // rebind records
                                  + 64 * sizeof(int)                          // scans
                                  + 2 * kRefitBlock * sizeof(int);            // Gaussian offsets, starts

// The Gaussians of a refit block's leaves, one per thread: leaf l (this
// thread's when l = threadIdx.x) holds gcnt Gaussians from index gs on and its
// record in rec.  A block whose Gaussian count overflows an int sets
// MESH_DEV_INDEX_RANGE and writes none (only an overlapping face CSR can).
__device__ __forceinline__ void bind_block(const float *__restrict__ rec, int *__restrict__ s_scan, int gs,
                                           int gcnt, const Rebind &RB, Header *__restrict__ hdr) {
    int *s_off = s_scan + 64, *s_gs = s_off + kRefitBlock;
    long long *s_wsum = reinterpret_cast<long long *>(s_scan);   // 16 warp totals (64-bit)
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    long long x = gcnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[wid] = x;
    __syncthreads();
    long long before = 0, total = 0;
    for (int w = 0; w < kRefitBlock / 32; ++w) {
        long long v = s_wsum[w];
        if (w < wid) before += v;
        total += v;
    }
    if (total > INT_MAX) {
        if (tid == 0) set_status(hdr, MESH_DEV_INDEX_RANGE);
        return;
    }
    s_off[tid] = (int)(before + x - gcnt);
    s_gs[tid] = gs;
    __syncthreads();
    for (int t = tid; t < (int)total; t += kRefitBlock) {
        int l = 0;                                       // the last leaf whose offset is <= t
#pragma unroll
        for (int h = kRefitBlock / 2; h > 0; h >>= 1)
            if (s_off[l + h] <= t) l += h;
        int64_t g = (int64_t)s_gs[l] + (t - s_off[l]);
        const float *r = rec + l;
        V3 a{r[0], r[kRefitBlock], r[2 * kRefitBlock]}, b{r[3 * kRefitBlock], r[4 * kRefitBlock], r[5 * kRefitBlock]};
        V3 c{r[6 * kRefitBlock], r[7 * kRefitBlock], r[8 * kRefitBlock]};
        V3 nrm{r[9 * kRefitBlock], r[10 * kRefitBlock], r[11 * kRefitBlock]};
        float q[4] = {r[12 * kRefitBlock], r[13 * kRefitBlock], r[14 * kRefitBlock], r[15 * kRefitBlock]};
        float sc[3] = {r[16 * kRefitBlock], r[17 * kRefitBlock], r[18 * kRefitBlock]};
        bool deg = r[19 * kRefitBlock] != 0.0f;
        V3 m = gaussian_centre(a, b, c, nrm, deg, RB.gbary[3 * g], RB.gbary[3 * g + 1], RB.gbary[3 * g + 2],
                               RB.goff ? RB.goff[g] : 0.0f);
        put_gaussian(g, m, q, sc, deg, RB.mu, RB.quat, RB.scale, &hdr->status, &hdr->n_degenerate);
    }
}

// The rebind of the leaves' Gaussians (kBind, mesh_refit_bind): after the
// rounds each leaf thread computes its face's normal, rotation and scale once
// (they depend on the face alone) into shared memory beside its corners, and
// the block's threads then take its Gaussians one per thread (offsets from a
// block scan of the faces' Gaussian counts), each computing only its centre.
template <bool kBind>
__global__ void __launch_bounds__(kRefitBlock, kBind ? 3 : 4)
k_refit_local(int n, const float *__restrict__ V3, int nV, float4 *__restrict__ V4,
              const int *__restrict__ perm, const int4 *__restrict__ faces,
              float4 *__restrict__ tris, float4 *__restrict__ nodes, const int *__restrict__ parent,
              const int *__restrict__ rend, float4 *__restrict__ pre, float4 *__restrict__ suf,
              float4 *__restrict__ bbox, int4 *__restrict__ xlist, int *__restrict__ xcnt,
              int *__restrict__ iperm, Header *__restrict__ hdr, Rebind RB, int leaf_size) {
    extern __shared__ float4 dsm[];
    pdl_wait();
    pdl_trigger();
    float *tab = reinterpret_cast<float *>(dsm);
    int *s_warp = reinterpret_cast<int *>(tab + (kBind ? kBindFloats : 12) * kRefitBlock);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int base = blockIdx.x * kRefitBlock, j = base + tid;
    // leaf j: box into level 0 and into its parent's record
    {
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
        float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
        if (j < n) {
            int pe_leaf = parent[(n - 1) + j];
            float4 a, b, c;
            load_tri(V3, V4, faces[perm[j]], a, b, c);
            lo = box_min(box_min(a, b), c);
            hi = box_max(box_max(a, b), c);
            put_box(nodes, hdr, pe_leaf, -(j + 1), 1, lo, hi);
        }
        SBox{tab}.put(tid, lo, hi);
    }
    // internal node j: its leaf range [ra, rb]
    int ra = 0, rb = 0, pe_node = -1;
    bool cross = false;
    if (j < n - 1) {
        int far = rend[j];
        ra = min(j, far);
        rb = max(j, far);
        cross = crosses_block(ra, rb);
        pe_node = parent[j];
    }
    // this block's crossing nodes, listed in index order
    unsigned int ball = __ballot_sync(0xffffffffu, cross);
    if (lane == 0) s_warp[wid] = __popc(ball);
    __syncthreads();
    if (wid == 0) {
        int c = lane < kRefitBlock / 32 ? s_warp[lane] : 0, x = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        s_warp[32 + lane] = x - c;
        if (lane == 31) xcnt[blockIdx.x] = x;
    }
    // Range queries, level by level: the union over [i0, i0 + L) with
    // 2^k <= L < 2^(k+1) is level k at i0 and at i0 + L - 2^k.  Asked here:
    // the owned node j (its range), and leaf j's prefix [0, tid] and suffix
    // [tid, kRefitBlock) inside the block (the block's box is the suffix of 0).
    const int node_level = (j < n - 1 && !cross) ? 31 - __clz(rb - ra + 1) : -1;
    const int pre_level = 31 - __clz(tid + 1), suf_level = 31 - __clz(kRefitBlock - tid);
    for (int k = 0; k <= kRefitLevels; ++k) {
        const SBox cur{tab + (k & 1) * 6 * kRefitBlock}, nxt{tab + ((k + 1) & 1) * 6 * kRefitBlock};
        const int h = 1 << k;
        if (node_level == k) {
            int i0 = ra - base, i1 = rb - base - h + 1;
            int link, cnt;
            node_link(j, ra, rb, leaf_size, link, cnt);
            put_box(nodes, hdr, pe_node, link, cnt, box_min(cur.lo(i0), cur.lo(i1)), box_max(cur.hi(i0), cur.hi(i1)));
        }
        if (pre_level == k && j < n) {
            int i1 = tid - h + 1;
            pre[2 * (size_t)j] = box_min(cur.lo(0), cur.lo(i1));
            pre[2 * (size_t)j + 1] = box_max(cur.hi(0), cur.hi(i1));
        }
        if (suf_level == k) {
            int i1 = kRefitBlock - h;
            float4 lo = box_min(cur.lo(tid), cur.lo(i1)), hi = box_max(cur.hi(tid), cur.hi(i1));
            if (j < n) {
                suf[2 * (size_t)j] = lo;
                suf[2 * (size_t)j + 1] = hi;
            }
            if (tid == 0) {
                bbox[2 * blockIdx.x] = lo;
                bbox[2 * blockIdx.x + 1] = hi;
            }
        }
        if (k == 1 && cross)                             // offsets written by warp 0 in round 0
            xlist[base + s_warp[32 + wid] + __popc(ball & ((1u << lane) - 1u))] = make_int4(j, ra, rb, pe_node);
        if (k < kRefitLevels) {
            if (tid + 2 * h <= kRefitBlock)
                nxt.put(tid, box_min(cur.lo(tid), cur.lo(tid + h)), box_max(cur.hi(tid), cur.hi(tid + h)));
            __syncthreads();
        }
    }
    int gs = 0, gcnt = 0;                                // kBind: this leaf's Gaussians
    if constexpr (kBind) __syncthreads();                // the table is read no more: records go there
    if (j < n) {
        int f = perm[j];                                 // reloaded: cheaper than keeping it live
        iperm[f] = j;
        float4 a, b, c;
        load_tri(V3, V4, faces[f], a, b, c);
        float deg = exactly_degenerate(a, b, c) ? 1.0f : 0.0f;
        tris[3 * (size_t)j + 0] = make_float4(a.x, a.y, a.z, __int_as_float(f));
        tris[3 * (size_t)j + 1] = make_float4(b.x, b.y, b.z, deg);
        tris[3 * (size_t)j + 2] = make_float4(c.x, c.y, c.z, 0.0f);
        if constexpr (kBind) {
            int g0 = RB.gstart[f], g1 = RB.gstart[f + 1];
            if (g0 < 0 || g1 < g0 || (int64_t)g1 > RB.nG) set_status(hdr, MESH_DEV_INDEX_RANGE);
            else { gs = g0; gcnt = g1 - g0; }
            FaceBind B = face_bind(v3(a), v3(b), v3(c));
            const float r[kBindFloats] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, B.n.x, B.n.y, B.n.z,
                                          B.q[0], B.q[1], B.q[2], B.q[3], B.s[0], B.s[1], B.s[2],
                                          B.degenerate ? 1.0f : 0.0f};
#pragma unroll
            for (int k = 0; k < kBindFloats; ++k) tab[k * kRefitBlock + tid] = r[k];
        }
    }
    if constexpr (kBind) bind_block(tab, s_warp, gs, gcnt, RB, hdr);
    // a1: this block's slice of the vertex repack (after every read of V4 above)
    if (V3) {
        int per = (nV + gridDim.x - 1) / gridDim.x;
        int v1 = min(nV, (int)(blockIdx.x + 1) * per);
        for (int v = blockIdx.x * per + tid; v < v1; v += kRefitBlock) {
            const float *p = V3 + 3 * (size_t)v;
            V4[v] = make_float4(p[0], p[1], p[2], 0.0f);
        }
    }
}

// One warp per crossing node: the suffix union in its first block, the prefix
// union in its last, and the boxes of the blocks between.
constexpr int kTopThreads = 256;

__global__ void __launch_bounds__(kTopThreads)
k_refit_top(const int4 *__restrict__ xlist, const int *__restrict__ xcnt, const float4 *__restrict__ pre,
            const float4 *__restrict__ suf, const float4 *__restrict__ bbox, float4 *__restrict__ nodes,
            Header *__restrict__ hdr, int leaf_size) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kTopThreads >> 5;
    const int cnt = xcnt[blockIdx.x];
    for (int r = wid; r < cnt; r += nw) {
        int4 e = xlist[(size_t)blockIdx.x * kRefitBlock + r];   // node, range start, range end, parent
        float4 lo = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
        float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.0f);
        if (lane == 0) {
            lo = box_min(__ldcg(suf + 2 * (size_t)e.y), __ldcg(pre + 2 * (size_t)e.z));
            hi = box_max(__ldcg(suf + 2 * (size_t)e.y + 1), __ldcg(pre + 2 * (size_t)e.z + 1));
        }
        for (int b = e.y / kRefitBlock + 1 + lane; b < e.z / kRefitBlock; b += 32) {
            lo = box_min(lo, __ldcg(bbox + 2 * b));
            hi = box_max(hi, __ldcg(bbox + 2 * b + 1));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
            lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
            hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
        }
        if (lane == 0) {
            int link, cnt;
            node_link(e.x, e.y, e.z, leaf_size, link, cnt);
            put_box(nodes, hdr, e.w, link, cnt, lo, hi);
        }
    }
}

// ---------------------------------------------------------------------------
// Batched build: the same steps over many scenes at once.  Faces carry scene-
// local vertex indices; offsets give each scene's vertex and face range.
// ---------------------------------------------------------------------------
__global__ void k_batch_init(unsigned int *__restrict__ cbox, int nscenes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * nscenes) cbox[i] = (i % 6 < 3) ? 0xffffffffu : 0u;
}

__global__ void k_batch_faces(const int *__restrict__ F3, int nF, const int *__restrict__ vert_off,
                              const int *__restrict__ face_off, int nscenes,
                              const float4 *__restrict__ V4, int4 *__restrict__ F4,
                              float4 *__restrict__ cent, unsigned int *__restrict__ cbox,
                              unsigned int *__restrict__ status) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = f < nF;
    int sc = valid ? segment_of(face_off, nscenes, f) : -1;
    float s3[3] = {0.f, 0.f, 0.f};
    if (valid) {
        int vb = __ldg(vert_off + sc), nv = __ldg(vert_off + sc + 1) - vb;
        const int *p = F3 + 3 * (size_t)f;
        int i0 = p[0], i1 = p[1], i2 = p[2];
        if ((unsigned)i0 >= (unsigned)nv || (unsigned)i1 >= (unsigned)nv || (unsigned)i2 >= (unsigned)nv) {
            atomicOr(status, (unsigned)MESH_DEV_INDEX_RANGE);
            if ((unsigned)i0 >= (unsigned)nv) i0 = 0;
            if ((unsigned)i1 >= (unsigned)nv) i1 = 0;
            if ((unsigned)i2 >= (unsigned)nv) i2 = 0;
        }
        i0 += vb; i1 += vb; i2 += vb;
        F4[f] = make_int4(i0, i1, i2, sc);
        float4 a = V4[i0], b = V4[i1], c = V4[i2];
        s3[0] = __fadd_rn(__fadd_rn(a.x, b.x), c.x);
        s3[1] = __fadd_rn(__fadd_rn(a.y, b.y), c.y);
        s3[2] = __fadd_rn(__fadd_rn(a.z, b.z), c.z);
        cent[f] = make_float4(s3[0], s3[1], s3[2], 0.0f);
    }
    // one atomic per scene present in the warp
    unsigned int peers = __match_any_sync(0xffffffffu, sc);
    for (int k = 0; k < 3; ++k) {
        unsigned int lo = __reduce_min_sync(peers, valid ? f2ord(s3[k]) : 0xffffffffu);
        unsigned int hi = __reduce_max_sync(peers, valid ? f2ord(s3[k]) : 0u);
        if (valid && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0u) {
            atomicMin(&cbox[6 * sc + k], lo);
            atomicMax(&cbox[6 * sc + 3 + k], hi);
        }
    }
}

__global__ void k_batch_morton(const float4 *__restrict__ cent, int nF, const int4 *__restrict__ F4,
                               const unsigned int *__restrict__ cbox,
                               unsigned int *__restrict__ key_of_face,
                               unsigned int *__restrict__ keys, int *__restrict__ vals) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    const unsigned int *bx = cbox + 6 * F4[f].w;
    float4 s = cent[f];
    float sv[3] = {s.x, s.y, s.z};
    unsigned int q[3];
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bx[k]);
        float ext = __fsub_rn(ord2f(bx[3 + k]), lo);
        float inv = ext > 0.0f ? __fdiv_rn(1.0f, ext) : 0.0f;
        float t = __fmul_rn(__fsub_rn(sv[k], lo), inv);
        int qi = (int)floorf(__fmul_rn(t, 1024.0f));
        qi = qi < 0 ? 0 : (qi > 1023 ? 1023 : qi);
        q[k] = (unsigned int)qi;
    }
    unsigned int key = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    key_of_face[f] = key;
    keys[f] = key;
    vals[f] = f;
}

// Scene id of each (Morton-sorted) face, as the key of the last, stable pass.
__global__ void k_batch_scene_keys(const int *__restrict__ vals, int n, const int4 *__restrict__ F4,
                                   unsigned int *__restrict__ keys) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) keys[j] = (unsigned int)F4[vals[j]].w;
}

__global__ void k_batch_gather_keys(const int *__restrict__ perm, int n,
                                    const unsigned int *__restrict__ key_of_face,
                                    unsigned int *__restrict__ keys) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) keys[j] = key_of_face[perm[j]];
}

__global__ void k_batch_karras(const unsigned int *__restrict__ keys, int nF,
                               const int *__restrict__ face_off, int nscenes,
                               float4 *__restrict__ nodes, int *__restrict__ parent_int,
                               int *__restrict__ parent_leaf) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nF) return;
    int sc = segment_of(face_off, nscenes, j);
    int base = __ldg(face_off + sc), n = __ldg(face_off + sc + 1) - base, i = j - base;
    if (n == 1) { parent_leaf[base] = -1; return; }
    if (i >= n - 1) return;
    int left, right, far_end;
    karras_children(keys + base, n, i, left, right, far_end);
    write_children(nodes + 4 * (size_t)base, i, left, right);
    if (left >= 0) parent_int[base + left] = 2 * i; else parent_leaf[base - left - 1] = 2 * i;
    if (right >= 0) parent_int[base + right] = 2 * i + 1; else parent_leaf[base - right - 1] = 2 * i + 1;
    if (i == 0) parent_int[base] = -1;
}

// Bottom-up boxes of every scene (build and refit).  One thread per leaf j
// writes the packed triangle of face perm[j] and climbs: at each internal node
// the first arriving child stops, the second computes the union (the
// sibling's box read from L2 after a fence) and continues, clearing the
// arrival counter for the next pass.  Each scene's root box goes to its slot.
__global__ void k_batch_leaves_up(int nF, const int *__restrict__ face_off, int nscenes,
                                  const int *__restrict__ perm, const int4 *__restrict__ faces,
                                  const float4 *__restrict__ verts, float4 *__restrict__ tris,
                                  float4 *__restrict__ nodes, const int *__restrict__ parent_int,
                                  const int *__restrict__ parent_leaf,
                                  unsigned int *__restrict__ flags, float4 *__restrict__ scene_box) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nF) return;
    int sc = segment_of(face_off, nscenes, j);
    int base = __ldg(face_off + sc);
    int f = perm[j];
    int4 fv = faces[f];
    float4 a = verts[fv.x], b = verts[fv.y], c = verts[fv.z];
    float deg = exactly_degenerate(a, b, c) ? 1.0f : 0.0f;
    tris[3 * (size_t)j + 0] = make_float4(a.x, a.y, a.z, __int_as_float(f));
    tris[3 * (size_t)j + 1] = make_float4(b.x, b.y, b.z, deg);
    tris[3 * (size_t)j + 2] = make_float4(c.x, c.y, c.z, 0.0f);
    float3 lo = make_float3(fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y),
                            fminf(fminf(a.z, b.z), c.z));
    float3 hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y),
                            fmaxf(fmaxf(a.z, b.z), c.z));
    float4 *snodes = nodes + 4 * (size_t)base;
    int self = -(j - base + 1);
    int pe = parent_leaf[j];
    while (pe >= 0) {
        int p = pe >> 1, side = pe & 1;
        float4 *rec = snodes + 4 * (size_t)p;
        rec[2 * side] = make_float4(lo.x, lo.y, lo.z, __int_as_float(self));
        rec[2 * side + 1] = make_float4(hi.x, hi.y, hi.z, __int_as_float(self < 0 ? 1 : self));
        __threadfence();
        unsigned int old = atomicAdd(&flags[base + p], 1u);
        if (old == 0u) return;
        __threadfence();
        int o = 1 - side;
        float4 olo = __ldcg(rec + 2 * o), ohi = __ldcg(rec + 2 * o + 1);
        lo = make_float3(fminf(lo.x, olo.x), fminf(lo.y, olo.y), fminf(lo.z, olo.z));
        hi = make_float3(fmaxf(hi.x, ohi.x), fmaxf(hi.y, ohi.y), fmaxf(hi.z, ohi.z));
        flags[base + p] = 0u;
        self = p;
        pe = parent_int[base + p];
    }
    scene_box[2 * sc] = make_float4(lo.x, lo.y, lo.z, 0.0f);
    scene_box[2 * sc + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
}

// ---------------------------------------------------------------------------
// Build workspace layout.
// ---------------------------------------------------------------------------
struct BuildWs {
    unsigned int *keysA, *keysB, *hist, *cbox, *dsum, *dbase, *ticket;
    int *valsA, *valsB;
    float4 *cent;
    int tiles;
    size_t bytes;
};

static BuildWs build_ws_layout(char *base, int64_t nF) {
    BuildWs w{};
    int64_t n = nF > 0 ? nF : 1;
    w.tiles = (int)((n + kSortTile - 1) / kSortTile);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return base + o; };
    w.keysA = (unsigned int *)take(4 * n);
    w.keysB = (unsigned int *)take(4 * n);
    w.valsA = (int *)take(4 * n);
    w.valsB = (int *)take(4 * n);
    w.cent = (float4 *)take(16 * n);
    w.hist = (unsigned int *)take((size_t)4 * kRadix * w.tiles);
    w.cbox = (unsigned int *)take(32);
    w.dsum = (unsigned int *)take(4 * kRadix);
    w.dbase = (unsigned int *)take(4 * kRadix);
    w.ticket = (unsigned int *)take(4);
    w.bytes = off;
    return w;
}

// Four 8-bit passes over (w.keysA, w.valsA): A -> B -> A -> B -> (out_keys,
// out_vals).  out_keys may be w.keysA (the last pass reads B).
static void radix_sort_pairs(const BuildWs &w, int n, unsigned int *out_keys, int *out_vals,
                             cudaStream_t s) {
    unsigned int *kin = w.keysA, *kout = w.keysB;
    int *vin = w.valsA, *vout = w.valsB;
    for (int pass = 0; pass < 4; ++pass) {
        if (pass == 3) { kout = out_keys; vout = out_vals; }
        int shift = 8 * pass;
        k_sort_upsweep<<<w.tiles, kSortThreads, 0, s>>>(kin, n, shift, w.hist, w.tiles, w.ticket);
        k_sort_scan<<<kRadix, kScanThreads, 0, s>>>(w.hist, w.tiles, w.dsum, w.dbase, w.ticket);
        k_sort_downsweep<<<w.tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, w.hist,
                                                          w.tiles, w.dbase);
        count_launch(3);
        unsigned int *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
}

// One pass for the other kernels of the library, its three kernels launched as
// programmatic dependents (the contact and Chamfer steps' orders run on a
// frame's critical path, where the launch latency counts).  The build's passes
// above use plain launches: there the early-launched grids measured slower.
static void radix_pass(const BuildWs &w, int n, int shift, const unsigned int *kin, const int *vin,
                       unsigned int *kout, int *vout, cudaStream_t s) {
    pdl_launch(k_sort_upsweep, w.tiles, kSortThreads, 0, s, kin, n, shift, w.hist, w.tiles, w.ticket);
    pdl_launch(k_sort_scan, kRadix, kScanThreads, 0, s, w.hist, w.tiles, w.dsum, w.dbase, w.ticket);
    pdl_launch(k_sort_downsweep, w.tiles, kSortThreads, 0, s, kin, vin, kout, vout, n, shift, w.hist, w.tiles,
               w.dbase);
    count_launch(3);
}

// Stable sort of (key, value) pairs on the low `bits` key bits (8 per pass),
// for other kernels of the library; ws holds sort_pairs_ws_bytes(n) bytes.
// vin NULL: the values are the indices 0 .. n-1 (the sorting permutation).
size_t sort_pairs_ws_bytes(int64_t n) { return build_ws_layout(nullptr, n).bytes + 256; }

void sort_pairs_u32(void *ws, int n, int bits, const unsigned int *kin, const int *vin, unsigned int *kout,
                    int *vout, cudaStream_t s) {
    BuildWs w = build_ws_layout((char *)ws, n);
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    unsigned int *kb[2] = {w.keysA, w.keysB};
    int *vb[2] = {w.valsA, w.valsB};
    for (int p = 0; p < passes; ++p) {
        const unsigned int *ki = p == 0 ? kin : kb[(p - 1) & 1];
        const int *vi = p == 0 ? vin : vb[(p - 1) & 1];
        unsigned int *ko = p == passes - 1 ? kout : kb[p & 1];
        int *vo = p == passes - 1 ? vout : vb[p & 1];
        radix_pass(w, n, 8 * p, ki, vi, ko, vo, s);
    }
}

struct BatchWs {
    BuildWs sort;
    unsigned int *key_of_face, *cbox;
    size_t bytes;
};

static BatchWs batch_ws_layout(char *base, int64_t nscenes, int64_t nF) {
    BatchWs w{};
    w.sort = build_ws_layout(base, nF);
    size_t off = w.sort.bytes;
    int64_t n = nF > 0 ? nF : 1;
    w.key_of_face = (unsigned int *)(base + off);
    off = align_up(off + 4 * n, 256);
    w.cbox = (unsigned int *)(base + off);
    off = align_up(off + 24 * (nscenes > 0 ? nscenes : 1), 256);
    w.bytes = off;
    return w;
}

static mesh_batch_layout batch_layout(int64_t maxB, int64_t maxV, int64_t maxF) {
    mesh_batch_layout L{};
    int64_t b = maxB > 0 ? maxB : 1, v = maxV > 0 ? maxV : 1, f = maxF > 0 ? maxF : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.max_scenes = maxB;
    L.max_verts = maxV;
    L.max_faces = maxF;
    L.off_scene = take(32 * b);
    L.off_status = take(sizeof(BatchStatus));
    L.off_vert_off = take(4 * (b + 1));
    L.off_face_off = take(4 * (b + 1));
    L.off_verts = take(16 * v);
    L.off_faces = take(16 * f);
    L.off_keys = take(4 * f);
    L.off_perm = take(4 * f);
    L.off_nodes = take(64 * f);
    L.off_parent_int = take(4 * f);
    L.off_parent_leaf = take(4 * f);
    L.off_tris = take(48 * f);
    L.off_flags = take(4 * f);
    L.storage_bytes = off;
    return L;
}

// Scratch of the bottom-up kernels: prefix and suffix unions of the leaf
// boxes inside each block (2 float4 per leaf each), the crossing nodes (int4
// per face), the blocks' boxes (2 float4 each) and the per-block counts.
static int64_t refit_blocks(int64_t f) { return (f + kRefitBlock - 1) / kRefitBlock; }
static size_t xlist_bytes(int64_t f) {
    int64_t nb = refit_blocks(f);
    return (size_t)(32 * f + 32 * f + 16 * f + 32 * nb + 4 * (nb + 1));
}

static mesh_bvh_layout storage_layout(int64_t maxV, int64_t maxF) {
    mesh_bvh_layout L{};
    int64_t v = maxV > 0 ? maxV : 1, f = maxF > 0 ? maxF : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.max_faces = maxF;
    L.max_verts = maxV;
    L.off_header = take(sizeof(Header));
    L.off_verts = take(16 * v);
    L.off_faces = take(16 * f);
    L.off_keys = take(4 * f);
    L.off_perm = take(4 * f);
    L.off_nodes = take(64 * (f > 1 ? f - 1 : 1));
    L.off_parent = take(4 * (2 * f - 1));
    L.off_tris = take(48 * f);
    L.off_rend = take(4 * f);
    L.off_iperm = take(4 * f);
    L.off_adj = take(12 * f);
    L.off_fnorm = take(16 * f);
    L.off_xlist = take(xlist_bytes(f));
    L.off_wide = take(128 * (f > 1 ? f - 1 : 1));
    L.storage_bytes = off;
    return L;
}

constexpr int64_t kMaxFaces = (int64_t)1 << 30;

// ---------------------------------------------------------------------------
// Agglomerative build for a mesh whose topology is fixed (built once from the
// template faces, then refit every frame): parallel locally-ordered
// clustering, PLOC (Meister & Bittner 2018), over the Morton-sorted leaves.
// One iteration: every cluster picks, among the clusters within kPlocRadius
// positions, the one whose union box has the least surface area (float32,
// (dx dy + dy dz) + dz dx, round-to-nearest without fused multiply-add; ties
// to the lower position); mutual pairs merge into a new node at the lower
// position (new nodes numbered in position order); the clusters are
// compacted in order.  The finished tree is laid out like the Karras tree:
// leaves in in-order, an internal node numbered by the end of its range not
// shared with its sibling (root 0; a left child by its last leaf, a right
// child by its first), which is a bijection for any binary tree over in-order
// leaves, so the bottom-up kernels and every traversal use it unchanged.
// ---------------------------------------------------------------------------
constexpr int kPlocRadius = 16;
constexpr int kPlocBlock = 256;

__device__ __forceinline__ float ploc_min(float a, float b) { return a < b ? a : b; }
__device__ __forceinline__ float ploc_max(float a, float b) { return a > b ? a : b; }

__device__ __forceinline__ float ploc_union_area(float4 la, float4 ha, float4 lb, float4 hb) {
    float dx = __fsub_rn(ploc_max(ha.x, hb.x), ploc_min(la.x, lb.x));
    float dy = __fsub_rn(ploc_max(ha.y, hb.y), ploc_min(la.y, lb.y));
    float dz = __fsub_rn(ploc_max(ha.z, hb.z), ploc_min(la.z, lb.z));
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}

// Leaf j of the Morton order: its face's box, cluster handle -(j+1).
__global__ void k_ploc_leaves(int n, const int *__restrict__ perm0, const int4 *__restrict__ faces,
                              const float4 *__restrict__ verts, int *__restrict__ cl,
                              float4 *__restrict__ cb) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int4 fv = faces[perm0[j]];
    float4 a = verts[fv.x], b = verts[fv.y], c = verts[fv.z];
    cb[2 * (size_t)j] = make_float4(ploc_min(ploc_min(a.x, b.x), c.x), ploc_min(ploc_min(a.y, b.y), c.y),
                                    ploc_min(ploc_min(a.z, b.z), c.z), 0.0f);
    cb[2 * (size_t)j + 1] = make_float4(ploc_max(ploc_max(a.x, b.x), c.x), ploc_max(ploc_max(a.y, b.y), c.y),
                                        ploc_max(ploc_max(a.z, b.z), c.z), 0.0f);
    cl[j] = -(j + 1);
}

// Nearest neighbour of every cluster within the radius; the block's clusters and
// the radius on either side are staged in shared memory.
__global__ void __launch_bounds__(kPlocBlock)
k_ploc_nn(int m, const float4 *__restrict__ cb, int *__restrict__ nn) {
    __shared__ float4 s_lo[kPlocBlock + 2 * kPlocRadius], s_hi[kPlocBlock + 2 * kPlocRadius];
    const int base = blockIdx.x * kPlocBlock;
    for (int t = threadIdx.x; t < kPlocBlock + 2 * kPlocRadius; t += kPlocBlock) {
        int g = base - kPlocRadius + t;
        if (g >= 0 && g < m) {
            s_lo[t] = cb[2 * (size_t)g];
            s_hi[t] = cb[2 * (size_t)g + 1];
        }
    }
    __syncthreads();
    const int i = base + threadIdx.x;
    if (i >= m) return;
    const int si = threadIdx.x + kPlocRadius;
    float4 lo = s_lo[si], hi = s_hi[si];
    float best = INFINITY;
    int bj = -1;
    for (int d = -kPlocRadius; d <= kPlocRadius; ++d) {
        int j = i + d;
        if (d == 0 || j < 0 || j >= m) continue;
        float a = ploc_union_area(lo, hi, s_lo[si + d], s_hi[si + d]);
        if (bj < 0 || a < best) { best = a; bj = j; }
    }
    nn[i] = bj;
}

// keep: the cluster survives the iteration (it is not the upper half of a pair);
// merge: it is the lower half of a mutual pair.
__global__ void k_ploc_flags(int m, const int *__restrict__ nn, int *__restrict__ keep,
                             int *__restrict__ merge) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    keep[i] = !(mutual && i > j);
    merge[i] = mutual && i < j;
}

// An iteration without a mutual pair (possible only for non-finite boxes) merges
// positions 0 and 1, as the oracle does.
__global__ void k_ploc_force(int *nn) {
    nn[0] = 1;
    nn[1] = 0;
}

__global__ void k_ploc_compact(int m, const int *__restrict__ cl_in, const float4 *__restrict__ cb_in,
                               const int *__restrict__ nn, const int *__restrict__ keep,
                               const int *__restrict__ kpos, const int *__restrict__ merge,
                               const int *__restrict__ mpos, int node_base, int *__restrict__ cl_out,
                               float4 *__restrict__ cb_out, int *__restrict__ cl_l, int *__restrict__ cl_r,
                               int *__restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !keep[i]) return;
    int dst = kpos[i];
    float4 lo = cb_in[2 * (size_t)i], hi = cb_in[2 * (size_t)i + 1];
    if (merge[i]) {
        int j = nn[i], c = node_base + mpos[i];
        int a = cl_in[i], b = cl_in[j];
        cl_l[c] = a;
        cl_r[c] = b;
        cnt[c] = (a < 0 ? 1 : cnt[a]) + (b < 0 ? 1 : cnt[b]);
        float4 lb = cb_in[2 * (size_t)j], hb = cb_in[2 * (size_t)j + 1];
        lo = make_float4(ploc_min(lo.x, lb.x), ploc_min(lo.y, lb.y), ploc_min(lo.z, lb.z), 0.0f);
        hi = make_float4(ploc_max(hi.x, hb.x), ploc_max(hi.y, hb.y), ploc_max(hi.z, hb.z), 0.0f);
        cl_out[dst] = c;
    } else {
        cl_out[dst] = cl_in[i];
    }
    cb_out[2 * (size_t)dst] = lo;
    cb_out[2 * (size_t)dst + 1] = hi;
}

__global__ void k_ploc_root(int root, int *pos, int *kid, int *parent) {
    pos[root] = 0;
    kid[root] = 0;
    parent[0] = -1;
}

// Top-down layout of the nodes made in one iteration (their parents, made
// later, are already placed): leaf positions, Karras numbers, parent links,
// far ends, and the leaf-order face ids and keys.
__global__ void k_ploc_place(int base, int count, int n, const int *__restrict__ cl_l,
                             const int *__restrict__ cl_r, const int *__restrict__ cnt, int *pos, int *kid,
                             const int *__restrict__ perm0, const unsigned int *__restrict__ sk,
                             int *__restrict__ perm, unsigned int *__restrict__ keys,
                             int *__restrict__ parent, int *__restrict__ rend) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    int c = base + t;
    int p = pos[c], k = kid[c];
    rend[k] = k == p ? p + cnt[c] - 1 : p;
    int a = cl_l[c], b = cl_r[c];
    int ca = a < 0 ? 1 : cnt[a];
    if (a < 0) {
        int j = -a - 1;
        perm[p] = perm0[j];
        keys[p] = sk[j];
        parent[(n - 1) + p] = 2 * k;
    } else {
        pos[a] = p;
        kid[a] = p + ca - 1;
        parent[p + ca - 1] = 2 * k;
    }
    int rp = p + ca;
    if (b < 0) {
        int j = -b - 1;
        perm[rp] = perm0[j];
        keys[rp] = sk[j];
        parent[(n - 1) + rp] = 2 * k + 1;
    } else {
        pos[b] = rp;
        kid[b] = rp;
        parent[rp] = 2 * k + 1;
    }
}

struct PlocWs {
    BuildWs sort;
    unsigned int *sk;
    int *perm0, *clA, *clB, *nn, *keep, *kpos, *merge, *mpos, *bsumA, *bsumB, *tot, *cl_l, *cl_r, *cnt,
        *pos, *kid;
    float4 *cbA, *cbB;
    size_t bytes;
};

// Depth check of a finished tree: leaf j climbs its parent links (2 p + side,
// -1 at the root) and flags the tree when it passes more than `limit`
// internal nodes.  The climb stops there, so a degenerate chain costs at most
// limit + 1 steps per leaf.
__global__ void k_depth_check(int n, const int *__restrict__ parent, int limit, int *__restrict__ flag) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int pe = parent[(n - 1) + j], d = 0;
    while (pe >= 0 && d <= limit) {
        ++d;
        pe = parent[pe >> 1];
    }
    if (d > limit) atomicOr(flag, 1);
}

__global__ void k_set_status(Header *hdr, unsigned int bits) { set_status(hdr, bits); }

static PlocWs ploc_ws_layout(char *base, int64_t nF) {
    PlocWs w{};
    w.sort = build_ws_layout(base, nF);
    int64_t n = nF > 0 ? nF : 1;
    size_t off = align_up(w.sort.bytes, 256);
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return base + o; };
    w.sk = (unsigned int *)take(4 * n);
    w.perm0 = (int *)take(4 * n);
    w.clA = (int *)take(4 * n);
    w.clB = (int *)take(4 * n);
    w.nn = (int *)take(4 * n);
    w.keep = (int *)take(4 * n);
    w.kpos = (int *)take(4 * n);
    w.merge = (int *)take(4 * n);
    w.mpos = (int *)take(4 * n);
    w.bsumA = (int *)take(4 * ((n + 1023) / 1024) + 4);
    w.bsumB = (int *)take(4 * ((n + 1023) / 1024) + 4);
    w.tot = (int *)take(16);
    w.cl_l = (int *)take(4 * n);
    w.cl_r = (int *)take(4 * n);
    w.cnt = (int *)take(4 * n);
    w.pos = (int *)take(4 * n);
    w.kid = (int *)take(4 * n);
    w.cbA = (float4 *)take(32 * n);
    w.cbB = (float4 *)take(32 * n);
    w.bytes = off;
    return w;
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

size_t mesh_bvh_storage_bytes(int64_t max_verts, int64_t max_faces) {
    if (max_verts < 0 || max_faces < 0 || max_faces > kMaxFaces || max_verts > kMaxFaces) return 0;
    return storage_layout(max_verts, max_faces).storage_bytes;
}

size_t mesh_build_workspace_bytes(int64_t max_faces) {
    if (max_faces < 0 || max_faces > kMaxFaces) return 0;
    return build_ws_layout(nullptr, max_faces).bytes;
}

mesh_status mesh_bvh_create(void *d_storage, size_t storage_bytes, int64_t max_verts,
                            int64_t max_faces, mesh_bvh **out) {
    if (!out || !d_storage || max_verts < 0 || max_faces < 0 || max_faces > kMaxFaces ||
        max_verts > kMaxFaces)
        return MESH_ERR_INVALID_ARG;
    if (((uintptr_t)d_storage & 255u) != 0) return MESH_ERR_INVALID_ARG;
    mesh_bvh_layout L = storage_layout(max_verts, max_faces);
    if (storage_bytes < L.storage_bytes) return MESH_ERR_WORKSPACE;
    mesh_bvh *h = (mesh_bvh *)std::calloc(1, sizeof(mesh_bvh));
    if (!h) return MESH_ERR_INVALID_ARG;
    h->base = (char *)d_storage;
    h->L = L;
    h->L.n_faces = 0;
    h->L.n_verts = 0;
    h->cfg_lanes = -1;
    h->cfg_variant = -1;
    h->cfg_block = 128;
    h->leaf_size = 1;
    h->wide_valid = false;
    h->adj_ready = false;
    *out = h;
    return MESH_OK;
}

void mesh_bvh_destroy(mesh_bvh *bvh) { std::free(bvh); }

mesh_status mesh_bvh_set_leaf_size(mesh_bvh *bvh, int leaf_size) {
    if (!bvh || leaf_size < 1 || leaf_size > kMaxLeafSize) return MESH_ERR_INVALID_ARG;
    bvh->leaf_size = leaf_size;
    return MESH_OK;
}

mesh_status mesh_bvh_get_layout(const mesh_bvh *bvh, mesh_bvh_layout *out) {
    if (!bvh || !out) return MESH_ERR_INVALID_ARG;
    *out = bvh->L;
    return MESH_OK;
}

mesh_status mesh_update_vertices(mesh_bvh *bvh, const float *d_V, int64_t nV, void *stream) {
    if (!bvh || nV < 0 || nV > bvh->L.max_verts || (nV > 0 && !d_V)) return MESH_ERR_INVALID_ARG;
    if (bvh->L.n_faces > 0 && nV != bvh->L.n_verts) return MESH_ERR_INVALID_ARG;
    bvh->L.n_verts = nV;
    if (nV == 0) return MESH_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_copy_verts<<<grid_for(nV, kBlock), kBlock, 0, s>>>(d_V, (int)nV, bvh->verts(), nullptr);
    count_launch();
    return check_launch();
}

// Launches the two bottom-up kernels (build and refit); V3 = new vertices or NULL.
static mesh_status bottom_up(mesh_bvh *bvh, const float *V3, cudaStream_t s,
                             Rebind rb = Rebind{nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr}) {
    static bool smem_set = false;                    // the dynamic shared memory the kernels take
    if (!smem_set) {
        if (cudaFuncSetAttribute(k_refit_local<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRefitLocalSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_refit_local<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRefitBindSmem) != cudaSuccess)
            return MESH_ERR_CUDA;
        smem_set = true;
    }
    int n = (int)bvh->L.n_faces;
    bvh->wide_valid = false;
    unsigned int nb = grid_for(n, kRefitBlock);
    int64_t fmax = bvh->L.max_faces, nbmax = refit_blocks(fmax);
    float4 *pre = reinterpret_cast<float4 *>(bvh->xlist()), *suf = pre + 2 * fmax;
    int4 *xlist = reinterpret_cast<int4 *>(suf + 2 * fmax);
    float4 *bbox = reinterpret_cast<float4 *>(xlist + fmax);
    int *xcnt = reinterpret_cast<int *>(bbox + 2 * nbmax);
    (rb.gstart ? k_refit_local<true> : k_refit_local<false>)<<<nb, kRefitBlock,
        rb.gstart ? kRefitBindSmem : kRefitLocalSmem, s>>>(
        n, V3, (int)bvh->L.n_verts, bvh->verts(), bvh->perm(), bvh->faces(), bvh->tris(),
        bvh->nodes(), bvh->parent(), bvh->rend(), pre, suf, bbox, xlist, xcnt, bvh->iperm(), bvh->hdr(), rb,
        bvh->leaf_size);
    count_launch();
    if (nb > 1) {
        pdl_launch(k_refit_top, nb, kTopThreads, 0, s, xlist, xcnt, pre, suf, bbox, bvh->nodes(), bvh->hdr(),
                   bvh->leaf_size);
        count_launch();
    }
    if (wide_wanted(bvh)) wide_refresh(bvh, s, true);     // the 4-wide records of variant 13
    return check_launch();
}

mesh_status mesh_refit_bind(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_gstart,
                            const float *d_gbary, const float *d_goff, int64_t nG, float *d_mu,
                            float *d_quat, float *d_scale, void *stream) {
    if (!bvh || nG < 0 || nG > INT_MAX) return MESH_ERR_INVALID_ARG;
    int n = (int)bvh->L.n_faces;
    if (n == 0) return mesh_refit(bvh, d_V, nV, stream);
    if (!d_gstart || (nG > 0 && (!d_gbary || !d_mu || !d_quat || !d_scale))) return MESH_ERR_INVALID_ARG;
    if (d_V && (nV != bvh->L.n_verts || nV > bvh->L.max_verts)) return MESH_ERR_INVALID_ARG;
    return bottom_up(bvh, d_V, (cudaStream_t)stream,
                     Rebind{d_gstart, d_gbary, d_goff, nG, d_mu, d_quat, d_scale});
}

mesh_status mesh_refit(mesh_bvh *bvh, const float *d_V, int64_t nV, void *stream) {
    if (!bvh) return MESH_ERR_INVALID_ARG;
    int n = (int)bvh->L.n_faces;
    if (d_V && n == 0) return mesh_update_vertices(bvh, d_V, nV, stream);
    if (d_V && (nV != bvh->L.n_verts || nV > bvh->L.max_verts)) return MESH_ERR_INVALID_ARG;
    if (n == 0) return MESH_OK;
    return bottom_up(bvh, d_V, (cudaStream_t)stream);
}

// The part both builds share: vertex and face tables, face centroids and
// their Morton keys (in w.keysA / w.valsA, ready for the sort).
static void build_keys(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_F, int64_t nF,
                       const BuildWs &w, cudaStream_t s) {
    bvh->L.n_verts = nV;
    bvh->L.n_faces = nF;
    bvh->adj_ready = false;
    bvh->wide_valid = false;
    int n = (int)nF;
    cudaMemsetAsync(bvh->hdr(), 0, sizeof(Header), s);
    if (nV > 0) {
        k_copy_verts<<<grid_for(nV > 6 ? nV : 6, kBlock), kBlock, 0, s>>>(
            d_V, (int)nV, bvh->verts(), n > 0 ? w.cbox : nullptr);
        count_launch();
    }
    if (n == 0) return;
    k_faces_centroids<<<grid_for(n, kBlock), kBlock, 0, s>>>(d_F, n, (int)nV, bvh->verts(),
                                                             bvh->faces(), w.cent, w.cbox, bvh->hdr());
    k_morton<<<grid_for(n, kBlock), kBlock, 0, s>>>(w.cent, n, w.cbox, w.keysA, w.valsA);
    count_launch(2);
}

mesh_status mesh_build_lbvh(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_F,
                            int64_t nF, void *d_ws, size_t ws_bytes, void *stream) {
    if (!bvh || nV < 0 || nF < 0 || nV > bvh->L.max_verts || nF > bvh->L.max_faces)
        return MESH_ERR_INVALID_ARG;
    if ((nV > 0 && !d_V) || (nF > 0 && (!d_F || nV == 0))) return MESH_ERR_INVALID_ARG;
    BuildWs w = build_ws_layout((char *)d_ws, nF);
    if (nF > 0 && (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u))) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int n = (int)nF;
    build_keys(bvh, d_V, nV, d_F, nF, w, s);
    if (n == 0) return check_launch();
    radix_sort_pairs(w, n, bvh->keys(), bvh->perm(), s);
    if (n > 1) {
        k_karras<<<grid_for(n - 1, kBlock), kBlock, 0, s>>>(bvh->keys(), n, bvh->nodes(),
                                                           bvh->parent(), bvh->rend());
        count_launch();
    } else {
        cudaMemsetAsync(bvh->parent(), 0xff, sizeof(int), s);   // lone leaf: no parent
    }
    return bottom_up(bvh, nullptr, s);
}

size_t mesh_build_ploc_workspace_bytes(int64_t max_faces) {
    if (max_faces < 0 || max_faces > kMaxFaces) return 0;
    return ploc_ws_layout(nullptr, max_faces).bytes;
}

mesh_status mesh_build_ploc(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_F,
                            int64_t nF, void *d_ws, size_t ws_bytes, void *stream) {
    if (!bvh || nV < 0 || nF < 0 || nV > bvh->L.max_verts || nF > bvh->L.max_faces)
        return MESH_ERR_INVALID_ARG;
    if ((nV > 0 && !d_V) || (nF > 0 && (!d_F || nV == 0))) return MESH_ERR_INVALID_ARG;
    PlocWs w = ploc_ws_layout((char *)d_ws, nF);
    if (nF > 0 && (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u))) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int n = (int)nF;
    build_keys(bvh, d_V, nV, d_F, nF, w.sort, s);
    if (n == 0) return check_launch();
    if (n == 1) {                                     // a lone leaf, as mesh_build_lbvh leaves it
        radix_sort_pairs(w.sort, n, bvh->keys(), bvh->perm(), s);
        cudaMemsetAsync(bvh->parent(), 0xff, sizeof(int), s);
        return bottom_up(bvh, nullptr, s);
    }
    radix_sort_pairs(w.sort, n, w.sk, w.perm0, s);
    k_ploc_leaves<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, w.perm0, bvh->faces(), bvh->verts(), w.clA, w.cbA);
    count_launch();
    std::vector<int2> batches;                        // (first node, count) made per iteration
    int m = n, made = 0;
    int *cl_in = w.clA, *cl_out = w.clB;
    float4 *cb_in = w.cbA, *cb_out = w.cbB;
    auto flags_and_counts = [&](int tot[2]) -> mesh_status {
        k_ploc_flags<<<grid_for(m, kBlock), kBlock, 0, s>>>(m, w.nn, w.keep, w.merge);
        count_launch();
        exclusive_scan_int(w.keep, w.kpos, m, w.bsumA, w.tot, s);
        exclusive_scan_int(w.merge, w.mpos, m, w.bsumB, w.tot + 1, s);
        if (cudaMemcpyAsync(tot, w.tot, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MESH_ERR_CUDA;
        return MESH_OK;
    };
    while (m > 1) {
        k_ploc_nn<<<(m + kPlocBlock - 1) / kPlocBlock, kPlocBlock, 0, s>>>(m, cb_in, w.nn);
        count_launch();
        int tot[2] = {0, 0};                          // clusters kept, nodes made
        mesh_status st = flags_and_counts(tot);
        if (st != MESH_OK) return st;
        if (tot[1] == 0) {
            k_ploc_force<<<1, 1, 0, s>>>(w.nn);
            count_launch();
            if ((st = flags_and_counts(tot)) != MESH_OK) return st;
        }
        // every node made removes one cluster; anything else means the device
        // state is not what the iteration wrote, so stop before using it
        if (tot[1] < 1 || tot[0] != m - tot[1] || made + tot[1] > n - 1) return MESH_ERR_CUDA;
        k_ploc_compact<<<grid_for(m, kBlock), kBlock, 0, s>>>(m, cl_in, cb_in, w.nn, w.keep, w.kpos, w.merge,
                                                            w.mpos, made, cl_out, cb_out, w.cl_l, w.cl_r,
                                                            w.cnt);
        count_launch();
        batches.push_back(make_int2(made, tot[1]));
        made += tot[1];
        m = tot[0];
        std::swap(cl_in, cl_out);
        std::swap(cb_in, cb_out);
    }
    k_ploc_root<<<1, 1, 0, s>>>(made - 1, w.pos, w.kid, bvh->parent());
    count_launch();
    for (auto it = batches.rbegin(); it != batches.rend(); ++it) {
        k_ploc_place<<<grid_for(it->y, kBlock), kBlock, 0, s>>>(it->x, it->y, n, w.cl_l, w.cl_r, w.cnt, w.pos,
                                                              w.kid, w.perm0, w.sk, bvh->perm(), bvh->keys(),
                                                              bvh->parent(), bvh->rend());
        count_launch();
    }
    // Agglomerative clustering gives no depth bound (equal boxes merge into a
    // chain), while every traversal keeps at most kMaxTreeDepth deferred
    // entries.  A deeper tree is replaced by the Karras tree over the same
    // faces (depth <= 30 key bits + log2 n + 1), with an informational bit.
    int deep = 0;
    if (cudaMemsetAsync(w.tot, 0, sizeof(int), s) != cudaSuccess) return MESH_ERR_CUDA;
    k_depth_check<<<grid_for(n, kBlock), kBlock, 0, s>>>(n, bvh->parent(), kMaxTreeDepth, w.tot);
    count_launch();
    if (cudaMemcpyAsync(&deep, w.tot, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MESH_ERR_CUDA;
    if (deep) {
        mesh_status st = mesh_build_lbvh(bvh, d_V, nV, d_F, nF, d_ws, ws_bytes, stream);
        if (st != MESH_OK) return st;
        k_set_status<<<1, 1, 0, s>>>(bvh->hdr(), MESH_DEV_DEEP_TREE);
        count_launch();
        return check_launch();
    }
    return bottom_up(bvh, nullptr, s);
}

size_t mesh_morton_order_workspace_bytes(int64_t n) { return mesh_build_workspace_bytes(n); }

mesh_status mesh_morton_order(const float *d_P, int64_t n, int32_t *d_order, void *d_ws,
                              size_t ws_bytes, void *stream) {
    if (n < 0 || n > kMaxFaces || (n > 0 && (!d_P || !d_order))) return MESH_ERR_INVALID_ARG;
    if (n == 0) return MESH_OK;
    BuildWs w = build_ws_layout((char *)d_ws, n);
    if (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int m = (int)n;
    k_init_box<<<1, 32, 0, s>>>(w.cbox);
    k_points_centroids<<<grid_for(m, kBlock), kBlock, 0, s>>>(d_P, m, w.cent, w.cbox);
    k_morton<<<grid_for(m, kBlock), kBlock, 0, s>>>(w.cent, m, w.cbox, w.keysA, w.valsA);
    count_launch(3);
    radix_sort_pairs(w, m, w.keysA, d_order, s);
    return check_launch();
}

size_t mesh_batch_storage_bytes(int64_t max_scenes, int64_t max_verts, int64_t max_faces) {
    if (max_scenes < 1 || max_scenes > 65536 || max_verts < 0 || max_faces < 0 ||
        max_faces > kMaxFaces || max_verts > kMaxFaces)
        return 0;
    return batch_layout(max_scenes, max_verts, max_faces).storage_bytes;
}

size_t mesh_batch_workspace_bytes(int64_t max_scenes, int64_t max_faces) {
    if (max_scenes < 1 || max_scenes > 65536 || max_faces < 0 || max_faces > kMaxFaces) return 0;
    return batch_ws_layout(nullptr, max_scenes, max_faces).bytes;
}

mesh_status mesh_batch_create(void *d_storage, size_t storage_bytes, int64_t max_scenes,
                              int64_t max_verts, int64_t max_faces, mesh_batch **out) {
    if (!out || !d_storage || ((uintptr_t)d_storage & 255u)) return MESH_ERR_INVALID_ARG;
    size_t need = mesh_batch_storage_bytes(max_scenes, max_verts, max_faces);
    if (need == 0) return MESH_ERR_INVALID_ARG;
    if (storage_bytes < need) return MESH_ERR_WORKSPACE;
    mesh_batch *h = (mesh_batch *)std::calloc(1, sizeof(mesh_batch));
    if (!h) return MESH_ERR_INVALID_ARG;
    h->base = (char *)d_storage;
    h->L = batch_layout(max_scenes, max_verts, max_faces);
    *out = h;
    return MESH_OK;
}

void mesh_batch_destroy(mesh_batch *batch) { std::free(batch); }

mesh_status mesh_batch_get_layout(const mesh_batch *batch, mesh_batch_layout *out) {
    if (!batch || !out) return MESH_ERR_INVALID_ARG;
    *out = batch->L;
    return MESH_OK;
}

mesh_status mesh_batch_build(mesh_batch *batch, int64_t n_scenes, const float *d_V,
                             const int32_t *d_vert_off, int64_t nV, const int32_t *d_F,
                             const int32_t *d_face_off, int64_t nF, void *d_ws, size_t ws_bytes,
                             void *stream) {
    if (!batch || n_scenes < 1 || n_scenes > batch->L.max_scenes || nV < 0 || nF < 0 ||
        nV > batch->L.max_verts || nF > batch->L.max_faces || !d_vert_off || !d_face_off)
        return MESH_ERR_INVALID_ARG;
    if ((nV > 0 && !d_V) || (nF > 0 && (!d_F || nV == 0))) return MESH_ERR_INVALID_ARG;
    BatchWs w = batch_ws_layout((char *)d_ws, n_scenes, nF);
    if (nF > 0 && (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u))) return MESH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    batch->L.n_scenes = n_scenes;
    batch->L.n_verts = nV;
    batch->L.n_faces = nF;
    int B = (int)n_scenes, n = (int)nF;
    cudaMemsetAsync(batch->st(), 0, sizeof(BatchStatus), s);
    cudaMemsetAsync(batch->scene_box(), 0, 32 * (size_t)B, s);
    cudaMemcpyAsync(batch->vert_off(), d_vert_off, 4 * (size_t)(B + 1), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(batch->face_off(), d_face_off, 4 * (size_t)(B + 1), cudaMemcpyDeviceToDevice, s);
    if (nV > 0) {
        k_copy_verts<<<grid_for(nV, kBlock), kBlock, 0, s>>>(d_V, (int)nV, batch->verts(), nullptr);
        count_launch();
    }
    if (n == 0) return check_launch();
    unsigned int *status = &batch->st()->status;
    k_batch_init<<<grid_for(6 * B, kBlock), kBlock, 0, s>>>(w.cbox, B);
    k_batch_faces<<<grid_for(n, kBlock), kBlock, 0, s>>>(d_F, n, batch->vert_off(), batch->face_off(),
                                                         B, batch->verts(), batch->faces(), w.sort.cent,
                                                         w.cbox, status);
    k_batch_morton<<<grid_for(n, kBlock), kBlock, 0, s>>>(w.sort.cent, n, batch->faces(), w.cbox,
                                                          w.key_of_face, w.sort.keysA, w.sort.valsA);
    count_launch(3);
    // Morton order over all faces, then a stable pass (two past 256 scenes) on
    // the scene id: faces end up grouped by scene in the order a per-scene
    // build would give them.
    radix_sort_pairs(w.sort, n, w.sort.keysA, w.sort.valsA, s);
    k_batch_scene_keys<<<grid_for(n, kBlock), kBlock, 0, s>>>(w.sort.valsA, n, batch->faces(),
                                                              w.sort.keysA);
    count_launch();
    if (B <= 256) {
        radix_pass(w.sort, n, 0, w.sort.keysA, w.sort.valsA, w.sort.keysB, batch->perm(), s);
    } else {
        radix_pass(w.sort, n, 0, w.sort.keysA, w.sort.valsA, w.sort.keysB, w.sort.valsB, s);
        radix_pass(w.sort, n, 8, w.sort.keysB, w.sort.valsB, w.sort.keysA, batch->perm(), s);
    }
    k_batch_gather_keys<<<grid_for(n, kBlock), kBlock, 0, s>>>(batch->perm(), n, w.key_of_face,
                                                               batch->keys());
    k_batch_karras<<<grid_for(n, kBlock), kBlock, 0, s>>>(batch->keys(), n, batch->face_off(), B,
                                                          batch->nodes(), batch->parent_int(),
                                                          batch->parent_leaf());
    count_launch(2);
    cudaMemsetAsync(batch->flags(), 0, sizeof(unsigned int) * (size_t)n, s);
    k_batch_leaves_up<<<grid_for(n, kBlock), kBlock, 0, s>>>(
        n, batch->face_off(), B, batch->perm(), batch->faces(), batch->verts(), batch->tris(),
        batch->nodes(), batch->parent_int(), batch->parent_leaf(), batch->flags(), batch->scene_box());
    count_launch();
    return check_launch();
}

mesh_status mesh_batch_refit(mesh_batch *batch, const float *d_V, int64_t nV, void *stream) {
    if (!batch || (d_V && nV != batch->L.n_verts)) return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_V && nV > 0) {
        k_copy_verts<<<grid_for(nV, kBlock), kBlock, 0, s>>>(d_V, (int)nV, batch->verts(), nullptr);
        count_launch();
    }
    int n = (int)batch->L.n_faces;
    if (n == 0) return check_launch();
    k_batch_leaves_up<<<grid_for(n, kBlock), kBlock, 0, s>>>(
        n, batch->face_off(), (int)batch->L.n_scenes, batch->perm(), batch->faces(), batch->verts(),
        batch->tris(), batch->nodes(), batch->parent_int(), batch->parent_leaf(), batch->flags(),
        batch->scene_box());
    count_launch();
    return check_launch();
}

mesh_status mesh_batch_status(mesh_batch *batch, uint32_t *bits, uint32_t *n_degenerate,
                              void *stream) {
    if (!batch) return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int h[2] = {0u, 0u};
    if (cudaMemcpyAsync(h, batch->st(), sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MESH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MESH_ERR_CUDA;
    if (cudaMemsetAsync(batch->st(), 0, sizeof(h), s) != cudaSuccess) return MESH_ERR_CUDA;
    if (bits) *bits = h[0];
    if (n_degenerate) *n_degenerate = h[1];
    return (h[0] & ~(unsigned)(MESH_DEV_DEGENERATE | MESH_DEV_DEEP_TREE)) ? MESH_ERR_DEVICE : MESH_OK;
}

uint64_t mesh_launch_count(void) { return (uint64_t)g_launches.load(); }

mesh_status mesh_mapped_pointer(const void *host, void **device) {
    if (!host || !device) return MESH_ERR_INVALID_ARG;
    void *d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<void *>(host), 0) != cudaSuccess || !d) {
        cudaGetLastError();                          // not page-locked: clear the error
        return MESH_ERR_CUDA;
    }
    *device = d;
    return MESH_OK;
}

}  // extern "C"
