// Internal definitions shared by the meshgs CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "meshgs.h"

namespace meshgs {

// Device-side header at the start of every BVH storage block.
struct __align__(16) Header {
    float4 root_lo;          // mesh box (all referenced vertices)
    float4 root_hi;
    unsigned int status;     // sticky MESH_DEV_* bits
    unsigned int n_degenerate;
    unsigned int pad[2];
};

struct mesh_bvh_impl {
    char *base;
    mesh_bvh_layout L;
    int cfg_lanes = -1;      // per-handle traversal choice; -1 = process-wide setting
    int cfg_variant = -1;
    int cfg_block = 128;     // threads per block of the one-thread traversal (variants 0, 2, 3)
    int leaf_size = 1;       // faces per collapsed leaf, written by the next build / refit
    mutable bool wide_valid = false;   // the 4-wide records match the node records
    Header *hdr() const { return reinterpret_cast<Header *>(base + L.off_header); }
    float4 *verts() const { return reinterpret_cast<float4 *>(base + L.off_verts); }
    int4 *faces() const { return reinterpret_cast<int4 *>(base + L.off_faces); }
    unsigned int *keys() const { return reinterpret_cast<unsigned int *>(base + L.off_keys); }
    int *perm() const { return reinterpret_cast<int *>(base + L.off_perm); }
    float4 *nodes() const { return reinterpret_cast<float4 *>(base + L.off_nodes); }
    int *parent() const { return reinterpret_cast<int *>(base + L.off_parent); }
    float4 *tris() const { return reinterpret_cast<float4 *>(base + L.off_tris); }
    float4 *wide() const { return reinterpret_cast<float4 *>(base + L.off_wide); }
    int *rend() const { return reinterpret_cast<int *>(base + L.off_rend); }
    int *iperm() const { return reinterpret_cast<int *>(base + L.off_iperm); }
    int *adj() const { return reinterpret_cast<int *>(base + L.off_adj); }
    float4 *fnorm() const { return reinterpret_cast<float4 *>(base + L.off_fnorm); }
    bool adj_ready = false;  // face adjacency matches the current topology
    int *xlist() const { return reinterpret_cast<int *>(base + L.off_xlist); }
};

struct BatchStatus {
    unsigned int status;
    unsigned int n_degenerate;
    unsigned int work;       // persistent-kernel work counter
    unsigned int pad;
};

struct mesh_batch_impl {
    char *base;
    mesh_batch_layout L;
    float4 *scene_box() const { return reinterpret_cast<float4 *>(base + L.off_scene); }
    BatchStatus *st() const { return reinterpret_cast<BatchStatus *>(base + L.off_status); }
    int *vert_off() const { return reinterpret_cast<int *>(base + L.off_vert_off); }
    int *face_off() const { return reinterpret_cast<int *>(base + L.off_face_off); }
    float4 *verts() const { return reinterpret_cast<float4 *>(base + L.off_verts); }
    int4 *faces() const { return reinterpret_cast<int4 *>(base + L.off_faces); }
    unsigned int *keys() const { return reinterpret_cast<unsigned int *>(base + L.off_keys); }
    int *perm() const { return reinterpret_cast<int *>(base + L.off_perm); }
    float4 *nodes() const { return reinterpret_cast<float4 *>(base + L.off_nodes); }
    int *parent_int() const { return reinterpret_cast<int *>(base + L.off_parent_int); }
    int *parent_leaf() const { return reinterpret_cast<int *>(base + L.off_parent_leaf); }
    float4 *tris() const { return reinterpret_cast<float4 *>(base + L.off_tris); }
    unsigned int *flags() const { return reinterpret_cast<unsigned int *>(base + L.off_flags); }
};

// Largest s in [0, n) with off[s] <= x (off non-decreasing, off[0] = 0): the
// non-empty segment that contains x.
__device__ __forceinline__ int segment_of(const int *__restrict__ off, int n, int64_t x) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits
// (lbvh.cu); the workspace is used for the intermediate passes.  vin NULL: the
// values are the indices (the output is the sorting permutation).
size_t sort_pairs_ws_bytes(int64_t n);
void sort_pairs_u32(void *ws, int n, int bits, const unsigned int *kin, const int *vin, unsigned int *kout,
                    int *vout, cudaStream_t s);

// Exclusive scan of n ints (splat.cu); bsum holds ceil(n / 1024) ints, total
// receives the sum.  Three launches on s.
void exclusive_scan_int(const int *in, int *out, int n, int *bsum, int *total, cudaStream_t s);

// Host-side bookkeeping shared by the entry points.
void count_launch(int n = 1);
mesh_status check_launch();

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// pdl_launch may be scheduled before the kernel ahead of it in the stream has
// finished: it calls pdl_wait() (griddepcontrol.wait) before its first access
// to memory, which returns once that kernel has completed and its writes are
// visible, so the ordering is that of a plain launch and only the launch
// latency is hidden.  pdl_trigger() (griddepcontrol.launch_dependents) lets the
// next such kernel be scheduled once every block of this one has started.  A
// kernel launched plainly passes both at once.  Errors surface through
// check_launch().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// launch_ex(pdl = false, ...) is a plain launch of the same kernel.
template <typename... KArgs, typename... Args>
inline void launch_ex(bool pdl, void (*kernel)(KArgs...), unsigned int grid, unsigned int block, size_t smem,
                      cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), unsigned int grid, unsigned int block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    launch_ex(true, kernel, grid, block, smem, s, std::forward<Args>(args)...);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

inline unsigned int grid_for(int64_t n, int block) {
    return (unsigned int)((n + block - 1) / block);
}

// Largest leaf size of the collapse (faces tested in one leaf range).
constexpr int kMaxLeafSize = 8;

// Deepest tree every traversal handles: the depth-first searches keep at most
// one deferred sibling per level, in stacks of this many entries.
constexpr int kMaxTreeDepth = 64;

// Tie rule of NearestSurface: faces within (1 + 1e-6) of the nearest distance
// (plus 1e-12 of the box diagonal) count as equally near; the lowest id wins.
constexpr float kTieRel = 1e-6f;
constexpr float kTieAbs = 1e-12f;

__device__ __forceinline__ float4 ldg4(const float4 *p) { return __ldg(p); }

__device__ __forceinline__ void set_status(Header *h, unsigned int bit) {
    atomicOr(&h->status, bit);
}

// The 4-wide records of traversal variant 13 (query.cu): wide_refresh writes them
// from the node records on stream s (as a programmatic dependent when pdl) and
// marks them current; wide_wanted tells whether the handle's traversal is
// variant 13, so that its builds and refits refresh them.
void wide_refresh(const mesh_bvh *b, cudaStream_t s, bool pdl);
bool wide_wanted(const mesh_bvh *b);

}  // namespace meshgs

struct mesh_bvh : meshgs::mesh_bvh_impl {};
struct mesh_batch : meshgs::mesh_batch_impl {};
