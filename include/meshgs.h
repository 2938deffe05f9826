/*
 * meshgs -- per-frame dynamic-mesh update on the GPU, C ABI.
 *
 * Ramlal & Zelek, "Real-Time Physics Simulation with Dynamic Mesh-Gaussian
 * Reconstructions" (CVIS 2026) keep a fixed-topology physics mesh and a set of
 * mesh-bound Gaussians in sync (Sec. 3.2).  Every frame the vertex buffer is
 * replaced (Sec. 3.4, Per-Frame Update), collision queries run against it
 * (Sec. 3.4, step 3), and the Gaussians follow their faces.  The
 * varying-topology baseline instead rebuilds the collision structure each
 * frame (Sec. 4.1).  This library provides those steps as CUDA kernels:
 *
 *   mesh_build_lbvh       full BVH build (Morton keys, radix sort, Karras
 *                         hierarchy, bottom-up boxes) -- the rebuild of Sec. 4.1
 *   mesh_build_ploc       the tree of a mesh built once and then refit
 *                         (agglomerative clustering; Sec. 3.4, Initialization)
 *   mesh_update_vertices  the O(N_v) vertex-buffer update of Sec. 3.4
 *   mesh_refit            boxes recomputed over the fixed topology
 *   mesh_closest_point    NearestSurface of Eq. 1 / Eq. 2 (exact closest point,
 *                         barycentric weights, optional contact cutoff)
 *   mesh_contact          the contact query of a physics step (warm-started,
 *                         ordered by the previous step's work)
 *   mesh_bind_gaussians   face-bound Gaussian centre / rotation / scale
 *   mesh_chamfer          point-to-mesh Chamfer distance of Sec. 4.2
 *   *_backward            gradients with respect to vertices and query points
 *   mesh_batch_*          many scenes in single launches
 *
 * Conventions (all entry points):
 *   - Pointers named d_* are DEVICE pointers owned by the caller (pinned host
 *     memory mapped by mesh_mapped_pointer qualifies); the library never
 *     allocates device memory (mesh_chamfer_noalloc's fixed scratch array is
 *     the one static exception).  A BVH lives in caller-provided storage
 *     (mesh_bvh_storage_bytes) and a build uses caller-provided scratch
 *     (mesh_build_workspace_bytes).  Host pointers are named without d_.
 *   - Positions are float32, row-major xyz: vertices [nV][3], queries [nQ][3].
 *     Faces are int32 [nF][3] vertex indices (0-based), counter-clockwise.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL is the legacy default stream) and may be captured in a CUDA graph,
 *     except the few that say they are synchronous (mesh_build_ploc,
 *     mesh_gs_render and mesh_emd read counts back on the host;
 *     mesh_gs_render_capacity is the render's asynchronous form).
 *     Host-side argument errors are returned at once and launch nothing.
 *     Device-side problems (an index out of range, a traversal stack
 *     overflow) set sticky bits in the BVH's status word, read and cleared by
 *     mesh_bvh_status(); the kernels never trap.
 *   - No call is thread-safe against concurrent calls on the same handle.
 */
#ifndef MESHGS_H
#define MESHGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MESH_OK = 0,
    MESH_ERR_INVALID_ARG = 1,   /* null pointer, negative or too-large size      */
    MESH_ERR_CUDA = 2,          /* a CUDA runtime call or launch failed            */
    MESH_ERR_WORKSPACE = 3,     /* caller storage / workspace smaller than needed  */
    MESH_ERR_DEVICE = 4         /* mesh_bvh_status found device-side status bits   */
} mesh_status;

/* Device status bits (mesh_bvh_status). */
#define MESH_DEV_INDEX_RANGE     0x1u  /* a face / Gaussian / sample index was out of range; the
                                          offending element was skipped or clamped to 0 */
#define MESH_DEV_STACK_OVERFLOW  0x2u  /* traversal stack exhausted (cannot happen: every tree is at
                                          most 64 levels deep, see MESH_DEV_DEEP_TREE)            */
#define MESH_DEV_DEGENERATE      0x4u  /* a Gaussian sat on a zero-area face (not an error)       */
#define MESH_DEV_NONMANIFOLD     0x8u  /* an edge shared by more than two faces (signed distance) */
#define MESH_DEV_DEEP_TREE       0x10u /* mesh_build_ploc's tree was deeper than the 64 levels every
                                          traversal handles; the Karras tree of mesh_build_lbvh was
                                          built instead (not an error)                            */

typedef struct mesh_bvh mesh_bvh;   /* opaque host handle describing device storage */

/* Child links in the node records: an internal node c >= 0, leaf j as -(j+1). */
typedef struct {
    int64_t n_faces, n_verts, max_faces, max_verts;
    /* byte offsets inside the storage block given to mesh_bvh_create */
    size_t off_header;   /* float4 root_lo, float4 root_hi, then uint32 status, uint32 n_degenerate */
    size_t off_verts;    /* float4 [max_verts]   vertex buffer, w = 0                          */
    size_t off_faces;    /* int4   [max_faces]   (v0, v1, v2, 0) in input face order           */
    size_t off_keys;     /* uint32 [max_faces]   Morton keys in leaf order (sorted for the
                            Karras tree of mesh_build_lbvh)                                    */
    size_t off_perm;     /* int32  [max_faces]   face id of leaf j                             */
    size_t off_nodes;    /* 4 x float4 per internal node: (lo_L, left) (hi_L, nL)
                                                          (lo_R, right) (hi_R, nR),
                            as int32 bits in .w: the child link (internal c >= 0, or a leaf
                            range -(first+1)) and n = the range's face count (1 without
                            leaf collapse), or c again for an internal child            */
    size_t off_parent;   /* int32  [2 max_faces - 1]  2 * parent + side (0 left, 1 right),
                            -1 at the root; internal nodes first, then leaves                 */
    size_t off_tris;     /* 3 x float4 per leaf: (v0, face id bits) (v1, 0) (v2, 0)           */
    size_t off_rend;     /* int32 [max_faces]   far end of internal node i's leaf range        */
    size_t off_iperm;    /* int32 [max_faces]   leaf of face f (inverse of perm)               */
    size_t off_adj;      /* int32 [max_faces][3] face across the edge opposite vertex k, or -1  */
    size_t off_fnorm;    /* float4 [max_faces]  unit face normals (signed distance)            */
    size_t off_xlist;    /* bottom-up scratch: per leaf the prefix and suffix box unions
                            inside its block of 512 leaves (2 x 32 B), the nodes whose leaf
                            ranges cross blocks int32x4 [max_faces] (node, range start, range
                            end, parent link), per block its box (32 B) and its count of
                            crossing nodes (int32)                                           */
    size_t off_wide;     /* 8 x float4 per internal node: its 4-wide record (traversal variant
                            13), four slots (lo, link) (hi, n) laid out as in the node records:
                            per side, the child's own node record when the child is internal
                            (its two children), else the node's slot for that leaf link and an
                            empty slot (link INT32_MIN, lo +inf, hi -inf, n 0).  Written from the
                            node records by every build or refit of a handle whose traversal is
                            variant 13, else by the first variant-13 query after one           */
    size_t storage_bytes;
} mesh_bvh_layout;

/* ---------------------------------------------------------------- */
/* Storage and handles                                               */
/* ---------------------------------------------------------------- */

/* Device bytes a BVH over up to max_faces faces / max_verts vertices occupies. */
size_t mesh_bvh_storage_bytes(int64_t max_verts, int64_t max_faces);

/* Device scratch bytes one mesh_build_lbvh over up to max_faces faces needs. */
size_t mesh_build_workspace_bytes(int64_t max_faces);

/* Wrap caller storage (>= mesh_bvh_storage_bytes, 256-byte aligned) in a handle.
 * Host-only: allocates the small host struct, touches no device memory. */
mesh_status mesh_bvh_create(void *d_storage, size_t storage_bytes, int64_t max_verts,
                            int64_t max_faces, mesh_bvh **out);

/* Free the host struct only; the storage stays the caller's. */
void mesh_bvh_destroy(mesh_bvh *bvh);

/* Offsets of every array inside the storage (for inspection and tests). */
mesh_status mesh_bvh_get_layout(const mesh_bvh *bvh, mesh_bvh_layout *out);

/* ---------------------------------------------------------------- */
/* The update steps                                                  */
/* ---------------------------------------------------------------- */

/* Full LBVH build from scratch over (V, F): the collision-structure rebuild the
 * varying-topology baseline pays every frame (Sec. 4.1) and the one-off build
 * from F0 (Sec. 3.4, Initialization).  Copies V into the handle's vertex
 * buffer and F into its face table, computes 30-bit Morton keys of face
 * centroids, radix-sorts them (stable), builds Karras's binary radix tree and
 * its boxes bottom-up.  nF may be 0 (every query then misses).  F indices
 * outside [0, nV) set MESH_DEV_INDEX_RANGE and are read as 0.
 * d_ws: >= mesh_build_workspace_bytes(nF) bytes of scratch, 256-byte aligned,
 * free for other use once the stream has passed this call. */
mesh_status mesh_build_lbvh(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_F,
                            int64_t nF, void *d_ws, size_t ws_bytes, void *stream);

/* Agglomerative build for a mesh whose topology is fixed (built once from the
 * template faces, Sec. 3.4, then refit every frame): the same vertex/face
 * tables and Morton order as mesh_build_lbvh, then parallel locally-ordered
 * clustering (PLOC, Meister & Bittner 2018) over the sorted leaves -- every
 * cluster picks the cluster within 16 positions whose union box has the least
 * surface area (float32, (dx dy + dy dz) + dz dx without fused multiply-add;
 * ties to the lower position), mutual pairs merge at the lower position, the
 * clusters are compacted, until one is left.  The tree is laid out like the
 * Karras tree (leaves in in-order, an internal node numbered by the end of its
 * leaf range not shared with its sibling, root 0), so refit, every query and
 * the batched and backward entry points use it unchanged; d_keys then holds
 * the leaves' Morton keys in leaf order (not sorted).  Its boxes have a lower
 * surface-area cost than the Karras tree's, so queries visit fewer nodes.
 * SYNCHRONOUS: the host reads the cluster count back after every iteration
 * (tens of iterations), so the call returns when the build is done and must
 * not be captured in a CUDA graph.  Clustering bounds no depth (equal boxes
 * merge into a chain), and every traversal handles at most 64 levels: the
 * build measures the finished tree's depth and, past 64, builds the Karras
 * tree of mesh_build_lbvh over the same faces instead and sets the
 * informational bit MESH_DEV_DEEP_TREE.  d_ws: mesh_build_ploc_workspace_bytes(nF),
 * 256-byte aligned.  Argument errors as mesh_build_lbvh; MESH_ERR_CUDA also
 * when an iteration's counts are inconsistent (the build then stops). */
size_t mesh_build_ploc_workspace_bytes(int64_t max_faces);
mesh_status mesh_build_ploc(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_F,
                            int64_t nF, void *d_ws, size_t ws_bytes, void *stream);

/* Morton order of a point set, for query coherence: d_order [n] receives the
 * permutation that sorts the points by the 30-bit key of mesh_build_lbvh (a
 * point p keyed as the zero-area face (p, p, p), over the points' own box),
 * ties by index.  Storing queries in this order (e.g. a particle set that
 * persists across frames) makes neighbouring threads traverse the same nodes.
 * d_ws: >= mesh_morton_order_workspace_bytes(n) bytes, 256-byte aligned. */
size_t mesh_morton_order_workspace_bytes(int64_t n);
mesh_status mesh_morton_order(const float *d_P, int64_t n, int32_t *d_order, void *d_ws,
                              size_t ws_bytes, void *stream);

/* Vertex-buffer update of Sec. 3.4 (step 2): copy V_k ([nV][3], nV equal to
 * the built mesh's) into the handle's vertex buffer.  Topology is untouched. */
mesh_status mesh_update_vertices(mesh_bvh *bvh, const float *d_V, int64_t nV, void *stream);

/* Recompute every node box over the fixed topology from the current vertex
 * buffer (after mesh_update_vertices).  If d_V is not NULL (nV equal to the
 * built mesh's) the vertex-buffer update is part of the same pass, with the
 * same result as mesh_update_vertices(bvh, d_V, nV) followed by
 * mesh_refit(bvh, NULL, 0).  Two kernels, the same the build ends with: one
 * block per 512 consecutive leaves answers every node whose leaf range lies
 * inside the block from a sparse table of its leaf boxes in shared memory
 * (and writes each leaf's prefix and suffix union in the block), then one
 * warp per node whose range crosses blocks unions the suffix, the prefix and
 * the boxes of the blocks between.  No atomics and no waits; nothing is
 * derived once per topology: a refit after any build is valid. */
mesh_status mesh_refit(mesh_bvh *bvh, const float *d_V, int64_t nV, void *stream);

/* mesh_refit and mesh_bind_gaussians in one pass (the fixed-topology frame of
 * Sec. 3.4: new vertices, new boxes, Gaussians moved with their faces).  The
 * refit's leaf threads, which gather their faces' corners for the leaf boxes,
 * also compute each face's normal, rotation and scale once (they depend on
 * the face alone); the block's threads then take the Gaussians of its 512
 * leaves one per thread, each computing its centre.  The Gaussians are
 * grouped by face: those of face f are g = d_gstart[f] .. d_gstart[f + 1] - 1
 * (int32 [nF + 1], non-decreasing, d_gstart[nF] = nG), with weights d_gbary
 * [nG][3] and normal offsets d_goff [nG] (NULL = 0); outputs as
 * mesh_bind_gaussians, indexed by g (writes are contiguous where the
 * Gaussians of neighbouring leaves are, e.g. when g follows the tree's leaf
 * order).  A face whose range is decreasing or past nG sets
 * MESH_DEV_INDEX_RANGE and its Gaussians are not written (so does a block
 * whose Gaussians number more than INT_MAX, possible only when ranges
 * overlap).  The same results as the two calls, bit for bit. */
mesh_status mesh_refit_bind(mesh_bvh *bvh, const float *d_V, int64_t nV, const int32_t *d_gstart,
                            const float *d_gbary, const float *d_goff, int64_t nG, float *d_mu,
                            float *d_quat, float *d_scale, void *stream);

/* NearestSurface (Eq. 1 / Eq. 2): for each query q the closest point of the
 * mesh, as face id, barycentric weights (u, v, w) of (v0, v1, v2), the point
 * u v0 + v v1 + w v2 and its squared distance.  Ties: the nearest face is the
 * lowest face id among the faces whose computed (float32) distance lies
 * within d* (1 + 1e-6) + 1e-12 x box diagonal, d* the least computed distance
 * (the spec rule of Eq. 1 / Eq. 2's NearestSurface).  The answer is a
 * function of the query and the mesh only: every tree (LBVH or agglomerative),
 * traversal variant, lane width and warm start gives the same face, weights,
 * point and distance, bit for bit.  It differs from a float64 evaluation of
 * the same rule only where float32 rounding moves a face across the window
 * (faces whose exact distances are within ~1e-7 x the coordinate magnitude of
 * each other or of the window's edge).  A query with no face within max_dist
 * (INFINITY = no cutoff) gets face -1, dist2 = +inf, bary = point = 0.  Any
 * output pointer may be NULL (not written).  With the one-thread depth-first
 * variants, a call that takes faces and distances and weights or points runs
 * as two launches: the search, then the weights and points of the hits. */
mesh_status mesh_closest_point(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                               float max_dist, int32_t *d_face, float *d_bary, float *d_point,
                               float *d_dist2, void *stream);

/* mesh_closest_point with a warm start: d_hint[i] (a face id, e.g. query i's
 * nearest face in the previous frame; -1 or out of range = none) is tested
 * before the traversal and its distance bounds the search.  Every face within
 * the final tie window is still reached, so the answer is the one without the
 * hint, bit for bit; the hint changes only the work.  d_hint may be the same
 * array as d_face (each query reads its hint before writing its face).  Used by
 * the depth-first one-thread variants (0, 2-9, 13), the warp packets (12) and
 * the cooperative groups (lanes > 1); variants 1, 10 and 11 ignore it. */
mesh_status mesh_closest_point_hinted(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                                      float max_dist, const int32_t *d_hint, int32_t *d_face,
                                      float *d_bary, float *d_point, float *d_dist2, void *stream);

/* k-NN weighted surface projection, the NearestSurface of temporal tracking
 * (Sec. 3.3, Strategy 1, Eq. 1), which the paper names without k or weights:
 * for query q the k (1..8) faces nearest to it (ties: the lower face id), each
 * giving its closest point p_j at distance d_j, blended as
 *   q' = sum w_j p_j / sum w_j,  w_j = 1 / max(d_j, 1e-6 x box diagonal);
 * with d_anchor (NULL = none), q'' = (1 - anchor_weight) q' + anchor_weight
 * anchor (the periodic re-anchoring to the template projection).  Outputs:
 * d_point [nQ][3] (may be the same array as d_Q: each query is read before it
 * is written), optional d_face [nQ][k] and d_dist2 [nQ][k], nearest first
 * (face -1 / +inf past the mesh's face count).  No faces: q' = q. */
mesh_status mesh_knn_project(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, int k,
                             const float *d_anchor, float anchor_weight, float *d_point,
                             int32_t *d_face, float *d_dist2, void *stream);

/* Workspace bytes for mesh_signed_distance's first call after a build (the
 * face-adjacency table over 3 nF half-edges); 0 for nF out of range. */
size_t mesh_signed_workspace_bytes(int64_t nF);

/* Signed NearestSurface distance for contact (inside negative), for
 * penetration depth: as mesh_closest_point (same face, weights, point, tie
 * rule and cutoff), plus d_sdist[i] = sign * distance with the sign of
 * (q - c) . N, N the angle-weighted pseudo-normal (Baerentzen & Aanaes 2005)
 * of the face, edge or vertex the nearest point c lies on; +inf beyond
 * max_dist.  The mesh must be closed, manifold and consistently
 * counter-clockwise seen from outside (an edge with one face uses that
 * face's normal; an edge of three or more faces sets MESH_DEV_NONMANIFOLD).
 * The first call after a build derives the face adjacency with d_ws
 * (mesh_signed_workspace_bytes(nF) bytes, 256-byte aligned; NULL is fine on
 * later calls) and every call recomputes the normals from the current
 * vertex buffer (two extra launches).  d_face, d_bary, d_point may be NULL. */
mesh_status mesh_signed_distance(mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                                 void *d_ws, size_t ws_bytes, int32_t *d_face, float *d_bary,
                                 float *d_point, float *d_sdist, void *stream);

/* Workspace bytes of mesh_emd for n points per set; 0 for n out of range. */
size_t mesh_emd_workspace_bytes(int64_t n);

/* Earth Mover's Distance between point sets A and B of n points each
 * (Sec. 4.2's EMD on sampled points): the minimum over bijections sigma of
 * the mean |a_i - b_sigma(i)|, by the auction algorithm with epsilon scaling.
 * The result is within eps_rel x (box diagonal of A and B) of the exact
 * minimum (an epsilon-optimal assignment).  d_out[0] = the mean (float64);
 * d_assign (NULL = not written) = sigma, int32 [n].  Synchronous: the host
 * runs the auction rounds on `stream` and reads a counter every 16 rounds,
 * so the call returns when the result is final.  max_iters bounds the rounds
 * (MESH_ERR_DEVICE if exceeded); *iters_out (NULL = not written) gets the
 * rounds used.  d_ws: mesh_emd_workspace_bytes(n) bytes, 256-byte aligned. */
mesh_status mesh_emd(const float *d_A, const float *d_B, int64_t n, float eps_rel, int64_t max_iters,
                     void *d_ws, size_t ws_bytes, double *d_out, int32_t *d_assign,
                     int64_t *iters_out, void *stream);

/* Pinhole camera for mesh_gs_render: x_c = R x + t (R row-major 3 x 3), image
 * point (fx x_c/z_c + cx, fy y_c/z_c + cy), pixel (px, py) samples the point
 * (px, py); Gaussians with z_c <= near_z are culled. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy, near_z;
    int width, height;
    float background[3];
} mesh_camera;

/* Workspace bytes of mesh_gs_render for nG Gaussians whose 3-sigma squares
 * touch n_instances tiles (of 16 x 16 pixels) in a width x height image. */
size_t mesh_gs_workspace_bytes(int64_t nG, int64_t n_instances, int width, int height);

/* Gaussian-splatting render of the face-bound Gaussians (Sec. 3.2's R_render)
 * by the forward equations of 3D Gaussian splatting: centres d_mu [nG][3],
 * rotations d_quat [nG][4] (w, x, y, z), scales d_scale [nG][3], opacities
 * d_opacity [nG], colours d_color [nG][3]; 2D covariance J R Sigma R^T J^T +
 * 0.3 I, 3-sigma tile squares, per-tile front-to-back blending (alpha =
 * min(0.99, o e^p), skipped below 1/255, a pixel stops before its
 * transmittance falls under 1e-4).  Writes d_image [height][width][3] (colour
 * plus T x background) and d_trans [height][width] (NULL = not written).
 * Synchronous: the host reads the instance count (one device-to-host copy)
 * before the tile sort.  If ws_bytes is too small for this view the call
 * writes the bytes needed to *ws_needed and returns MESH_ERR_WORKSPACE
 * without drawing; grow the workspace and call again. */
mesh_status mesh_gs_render(const float *d_mu, const float *d_quat, const float *d_scale,
                           const float *d_opacity, const float *d_color, int64_t nG,
                           const mesh_camera *cam, void *d_ws, size_t ws_bytes, size_t *ws_needed,
                           float *d_image, float *d_trans, void *stream);

/* mesh_gs_render with a caller-chosen instance capacity instead of the host
 * read of the instance count: asynchronous, no host synchronisation, so it
 * can be captured in a CUDA graph and replayed every frame (R_render of
 * Sec. 3.2 as a per-frame step).  max_instances bounds the (tile, Gaussian)
 * instances of one frame (e.g. the count of an earlier frame with a margin);
 * d_ws must hold mesh_gs_workspace_bytes(nG, max_instances, width, height)
 * bytes.  d_counts (DEVICE uint32 [2], may be NULL) receives {overflow, count}:
 * overflow = 1 when the frame had more instances than max_instances (the
 * instances of the farthest Gaussians, past the capacity, are dropped and the
 * image is incomplete), count = the frame's instances.  With enough capacity
 * the image and transmittance equal mesh_gs_render's bit for bit; the tile
 * sort runs over max_instances slots (the unused ones are keyed after every
 * real instance). */
mesh_status mesh_gs_render_capacity(const float *d_mu, const float *d_quat, const float *d_scale,
                                    const float *d_opacity, const float *d_color, int64_t nG,
                                    const mesh_camera *cam, int64_t max_instances, void *d_ws,
                                    size_t ws_bytes, float *d_image, float *d_trans, uint32_t *d_counts,
                                    void *stream);

/* Workspace bytes of mesh_contact for nQ queries. */
size_t mesh_contact_workspace_bytes(int64_t nQ);

/* The contact query of a physics step: NearestSurface of the nQ particles
 * with cutoff max_dist, with d_face both the previous step's answers (read
 * first, as warm-start hints: -1 = none) and this step's (written).  The
 * queries run in the order of the previous step's work: each query's node
 * visits give it a class (48 or more, 24-47, 12-23, fewer), kept in d_ws,
 * and the next call runs the classes heaviest first, each in the given
 * order, so that a warp holds searches of similar depth.  d_ws therefore
 * carries state from one step to the next: pass the same workspace every
 * step for the same particles; its contents steer only the order (a fresh
 * or unrelated workspace gives a worse order, never a wrong answer).
 * Answers equal mesh_closest_point's bit for bit.  The one-thread searches
 * write face and distance; the weights and closest points (when asked for)
 * follow in a second launch with one thread per query (the distances are kept
 * in d_ws when d_dist2 is NULL).
 * Traversal variants 1, 10, 11 and cooperative groups run unordered without
 * classes (the warp packets of variant 12 take the classes, counting for each
 * query the nodes whose children it needed).  d_ws:
 * mesh_contact_workspace_bytes(nQ), 256-byte aligned. */
mesh_status mesh_contact(const mesh_bvh *bvh, const float *d_Q, int64_t nQ, float max_dist,
                         int32_t *d_face, float *d_bary, float *d_point, float *d_dist2, void *d_ws,
                         size_t ws_bytes, void *stream);

/* Work counters of the one-thread depth-first traversal for these queries:
 * d_counts[0] = node visits (each reads one 64-byte record holding two child
 * boxes; with traversal variant 13, 4-wide records of 128 bytes), d_counts[1] =
 * triangle tests, d_counts[2] = queries with a face
 * within max_dist; uint64, summed over all queries.  Runs a separate counting
 * kernel; writes no query results.  For roofline accounting and diagnosis. */
mesh_status mesh_closest_point_stats(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                                     float max_dist, unsigned long long *d_counts, void *stream);

/* Lanes that cooperate on one query in mesh_closest_point and mesh_chamfer.
 * 0 (default) picks from the query count: one thread per query when the
 * queries fill the GPU, else the smallest power of two up to 32 that does (a
 * group pops several stack entries per step and merges its candidates with
 * the same tie rule).  1, 2, 4, 8, 16 or 32 force a width.  Process-wide,
 * not thread-safe; for tuning and tests.  Results are the same for every
 * width, bit for bit. */
mesh_status mesh_set_query_group(int lanes);

/* One-thread-per-query traversal variant for mesh_closest_point (tuning):
 *   0 depth-first, 24-entry shared-memory stack per thread (default)
 *   1 while-while: leaf children queued while internal nodes are traversed
 *   2 depth-first, 8 shared entries    3 depth-first, stack in local memory only
 *   4 as 0 with one leaf-test site     5 as 3 with one leaf-test site
 *   6 as 2, 9 blocks per SM (<= 56 registers)    7 as 3, 9 blocks per SM
 *   8 as 3, 16 blocks per SM (<= 32 registers)   9 as 5, 12 blocks per SM
 *  10 persistent, dynamic fetch: lanes take new queries as they finish
 *     (8 shared entries)                          11 as 10, local stack only
 *     (10 and 11 keep a work counter in the handle: calls on one handle must
 *     not overlap on the GPU)
 *  12 warp packet: the 32 queries of a warp share one node sequence, a node
 *     entered when any lane needs it (for queries kept in Morton order; it
 *     gains most from leaf collapse, mesh_bvh_set_leaf_size)
 *  13 depth-first over 4-wide records (each visit tests up to four boxes:
 *     the node's children, an internal child replaced by its two; about half
 *     the visits of the binary tree), 8 shared entries; the records are
 *     written from the binary tree by every build or refit of a handle whose
 *     traversal is 13, else by the first such query after one (layout
 *     off_wide; a host-side flag per handle: a captured graph that queries
 *     with 13 relies on the handle's refits writing them, so keep the handle
 *     at 13 while such a graph is replayed)
 * (the shared part of the stack spills to local memory; local-only leaves the
 * SM's L1 to the node cache).  Process-wide; the same answers, bit for bit,
 * for every variant. */
mesh_status mesh_set_traversal(int variant);

/* Traversal choice for mesh_closest_point calls on this handle (host-side
 * setting, read when a call is made, so a captured graph keeps the choice it
 * was captured with): lanes as mesh_set_query_group (0 = from the query
 * count), variant as mesh_set_traversal; -1 for either = follow the
 * process-wide setting (the default).  Set by the autotuner. */
mesh_status mesh_bvh_set_query_config(mesh_bvh *bvh, int lanes, int variant);

/* Leaf size L (1..8) of this handle's tree: from the next build or refit on,
 * every child whose subtree holds at most L faces is linked from its parent as
 * one leaf over its contiguous range of faces in leaf order (the topmost such
 * subtree; lo.w = -(first + 1), hi.w = the face count), and a search tests
 * those faces in one loop instead of visiting the nodes below.  The tree, its
 * boxes and every other array are those of L = 1 (the nodes below a collapsed
 * link are still refit, unreachable).  Answers do not depend on L, bit for
 * bit; the autotuner picks it.  Default 1.  Host-side setting. */
mesh_status mesh_bvh_set_leaf_size(mesh_bvh *bvh, int leaf_size);

/* Threads per block of this handle's one-thread traversals (mesh_closest_point
 * and mesh_contact with variants 0, 2 and 3): 128 (default; 0 = default), 64 or
 * 32.  Each form keeps the same register budget, so the same number of warps
 * fits an SM; smaller blocks free their slot as soon as their own searches end
 * (the searches of one block end at very different times).  Host-side setting,
 * read when a call is made (a captured graph keeps it); set by the autotuner.
 * The answers do not depend on it. */
mesh_status mesh_bvh_set_query_block(mesh_bvh *bvh, int threads);

/* Face-bound Gaussians from the handle's current vertex buffer.  For Gaussian
 * g on face f = d_gface[g] with weights b = d_gbary[g] and normal offset
 * delta = d_goff[g] (NULL = 0):
 *   e1 = (v1 - v0)/|v1 - v0|, n = unit((v1 - v0) x (v2 - v0)), e2 = n x e1,
 *   mu = b0 v0 + b1 v1 + b2 v2 + delta n,
 *   quat = unit quaternion (w, x, y, z) of [e1 e2 n] with w >= 0,
 *   scale = (l/3, h/3, 0.01 (l + h)/6), l = |v1 - v0|, h = 2 area / l.
 * Zero-area faces give mu from b alone, quat (1,0,0,0), scale 0 and set
 * MESH_DEV_DEGENERATE.  Outputs: d_mu [nG][3], d_quat [nG][4], d_scale [nG][3]. */
mesh_status mesh_bind_gaussians(const mesh_bvh *bvh, const int32_t *d_gface, const float *d_gbary,
                                const float *d_goff, int64_t nG, float *d_mu, float *d_quat,
                                float *d_scale, void *stream);

/* Points given by face id and barycentric weights on the current vertex
 * buffer: out[i] = sum_j bary[i][j] v_j(face[i]).  [n][3] float32. */
mesh_status mesh_interpolate(const mesh_bvh *bvh, const int32_t *d_face, const float *d_bary,
                             int64_t n, float *d_out, void *stream);

/* Chamfer distance (Sec. 4.2): d_out[0] = mean over SA of d(a, mesh B)^2,
 * d_out[1] = mean over SB of d(b, mesh A)^2, float64, summed in a fixed order
 * (bit-reproducible run to run).  Per-sample results for the backward pass
 * may be requested (any of the pointers may be NULL).
 * d_ws: >= mesh_chamfer_workspace_bytes(nSA, nSB) bytes of scratch. */
size_t mesh_chamfer_workspace_bytes(int64_t nSA, int64_t nSB);
mesh_status mesh_chamfer(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                         const mesh_bvh *B, const float *d_SB, int64_t nSB,
                         void *d_ws, size_t ws_bytes, double *d_out,
                         int32_t *d_faceA, float *d_baryA, float *d_dist2A,
                         int32_t *d_faceB, float *d_baryB, float *d_dist2B, void *stream);

/* mesh_chamfer with warm starts: d_hintA[i] is a face of mesh B for sample
 * SA[i] (e.g. its nearest face in the previous frame), d_hintB[i] a face of
 * mesh A for SB[i]; -1 or out of range = none, either pointer may be NULL,
 * and each may be the same array as the matching face output.  The answers
 * are those without hints, bit for bit; the hints change only the traversal
 * work. */
mesh_status mesh_chamfer_hinted(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                                const mesh_bvh *B, const float *d_SB, int64_t nSB, void *d_ws,
                                size_t ws_bytes, double *d_out, const int32_t *d_hintA,
                                const int32_t *d_hintB, int32_t *d_faceA, float *d_baryA,
                                float *d_dist2A, int32_t *d_faceB, float *d_baryB,
                                float *d_dist2B, void *stream);

/* Workspace bytes of mesh_chamfer_step for nSA + nSB samples (0 when their sum
 * exceeds INT32_MAX). */
size_t mesh_chamfer_step_workspace_bytes(int64_t nSA, int64_t nSB);

/* The Chamfer distance of Sec. 4.2 for a sequence of frames (a physics step or
 * an optimisation step on the same samples): mesh_chamfer with d_faceA /
 * d_faceB both the previous call's faces (read first, as warm-start hints:
 * -1 = none) and this call's (written), and the samples of each side run in
 * the order of the previous call's costs, heaviest first: each sample's cost
 * (its node visits / 8 with one lane per sample, its group steps with
 * several, capped at 127) is kept in d_ws as an 8-bit key with the side in bit
 * 7, and the next call sorts the keys of both sides with one stable radix
 * pass, so that the samples sharing a block end together and the longest
 * searches start first.  d_ws therefore carries state from one call to the
 * next: pass the same workspace for the same samples; its contents steer only
 * the order (a fresh or unrelated workspace gives a worse order, never a
 * wrong answer).  The per-sample outputs equal mesh_chamfer's bit for bit;
 * d_out equals it up to the order of the float64 sums (each block sums its
 * samples, and the blocks hold other samples in another order).  d_faceA is
 * required when nSA > 0, d_faceB when nSB > 0; the other outputs may be NULL.
 * d_ws: mesh_chamfer_step_workspace_bytes(nSA, nSB), 256-byte aligned;
 * MESH_ERR_WORKSPACE otherwise. */
mesh_status mesh_chamfer_step(const mesh_bvh *A, const float *d_SA, int64_t nSA, const mesh_bvh *B,
                              const float *d_SB, int64_t nSB, void *d_ws, size_t ws_bytes, double *d_out,
                              int32_t *d_faceA, float *d_baryA, float *d_dist2A, int32_t *d_faceB,
                              float *d_baryB, float *d_dist2B, void *stream);

/* mesh_chamfer for callers that cannot allocate device memory.  (The paper has
 * no counterpart; this exists for integrations, not for the method.)  Some
 * callers cannot call cudaMalloc -- a physics or renderer plugin whose host
 * application owns every device allocation, or code running while another
 * framework captures the stream into a CUDA graph and forbids allocation --
 * so they cannot supply mesh_chamfer's workspace.  This variant runs
 * mesh_chamfer's kernel, keeping its scratch in one fixed array inside the
 * library (128 KB of device memory, held by every GPU that loads the library
 * until the process exits) and allocates nothing.  It uses the lanes per
 * sample mesh_chamfer would use, or fewer when those blocks exceed the array:
 * the per-sample results are mesh_chamfer's bit for bit, and so are the two
 * means when the lanes agree (otherwise they differ only in the float64
 * summation order).
 *   - Limit: ceil(nSA/128) + ceil(nSB/128) <= 16384 blocks with one lane per
 *     sample (about 2M samples in total); larger inputs return
 *     MESH_ERR_WORKSPACE and launch nothing.
 *   - The first call on each device looks up that device's address of the
 *     array (cudaGetSymbolAddress, with that device current); make that first
 *     call before any stream capture.  The address is kept for the process's
 *     life: after a cudaDeviceReset the call must not be used again.
 *   - All calls share the array: calls that may overlap on the GPU (different
 *     streams, or concurrent threads) race and give wrong results; serialise
 *     them.  Each call clears the part that must start at zero itself.
 * Arguments and outputs are those of mesh_chamfer. */
mesh_status mesh_chamfer_noalloc(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                                 const mesh_bvh *B, const float *d_SB, int64_t nSB,
                                 double *d_out, int32_t *d_faceA, float *d_baryA, float *d_dist2A,
                                 int32_t *d_faceB, float *d_baryB, float *d_dist2B, void *stream);

/* ---------------------------------------------------------------- */
/* Gradients (nearest face and weights held fixed: envelope theorem) */
/* ---------------------------------------------------------------- */

/* Given dL/d(dist2) per query (d_g [nQ]) and the forward face / bary:
 *   dL/dq   = 2 g (q - c)                 -> d_gQ [nQ][3] (written; may be NULL)
 *   dL/dv_j = -2 g b_j (q - c)            -> d_gV [nV][3] (accumulated; may be NULL)
 * with c = sum_j b_j v_j on the current vertex buffer.  face -1 contributes 0. */
mesh_status mesh_closest_point_backward(const mesh_bvh *bvh, const float *d_Q, int64_t nQ,
                                        const int32_t *d_face, const float *d_bary,
                                        const float *d_g, float *d_gQ, float *d_gV,
                                        void *stream);

/* Reverse mode of mesh_chamfer (Sec. 4.2's Chamfer distance as a loss), both
 * directions in one launch.  d_g: DEVICE float64 [2] = dL/d(out[0]), dL/d(out[1])
 * (read on the device: no host synchronisation).  With the forward's per-sample
 * faces and weights (d_faceA / d_baryA: SA's nearest faces on mesh B; d_faceB /
 * d_baryB: SB's on mesh A) and each mesh's current vertex buffer, every sample of
 * SA carries dL/d(dist2) = g[0] / nSA and every sample of SB g[1] / nSB:
 *   dL/dSA[i] =  2 (g[0]/nSA) (a_i - c_i)           -> d_gSA [nSA][3] (written)
 *   dL/dV_B  += -2 (g[0]/nSA) b_ij (a_i - c_i)       -> d_gVB [nVB][3] (accumulated)
 *   dL/dSB[i] =  2 (g[1]/nSB) (b_i - c_i)           -> d_gSB [nSB][3] (written)
 *   dL/dV_A  += -2 (g[1]/nSB) b_ij (b_i - c_i)       -> d_gVA [nVA][3] (accumulated)
 * c_i = sum_j b_ij v_j, the nearest face and weights held fixed (envelope
 * theorem).  Any gradient output may be NULL; a direction whose outputs are
 * both NULL is skipped.  Face -1 contributes 0; a face id out of range sets
 * MESH_DEV_INDEX_RANGE on the mesh it indexes and contributes 0. */
mesh_status mesh_chamfer_backward(const mesh_bvh *A, const float *d_SA, int64_t nSA,
                                  const mesh_bvh *B, const float *d_SB, int64_t nSB,
                                  const double *d_g, const int32_t *d_faceA, const float *d_baryA,
                                  const int32_t *d_faceB, const float *d_baryB, float *d_gSA,
                                  float *d_gVA, float *d_gSB, float *d_gVB, void *stream);

/* dL/dV += sum_i b_ij dL/dp_i over the vertices of face[i] (d_gV accumulated). */
mesh_status mesh_interpolate_backward(const mesh_bvh *bvh, const int32_t *d_face,
                                      const float *d_bary, int64_t n, const float *d_gP,
                                      float *d_gV, void *stream);

/* Reverse mode of mesh_bind_gaussians with respect to vertex positions:
 * d_gmu [nG][3], d_gquat [nG][4], d_gscale [nG][3] (any may be NULL = 0);
 * dL/dV accumulated into d_gV [nV][3]. */
mesh_status mesh_bind_gaussians_backward(const mesh_bvh *bvh, const int32_t *d_gface,
                                         const float *d_gbary, const float *d_goff, int64_t nG,
                                         const float *d_gmu, const float *d_gquat,
                                         const float *d_gscale, float *d_gV, void *stream);

/* ---------------------------------------------------------------- */
/* Batched forms: many independent scenes in one storage block       */
/* ---------------------------------------------------------------- */
/* Scenes are concatenated: vertices [nV][3] with device offsets vert_off
 * [B+1], faces [nF][3] holding SCENE-LOCAL vertex indices with face_off [B+1]
 * (int32, non-decreasing, off[0] = 0, off[B] = total; empty scenes allowed).
 * Each scene gets its own LBVH, identical to the one mesh_build_lbvh builds for
 * that scene alone, but every phase runs as one launch over all scenes, and
 * queries / Gaussians of all scenes go through one persistent launch (warps
 * pull work in chunks from a counter), so per-scene launch overhead vanishes
 * and the whole frame can be captured in one CUDA graph. */
typedef struct mesh_batch mesh_batch;

typedef struct {
    int64_t n_scenes, n_verts, n_faces, max_scenes, max_verts, max_faces;
    size_t off_scene;        /* per scene: float4 root_lo, float4 root_hi            */
    size_t off_status;       /* uint32 status, uint32 n_degenerate, uint32 work counter */
    size_t off_vert_off;     /* int32 [max_scenes + 1] copy of vert_off              */
    size_t off_face_off;     /* int32 [max_scenes + 1] copy of face_off              */
    size_t off_verts;        /* float4 [max_verts]                                   */
    size_t off_faces;        /* int4 [max_faces]  GLOBAL vertex indices, .w = scene    */
    size_t off_keys;         /* uint32 [max_faces] Morton keys, leaf order per scene  */
    size_t off_perm;         /* int32 [max_faces]  global face id of leaf (face_off[s] + j) */
    size_t off_nodes;        /* 64 B records; scene s's internal node i at face_off[s] + i */
    size_t off_parent_int;   /* int32 [max_faces]  2 * local parent + side, -1 at a root  */
    size_t off_parent_leaf;  /* int32 [max_faces]                                        */
    size_t off_tris;         /* 48 B per leaf, global leaf order                          */
    size_t off_flags;        /* uint32 [max_faces]                                        */
    size_t storage_bytes;
} mesh_batch_layout;

size_t mesh_batch_storage_bytes(int64_t max_scenes, int64_t max_verts, int64_t max_faces);
size_t mesh_batch_workspace_bytes(int64_t max_scenes, int64_t max_faces);
mesh_status mesh_batch_create(void *d_storage, size_t storage_bytes, int64_t max_scenes,
                              int64_t max_verts, int64_t max_faces, mesh_batch **out);
void mesh_batch_destroy(mesh_batch *batch);
mesh_status mesh_batch_get_layout(const mesh_batch *batch, mesh_batch_layout *out);

/* Build all scenes' LBVHs (one launch per phase for the whole batch). */
mesh_status mesh_batch_build(mesh_batch *batch, int64_t n_scenes, const float *d_V,
                             const int32_t *d_vert_off, int64_t nV, const int32_t *d_F,
                             const int32_t *d_face_off, int64_t nF, void *d_ws, size_t ws_bytes,
                             void *stream);

/* Vertex-buffer update [nV][3] (same offsets) and refit of every scene. */
mesh_status mesh_batch_refit(mesh_batch *batch, const float *d_V, int64_t nV, void *stream);

/* Closest point for queries of every scene: query i belongs to scene s with
 * query_off[s] <= i < query_off[s+1] (device, int32 [B+1]).  Outputs as
 * mesh_closest_point, face ids SCENE-LOCAL.  One persistent launch. */
mesh_status mesh_batch_closest_point(mesh_batch *batch, const float *d_Q,
                                     const int32_t *d_query_off, int64_t nQ, float max_dist,
                                     int32_t *d_face, float *d_bary, float *d_point,
                                     float *d_dist2, void *stream);

/* Face-bound Gaussians of every scene: Gaussian g belongs to scene s with
 * gauss_off[s] <= g < gauss_off[s+1]; d_gface holds SCENE-LOCAL face ids.
 * Formula and outputs as mesh_bind_gaussians. */
mesh_status mesh_batch_bind_gaussians(mesh_batch *batch, const int32_t *d_gface,
                                      const int32_t *d_gauss_off, const float *d_gbary,
                                      const float *d_goff, int64_t nG, float *d_mu,
                                      float *d_quat, float *d_scale, void *stream);

/* Read and clear the batch's device status bits (as mesh_bvh_status). */
mesh_status mesh_batch_status(mesh_batch *batch, uint32_t *bits, uint32_t *n_degenerate,
                              void *stream);

/* ---------------------------------------------------------------- */
/* Status and diagnostics                                            */
/* ---------------------------------------------------------------- */

/* Synchronise `stream`, read and clear the BVH's device status bits into
 * *bits (may be NULL) and the count of degenerate Gaussians seen into
 * *n_degenerate (may be NULL).  Returns MESH_ERR_DEVICE if an error bit
 * (anything but MESH_DEV_DEGENERATE and MESH_DEV_DEEP_TREE) was set, else
 * MESH_OK. */
mesh_status mesh_bvh_status(mesh_bvh *bvh, uint32_t *bits, uint32_t *n_degenerate, void *stream);

const char *mesh_status_string(mesh_status s);

/* L2 read-bandwidth probe (the roofline denominator of the traversal kernels,
 * whose trees stay resident in L2): reads the first `bytes` of d_buf (16-byte
 * aligned, a multiple of 16; choose a size well inside L2, e.g. 48 MB) `passes`
 * times with L2-only loads from a grid of four 256-thread blocks per SM, and
 * writes one word per thread to d_sink (mesh_probe_sink_bytes() bytes).  Time
 * it with CUDA events after one warm-up call: bytes x passes / time is the
 * sustained L2 read bandwidth.  Not part of the method; a measurement aid. */
size_t mesh_probe_sink_bytes(void);
mesh_status mesh_probe_l2_read(const void *d_buf, size_t bytes, int passes, void *d_sink,
                               size_t sink_bytes, void *stream);

/* Number of kernels this library has launched in the process so far. */
uint64_t mesh_launch_count(void);

/* The device address of page-locked host memory (cudaHostAlloc / pinned),
 * so that an entry point can read its inputs from, or write its outputs to,
 * host memory directly: on a Grace-Blackwell node the kernel's loads and
 * stores then cross NVLink-C2C while it runs, with no separate copy (e.g.
 * mesh_contact writing each step's faces and distances where the host reads
 * them).  Host-only call; MESH_ERR_INVALID_ARG for NULL arguments,
 * MESH_ERR_CUDA when the memory is not page-locked host memory. */
mesh_status mesh_mapped_pointer(const void *host, void **device);

#ifdef __cplusplus
}
#endif
#endif /* MESHGS_H */
