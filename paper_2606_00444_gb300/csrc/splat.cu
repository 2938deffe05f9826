// Gaussian-splatting render of the face-bound Gaussians (Sec. 3.2's R_render),
// by the forward equations of 3D Gaussian splatting (Kerbl et al. 2023) into a
// headless device image.  Pipeline: (1) per Gaussian, project the centre,
// the 2D covariance J Rc Sigma Rc^T J^T + 0.3 I and its inverse (the conic),
// a 3-sigma radius and the rectangle of 16 x 16-pixel tiles it touches;
// (2) a stable radix sort of the Gaussians by depth (ties by index) and an
// exclusive scan of their tile counts in that order give each its slots;
// (3) one (tile, Gaussian) instance per touched tile, in depth order; (4) a
// stable radix sort of the instances by tile, so each tile's instances are
// contiguous and front to back; (5) each tile's range; (6) one block
// of 16 x 16 threads per tile, the tiles with the most instances first,
// composites its pixels front to back, the instances streamed through shared
// memory 256 at a time, until every pixel's transmittance would fall below
// 1e-4; a warp (two rows of the tile) blends only the instances whose reach
// box meets its pixels (elsewhere an alpha is below 1/255 for certain), found
// 32 at a time with one vote.
//
// A pixel (px, py) samples the image point (px, py); u = fx x_c / z_c + cx.
// Per instance and pixel: p = -0.5 (a dx^2 + c dy^2) - b dx dy with
// d = (u - px, v - py); skip if p > 0; alpha = min(0.99, opacity e^p); skip
// if alpha < 1/255; stop if T (1 - alpha) < 1e-4; else C += color alpha T,
// T *= 1 - alpha.  Output: C + T background, and T.
#include <math.h>

#include "common.cuh"

namespace meshgs {

constexpr int kTile = 16;
constexpr int kTilePix = kTile * kTile;
constexpr int kScanBlock = 1024;

// reach: the box (x0, x1, y0, y1) in pixels outside which the Gaussian's alpha is
// below 1/255 for certain (its ellipse d^T conic d <= 2 ln(255 opacity), the bound
// grown by 1 % and half a pixel so that float32 rounding cannot shrink it past a
// pixel the per-pixel test would keep).
__global__ void k_gs_preprocess(int n, const float *__restrict__ mu, const float *__restrict__ quat,
                                const float *__restrict__ scale, const float *__restrict__ opac,
                                mesh_camera cam, int gx, int gy, float2 *uv, float4 *conic_o,
                                int4 *rect, int *count, float4 *reach, unsigned *gkey) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    count[g] = 0;
    gkey[g] = 0xffffffffu;                               // culled: after every drawn Gaussian
    const float *m = mu + 3 * (size_t)g;
    float xc[3];
    for (int r = 0; r < 3; ++r)
        xc[r] = cam.R[3 * r] * m[0] + cam.R[3 * r + 1] * m[1] + cam.R[3 * r + 2] * m[2] + cam.t[r];
    if (!(xc[2] > cam.near_z)) return;
    const float *q = quat + 4 * (size_t)g, *s = scale + 3 * (size_t)g;
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float qn = rsqrtf(w * w + x * x + y * y + z * z);
    w *= qn; x *= qn; y *= qn; z *= qn;
    float R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                     {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                     {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * s[j];
    float S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) S[i][j] = M[i][0] * M[j][0] + M[i][1] * M[j][1] + M[i][2] * M[j][2];
    // Rc S Rc^T
    float T1[3][3], Sc[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T1[i][j] = cam.R[3 * i] * S[0][j] + cam.R[3 * i + 1] * S[1][j] + cam.R[3 * i + 2] * S[2][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Sc[i][j] = T1[i][0] * cam.R[3 * j] + T1[i][1] * cam.R[3 * j + 1] + T1[i][2] * cam.R[3 * j + 2];
    float iz = 1.0f / xc[2];
    float J0[3] = {cam.fx * iz, 0.0f, -cam.fx * xc[0] * iz * iz};
    float J1[3] = {0.0f, cam.fy * iz, -cam.fy * xc[1] * iz * iz};
    float A0[3], A1[3];
    for (int j = 0; j < 3; ++j) {
        A0[j] = J0[0] * Sc[0][j] + J0[1] * Sc[1][j] + J0[2] * Sc[2][j];
        A1[j] = J1[0] * Sc[0][j] + J1[1] * Sc[1][j] + J1[2] * Sc[2][j];
    }
    float a = A0[0] * J0[0] + A0[1] * J0[1] + A0[2] * J0[2] + 0.3f;
    float b = A0[0] * J1[0] + A0[1] * J1[1] + A0[2] * J1[2];
    float c = A1[0] * J1[0] + A1[1] * J1[1] + A1[2] * J1[2] + 0.3f;
    float det = a * c - b * b;
    if (!(det > 0.0f)) return;
    float mid = 0.5f * (a + c);
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    int r = (int)ceilf(3.0f * sqrtf(lam));
    float u = cam.fx * xc[0] * iz + cam.cx, v = cam.fy * xc[1] * iz + cam.cy;
    int x0 = (int)((u - r) / (float)kTile), x1 = (int)((u + r + kTile - 1) / (float)kTile);
    int y0 = (int)((v - r) / (float)kTile), y1 = (int)((v + r + kTile - 1) / (float)kTile);
    x0 = min(max(x0, 0), gx); x1 = min(max(x1, 0), gx);
    y0 = min(max(y0, 0), gy); y1 = min(max(y1, 0), gy);
    int cnt = (x1 - x0) * (y1 - y0);
    if (cnt <= 0) return;
    float id = 1.0f / det;
    uv[g] = make_float2(u, v);
    conic_o[g] = make_float4(c * id, -b * id, a * id, opac[g]);
    rect[g] = make_int4(x0, y0, x1, y1);
    count[g] = cnt;
    gkey[g] = __float_as_uint(xc[2]);                    // positive: bit order is value order
    float k = 2.0f * logf(fmaxf(255.0f * opac[g], 1.0f));          // the ellipse's squared radius
    float rx = 1.01f * sqrtf(k * a) + 0.5f, ry = 1.01f * sqrtf(k * c) + 0.5f;
    reach[g] = make_float4(u - rx, u + rx, v - ry, v + ry);
}

// Exclusive scan of n ints: per-block scans, a scan of the block totals by one
// block, then the block offsets added.
__global__ void __launch_bounds__(kScanBlock) k_scan_local(int n, const int *in, int *out, int *bsum) {
    __shared__ int ws[32];
    int i = blockIdx.x * kScanBlock + threadIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = i < n ? in[i] : 0, x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = ws[lane], z = t;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        ws[lane] = z - t;
        if (lane == 31) bsum[blockIdx.x] = z;
    }
    __syncthreads();
    if (i < n) out[i] = x - v + ws[wid];
}

__global__ void __launch_bounds__(32) k_scan_sums(int nb, int *bsum, int *total) {
    int run = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        int b = b0 + threadIdx.x;
        int v = b < nb ? bsum[b] : 0, x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)threadIdx.x >= o) x += y;
        }
        if (b < nb) bsum[b] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (threadIdx.x == 0) *total = run;
}

__global__ void k_scan_add(int n, int *out, const int *bsum) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / kScanBlock];
}

void exclusive_scan_int(const int *in, int *out, int n, int *bsum, int *total, cudaStream_t s) {
    int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_local<<<nb, kScanBlock, 0, s>>>(n, in, out, bsum);
    k_scan_sums<<<1, 32, 0, s>>>(nb, bsum, total);
    k_scan_add<<<grid_for(n, 256), 256, 0, s>>>(n, out, bsum);
    count_launch(3);
}

// The instances of the Gaussians in depth order (sorted position i holds Gaussian
// gorder[i]; its instances start at offset[i]), so that a stable sort by tile
// leaves each tile's instances front to back.  Slots at or past cap are dropped.
__global__ void k_gs_duplicate(int n, const int *__restrict__ gorder, const int *__restrict__ offset,
                               const int *__restrict__ count, const int4 *__restrict__ rect, int gx, int cap,
                               unsigned *tile_key, int *gid) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = gorder[i];
    if (count[g] == 0) return;
    int4 r = rect[g];
    int k = offset[i];
    for (int ty = r.y; ty < r.w; ++ty)
        for (int tx = r.x; tx < r.z; ++tx, ++k) {
            if (k >= cap) return;
            tile_key[k] = (unsigned)(ty * gx + tx);
            gid[k] = g;
        }
}

// The tile counts in depth order, for the scan of the instance offsets.
__global__ void k_gs_gather_count(int n, const int *__restrict__ gorder, const int *__restrict__ count,
                                  int *__restrict__ count_s) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) count_s[i] = count[gorder[i]];
}

__global__ void k_gs_pad(int cap, const int *__restrict__ total, unsigned pad_tile, unsigned *tile_key, int *gid,
                         unsigned int *counts) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = *total;
    if (k == 0 && counts) {
        counts[0] = m > cap ? 1u : 0u;                 // overflow: instances were dropped
        counts[1] = (unsigned)m;
    }
    if (k >= cap || k < m) return;
    tile_key[k] = pad_tile;
    gid[k] = 0;
}

__global__ void k_gs_ranges_cap(int cap, int tiles, const unsigned *__restrict__ tk, int2 *range) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap) return;
    unsigned t = tk[i];
    if (t >= (unsigned)tiles) return;                  // a padding slot
    if (i == 0 || tk[i - 1] != t) range[t].x = i;
    if (i == cap - 1 || tk[i + 1] != t) range[t].y = i + 1;
}

__global__ void k_gs_ranges(int m, const unsigned *__restrict__ tk, int2 *range) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    unsigned t = tk[i];
    if (i == 0 || tk[i - 1] != t) range[t].x = i;
    if (i == m - 1 || tk[i + 1] != t) range[t].y = i + 1;
}

__global__ void __launch_bounds__(kTilePix)
k_gs_render(mesh_camera cam, int gx, const int *__restrict__ order, const int2 *__restrict__ range,
            const int *__restrict__ inst, const int *__restrict__ gid, const float2 *__restrict__ uv,
            const float4 *__restrict__ conic_o, const float4 *__restrict__ reach,
            const float *__restrict__ color, float *image, float *trans) {
    __shared__ float2 s_uv[kTilePix];
    __shared__ float4 s_co[kTilePix];
    __shared__ float4 s_col[kTilePix];
    __shared__ float4 s_reach[kTilePix];
    const int tile = order[blockIdx.x];                     // the heaviest tiles first
    const int tx = tile % gx, ty = tile / gx;
    const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
    const bool inside = px < cam.width && py < cam.height;
    bool done = !inside;
    // this warp's pixels: two rows of the tile
    const int lane = threadIdx.x & 31;
    const float wx0 = (float)(tx * kTile), wx1 = wx0 + (float)(kTile - 1);
    const float wy0 = (float)(ty * kTile + 2 * (threadIdx.x / 32)), wy1 = wy0 + 1.0f;
    const int2 rg = range[tile];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    for (int b0 = rg.x; b0 < rg.y; b0 += kTilePix) {
        if (__syncthreads_count(done) == kTilePix) break;
        int k = b0 + threadIdx.x;
        if (k < rg.y) {
            int g = gid[inst[k]];
            s_uv[threadIdx.x] = uv[g];
            s_co[threadIdx.x] = conic_o[g];
            s_col[threadIdx.x] = make_float4(color[3 * (size_t)g], color[3 * (size_t)g + 1], color[3 * (size_t)g + 2],
                                             0.0f);
            s_reach[threadIdx.x] = reach[g];
        }
        __syncthreads();
        int m = min(kTilePix, rg.y - b0);
        // 32 instances at a time: each lane tests one instance's reach box against the
        // warp's pixels, and the warp then blends only the instances that reach them, in
        // order (the others have alpha below 1/255 at every pixel of the warp)
        for (int j0 = 0; j0 < m; j0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const int jl = j0 + lane;
            bool reaches = false;
            if (jl < m) {
                const float4 rb = s_reach[jl];
                reaches = !(rb.y < wx0 || rb.x > wx1 || rb.w < wy0 || rb.z > wy1);
            }
            unsigned int todo = __ballot_sync(0xffffffffu, reaches);
            // two instances per step: their exponents do not depend on the blend, so
            // both are evaluated before the two blends (which stay in order)
            while (todo) {
                const int ja = j0 + __ffs(todo) - 1;
                todo &= todo - 1u;
                const int jb = todo ? j0 + __ffs(todo) - 1 : ja;
                const bool two = todo != 0u;
                todo &= todo - 1u;
                if (done) continue;
                const float2 ua = s_uv[ja], ub = s_uv[jb];
                const float4 ca = s_co[ja], cb = s_co[jb];
                const float dxa = ua.x - (float)px, dya = ua.y - (float)py;
                const float dxb = ub.x - (float)px, dyb = ub.y - (float)py;
                const float pa = -0.5f * (ca.x * dxa * dxa + ca.z * dya * dya) - ca.y * dxa * dya;
                const float pb = -0.5f * (cb.x * dxb * dxb + cb.z * dyb * dyb) - cb.y * dxb * dyb;
                const float ea = expf(pa), eb = expf(pb);
                if (!(pa > 0.0f)) {
                    const float alpha = fminf(0.99f, ca.w * ea);
                    if (alpha >= 1.0f / 255.0f) {
                        const float tt = T * (1.0f - alpha);
                        if (tt < 1e-4f) { done = true; continue; }
                        const float4 c = s_col[ja];
                        C0 += c.x * alpha * T;
                        C1 += c.y * alpha * T;
                        C2 += c.z * alpha * T;
                        T = tt;
                    }
                }
                if (two && !(pb > 0.0f)) {
                    const float alpha = fminf(0.99f, cb.w * eb);
                    if (alpha >= 1.0f / 255.0f) {
                        const float tt = T * (1.0f - alpha);
                        if (tt < 1e-4f) { done = true; continue; }
                        const float4 c = s_col[jb];
                        C0 += c.x * alpha * T;
                        C1 += c.y * alpha * T;
                        C2 += c.z * alpha * T;
                        T = tt;
                    }
                }
            }
        }
    }
    if (!inside) return;
    size_t o = (size_t)py * cam.width + px;
    image[3 * o] = C0 + T * cam.background[0];
    image[3 * o + 1] = C1 + T * cam.background[1];
    image[3 * o + 2] = C2 + T * cam.background[2];
    if (trans) trans[o] = T;
}

// Tile order for the compositing launch, the tiles with the most instances
// first (longest-first scheduling: the longest tiles start in the first wave
// instead of trailing the launch).  One block: a counting sort of the tiles by
// the bit length of their instance count, descending; within a bucket the order
// is that of the atomics (any order gives the same image: tiles are
// independent).
__global__ void __launch_bounds__(1024) k_gs_tile_order(int tiles, const int2 *__restrict__ range,
                                                       int *__restrict__ order) {
    __shared__ int s_cnt[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        int2 r = range[t];
        int len = r.y - r.x;
        int bucket = len > 0 ? 32 - __clz(len) : 0;        // 0 (empty) .. 32
        atomicAdd(&s_cnt[32 - bucket], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 33; ++b) { int c = s_cnt[b]; s_cnt[b] = run; run += c; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        int2 r = range[t];
        int len = r.y - r.x;
        int bucket = len > 0 ? 32 - __clz(len) : 0;
        order[atomicAdd(&s_cnt[32 - bucket], 1)] = t;
    }
}

struct SplatWs {
    float2 *uv;
    float4 *conic_o, *reach;
    int *torder;
    int4 *rect;
    int *count, *count_s, *offset, *bsum, *total;
    int2 *range;
    unsigned *gkey, *gkey_s;
    int *gorder;
    char *gsort_ws;                // the Gaussians' depth sort
    size_t base_bytes;
    // per instance
    unsigned *tile_key, *tk_s;
    int *gid, *inst;
    char *sort_ws;                 // the instances' tile sort
    size_t bytes;
};

static SplatWs splat_ws(void *ws, int64_t n, int64_t m, int64_t tiles) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    int64_t nn = n > 0 ? n : 1, mm = m > 0 ? m : 1, tt = tiles > 0 ? tiles : 1;
    size_t oUV = take(8 * nn), oCO = take(16 * nn), oR = take(16 * nn), oC = take(4 * nn),
           oCS = take(4 * nn), oO = take(4 * nn), oB = take(4 * ((nn + kScanBlock - 1) / kScanBlock) + 4),
           oT = take(16), oRg = take(8 * tt), oRe = take(16 * nn), oTo = take(4 * tt), oGK = take(4 * nn),
           oGS = take(4 * nn), oGO = take(4 * nn), oGW = take(sort_pairs_ws_bytes(nn));
    size_t base = off;
    size_t oTK = take(4 * mm), oTS = take(4 * mm), oG = take(4 * mm), oI = take(4 * mm),
           oS = take(sort_pairs_ws_bytes(mm));
    char *b = (char *)ws;
    SplatWs w;
    w.uv = (float2 *)(b + oUV); w.conic_o = (float4 *)(b + oCO);
    w.rect = (int4 *)(b + oR); w.count = (int *)(b + oC); w.count_s = (int *)(b + oCS); w.offset = (int *)(b + oO);
    w.bsum = (int *)(b + oB); w.total = (int *)(b + oT); w.range = (int2 *)(b + oRg);
    w.reach = (float4 *)(b + oRe); w.torder = (int *)(b + oTo);
    w.gkey = (unsigned *)(b + oGK); w.gkey_s = (unsigned *)(b + oGS); w.gorder = (int *)(b + oGO);
    w.gsort_ws = b + oGW;
    w.base_bytes = base;
    w.tile_key = (unsigned *)(b + oTK); w.tk_s = (unsigned *)(b + oTS);
    w.gid = (int *)(b + oG); w.inst = (int *)(b + oI);
    w.sort_ws = b + oS;
    w.bytes = off;
    return w;
}

// Steps (1) and (2): project, sort the Gaussians by depth (ties by index), and
// scan their tile counts in that order into instance offsets (total in w.total).
static void gs_front(const SplatWs &w, int n, const float *d_mu, const float *d_quat, const float *d_scale,
                     const float *d_opacity, const mesh_camera &cam, int gx, int gy, cudaStream_t s) {
    k_gs_preprocess<<<grid_for(n, 256), 256, 0, s>>>(n, d_mu, d_quat, d_scale, d_opacity, cam, gx, gy, w.uv,
                                                     w.conic_o, w.rect, w.count, w.reach, w.gkey);
    count_launch();
    sort_pairs_u32(w.gsort_ws, n, 32, w.gkey, nullptr, w.gkey_s, w.gorder, s);
    k_gs_gather_count<<<grid_for(n, 256), 256, 0, s>>>(n, w.gorder, w.count, w.count_s);
    int nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_local<<<nb, kScanBlock, 0, s>>>(n, w.count_s, w.offset, w.bsum);
    k_scan_sums<<<1, 32, 0, s>>>(nb, w.bsum, w.total);
    k_scan_add<<<grid_for(n, 256), 256, 0, s>>>(n, w.offset, w.bsum);
    count_launch(4);
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

size_t mesh_gs_workspace_bytes(int64_t nG, int64_t n_instances, int width, int height) {
    if (nG < 0 || n_instances < 0 || n_instances > INT32_MAX || width <= 0 || height <= 0) return 0;
    int64_t tiles = (int64_t)((width + kTile - 1) / kTile) * ((height + kTile - 1) / kTile);
    return splat_ws(nullptr, nG, n_instances, tiles).bytes;
}

mesh_status mesh_gs_render(const float *d_mu, const float *d_quat, const float *d_scale,
                           const float *d_opacity, const float *d_color, int64_t nG,
                           const mesh_camera *cam, void *d_ws, size_t ws_bytes, size_t *ws_needed,
                           float *d_image, float *d_trans, void *stream) {
    if (!cam || nG < 0 || nG > INT32_MAX || cam->width <= 0 || cam->height <= 0 || !d_image ||
        (nG > 0 && (!d_mu || !d_quat || !d_scale || !d_opacity || !d_color)) || !(cam->near_z > 0.0f))
        return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)nG;
    const int gx = (cam->width + kTile - 1) / kTile, gy = (cam->height + kTile - 1) / kTile;
    const int64_t tiles = (int64_t)gx * gy;
    SplatWs w0 = splat_ws(d_ws, n, 0, tiles);
    if (ws_needed) *ws_needed = w0.bytes;
    if (!d_ws || ws_bytes < w0.base_bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    int m = 0;
    if (n > 0) {
        gs_front(w0, n, d_mu, d_quat, d_scale, d_opacity, *cam, gx, gy, s);
        if (cudaMemcpyAsync(&m, w0.total, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MESH_ERR_CUDA;
    }
    SplatWs w = splat_ws(d_ws, n, m, tiles);
    if (ws_needed) *ws_needed = w.bytes;
    if (ws_bytes < w.bytes) return MESH_ERR_WORKSPACE;
    cudaMemsetAsync(w.range, 0, 8 * (size_t)tiles, s);
    if (m > 0) {
        k_gs_duplicate<<<grid_for(n, 256), 256, 0, s>>>(n, w.gorder, w.offset, w.count, w.rect, gx, m, w.tile_key,
                                                        w.gid);
        count_launch();
        int bits = 1;
        while (((int64_t)1 << bits) < tiles) ++bits;
        sort_pairs_u32(w.sort_ws, m, bits, w.tile_key, nullptr, w.tk_s, w.inst, s);
        k_gs_ranges<<<grid_for(m, 256), 256, 0, s>>>(m, w.tk_s, w.range);
        count_launch();
    }
    k_gs_tile_order<<<1, 1024, 0, s>>>((int)tiles, w.range, w.torder);
    k_gs_render<<<(unsigned)tiles, kTilePix, 0, s>>>(*cam, gx, w.torder, w.range, w.inst, w.gid, w.uv, w.conic_o,
                                                     w.reach, d_color, d_image, d_trans);
    count_launch(2);
    return check_launch();
}

mesh_status mesh_gs_render_capacity(const float *d_mu, const float *d_quat, const float *d_scale,
                                    const float *d_opacity, const float *d_color, int64_t nG,
                                    const mesh_camera *cam, int64_t max_instances, void *d_ws,
                                    size_t ws_bytes, float *d_image, float *d_trans, uint32_t *d_counts,
                                    void *stream) {
    if (!cam || nG < 0 || nG > INT32_MAX || cam->width <= 0 || cam->height <= 0 || !d_image ||
        max_instances < 1 || max_instances > INT32_MAX ||
        (nG > 0 && (!d_mu || !d_quat || !d_scale || !d_opacity || !d_color)) || !(cam->near_z > 0.0f))
        return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)nG, cap = (int)max_instances;
    const int gx = (cam->width + kTile - 1) / kTile, gy = (cam->height + kTile - 1) / kTile;
    const int64_t tiles = (int64_t)gx * gy;
    SplatWs w = splat_ws(d_ws, n, cap, tiles);
    if (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    cudaMemsetAsync(w.range, 0, 8 * (size_t)tiles, s);
    cudaMemsetAsync(w.total, 0, sizeof(int), s);
    if (n > 0) {
        gs_front(w, n, d_mu, d_quat, d_scale, d_opacity, *cam, gx, gy, s);
        k_gs_duplicate<<<grid_for(n, 256), 256, 0, s>>>(n, w.gorder, w.offset, w.count, w.rect, gx, cap, w.tile_key,
                                                        w.gid);
        count_launch();
    }
    // tile keys take `bits` bits with room above the last tile for the padding key
    int bits = 1;
    while (((int64_t)1 << bits) <= tiles) ++bits;
    const unsigned pad_tile = (unsigned)(((int64_t)1 << bits) - 1);
    k_gs_pad<<<grid_for(cap, 256), 256, 0, s>>>(cap, w.total, pad_tile, w.tile_key, w.gid, d_counts);
    count_launch();
    sort_pairs_u32(w.sort_ws, cap, bits, w.tile_key, nullptr, w.tk_s, w.inst, s);
    k_gs_ranges_cap<<<grid_for(cap, 256), 256, 0, s>>>(cap, (int)tiles, w.tk_s, w.range);
    count_launch();
    k_gs_tile_order<<<1, 1024, 0, s>>>((int)tiles, w.range, w.torder);
    k_gs_render<<<(unsigned)tiles, kTilePix, 0, s>>>(*cam, gx, w.torder, w.range, w.inst, w.gid, w.uv, w.conic_o,
                                                     w.reach, d_color, d_image, d_trans);
    count_launch(2);
    return check_launch();
}

}  // extern "C"
