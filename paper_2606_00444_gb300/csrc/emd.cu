// Earth Mover's Distance between two equal-size point sets (the EMD of
// Sec. 4.2, on 10K points sampled from each mesh): the minimum over bijections
// of the mean Euclidean distance, by Bertsekas's auction algorithm with
// epsilon scaling (Jacobi form: every unassigned point bids at once).  Each
// phase ends with every point assigned and prices epsilon-complementary, so
// the final assignment costs at most n * eps_final more than the optimum: the
// mean is within eps_final of the exact EMD.
//
// Bid kernel: one warp per unassigned point of A; the points of B and their
// prices are streamed through shared memory in tiles; each lane keeps the best
// and second-best value (-distance - price) and the warp merges them; the bid
// (price + best - second + eps) goes to the object with a 64-bit atomic max of
// (bid bits, bidder) -- bids are positive floats, so their bits order like
// the values, and equal bids resolve to the higher bidder id.  Resolve kernel:
// one thread per object with a bid moves the object to the winner and frees
// its previous owner.  The host runs the iterations, reading the count of
// unassigned points every 16 iterations; the call returns when done.
#include <math.h>

#include <cstring>

#include "common.cuh"

namespace meshgs {

constexpr int kEmdBlock = 256;
constexpr int kEmdWarps = kEmdBlock / 32;
constexpr int kEmdTile = 1024;
constexpr int kEmdCheck = 16;

__device__ __forceinline__ unsigned f2ord_emd(float f) {
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f_emd(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_emd_init(const float *__restrict__ A, const float *__restrict__ B, int n, float4 *A4,
                           float4 *B4, float *price, int *owner, int *assign, unsigned long long *bids,
                           unsigned *box) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a = make_float4(A[3 * i], A[3 * i + 1], A[3 * i + 2], 0.0f);
    float4 b = make_float4(B[3 * i], B[3 * i + 1], B[3 * i + 2], 0.0f);
    A4[i] = a;
    B4[i] = b;
    price[i] = 0.0f;
    owner[i] = -1;
    assign[i] = -1;
    bids[i] = 0ull;
    atomicMin(&box[0], f2ord_emd(fminf(a.x, b.x)));
    atomicMin(&box[1], f2ord_emd(fminf(a.y, b.y)));
    atomicMin(&box[2], f2ord_emd(fminf(a.z, b.z)));
    atomicMax(&box[3], f2ord_emd(fmaxf(a.x, b.x)));
    atomicMax(&box[4], f2ord_emd(fmaxf(a.y, b.y)));
    atomicMax(&box[5], f2ord_emd(fmaxf(a.z, b.z)));
}

__global__ void k_emd_unassign(int n, int *owner, int *assign) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    owner[i] = -1;
    assign[i] = -1;
}

// (best, second best) of a lane merged with another lane's
__device__ __forceinline__ void merge2(float &b1, int &j1, float &b2, float o1, int oj, float o2) {
    if (o1 > b1 || (o1 == b1 && oj < j1)) {
        b2 = fmaxf(b1, o2);
        b1 = o1;
        j1 = oj;
    } else {
        b2 = fmaxf(b2, o1);
    }
}

__global__ void __launch_bounds__(kEmdBlock)
k_emd_bid(int n, const float4 *__restrict__ A4, const float4 *__restrict__ B4, const float *__restrict__ price,
          const int *__restrict__ assign, unsigned long long *bids, float eps, unsigned *active) {
    __shared__ float4 sb[kEmdTile];
    __shared__ float sp[kEmdTile];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * kEmdWarps + wid;
    const bool mine = i < n && assign[i] < 0;
    if (!__syncthreads_or(mine)) return;
    float4 a = mine ? A4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    float b1 = -INFINITY, b2 = -INFINITY;
    int j1 = 0x7fffffff;
    for (int t0 = 0; t0 < n; t0 += kEmdTile) {
        int m = min(kEmdTile, n - t0);
        for (int t = threadIdx.x; t < m; t += kEmdBlock) {
            sb[t] = B4[t0 + t];
            sp[t] = price[t0 + t];
        }
        __syncthreads();
        if (mine) {
            for (int t = lane; t < m; t += 32) {
                float4 b = sb[t];
                float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
                float v = -sqrtf(dx * dx + dy * dy + dz * dz) - sp[t];
                merge2(b1, j1, b2, v, t0 + t, -INFINITY);
            }
        }
        __syncthreads();
    }
    if (!mine) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float o1 = __shfl_xor_sync(0xffffffffu, b1, o), o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        merge2(b1, j1, b2, o1, oj, o2);
    }
    if (lane == 0) {
        atomicAdd(active, 1u);
        float inc = (b2 == -INFINITY ? 0.0f : b1 - b2) + eps;
        float bid = price[j1] + inc;
        atomicMax(&bids[j1], ((unsigned long long)__float_as_uint(bid) << 32) | (unsigned)i);
    }
}

__global__ void k_emd_resolve(int n, float *price, int *owner, int *assign, unsigned long long *bids) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    unsigned long long b = bids[j];
    if (b == 0ull) return;
    bids[j] = 0ull;
    int winner = (int)(b & 0xffffffffull);
    int old = owner[j];
    if (old >= 0) assign[old] = -1;
    owner[j] = winner;
    assign[winner] = j;
    price[j] = __uint_as_float((unsigned)(b >> 32));
}

// Gauss-Seidel tail: once few points are unassigned, one block finishes the
// phase, one bid at a time, with the other set and its prices held in shared
// memory (n <= kTailMaxN): the unassigned points are queued in index order,
// each bid is a block-wide scan for the best and second-best object, and an
// evicted owner joins the back of the queue.  At most max_bids bids; *active
// gets the points still queued.
constexpr int kTailThreads = 1024;
constexpr int kTailQueue = 256;

__device__ __forceinline__ void block_best2(float &b1, int &j1, float &b2, float *r1, float *r2, int *rj) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float o1 = __shfl_xor_sync(0xffffffffu, b1, o), o2 = __shfl_xor_sync(0xffffffffu, b2, o);
        int oj = __shfl_xor_sync(0xffffffffu, j1, o);
        merge2(b1, j1, b2, o1, oj, o2);
    }
    if (lane == 0) { r1[wid] = b1; r2[wid] = b2; rj[wid] = j1; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        b1 = lane < nw ? r1[lane] : -INFINITY;
        b2 = lane < nw ? r2[lane] : -INFINITY;
        j1 = lane < nw ? rj[lane] : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float o1 = __shfl_xor_sync(0xffffffffu, b1, o), o2 = __shfl_xor_sync(0xffffffffu, b2, o);
            int oj = __shfl_xor_sync(0xffffffffu, j1, o);
            merge2(b1, j1, b2, o1, oj, o2);
        }
        if (lane == 0) { r1[0] = b1; r2[0] = b2; rj[0] = j1; }
    }
    __syncthreads();
    b1 = r1[0]; b2 = r2[0]; j1 = rj[0];
    __syncthreads();
}

__global__ void __launch_bounds__(kTailThreads)
k_emd_tail(int n, const float4 *__restrict__ A4, const float4 *__restrict__ B4, float *price, int *owner,
           int *assign, float eps, int max_bids, unsigned *active) {
    extern __shared__ float4 tsm[];
    float4 *sB = tsm;
    float *sp = reinterpret_cast<float *>(sB + n);
    __shared__ int queue[kTailQueue];
    __shared__ float r1[32], r2[32];
    __shared__ int rj[32], s_cnt[32];
    __shared__ int s_len;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int j = tid; j < n; j += kTailThreads) { sB[j] = B4[j]; sp[j] = price[j]; }
    if (tid == 0) s_len = 0;
    __syncthreads();
    // unassigned points in index order (up to the queue's size)
    for (int c0 = 0; c0 < n; c0 += kTailThreads) {
        int i = c0 + tid;
        bool un = i < n && assign[i] < 0;
        unsigned ball = __ballot_sync(0xffffffffu, un);
        if (lane == 0) s_cnt[wid] = __popc(ball);
        __syncthreads();
        int before = s_len;
        for (int w = 0; w < wid; ++w) before += s_cnt[w];
        int pos = before + __popc(ball & ((1u << lane) - 1u));
        if (un && pos < kTailQueue) queue[pos] = i;
        __syncthreads();
        if (tid == 0) {
            int tot = s_len;
            for (int w = 0; w < (kTailThreads >> 5); ++w) tot += s_cnt[w];
            s_len = min(tot, kTailQueue);
        }
        __syncthreads();
    }
    int head = 0, len = s_len;
    for (int bids = 0; bids < max_bids && len > 0; ++bids) {
        const int i = queue[head % kTailQueue];
        const float4 a = A4[i];
        float b1 = -INFINITY, b2 = -INFINITY;
        int j1 = 0x7fffffff;
        for (int j = tid; j < n; j += kTailThreads) {
            float4 b = sB[j];
            float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
            merge2(b1, j1, b2, -sqrtf(dx * dx + dy * dy + dz * dz) - sp[j], j, -INFINITY);
        }
        block_best2(b1, j1, b2, r1, r2, rj);
        int old = owner[j1];                          // read by every thread, written by thread 0 below
        __syncthreads();
        if (tid == 0) {
            sp[j1] += (b2 == -INFINITY ? 0.0f : b1 - b2) + eps;
            owner[j1] = i;
            assign[i] = j1;
            if (old >= 0) {
                assign[old] = -1;
                queue[(head + len) % kTailQueue] = old;
            }
        }
        ++head;
        if (old < 0) --len;
        __syncthreads();
    }
    for (int j = tid; j < n; j += kTailThreads) price[j] = sp[j];
    if (tid == 0) *active = (unsigned)len;
}

// Mean cost of the assignment in float64, summed in a fixed order.
__global__ void __launch_bounds__(kEmdBlock)
k_emd_cost(int n, const float4 *__restrict__ A4, const float4 *__restrict__ B4, const int *__restrict__ assign,
           int *out_assign, double *partial, unsigned *ticket, double *out) {
    __shared__ double red[kEmdWarps];
    __shared__ bool last;
    int i = blockIdx.x * kEmdBlock + threadIdx.x;
    double c = 0.0;
    if (i < n) {
        int j = assign[i];
        if (out_assign) out_assign[i] = j;
        float4 a = A4[i], b = B4[j];
        double dx = (double)a.x - b.x, dy = (double)a.y - b.y, dz = (double)a.z - b.z;
        c = sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kEmdWarps; ++w) s += red[w];
        partial[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double s = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partial + k);
    out[0] = s / (double)n;
    *ticket = 0u;
}

struct EmdWs {
    float4 *A4, *B4;
    float *price;
    int *owner, *assign;
    unsigned long long *bids;
    unsigned *box, *active, *ticket;
    double *partial;
    size_t bytes;
};

static EmdWs emd_ws(void *ws, int64_t n) {
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off = align_up(off + b, 256); return o; };
    int64_t m = n > 0 ? n : 1;
    size_t oA = take(16 * m), oB = take(16 * m), oP = take(4 * m), oO = take(4 * m), oS = take(4 * m),
           oBid = take(8 * m), oBox = take(64), oPart = take(8 * (size_t)((m + kEmdBlock - 1) / kEmdBlock));
    char *b = (char *)ws;
    EmdWs w;
    w.A4 = (float4 *)(b + oA);
    w.B4 = (float4 *)(b + oB);
    w.price = (float *)(b + oP);
    w.owner = (int *)(b + oO);
    w.assign = (int *)(b + oS);
    w.bids = (unsigned long long *)(b + oBid);
    w.box = (unsigned *)(b + oBox);
    w.active = w.box + 8;
    w.ticket = w.box + 9;
    w.partial = (double *)(b + oPart);
    w.bytes = off;
    return w;
}

}  // namespace meshgs

using namespace meshgs;

extern "C" {

size_t mesh_emd_workspace_bytes(int64_t n) {
    if (n < 0 || n > ((int64_t)1 << 26)) return 0;
    return emd_ws(nullptr, n).bytes;
}

mesh_status mesh_emd(const float *d_A, const float *d_B, int64_t n, float eps_rel, int64_t max_iters,
                     void *d_ws, size_t ws_bytes, double *d_out, int32_t *d_assign, int64_t *iters_out,
                     void *stream) {
    if (n < 0 || n > ((int64_t)1 << 26) || !d_out || (n > 0 && (!d_A || !d_B)) || !(eps_rel > 0.0f) ||
        max_iters < 1)
        return MESH_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        cudaMemsetAsync(d_out, 0, sizeof(double), s);
        if (iters_out) *iters_out = 0;
        return check_launch();
    }
    EmdWs w = emd_ws(d_ws, n);
    if (!d_ws || ws_bytes < w.bytes || ((uintptr_t)d_ws & 255u)) return MESH_ERR_WORKSPACE;
    const int N = (int)n;
    unsigned init_box[10] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (cudaMemcpyAsync(w.box, init_box, sizeof(init_box), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MESH_ERR_CUDA;
    k_emd_init<<<grid_for(N, 256), 256, 0, s>>>(d_A, d_B, N, w.A4, w.B4, w.price, w.owner, w.assign, w.bids,
                                               w.box);
    count_launch();
    unsigned hb[6];
    if (cudaMemcpyAsync(hb, w.box, sizeof(hb), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MESH_ERR_CUDA;
    auto dec = [](unsigned u) {
        unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
        float f;
        memcpy(&f, &b, 4);
        return (double)f;
    };
    double dx = dec(hb[3]) - dec(hb[0]), dy = dec(hb[4]) - dec(hb[1]), dz = dec(hb[5]) - dec(hb[2]);
    double C = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(C > 0.0)) C = 1.0;
    const double eps_final = eps_rel * C;
    const unsigned bid_grid = grid_for(N, kEmdWarps);
    static int64_t tail_max = -1;                    // largest n whose set fits the tail's shared memory
    auto tail_smem = [](int m) { return (size_t)m * (sizeof(float4) + sizeof(float)); };
    if (tail_max < 0) {
        int dev = 0, optin = 0;
        tail_max = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            optin > 4096 && cudaFuncSetAttribute(k_emd_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 optin - 4096) == cudaSuccess)
            tail_max = (optin - 4096) / (int64_t)(sizeof(float4) + sizeof(float));
        cudaGetLastError();
    }
    int64_t iters = 0;
    for (double eps = C / 10.0;; eps /= 8.0) {
        if (eps < eps_final) eps = eps_final;
        k_emd_unassign<<<grid_for(N, 256), 256, 0, s>>>(N, w.owner, w.assign);
        count_launch();
        bool done = false;
        while (!done) {
            for (int k = 0; k < kEmdCheck; ++k) {
                cudaMemsetAsync(w.active, 0, sizeof(unsigned), s);
                k_emd_bid<<<bid_grid, kEmdBlock, 0, s>>>(N, w.A4, w.B4, w.price, w.assign, w.bids, (float)eps,
                                                         w.active);
                k_emd_resolve<<<grid_for(N, 256), 256, 0, s>>>(N, w.price, w.owner, w.assign, w.bids);
                count_launch(2);
                ++iters;
            }
            unsigned act = 0;
            if (cudaMemcpyAsync(&act, w.active, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return MESH_ERR_CUDA;
            done = act == 0;
            if (!done && act <= (unsigned)kTailQueue && n <= tail_max) {
                int64_t left = max_iters > iters ? max_iters - iters : 1;
                int cap = (int)(left < (int64_t)(1 << 24) ? left : (int64_t)(1 << 24));
                k_emd_tail<<<1, kTailThreads, tail_smem(N), s>>>(N, w.A4, w.B4, w.price, w.owner, w.assign,
                                                                 (float)eps, cap, w.active);
                count_launch();
                if (cudaMemcpyAsync(&act, w.active, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return MESH_ERR_CUDA;
                done = act == 0;
                iters += 1;
            }
            if (!done && iters >= max_iters) {
                if (iters_out) *iters_out = iters;
                return MESH_ERR_DEVICE;
            }
        }
        if (eps <= eps_final) break;
    }
    cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), s);
    k_emd_cost<<<grid_for(N, kEmdBlock), kEmdBlock, 0, s>>>(N, w.A4, w.B4, w.assign, d_assign, w.partial,
                                                           w.ticket, d_out);
    count_launch();
    if (iters_out) *iters_out = iters;
    return check_launch();
}

}  // extern "C"
