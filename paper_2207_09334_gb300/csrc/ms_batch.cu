// ms_batch.cu -- batched voxel-robot populations: one persistent launch
// advances thousands of independent robots of uneven size.
//
// Each robot is small (at most 4096 masses), so its whole state lives in
// shared memory for the length of the run: positions+inverse mass, velocity
// and the force accumulator, 48 bytes per mass.  Spring records stay in
// global memory and are re-read every step from L2: sliced-ELL rows (32
// masses per slice, robot-local mass indices) in which every mass lists all
// of its springs, both directions, one slot per lattice direction, so the
// force sum is one pass of coalesced loads with no dependent back-reference
// gathers, and a warp's partner reads from shared memory rarely collide in
// a bank.  (The robot-by-robot loop
// and the adjoint use the owner-row + back-reference layout.)  A step is
// two phases separated by a barrier: every mass gathers its spring forces
// from the shared-memory state at t_n (Jacobi, like the paper's grid-wide
// synchronisation in Algorithm 1), then every mass integrates in place.
//
// Schedules share one kernel (CTAs of 512 or 1024 threads):
//   block-per-robot  all threads of a CTA work on one robot (__syncthreads);
//   pair / quad      (1024-thread CTAs) two robots of at most 512 masses, or
//                    four of at most 256, one per half or quarter of the CTA,
//                    so that each mass has its own thread (named barriers);
//   warp-per-robot   each warp of a CTA owns a small robot (__syncwarp only).
// The CTAs are persistent: they pull work items (a robot, or a group of up to
// sixteen small robots (one per warp)) from a queue ordered by decreasing cost, and the
// choice of schedule per robot-size bucket is made by timing both
// (msb_autotune).  At the end of its item a CTA reduces the robot's centre of
// mass with warp shuffles and writes the x-travel.
#include "ms_voxel.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <vector>

namespace ms {
namespace {

// CTA size of the persistent kernel: 512 or 1024 threads (msb_autotune times
// both on the population and keeps the faster; msb_set_threads sets one).  A
// block item has the whole CTA; a warp item holds one robot per warp.
constexpr int kBatchThreadsDefault = 512;
constexpr int kComThreads = 256;    // k_com_travel
constexpr int kWarpModeMax = 256;   // robots up to this many masses may run warp-per-robot
constexpr int kPairMax = 512;       // block robots up to this many masses run two per 1024-thread CTA
constexpr int kQuadMax = 256;       // ... and up to this many, four per 1024-thread CTA

struct BatchArgs {
    const RobotDev *robots;
    const int4 *items;     // (x, count, mode, cost): mode 0 = block (x = robot),
                           // mode 1 = warp (robots wlist[x .. x+count)),
                           // mode 2 = pair, 3 = quad (robots wlist[x .. x+count): one per
                           // half / quarter of a 1024-thread CTA)
    const int *wlist;
    int n_items;
    int *queue;            // next item (zeroed before each launch)
    float4 *st;            // population state, 2 float4 per mass
    AllRows rows;
    Env env;
    const float2 *sc;      // (sin, cos)(2 pi f t_n) per step of this run
    int nsteps;
    int warp_cap;          // masses per warp region in warp mode
    int pair_cap;          // masses per half in a pair item (1024-thread CTAs)
    int quad_cap;          // masses per quarter in a quad item
    float *travel;         // per robot
    int *err;
};

// Barrier of the NT threads that work on one robot: the whole CTA
// (BAR = 0), or a half or a quarter of it (named barrier BAR, for a pair or
// quad item).
template <int NT, int BAR>
__device__ __forceinline__ void group_sync()
{
    if (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// All steps of one robot by a group of NT threads (t = 0 .. NT-1 within the
// group), its state and forces in xs, vs, fs (shared memory); red holds
// NT / 32 pairs of warp partial sums for the centre-of-mass travel.
template <int NT, int BAR>
__device__ __forceinline__ void run_robot(const BatchArgs &a, int r, int t, float4 *xs, float4 *vs, float4 *fs,
                                          float *red0, float *red1)
{
    const RobotDev R = a.robots[r];
    const int n = R.n;
    const float4 *g = a.st + 2 * R.mass_base;
    for (int i = t; i < n; i += NT) { xs[i] = g[2 * i]; vs[i] = g[2 * i + 1]; }
    group_sync<NT, BAR>();
    for (int step = 0; step < a.nsteps; ++step) {
        const float2 sc = __ldg(&a.sc[step]);
        for (int i = t; i < n; i += NT)
            fs[i] = robot_force_all<4>(a.rows, R.slice_base, i, xs, vs, sc.x, sc.y);
        group_sync<NT, BAR>();
        for (int i = t; i < n; i += NT) {
            float4 x = xs[i], v = vs[i];
            robot_integrate(a.env, x, v, fs[i]);
            xs[i] = x; vs[i] = v;
        }
        group_sync<NT, BAR>();
    }
    float mx = 0.f, m = 0.f;
    bool bad = false;
    for (int i = t; i < n; i += NT) {
        const float4 x = xs[i], v = vs[i];
        float4 *gw = a.st + 2 * R.mass_base;
        gw[2 * i] = x; gw[2 * i + 1] = v;
        if (x.w > 0.f) { const float mi = 1.0f / x.w; mx += mi * x.x; m += mi; }
        bad |= !isfinite(x.x + x.y + x.z + v.x + v.y + v.z);
    }
    const int w = t >> 5, lane = t & 31;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonFinite);
    mx = warp_sum(mx); m = warp_sum(m);
    if (lane == 0) { red0[w] = mx; red1[w] = m; }
    group_sync<NT, BAR>();
    if (t == 0) {
        float smx = 0.f, sm = 0.f;
        for (int q = 0; q < NT / 32; ++q) { smx += red0[q]; sm += red1[q]; }
        a.travel[r] = smx / sm - R.com0_x;
    }
}

template <int T>
__global__ void __launch_bounds__(T, 65536 / (64 * T)) k_batch(const BatchArgs a)
{
    extern __shared__ float4 smem[];
    __shared__ int item_sh;
    __shared__ float red_sh[2][T / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (;;) {
        if (tid == 0) item_sh = atomicAdd(a.queue, 1);
        __syncthreads();
        const int it = item_sh;
        __syncthreads();
        if (it >= a.n_items) break;
        const int4 item = a.items[it];

        if (item.z == 0) {
            // ---------------- block-per-robot ----------------
            const int n = a.robots[item.x].n;
            run_robot<T, 0>(a, item.x, tid, smem, smem + n, smem + 2 * n, red_sh[0], red_sh[1]);
            __syncthreads();
        } else if (item.z == 2) {
            // ---------------- a pair of robots, one per half of the CTA ----------------
            if constexpr (T == 1024) {
                const int half = tid >> 9;
                if (half < item.y) {
                    const int r = a.wlist[item.x + half];
                    float4 *xs = smem + (size_t)half * 3 * a.pair_cap;
                    if (half == 0)
                        run_robot<512, 1>(a, r, tid & 511, xs, xs + a.pair_cap, xs + 2 * a.pair_cap, red_sh[0],
                                          red_sh[1]);
                    else
                        run_robot<512, 2>(a, r, tid & 511, xs, xs + a.pair_cap, xs + 2 * a.pair_cap,
                                          red_sh[0] + 16, red_sh[1] + 16);
                }
            }
            __syncthreads();
        } else if (item.z == 3) {
            // ---------------- four robots, one per quarter of the CTA ----------------
            if constexpr (T == 1024) {
                const int qr = tid >> 8;
                if (qr < item.y) {
                    const int r = a.wlist[item.x + qr];
                    float4 *xs = smem + (size_t)qr * 3 * a.quad_cap, *vs = xs + a.quad_cap, *fs = vs + a.quad_cap;
                    float *r0 = red_sh[0] + 8 * qr, *r1 = red_sh[1] + 8 * qr;
                    switch (qr) {
                    case 0: run_robot<256, 1>(a, r, tid & 255, xs, vs, fs, r0, r1); break;
                    case 1: run_robot<256, 2>(a, r, tid & 255, xs, vs, fs, r0, r1); break;
                    case 2: run_robot<256, 3>(a, r, tid & 255, xs, vs, fs, r0, r1); break;
                    default: run_robot<256, 4>(a, r, tid & 255, xs, vs, fs, r0, r1); break;
                    }
                }
            }
            __syncthreads();
        } else {
            // ---------------- warp-per-robot ----------------
            if (warp < item.y) {
                const int r = a.wlist[item.x + warp];
                const RobotDev R = a.robots[r];
                const int n = R.n;
                float4 *xs = smem + (size_t)warp * 3 * a.warp_cap, *vs = xs + a.warp_cap, *fs = vs + a.warp_cap;
                const float4 *g = a.st + 2 * R.mass_base;
                for (int i = lane; i < n; i += 32) { xs[i] = g[2 * i]; vs[i] = g[2 * i + 1]; }
                __syncwarp();
                for (int step = 0; step < a.nsteps; ++step) {
                    const float2 sc = __ldg(&a.sc[step]);
                    for (int i = lane; i < n; i += 32)
                        fs[i] = robot_force_all<4>(a.rows, R.slice_base, i, xs, vs, sc.x, sc.y);
                    __syncwarp();
                    for (int i = lane; i < n; i += 32) {
                        float4 x = xs[i], v = vs[i];
                        robot_integrate(a.env, x, v, fs[i]);
                        xs[i] = x; vs[i] = v;
                    }
                    __syncwarp();
                }
                float mx = 0.f, m = 0.f;
                bool bad = false;
                for (int i = lane; i < n; i += 32) {
                    const float4 x = xs[i], v = vs[i];
                    float4 *gw = a.st + 2 * R.mass_base;
                    gw[2 * i] = x; gw[2 * i + 1] = v;
                    if (x.w > 0.f) { const float mi = 1.0f / x.w; mx += mi * x.x; m += mi; }
                    bad |= !isfinite(x.x + x.y + x.z + v.x + v.y + v.z);
                }
                if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, kErrNonFinite);
                mx = warp_sum(mx); m = warp_sum(m);
                if (lane == 0) a.travel[r] = mx / m - R.com0_x;
            }
            __syncthreads();
        }
    }
}

// (sin, cos)(2 pi f t_n) for the steps of one run, t_n = (counter + n) dt,
// evaluated in double precision.
__global__ void k_sc_table(const long long *counter, int nsteps, double dt, double two_pi_f, float2 *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nsteps) return;
    const double t = (double)(*counter + n) * dt;
    double s, c;
    sincos(two_pi_f * t, &s, &c);
    out[n] = make_float2((float)s, (float)c);
}

__global__ void k_advance(long long *counter, int nsteps) { *counter += nsteps; }

__global__ void k_sc_table_from(long long n0, int nsteps, double dt, double two_pi_f, float2 *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nsteps) return;
    double s, c;
    sincos(two_pi_f * ((double)(n0 + n) * dt), &s, &c);
    out[n] = make_float2((float)s, (float)c);
}

// Centre-of-mass x travel of every robot from the global state (one CTA per robot).
__global__ void k_com_travel(const RobotDev *robots, const float4 *st, float *travel)
{
    __shared__ float red[2][kComThreads / 32];
    const RobotDev R = robots[blockIdx.x];
    float mx = 0.f, m = 0.f;
    for (int i = threadIdx.x; i < R.n; i += blockDim.x) {
        const float4 x = st[2 * (R.mass_base + i)];
        if (x.w > 0.f) { const float mi = 1.0f / x.w; mx += mi * x.x; m += mi; }
    }
    mx = warp_sum(mx); m = warp_sum(m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[0][warp] = mx; red[1][warp] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float smx = 0.f, sm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { smx += red[0][w]; sm += red[1][w]; }
        travel[blockIdx.x] = smx / sm - R.com0_x;
    }
}

}  // namespace
}  // namespace ms

using namespace ms;

struct msb_batch {
    ms_params p{};
    msb_voxel_spec spec{};
    double freq = 0.0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    ms_allocator alloc{};
    bool custom_alloc = false;
    std::vector<std::pair<void *, size_t>> allocs;
    int64_t device_bytes = 0;

    int n_robots = 0;
    int64_t n_masses = 0, n_records = 0, n_slots = 0, n_back = 0;
    int n_slices = 0;
    int max_n = 0;
    std::vector<RobotDev> h_robots;
    std::vector<float4> h_st0;                 // initial state (for reset)

    RobotDev *robots = nullptr;
    float4 *st = nullptr, *st2 = nullptr;
    // robot-by-robot loop (msb_run_loop): the population in the single-system
    // step's packed layout, allocated on first use
    float4 *loop_a[2] = {nullptr, nullptr};
    float2 *loop_b[2] = {nullptr, nullptr};
    float *loop_w = nullptr;
    uint4 *slice = nullptr;
    int32_t *f_nbr = nullptr;
    float2 *f_kl = nullptr, *f_ab = nullptr;
    float *f_c = nullptr;
    uint32_t *b_ent = nullptr;
    // every-spring rows (the persistent population kernel)
    uint2 *a_slice = nullptr;
    uint16_t *a_nbr = nullptr;
    float2 *a_kl = nullptr, *a_ab = nullptr;
    float *a_c = nullptr;
    float *travel = nullptr;
    int *err = nullptr;
    int *queue = nullptr;
    long long *counter = nullptr;
    float2 *sc = nullptr;
    int sc_cap = 0;
    int4 *items = nullptr;
    int items_cap = 0;
    std::vector<int4> h_items;
    int *wlist = nullptr;
    int wlist_cap = 0;
    std::vector<int> h_wlist;
    std::vector<uint8_t> warp_mode;           // per robot: 1 = warp-per-robot
    int threads = kBatchThreadsDefault;       // CTA size of the persistent kernel (512 or 1024)
    int warp_cap = 32;
    int pair_cap = 32;
    int quad_cap = 32;
    size_t smem_bytes = 0;
    int grid = 0;
    int64_t step_count = 0;
    std::map<int, cudaGraphExec_t> graphs;

    void *dev_alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *ptr = nullptr;
        if (custom_alloc) ptr = alloc.alloc(bytes, stream, alloc.ctx);
        else if (cudaMalloc(&ptr, bytes) != cudaSuccess) { cudaGetLastError(); ptr = nullptr; }
        if (ptr) { allocs.push_back({ptr, bytes}); device_bytes += (int64_t)bytes; }
        return ptr;
    }
    void drop_graphs()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        graphs.clear();
    }
    void release()
    {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        drop_graphs();
        for (auto &a : allocs) {
            if (custom_alloc) alloc.free(a.first, a.second, stream, alloc.ctx);
            else cudaFree(a.first);
        }
        allocs.clear();
        if (cap_stream) { cudaStreamDestroy(cap_stream); cap_stream = nullptr; }
    }
};

namespace {

#define MSB_CUDA_TRY(expr)                                                                     \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return fail(MS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));     \
    } while (0)

template <class T>
ms_status bupload(msb_batch *b, T **dst, const T *src, size_t count)
{
    *dst = (T *)b->dev_alloc(sizeof(T) * count);
    if (!*dst) return fail(MS_ERR_OOM, "device allocation failed");
    if (src && count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    return MS_OK;
}

// The 13 forward neighbour directions (dx, dy, dz) of the 26-neighbourhood:
// (dz, dy, dx) lexicographically positive, so the partner is later in
// raster (x fastest) order.
struct Dir { int dx, dy, dz; };
std::vector<Dir> forward_dirs()
{
    std::vector<Dir> d;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                if (dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)))) d.push_back({dx, dy, dz});
    return d;
}

int dir_index(int dx, int dy, int dz)
{
    static const std::vector<Dir> d = forward_dirs();
    for (int q = 0; q < (int)d.size(); ++q)
        if (d[q].dx == dx && d[q].dy == dy && d[q].dz == dz) return q;
    return -1;
}

// Build the schedule items from per-robot modes: block items one per robot,
// warp items groups of up to threads / 32 robots of similar size, and (with
// 1024-thread CTAs) pair and quad items: two block robots of at most kPairMax
// masses, or four of at most kQuadMax, one per half / quarter of the CTA
// (one thread per mass); ordered by decreasing cost so the persistent CTAs
// balance (longest item first).
void set_items(msb_batch *b, const std::vector<int> &block_robots, std::vector<int> warp_robots)
{
    b->h_items.clear();
    b->h_wlist.clear();
    int cap = 32;
    std::vector<int> paired, quads;
    for (int r : block_robots) {
        const int n = b->h_robots[r].n;
        if (b->threads == 1024 && n <= kQuadMax) quads.push_back(r);
        else if (b->threads == 1024 && n <= kPairMax) paired.push_back(r);
        else b->h_items.push_back(make_int4(r, 1, 0, n));
    }
    std::stable_sort(warp_robots.begin(), warp_robots.end(),
                     [&](int x, int y) { return b->h_robots[x].n > b->h_robots[y].n; });
    const size_t wpc = (size_t)b->threads / 32;
    for (size_t q = 0; q < warp_robots.size(); q += wpc) {
        const int cnt = (int)std::min<size_t>(wpc, warp_robots.size() - q);
        int cost = 0;
        for (int u = 0; u < cnt; ++u) {
            const int r = warp_robots[q + u];
            b->h_wlist.push_back(r);
            cost = std::max(cost, b->h_robots[r].n);
            cap = std::max(cap, b->h_robots[r].n);
        }
        b->h_items.push_back(make_int4((int)q, cnt, 1, cost));
    }
    b->warp_cap = (cap + 31) / 32 * 32;
    // groups of G robots of similar size, one per 1024 / G threads (mode 2: G = 2, mode 3: G = 4)
    auto group = [&](std::vector<int> &rs, int G, int mode) {
        std::stable_sort(rs.begin(), rs.end(), [&](int x, int y) { return b->h_robots[x].n > b->h_robots[y].n; });
        int gcap = 32;
        for (size_t q = 0; q < rs.size(); q += G) {
            const int cnt = (int)std::min<size_t>((size_t)G, rs.size() - q);
            const int first = (int)b->h_wlist.size();
            int cost = 0;
            for (int u = 0; u < cnt; ++u) {
                const int r = rs[q + u];
                b->h_wlist.push_back(r);
                cost = std::max(cost, b->h_robots[r].n);
                gcap = std::max(gcap, b->h_robots[r].n);
            }
            b->h_items.push_back(make_int4(first, cnt, mode, cost));
        }
        return (gcap + 31) / 32 * 32;
    };
    b->pair_cap = group(paired, 2, 2);
    b->quad_cap = group(quads, 4, 3);
    std::stable_sort(b->h_items.begin(), b->h_items.end(), [](const int4 &x, const int4 &y) {
        // a warp robot advances with 1/8 of the CTA's threads
        const long long cx = (long long)x.w * (x.z == 0 ? 1 : 8), cy = (long long)y.w * (y.z == 0 ? 1 : 8);
        return cx > cy;
    });
    size_t blk = 0;
    for (auto &it : b->h_items) if (it.z == 0) blk = std::max(blk, (size_t)b->h_robots[it.x].n);
    const size_t warp_bytes = warp_robots.empty() ? 0 : wpc * 3 * b->warp_cap * sizeof(float4);
    const size_t pair_bytes = paired.empty() ? 0 : 2 * 3 * (size_t)b->pair_cap * sizeof(float4);
    const size_t quad_bytes = quads.empty() ? 0 : 4 * 3 * (size_t)b->quad_cap * sizeof(float4);
    b->smem_bytes = std::max<size_t>(
        std::max(std::max(blk * 3 * sizeof(float4), warp_bytes), std::max(pair_bytes, quad_bytes)), 16);
}

void build_items(msb_batch *b)
{
    std::vector<int> blk, wrp;
    for (int r = 0; r < b->n_robots; ++r) (b->warp_mode[r] ? wrp : blk).push_back(r);
    set_items(b, blk, wrp);
}

ms_status upload_items(msb_batch *b)
{
    const int n = (int)b->h_items.size();
    if (n > b->items_cap) {
        ms_status st = bupload<int4>(b, &b->items, nullptr, n);
        if (st != MS_OK) return st;
        b->items_cap = n;
    }
    MSB_CUDA_TRY(cudaMemcpyAsync(b->items, b->h_items.data(), sizeof(int4) * n, cudaMemcpyHostToDevice, b->stream));
    const int nw = (int)b->h_wlist.size();
    if (nw > b->wlist_cap || !b->wlist) {
        ms_status st = bupload<int>(b, &b->wlist, nullptr, std::max(nw, 1));
        if (st != MS_OK) return st;
        b->wlist_cap = std::max(nw, 1);
    }
    if (nw) MSB_CUDA_TRY(cudaMemcpyAsync(b->wlist, b->h_wlist.data(), sizeof(int) * nw, cudaMemcpyHostToDevice, b->stream));
    int dev = 0, sms = 0, per_sm = 0;
    MSB_CUDA_TRY(cudaGetDevice(&dev));
    MSB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (b->threads == 1024) {
        MSB_CUDA_TRY(cudaFuncSetAttribute(k_batch<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes));
        MSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<1024>, 1024, b->smem_bytes));
    } else {
        MSB_CUDA_TRY(cudaFuncSetAttribute(k_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes));
        MSB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<512>, 512, b->smem_bytes));
    }
    if (per_sm < 1) return fail(MS_ERR_ARG, "a robot does not fit in one CTA's shared memory");
    b->grid = std::max(1, std::min(n, sms * per_sm));
    MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->drop_graphs();
    return MS_OK;
}

ms_status ensure_sc(msb_batch *b, int nsteps)
{
    if (nsteps <= b->sc_cap) return MS_OK;
    b->drop_graphs();                          // graphs hold the old table pointer
    ms_status st = bupload<float2>(b, &b->sc, nullptr, std::max(nsteps, 1));
    if (st != MS_OK) return st;
    b->sc_cap = nsteps;
    return MS_OK;
}

BatchArgs batch_args(msb_batch *b, int nsteps)
{
    BatchArgs a{};
    a.robots = b->robots; a.items = b->items; a.wlist = b->wlist; a.n_items = (int)b->h_items.size(); a.queue = b->queue;
    a.st = b->st;
    a.rows = AllRows{b->a_slice, b->a_nbr, b->a_kl, b->a_ab, b->a_c};
    a.env = make_env(b->p);
    a.sc = b->sc; a.nsteps = nsteps;
    a.warp_cap = b->warp_cap; a.pair_cap = b->pair_cap; a.quad_cap = b->quad_cap;
    a.travel = b->travel; a.err = b->err;
    return a;
}

// Enqueue one run (table, persistent kernel, clock advance) on stream s.
ms_status enqueue_run(msb_batch *b, int nsteps, cudaStream_t s)
{
    MSB_CUDA_TRY(cudaMemsetAsync(b->queue, 0, sizeof(int), s));
    const double two_pi_f = 2.0 * M_PI * b->freq;
    k_sc_table<<<(nsteps + 255) / 256, 256, 0, s>>>(b->counter, nsteps, (double)b->p.dt, two_pi_f, b->sc);
    MSB_CUDA_TRY(cudaGetLastError());
    if (b->threads == 1024) k_batch<1024><<<b->grid, 1024, b->smem_bytes, s>>>(batch_args(b, nsteps));
    else k_batch<512><<<b->grid, 512, b->smem_bytes, s>>>(batch_args(b, nsteps));
    MSB_CUDA_TRY(cudaGetLastError());
    k_advance<<<1, 1, 0, s>>>(b->counter, nsteps);
    MSB_CUDA_TRY(cudaGetLastError());
    return MS_OK;
}

}  // namespace

namespace ms {
void launch_sc_table(const long long *counter, int nsteps, double dt, double two_pi_f, float2 *out, cudaStream_t s)
{
    if (nsteps > 0) k_sc_table<<<(nsteps + 255) / 256, 256, 0, s>>>(counter, nsteps, dt, two_pi_f, out);
}

void launch_sc_table_from(long long n0, int nsteps, double dt, double two_pi_f, float2 *out, cudaStream_t s)
{
    if (nsteps > 0) k_sc_table_from<<<(nsteps + 255) / 256, 256, 0, s>>>(n0, nsteps, dt, two_pi_f, out);
}


ms_status build_voxels(const msb_voxel_spec *spec, int n_robots, const int32_t *dims, const uint8_t *materials,
                       const float *phase, const float *logk, bool adjoint_maps, VoxelBuild &out)
{
    out = VoxelBuild();
    std::vector<uint4> &h_slice = out.slice;
    std::vector<int32_t> &h_nbr = out.nbr;
    std::vector<float2> &h_kl = out.kl, &h_ab = out.ab;
    std::vector<float> &h_c = out.c;
    std::vector<uint32_t> &h_b = out.bent;
    const std::vector<Dir> dirs = forward_dirs();
    const double a = spec->voxel_edge;
    float L0dir[13];
    for (int d = 0; d < 13; ++d)
        L0dir[d] = (float)(a * std::sqrt((double)(dirs[d].dx * dirs[d].dx + dirs[d].dy * dirs[d].dy + dirs[d].dz * dirs[d].dz)));

    out.robots.resize(n_robots);
    int64_t vox_off = 0;
    for (int r = 0; r < n_robots; ++r) {
        const int nx = dims[3 * r], ny = dims[3 * r + 1], nz = dims[3 * r + 2];
        if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz > (1 << 20)) return fail(MS_ERR_ARG, "bad dims for robot " + std::to_string(r));
        const int cx = nx + 1, cy = ny + 1, cz = nz + 1;
        const int64_t nvox = (int64_t)nx * ny * nz;
        const uint8_t *mat = materials + vox_off;
        const float *ph = phase ? phase + vox_off : nullptr;
        const float *lk = logk ? logk + vox_off : nullptr;
        std::vector<int32_t> cmap((size_t)cx * cy * cz, -1);
        std::vector<double> cmass((size_t)cx * cy * cz, 0.0);
        int nonempty = 0;
        for (int64_t v = 0; v < nvox; ++v) {
            if (mat[v] >= spec->n_materials) return fail(MS_ERR_ARG, "material id out of range in robot " + std::to_string(r));
            if (mat[v] == 0) continue;
            if (ph && !std::isfinite(ph[v])) return fail(MS_ERR_ARG, "non-finite phase in robot " + std::to_string(r));
            if (lk && !std::isfinite(lk[v])) return fail(MS_ERR_ARG, "non-finite logk in robot " + std::to_string(r));
            ++nonempty;
            const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((int64_t)nx * ny));
            for (int c8 = 0; c8 < 8; ++c8) {
                const int q = (ix + (c8 & 1)) + cx * ((iy + ((c8 >> 1) & 1)) + cy * (iz + (c8 >> 2)));
                cmap[q] = 1;
                cmass[q] += spec->voxel_mass / 8.0;
            }
        }
        if (!nonempty) return fail(MS_ERR_ARG, "robot " + std::to_string(r) + " has no non-empty voxel");
        int n = 0;
        for (size_t q = 0; q < cmap.size(); ++q) if (cmap[q] > 0) cmap[q] = n++;
        if (n > kMaxRobotMasses) return fail(MS_ERR_ARG, "robot " + std::to_string(r) + " has " + std::to_string(n) + " masses; at most 4096 are supported");
        // merged springs per (owner corner, forward direction)
        std::vector<double> K((size_t)n * 13, 0.0), Cc((size_t)n * 13, 0.0), SA((size_t)n * 13, 0.0), SB((size_t)n * 13, 0.0);
        std::vector<uint8_t> has((size_t)n * 13, 0);
        std::vector<short4> key_vox;                 // adjoint: voxels sharing each merged spring
        std::vector<uint32_t> vkey;                  // adjoint: key of each voxel's 28 corner pairs
        if (adjoint_maps) {
            if (nvox > 32767) return fail(MS_ERR_ARG, "robot " + std::to_string(r) + " has too many voxels for the adjoint maps");
            key_vox.assign((size_t)n * 13, make_short4(-1, -1, -1, -1));
            vkey.assign((size_t)nvox * 28, UINT32_MAX);
        }
        for (int64_t v = 0; v < nvox; ++v) {
            if (mat[v] == 0) continue;
            const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((int64_t)nx * ny));
            const double kv = lk ? std::exp((double)lk[v]) : (double)spec->mat_k[mat[v]];
            const double cv = spec->mat_c[mat[v]], av = spec->mat_amp[mat[v]];
            const double phv = ph ? (double)ph[v] : 0.0;
            for (int p8 = 0; p8 < 8; ++p8)
                for (int q8 = p8 + 1; q8 < 8; ++q8) {
                    // corner offsets inside the voxel; q8 > p8 means q is later in raster order
                    const int px = p8 & 1, py = (p8 >> 1) & 1, pz = p8 >> 2;
                    const int qx = q8 & 1, qy = (q8 >> 1) & 1, qz = q8 >> 2;
                    const int d = dir_index(qx - px, qy - py, qz - pz);
                    const int owner = cmap[(ix + px) + cx * ((iy + py) + cy * (iz + pz))];
                    const size_t key = (size_t)owner * 13 + d;
                    K[key] += kv; Cc[key] += cv;
                    SA[key] += kv * av * std::cos(phv); SB[key] += kv * av * std::sin(phv);
                    has[key] = 1;
                    if (adjoint_maps) {
                        short4 &kvx = key_vox[key];
                        if (kvx.x < 0) kvx.x = (short)v; else if (kvx.y < 0) kvx.y = (short)v;
                        else if (kvx.z < 0) kvx.z = (short)v; else kvx.w = (short)v;
                        int pair = 0;
                        for (int a8 = 0; a8 < p8; ++a8) pair += 7 - a8;
                        pair += q8 - p8 - 1;
                        vkey[(size_t)v * 28 + pair] = (uint32_t)key;
                    }
                }
        }
        // corner positions, masses
        RobotDev &R = out.robots[r];
        R.mass_base = out.n_masses; R.n = n; R.slice_base = out.n_slices;
        double M = 0, MX = 0;
        std::vector<int> pos_of(n);
        for (size_t q = 0; q < cmap.size(); ++q) {
            if (cmap[q] < 0) continue;
            const int qx = (int)(q % cx), qy = (int)((q / cx) % cy), qz = (int)(q / ((size_t)cx * cy));
            const double m = cmass[q];
            const float w = (float)(1.0 / m);
            out.st0.push_back(make_float4((float)(qx * a), (float)(qy * a), (float)(qz * a), w));
            out.st0.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
            M += m; MX += m * (double)(float)(qx * a);
            pos_of[cmap[q]] = (int)q;
        }
        R.com0_x = (float)(MX / M);
        R.inv_mass = (float)(1.0 / M);
        R.vox_base = (int)vox_off;
        R.n_vox = (int)nvox;
        // forward degrees and sliced-ELL rows
        std::vector<int> deg(n, 0), bdeg(n, 0);
        for (int o = 0; o < n; ++o)
            for (int d = 0; d < 13; ++d) if (has[(size_t)o * 13 + d]) deg[o]++;
        const int ns = (n + 31) / 32;
        const size_t slice0 = h_slice.size();
        R.rec_base = (uint32_t)h_nbr.size();              // the first slice's first record
        for (int s_ = 0; s_ < ns; ++s_) {
            int mx = 0;
            for (int l = 0; l < 32 && 32 * s_ + l < n; ++l) mx = std::max(mx, deg[32 * s_ + l]);
            h_slice.push_back(make_uint4((uint32_t)h_nbr.size(), 0u, (uint32_t)mx, 0u));
            h_nbr.resize(h_nbr.size() + 32 * (size_t)mx, -1);
        }
        h_kl.resize(h_nbr.size(), make_float2(0.f, 0.f));
        h_ab.resize(h_nbr.size(), make_float2(0.f, 0.f));
        h_c.resize(h_nbr.size(), 0.f);
        std::vector<int8_t> rdir(h_nbr.size() - R.rec_base, -1);    // forward direction of each record
        std::vector<uint32_t> key_slot;
        if (adjoint_maps) {
            out.slot_vox.resize(h_nbr.size(), make_short4(-1, -1, -1, -1));
            key_slot.assign((size_t)n * 13, UINT32_MAX);
        }
        for (int o = 0; o < n; ++o) {
            const int q = pos_of[o];
            const int ox = q % cx, oy = (q / cx) % cy, oz = q / (cx * cy);
            int slot = 0;
            for (int d = 0; d < 13; ++d) {
                const size_t key = (size_t)o * 13 + d;
                if (!has[key]) continue;
                const int j = cmap[(ox + dirs[d].dx) + cx * ((oy + dirs[d].dy) + cy * (oz + dirs[d].dz))];
                const uint32_t rr = h_slice[slice0 + (o >> 5)].x + 32u * slot + (uint32_t)(o & 31);
                h_nbr[rr] = j;
                rdir[rr - R.rec_base] = (int8_t)d;
                h_kl[rr] = make_float2((float)K[key], L0dir[d]);
                h_c[rr] = (float)Cc[key];
                h_ab[rr] = K[key] > 0 ? make_float2((float)(SA[key] / K[key]), (float)(SB[key] / K[key])) : make_float2(0.f, 0.f);
                if (adjoint_maps) { out.slot_vox[rr] = key_vox[key]; key_slot[key] = rr; }
                bdeg[j]++;
                ++slot;
                ++out.n_records;
            }
        }
        // back references
        const size_t b0 = h_b.size();
        for (int s_ = 0; s_ < ns; ++s_) {
            int mx = 0;
            for (int l = 0; l < 32 && 32 * s_ + l < n; ++l) mx = std::max(mx, bdeg[32 * s_ + l]);
            h_slice[slice0 + s_].y = (uint32_t)h_b.size();
            h_slice[slice0 + s_].z |= (uint32_t)mx << 16;
            h_b.resize(h_b.size() + 32 * (size_t)mx, kBackPad);
        }
        (void)b0;
        std::vector<int> bfill(n, 0);
        const uint32_t rec0 = h_slice[slice0].x;           // the robot's first record
        for (int o = 0; o < n; ++o) {
            const uint32_t base = h_slice[slice0 + (o >> 5)].x + (uint32_t)(o & 31);
            for (int s_ = 0; s_ < deg[o]; ++s_) {
                const uint32_t rr = base + 32u * s_;
                const int j = h_nbr[rr];
                const int t = bfill[j]++;
                if (rr - rec0 >= (1u << (32 - kRobotOwnerBits))) return fail(MS_ERR_ARG, "robot has too many spring records");
                h_b[h_slice[slice0 + (j >> 5)].y + 32u * t + (uint32_t)(j & 31)] = (uint32_t)o | ((rr - rec0) << kRobotOwnerBits);
            }
        }
        if (!adjoint_maps) {
            // every-spring rows, one slot per lattice direction: slot q of a
            // slice holds, for each of its 32 masses, the spring in direction
            // D_q (the directions any of them has, in a fixed order: the 13
            // forward ones, then their opposites), or padding that points at
            // the mass itself.  The lanes of a warp then read partners at
            // nearly the same offset from their own masses, so their
            // shared-memory reads fall in distinct banks.  A mass sums its
            // springs in this direction order.
            std::vector<int> drec((size_t)n * 26, -1), dpart((size_t)n * 26, -1);
            for (int i = 0; i < n; ++i) {
                const uint32_t fbase = h_slice[slice0 + (i >> 5)].x + (uint32_t)(i & 31);
                for (int s_ = 0; s_ < deg[i]; ++s_) {
                    const uint32_t rr = fbase + 32u * s_;
                    const int d = rdir[rr - R.rec_base];
                    drec[(size_t)i * 26 + d] = (int)rr;
                    dpart[(size_t)i * 26 + d] = h_nbr[rr];
                }
                const uint32_t bbase = h_slice[slice0 + (i >> 5)].y + (uint32_t)(i & 31);
                for (int t = 0; t < bdeg[i]; ++t) {
                    const uint32_t e = h_b[bbase + 32u * t];
                    const uint32_t rr = rec0 + (e >> kRobotOwnerBits);
                    const int d = rdir[rr - R.rec_base];
                    drec[(size_t)i * 26 + 13 + d] = (int)rr;
                    dpart[(size_t)i * 26 + 13 + d] = (int)(e & kRobotOwnerMask);
                }
            }
            for (int s_ = 0; s_ < ns; ++s_) {
                uint32_t mask = 0;
                for (int l = 0; l < 32 && 32 * s_ + l < n; ++l)
                    for (int D = 0; D < 26; ++D)
                        if (drec[(size_t)(32 * s_ + l) * 26 + D] >= 0) mask |= 1u << D;
                const int mx = __builtin_popcount(mask);
                out.aslice.push_back(make_uint2((uint32_t)out.anbr.size(), (uint32_t)mx));
                const size_t first = out.anbr.size();
                out.anbr.resize(first + 32 * (size_t)mx, 0);
                out.akl.resize(out.anbr.size(), make_float2(0.f, 0.f));
                out.aab.resize(out.anbr.size(), make_float2(0.f, 0.f));
                out.ac.resize(out.anbr.size(), 0.f);
                int q = 0;
                for (int D = 0; D < 26; ++D) {
                    if (!((mask >> D) & 1u)) continue;
                    for (int l = 0; l < 32; ++l) {
                        const int i = std::min(32 * s_ + l, n - 1);
                        const size_t w = first + 32 * (size_t)q + l;
                        const int rr = 32 * s_ + l < n ? drec[(size_t)i * 26 + D] : -1;
                        if (rr >= 0) {
                            out.anbr[w] = (uint16_t)dpart[(size_t)i * 26 + D];
                            out.akl[w] = h_kl[rr]; out.aab[w] = h_ab[rr]; out.ac[w] = h_c[rr];
                        } else {
                            out.anbr[w] = (uint16_t)i;     // k = 0 and zero length: no force
                        }
                    }
                    ++q;
                }
            }
            if (out.anbr.size() >= (size_t)UINT32_MAX / 2) return fail(MS_ERR_ARG, "population too large for 32-bit record offsets");
        }
        if (adjoint_maps) {
            for (int64_t v = 0; v < nvox; ++v) {
                for (int pr = 0; pr < 28; ++pr) {
                    const uint32_t key = vkey[(size_t)v * 28 + pr];
                    out.vox_slots.push_back(key == UINT32_MAX ? UINT32_MAX : key_slot[key]);
                }
                out.vox_amp.push_back(mat[v] ? spec->mat_amp[mat[v]] : 0.f);
            }
        }
        out.n_slices += ns;
        out.n_masses += n;
        out.max_n = std::max(out.max_n, n);
        vox_off += nvox;
        if (h_nbr.size() >= (size_t)UINT32_MAX / 2 || h_b.size() >= (size_t)UINT32_MAX / 2)
            return fail(MS_ERR_ARG, "population too large for 32-bit record offsets");
    }

    return MS_OK;
}

}  // namespace ms

extern "C" {

ms_status msb_create(const ms_params *p, const msb_voxel_spec *spec, int32_t n_robots, const int32_t *dims,
                     const uint8_t *materials, const float *phase, const float *logk,
                     const ms_allocator *alloc, void *stream, msb_batch **out)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !spec || !dims || !materials) return fail(MS_ERR_ARG, "p, spec, dims and materials are required");
    if (n_robots < 1) return fail(MS_ERR_ARG, "n_robots must be >= 1");
    if (!(p->dt > 0.f) || !std::isfinite(p->dt)) return fail(MS_ERR_ARG, "dt must be positive and finite");
    if (p->integrator != 0) return fail(MS_ERR_ARG, "the GPU path implements integrator 0 (symplectic Euler) only");
    if (!(p->vel_damping >= 0.f && p->vel_damping < 1.f)) return fail(MS_ERR_ARG, "vel_damping must be in [0, 1)");
    if (spec->n_materials < 1 || !spec->mat_k || !spec->mat_c || !spec->mat_amp) return fail(MS_ERR_ARG, "material table incomplete");
    if (!(spec->voxel_edge > 0.f) || !(spec->voxel_mass > 0.f) || !std::isfinite(spec->freq)) return fail(MS_ERR_ARG, "voxel_edge and voxel_mass must be > 0");
    for (int m = 0; m < spec->n_materials; ++m)
        if (!(spec->mat_k[m] >= 0.f) || !(spec->mat_c[m] >= 0.f) || !std::isfinite(spec->mat_amp[m]) || !std::isfinite(spec->mat_k[m]) || !std::isfinite(spec->mat_c[m]))
            return fail(MS_ERR_ARG, "material " + std::to_string(m) + " has a negative or non-finite entry");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(MS_ERR_ARG, "allocator needs alloc and free");

    msb_batch *b = new (std::nothrow) msb_batch();
    if (!b) return fail(MS_ERR_OOM, "host allocation failed");
    struct Guard { msb_batch *b; ~Guard() { if (b) { b->release(); delete b; } } } guard{b};
    b->p = *p; b->spec = *spec; b->freq = spec->freq;
    b->stream = (cudaStream_t)stream;
    if (alloc) { b->alloc = *alloc; b->custom_alloc = true; }
    b->n_robots = n_robots;

    VoxelBuild vb;
    ms_status st = build_voxels(spec, n_robots, dims, materials, phase, logk, false, vb);
    if (st != MS_OK) return st;
    b->h_robots = vb.robots;
    b->h_st0 = vb.st0;
    b->n_masses = vb.n_masses; b->n_records = vb.n_records; b->n_slices = vb.n_slices; b->max_n = vb.max_n;
    b->n_slots = (int64_t)vb.nbr.size();
    b->n_back = (int64_t)vb.bent.size();
    std::vector<uint4> &h_slice = vb.slice;
    std::vector<int32_t> &h_nbr = vb.nbr;
    std::vector<float2> &h_kl = vb.kl, &h_ab = vb.ab;
    std::vector<float> &h_c = vb.c;
    std::vector<uint32_t> &h_b = vb.bent;

    if ((st = bupload(b, &b->robots, b->h_robots.data(), n_robots)) != MS_OK) return st;
    if ((st = bupload(b, &b->st, b->h_st0.data(), b->h_st0.size())) != MS_OK) return st;
    if ((st = bupload<float4>(b, &b->st2, nullptr, b->h_st0.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->slice, h_slice.data(), h_slice.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->f_nbr, h_nbr.data(), h_nbr.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->f_kl, h_kl.data(), h_kl.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->f_ab, h_ab.data(), h_ab.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->f_c, h_c.data(), h_c.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->b_ent, h_b.data(), h_b.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->a_slice, vb.aslice.data(), vb.aslice.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->a_nbr, vb.anbr.data(), vb.anbr.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->a_kl, vb.akl.data(), vb.akl.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->a_ab, vb.aab.data(), vb.aab.size())) != MS_OK) return st;
    if ((st = bupload(b, &b->a_c, vb.ac.data(), vb.ac.size())) != MS_OK) return st;
    if ((st = bupload<float>(b, &b->travel, nullptr, n_robots)) != MS_OK) return st;
    if ((st = bupload<int>(b, &b->err, nullptr, 1)) != MS_OK) return st;
    if ((st = bupload<int>(b, &b->queue, nullptr, 1)) != MS_OK) return st;
    if ((st = bupload<long long>(b, &b->counter, nullptr, 1)) != MS_OK) return st;
    MSB_CUDA_TRY(cudaMemsetAsync(b->err, 0, sizeof(int), b->stream));
    MSB_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(long long), b->stream));
    MSB_CUDA_TRY(cudaMemsetAsync(b->travel, 0, sizeof(float) * n_robots, b->stream));
    MSB_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    b->warp_mode.assign(n_robots, 0);
    for (int r = 0; r < n_robots; ++r) b->warp_mode[r] = b->h_robots[r].n <= 64 ? 1 : 0;
    build_items(b);
    if ((st = upload_items(b)) != MS_OK) return st;
    MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    guard.b = nullptr;
    *out = b;
    return MS_OK;
}

ms_status msb_run(msb_batch *b, int32_t nsteps)
{
    ms::Range range_("msb_run");
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return fail(MS_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return MS_OK;
    ms_status st = ensure_sc(b, nsteps);
    if (st != MS_OK) return st;
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        MSB_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_run(b, nsteps, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != MS_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = b->graphs.emplace(nsteps, ge).first;
    }
    MSB_CUDA_TRY(cudaGraphLaunch(it->second, b->stream));
    b->step_count += nsteps;
    return MS_OK;
}

ms_status msb_run_loop(msb_batch *b, int32_t nsteps)
{
    ms::Range range_("msb_run_loop");
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    if (nsteps < 0) return fail(MS_ERR_ARG, "nsteps must be >= 0");
    if (!b->loop_w) {
        ms_status st;
        for (int q = 0; q < 2; ++q) {
            if ((st = bupload<float4>(b, &b->loop_a[q], nullptr, (size_t)b->n_masses)) != MS_OK) return st;
            if ((st = bupload<float2>(b, &b->loop_b[q], nullptr, (size_t)b->n_masses)) != MS_OK) return st;
        }
        if ((st = bupload<float>(b, &b->loop_w, nullptr, (size_t)b->n_masses)) != MS_OK) return st;
    }
    // the single-system step kernel keeps the state packed: convert, step robot by robot, convert back
    MSB_CUDA_TRY(launch_pack_state(b->st, (int)b->n_masses, b->loop_a[0], b->loop_b[0], b->loop_w, b->stream));
    StepArgs a{};
    a.f_nbr = b->f_nbr; a.f_kl = b->f_kl; a.f_c = b->f_c; a.f_ab = b->f_ab; a.b_ent = b->b_ent;
    a.err = b->err; a.dt = b->p.dt; a.gx = b->p.g[0]; a.gy = b->p.g[1]; a.gz = b->p.g[2];
    a.k_c = b->p.k_c; a.mu = b->p.mu; a.keep = 1.0f - b->p.vel_damping; a.contact = b->p.contact_on;
    const double two_pi_f = 2.0 * M_PI * b->freq;
    int cur = 0;
    for (int n = 0; n < nsteps; ++n) {
        const double t = (double)(b->step_count + n) * (double)b->p.dt;
        a.s_n = (float)std::sin(two_pi_f * t);
        a.c_n = (float)std::cos(two_pi_f * t);
        for (int r = 0; r < b->n_robots; ++r) {
            const RobotDev &R = b->h_robots[r];
            a.N = R.n;
            a.slice = b->slice + R.slice_base;
            a.back_local = 1;                  // robot records use robot-local back references
            a.back_base = R.rec_base;
            a.sa = b->loop_a[cur] + R.mass_base; a.sb = b->loop_b[cur] + R.mass_base;
            a.oa = b->loop_a[cur ^ 1] + R.mass_base; a.ob = b->loop_b[cur ^ 1] + R.mass_base;
            a.w = b->loop_w + R.mass_base;
            MSB_CUDA_TRY(launch_step(a, b->stream));
        }
        cur ^= 1;
    }
    MSB_CUDA_TRY(launch_unpack_state(b->loop_a[cur], b->loop_b[cur], b->loop_w, (int)b->n_masses, b->st, b->stream));
    // keep the batched kernel's clock in step with this one
    if (nsteps > 0) {
        k_advance<<<1, 1, 0, b->stream>>>(b->counter, nsteps);
        MSB_CUDA_TRY(cudaGetLastError());
    }
    k_com_travel<<<b->n_robots, kComThreads, 0, b->stream>>>(b->robots, b->st, b->travel);
    MSB_CUDA_TRY(cudaGetLastError());
    b->step_count += nsteps;
    return MS_OK;
}

ms_status msb_autotune(msb_batch *b, int32_t sample_steps, int32_t policy)
{
    ms::Range range_("msb_autotune");
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    if (policy < 0 || policy > 2) return fail(MS_ERR_ARG, "policy must be 0, 1 or 2");
    const size_t smem_limit = 200 * 1024;
    auto warp_ok = [&](int n) {
        return n <= kWarpModeMax && (size_t)(b->threads / 32) * 3 * ((n + 31) / 32 * 32) * sizeof(float4) <= smem_limit;
    };
    if (policy == 1) { std::fill(b->warp_mode.begin(), b->warp_mode.end(), 0); }
    else if (policy == 2) { for (int r = 0; r < b->n_robots; ++r) b->warp_mode[r] = warp_ok(b->h_robots[r].n) ? 1 : 0; }
    else {
        if (sample_steps < 1) return fail(MS_ERR_ARG, "sample_steps must be >= 1");
        // save the state: the timing runs advance the robots
        MSB_CUDA_TRY(cudaMemcpyAsync(b->st2, b->st, sizeof(float4) * 2 * b->n_masses, cudaMemcpyDeviceToDevice, b->stream));
        ms_status st = ensure_sc(b, sample_steps);
        if (st != MS_OK) return st;
        // size buckets by mass count: (0,32], (32,64], (64,128], (128,256]
        const int edges[] = {0, 32, 64, 128, 256};
        cudaEvent_t e0, e1;
        MSB_CUDA_TRY(cudaEventCreate(&e0));
        MSB_CUDA_TRY(cudaEventCreate(&e1));
        // two runs of sample_steps steps with the current items; the second is timed
        auto time_items = [&](float &ms_out) -> ms_status {
            ms_status s2 = upload_items(b);
            if (s2 != MS_OK) return s2;
            for (int rep = 0; rep < 2; ++rep) {
                MSB_CUDA_TRY(cudaEventRecord(e0, b->stream));
                if ((s2 = enqueue_run(b, sample_steps, b->stream)) != MS_OK) return s2;
                MSB_CUDA_TRY(cudaEventRecord(e1, b->stream));
                MSB_CUDA_TRY(cudaEventSynchronize(e1));
            }
            MSB_CUDA_TRY(cudaEventElapsedTime(&ms_out, e0, e1));
            return MS_OK;
        };
        // For each CTA size: from the default schedules (warp-per-robot up to 64
        // masses), flip one size bucket at a time between warp- and
        // block-per-robot, and keep a flip when the whole population, run for
        // sample_steps from the saved state, gets faster.  Timing the whole
        // population measures throughput; a sample of one bucket alone would
        // not fill the GPU.  Then keep the faster CTA size.
        auto bucket_of = [&](int n) {
            int bk = 0;
            for (int q = 1; q < 5; ++q) if (n > edges[q - 1] && n <= edges[q]) bk = q;
            return bk;
        };
        auto time_all = [&](float &t) -> ms_status {
            build_items(b);
            MSB_CUDA_TRY(cudaMemcpyAsync(b->st, b->st2, sizeof(float4) * 2 * b->n_masses, cudaMemcpyDeviceToDevice, b->stream));
            return time_items(t);
        };
        float best_t = -1.f;
        int best_threads = b->threads;
        std::vector<uint8_t> best_mode = b->warp_mode;
        for (const int T : {512, 1024}) {
            b->threads = T;
            for (int r = 0; r < b->n_robots; ++r) {
                const int n = b->h_robots[r].n;
                b->warp_mode[r] = (n <= 64 && warp_ok(n)) ? 1 : 0;
            }
            float t_cur = 0.f;
            if ((st = time_all(t_cur)) != MS_OK) return st;
            for (int bk = 1; bk < 5; ++bk) {
                std::vector<uint8_t> trial = b->warp_mode;
                bool any = false;
                for (int r = 0; r < b->n_robots; ++r) {
                    const int n = b->h_robots[r].n;
                    if (bucket_of(n) == bk && warp_ok(n)) { trial[r] ^= 1; any = true; }
                }
                if (!any) continue;
                std::swap(b->warp_mode, trial);
                float t = 0.f;
                if ((st = time_all(t)) != MS_OK) return st;
                if (t < t_cur) t_cur = t;
                else std::swap(b->warp_mode, trial);      // keep the previous schedules
            }
            if (best_t < 0.f || t_cur < best_t) { best_t = t_cur; best_threads = T; best_mode = b->warp_mode; }
        }
        b->threads = best_threads;
        b->warp_mode = best_mode;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        // restore the state, the clock and the travel record
        MSB_CUDA_TRY(cudaMemcpyAsync(b->st, b->st2, sizeof(float4) * 2 * b->n_masses, cudaMemcpyDeviceToDevice, b->stream));
        k_com_travel<<<b->n_robots, kComThreads, 0, b->stream>>>(b->robots, b->st, b->travel);
        MSB_CUDA_TRY(cudaGetLastError());
        const long long sc_now = b->step_count;
        MSB_CUDA_TRY(cudaMemcpyAsync(b->counter, &sc_now, sizeof(long long), cudaMemcpyHostToDevice, b->stream));
        MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    }
    build_items(b);
    return upload_items(b);
}

ms_status msb_set_threads(msb_batch *b, int32_t threads)
{
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    if (threads != 512 && threads != 1024) return fail(MS_ERR_ARG, "threads per CTA must be 512 or 1024");
    b->threads = threads;
    // robots whose warp share no longer fits shared memory run block-per-robot
    const size_t smem_limit = 200 * 1024;
    for (int r = 0; r < b->n_robots; ++r) {
        const int n = b->h_robots[r].n;
        if ((size_t)(threads / 32) * 3 * ((n + 31) / 32 * 32) * sizeof(float4) > smem_limit) b->warp_mode[r] = 0;
    }
    build_items(b);
    return upload_items(b);
}

ms_status msb_com_travel(msb_batch *b, float *out, int32_t on_device)
{
    if (!b || !out) return fail(MS_ERR_ARG, "batch and out are required");
    if (on_device) {
        MSB_CUDA_TRY(cudaMemcpyAsync(out, b->travel, sizeof(float) * b->n_robots, cudaMemcpyDeviceToDevice, b->stream));
        return MS_OK;
    }
    MSB_CUDA_TRY(cudaMemcpyAsync(out, b->travel, sizeof(float) * b->n_robots, cudaMemcpyDeviceToHost, b->stream));
    MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    int flag = 0;
    MSB_CUDA_TRY(cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(MS_ERR_NONFINITE, "a robot reached a non-finite position or velocity");
    return MS_OK;
}

ms_status msb_robot_info(const msb_batch *b, int32_t robot, int32_t *n_masses, int64_t *first_mass)
{
    if (!b || robot < 0 || robot >= b->n_robots) return fail(MS_ERR_ARG, "bad batch or robot index");
    if (n_masses) *n_masses = b->h_robots[robot].n;
    if (first_mass) *first_mass = b->h_robots[robot].mass_base;
    return MS_OK;
}

ms_status msb_get_state(msb_batch *b, float *x, float *v)
{
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    std::vector<float4> h(2 * (size_t)b->n_masses);
    MSB_CUDA_TRY(cudaMemcpyAsync(h.data(), b->st, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost, b->stream));
    MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int64_t i = 0; i < b->n_masses; ++i) {
        if (x) { x[3 * i] = h[2 * i].x; x[3 * i + 1] = h[2 * i].y; x[3 * i + 2] = h[2 * i].z; }
        if (v) { v[3 * i] = h[2 * i + 1].x; v[3 * i + 1] = h[2 * i + 1].y; v[3 * i + 2] = h[2 * i + 1].z; }
    }
    return MS_OK;
}

ms_status msb_reset(msb_batch *b)
{
    if (!b) return fail(MS_ERR_ARG, "batch is NULL");
    MSB_CUDA_TRY(cudaMemcpyAsync(b->st, b->h_st0.data(), sizeof(float4) * b->h_st0.size(), cudaMemcpyHostToDevice, b->stream));
    MSB_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(long long), b->stream));
    MSB_CUDA_TRY(cudaMemsetAsync(b->travel, 0, sizeof(float) * b->n_robots, b->stream));
    MSB_CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->step_count = 0;
    return MS_OK;
}

ms_status msb_get_info(const msb_batch *b, msb_info_t *out)
{
    if (!b || !out) return fail(MS_ERR_ARG, "batch or out is NULL");
    out->n_robots = b->n_robots; out->n_masses = b->n_masses; out->n_records = b->n_records;
    out->max_robot_masses = b->max_n;
    int nb = 0, nw = 0;
    for (int r = 0; r < b->n_robots; ++r) (b->warp_mode[r] ? nw : nb)++;
    out->n_block_items = nb; out->n_warp_items = nw;
    out->threads = b->threads;
    out->device_bytes = b->device_bytes; out->step_count = b->step_count;
    return MS_OK;
}

ms_status msb_destroy(msb_batch *b)
{
    if (!b) return MS_OK;
    b->release();
    delete b;
    return MS_OK;
}

}  // extern "C"
