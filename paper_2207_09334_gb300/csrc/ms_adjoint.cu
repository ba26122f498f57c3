// ms_adjoint.cu -- reverse-mode gradients of voxel-robot rollouts.
//
// One CTA per robot.  The robot's state lives in shared memory; the forward
// pass stores a checkpoint (x, v) every K steps; the reverse pass, segment
// by segment from the last, recomputes the K forward steps from the
// checkpoint (keeping x_n, v_n and the pre-clamp velocity with its contact
// flag in a global segment buffer) and then walks them backwards:
//
//   forward step n (per free mass, w = 1/m):
//     F   = sum_springs f(x_n, v_n, t_n) + [z < 0] (0, 0, -k_c z)
//     vt  = v_n + dt (F w + g)
//     vc  = Coulomb clamp of (vt_x, vt_y) by D = mu (-k_c z) dt w     (if z < 0)
//     v'  = keep vc,   x' = x_n + dt v'
//
//   reverse step n, given lx = dL/dx', lv = dL/dv':
//     G   = lv + dt lx                    (total derivative w.r.t. v')
//     gc  = keep G
//     clamp, slipping: gvt_t = (1 - D/|vt|) gc_t + D (vt.gc_t) vt_t / |vt|^3,
//                      gD = -(vt.gc_t)/|vt|;   sticking: gvt_t = 0, gD = 0
//     a   = dt w gvt                      (dL/dF)
//     dL/dx_n = lx + (0, 0, -k_c a_z [z<0] - mu k_c dt w gD [clamp active])
//               - sum_springs g_d,     dL/dv_n = gvt - sum_springs c (w.u) u
//   where, for a spring with d = x_j - x_i, u = d/l, s = k (l - L) + c dv.u,
//   W = a_i - a_j:
//     g_d = (W.u) (k u + c (dv - (dv.u) u)/l) + s (W - (W.u) u)/l.
//   Parameters: voxel v contributes k_v (l - L_v(t_n)) to s of each of its
//   28 springs, with k_v = exp(logk_v), L_v = L0 (1 + A_v sin(w t_n + phi_v)),
//   so dL/dlogk_v += (W.u) k_v (l - L_v) and
//      dL/dphi_v  -= (W.u) k_v L0 A_v cos(w t_n + phi_v), summed over its springs.
// The spring owner writes (W.u, l) per merged spring to a scratch array; a
// voxel pass then gathers its 28 springs in a fixed order (deterministic).
#include "ms_voxel.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ms {
namespace {

// Threads per robot (one CTA each): 1024, 768, 512 or 256.  More threads per
// robot hide more of the latency of each step's record loads; fewer let more
// robots run at once.  Each size has its CTAs per multiprocessor fixed by its
// register budget: 1024 x 64 registers (one), 768 x 40 (two: one thread per
// mass of an 8^3-voxel walker, and 256 walkers in one wave), 512 x 64 (two),
// 256 x 64 (four).  msa_create picks the size from the population
// (choose_threads), msa_set_threads overrides it.
constexpr int kAdjThreadChoices[4] = {1024, 768, 512, 256};
__host__ __device__ constexpr int adj_ctas_per_sm(int T) { return T == 1024 ? 1 : T == 768 ? 2 : T == 512 ? 2 : 4; }
constexpr int kAdjMaxMasses = 1024;
constexpr int kAdjMaxVoxels = 4096;

struct AdjArgs {
    const RobotDev *robots;
    const int2 *slot_range;     // per robot: [first slot, end slot)
    Records rec;
    const short4 *slot_vox;
    const uint32_t *vox_slots;  // 28 per voxel
    const float *vox_amp;
    const float *phase;         // per voxel
    const float *logk;
    const float4 *st0;          // initial state, 2 float4 per mass
    const float4 *seed;         // per mass (xyz), or nullptr for centre-of-mass x travel
    float4 *ckpt;               // [robot][n_ckpt][n_cap] x,v pairs
    float4 *seg;                // [robot][K][n_cap] x, v, vt triples
    float2 *scratch;            // per slot: (W.u, l)
    const float2 *sc;           // (sin, cos)(2 pi f t_n), n = 0 .. nsteps-1
    Env env;
    int nsteps, K, n_ckpt, n_cap;
    float *loss;
    float *g_phase, *g_logk;
    int *err;
};

__global__ void k_zero_counter(long long *c) { *c = 0; }

// merged stiffness and actuation of every spring from the voxel parameters
__global__ void k_adj_merge(const int2 *slot_range, const RobotDev *robots, const short4 *slot_vox,
                            const float *phase, const float *logk, const float *amp, float2 *kl, float2 *ab)
{
    const int r = blockIdx.x;
    const int2 rg = slot_range[r];
    const int vb = robots[r].vox_base;
    for (int m = rg.x + threadIdx.x; m < rg.y; m += blockDim.x) {
        const short4 vv = slot_vox[m];
        const short ids[4] = {vv.x, vv.y, vv.z, vv.w};
        float K = 0.f, SA = 0.f, SB = 0.f;
        for (int q = 0; q < 4; ++q) {
            if (ids[q] < 0) continue;
            const int v = vb + ids[q];
            const float kv = expf(logk[v]);
            float sp, cp;
            sincosf(phase[v], &sp, &cp);
            K += kv; SA += kv * amp[v] * cp; SB += kv * amp[v] * sp;
        }
        kl[m].x = K;
        ab[m] = K > 0.f ? make_float2(SA / K, SB / K) : make_float2(0.f, 0.f);
    }
}

template <int T>
__device__ __forceinline__ float block_sum(float v, float *red)
{
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < T / 32; ++w) t += red[w];
    return t;
}

// reverse spring terms of mass i against partner j (frame of i); returns W.u
__device__ __forceinline__ float spring_adjoint(const float4 xi, const float4 vi, const float4 ai, const float4 xj,
                                                const float4 vj, const float4 aj, float k, float L, float c,
                                                float3 &gx, float3 &gv, float &l_out)
{
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    l_out = 0.f;
    if (!(l2 > 0.f)) return 0.f;
    const float il = rsqrtf(l2);
    const float l = l2 * il;
    const float ux = dx * il, uy = dy * il, uz = dz * il;
    const float dvx = vj.x - vi.x, dvy = vj.y - vi.y, dvz = vj.z - vi.z;
    const float dvu = dvx * ux + dvy * uy + dvz * uz;
    const float s = k * (l - L) + c * dvu;
    const float Wx = ai.x - aj.x, Wy = ai.y - aj.y, Wz = ai.z - aj.z;
    const float wu = Wx * ux + Wy * uy + Wz * uz;
    // g_d = wu (k u + c (dv - dvu u)/l) + s (W - wu u)/l
    const float gdx = wu * (k * ux + c * (dvx - dvu * ux) * il) + s * (Wx - wu * ux) * il;
    const float gdy = wu * (k * uy + c * (dvy - dvu * uy) * il) + s * (Wy - wu * uy) * il;
    const float gdz = wu * (k * uz + c * (dvz - dvu * uz) * il) + s * (Wz - wu * uz) * il;
    gx.x -= gdx; gx.y -= gdy; gx.z -= gdz;
    gv.x -= c * wu * ux; gv.y -= c * wu * uy; gv.z -= c * wu * uz;
    l_out = l;
    return wu;
}

template <int T>
__global__ void __launch_bounds__(T, adj_ctas_per_sm(T)) k_adjoint(const AdjArgs a)
{
    extern __shared__ float4 sm4[];
    __shared__ float red[T / 32];
    const int r = blockIdx.x, tid = threadIdx.x;
    const RobotDev R = a.robots[r];
    const int n = R.n, nv = R.n_vox;
    float4 *xs = sm4, *vs = xs + n, *vts = vs + n, *lx = vts + n, *lv = lx + n, *aa = lv + n;
    float *gph = reinterpret_cast<float *>(aa + n), *glk = gph + nv;
    const Env &e = a.env;
    const Records &rc = a.rec;
    const unsigned rec_base = R.rec_base;          // the robot's first record
    float4 *ck = a.ckpt + (size_t)r * a.n_ckpt * a.n_cap * 2;
    float4 *sg = a.seg + (size_t)r * a.K * a.n_cap * 3;

    for (int i = tid; i < n; i += T) {
        xs[i] = a.st0[2 * (R.mass_base + i)];
        vs[i] = a.st0[2 * (R.mass_base + i) + 1];
    }
    for (int v = tid; v < nv; v += T) { gph[v] = 0.f; glk[v] = 0.f; }
    __syncthreads();

    // ---- forward pass with checkpoints ----
    for (int step = 0; step < a.nsteps; ++step) {
        if (step % a.K == 0) {
            float4 *c = ck + (size_t)(step / a.K) * a.n_cap * 2;
            for (int i = tid; i < n; i += T) { c[2 * i] = xs[i]; c[2 * i + 1] = vs[i]; }
        }
        const float2 sc = a.sc[step];
        for (int i = tid; i < n; i += T) aa[i] = robot_force(rc, R.slice_base, rec_base, i, xs, vs, sc.x, sc.y);
        __syncthreads();
        for (int i = tid; i < n; i += T) {
            float4 x = xs[i], v = vs[i];
            robot_integrate(e, x, v, aa[i]);
            xs[i] = x; vs[i] = v;
        }
        __syncthreads();
    }

    // ---- loss and terminal adjoint ----
    float part = 0.f;
    for (int i = tid; i < n; i += T) {
        const float4 x = xs[i];
        float4 s4;
        if (a.seed) s4 = a.seed[R.mass_base + i];
        else s4 = make_float4(x.w > 0.f ? R.inv_mass / x.w : 0.f, 0.f, 0.f, 0.f);
        part += s4.x * x.x + s4.y * x.y + s4.z * x.z;
        lx[i] = make_float4(s4.x, s4.y, s4.z, 0.f);
        lv[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!isfinite(x.x + x.y + x.z)) atomicOr(a.err, kErrNonFinite);
    }
    const float L = block_sum<T>(part, red);
    if (tid == 0) a.loss[r] = a.seed ? L : L - R.com0_x;

    // ---- reverse pass, segment by segment ----
    const int nseg = (a.nsteps + a.K - 1) / a.K;
    for (int cseg = nseg - 1; cseg >= 0; --cseg) {
        const int n0 = cseg * a.K, n1 = min(n0 + a.K, a.nsteps);
        const float4 *c = ck + (size_t)cseg * a.n_cap * 2;
        __syncthreads();
        for (int i = tid; i < n; i += T) { xs[i] = c[2 * i]; vs[i] = c[2 * i + 1]; }
        __syncthreads();
        for (int step = n0; step < n1; ++step) {            // recompute the segment
            float4 *sgn = sg + (size_t)(step - n0) * a.n_cap * 3;
            const float2 sc = a.sc[step];
            for (int i = tid; i < n; i += T) aa[i] = robot_force(rc, R.slice_base, rec_base, i, xs, vs, sc.x, sc.y);
            __syncthreads();
            for (int i = tid; i < n; i += T) {
                float4 x = xs[i], v = vs[i], vt;
                sgn[3 * i] = x; sgn[3 * i + 1] = v;
                robot_integrate(e, x, v, aa[i], &vt);
                sgn[3 * i + 2] = vt;
                xs[i] = x; vs[i] = v;
            }
            __syncthreads();
        }
        for (int step = n1 - 1; step >= n0; --step) {       // and walk it backwards
            const float4 *sgn = sg + (size_t)(step - n0) * a.n_cap * 3;
            const float2 sc = a.sc[step];
            for (int i = tid; i < n; i += T) { xs[i] = sgn[3 * i]; vs[i] = sgn[3 * i + 1]; vts[i] = sgn[3 * i + 2]; }
            __syncthreads();
            // phase A: through the update, the clamp and the contact force
            for (int i = tid; i < n; i += T) {
                const float4 x = xs[i], vt = vts[i], lxi = lx[i], lvi = lv[i];
                const float w = x.w;
                if (w < 0.f) { aa[i] = make_float4(0.f, 0.f, 0.f, 0.f); lv[i] = aa[i]; continue; }
                const float Gx = lvi.x + e.dt * lxi.x, Gy = lvi.y + e.dt * lxi.y, Gz = lvi.z + e.dt * lxi.z;
                float gx = e.keep * Gx, gy = e.keep * Gy, gz = e.keep * Gz;
                const bool pen = vt.w > 0.5f;
                float gzx = 0.f;
                if (pen && e.mu > 0.f) {
                    const float D = e.mu * (-e.k_c * x.z) * e.dt * w;
                    const float vtn = sqrtf(vt.x * vt.x + vt.y * vt.y);
                    if (vtn <= D) { gx = 0.f; gy = 0.f; }
                    else {
                        const float dot = vt.x * gx + vt.y * gy;
                        const float q = 1.f - D / vtn, h = D * dot / (vtn * vtn * vtn);
                        const float gD = -dot / vtn;
                        gx = q * gx + h * vt.x;
                        gy = q * gy + h * vt.y;
                        gzx = gD * (-e.mu * e.k_c * e.dt * w);
                    }
                }
                const float4 ai = make_float4(e.dt * w * gx, e.dt * w * gy, e.dt * w * gz, 0.f);
                aa[i] = ai;
                lv[i] = make_float4(gx, gy, gz, 0.f);
                lx[i] = make_float4(lxi.x, lxi.y, lxi.z + gzx + (pen ? -e.k_c * ai.z : 0.f), 0.f);
            }
            __syncthreads();
            // phase B: through the spring forces (each mass gathers its springs)
            for (int i = tid; i < n; i += T) {
                const float4 xi = xs[i], vi = vs[i], ai = aa[i];
                float3 gx = make_float3(0.f, 0.f, 0.f), gv = make_float3(0.f, 0.f, 0.f);
                const unsigned lane = (unsigned)i & 31u;
                const uint4 meta = __ldg(&rc.slice[R.slice_base + (i >> 5)]);
                const unsigned flen = meta.z & 0xffffu, blen = meta.z >> 16;
                unsigned rr = meta.x + lane;
                for (unsigned s = 0; s < flen; ++s, rr += 32u) {
                    const int j = __ldg(&rc.f_nbr[rr]);
                    if (j < 0) continue;
                    const float2 kl = __ldg(&rc.f_kl[rr]);
                    const float2 ab = __ldg(&rc.f_ab[rr]);
                    const float Lr = kl.y * (1.0f + (ab.x * sc.x + ab.y * sc.y));
                    float l;
                    const float wu = spring_adjoint(xi, vi, ai, xs[j], vs[j], aa[j], kl.x, Lr, __ldg(&rc.f_c[rr]), gx, gv, l);
                    a.scratch[rr] = make_float2(wu, l);
                }
                unsigned q = meta.y + lane;
                for (unsigned s = 0; s < blen; ++s, q += 32u) {
                    const uint32_t be = __ldg(&rc.b_ent[q]);
                    if (be == kBackPad) continue;
                    const int o = (int)(be & kRobotOwnerMask);
                    const unsigned r2 = rec_base + (be >> kRobotOwnerBits);
                    const float2 kl = __ldg(&rc.f_kl[r2]);
                    const float2 ab = __ldg(&rc.f_ab[r2]);
                    const float Lr = kl.y * (1.0f + (ab.x * sc.x + ab.y * sc.y));
                    float l;
                    spring_adjoint(xi, vi, ai, xs[o], vs[o], aa[o], kl.x, Lr, __ldg(&rc.f_c[r2]), gx, gv, l);
                }
                const float4 lxi = lx[i], lvi = lv[i];
                lx[i] = make_float4(lxi.x + gx.x, lxi.y + gx.y, lxi.z + gx.z, 0.f);
                lv[i] = make_float4(lvi.x + gv.x, lvi.y + gv.y, lvi.z + gv.z, 0.f);
            }
            __syncthreads();
            // phase C: parameter gradients, voxel by voxel over its 28 springs
            for (int v = tid; v < nv; v += T) {
                const int gvx = R.vox_base + v;
                const uint32_t *vsl = a.vox_slots + (size_t)gvx * 28;
                if (vsl[0] == 0xffffffffu) continue;               // empty voxel
                const float kv = expf(a.logk[gvx]);
                const float A = a.vox_amp[gvx];
                float sp, cp;
                sincosf(a.phase[gvx], &sp, &cp);
                const float sinT = sc.x * cp + sc.y * sp;          // sin(w t + phi)
                const float cosT = sc.y * cp - sc.x * sp;          // cos(w t + phi)
                float dk = 0.f, dp = 0.f;
                for (int pr = 0; pr < 28; ++pr) {
                    const uint32_t m = vsl[pr];
                    const float2 gl = a.scratch[m];
                    const float L0 = __ldg(&rc.f_kl[m]).y;
                    dk += gl.x * kv * (gl.y - L0 * (1.f + A * sinT));
                    dp -= gl.x * kv * L0 * A * cosT;
                }
                glk[v] += dk;
                gph[v] += dp;
            }
            __syncthreads();
        }
    }
    for (int v = tid; v < nv; v += T) {
        a.g_phase[R.vox_base + v] = gph[v];
        a.g_logk[R.vox_base + v] = glk[v];
    }
}

// Threads per robot for a population: the choice T whose estimated time,
// waves(T) * ceil(n_cap / T), is smallest (the larger T on a tie), where a
// wave is one CTA per robot on every multiprocessor, as many at once as the
// register budget (adj_ctas_per_sm) and the shared memory of a
// multiprocessor allow.
int choose_threads(int n_robots, int n_cap, size_t smem, int n_sms, int smem_per_sm)
{
    int best = kAdjThreadChoices[0];
    long long best_cost = -1;
    for (int T : kAdjThreadChoices) {
        int per_sm = adj_ctas_per_sm(T);
        if (smem_per_sm > 0) per_sm = std::min<int>(per_sm, (int)((size_t)smem_per_sm / (smem + 1024)));
        per_sm = std::max(per_sm, 1);
        const long long slots = (long long)per_sm * std::max(n_sms, 1);
        const long long cost = ((n_robots + slots - 1) / slots) * (long long)((n_cap + T - 1) / T);
        if (best_cost < 0 || cost < best_cost) { best = T; best_cost = cost; }
    }
    return best;
}

}  // namespace
}  // namespace ms

using namespace ms;

struct msa_adjoint {
    ms_params p{};
    msb_voxel_spec spec{};
    cudaStream_t stream = nullptr;
    ms_allocator alloc{};
    bool custom_alloc = false;
    std::vector<std::pair<void *, size_t>> allocs;
    int n_robots = 0, K = 100, max_steps = 0, n_ckpt = 0, n_cap = 0, max_vox = 0;
    int threads = 0;                   // threads per robot (one of kAdjThreadChoices)
    int64_t n_masses = 0, n_voxels = 0, n_slots = 0;
    RobotDev *robots = nullptr;
    int2 *slot_range = nullptr;
    uint4 *slice = nullptr;
    int32_t *f_nbr = nullptr;
    float2 *f_kl = nullptr, *f_ab = nullptr, *scratch = nullptr, *sc = nullptr;
    float *f_c = nullptr, *vox_amp = nullptr;
    uint32_t *b_ent = nullptr, *vox_slots = nullptr;
    short4 *slot_vox = nullptr;
    float4 *st0 = nullptr, *ckpt = nullptr, *seg = nullptr, *seed = nullptr;
    float *phase = nullptr, *logk = nullptr, *loss = nullptr, *g_phase = nullptr, *g_logk = nullptr;
    long long *counter = nullptr;
    int *err = nullptr;
    size_t smem = 0;

    void *dev_alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *ptr = nullptr;
        if (custom_alloc) ptr = alloc.alloc(bytes, stream, alloc.ctx);
        else if (cudaMalloc(&ptr, bytes) != cudaSuccess) { cudaGetLastError(); ptr = nullptr; }
        if (ptr) allocs.push_back({ptr, bytes});
        return ptr;
    }
    void release()
    {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        for (auto &a : allocs) {
            if (custom_alloc) alloc.free(a.first, a.second, stream, alloc.ctx);
            else cudaFree(a.first);
        }
        allocs.clear();
    }
};

namespace {

#define MSA_CUDA_TRY(expr)                                                                     \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return fail(MS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));     \
    } while (0)

template <class T>
ms_status aupload(msa_adjoint *b, T **dst, const T *src, size_t count)
{
    *dst = (T *)b->dev_alloc(sizeof(T) * count);
    if (!*dst) return fail(MS_ERR_OOM, "device allocation failed");
    if (src && count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, b->stream);
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    return MS_OK;
}

}  // namespace

extern "C" {

ms_status msa_create(const ms_params *p, const msb_voxel_spec *spec, int32_t n_robots, const int32_t *dims,
                     const uint8_t *materials, int32_t checkpoint_every, int32_t max_steps,
                     const ms_allocator *alloc, void *stream, msa_adjoint **out)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !spec || !dims || !materials) return fail(MS_ERR_ARG, "p, spec, dims and materials are required");
    if (n_robots < 1 || checkpoint_every < 1 || max_steps < 1) return fail(MS_ERR_ARG, "n_robots, checkpoint_every and max_steps must be >= 1");
    if (!(p->dt > 0.f) || p->integrator != 0 || !(p->vel_damping >= 0.f && p->vel_damping < 1.f))
        return fail(MS_ERR_ARG, "bad step parameters");
    if (spec->n_materials < 1 || !spec->mat_k || !spec->mat_c || !spec->mat_amp) return fail(MS_ERR_ARG, "material table incomplete");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(MS_ERR_ARG, "allocator needs alloc and free");
    msa_adjoint *b = new (std::nothrow) msa_adjoint();
    if (!b) return fail(MS_ERR_OOM, "host allocation failed");
    struct Guard { msa_adjoint *b; ~Guard() { if (b) { b->release(); delete b; } } } guard{b};
    b->p = *p; b->spec = *spec; b->stream = (cudaStream_t)stream;
    if (alloc) { b->alloc = *alloc; b->custom_alloc = true; }
    b->n_robots = n_robots; b->K = checkpoint_every; b->max_steps = max_steps;

    VoxelBuild vb;
    ms_status st = build_voxels(spec, n_robots, dims, materials, nullptr, nullptr, true, vb);
    if (st != MS_OK) return st;
    std::vector<int2> ranges(n_robots);
    for (int r = 0; r < n_robots; ++r) {
        const RobotDev &R = vb.robots[r];
        if (R.n > kAdjMaxMasses) return fail(MS_ERR_ARG, "robot " + std::to_string(r) + " has more than 1024 masses");
        if (R.n_vox > kAdjMaxVoxels) return fail(MS_ERR_ARG, "robot " + std::to_string(r) + " has more than 4096 voxels");
        b->max_vox = std::max(b->max_vox, R.n_vox);
        const int first = (int)vb.slice[R.slice_base].x;
        const int end = r + 1 < n_robots ? (int)vb.slice[vb.robots[r + 1].slice_base].x : (int)vb.nbr.size();
        ranges[r] = make_int2(first, end);
    }
    b->n_cap = vb.max_n;
    b->n_masses = vb.n_masses;
    b->n_voxels = (int64_t)vb.vox_amp.size();
    b->n_slots = (int64_t)vb.nbr.size();
    b->n_ckpt = (max_steps + b->K - 1) / b->K;
    const size_t ck = (size_t)n_robots * b->n_ckpt * b->n_cap * 2, sg = (size_t)n_robots * b->K * b->n_cap * 3;
    if ((st = aupload(b, &b->robots, vb.robots.data(), vb.robots.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->slot_range, ranges.data(), ranges.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->slice, vb.slice.data(), vb.slice.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->f_nbr, vb.nbr.data(), vb.nbr.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->f_kl, vb.kl.data(), vb.kl.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->f_ab, vb.ab.data(), vb.ab.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->f_c, vb.c.data(), vb.c.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->b_ent, vb.bent.data(), vb.bent.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->slot_vox, vb.slot_vox.data(), vb.slot_vox.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->vox_slots, vb.vox_slots.data(), vb.vox_slots.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->vox_amp, vb.vox_amp.data(), vb.vox_amp.size())) != MS_OK) return st;
    if ((st = aupload(b, &b->st0, vb.st0.data(), vb.st0.size())) != MS_OK) return st;
    if ((st = aupload<float4>(b, &b->ckpt, nullptr, ck)) != MS_OK) return st;
    if ((st = aupload<float4>(b, &b->seg, nullptr, sg)) != MS_OK) return st;
    if ((st = aupload<float2>(b, &b->scratch, nullptr, vb.nbr.size())) != MS_OK) return st;
    if ((st = aupload<float2>(b, &b->sc, nullptr, max_steps)) != MS_OK) return st;
    if ((st = aupload<float4>(b, &b->seed, nullptr, vb.n_masses)) != MS_OK) return st;
    if ((st = aupload<float>(b, &b->phase, nullptr, b->n_voxels)) != MS_OK) return st;
    if ((st = aupload<float>(b, &b->logk, nullptr, b->n_voxels)) != MS_OK) return st;
    if ((st = aupload<float>(b, &b->g_phase, nullptr, b->n_voxels)) != MS_OK) return st;
    if ((st = aupload<float>(b, &b->g_logk, nullptr, b->n_voxels)) != MS_OK) return st;
    if ((st = aupload<float>(b, &b->loss, nullptr, n_robots)) != MS_OK) return st;
    if ((st = aupload<long long>(b, &b->counter, nullptr, 1)) != MS_OK) return st;
    if ((st = aupload<int>(b, &b->err, nullptr, 1)) != MS_OK) return st;
    MSA_CUDA_TRY(cudaMemsetAsync(b->err, 0, sizeof(int), b->stream));
    MSA_CUDA_TRY(cudaMemsetAsync(b->scratch, 0, sizeof(float2) * vb.nbr.size(), b->stream));
    b->smem = (size_t)b->n_cap * 6 * sizeof(float4) + (size_t)b->max_vox * 2 * sizeof(float);
    if (b->smem > 200 * 1024) return fail(MS_ERR_ARG, "a robot's adjoint state does not fit in shared memory");
    MSA_CUDA_TRY(cudaFuncSetAttribute(k_adjoint<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    MSA_CUDA_TRY(cudaFuncSetAttribute(k_adjoint<768>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    MSA_CUDA_TRY(cudaFuncSetAttribute(k_adjoint<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    MSA_CUDA_TRY(cudaFuncSetAttribute(k_adjoint<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    {
        int dev = 0, n_sms = 1, smem_sm = 0;
        MSA_CUDA_TRY(cudaGetDevice(&dev));
        MSA_CUDA_TRY(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
        MSA_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        b->threads = choose_threads(b->n_robots, b->n_cap, b->smem, n_sms, smem_sm);
    }
    MSA_CUDA_TRY(cudaStreamSynchronize(b->stream));
    guard.b = nullptr;
    *out = b;
    return MS_OK;
}

ms_status msa_gradients(msa_adjoint *b, int32_t nsteps, const float *phase, const float *logk,
                        const float *seed_x, float *loss, float *g_phase, float *g_logk, int32_t on_device)
{
    ms::Range range_("msa_gradients");
    if (!b || !phase || !logk || !loss || !g_phase || !g_logk) return fail(MS_ERR_ARG, "missing argument");
    if (nsteps < 1 || nsteps > b->max_steps) return fail(MS_ERR_ARG, "nsteps must be in [1, max_steps]");
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind outk = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!on_device) {
        for (int64_t v = 0; v < b->n_voxels; ++v)
            if (!std::isfinite(phase[v]) || !std::isfinite(logk[v])) return fail(MS_ERR_ARG, "non-finite phase or logk at voxel " + std::to_string(v));
    }
    MSA_CUDA_TRY(cudaMemcpyAsync(b->phase, phase, sizeof(float) * b->n_voxels, in, b->stream));
    MSA_CUDA_TRY(cudaMemcpyAsync(b->logk, logk, sizeof(float) * b->n_voxels, in, b->stream));
    const float4 *seed = nullptr;
    if (seed_x) {
        // (n,3) -> float4 via a strided 2-D copy
        MSA_CUDA_TRY(cudaMemsetAsync(b->seed, 0, sizeof(float4) * b->n_masses, b->stream));
        MSA_CUDA_TRY(cudaMemcpy2DAsync(b->seed, sizeof(float4), seed_x, 3 * sizeof(float), 3 * sizeof(float),
                                       b->n_masses, in, b->stream));
        seed = b->seed;
    }
    k_adj_merge<<<b->n_robots, 256, 0, b->stream>>>(b->slot_range, b->robots, b->slot_vox, b->phase, b->logk,
                                                   b->vox_amp, b->f_kl, b->f_ab);
    MSA_CUDA_TRY(cudaGetLastError());
    k_zero_counter<<<1, 1, 0, b->stream>>>(b->counter);
    MSA_CUDA_TRY(cudaGetLastError());
    launch_sc_table(b->counter, nsteps, (double)b->p.dt, 2.0 * M_PI * (double)b->spec.freq, b->sc, b->stream);
    MSA_CUDA_TRY(cudaGetLastError());
    AdjArgs a{};
    a.robots = b->robots; a.slot_range = b->slot_range;
    a.rec = Records{b->slice, b->f_nbr, b->f_kl, b->f_c, b->f_ab, b->b_ent, 0.f};
    a.slot_vox = b->slot_vox; a.vox_slots = b->vox_slots; a.vox_amp = b->vox_amp;
    a.phase = b->phase; a.logk = b->logk; a.st0 = b->st0; a.seed = seed;
    a.ckpt = b->ckpt; a.seg = b->seg; a.scratch = b->scratch; a.sc = b->sc;
    a.env = make_env(b->p);
    a.nsteps = nsteps; a.K = b->K; a.n_ckpt = b->n_ckpt; a.n_cap = b->n_cap;
    a.loss = b->loss; a.g_phase = b->g_phase; a.g_logk = b->g_logk; a.err = b->err;
    switch (b->threads) {
    case 1024: k_adjoint<1024><<<b->n_robots, 1024, b->smem, b->stream>>>(a); break;
    case 768: k_adjoint<768><<<b->n_robots, 768, b->smem, b->stream>>>(a); break;
    case 512: k_adjoint<512><<<b->n_robots, 512, b->smem, b->stream>>>(a); break;
    default: k_adjoint<256><<<b->n_robots, 256, b->smem, b->stream>>>(a); break;
    }
    MSA_CUDA_TRY(cudaGetLastError());
    MSA_CUDA_TRY(cudaMemcpyAsync(loss, b->loss, sizeof(float) * b->n_robots, outk, b->stream));
    MSA_CUDA_TRY(cudaMemcpyAsync(g_phase, b->g_phase, sizeof(float) * b->n_voxels, outk, b->stream));
    MSA_CUDA_TRY(cudaMemcpyAsync(g_logk, b->g_logk, sizeof(float) * b->n_voxels, outk, b->stream));
    if (!on_device) {
        MSA_CUDA_TRY(cudaStreamSynchronize(b->stream));
        int flag = 0;
        MSA_CUDA_TRY(cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return fail(MS_ERR_NONFINITE, "a rollout reached a non-finite state");
    }
    return MS_OK;
}

ms_status msa_set_threads(msa_adjoint *b, int32_t threads)
{
    if (!b) return fail(MS_ERR_ARG, "adjoint is NULL");
    if (threads != 1024 && threads != 768 && threads != 512 && threads != 256)
        return fail(MS_ERR_ARG, "threads per robot must be 256, 512, 768 or 1024");
    b->threads = threads;
    return MS_OK;
}

int32_t msa_threads(const msa_adjoint *b) { return b ? b->threads : 0; }

ms_status msa_sizes(const msa_adjoint *b, int64_t *n_voxels, int64_t *n_masses)
{
    if (!b) return fail(MS_ERR_ARG, "adjoint is NULL");
    if (n_voxels) *n_voxels = b->n_voxels;
    if (n_masses) *n_masses = b->n_masses;
    return MS_OK;
}

ms_status msa_destroy(msa_adjoint *b)
{
    if (!b) return MS_OK;
    b->release();
    delete b;
    return MS_OK;
}

}  // extern "C"
