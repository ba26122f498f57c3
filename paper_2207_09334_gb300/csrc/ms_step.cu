// ms_step.cu -- the explicit mass-spring step on sm_103a: three kernels over
// the same arithmetic (spring_term_packed, integrate_mass).
//   * k_step (gather layout, kernel = 1): one thread per mass, one launch per
//     time step (below).
//   * k_step_tiled (tiled layout, the default): one CTA per 512-mass tile
//     with its halo staged in shared memory and the spring rows streamed by
//     TMA bulk copies; one launch per time step.
//   * k_step_grid (tiled layout, kernel = 3 above the cluster kernel's size):
//     all steps of a call in one cooperative launch with a grid barrier.
//
// The gather kernel: each thread gathers every spring attached to its mass --
// the springs it owns from its own sliced-ELL row, the others through back
// references into the owners' rows -- evaluates eq. 2's Hooke term plus the
// axial dashpot with the partner's state at t_n, adds gravity, external force
// and ground contact, and integrates (symplectic Euler) into the other state
// buffer.
//
// This replaces Algorithm 1's two passes (spring pass appending forces to
// per-mass slots reserved with an integer atomicAdd, grid-wide sync, mass
// pass summing the slots) by a single fused mass-centric pass: the kernel
// boundary between steps is the grid-wide synchronisation, the per-mass sum
// happens in registers in a fixed order, and there are no atomics, so two
// runs are bit-identical.  Each spring force is evaluated by both endpoints;
// with d = x_partner - x_self the two evaluations are exact negatives of each
// other in IEEE arithmetic, so momentum balance is broken only by the
// rounding of each mass's own sum.
// The step is memory bound (about 30 flops per spring evaluation), so the
// design goal is to read every spring record from DRAM once: the partner's
// read of a record is a gather that normally hits L2 because owner and
// partner are close in the mass order.
#include "ms_internal.h"
#include "ms_device.cuh"

#include <atomic>

namespace ms {

template <bool HAS_C, bool HAS_ACT, bool HAS_FEXT, bool RK4>
__global__ void __launch_bounds__(256) k_step(const StepArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const unsigned lane = (unsigned)i & 31u;
    const uint4 meta = __ldg(&a.slice[i >> 5]);
    float4 xi, vi;
    load_mass(a.sa, a.sb, a.w, i, xi, vi);
    float fx = 0.f, fy = 0.f, fz = 0.f;

    // springs owned by this mass
    const unsigned flen = meta.z & 0xffffu, blen = meta.z >> 16;
    unsigned r = meta.x + lane;
#pragma unroll 2
    for (unsigned s = 0; s < flen; ++s, r += 32u) {
        int j = __ldg(&a.f_nbr[r]);
        j = (j < 0) ? i : j;               // padding slot: self, zero length
        const float2 kl = __ldg(&a.f_kl[r]);
        float L = kl.y;
        const float c = HAS_C ? __ldg(&a.f_c[r]) : a.c_uniform;
        if (HAS_ACT) { const float2 ab = __ldg(&a.f_ab[r]); L = L * (1.0f + fmaf(ab.x, a.s_n, ab.y * a.c_n)); }
        spring_term_packed(xi, vi, __ldg(&a.sa[j]), __ldg(&a.sb[j]), kl.x, L, c, fx, fy, fz);
    }
    // springs owned by partners, reached through back references
    unsigned q = meta.y + lane;
#pragma unroll 2
    for (unsigned s = 0; s < blen; ++s, q += 32u) {
        const uint32_t e = __ldg(&a.b_ent[q]);
        int o = i;
        unsigned rr = 0;
        if (e != kBackPad) {
            if (a.back_local) {            // robot-local form (populations stepped robot by robot)
                o = (int)(e & kRobotOwnerMask);
                rr = a.back_base + (e >> kRobotOwnerBits);
            } else {
                o = (int)(e & kOwnerMask);
                rr = __ldg(&a.slice[o >> 5].x) + (e >> kOwnerBits) * 32u + ((unsigned)o & 31u);
            }
        }
        const float2 kl = __ldg(&a.f_kl[rr]);
        float L = kl.y;
        const float c = HAS_C ? __ldg(&a.f_c[rr]) : a.c_uniform;
        if (HAS_ACT) { const float2 ab = __ldg(&a.f_ab[rr]); L = L * (1.0f + fmaf(ab.x, a.s_n, ab.y * a.c_n)); }
        spring_term_packed(xi, vi, __ldg(&a.sa[o]), __ldg(&a.sb[o]), kl.x, L, c, fx, fy, fz);
    }

    float4 xn, vn;
    integrate_mass<HAS_FEXT, RK4>(a, i, xi, vi, fx, fy, fz, xn, vn);
    store_mass(a, i, xn, vn);
}

// ---------------------------------------------------------------------------
// Tiled variant: one CTA per tile of kTileMasses consecutive masses (a
// compact block in Morton order).
//   * The CTA stages the state of its members and of their halo (every
//     outside partner, listed per tile) in shared memory; every partner read
//     is then a shared-memory read.
//   * Each mass's row holds all of its springs, with the partner as a 16-bit
//     tile-local index.  Rows are slot-major over the tile, so kTileGroup
//     slots of the whole tile are one contiguous range per array; they are
//     streamed into shared memory by TMA bulk copies (cp.async.bulk) through
//     a kTileStages-deep mbarrier pipeline, so DRAM stays busy while the
//     warps compute.  One elected thread issues the copies.
//   * Every wait on an mbarrier is bounded: after kMaxSpins polls the CTA
//     records kErrTimeout in the error flag and stops using the pipeline.
// ---------------------------------------------------------------------------
namespace {

template <bool HAS_C, bool HAS_ACT>
struct StageLayout {
    static constexpr uint32_t nbr = kTileGroup * kTileMasses * 2;
    static constexpr uint32_t kl = kTileGroup * kTileMasses * 8;
    static constexpr uint32_t c = HAS_C ? kTileGroup * kTileMasses * 4 : 0;
    static constexpr uint32_t ab = HAS_ACT ? kTileGroup * kTileMasses * 8 : 0;
    static constexpr uint32_t bytes = nbr + kl + c + ab;
};

}  // namespace

template <bool HAS_C, bool HAS_ACT, bool HAS_FEXT, bool RK4, int STAGES>
__global__ void __launch_bounds__(kTileMasses, STAGES == kTileStages ? 4 : 1) k_step_tiled(const StepArgs a)
{
    using SL = StageLayout<HAS_C, HAS_ACT>;
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ int give_up;
    const int tid = threadIdx.x;
    const int4 T = __ldg(&a.tiles[2 * blockIdx.x]);
    const int4 R = __ldg(&a.tiles[2 * blockIdx.x + 1]);
    const int base = T.x, nb = T.y, hoff = T.z, nh = T.w;
    const unsigned rec0 = (unsigned)R.x, nslots = (unsigned)R.y;
    const unsigned ngroups = (nslots + kTileGroup - 1) / kTileGroup;
    // shared partner state, packed: (x, y, z, vx) and (vy, vz) per tile-local mass
    float4 *spa = reinterpret_cast<float4 *>(dyn);
    float2 *spb = reinterpret_cast<float2 *>(spa + a.tile_local);
    unsigned char *stage0 = dyn + (((size_t)a.tile_local * 24 + 127) & ~(size_t)127);

    auto stage_ptr = [&](unsigned p) { return stage0 + (size_t)p * SL::bytes; };
    const uint64_t pol = l2_evict_first();
    auto issue = [&](unsigned g) {          // one thread: bulk-copy slot group g into its stage
        const unsigned p = g % STAGES;
        const unsigned s0 = g * kTileGroup;
        const unsigned ns = min((unsigned)kTileGroup, nslots - s0);
        const size_t first = (size_t)rec0 + (size_t)s0 * kTileMasses;
        const uint32_t cnt = ns * kTileMasses;
        unsigned char *st = stage_ptr(p);
        mbar_expect_tx(&bar[p], cnt * (2u + 8u + (HAS_C ? 4u : 0u) + (HAS_ACT ? 8u : 0u)));
        bulk_g2s(st, a.t_nbr + first, cnt * 2u, &bar[p], pol);
        bulk_g2s(st + SL::nbr, a.f_kl + first, cnt * 8u, &bar[p], pol);
        if (HAS_C) bulk_g2s(st + SL::nbr + SL::kl, a.f_c + first, cnt * 4u, &bar[p], pol);
        if (HAS_ACT) bulk_g2s(st + SL::nbr + SL::kl + SL::c, a.f_ab + first, cnt * 8u, &bar[p], pol);
    };

    if (tid == 0) {
        give_up = 0;
        for (int p = 0; p < STAGES; ++p) mbar_init(&bar[p], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0)
        for (unsigned g = 0; g < min(ngroups, (unsigned)STAGES); ++g) issue(g);

    // stage the state of the members and the halo while the first groups stream in
    const bool active = tid < nb;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f), vi = xi;
    if (active) {
        const float4 p = __ldg(&a.sa[base + tid]);
        const float2 q = __ldg(&a.sb[base + tid]);
        xi = make_float4(p.x, p.y, p.z, __ldg(&a.w[base + tid]));
        vi = make_float4(p.w, q.x, q.y, 0.f);
        spa[tid] = p;
        spb[tid] = q;
    }
    for (int h = tid; h < nh; h += kTileMasses) {
        const int g = __ldg(&a.halo[hoff + h]);
        spa[nb + h] = __ldg(&a.sa[g]);
        spb[nb + h] = __ldg(&a.sb[g]);
    }
    __syncthreads();
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (unsigned g = 0; g < ngroups; ++g) {
        const unsigned p = g % STAGES;
        const bool late = !mbar_wait(&bar[p], (g / STAGES) & 1u);
        if (late) give_up = 1;              // the stage never landed: its contents are not used
        const unsigned char *st = stage_ptr(p);
        const uint16_t *snbr = reinterpret_cast<const uint16_t *>(st);
        const float2 *skl = reinterpret_cast<const float2 *>(st + SL::nbr);
        const float *sc = reinterpret_cast<const float *>(st + SL::nbr + SL::kl);
        const float2 *sab = reinterpret_cast<const float2 *>(st + SL::nbr + SL::kl + SL::c);
        const unsigned ns = min((unsigned)kTileGroup, nslots - g * kTileGroup);
        if (active && !late) {
#pragma unroll
            for (unsigned u = 0; u < (unsigned)kTileGroup; ++u) {
                if (u < ns) {
                    const unsigned e = u * kTileMasses + tid;
                    const unsigned j = snbr[e];    // a padding slot points at the mass itself
                    const float2 kl = skl[e];
                    float L = kl.y;
                    const float c = HAS_C ? sc[e] : a.c_uniform;
                    if (HAS_ACT) { const float2 ab = sab[e]; L = L * (1.0f + fmaf(ab.x, a.s_n, ab.y * a.c_n)); }
                    spring_term_packed(xi, vi, spa[j], spb[j], kl.x, L, c, fx, fy, fz);
                }
            }
        }
        __syncthreads();                    // stage p fully consumed
        if (give_up) break;
        if (tid == 0 && g + STAGES < ngroups) {
            fence_proxy_async();
            issue(g + STAGES);
        }
    }
    if (give_up) {
        // a copy never completed: flag it, and give in-flight copies a bounded
        // chance to land before the CTA's shared memory is released
        if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            for (unsigned g = 0; g < ngroups && g < (unsigned)STAGES; ++g) mbar_wait(&bar[g], 0);
        }
        return;
    }
    if (!active) return;
    const int i = base + tid;
    float4 xn, vn;
    integrate_mass<HAS_FEXT, RK4>(a, i, xi, vi, fx, fy, fz, xn, vn);
    store_mass(a, i, xn, vn);
}

size_t tiled_smem_bytes(int tile_local, bool has_c, bool has_act, int stages)
{
    const size_t stage = (size_t)kTileGroup * kTileMasses * (2 + 8 + (has_c ? 4 : 0) + (has_act ? 8 : 0));
    return ((((size_t)tile_local * 24 + 127) & ~(size_t)127)) + (size_t)stages * stage;
}

// Opt a kernel in to the largest dynamic shared memory any tiled layout may
// need, once per device (a per-launch attribute call would cost more host
// time than a small system's step takes on the GPU).
template <class Kernel>
cudaError_t tiled_smem_opt_in(Kernel kfn, std::atomic<uint64_t> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmemMax);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

template <bool RK4>
cudaError_t launch_step_t(const StepArgs &a, cudaStream_t st)
{
    const bool hc = a.f_c != nullptr, ha = a.f_ab != nullptr, hf = a.fext != nullptr;
    if (a.tiled) {
        // A grid of at most one wave with few slot groups (small systems):
        // every group gets its own stage, so all bulk copies are issued at
        // once and their latencies overlap instead of adding up group by group.
        const bool deep = !RK4 && a.n_tiles <= a.n_sms && a.max_slots <= kTileGroup * kTileStagesDeep &&
                          tiled_smem_bytes(a.tile_local, hc, ha, kTileStagesDeep) <= kTileSmemMax;
        const int stages = deep ? kTileStagesDeep : kTileStages;
        const size_t smem = tiled_smem_bytes(a.tile_local, hc, ha, stages);
        const int grid = a.n_tiles;
#define MS_LAUNCH_TS(C, A, F, S)                                                                    \
    do {                                                                                            \
        static std::atomic<uint64_t> opted_in{0};                                                   \
        cudaError_t e_ = tiled_smem_opt_in(k_step_tiled<C, A, F, RK4, S>, opted_in);                \
        if (e_ != cudaSuccess) return e_;                                                           \
        k_step_tiled<C, A, F, RK4, S><<<grid, kTileMasses, smem, st>>>(a);                          \
    } while (0)
#define MS_LAUNCH_T(C, A, F)                                                                        \
    do {                                                                                            \
        if (!RK4 && deep) MS_LAUNCH_TS(C, A, F, (RK4 ? kTileStages : kTileStagesDeep));             \
        else MS_LAUNCH_TS(C, A, F, kTileStages);                                                    \
    } while (0)
        if (hc) {
            if (ha) { if (hf) MS_LAUNCH_T(true, true, true); else MS_LAUNCH_T(true, true, false); }
            else    { if (hf) MS_LAUNCH_T(true, false, true); else MS_LAUNCH_T(true, false, false); }
        } else {
            if (ha) { if (hf) MS_LAUNCH_T(false, true, true); else MS_LAUNCH_T(false, true, false); }
            else    { if (hf) MS_LAUNCH_T(false, false, true); else MS_LAUNCH_T(false, false, false); }
        }
#undef MS_LAUNCH_T
#undef MS_LAUNCH_TS
        return cudaGetLastError();
    }
    const int bs = 256;
    const int grid = (a.N + bs - 1) / bs;
#define MS_LAUNCH(C, A, F) k_step<C, A, F, RK4><<<grid, bs, 0, st>>>(a)
    if (hc) {
        if (ha) { if (hf) MS_LAUNCH(true, true, true); else MS_LAUNCH(true, true, false); }
        else    { if (hf) MS_LAUNCH(true, false, true); else MS_LAUNCH(true, false, false); }
    } else {
        if (ha) { if (hf) MS_LAUNCH(false, true, true); else MS_LAUNCH(false, true, false); }
        else    { if (hf) MS_LAUNCH(false, false, true); else MS_LAUNCH(false, false, false); }
    }
#undef MS_LAUNCH
    return cudaGetLastError();
}

// RK4 stages run their own instantiations, so the other schemes' kernels
// keep the register budget of the plain update.
cudaError_t launch_step(const StepArgs &a, cudaStream_t st)
{
    if (a.N <= 0) return cudaSuccess;
    return a.integrator == 3 ? launch_step_t<true>(a, st) : launch_step_t<false>(a, st);
}

// ---------------------------------------------------------------------------
// Persistent grid variant of the tiled step (kernel = 3 above the cluster
// kernel's size): all steps of one call in ONE cooperative launch, one CTA
// per tile and at most one wave of tiles, so every CTA is resident.  Each CTA
// loads its tile's spring records (and halo list) into shared memory once;
// per step it stages the halo's state from global memory (L2), evaluates its
// members' springs from shared memory, integrates, writes the new state to
// the other global buffer and meets the other CTAs at a grid barrier.  The
// members' own state stays in registers across steps.
// The barrier is a counter and a generation word in global memory; every
// wait on it is bounded (GridArgs::max_polls polls, 2^22 by default), after
// which the CTA records kErrTimeout and leaves its step loop.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// every CTA of the grid: global writes before it are visible after it (the
// CTA barrier orders its threads' stores before thread 0's fence, which then
// releases them with the arrival); false when the wait gave up
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks, unsigned max_polls,
                                             unsigned &my_gen, int *ok_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g0 = my_gen;
        bool ok = true;
        __threadfence();                                  // release this CTA's writes
        if (atomicAdd(count, 1u) + 1u == nblocks) {
            atomicExch(count, 0u);
            __threadfence();
            atomicExch(gen, g0 + 1u);
        } else {
            unsigned spins = 0;
            while (ld_acquire_gpu(gen) == g0) {
                if (++spins > max_polls) { ok = false; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        my_gen = g0 + 1u;
        *ok_sh = ok ? 1 : 0;
    }
    __syncthreads();
    return *ok_sh != 0;
}

}  // namespace

template <bool HAS_C, bool HAS_ACT, bool HAS_FEXT>
__global__ void __launch_bounds__(kTileMasses, 1) k_step_grid(const StepArgs a, const GridArgs gr)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ int ok_sh;
    const int tid = threadIdx.x;
    const int4 T = __ldg(&a.tiles[2 * blockIdx.x]);
    const int4 R = __ldg(&a.tiles[2 * blockIdx.x + 1]);
    const int base = T.x, nb = T.y, hoff = T.z, nh = T.w;
    const unsigned nrec = (unsigned)R.y * kTileMasses;
    float4 *spa = reinterpret_cast<float4 *>(dyn);
    float2 *spb = reinterpret_cast<float2 *>(spa + a.tile_local);
    int32_t *hidx = reinterpret_cast<int32_t *>(dyn + (((size_t)a.tile_local * 24 + 127) & ~(size_t)127));
    uint16_t *rn = reinterpret_cast<uint16_t *>(hidx + ((a.tile_local + 3) & ~3));
    float2 *rkl = reinterpret_cast<float2 *>(rn + ((nrec + 7) & ~7u));
    float *rc = reinterpret_cast<float *>(rkl + nrec);
    float2 *rab = reinterpret_cast<float2 *>(rc + (HAS_C ? nrec : 0));

    // once per call: the tile's records and halo list
    for (unsigned e = tid; e < nrec; e += kTileMasses) {
        const size_t r = (size_t)R.x + e;
        rn[e] = __ldg(&a.t_nbr[r]);
        rkl[e] = __ldg(&a.f_kl[r]);
        if (HAS_C) rc[e] = __ldg(&a.f_c[r]);
        if (HAS_ACT) rab[e] = __ldg(&a.f_ab[r]);
    }
    for (int h = tid; h < nh; h += kTileMasses) hidx[h] = __ldg(&a.halo[hoff + h]);
    const bool active = tid < nb;
    const int i = base + tid;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f), vi = xi;
    if (active) load_mass(gr.buf_a[0], gr.buf_b[0], a.w, i, xi, vi);
    unsigned my_gen = ld_acquire_gpu(gr.bar_gen);         // no CTA moves it before all have arrived once
    bool ok = true;
    for (int step = 0; step < gr.nsteps && ok; ++step) {
        const int cur = step & 1;
        // stage members (from registers) and halo (written by other CTAs, read
        // through L2); the grid barrier's CTA barriers ordered the previous
        // step's shared reads before these writes, and each thread reads back
        // only the halo indices it wrote itself
        if (active) { spa[tid] = make_float4(xi.x, xi.y, xi.z, vi.x); spb[tid] = make_float2(vi.y, vi.z); }
        for (int h = tid; h < nh; h += kTileMasses) {
            const int g = hidx[h];
            spa[nb + h] = __ldcg(&gr.buf_a[cur][g]);
            spb[nb + h] = __ldcg(&gr.buf_b[cur][g]);
        }
        __syncthreads();
        if (active) {
            float s_n = 0.f, c_n = 0.f;
            if (HAS_ACT) { const float2 t = __ldg(&gr.sc[step]); s_n = t.x; c_n = t.y; }
            float fx = 0.f, fy = 0.f, fz = 0.f;
            for (unsigned sl = 0; sl < (unsigned)R.y; ++sl) {
                const unsigned e = sl * kTileMasses + tid;
                const unsigned j = rn[e];                 // a padding slot points at the mass itself
                const float2 kl = rkl[e];
                float L = kl.y;
                const float c = HAS_C ? rc[e] : a.c_uniform;
                if (HAS_ACT) { const float2 ab = rab[e]; L = L * (1.0f + fmaf(ab.x, s_n, ab.y * c_n)); }
                spring_term_packed(xi, vi, spa[j], spb[j], kl.x, L, c, fx, fy, fz);
            }
            float4 xn, vn;
            integrate_mass<HAS_FEXT, false>(a, i, xi, vi, fx, fy, fz, xn, vn);
            gr.buf_a[cur ^ 1][i] = make_float4(xn.x, xn.y, xn.z, vn.x);
            gr.buf_b[cur ^ 1][i] = make_float2(vn.y, vn.z);
            xi = xn; vi = vn;
        }
        ok = grid_barrier(gr.bar_count, gr.bar_gen, gr.expected, gr.max_polls, my_gen, &ok_sh);
    }
    if (!ok && tid == 0) atomicOr(a.err, kErrTimeout);
}

size_t grid_smem_bytes(int tile_local, int slots, bool has_c, bool has_act)
{
    const size_t nrec = (size_t)slots * kTileMasses;
    return (((size_t)tile_local * 24 + 127) & ~(size_t)127) + (size_t)((tile_local + 3) & ~3) * 4 +
           ((nrec + 7) & ~(size_t)7) * 2 + nrec * 8 + (has_c ? nrec * 4 : 0) + (has_act ? nrec * 8 : 0);
}

cudaError_t launch_step_grid(const StepArgs &a, const GridArgs &gr, cudaStream_t st)
{
    if (a.N <= 0 || gr.nsteps <= 0) return cudaSuccess;
    if (!a.tiled || a.integrator != 0 || a.n_tiles > a.n_sms || gr.expected < (unsigned)a.n_tiles)
        return cudaErrorInvalidValue;
    const bool hc = a.f_c != nullptr, ha = a.f_ab != nullptr, hf = a.fext != nullptr;
    const size_t smem = grid_smem_bytes(a.tile_local, a.max_slots, hc, ha);
    if (smem > kTileSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(gr.bar_count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    StepArgs ac = a;
    GridArgs gc = gr;
    void *args[] = {&ac, &gc};
#define MS_LAUNCH_G(C, A, F)                                                                        \
    do {                                                                                            \
        auto kfn = k_step_grid<C, A, F>;                                                            \
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
        if (e != cudaSuccess) return e;                                                             \
        return cudaLaunchCooperativeKernel((const void *)kfn, dim3((unsigned)a.n_tiles), dim3(kTileMasses), args, smem, st); \
    } while (0)
    if (hc) {
        if (ha) { if (hf) MS_LAUNCH_G(true, true, true); else MS_LAUNCH_G(true, true, false); }
        else    { if (hf) MS_LAUNCH_G(true, false, true); else MS_LAUNCH_G(true, false, false); }
    } else {
        if (ha) { if (hf) MS_LAUNCH_G(false, true, true); else MS_LAUNCH_G(false, true, false); }
        else    { if (hf) MS_LAUNCH_G(false, false, true); else MS_LAUNCH_G(false, false, false); }
    }
#undef MS_LAUNCH_G
}


}  // namespace ms
