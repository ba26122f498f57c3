// ms_cluster.cu -- the persistent multi-step kernel for small systems
// (kernel = 3): all steps of one ms_step call in ONE launch of a thread-block
// cluster, the system held entirely in shared memory.
//
// The system (at most kClusterMax x TM masses, internal Morton order) is cut
// into tiles of TM consecutive masses, one CTA of kClThreads threads per
// tile, all CTAs in one cluster (co-scheduled by the hardware).  TM is the
// smallest of 64, 128, 256, 512 that needs at most kClusterMax tiles, so the
// work of a step is spread over as many SMs as a cluster may hold.  Each mass
// has L = kClThreads / TM threads ("lanes"): lane l takes the mass's slots
// l, l + L, ...  Each CTA keeps in its own shared memory, for the whole call:
//   * the spring records of its masses, both directions, laid out so that
//     group g of the thread t's slots is entry g * kClThreads + t (a warp
//     reads 32 consecutive entries); the partner is coded by its mass index;
//   * the state of its masses, packed as (x, y, z, vx) and (vy, vz) in two
//     arrays (16- and 8-byte strides, so that gathers use every bank),
//     double buffered: step n reads buffer n & 1 and writes the other.
// A partner in another tile is read from that CTA's shared memory through
// distributed shared memory (mapa + ld.shared::cluster).  The only
// synchronisation is one cluster barrier per step, after which every CTA may
// read the new buffer and overwrite the old one.  The lanes' partial forces
// are combined by shuffles in a fixed order, then lane 0 integrates:
// symplectic Euler with gravity, external force, ground contact, Coulomb
// friction and global damping (the robot routines).
#include <cooperative_groups.h>

#include "ms_internal.h"
#include "ms_voxel.h"

namespace ms {
namespace {

namespace cg = cooperative_groups;

__device__ __forceinline__ uint32_t cl_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared::cluster address of the shared::cta address `a` in the CTA of rank r
__device__ __forceinline__ uint32_t cl_map(uint32_t a, uint32_t r)
{
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(r));
    return d;
}

__device__ __forceinline__ float4 cl_load4(uint32_t addr)
{
    float4 p;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(p.x), "=f"(p.y), "=f"(p.z), "=f"(p.w) : "r"(addr));
    return p;
}

__device__ __forceinline__ float2 cl_load2(uint32_t addr)
{
    float2 q;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(q.x), "=f"(q.y) : "r"(addr));
    return q;
}

// every thread of the cluster: writes before it are visible to reads after it
__device__ __forceinline__ void cl_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 1/sqrt(x), hardware approximation; x = 0 is handled by the caller
__device__ __forceinline__ float cl_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int TM, bool HAS_C, bool HAS_ACT, bool HAS_FEXT>
__global__ void __launch_bounds__(kClThreads) k_cluster(const ClusterArgs a)
{
    constexpr int L = kClThreads / TM;                // lanes per mass
    constexpr int TM_SHIFT = TM == 64 ? 6 : TM == 128 ? 7 : TM == 256 ? 8 : 9;
    static_assert((1 << TM_SHIFT) == TM && L * TM == kClThreads, "tile shape");
    extern __shared__ __align__(16) unsigned char dyn[];
    const uint32_t rank = cg::this_cluster().block_rank();
    const int tid = threadIdx.x;
    const int base = (int)rank * TM;
    const int nb = min(TM, a.N - base);
    const int groups = a.slots / L;
    float4 *sa = reinterpret_cast<float4 *>(dyn);                    // [2][TM]
    float2 *sb = reinterpret_cast<float2 *>(sa + 2 * TM);            // [2][TM]
    uint16_t *rn = reinterpret_cast<uint16_t *>(sb + 2 * TM);
    const int nrec = groups * kClThreads;
    float2 *rkl = reinterpret_cast<float2 *>(rn + ((nrec + 7) & ~7));
    float *rc = reinterpret_cast<float *>(rkl + nrec);
    float2 *rab = reinterpret_cast<float2 *>(rc + (HAS_C ? nrec : 0));

    // records of this tile, once per call (same layout as in global memory)
    const size_t off = (size_t)rank * (size_t)nrec;
    for (int e = tid; e < nrec; e += kClThreads) {
        rn[e] = __ldg(&a.nbr[off + e]);
        rkl[e] = __ldg(&a.kl[off + e]);
        if (HAS_C) rc[e] = __ldg(&a.c[off + e]);
        if (HAS_ACT) rab[e] = __ldg(&a.ab[off + e]);
    }
    const int mi = tid / L, lane = tid % L;         // this thread's mass and slot lane
    const bool owner = mi < nb;
    float w = 0.f;
    float4 fe = make_float4(0.f, 0.f, 0.f, 0.f);
    if (owner && lane == 0) {
        sa[mi] = a.sa[base + mi];
        sb[mi] = a.sb[base + mi];
        w = __ldg(&a.w[base + mi]);
        if (HAS_FEXT) fe = __ldg(&a.fext[base + mi]);
    }
    const uint32_t sa0 = cl_smem_addr(sa), sb0 = cl_smem_addr(sb);
    float2 sc_next = make_float2(0.f, 0.f);
    if (HAS_ACT) sc_next = __ldg(&a.sc[0]);
    cl_barrier();                                   // every tile's state is in place

    bool bad = false;
    for (int step = 0; step < a.nsteps; ++step) {
        const uint32_t cur = (uint32_t)step & 1u;
        const uint32_t cur_a = sa0 + cur * (uint32_t)(TM * 16), cur_b = sb0 + cur * (uint32_t)(TM * 8);
        const float2 scn = sc_next;                 // (sin, cos) of this step; the next one is fetched early
        if (HAS_ACT && step + 1 < a.nsteps) sc_next = __ldg(&a.sc[step + 1]);
        float fx = 0.f, fy = 0.f, fz = 0.f;
        float4 x = make_float4(0.f, 0.f, 0.f, w), v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (owner) {
            const float4 p = sa[cur * TM + mi];
            const float2 q = sb[cur * TM + mi];
            x = make_float4(p.x, p.y, p.z, w);
            v = make_float4(p.w, q.x, q.y, 0.f);
#pragma unroll 2
            for (int g = 0; g < groups; ++g) {
                const int e = g * kClThreads + tid;
                const uint32_t code = rn[e];
                const uint32_t pm = code & (TM - 1), pt = code >> TM_SHIFT;
                const float4 pa = cl_load4(cl_map(cur_a + (pm << 4), pt));
                const float2 pb = cl_load2(cl_map(cur_b + (pm << 3), pt));
                const float2 kl = rkl[e];
                float Lr = kl.y;
                if (HAS_ACT) { const float2 ab = rab[e]; Lr = Lr * (1.0f + fmaf(ab.x, scn.x, ab.y * scn.y)); }
                const float c = HAS_C ? rc[e] : a.c_uniform;
                // Hooke term of eq. 2 plus the axial dashpot, d = x_partner - x_self
                const float dx = pa.x - x.x, dy = pa.y - x.y, dz = pa.z - x.z;
                const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float il = cl_rsqrt(l2);
                const float l = l2 * il;
                const float rv = fmaf(pa.w - v.x, dx, fmaf(pb.x - v.y, dy, (pb.y - v.z) * dz)) * il;
                float fs = fmaf(kl.x, l - Lr, c * rv) * il;
                fs = (l2 > 0.0f) ? fs : 0.0f;
                fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
            }
        }
        // combine the lanes of each mass (fixed order: pairs, then pairs of pairs)
#pragma unroll
        for (int o = 1; o < L; o <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (owner && lane == 0) {
            robot_integrate(a.env, x, v, make_float4(fx + fe.x, fy + fe.y, fz + fe.z, 0.f));
            sa[(cur ^ 1u) * TM + mi] = make_float4(x.x, x.y, x.z, v.x);
            sb[(cur ^ 1u) * TM + mi] = make_float2(v.y, v.z);
            bad |= !isfinite(x.x + x.y + x.z + v.x + v.y + v.z);
        }
        cl_barrier();                               // the new state is complete in every tile
    }
    if (owner && lane == 0) {
        const uint32_t fin = (uint32_t)a.nsteps & 1u;
        a.sa[base + mi] = sa[fin * TM + mi];
        a.sb[base + mi] = sb[fin * TM + mi];
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(a.err, kErrNonFinite);
    cl_barrier();                                   // no CTA leaves while others may read its memory
}

}  // namespace

size_t cluster_smem_bytes(int tm, int slots, bool has_c, bool has_act)
{
    const size_t nrec = (size_t)slots * tm;
    return (size_t)tm * 48 + ((nrec + 7) & ~(size_t)7) * 2 + nrec * 8 + (has_c ? nrec * 4 : 0) +
           (has_act ? nrec * 8 : 0);
}

cudaError_t launch_cluster(const ClusterArgs &a, cudaStream_t st)
{
    if (a.N <= 0 || a.nsteps <= 0) return cudaSuccess;
    if (a.tm != 64 && a.tm != 128 && a.tm != 256 && a.tm != 512) return cudaErrorInvalidValue;
    const int tiles = (a.N + a.tm - 1) / a.tm;
    if (tiles > kClusterMax || a.slots % (kClThreads / a.tm) != 0) return cudaErrorInvalidValue;
    const bool hc = a.c != nullptr, ha = a.ab != nullptr, hf = a.fext != nullptr;
    const size_t smem = cluster_smem_bytes(a.tm, a.slots, hc, ha);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)tiles;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define MS_LAUNCH_CL(TM, C, A, F)                                                                    \
    do {                                                                                             \
        auto kfn = k_cluster<TM, C, A, F>;                                                           \
        cudaError_t e_ = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e_ == cudaSuccess && tiles > 8)                                                          \
            e_ = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);       \
        if (e_ != cudaSuccess) return e_;                                                            \
        return cudaLaunchKernelEx(&cfg, kfn, a);                                                     \
    } while (0)
#define MS_LAUNCH_CL_TM(TM)                                                                            \
    if (hc) {                                                                                        \
        if (ha) { if (hf) MS_LAUNCH_CL(TM, true, true, true); else MS_LAUNCH_CL(TM, true, true, false); }    \
        else    { if (hf) MS_LAUNCH_CL(TM, true, false, true); else MS_LAUNCH_CL(TM, true, false, false); }  \
    } else {                                                                                         \
        if (ha) { if (hf) MS_LAUNCH_CL(TM, false, true, true); else MS_LAUNCH_CL(TM, false, true, false); }  \
        else    { if (hf) MS_LAUNCH_CL(TM, false, false, true); else MS_LAUNCH_CL(TM, false, false, false); } \
    }
    switch (a.tm) {
        case 64: MS_LAUNCH_CL_TM(64) break;
        case 128: MS_LAUNCH_CL_TM(128) break;
        case 256: MS_LAUNCH_CL_TM(256) break;
        default: MS_LAUNCH_CL_TM(512) break;
    }
    return cudaErrorInvalidValue;
#undef MS_LAUNCH_CL_TM
#undef MS_LAUNCH_CL
}

}  // namespace ms
