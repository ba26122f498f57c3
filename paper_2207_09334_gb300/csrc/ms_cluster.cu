// ms_cluster.cu -- the persistent multi-step kernel for small systems
// (kernel = 3): all steps of one ms_step call in ONE launch of a thread-block
// cluster, the system held entirely in shared memory.
//
// The system (at most kClusterMax x kClMasses masses, internal Morton order)
// is cut into tiles of kClMasses consecutive masses, one CTA per tile, all
// CTAs in one cluster (co-scheduled by the hardware).  Each CTA keeps in its
// own shared memory, for the whole call:
//   * the spring records of its masses, both directions (slot-major: record
//     s of member m at s * kClMasses + m; the partner coded as
//     (tile << 8) | member), loaded once;
//   * the state of its masses, packed (x, y, z, vx), (vy, vz), double
//     buffered: step n reads buffer n & 1 and writes the other.
// A partner in another tile is read straight from that CTA's shared memory
// (distributed shared memory, through the generic address of the remote
// buffer).  The only synchronisation is one cluster barrier per step, after
// which every CTA may read the new buffer and overwrite the old one.
// Each mass has kClLanes threads: lane l sums the springs of slots l,
// l + kClLanes, ..., and the lanes' partial forces are combined by shuffles in
// a fixed order, so a step's latency is a quarter of one thread walking every
// spring.  Integration is symplectic Euler with gravity, external force,
// ground contact, Coulomb friction and global damping (the robot routines).
#include <cooperative_groups.h>

#include "ms_internal.h"
#include "ms_voxel.h"

namespace ms {
namespace {

namespace cg = cooperative_groups;

constexpr int kClLanes = 4;                          // threads per mass
constexpr int kClThreads = kClMasses * kClLanes;

template <bool HAS_C, bool HAS_ACT, bool HAS_FEXT>
__global__ void __launch_bounds__(kClThreads) k_cluster(const ClusterArgs a)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ const float4 *rem_a[kClusterMax];   // buffer 0 of every CTA's state (generic addresses)
    __shared__ const float2 *rem_b[kClusterMax];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    const int base = rank * kClMasses;
    const int nb = min(kClMasses, a.N - base);
    const int slots = a.slots;
    float4 *sa = reinterpret_cast<float4 *>(dyn);                    // [2][kClMasses]
    float2 *sb = reinterpret_cast<float2 *>(sa + 2 * kClMasses);     // [2][kClMasses]
    uint16_t *rn = reinterpret_cast<uint16_t *>(sb + 2 * kClMasses);
    const size_t nrec = (size_t)slots * kClMasses;
    float2 *rkl = reinterpret_cast<float2 *>(rn + ((nrec + 7) & ~(size_t)7));
    float *rc = reinterpret_cast<float *>(rkl + nrec);
    float2 *rab = reinterpret_cast<float2 *>(rc + (HAS_C ? nrec : 0));

    // records of this tile, once per call
    const size_t off = (size_t)rank * nrec;
    for (size_t e = tid; e < nrec; e += kClThreads) {
        rn[e] = __ldg(&a.nbr[off + e]);
        rkl[e] = __ldg(&a.kl[off + e]);
        if (HAS_C) rc[e] = __ldg(&a.c[off + e]);
        if (HAS_ACT) rab[e] = __ldg(&a.ab[off + e]);
    }
    const int mi = tid / kClLanes, lane = tid % kClLanes;  // this thread's mass and slot lane
    const bool owner = mi < nb;
    float w = 0.f;
    float4 fe = make_float4(0.f, 0.f, 0.f, 0.f);
    if (owner && lane == 0) {
        sa[mi] = a.sa[base + mi];
        sb[mi] = a.sb[base + mi];
        w = __ldg(&a.w[base + mi]);
        if (HAS_FEXT) fe = __ldg(&a.fext[base + mi]);
    }
    if (tid < (int)cl.num_blocks()) {
        rem_a[tid] = cl.map_shared_rank(sa, tid);
        rem_b[tid] = cl.map_shared_rank(sb, tid);
    }
    cl.sync();                                      // every tile's state is in place

    bool bad = false;
    for (int step = 0; step < a.nsteps; ++step) {
        const unsigned cur = (unsigned)step & 1u;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        float4 x = make_float4(0.f, 0.f, 0.f, w), v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (owner) {
            const float4 p = sa[cur * kClMasses + mi];
            const float2 q = sb[cur * kClMasses + mi];
            x = make_float4(p.x, p.y, p.z, w);
            v = make_float4(p.w, q.x, q.y, 0.f);
            float s_n = 0.f, c_n = 0.f;
            if (HAS_ACT) { const float2 t = __ldg(&a.sc[step]); s_n = t.x; c_n = t.y; }
#pragma unroll 2
            for (int s = lane; s < slots; s += kClLanes) {
                const unsigned e = (unsigned)s * kClMasses + mi;
                const unsigned code = rn[e];
                const unsigned pt = code >> 8, pm = cur * kClMasses + (code & 0xffu);
                const float4 pa = rem_a[pt][pm];
                const float2 pb = rem_b[pt][pm];
                const float2 kl = rkl[e];
                float L = kl.y;
                if (HAS_ACT) { const float2 ab = rab[e]; L = L * (1.0f + (ab.x * s_n + ab.y * c_n)); }
                const float c = HAS_C ? rc[e] : a.c_uniform;
                // Hooke term of eq. 2 plus the axial dashpot, d = x_partner - x_self
                const float dx = pa.x - x.x, dy = pa.y - x.y, dz = pa.z - x.z;
                const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float il = rsqrtf(l2);
                const float l = l2 * il;
                const float rv = fmaf(pa.w - v.x, dx, fmaf(pb.x - v.y, dy, (pb.y - v.z) * dz)) * il;
                float fs = fmaf(kl.x, l - L, c * rv) * il;
                fs = (l2 > 0.0f) ? fs : 0.0f;
                fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
            }
        }
        // combine the lanes of each mass (fixed order: pairs, then pairs of pairs)
#pragma unroll
        for (int o = 1; o < kClLanes; o <<= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (owner && lane == 0) {
            robot_integrate(a.env, x, v, make_float4(fx + fe.x, fy + fe.y, fz + fe.z, 0.f));
            sa[(cur ^ 1u) * kClMasses + mi] = make_float4(x.x, x.y, x.z, v.x);
            sb[(cur ^ 1u) * kClMasses + mi] = make_float2(v.y, v.z);
            bad |= !isfinite(x.x + x.y + x.z + v.x + v.y + v.z);
        }
        cl.sync();                                  // the new state is complete in every tile
    }
    if (owner && lane == 0) {
        const unsigned fin = (unsigned)a.nsteps & 1u;
        a.sa[base + mi] = sa[fin * kClMasses + mi];
        a.sb[base + mi] = sb[fin * kClMasses + mi];
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(a.err, kErrNonFinite);
    cl.sync();                                      // no CTA leaves while others may read its memory
}

}  // namespace

size_t cluster_smem_bytes(int slots, bool has_c, bool has_act)
{
    const size_t nrec = (size_t)slots * kClMasses;
    return (size_t)2 * kClMasses * (16 + 8) + ((nrec + 7) & ~(size_t)7) * 2 + nrec * 8 + (has_c ? nrec * 4 : 0) +
           (has_act ? nrec * 8 : 0);
}

cudaError_t launch_cluster(const ClusterArgs &a, cudaStream_t st)
{
    if (a.N <= 0 || a.nsteps <= 0) return cudaSuccess;
    const int tiles = (a.N + kClMasses - 1) / kClMasses;
    if (tiles > kClusterMax) return cudaErrorInvalidValue;
    const bool hc = a.c != nullptr, ha = a.ab != nullptr, hf = a.fext != nullptr;
    const size_t smem = cluster_smem_bytes(a.slots, hc, ha);
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
#define MS_LAUNCH_CL(C, A, F)                                                                        \
    do {                                                                                             \
        auto kfn = k_cluster<C, A, F>;                                                               \
        cudaError_t e_ = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e_ == cudaSuccess && tiles > 8)                                                          \
            e_ = cudaFuncSetAttribute(kfn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);       \
        if (e_ != cudaSuccess) return e_;                                                            \
        return cudaLaunchKernelEx(&cfg, kfn, a);                                                     \
    } while (0)
    if (hc) {
        if (ha) { if (hf) MS_LAUNCH_CL(true, true, true); else MS_LAUNCH_CL(true, true, false); }
        else    { if (hf) MS_LAUNCH_CL(true, false, true); else MS_LAUNCH_CL(true, false, false); }
    } else {
        if (ha) { if (hf) MS_LAUNCH_CL(false, true, true); else MS_LAUNCH_CL(false, true, false); }
        else    { if (hf) MS_LAUNCH_CL(false, false, true); else MS_LAUNCH_CL(false, false, false); }
    }
#undef MS_LAUNCH_CL
}

}  // namespace ms
