// ms_lattice.cu -- the explicit step on the lattice layout (kernel 4).
//
// For a box lattice with 26-neighbourhood springs (the benchmark's
// throughput lattice; the paper's voxel and cubic lattices of "Generating a
// Lattice"), the topology and the rest lengths follow from the lattice
// itself, so the step reads per spring only its stiffness.  That is a
// quarter of the spring bytes of the general (tiled) layout, which stores
// partner indices and rest lengths and lists every spring at both masses.
//
// Bricks of 16 x 16 x 8 cells; 1024 threads per brick, each thread two cells
// stacked in z (a at z, b at z + 1):
//   * the state of the brick and of its one-cell halo (18 x 18 x 10 cells) is
//     staged in shared memory; a partner in direction d is then the shared
//     entry at a constant offset, with no index stored anywhere;
//   * the CTAs are persistent (one per multiprocessor: two stages of 76 KB;
//     a brick of this size stages 1.58 cells per cell, against 1.76 for
//     16 x 8 x 8 bricks at two CTAs per multiprocessor) and walk the bricks
//     in raster order through two shared buffers: two TMA tensor copies
//     (completing on the buffer's mbarrier) stage a brick's block, and a TMA
//     prefetch brings its stiffness into L2.  There is no block-wide barrier
//     between bricks: a warp done with brick n goes on to brick n + 1 (staged
//     in the other buffer), and the last warp done with brick n issues brick
//     n + 2 into the freed buffer, so the warps drift apart by up to a brick
//     and one warp's loads overlap another's arithmetic;
//   * a thread walks the 3 x 3 columns around its pair and reads the four
//     cells z - 1 .. z + 2 of each column once: they are partners of a (z - 1
//     .. z + 1) and of b (z .. z + 2), so each shared-memory read of a partner
//     state serves both cells (the shared-memory pipe, not DRAM, bounds a
//     one-cell-per-thread form), and the spring between a and b is evaluated
//     once;
//   * each spring term is eq. 2's Hooke term plus the axial dashpot (reading
//     R2), written as f = s d, s = k + (c (dv . d)/l - k L)/l, with one
//     hardware reciprocal square root; k comes from the cell's own array for a
//     forward direction and from the partner's (kb[d][i] = kf[d][i - off(d)])
//     for a backward one; an actuated lattice (ACT) reads the spring's
//     (alpha, beta) the same way and uses L (1 + alpha sin + beta cos) of the
//     step's 2 pi f t (reading R3).  A cell without a mass sits at a far sentinel
//     position with k = 0 on its springs, so its terms vanish exactly; only a
//     lattice where some neighbouring masses lack a spring (k = NaN there)
//     runs the variant that tests each term (GUARD);
//   * then gravity, external force, ground contact, damping and the update of
//     both masses (integrate_mass, shared with the other step kernels); the
//     new state goes to the other buffer (Algorithm 1's synchronisation is
//     the kernel boundary).
// Each mass sums its springs in a fixed order, so runs are bit-reproducible.
#include <cudaTypedefs.h>

#include "ms_internal.h"
#include "ms_device.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

namespace ms {
namespace {

// shared-memory offset of the cell (dx, dy, dz) away inside the staged block
__host__ __device__ constexpr int halo_off(int dx, int dy, int dz) { return dx + kHaloX * (dy + kHaloY * dz); }

// forward direction index of (dx, dy, dz) (lat_dx/dy/dz), or -1 for a backward one
__host__ __device__ constexpr int fwd_index(int dx, int dy, int dz)
{
    return dz == 1 ? 4 + (dx + 1) + 3 * (dy + 1)
         : (dz == 0 && dy == 1) ? dx + 2
         : (dz == 0 && dy == 0 && dx == 1) ? 0
         : -1;
}

// k of the spring of cell i in direction (dx, dy, dz): from the cell's own
// array for a forward direction, from the partner's for a backward one
template <int DX, int DY, int DZ>
__device__ __forceinline__ float spring_k(const LatticeArgs &g, int i)
{
    constexpr int f = fwd_index(DX, DY, DZ);
    constexpr int b = fwd_index(-DX, -DY, -DZ);
    if constexpr (f >= 0) return __ldg(g.kf[f] + i);
    else return __ldg(g.kb[b] + i);
}

// rest length of the spring of cell i in direction (dx, dy, dz): the
// direction's L, actuated (ACT) by the spring's (alpha, beta) at the step's
// (sin, cos)(2 pi f t) = (s_n, c_n), read like k
template <bool ACT, int DX, int DY, int DZ>
__device__ __forceinline__ float spring_L(const LatticeArgs &g, int i, float s_n, float c_n)
{
    constexpr int f = fwd_index(DX, DY, DZ);
    constexpr int b = fwd_index(-DX, -DY, -DZ);
    const float L = g.L[f >= 0 ? f : b];
    if constexpr (!ACT) {
        return L;
    } else if constexpr (f >= 0) {
        const float2 ab = __ldg(g.abf[f] + i);
        return L * (1.0f + fmaf(ab.x, s_n, ab.y * c_n));
    } else {
        const float2 ab = __ldg(g.abb[b] + i);
        return L * (1.0f + fmaf(ab.x, s_n, ab.y * c_n));
    }
}

// Magnitude s of the spring term f = s d on the mass at (xi, vi) from the
// partner (pa, pb) = ((x, y, z, vx), (vy, vz)), d = x_partner - x_self:
//   s = k (l - L)/l + c (v_partner - v_self) . d / l^2 = k + (c dv.d / l - k L) / l.
// A partner without a mass (at kLatEmptyPos, k = 0) gives l^2 = +inf, 1/l = 0
// and s = 0.  A spring of zero length adds nothing: GUARD turns its NaN into
// 0 (as it does for k = NaN, a missing spring between two masses); without
// GUARD, 1e-30 is added into l^2 (in the FMA that forms dz^2, so it costs no
// instruction and leaves any l^2 above about 1e-22 as it was, up to the
// rounding of an exact tie), s stays finite and d = 0.
constexpr float kLatMinL2 = 1e-30f;

// A mass as the spring terms use it: the negated pairs (-x, -y), (-z, -vx) and
// (-vy, -vz).  A partner's state arrives from shared memory as the register
// pairs (x, y), (z, vx) of one 16-byte load and (vy, vz) of one 8-byte load,
// so each pair of differences is one packed FP32x2 add (sm_100 and later),
// rounded as the two scalar subtractions would be.  The force accumulates as
// (fx, fy) in one packed FMA and fz.
struct Own { float2 nxy, nzv, nvyz; };
struct Force { float2 xy; float z; };

__device__ __forceinline__ Own own_of(const float4 x, const float3 v)
{
    return {make_float2(-x.x, -x.y), make_float2(-x.z, -v.x), make_float2(-v.y, -v.z)};
}

template <bool GUARD>
__device__ __forceinline__ float lattice_term(const Own &o, const float4 pa, const float2 pb, float k, float L,
                                              float c, float2 &dxy, float &dz)
{
    dxy = __fadd2_rn(make_float2(pa.x, pa.y), o.nxy);
    const float2 zv = __fadd2_rn(make_float2(pa.z, pa.w), o.nzv);       // (dz, dvx)
    const float2 vyz = __fadd2_rn(pb, o.nvyz);                          // (dvy, dvz)
    dz = zv.x;
    const float l2 = fmaf(dxy.x, dxy.x, fmaf(dxy.y, dxy.y, GUARD ? dz * dz : fmaf(dz, dz, kLatMinL2)));
    const float il = rsqrt_hw(l2);
    const float dot = fmaf(zv.y, dxy.x, fmaf(vyz.x, dxy.y, vyz.y * dz));
    const float s = fmaf(fmaf(c * dot, il, -(k * L)), il, k);
    if (GUARD) return s == s ? s : 0.0f;
    return s;
}

template <bool GUARD>
__device__ __forceinline__ void add_term(const Own &o, const float4 pa, const float2 pb, float k, float L, float c,
                                         Force &F)
{
    float2 dxy;
    float dz;
    const float s = lattice_term<GUARD>(o, pa, pb, k, L, c, dxy, dz);
    F.xy = __ffma2_rn(make_float2(s, s), dxy, F.xy);
    F.z = fmaf(s, dz, F.z);
}

// Springs of the pair (a at z, b at z + 1) into the column (DX, DY): partner
// cells z - 1 .. z + 2 read once each.  The centre column (0, 0) holds a and b
// themselves: a's spring to z - 1, the a-b spring once, b's spring to z + 2.
template <bool GUARD, bool ACT, int DX, int DY>
__device__ __forceinline__ void column(const LatticeArgs &g, const float4 *spa, const float2 *spb, int sa_, int ia,
                                       int ib, const Own &oa, const Own &ob, float s_n, float c_n, Force &Fa,
                                       Force &Fb)
{
    const int c0 = sa_ + halo_off(DX, DY, 0);
    const float c = g.c;
    {   // z - 1: a only
        const float4 p = spa[c0 - halo_off(0, 0, 1)];
        const float2 q = spb[c0 - halo_off(0, 0, 1)];
        add_term<GUARD>(oa, p, q, spring_k<DX, DY, -1>(g, ia), spring_L<ACT, DX, DY, -1>(g, ia, s_n, c_n), c, Fa);
    }
    if constexpr (DX != 0 || DY != 0) {
        {   // z: a in-plane, b one below
            const float4 p = spa[c0];
            const float2 q = spb[c0];
            add_term<GUARD>(oa, p, q, spring_k<DX, DY, 0>(g, ia), spring_L<ACT, DX, DY, 0>(g, ia, s_n, c_n), c, Fa);
            add_term<GUARD>(ob, p, q, spring_k<DX, DY, -1>(g, ib), spring_L<ACT, DX, DY, -1>(g, ib, s_n, c_n), c, Fb);
        }
        {   // z + 1: a one above, b in-plane
            const float4 p = spa[c0 + halo_off(0, 0, 1)];
            const float2 q = spb[c0 + halo_off(0, 0, 1)];
            add_term<GUARD>(oa, p, q, spring_k<DX, DY, 1>(g, ia), spring_L<ACT, DX, DY, 1>(g, ia, s_n, c_n), c, Fa);
            add_term<GUARD>(ob, p, q, spring_k<DX, DY, 0>(g, ib), spring_L<ACT, DX, DY, 0>(g, ib, s_n, c_n), c, Fb);
        }
    } else {
        // the a-b spring, once: +s d on a, -s d on b
        float2 dxy;
        float dz;
        const float s = lattice_term<GUARD>(oa, spa[c0 + halo_off(0, 0, 1)], spb[c0 + halo_off(0, 0, 1)],
                                            __ldg(g.kf[fwd_index(0, 0, 1)] + ia),
                                            spring_L<ACT, 0, 0, 1>(g, ia, s_n, c_n), c, dxy, dz);
        Fa.xy = __ffma2_rn(make_float2(s, s), dxy, Fa.xy);
        Fa.z = fmaf(s, dz, Fa.z);
        Fb.xy = __ffma2_rn(make_float2(-s, -s), dxy, Fb.xy);
        Fb.z = fmaf(-s, dz, Fb.z);
    }
    {   // z + 2: b only
        const float4 p = spa[c0 + halo_off(0, 0, 2)];
        const float2 q = spb[c0 + halo_off(0, 0, 2)];
        add_term<GUARD>(ob, p, q, spring_k<DX, DY, 1>(g, ib), spring_L<ACT, DX, DY, 1>(g, ib, s_n, c_n), c, Fb);
    }
}

// all springs of the pair (a, b), column by column
template <bool GUARD, bool ACT>
__device__ __forceinline__ void pair_forces(const LatticeArgs &g, const float4 *spa, const float2 *spb, int s0, int ia,
                                            int ib, const Own &oa, const Own &ob, float s_n, float c_n,
                                            float3 &Fa3, float3 &Fb3)
{
    Force Fa{make_float2(0.f, 0.f), 0.f}, Fb = Fa;
    column<GUARD, ACT, -1, -1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  0, -1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  1, -1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT, -1,  0>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  0,  0>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  1,  0>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT, -1,  1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  0,  1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    column<GUARD, ACT,  1,  1>(g, spa, spb, s0, ia, ib, oa, ob, s_n, c_n, Fa, Fb);
    Fa3 = make_float3(Fa.xy.x, Fa.xy.y, Fa.z);
    Fb3 = make_float3(Fb.xy.x, Fb.xy.y, Fb.z);
}

// one staged block: (x, y, z, vx) then (vy, vz) of the 18 x 18 x 10 cells
constexpr uint32_t kStageA = kHaloCells * sizeof(float4);       // 51 840 bytes (a multiple of 128)
constexpr uint32_t kStageB = kHaloCells * sizeof(float2);       // 25 920 bytes
constexpr uint32_t kStageCopied = kStageA + kStageB;            // bytes the two copies of a stage bring
constexpr uint32_t kStageBytes = (kStageCopied + 127) / 128 * 128;   // stage stride: copies land 128-byte aligned
static_assert(kStageA % 128 == 0 && kStageBytes % 128 == 0, "tensor copies need 128-byte aligned destinations");
constexpr int kLatCtasPerSm = 1;
constexpr int kLatWarps = kLatThreads / 32;

template <bool HAS_FEXT, bool RK4, bool GUARD, bool ACT>
__global__ void __launch_bounds__(kLatThreads, kLatCtasPerSm)
k_step_lattice(const StepArgs a, const LatticeArgs g, const __grid_constant__ CUtensorMap map_a,
               const __grid_constant__ CUtensorMap map_b, const __grid_constant__ CUtensorMap map_k)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int done[2];                       // warps done with each buffer, over all its uses
    __shared__ int issued[2];                     // copies issued into each buffer
    __shared__ int give_up;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nbricks = g.nbx * g.nby * g.nbz;
    const int XY = g.X * g.Y;
    // brick b: its staged block starts at padded cell (bx kBrickX, by kBrickY, bz kBrickZ)
    auto origin = [&](int b, int &ox, int &oy, int &oz) {
        const int bx = b % g.nbx, byz = b / g.nbx;
        ox = bx * kBrickX; oy = (byz % g.nby) * kBrickY; oz = (byz / g.nby) * kBrickZ;
    };
    auto issue = [&](int b, int stage) {          // one thread: stage brick b, prefetch its stiffness
        int ox, oy, oz;
        origin(b, ox, oy, oz);
        unsigned char *dst = dyn + (size_t)stage * kStageBytes;
        mbar_expect_tx(&bar[stage], kStageCopied);
        tma_load_4d(dst, &map_a, 0, ox, oy, oz, &bar[stage]);
        tma_load_3d(dst + kStageA, &map_b, ox, oy, oz, &bar[stage]);
        tma_prefetch_4d(&map_k, ox, oy, oz, 0);
        ++issued[stage];
    };
    if (tid == 0) {
        give_up = 0;
        done[0] = done[1] = 0;
        issued[0] = issued[1] = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        if ((int)blockIdx.x < nbricks) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < nbricks) issue(blockIdx.x + gridDim.x, 1);
    }
    __syncthreads();
    const int cx = tid % kBrickX, cy = (tid / kBrickX) % kBrickY, cz = 2 * (tid / (kBrickX * kBrickY));
    const int s0 = (cx + 1) + kHaloX * ((cy + 1) + kHaloY * (cz + 1));     // cell a; b is one layer up
    int n = 0;
    // No block-wide barrier between bricks: a warp that is done with brick n
    // goes on to brick n + 1 (already staged in the other buffer), and the last
    // warp done with brick n refills its buffer with brick n + 2, so the warps
    // drift apart by up to a brick and their load and arithmetic phases overlap.
    for (int b = blockIdx.x; b < nbricks; b += gridDim.x, ++n) {
        const int stage = n & 1;
        int ox, oy, oz;
        origin(b, ox, oy, oz);
        const int ia = (ox + cx + 1) + g.X * (oy + cy + 1) + XY * (oz + cz + 1), ib = ia + XY;
        const float wa = __ldg(&a.w[ia]), wb = __ldg(&a.w[ib]);
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[stage], (n >> 1) & 1))) {   // warp-uniform
            if (lane == 0) give_up = 1;
            break;
        }
        const float4 *spa = reinterpret_cast<const float4 *>(dyn + (size_t)stage * kStageBytes);
        const float2 *spb = reinterpret_cast<const float2 *>(dyn + (size_t)stage * kStageBytes + kStageA);
        if (wa == wa || wb == wb) {
            // the pair's own states, negated (Own); the integration takes them back
            // from there (negation is exact), so no second copy stays live
            const float4 p = spa[s0];
            const float2 q = spb[s0];
            const float4 r = spa[s0 + halo_off(0, 0, 1)];
            const float2 t = spb[s0 + halo_off(0, 0, 1)];
            const Own oa = own_of(p, make_float3(p.w, q.x, q.y)), ob = own_of(r, make_float3(r.w, t.x, t.y));
            float3 Fa, Fb;
            pair_forces<GUARD, ACT>(g, spa, spb, s0, ia, ib, oa, ob, a.s_n, a.c_n, Fa, Fb);
            float4 xn, vn;
            if (wa == wa) {
                integrate_mass<HAS_FEXT, RK4>(a, ia, make_float4(-oa.nxy.x, -oa.nxy.y, -oa.nzv.x, wa),
                                              make_float4(-oa.nzv.y, -oa.nvyz.x, -oa.nvyz.y, 0.f), Fa.x, Fa.y, Fa.z,
                                              xn, vn);
                store_mass(a, ia, xn, vn);
            }
            if (wb == wb) {
                integrate_mass<HAS_FEXT, RK4>(a, ib, make_float4(-ob.nxy.x, -ob.nxy.y, -ob.nzv.x, wb),
                                              make_float4(-ob.nzv.y, -ob.nvyz.x, -ob.nvyz.y, 0.f), Fb.x, Fb.y, Fb.z,
                                              xn, vn);
                store_mass(a, ib, xn, vn);
            }
        }
        // this warp's reads of the buffer are done; the last warp refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int prev = atomicAdd(&done[stage], 1);
            if ((prev + 1) % kLatWarps == 0) {
                __threadfence_block();
                const int nb = b + 2 * (int)gridDim.x;
                if (nb < nbricks) {
                    fence_proxy_async();
                    issue(nb, stage);
                }
            }
        }
    }
    __syncthreads();
    if (give_up && tid == 0) {
        // a stage never landed: flag it, and give the copies still in flight a
        // bounded chance to land before the shared memory is released
        atomicOr(a.err, kErrTimeout);
        for (int st = 0; st < 2; ++st)
            if (issued[st] > 0) mbar_wait(&bar[st], (issued[st] - 1) & 1);
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

ms_status encode(CUtensorMap *map, CUtensorMapDataType type, int rank, const void *ptr, const cuuint64_t *dims,
                 const cuuint64_t *strides, const cuuint32_t *box)
{
    auto fn = tensor_map_encoder();
    if (!fn) return fail(MS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((uintptr_t)ptr & 15) return fail(MS_ERR_CUDA, "lattice tensor map: base not 16-byte aligned");
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(map, type, (cuuint32_t)rank, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return MS_OK;
}

}  // namespace

ms_status lattice_maps_add(LatticeMaps &m, const LatticeArgs &g, const float4 *sa, const float2 *sb)
{
    const cuuint64_t X = (cuuint64_t)g.X, Y = (cuuint64_t)g.Y, Z = (cuuint64_t)g.Z;
    ms_status st;
    if (m.n == 0) {
        // the 13 stiffness arrays, one allocation P floats apart: (x, y, z, d);
        // prefetch box = the cells whose k a brick reads, every direction
        const cuuint64_t dims[4] = {X, Y, Z, (cuuint64_t)kLatDirs};
        const cuuint64_t strides[3] = {X * 4, X * Y * 4, X * Y * Z * 4};
        // x rounded up to 16 bytes; z from one below the brick to its top layer
        // (a spring's k is read at its lower-or-equal end, never above the brick)
        const cuuint32_t box[4] = {kHaloX + 2, kHaloY, kBrickZ + 1, (cuuint32_t)kLatDirs};
        if ((st = encode(&m.k, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.kf[0], dims, strides, box)) != MS_OK) return st;
    }
    if (m.n >= LatticeMaps::kMax) return fail(MS_ERR_ARG, "too many lattice state buffers");
    {   // (x, y, z, vx): 4 floats per cell
        const cuuint64_t dims[4] = {4, X, Y, Z};
        const cuuint64_t strides[3] = {16, X * 16, X * Y * 16};
        const cuuint32_t box[4] = {4, kHaloX, kHaloY, kHaloZ};
        if ((st = encode(&m.a[m.n], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, sa, dims, strides, box)) != MS_OK) return st;
    }
    {   // (vy, vz): one 8-byte element per cell (copied verbatim)
        const cuuint64_t dims[3] = {X, Y, Z};
        const cuuint64_t strides[2] = {X * 8, X * Y * 8};
        const cuuint32_t box[3] = {kHaloX, kHaloY, kHaloZ};
        if ((st = encode(&m.b[m.n], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, sb, dims, strides, box)) != MS_OK) return st;
    }
    m.sa[m.n] = sa;
    m.sb[m.n] = sb;
    ++m.n;
    return MS_OK;
}

cudaError_t launch_step_lattice(const StepArgs &a, const LatticeArgs &g, const LatticeMaps &m, int n_sms,
                                cudaStream_t st)
{
    const long long nbricks = (long long)g.nbx * g.nby * g.nbz;
    if (nbricks <= 0) return cudaSuccess;
    if (nbricks > 0x7fffffffLL) return cudaErrorInvalidValue;
    int q = 0;
    while (q < m.n && !(m.sa[q] == a.sa && m.sb[q] == a.sb)) ++q;
    if (q == m.n) return cudaErrorInvalidValue;                // a buffer without tensor maps
    const unsigned grid = (unsigned)std::min<long long>(nbricks, (long long)kLatCtasPerSm * std::max(n_sms, 1));
    const size_t smem = 2 * (size_t)kStageBytes;
#define MS_LAUNCH_L(F, R, G, A)                                                                            \
    do {                                                                                                   \
        static std::atomic<uint64_t> opted{0};                                                             \
        int dev = 0;                                                                                       \
        cudaError_t e_ = cudaGetDevice(&dev);                                                              \
        if (e_ != cudaSuccess) return e_;                                                                  \
        const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;                                            \
        if (!bit || !(opted.load() & bit)) {                                                               \
            e_ = cudaFuncSetAttribute(k_step_lattice<F, R, G, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)smem);                                                          \
            if (e_ != cudaSuccess) return e_;                                                              \
            if (bit) opted.fetch_or(bit);                                                                  \
        }                                                                                                  \
        k_step_lattice<F, R, G, A><<<grid, kLatThreads, smem, st>>>(a, g, m.a[q], m.b[q], m.k);            \
    } while (0)
#define MS_LAUNCH_L2(G, A)                                                                                 \
    do {                                                                                                   \
        if (a.integrator == 3) { if (hf) MS_LAUNCH_L(true, true, G, A); else MS_LAUNCH_L(false, true, G, A); } \
        else { if (hf) MS_LAUNCH_L(true, false, G, A); else MS_LAUNCH_L(false, false, G, A); }             \
    } while (0)
    const bool hf = a.fext != nullptr;
    if (g.guard) { if (g.act) MS_LAUNCH_L2(true, true); else MS_LAUNCH_L2(true, false); }
    else { if (g.act) MS_LAUNCH_L2(false, true); else MS_LAUNCH_L2(false, false); }
#undef MS_LAUNCH_L2
#undef MS_LAUNCH_L
    return cudaGetLastError();
}

}  // namespace ms
