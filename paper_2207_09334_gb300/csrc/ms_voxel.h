// ms_voxel.h -- voxel robots shared by the batched population (ms_batch.cu)
// and the adjoint (ms_adjoint.cu): the host builder of the voxel lattice
// and the device routines of one step on a robot held in shared memory.
#pragma once
#include "ms_internal.h"

#include <vector>

namespace ms {

constexpr int kMaxRobotMasses = 4096;   // <= 2^kRobotOwnerBits (robot-local back references)

struct RobotDev {
    long long mass_base;   // first mass in the population-wide numbering
    int n;                 // masses
    int slice_base;        // first sliced-ELL slice of this robot
    float com0_x;          // centre-of-mass x at t = 0
    int vox_base;          // first voxel of this robot in the concatenated grids
    int n_vox;             // voxels (including empty ones) of this robot
    float inv_mass;        // 1 / total mass
    uint32_t rec_base;     // the robot's first record (= slice[slice_base].fwd_off)
};

// Host image of a population (robots concatenated; sliced-ELL rows with
// robot-local mass indices, absolute record offsets).
struct VoxelBuild {
    std::vector<RobotDev> robots;
    std::vector<float4> st0;           // 2 float4 per mass
    std::vector<uint4> slice;
    std::vector<int32_t> nbr;
    std::vector<float2> kl;            // (k, L0)
    std::vector<float2> ab;            // (alpha, beta)
    std::vector<float> c;
    std::vector<uint32_t> bent;
    // every-spring rows (population kernel; filled when the adjoint maps are
    // not requested): per slice (same index as `slice`) the first slot and
    // the row length; per slot the partner (robot-local, the mass itself for
    // padding) and the spring's (k, L0), (alpha, beta) and c
    std::vector<uint2> aslice;
    std::vector<uint16_t> anbr;
    std::vector<float2> akl, aab;
    std::vector<float> ac;
    // adjoint maps (filled when requested):
    std::vector<short4> slot_vox;      // per slot: up to 4 robot-local voxels sharing the spring (-1 = none)
    std::vector<uint32_t> vox_slots;   // per voxel (concatenated): slot of each of its 28 corner pairs (or 0xffffffff)
    std::vector<float> vox_amp;        // per voxel: actuation amplitude of its material (0 for empty)
    int64_t n_masses = 0, n_records = 0;
    int n_slices = 0;
    int max_n = 0;
};

// Builds the voxel lattice of every robot: masses at the corners of its
// non-empty voxels (raster order, x fastest), every voxel linking its 28
// corner pairs, springs shared by neighbouring voxels merged exactly.
ms_status build_voxels(const msb_voxel_spec *spec, int n_robots, const int32_t *dims, const uint8_t *materials,
                       const float *phase, const float *logk, bool adjoint_maps, VoxelBuild &out);

// (sin, cos)(two_pi_f * (counter + n) * dt) for n < nsteps, in double precision.
void launch_sc_table(const long long *counter, int nsteps, double dt, double two_pi_f, float2 *out, cudaStream_t s);

// Step parameters of a voxel population.
struct Env {
    float dt, gx, gy, gz, k_c, mu, keep;
    int contact;
};

inline Env make_env(const ms_params &p)
{
    Env e;
    e.dt = p.dt; e.gx = p.g[0]; e.gy = p.g[1]; e.gz = p.g[2];
    e.k_c = p.k_c; e.mu = p.mu; e.keep = 1.0f - p.vel_damping; e.contact = p.contact_on;
    return e;
}

// Persistent cluster step (ms_cluster.cu): tiles of tm masses (64 to
// kClMassesMax), one CTA of kClThreads threads each, at most kClusterMax CTAs
// in one cluster.
constexpr int kClMassesMax = 512;
constexpr int kClThreads = 1024;
constexpr int kClusterMax = 16;

struct ClusterArgs {
    float4 *sa;              // packed state (internal order): read at the start, written at the end
    float2 *sb;
    const float *w;          // 1/m, or -m for an anchored mass
    const float4 *fext;      // or nullptr
    // records, both directions, per tile; with L = kClThreads / tm lanes per
    // mass, slot q of member m is at [tile][q / L][m][q % L] (slots padded to
    // a multiple of L); partner coded by its mass index, padding = the mass
    // itself with (k, L0) = 0
    const uint16_t *nbr;
    const float2 *kl;
    const float *c;          // or nullptr (then c_uniform)
    const float2 *ab;        // or nullptr (passive)
    float c_uniform;
    int N, slots;            // slots: a multiple of L
    int tm;                  // masses per tile: 64, 128, 256 or 512
    const float2 *sc;        // (sin, cos)(2 pi f t_n) for the nsteps steps, if ab
    int nsteps;
    Env env;
    int *err;
};
size_t cluster_smem_bytes(int tm, int slots, bool has_c, bool has_act);
cudaError_t launch_cluster(const ClusterArgs &a, cudaStream_t st);

#ifdef __CUDACC__
// Spring records of a population (device pointers).
struct Records {
    const uint4 *slice;
    const int32_t *f_nbr;
    const float2 *f_kl;
    const float *f_c;      // or nullptr: every spring has c_uniform
    const float2 *f_ab;    // or nullptr: passive springs
    const uint32_t *b_ent;
    float c_uniform;
};

// Every-spring rows of a population (device pointers): each mass's row lists
// all of its springs, both directions, so one pass of coalesced loads serves
// the whole force sum.
struct AllRows {
    const uint2 *slice;    // per slice: (first slot, slots per lane)
    const uint16_t *nbr;
    const float2 *kl;
    const float2 *ab;
    const float *c;
};

// Hooke + dashpot term (eq. 2), the same arithmetic as the single-system step.
__device__ __forceinline__ void vox_spring(const float4 xi, const float4 vi, const float4 xj, const float4 vj,
                                           float k, float L, float c, float &fx, float &fy, float &fz)
{
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float il = rsqrtf(l2);
    const float l = l2 * il;
    const float rv = fmaf(vj.x - vi.x, dx, fmaf(vj.y - vi.y, dy, (vj.z - vi.z) * dz)) * il;
    float fs = fmaf(k, l - L, c * rv) * il;
    fs = (l2 > 0.0f) ? fs : 0.0f;
    fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
}

// Spring force on robot-local mass i from the shared-memory state; rec_base
// is the robot's first record (slice[slice_base].x).  UNROLL springs are
// unrolled together so that their record loads (L2 round trips) overlap;
// the population kernel gains from it, the register-heavy adjoint does not.
template <int UNROLL = 1>
__device__ __forceinline__ float4 robot_force(const Records &a, int slice_base, unsigned rec_base, int i,
                                              const float4 *xs, const float4 *vs, float s_n, float c_n)
{
    const unsigned lane = (unsigned)i & 31u;
    const uint4 meta = __ldg(&a.slice[slice_base + (i >> 5)]);
    const float4 xi = xs[i], vi = vs[i];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const unsigned flen = meta.z & 0xffffu, blen = meta.z >> 16;
    unsigned r = meta.x + lane;
#pragma unroll UNROLL
    for (unsigned s = 0; s < flen; ++s, r += 32u) {
        int j = __ldg(&a.f_nbr[r]);
        j = (j < 0) ? i : j;
        const float2 kl = __ldg(&a.f_kl[r]);
        const float2 ab = a.f_ab ? __ldg(&a.f_ab[r]) : make_float2(0.f, 0.f);
        const float L = kl.y * (1.0f + fmaf(ab.x, s_n, ab.y * c_n));
        vox_spring(xi, vi, xs[j], vs[j], kl.x, L, a.f_c ? __ldg(&a.f_c[r]) : a.c_uniform, fx, fy, fz);
    }
    unsigned q = meta.y + lane;
#pragma unroll UNROLL
    for (unsigned s = 0; s < blen; ++s, q += 32u) {
        const uint32_t e = __ldg(&a.b_ent[q]);
        int o = i;
        unsigned rr = 0;
        if (e != kBackPad) {
            o = (int)(e & kRobotOwnerMask);
            rr = rec_base + (e >> kRobotOwnerBits);
        }
        const float2 kl = __ldg(&a.f_kl[rr]);
        const float2 ab = a.f_ab ? __ldg(&a.f_ab[rr]) : make_float2(0.f, 0.f);
        const float L = kl.y * (1.0f + fmaf(ab.x, s_n, ab.y * c_n));
        vox_spring(xi, vi, xs[o], vs[o], kl.x, L, a.f_c ? __ldg(&a.f_c[rr]) : a.c_uniform, fx, fy, fz);
    }
    return make_float4(fx, fy, fz, 0.f);
}

// The same force from the every-spring rows: the springs of mass i one slot
// per lattice direction (the 13 forward directions, then their opposites), so
// the sum agrees with robot_force's (own records, then back references) up
// to the rounding of a different order.
template <int UNROLL = 1>
__device__ __forceinline__ float4 robot_force_all(const AllRows &g, int slice_base, int i, const float4 *xs,
                                                  const float4 *vs, float s_n, float c_n)
{
    const uint2 meta = __ldg(&g.slice[slice_base + (i >> 5)]);
    const float4 xi = xs[i], vi = vs[i];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    unsigned r = meta.x + ((unsigned)i & 31u);
#pragma unroll UNROLL
    for (unsigned s = 0; s < meta.y; ++s, r += 32u) {
        const int j = __ldg(&g.nbr[r]);
        const float2 kl = __ldg(&g.kl[r]);
        const float2 ab = __ldg(&g.ab[r]);
        const float L = kl.y * (1.0f + fmaf(ab.x, s_n, ab.y * c_n));
        vox_spring(xi, vi, xs[j], vs[j], kl.x, L, __ldg(&g.c[r]), fx, fy, fz);
    }
    return make_float4(fx, fy, fz, 0.f);
}

// Gravity, ground contact, friction clamp, damping and the symplectic Euler
// update of one mass, in place.  vt (optional) receives the velocity before
// the friction clamp and damping, with w = 1 if the mass penetrates the
// ground (the branch record the adjoint needs).
__device__ __forceinline__ void robot_integrate(const Env &e, float4 &x, float4 &v, float4 f, float4 *vt = nullptr)
{
    const float w = x.w;
    if (w < 0.0f) { v = make_float4(0.f, 0.f, 0.f, 0.f); if (vt) *vt = v; return; }
    const bool pen = e.contact && x.z < 0.0f;
    float Fn = 0.f;
    // explicit fused operations: every inlined copy rounds the same way,
    // whatever the compiler's contraction choices in its context
    if (pen) { Fn = -e.k_c * x.z; f.z = fmaf(-e.k_c, x.z, f.z); }
    float vx = fmaf(e.dt, fmaf(f.x, w, e.gx), v.x);
    float vy = fmaf(e.dt, fmaf(f.y, w, e.gy), v.y);
    float vz = fmaf(e.dt, fmaf(f.z, w, e.gz), v.z);
    if (vt) *vt = make_float4(vx, vy, vz, pen ? 1.0f : 0.0f);
    if (pen && e.mu > 0.0f) {
        const float D = e.mu * Fn * e.dt * w;
        const float vtn = sqrtf(fmaf(vx, vx, vy * vy));
        if (vtn <= D) { vx = 0.f; vy = 0.f; }
        else { const float sc = 1.0f - D / vtn; vx *= sc; vy *= sc; }
    }
    vx *= e.keep; vy *= e.keep; vz *= e.keep;
    v = make_float4(vx, vy, vz, 0.f);
    x = make_float4(fmaf(e.dt, vx, x.x), fmaf(e.dt, vy, x.y), fmaf(e.dt, vz, x.z), w);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
#endif  // __CUDACC__

#ifdef __CUDACC__

// (sin, cos)(two_pi_f * (n0 + n) * dt) for n < nsteps.
void launch_sc_table_from(long long n0, int nsteps, double dt, double two_pi_f, float2 *out, cudaStream_t s);
#endif

}  // namespace ms
