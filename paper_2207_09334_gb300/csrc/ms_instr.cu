// ms_instr.cu -- instrumentation kernels of the single-system path: the
// energy of the state on the device and a per-step trace of chosen masses.
//
// The paper checks its simulator against energy conservation and follows
// the tip of a cantilever over time (Energy Conservation Tests, the
// cantilever and damping experiments).  At scale those quantities are
// reduced on the device, so a run can record them every few steps without
// copying the state to the host.
//
// Energy, at the current state and time t_n = step_count dt:
//   kinetic      sum_i  m_i |v_i|^2 / 2
//   elastic      sum_s  k_s (l_s - L_s(t_n))^2 / 2      (eq. 2's Hooke term)
//   gravity      -sum_i m_i g . x_i
//   ground       sum_i  k_c z_i^2 / 2 over z_i < 0      (penalty contact)
// Anchored masses keep their mass in the state (stored as -m), so they
// count in the gravity and ground terms like every other mass.
//
// Reduction order is fixed (no atomics): each thread sums its own terms in
// FP32, a warp reduces by shuffles in FP32, warps are combined in FP64 per
// block, and one block sums the per-block partials in FP64 in block order.
#include "ms_internal.h"

namespace ms {
namespace {

constexpr int kEnergyThreads = 256;

struct Terms {
    float ke, pe, gpe, cpe;
};

__device__ __forceinline__ void mass_terms(const EnergyArgs &a, int i, Terms &t)
{
    const float4 p = __ldg(&a.sa[i]);
    const float2 q = __ldg(&a.sb[i]);
    const float4 x = make_float4(p.x, p.y, p.z, __ldg(&a.w[i]));
    const float3 v = make_float3(p.w, q.x, q.y);
    const float m = x.w > 0.0f ? 1.0f / x.w : -x.w;     // free: 1/m stored; anchored: -m
    t.ke += 0.5f * m * fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z));
    t.gpe -= m * fmaf(a.gx, x.x, fmaf(a.gy, x.y, a.gz * x.z));
    if (a.contact && x.z < 0.0f) t.cpe += 0.5f * a.k_c * x.z * x.z;
}

// k (l - L)^2 for the spring from xi to xj with record r
__device__ __forceinline__ float spring_pe(const EnergyArgs &a, const float4 xi, const float4 xj, unsigned r)
{
    const float2 kl = __ldg(&a.f_kl[r]);
    float L = kl.y;
    if (a.f_ab) { const float2 ab = __ldg(&a.f_ab[r]); L = L * (1.0f + fmaf(ab.x, a.s_n, ab.y * a.c_n)); }
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float e = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - L;
    return kl.x * e * e;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block sum of the four terms into partial[4 * blockIdx.x .. +3] (FP64)
__device__ void block_reduce(Terms t, double *partial)
{
    __shared__ double wsum[32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    t.ke = warp_sum_f(t.ke); t.pe = warp_sum_f(t.pe); t.gpe = warp_sum_f(t.gpe); t.cpe = warp_sum_f(t.cpe);
    if (lane == 0) { wsum[warp][0] = t.ke; wsum[warp][1] = t.pe; wsum[warp][2] = t.gpe; wsum[warp][3] = t.cpe; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w][threadIdx.x];
        partial[4 * blockIdx.x + threadIdx.x] = s;
    }
}

// gather layout: one thread per mass; each spring once, from its owner's row
__global__ void __launch_bounds__(kEnergyThreads) k_energy_gather(const EnergyArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    Terms t{0.f, 0.f, 0.f, 0.f};
    if (i < a.N) {
        mass_terms(a, i, t);
        const uint4 meta = __ldg(&a.slice[i >> 5]);
        const float4 xi = __ldg(&a.sa[i]);
        const unsigned flen = meta.z & 0xffffu;
        unsigned r = meta.x + ((unsigned)i & 31u);
        float pe = 0.f;
        for (unsigned s = 0; s < flen; ++s, r += 32u) {
            const int j = __ldg(&a.f_nbr[r]);
            if (j < 0) continue;                              // padding slot
            pe += spring_pe(a, xi, __ldg(&a.sa[j]), r);
        }
        t.pe = 0.5f * pe;
    }
    block_reduce(t, a.partial);
}

// tiled layout: one CTA per tile; every spring is listed at both of its
// masses, so each listing counts one half of the spring's energy
__global__ void __launch_bounds__(kTileMasses) k_energy_tiled(const EnergyArgs a)
{
    const int4 T = __ldg(&a.tiles[2 * blockIdx.x]);
    const int4 R = __ldg(&a.tiles[2 * blockIdx.x + 1]);
    const int m = threadIdx.x;
    Terms t{0.f, 0.f, 0.f, 0.f};
    if (m < T.y) {
        const int i = T.x + m;
        mass_terms(a, i, t);
        const float4 xi = __ldg(&a.sa[i]);
        float pe = 0.f;
        for (int s = 0; s < R.y; ++s) {
            const unsigned r = (unsigned)R.x + (unsigned)s * kTileMasses + (unsigned)m;
            const unsigned loc = __ldg(&a.t_nbr[r]);
            if (loc == 0xffffu || (int)loc == m) continue;  // padding slot (marked, or the mass itself)
            const int j = (int)loc < T.y ? T.x + (int)loc : __ldg(&a.halo[T.z + (int)loc - T.y]);
            pe += spring_pe(a, xi, __ldg(&a.sa[j]), r);
        }
        t.pe = 0.25f * pe;
    }
    block_reduce(t, a.partial);
}

// lattice layout: the terms of cell i; each spring once, from the cell it
// leaves in a forward direction (k = NaN: no spring between two masses; k = 0:
// a slot that touches a cell without a mass, or a spring of zero stiffness,
// either way no energy)
__device__ __forceinline__ void lattice_cell_terms(const EnergyArgs &a, const LatticeArgs &g, int i, Terms &t)
{
    const float w = __ldg(&a.w[i]);
    if (!(w == w)) return;                               // a cell without a mass
    mass_terms(a, i, t);
    const float4 xi = __ldg(&a.sa[i]);
    float pe = 0.f;
#pragma unroll
    for (int d = 0; d < kLatDirs; ++d) {
        const float k = __ldg(g.kf[d] + i);
        if (!(k == k) || k == 0.f) continue;                // no spring, or one that adds no energy
        const float4 xj = __ldg(&a.sa[i + lat_dx(d) + g.X * (lat_dy(d) + g.Y * lat_dz(d))]);
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        float L = g.L[d];
        if (g.act) {                                        // the actuated rest length at t_n
            const float2 ab = __ldg(g.abf[d] + i);
            L = L * (1.0f + fmaf(ab.x, a.s_n, ab.y * a.c_n));
        }
        const float e = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - L;
        pe += k * e * e;
    }
    t.pe += 0.5f * pe;
}

// one CTA per brick, each thread the two cells stacked in z that the step
// kernel gives it
__global__ void __launch_bounds__(kLatThreads) k_energy_lattice(const EnergyArgs a, const LatticeArgs g)
{
    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    const int bx = b % g.nbx, byz = b / g.nbx, by = byz % g.nby, bz = byz / g.nby;
    const int cx = tid % kBrickX, cy = (tid / kBrickX) % kBrickY, cz = 2 * (tid / (kBrickX * kBrickY));
    const int i = (bx * kBrickX + cx + 1) + g.X * ((by * kBrickY + cy + 1) + g.Y * (bz * kBrickZ + cz + 1));
    Terms t{0.f, 0.f, 0.f, 0.f};
    lattice_cell_terms(a, g, i, t);
    lattice_cell_terms(a, g, i + g.X * g.Y, t);
    block_reduce(t, a.partial);
}

// one block: out[c] = sum over blocks of partial[4 b + c], in block order
// per thread, then a fixed tree over the threads
__global__ void __launch_bounds__(kEnergyThreads) k_energy_final(const double *partial, int n_blocks, double *out)
{
    __shared__ double s[4][kEnergyThreads];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < n_blocks; b += kEnergyThreads)
        for (int c = 0; c < 4; ++c) acc[c] += partial[4 * b + c];
    for (int c = 0; c < 4; ++c) s[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int w = kEnergyThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_trace(const float4 *__restrict__ sa, const int32_t *__restrict__ idx, int n, float *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float4 p = sa[idx[q]];
    out[3 * q] = p.x; out[3 * q + 1] = p.y; out[3 * q + 2] = p.z;
}

}  // namespace

int energy_blocks(const EnergyArgs &a, const LatticeArgs *lat)
{
    if (lat) return lat->nbx * lat->nby * lat->nbz;
    return a.tiled ? a.n_tiles : (a.N + kEnergyThreads - 1) / kEnergyThreads;
}

cudaError_t launch_energy(const EnergyArgs &a, const LatticeArgs *lat, double *out, cudaStream_t s)
{
    const int nb = energy_blocks(a, lat);
    if (lat) k_energy_lattice<<<nb, kLatThreads, 0, s>>>(a, *lat);
    else if (a.tiled) k_energy_tiled<<<nb, kTileMasses, 0, s>>>(a);
    else k_energy_gather<<<nb, kEnergyThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_final<<<1, kEnergyThreads, 0, s>>>(a.partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_trace(const float4 *sa, const int32_t *idx, int n, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_trace<<<(n + 127) / 128, 128, 0, s>>>(sa, idx, n, out);
    return cudaGetLastError();
}

}  // namespace ms
