// ms_lattice.cu -- the explicit step on the lattice layout (kernel 4).
//
// For a box lattice with 26-neighbourhood springs (the benchmark's
// throughput lattice; the paper's voxel and cubic lattices of "Generating a
// Lattice"), the topology and the rest lengths follow from the lattice
// itself, so the step reads per spring only its stiffness.  That halves the
// bytes of the general (tiled) layout, which stores partner indices and rest
// lengths and lists every spring at both of its masses.
//
// One CTA per brick of 16 x 8 x 4 cells (one thread per cell):
//   * the state of the brick and of its one-cell halo (18 x 10 x 6 cells) is
//     staged in shared memory; a partner in direction d is then the shared
//     entry at a constant offset, with no index stored anywhere;
//   * each thread evaluates its cell's 26 springs (eq. 2's Hooke term plus
//     the axial dashpot, reading R2): the 13 forward springs with k from its
//     own cell's arrays kf[d][i], the 13 backward springs with k from the
//     partner's arrays (kb[d][i] = kf[d][i - off(d)], a read that hits L1 or
//     L2 because the partner sits in this brick or in one processed just
//     before);
//   * then gravity, external force, ground contact, damping and the update of
//     the cell's mass (integrate_mass, shared with the other step kernels), and
//     the new state goes to the other buffer (Algorithm 1's synchronisation
//     is the kernel boundary).
// Every spring is evaluated at both ends; the two evaluations are exact
// negatives, and each mass sums its springs in a fixed order (forward
// directions 0..12, then backward 0..12), so runs are bit-reproducible.
#include "ms_internal.h"
#include "ms_device.cuh"

namespace ms {
namespace {

// spring_term_packed for a lattice spring with stiffness k; k < 0 marks a
// spring that does not exist (its partner cell may hold no mass), which adds
// nothing.  For an existing spring the result is spring_term_packed's.
__device__ __forceinline__ void lattice_spring(const float4 xi, const float4 vi, const float4 pa, const float2 pb,
                                               float k, float L, float c, float &fx, float &fy, float &fz)
{
    const float dx = pa.x - xi.x, dy = pa.y - xi.y, dz = pa.z - xi.z;
    const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float il = rsqrt_hw(l2);
    const float l = l2 * il;
    const float rv = fmaf(pa.w - vi.x, dx, fmaf(pb.x - vi.y, dy, (pb.y - vi.z) * dz)) * il;
    float fs = fmaf(k, l - L, c * rv) * il;
    fs = (l2 > 0.0f && k >= 0.0f) ? fs : 0.0f;
    fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
}

// shared-memory offset of the partner in direction d inside the staged block
__host__ __device__ constexpr int halo_off(int d) { return lat_dx(d) + kHaloX * (lat_dy(d) + kHaloY * lat_dz(d)); }

template <bool HAS_FEXT, bool RK4>
__global__ void __launch_bounds__(kBrickCells, 3) k_step_lattice(const StepArgs a, const LatticeArgs g)
{
    __shared__ float4 spa[kHaloCells];     // (x, y, z, vx) of the brick and its halo
    __shared__ float2 spb[kHaloCells];     // (vy, vz)
    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    const int bx = b % g.nbx, byz = b / g.nbx, by = byz % g.nby, bz = byz / g.nby;
    const int XY = g.X * g.Y;
    // padded index of the staged block's first cell (the brick's origin less one cell on each axis)
    const int base = bx * kBrickX + g.X * (by * kBrickY) + XY * (bz * kBrickZ);
    for (int e = tid; e < kHaloCells; e += kBrickCells) {
        const int hx = e % kHaloX, hy = (e / kHaloX) % kHaloY, hz = e / (kHaloX * kHaloY);
        const int gi = base + hx + g.X * hy + XY * hz;
        spa[e] = __ldg(&a.sa[gi]);
        spb[e] = __ldg(&a.sb[gi]);
    }
    __syncthreads();
    const int cx = tid % kBrickX, cy = (tid / kBrickX) % kBrickY, cz = tid / (kBrickX * kBrickY);
    const int s = (cx + 1) + kHaloX * ((cy + 1) + kHaloY * (cz + 1));
    const int i = base + (cx + 1) + g.X * (cy + 1) + XY * (cz + 1);
    const float w = __ldg(&a.w[i]);
    if (w != w) return;                    // a cell without a mass
    const float4 p = spa[s];
    const float2 q = spb[s];
    const float4 xi = make_float4(p.x, p.y, p.z, w), vi = make_float4(p.w, q.x, q.y, 0.f);
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int d = 0; d < kLatDirs; ++d)
        lattice_spring(xi, vi, spa[s + halo_off(d)], spb[s + halo_off(d)], __ldg(g.kf[d] + i), g.L[d], g.c, fx, fy, fz);
#pragma unroll
    for (int d = 0; d < kLatDirs; ++d)
        lattice_spring(xi, vi, spa[s - halo_off(d)], spb[s - halo_off(d)], __ldg(g.kb[d] + i), g.L[d], g.c, fx, fy, fz);
    float4 xn, vn;
    integrate_mass<HAS_FEXT, RK4>(a, i, xi, vi, fx, fy, fz, xn, vn);
    store_mass(a, i, xn, vn);
}

}  // namespace

cudaError_t launch_step_lattice(const StepArgs &a, const LatticeArgs &g, cudaStream_t st)
{
    const long long grid = (long long)g.nbx * g.nby * g.nbz;
    if (grid <= 0) return cudaSuccess;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    const bool hf = a.fext != nullptr;
    if (a.integrator == 3) {
        if (hf) k_step_lattice<true, true><<<(unsigned)grid, kBrickCells, 0, st>>>(a, g);
        else k_step_lattice<false, true><<<(unsigned)grid, kBrickCells, 0, st>>>(a, g);
    } else {
        if (hf) k_step_lattice<true, false><<<(unsigned)grid, kBrickCells, 0, st>>>(a, g);
        else k_step_lattice<false, false><<<(unsigned)grid, kBrickCells, 0, st>>>(a, g);
    }
    return cudaGetLastError();
}

}  // namespace ms
