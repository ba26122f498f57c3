// ms_step.cu -- the explicit mass-spring step on sm_103a.
//
// One thread per mass (internal order), one launch per time step.  Each
// thread gathers every spring attached to its mass -- the springs it owns
// from its own sliced-ELL row, the others through back references into the
// owners' rows -- evaluates eq. 2's Hooke term plus the axial dashpot with the
// partner's state at t_n, adds gravity, external force and ground contact,
// and integrates (symplectic Euler) into the other state buffer.
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

namespace ms {

__device__ __forceinline__ void spring_term(const float4 xi, const float4 vi, const float4 xj,
                                            const float4 vj, float k, float L, float c,
                                            float &fx, float &fy, float &fz)
{
    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    if (l2 > 0.0f) {                       // a zero-length spring exerts no force
        const float l = sqrtf(l2);
        const float il = 1.0f / l;
        const float ux = dx * il, uy = dy * il, uz = dz * il;
        const float rv = (vj.x - vi.x) * ux + (vj.y - vi.y) * uy + (vj.z - vi.z) * uz;
        const float fs = k * (l - L) + c * rv;
        fx += fs * ux; fy += fs * uy; fz += fs * uz;
    }
}

template <bool HAS_C, bool HAS_ACT, bool HAS_FEXT>
__global__ void __launch_bounds__(256) k_step(const StepArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const unsigned lane = (unsigned)i & 31u;
    const uint4 meta = __ldg(&a.slice[i >> 5]);
    const float4 xi = __ldg(&a.x[i]);
    const float4 vi = __ldg(&a.v[i]);
    float fx = 0.f, fy = 0.f, fz = 0.f;

    // springs owned by this mass
    const unsigned flen = meta.z & 0xffffu, blen = meta.z >> 16;
    unsigned r = meta.x + lane;
#pragma unroll 2
    for (unsigned s = 0; s < flen; ++s, r += 32u) {
        int j = __ldg(&a.f_nbr[r]);
        j = (j < 0) ? i : j;               // padding slot: self, zero length
        const float k = __ldg(&a.f_k[r]);
        float L = __ldg(&a.f_L0[r]);
        const float c = HAS_C ? __ldg(&a.f_c[r]) : a.c_uniform;
        if (HAS_ACT) L = L * (1.0f + (__ldg(&a.f_al[r]) * a.s_n + __ldg(&a.f_be[r]) * a.c_n));
        spring_term(xi, vi, __ldg(&a.x[j]), __ldg(&a.v[j]), k, L, c, fx, fy, fz);
    }
    // springs owned by partners, reached through back references
    unsigned q = meta.y + lane;
#pragma unroll 2
    for (unsigned s = 0; s < blen; ++s, q += 32u) {
        const uint32_t e = __ldg(&a.b_ent[q]);
        int o = i;
        unsigned rr = 0;
        if (e != kBackPad) {
            o = (int)(e & kOwnerMask);
            rr = __ldg(&a.slice[o >> 5].x) + (e >> kOwnerBits) * 32u + ((unsigned)o & 31u);
        }
        const float k = __ldg(&a.f_k[rr]);
        float L = __ldg(&a.f_L0[rr]);
        const float c = HAS_C ? __ldg(&a.f_c[rr]) : a.c_uniform;
        if (HAS_ACT) L = L * (1.0f + (__ldg(&a.f_al[rr]) * a.s_n + __ldg(&a.f_be[rr]) * a.c_n));
        spring_term(xi, vi, __ldg(&a.x[o]), __ldg(&a.v[o]), k, L, c, fx, fy, fz);
    }

    float4 xn = xi, vn = make_float4(0.f, 0.f, 0.f, 0.f);
    const float w = xi.w;                  // 1/m, or -1 for an anchored mass
    if (w >= 0.0f) {
        if (HAS_FEXT) {
            const float4 fe = __ldg(&a.fext[i]);
            fx += fe.x; fy += fe.y; fz += fe.z;
        }
        const bool pen = a.contact && xi.z < 0.0f;
        float Fn = 0.f;
        if (pen) { Fn = -a.k_c * xi.z; fz += Fn; }
        float vx = vi.x + a.dt * (fx * w + a.gx);
        float vy = vi.y + a.dt * (fy * w + a.gy);
        float vz = vi.z + a.dt * (fz * w + a.gz);
        if (pen && a.mu > 0.0f) {          // Coulomb impulse clamp on (vx, vy)
            const float D = a.mu * Fn * a.dt * w;
            const float vt = sqrtf(vx * vx + vy * vy);
            if (vt <= D) { vx = 0.f; vy = 0.f; }
            else { const float sc = 1.0f - D / vt; vx *= sc; vy *= sc; }
        }
        vx *= a.keep; vy *= a.keep; vz *= a.keep;
        vn = make_float4(vx, vy, vz, 0.f);
        xn = make_float4(xi.x + a.dt * vx, xi.y + a.dt * vy, xi.z + a.dt * vz, w);
        if (!isfinite(xn.x + xn.y + xn.z + vx + vy + vz)) atomicOr(a.err, 1);
    }
    a.xo[i] = xn;
    a.vo[i] = vn;
}

cudaError_t launch_step(const StepArgs &a, cudaStream_t st)
{
    if (a.N <= 0) return cudaSuccess;
    const int bs = 256;
    const int grid = (a.N + bs - 1) / bs;
    const bool hc = a.f_c != nullptr, ha = a.f_al != nullptr, hf = a.fext != nullptr;
#define MS_LAUNCH(C, A, F) k_step<C, A, F><<<grid, bs, 0, st>>>(a)
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

__global__ void k_gather_state(const float4 *__restrict__ x4, const float4 *__restrict__ v4,
                               const int32_t *__restrict__ perm, int N, float *__restrict__ xo,
                               float *__restrict__ vo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = perm ? perm[i] : i;
    if (xo) { const float4 p = x4[i]; xo[3 * c] = p.x; xo[3 * c + 1] = p.y; xo[3 * c + 2] = p.z; }
    if (vo) { const float4 p = v4[i]; vo[3 * c] = p.x; vo[3 * c + 1] = p.y; vo[3 * c + 2] = p.z; }
}

__global__ void k_scatter_state(float4 *__restrict__ x4, float4 *__restrict__ v4,
                                const int32_t *__restrict__ perm, int N, const float *__restrict__ xi,
                                const float *__restrict__ vi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = perm ? perm[i] : i;
    const float w = x4[i].w;
    if (xi) x4[i] = make_float4(xi[3 * c], xi[3 * c + 1], xi[3 * c + 2], w);
    if (vi) {
        if (w < 0.0f) v4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        else v4[i] = make_float4(vi[3 * c], vi[3 * c + 1], vi[3 * c + 2], 0.f);
    }
}

cudaError_t launch_gather_state(const float4 *x4, const float4 *v4, const int32_t *perm, int N,
                                float *x_out, float *v_out, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    k_gather_state<<<(N + 255) / 256, 256, 0, st>>>(x4, v4, perm, N, x_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(float4 *x4, float4 *v4, const int32_t *perm, int N,
                                 const float *x_in, const float *v_in, cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    k_scatter_state<<<(N + 255) / 256, 256, 0, st>>>(x4, v4, perm, N, x_in, v_in);
    return cudaGetLastError();
}

}  // namespace ms
