// ms_device.cuh -- the per-spring and per-mass arithmetic of the explicit
// step, shared by every single-system step kernel (ms_step.cu, ms_lattice.cu)
// so that they all round alike: eq. 2's Hooke term with the axial dashpot,
// and gravity, external force, ground contact, damping and the update of one
// mass (symplectic Euler, forward Euler eq. 4, position Verlet eq. 5-6, or a
// stage of classical RK4 eq. 7-8).
#pragma once
#include "ms_internal.h"

namespace ms {

// 1/sqrt(x) by the hardware approximation (PTX rsqrt.approx.ftz.f32, relative
// error below 2^-22); subnormal inputs count as zero.  Squared spring lengths
// are never subnormal: a zero length is handled by the caller.
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Hooke term of eq. 2 plus the axial dashpot, added to (fx, fy, fz) for the
// mass at (xi, vi) with the partner's state packed as pa = (x, y, z, vx),
// pb = (vy, vz) (d = x_partner - x_self):
//   f = (k (l - L) + c (v_partner - v_self).d / l) d / l.
// One reciprocal square root serves both l and the unit vector.  The result
// is an exact negation when the endpoints are swapped, and a spring of zero
// length (or a padding slot pointing at the mass itself) adds nothing.
__device__ __forceinline__ void spring_term_packed(const float4 xi, const float4 vi, const float4 pa,
                                                   const float2 pb, float k, float L, float c,
                                                   float &fx, float &fy, float &fz)
{
    const float dx = pa.x - xi.x, dy = pa.y - xi.y, dz = pa.z - xi.z;
    const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float il = rsqrt_hw(l2);
    const float l = l2 * il;
    const float rv = fmaf(pa.w - vi.x, dx, fmaf(pb.x - vi.y, dy, (pb.y - vi.z) * dz)) * il;
    float fs = fmaf(k, l - L, c * rv) * il;
    fs = (l2 > 0.0f) ? fs : 0.0f;
    fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
}

// Packed state of mass i as the kernels use it: xi = (x, w), vi = (v, 0).
__device__ __forceinline__ void load_mass(const float4 *sa, const float2 *sb, const float *w, int i, float4 &xi,
                                          float4 &vi)
{
    const float4 p = __ldg(&sa[i]);
    const float2 q = __ldg(&sb[i]);
    xi = make_float4(p.x, p.y, p.z, __ldg(&w[i]));
    vi = make_float4(p.w, q.x, q.y, 0.f);
}

__device__ __forceinline__ void store_mass(const StepArgs &a, int i, const float4 xn, const float4 vn)
{
    a.oa[i] = make_float4(xn.x, xn.y, xn.z, vn.x);
    a.ob[i] = make_float2(vn.y, vn.z);
}

// Gravity, external force, ground contact (penalty normal force, Coulomb
// impulse clamp), global damping and the update of mass i: symplectic Euler
// (default), forward Euler (eq. 4), position Verlet (eq. 5-6) or one stage
// of classical RK4 (eq. 7-8).
template <bool HAS_FEXT, bool RK4>
__device__ __forceinline__ void integrate_mass(const StepArgs &a, int i, const float4 xi, const float4 vi,
                                               float fx, float fy, float fz, float4 &xn, float4 &vn)
{
    xn = xi;
    vn = make_float4(0.f, 0.f, 0.f, 0.f);
    const float w = xi.w;                  // 1/m, or -m for an anchored mass
    if (w < 0.0f) return;
    if (HAS_FEXT) {
        const float4 fe = __ldg(&a.fext[i]);
        fx += fe.x; fy += fe.y; fz += fe.z;
    }
    // fused operations written out, so every kernel that inlines this rounds alike
    const bool pen = a.contact && xi.z < 0.0f;
    float Fn = 0.f;
    if (pen) { Fn = -a.k_c * xi.z; fz = fmaf(-a.k_c, xi.z, fz); }
    if (RK4) {
        // RK4 stage q on d/dt (x, v) = (v, f/m): (xi, vi) is the stage state
        // Y_q, its slope is K_q = (vi, f/m).  The slopes are summed with
        // weights 1, 2, 2, 1 into rk_acc; stages 0-2 write the next stage
        // state Y_n + c h K_q (c = 1/2, 1/2, 1), stage 3 writes
        // Y_{n+1} = Y_n + h/6 (K_0 + 2 K_1 + 2 K_2 + K_3).
        const int q = a.rk_stage;
        const float ax = fx * w + a.gx, ay = fy * w + a.gy, az = fz * w + a.gz;
        const float4 ba = __ldg(&a.rk_ba[i]);
        const float2 bb = __ldg(&a.rk_bb[i]);
        const float3 bx = make_float3(ba.x, ba.y, ba.z), bv = make_float3(ba.w, bb.x, bb.y);
        float4 sx = make_float4(vi.x, vi.y, vi.z, 0.f), sv = make_float4(ax, ay, az, 0.f);
        if (q > 0) {
            const float wq = q == 3 ? 1.0f : 2.0f;
            const float4 px = a.rk_acc[2 * i], pv = a.rk_acc[2 * i + 1];
            sx = make_float4(fmaf(wq, sx.x, px.x), fmaf(wq, sx.y, px.y), fmaf(wq, sx.z, px.z), 0.f);
            sv = make_float4(fmaf(wq, sv.x, pv.x), fmaf(wq, sv.y, pv.y), fmaf(wq, sv.z, pv.z), 0.f);
        }
        if (q < 3) {
            a.rk_acc[2 * i] = sx;
            a.rk_acc[2 * i + 1] = sv;
            const float c = q == 2 ? a.dt : 0.5f * a.dt;
            xn = make_float4(fmaf(c, vi.x, bx.x), fmaf(c, vi.y, bx.y), fmaf(c, vi.z, bx.z), w);
            vn = make_float4(fmaf(c, ax, bv.x), fmaf(c, ay, bv.y), fmaf(c, az, bv.z), 0.f);
        } else {
            const float h6 = a.dt / 6.0f;
            xn = make_float4(fmaf(h6, sx.x, bx.x), fmaf(h6, sx.y, bx.y), fmaf(h6, sx.z, bx.z), w);
            vn = make_float4(fmaf(h6, sv.x, bv.x), fmaf(h6, sv.y, bv.y), fmaf(h6, sv.z, bv.z), 0.f);
        }
        if (!isfinite(xn.x + xn.y + xn.z + vn.x + vn.y + vn.z)) atomicOr(a.err, kErrNonFinite);
        return;
    }
    float vx = fmaf(a.dt, fmaf(fx, w, a.gx), vi.x);
    float vy = fmaf(a.dt, fmaf(fy, w, a.gy), vi.y);
    float vz = fmaf(a.dt, fmaf(fz, w, a.gz), vi.z);
    if (pen && a.mu > 0.0f) {              // Coulomb impulse clamp on (vx, vy)
        const float D = a.mu * Fn * a.dt * w;
        const float vt = sqrtf(fmaf(vx, vx, vy * vy));
        if (vt <= D) { vx = 0.f; vy = 0.f; }
        else { const float sc = 1.0f - D / vt; vx *= sc; vy *= sc; }
    }
    vx *= a.keep; vy *= a.keep; vz *= a.keep;
    vn = make_float4(vx, vy, vz, 0.f);
    if (a.integrator == 1) {
        // forward Euler (eq. 4): the position moves with the velocity at t_n
        xn = make_float4(xi.x + a.dt * vi.x, xi.y + a.dt * vi.y, xi.z + a.dt * vi.z, w);
    } else if (a.integrator == 2) {
        // position Verlet (eq. 5-6) in velocity form.  With v_n = (x_n - x_{n-1})/dt,
        // eq. 6 is x_{n+1} = x_n + dt (v_n + dt f/m) and eq. 5 the same with dt/2
        // in the inner product, so v_{n+1} = v_n + h dt f/m (h = 1/2 on the first
        // step, 1 after) and x_{n+1} = x_n + dt v_{n+1}: no difference of
        // positions is formed, so no precision is lost to cancellation.
        const float h = a.first_step ? 0.5f : 1.0f;
        const float ax = fx * w + a.gx, ay = fy * w + a.gy, az = fz * w + a.gz;
        vn = make_float4(vi.x + h * a.dt * ax, vi.y + h * a.dt * ay, vi.z + h * a.dt * az, 0.f);
        xn = make_float4(xi.x + a.dt * vn.x, xi.y + a.dt * vn.y, xi.z + a.dt * vn.z, w);
    } else {
        // symplectic Euler: the position moves with the updated velocity
        xn = make_float4(fmaf(a.dt, vx, xi.x), fmaf(a.dt, vy, xi.y), fmaf(a.dt, vz, xi.z), w);
    }
    if (!isfinite(xn.x + xn.y + xn.z + vn.x + vn.y + vn.z)) atomicOr(a.err, kErrNonFinite);
}

// ---- mbarriers and bulk copies (TMA) -------------------------------------
// Every wait is bounded: after kMaxSpins polls it reports failure, and the
// kernel records kErrTimeout instead of hanging.
constexpr unsigned kMaxSpins = 1u << 26;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// L2 policy for data read once per step (the spring records): evicted first,
// so that the state, whose halo is read again by neighbouring tiles, stays in L2
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// global -> shared bulk copy completing on an mbarrier, with an L2 policy
// (sizes and both addresses are multiples of 16 bytes by construction of the
// layout)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait: true when the phase completed, false after kMaxSpins polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (unsigned n = 0; n < kMaxSpins; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// tiled global -> shared copies of a 3-D / 4-D box (tensor map in kernel
// parameter space), completing on an mbarrier; the innermost coordinate is a
// multiple of 16 bytes by construction of the layouts that use them
__device__ __forceinline__ void tma_load_3d(void *dst, const void *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2),
                   "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const void *map, int c0, int c1, int c2, int c3, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
                   "r"(smem_addr(bar)) : "memory");
}

// bring a 4-D box into L2 ahead of its use (no shared memory, no completion)
__device__ __forceinline__ void tma_prefetch_4d(const void *map, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global [%0, {%1, %2, %3, %4}];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3) : "memory");
}

}  // namespace ms
