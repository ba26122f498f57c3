// ms_noalloc.cu -- a step entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want
// to advance a spring network: code that runs while a CUDA graph is being
// captured, plugins living inside a host framework that owns every
// allocation, or real-time loops that forbid allocator calls.  This entry
// point serves them: the caller passes every input and output as device
// memory, and the only working memory -- the intermediate states of a
// multi-step call -- is a fixed array in the library's own device memory
// (`noalloc_scratch` below), which every GPU that loads the library holds
// until the process exits.
//
// The kernel is the gather form of the step (one thread per mass, every
// spring of the mass read from a caller-supplied CSR incidence list, so no
// atomics), double buffered through the scratch array.
#include "ms_internal.h"

#include <mutex>

namespace ms {
namespace {

constexpr int kNoallocMaxMasses = MS_NOALLOC_MAX_MASSES;
constexpr int kMaxDevices = 64;

// two state buffers of (x, w), (v, 0) float4 pairs: 2 x 2 x 16 B per mass
// (16 MiB).  Every call writes a buffer completely before reading it, so
// nothing in it needs clearing between calls.
__device__ __align__(256) float4 noalloc_scratch[4 * kNoallocMaxMasses];

std::mutex g_mu;
// per device: the context the address was looked up in, and the address
struct ScratchAddr {
    unsigned long long ctx_id;
    float4 *ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

struct CsrArgs {
    const float4 *st;    // state at t_n (2 float4 per mass); nullptr on the first step
    const float *x_in, *v_in, *mass;
    const uint8_t *fixed;
    const int32_t *row, *partner;
    const float *k, *c, *L0;
    float4 *sto;         // state at t_{n+1} (scratch), or nullptr on the last step
    float *x_out, *v_out;
    int N;
    float dt, gx, gy, gz, k_c, mu, keep;
    int contact;
};

__device__ __forceinline__ void load_state(const CsrArgs &a, int i, float4 &x, float4 &v)
{
    if (a.st) { x = a.st[2 * i]; v = a.st[2 * i + 1]; return; }
    const bool anchored = a.fixed && a.fixed[i];
    x = make_float4(a.x_in[3 * i], a.x_in[3 * i + 1], a.x_in[3 * i + 2], anchored ? -1.0f : 1.0f / a.mass[i]);
    v = anchored ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(a.v_in[3 * i], a.v_in[3 * i + 1], a.v_in[3 * i + 2], 0.f);
}

__global__ void k_step_csr(const CsrArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    float4 xi, vi;
    load_state(a, i, xi, vi);
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int q = a.row[i]; q < a.row[i + 1]; ++q) {
        float4 xj, vj;
        load_state(a, a.partner[q], xj, vj);
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float il = rsqrtf(l2);
        const float l = l2 * il;
        const float rv = fmaf(vj.x - vi.x, dx, fmaf(vj.y - vi.y, dy, (vj.z - vi.z) * dz)) * il;
        float fs = fmaf(a.k[q], l - a.L0[q], a.c[q] * rv) * il;
        fs = (l2 > 0.0f) ? fs : 0.0f;
        fx = fmaf(fs, dx, fx); fy = fmaf(fs, dy, fy); fz = fmaf(fs, dz, fz);
    }
    float4 xn = xi, vn = make_float4(0.f, 0.f, 0.f, 0.f);
    const float w = xi.w;
    if (w >= 0.0f) {
        const bool pen = a.contact && xi.z < 0.0f;
        float Fn = 0.f;
        if (pen) { Fn = -a.k_c * xi.z; fz += Fn; }
        float vx = vi.x + a.dt * (fx * w + a.gx);
        float vy = vi.y + a.dt * (fy * w + a.gy);
        float vz = vi.z + a.dt * (fz * w + a.gz);
        if (pen && a.mu > 0.0f) {
            const float D = a.mu * Fn * a.dt * w;
            const float vt = sqrtf(vx * vx + vy * vy);
            if (vt <= D) { vx = 0.f; vy = 0.f; }
            else { const float sc = 1.0f - D / vt; vx *= sc; vy *= sc; }
        }
        vx *= a.keep; vy *= a.keep; vz *= a.keep;
        vn = make_float4(vx, vy, vz, 0.f);
        xn = make_float4(xi.x + a.dt * vx, xi.y + a.dt * vy, xi.z + a.dt * vz, w);
    }
    if (a.sto) { a.sto[2 * i] = xn; a.sto[2 * i + 1] = vn; }
    else {
        a.x_out[3 * i] = xn.x; a.x_out[3 * i + 1] = xn.y; a.x_out[3 * i + 2] = xn.z;
        a.v_out[3 * i] = vn.x; a.v_out[3 * i + 1] = vn.y; a.v_out[3 * i + 2] = vn.z;
    }
}

// Unique id of the calling thread's current CUDA context (0 when none is
// current), through driver entry points that the runtime hands out, so the
// library links no driver library.  A context that is destroyed and created
// again (a device reset) gets a new id.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

ms_status current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return fail(MS_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not available");
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0) return fail(MS_ERR_CUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != 0) return fail(MS_ERR_CUDA, "cuCtxGetId failed");
    return MS_OK;
}

// Device address of the scratch array in the current context.  Host code
// only has a stand-in symbol for a __device__ array, so the real address is
// looked up with cudaGetSymbolAddress, with the device current, and cached
// per device together with the id of the context it belongs to; a call in a
// different context (after a device reset) looks the address up again.
ms_status scratch_for_current_device(float4 **scratch)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(MS_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    ms_status st = current_context_id(&id);
    if (st != MS_OK) return st;
    if (id == 0 || g_scratch[dev].ctx_id != id || !g_scratch[dev].ptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, noalloc_scratch);    // makes the device's primary context current if none is
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        if ((st = current_context_id(&id)) != MS_OK) return st;
        g_scratch[dev] = ScratchAddr{id, (float4 *)p};
    }
    *scratch = g_scratch[dev].ptr;
    return MS_OK;
}

}  // namespace
}  // namespace ms

extern "C" ms_status ms_step_csr_noalloc(const ms_params *p, int32_t N, const float *x_in, const float *v_in,
                                         const float *mass, const uint8_t *fixed, const int32_t *row_ptr,
                                         const int32_t *partner, const float *k, const float *c,
                                         const float *rest_len, int32_t nsteps, float *x_out, float *v_out,
                                         void *stream)
{
    using namespace ms;
    if (!p || !x_in || !v_in || !mass || !row_ptr || !partner || !k || !c || !rest_len || !x_out || !v_out)
        return fail(MS_ERR_ARG, "missing argument");
    if (N < 1) return fail(MS_ERR_ARG, "N must be >= 1");
    if (N > kNoallocMaxMasses)
        return fail(MS_ERR_ARG, "N = " + std::to_string(N) + " exceeds the fixed scratch capacity of " +
                                    std::to_string(kNoallocMaxMasses) + " masses (MS_NOALLOC_MAX_MASSES)");
    if (nsteps < 1) return fail(MS_ERR_ARG, "nsteps must be >= 1");
    if (!(p->dt > 0.f) || p->integrator != 0 || !(p->vel_damping >= 0.f && p->vel_damping < 1.f))
        return fail(MS_ERR_ARG, "bad step parameters");
    float4 *scratch = nullptr;
    ms_status st = scratch_for_current_device(&scratch);
    if (st != MS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    CsrArgs a{};
    a.x_in = x_in; a.v_in = v_in; a.mass = mass; a.fixed = fixed; a.row = row_ptr; a.partner = partner;
    a.k = k; a.c = c; a.L0 = rest_len; a.x_out = x_out; a.v_out = v_out; a.N = N;
    a.dt = p->dt; a.gx = p->g[0]; a.gy = p->g[1]; a.gz = p->g[2];
    a.k_c = p->k_c; a.mu = p->mu; a.keep = 1.0f - p->vel_damping; a.contact = p->contact_on;
    float4 *buf[2] = {scratch, scratch + 2 * (size_t)kNoallocMaxMasses};
    for (int n = 0; n < nsteps; ++n) {
        a.st = n == 0 ? nullptr : buf[(n - 1) & 1];
        a.sto = n == nsteps - 1 ? nullptr : buf[n & 1];
        k_step_csr<<<(N + 255) / 256, 256, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    return MS_OK;
}

