// ms_state.cu -- moving the state of a single system between the caller's
// (N, 3) arrays in caller order and the library's internal buffers (2 float4
// per mass in internal order: (x, 1/m or -m), (v, 0)).
#include "ms_internal.h"

#include <climits>

namespace ms {
namespace {

__global__ void k_gather_state(const float4 *__restrict__ st, const int32_t *__restrict__ perm, int N,
                               float *__restrict__ xo, float *__restrict__ vo)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = perm ? perm[i] : i;
    if (xo) { const float4 p = st[2 * i]; xo[3 * c] = p.x; xo[3 * c + 1] = p.y; xo[3 * c + 2] = p.z; }
    if (vo) { const float4 p = st[2 * i + 1]; vo[3 * c] = p.x; vo[3 * c + 1] = p.y; vo[3 * c + 2] = p.z; }
}

// skip: if not null and no longer INT_MAX (a non-finite input was found), nothing is written
__global__ void k_scatter_state(float4 *__restrict__ st, const int32_t *__restrict__ perm, int N,
                                const float *__restrict__ xi, const float *__restrict__ vi, const int *skip)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (skip && *skip != INT_MAX) return;
    const int c = perm ? perm[i] : i;
    const float w = st[2 * i].w;
    if (xi) st[2 * i] = make_float4(xi[3 * c], xi[3 * c + 1], xi[3 * c + 2], w);
    if (vi) {
        if (w < 0.0f) st[2 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        else st[2 * i + 1] = make_float4(vi[3 * c], vi[3 * c + 1], vi[3 * c + 2], 0.f);
    }
}

// first_bad = min over masses (caller order) with a non-finite coordinate
__global__ void k_check_finite(const float *__restrict__ x, const float *__restrict__ v, int N, int *first_bad)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    bool ok = true;
    if (x) ok = isfinite(x[3 * c]) && isfinite(x[3 * c + 1]) && isfinite(x[3 * c + 2]);
    if (v) ok = ok && isfinite(v[3 * c]) && isfinite(v[3 * c + 1]) && isfinite(v[3 * c + 2]);
    if (!ok) atomicMin(first_bad, c);
}

__global__ void k_set_int(int *p, int v) { *p = v; }

}  // namespace

cudaError_t launch_gather_state(const float4 *st, const int32_t *perm, int N,
                                float *x_out, float *v_out, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_gather_state<<<(N + 255) / 256, 256, 0, stream>>>(st, perm, N, x_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(float4 *st, const int32_t *perm, int N,
                                 const float *x_in, const float *v_in, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_scatter_state<<<(N + 255) / 256, 256, 0, stream>>>(st, perm, N, x_in, v_in, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_checked_scatter_state(float4 *st, const int32_t *perm, int N, const float *x_in,
                                         const float *v_in, int *first_bad, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_set_int<<<1, 1, 0, stream>>>(first_bad, INT_MAX);
    k_check_finite<<<(N + 255) / 256, 256, 0, stream>>>(x_in, v_in, N, first_bad);
    k_scatter_state<<<(N + 255) / 256, 256, 0, stream>>>(st, perm, N, x_in, v_in, first_bad);
    return cudaGetLastError();
}

}  // namespace ms
