// ms_state.cu -- moving the state of a single system between the caller's
// (N, 3) arrays in caller order and the library's internal packed buffers
// (internal order: a = (x, y, z, vx), b = (vy, vz), w = 1/m or -m), and
// between the packed form and 2 float4 per mass ((x, w), (v, 0)).
// The internal order is given either as perm (internal index -> caller
// index, for layouts whose internal indices are 0..N-1) or as cidx (caller
// index -> internal index, for the lattice layout, whose padded index space
// is larger than N).
#include "ms_internal.h"

#include <climits>

namespace ms {
namespace {

// (internal i, caller c) of thread t
__device__ __forceinline__ void index_pair(const int32_t *perm, const int32_t *cidx, int t, int &i, int &c)
{
    if (cidx) { c = t; i = cidx[t]; }
    else { i = t; c = perm ? perm[t] : t; }
}

__global__ void k_gather_state(const float4 *__restrict__ sa, const float2 *__restrict__ sb,
                               const int32_t *__restrict__ perm, const int32_t *__restrict__ cidx, int N,
                               float *__restrict__ xo, float *__restrict__ vo)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int i, c;
    index_pair(perm, cidx, t, i, c);
    const float4 p = sa[i];
    if (xo) { xo[3 * c] = p.x; xo[3 * c + 1] = p.y; xo[3 * c + 2] = p.z; }
    if (vo) { const float2 q = sb[i]; vo[3 * c] = p.w; vo[3 * c + 1] = q.x; vo[3 * c + 2] = q.y; }
}

// skip: if not null and no longer INT_MAX (a non-finite input was found), nothing is written
__global__ void k_scatter_state(float4 *__restrict__ sa, float2 *__restrict__ sb, const float *__restrict__ w,
                                const int32_t *__restrict__ perm, const int32_t *__restrict__ cidx, int N,
                                const float *__restrict__ xi, const float *__restrict__ vi, const int *skip)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    if (skip && *skip != INT_MAX) return;
    int i, c;
    index_pair(perm, cidx, t, i, c);
    float4 p = sa[i];
    if (xi) { p.x = xi[3 * c]; p.y = xi[3 * c + 1]; p.z = xi[3 * c + 2]; }
    if (vi) {
        const bool anchored = w[i] < 0.0f;             // anchored masses keep v = 0
        p.w = anchored ? 0.f : vi[3 * c];
        sb[i] = anchored ? make_float2(0.f, 0.f) : make_float2(vi[3 * c + 1], vi[3 * c + 2]);
    }
    sa[i] = p;
}

__global__ void k_pack_state(const float4 *__restrict__ pairs, int n, float4 *__restrict__ sa,
                             float2 *__restrict__ sb, float *__restrict__ w)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 x = pairs[2 * i], v = pairs[2 * i + 1];
    sa[i] = make_float4(x.x, x.y, x.z, v.x);
    sb[i] = make_float2(v.y, v.z);
    if (w) w[i] = x.w;
}

__global__ void k_unpack_state(const float4 *__restrict__ sa, const float2 *__restrict__ sb,
                               const float *__restrict__ w, int n, float4 *__restrict__ pairs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = sa[i];
    const float2 q = sb[i];
    pairs[2 * i] = make_float4(p.x, p.y, p.z, w[i]);
    pairs[2 * i + 1] = make_float4(p.w, q.x, q.y, 0.f);
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

cudaError_t launch_gather_state(const float4 *sa, const float2 *sb, const int32_t *perm, const int32_t *cidx, int N,
                                float *x_out, float *v_out, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_gather_state<<<(N + 255) / 256, 256, 0, stream>>>(sa, sb, perm, cidx, N, x_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(float4 *sa, float2 *sb, const float *w, const int32_t *perm, const int32_t *cidx,
                                 int N, const float *x_in, const float *v_in, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_scatter_state<<<(N + 255) / 256, 256, 0, stream>>>(sa, sb, w, perm, cidx, N, x_in, v_in, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_checked_scatter_state(float4 *sa, float2 *sb, const float *w, const int32_t *perm,
                                         const int32_t *cidx, int N, const float *x_in, const float *v_in,
                                         int *first_bad, cudaStream_t stream)
{
    if (N <= 0) return cudaSuccess;
    k_set_int<<<1, 1, 0, stream>>>(first_bad, INT_MAX);
    k_check_finite<<<(N + 255) / 256, 256, 0, stream>>>(x_in, v_in, N, first_bad);
    k_scatter_state<<<(N + 255) / 256, 256, 0, stream>>>(sa, sb, w, perm, cidx, N, x_in, v_in, first_bad);
    return cudaGetLastError();
}

cudaError_t launch_pack_state(const float4 *pairs, int n, float4 *sa, float2 *sb, float *w, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    k_pack_state<<<(n + 255) / 256, 256, 0, stream>>>(pairs, n, sa, sb, w);
    return cudaGetLastError();
}

cudaError_t launch_unpack_state(const float4 *sa, const float2 *sb, const float *w, int n, float4 *pairs,
                                cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    k_unpack_state<<<(n + 255) / 256, 256, 0, stream>>>(sa, sb, w, n, pairs);
    return cudaGetLastError();
}

}  // namespace ms
