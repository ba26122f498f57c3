// ms_internal.h -- structures shared by the host builder and the step kernels
// of the mass-spring library (library-internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ms {

// Device layout of one simulation (all pointers are device memory).
//
// Masses are stored in the library's internal order as two float4 streams,
// double buffered (the step reads buffer `cur` and writes `cur ^ 1`):
//   x4[i] = (x, y, z, w)   w = 1/m for a free mass, -1 for an anchored mass
//   v4[i] = (vx, vy, vz, 0)
//
// Springs are stored once, in the row of their lower-indexed endpoint (the
// "owner"), in a sliced-ELL layout with slices of 32 masses (one warp):
//   record (owner o, slot s) lives at  slice[o/32].fwd_off + 32*s + o%32
// with arrays f_nbr (partner index, -1 = padding), f_k, f_L0 and optionally
// f_c (per-record damping) and f_al/f_be (actuation coefficients).
// The partner reaches the same record through a back reference stored in
// its own row, also sliced-ELL:
//   b_ent[slice[j/32].bwd_off + 32*t + j%32] = o | (s << 27)  (0xffffffff = padding)
// so every mass can gather all of its springs without atomics.
struct Slice {                 // 16 bytes, read as one uint4
    uint32_t fwd_off;          // first forward record slot of the slice
    uint32_t bwd_off;          // first back-reference slot of the slice
    uint32_t lens;             // fwd_len | (bwd_len << 16): slots per lane
    uint32_t pad;
};

constexpr uint32_t kOwnerBits = 27;
constexpr uint32_t kOwnerMask = (1u << kOwnerBits) - 1u;
constexpr uint32_t kBackPad = 0xffffffffu;
constexpr int kMaxFwdDegree = 31;

struct StepArgs {
    const float4 *x;     // state at t_n
    const float4 *v;
    float4 *xo;          // state at t_{n+1}
    float4 *vo;
    const float4 *fext;  // or nullptr
    const uint4 *slice;
    const int32_t *f_nbr;
    const float *f_k;
    const float *f_L0;
    const float *f_c;    // or nullptr (then c_uniform)
    const float *f_al;   // or nullptr (passive)
    const float *f_be;
    const uint32_t *b_ent;
    int *err;            // non-finite flag (sticky)
    int N;
    float c_uniform;
    float dt, gx, gy, gz;
    float k_c, mu, keep; // keep = 1 - vel_damping
    float s_n, c_n;      // sin, cos of 2 pi f t_n
    int contact;
};

// Launchers (ms_step.cu).
cudaError_t launch_step(const StepArgs &a, cudaStream_t st);
cudaError_t launch_gather_state(const float4 *x4, const float4 *v4, const int32_t *perm, int N,
                                float *x_out, float *v_out, cudaStream_t st);
cudaError_t launch_scatter_state(float4 *x4, float4 *v4, const int32_t *perm, int N,
                                 const float *x_in, const float *v_in, cudaStream_t st);

}  // namespace ms
