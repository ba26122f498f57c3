// mlp_tc.cu -- the design surrogate: an MLP 2048 -> 512 -> 512 -> 1 (GELU)
// trained and run on the 5th-generation tensor cores.
//
// Every matrix product is C = A . B^T with A [M x K] and B [N x K] both
// row-major bf16 (K-major), accumulated in fp32 in tensor memory:
//   * one CTA computes a 128 x BN tile of C (BN = 256 when N allows, else
//     128) with four warps, specialised while the K loop runs:
//       - a producer thread (warp 0) streams 128 x 64 tiles of A and BN x 64
//         tiles of B by TMA (cp.async.bulk.tensor, 128-byte swizzle) into a
//         kStages-deep shared-memory ring, refilling a stage as soon as its
//         "empty" mbarrier says the MMAs that read it are done;
//       - an MMA thread (warp 1) waits on each stage's "full" mbarrier and
//         issues tcgen05.mma (cta_group::1, kind::f16, M = 128, N = BN,
//         K = 16 per instruction) into a 128 x BN fp32 accumulator in TMEM,
//         then tcgen05.commit to the stage's "empty" mbarrier;
//     so loads run kStages tiles ahead and the MMAs are issued back to back;
//   * the epilogue warps (sixteen, or eight in the one-hot variant) read the
//     accumulator back with tcgen05.ld (warp w owns TMEM lanes 32(w mod 4)..+31
//     = rows, and one of the column parts) and apply the fused epilogue: plain fp32 store, bias + GELU (forward), or
//     GELU' (backward), writing row-major and transposed bf16 copies as the
//     next product needs.  The last layer's n_hidden -> 1 head is folded into
//     the second layer's epilogue as 16-column partial dot products (summed
//     in a fixed order by a small kernel), so inference never stores H2.
// Every wait is bounded by %globaltimer; on expiry the kernel records a
// timeout in the error flag, stops issuing work and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "ms_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <vector>

namespace ms {
namespace {

constexpr int kBM = 128, kBK = 64;
constexpr int kStages = 4;
// Warp roles: warp 0 loads, warp 1 issues MMAs, the next epi_warps() warps run
// the epilogue, and (one-hot variant) four more warps build the A tiles.
// Sixteen epilogue warps when the K loop is short (the epilogue then sets the
// pace: bias + erf-GELU of the whole tile against a few k-steps of MMAs);
// eight in the one-hot variant, whose long K loop hides its epilogue.
template <bool ONEHOT>
constexpr int epi_warps() { return ONEHOT ? 8 : 16; }
template <bool ONEHOT>
constexpr int gemm_threads() { return 64 + 32 * epi_warps<ONEHOT>() + (ONEHOT ? 128 : 0); }
constexpr uint32_t kTileBytes = kBM * kBK * 2;                  // 16 KB: one 128 x 64 bf16 box
constexpr uint64_t kWaitNs = 2000000000ull;                       // 2 s

enum Epi { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_DGELU = 2 };

struct GemmArgs {
    int M, N, K;
    int epi;
    float *C;                 // EPI_F32: [M][N] fp32
    const float *bias;        // EPI_BIAS_GELU: [N]
    __nv_bfloat16 *Z;         // EPI_BIAS_GELU: pre-activation out [M][N] (or nullptr); EPI_DGELU: pre-activation in
    __nv_bfloat16 *H;         // row-major out [M][N] (GELU(z) or dz)
    __nv_bfloat16 *Ht;        // transposed out [N][M] (or nullptr)
    const uint8_t *mats;      // one-hot A operand: materials [M][n_vox] (ids 0..3), K = 4 n_vox
    int n_vox;
    const float *w3;          // EPI_BIAS_GELU, fused head (or nullptr): head weights [N]
    float *hpart;             // fused head: partial dot products [N / 16][M]
    int *err;
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(n) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(saddr(b)), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait on an mbarrier phase (time limit kWaitNs)
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity)
{
    if (mbar_try(b, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(b, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(saddr(bar))
                 : "memory");
}

// bring [p, p + bytes) into L2 in pieces of at most 16 KB (bytes a multiple
// of 16, p 16-byte aligned)
__device__ __forceinline__ void bulk_prefetch_l2(const uint8_t *p, uint32_t bytes)
{
    for (uint32_t o = 0; o < bytes; o += 16384u) {
        const uint32_t n = bytes - o < 16384u ? bytes - o : 16384u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p + o)), "r"(n) : "memory");
    }
}

// shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), version 1, layout type 2
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fff);
    d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
    d |= (uint64_t)1 << 46;                        // descriptor version
    d |= (uint64_t)2 << 61;                        // SWIZZLE_128B
    return d;
}

// instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = BN
template <int BN>
__host__ __device__ constexpr uint32_t idesc() { return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24); }

template <int BN>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(tmem), "l"(a), "l"(b), "r"(idesc<BN>()), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}

// Epilogue of one CW-column chunk of a thread's row (CW = 16 or 32): r holds
// the fp32 accumulator C[row][nb .. nb + CW - 1].
template <int CW>
__device__ __forceinline__ void epilogue_chunk(const GemmArgs &g, const uint32_t (&r)[CW], int row, int nb)
{
    if (g.epi == EPI_F32) {
        float *dst = g.C + (size_t)row * g.N + nb;
#pragma unroll
        for (int q = 0; q < CW; q += 4)
            *reinterpret_cast<float4 *>(dst + q) = make_float4(__uint_as_float(r[q]), __uint_as_float(r[q + 1]),
                                                               __uint_as_float(r[q + 2]), __uint_as_float(r[q + 3]));
        return;
    }
    __align__(16) __nv_bfloat16 hv[CW], zv[CW];
    if (g.epi == EPI_BIAS_GELU) {
        // bias offsets are multiples of 16 floats by construction: float4 loads
        const float4 *b4 = reinterpret_cast<const float4 *>(g.bias + nb);
#pragma unroll
        for (int q4 = 0; q4 < CW / 4; ++q4) {
            const float4 bq = __ldg(&b4[q4]);
            const float bb[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = 4 * q4 + e;
                zv[q] = __float2bfloat16(__uint_as_float(r[q]) + bb[e]);
                hv[q] = __float2bfloat16(gelu(__bfloat162float(zv[q])));
            }
        }
        if (g.w3) {
            // fused head: this row's dot product with w3 over each 16 columns
#pragma unroll
            for (int q0 = 0; q0 < CW; q0 += 16) {
                const float4 *w4 = reinterpret_cast<const float4 *>(g.w3 + nb + q0);
                float hs = 0.f;
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const float4 w = __ldg(&w4[q4]);
                    const int q = q0 + 4 * q4;
                    hs = fmaf(__bfloat162float(hv[q]), w.x, hs);
                    hs = fmaf(__bfloat162float(hv[q + 1]), w.y, hs);
                    hs = fmaf(__bfloat162float(hv[q + 2]), w.z, hs);
                    hs = fmaf(__bfloat162float(hv[q + 3]), w.w, hs);
                }
                g.hpart[(size_t)((nb + q0) >> 4) * g.M + row] = hs;
            }
        }
    } else {
        const uint4 *zr = reinterpret_cast<const uint4 *>(g.Z + (size_t)row * g.N + nb);
#pragma unroll
        for (int q = 0; q < CW / 8; ++q) reinterpret_cast<uint4 *>(zv)[q] = zr[q];
#pragma unroll
        for (int q = 0; q < CW; ++q)
            hv[q] = __float2bfloat16(__uint_as_float(r[q]) * gelu_grad(__bfloat162float(zv[q])));
    }
    if (g.H) {
        uint4 *dh = reinterpret_cast<uint4 *>(g.H + (size_t)row * g.N + nb);
#pragma unroll
        for (int q = 0; q < CW / 8; ++q) dh[q] = reinterpret_cast<const uint4 *>(hv)[q];
    }
    if (g.epi == EPI_BIAS_GELU && g.Z) {                    // pre-activation kept for the backward pass
        uint4 *dz = reinterpret_cast<uint4 *>(g.Z + (size_t)row * g.N + nb);
#pragma unroll
        for (int q = 0; q < CW / 8; ++q) dz[q] = reinterpret_cast<const uint4 *>(zv)[q];
    }
    if (g.Ht)
#pragma unroll
        for (int q = 0; q < CW; ++q) g.Ht[(size_t)(nb + q) * g.M + row] = hv[q];
}

// tcgen05.ld of CW consecutive fp32 columns of this warp's 32 TMEM lanes
template <int CW>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[CW]);

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                   "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

// Persistent tile loop.  Tiles are 128 x BN, numbered with N fastest (CTAs
// that run at the same time share rows of A in L2); CTA c takes tiles c,
// c + gridDim.x, ...  Warp 0 (one thread) loads, warp 1 (one thread) issues
// the MMAs, the epilogue warps drain the accumulators.  Two accumulators of BN TMEM
// columns alternate between tiles, so the epilogue of one tile overlaps the
// main loop of the next:
//   full[s] / empty[s]        shared-memory stage loaded / read by the MMAs
//   acc_full[a] / acc_empty[a] accumulator a complete / drained by all 256
//                              epilogue threads
// One-hot A tile (ONEHOT): four builder warps write the 128 x 64 bf16 tile of
// X[b][4 v + m] = (materials[b][v] == m) for 16 voxels straight into shared
// memory, in the layout a 128-byte-swizzled TMA load of X would give (row r
// at r * 128 bytes, 16-byte chunk j of the row at chunk j ^ (r mod 8)), so the
// one-hot matrix never exists in global memory.  Builder thread r owns row r;
// the material rows of a CTA's next tile are prefetched into L2 (one bulk
// prefetch) while the current tile is built.
__device__ __forceinline__ uint64_t onehot4(uint32_t m)
{   // the four bf16 (m == 0, .., m == 3) of one voxel, 1.0 = 0x3f80; all zero for m > 3
    return m < 4u ? (uint64_t)0x3f80u << (16u * m) : 0ull;
}

// row r of the tile from its 16 material bytes mv
__device__ __forceinline__ void build_onehot_row(unsigned char *tile, int r, const uint4 mv)
{
    const uint32_t w[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {                    // chunk j: voxels 2j, 2j + 1
        const uint64_t a = onehot4((w[j >> 1] >> (16 * (j & 1))) & 0xffu);
        const uint64_t b = onehot4((w[j >> 1] >> (16 * (j & 1) + 8)) & 0xffu);
        const uint4 c = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
        *reinterpret_cast<uint4 *>(tile + r * 128 + ((j ^ (r & 7)) << 4)) = c;
    }
}

template <int BN, bool ONEHOT>
__global__ void __launch_bounds__(gemm_threads<ONEHOT>(), 1) k_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                             const __grid_constant__ CUtensorMap mapB, const GemmArgs g)
{
    constexpr uint32_t kStageBytes = kTileBytes * (1 + BN / kBM);   // A tile + BN/128 B boxes
    constexpr uint32_t kTxBytes = ONEHOT ? kStageBytes - kTileBytes : kStageBytes;   // bytes the TMA brings
    constexpr int kEW = epi_warps<ONEHOT>();
    static_assert(kEW % 4 == 0 && BN % (32 * (kEW / 4)) == 0, "epilogue split");
    extern __shared__ __align__(1024) unsigned char dyn[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    // 1024-byte aligned ring of stages: A tile then the B tile (BN rows)
    unsigned char *ring = reinterpret_cast<unsigned char *>(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_n = g.N / BN, n_tiles = (g.M / kBM) * tiles_n;
    const int KT = g.K / kBK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)), "r"(2 * BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        // full[s]: the TMA thread's expect_tx arrival, plus the 128 builders after writing a one-hot tile
        for (int s = 0; s < kStages; ++s) { mbar_init(&full[s], ONEHOT ? 1 + kBM : 1); mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { mbar_init(&acc_full[a], 1); mbar_init(&acc_empty[a], 32 * kEW); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // producer: stage s is refilled once the MMAs of k-step it - kStages released it
            unsigned it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                const int n0 = (tile % tiles_n) * BN;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const unsigned s = it % kStages;
                    if (it >= (unsigned)kStages && !mbar_wait(&empty[s], ((it / kStages) - 1) & 1)) { ok = false; break; }
                    unsigned char *a = ring + (size_t)s * kStageBytes;
                    mbar_expect_tx(&full[s], kTxBytes);
                    if (!ONEHOT) tma_load_2d(a, &mapA, kt * kBK, (tile / tiles_n) * kBM, &full[s]);
#pragma unroll
                    for (int q = 0; q < BN / kBM; ++q)
                        tma_load_2d(a + kTileBytes * (1 + q), &mapB, kt * kBK, n0 + q * kBM, &full[s]);
                }
            }
            if (!ok) atomicOr(g.err, kErrTimeout);
        }
    } else if (ONEHOT && warp >= 2 + kEW) {
        // one-hot builders: thread r writes row r of every A tile, with the
        // next k-step's material bytes loaded while the current row is built
        const int r = tid - 32 * (2 + kEW);
        unsigned it = 0;
        bool ok = true;
        if (r == 0 && (int)blockIdx.x < n_tiles)             // the first tile's material rows into L2
            bulk_prefetch_l2(g.mats + (size_t)((blockIdx.x / tiles_n) * kBM) * g.n_vox, kBM * g.n_vox);
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            const int m0 = (tile / tiles_n) * kBM;
            if (r == 0 && tile + (int)gridDim.x < n_tiles)    // and the next tile's, while this one is built
                bulk_prefetch_l2(g.mats + (size_t)(((tile + gridDim.x) / tiles_n) * kBM) * g.n_vox, kBM * g.n_vox);
            const uint4 *src = reinterpret_cast<const uint4 *>(g.mats + (size_t)(m0 + r) * g.n_vox);
            uint4 mv = __ldg(&src[0]);
            for (int kt = 0; kt < KT; ++kt, ++it) {
                const uint4 next = kt + 1 < KT ? __ldg(&src[kt + 1]) : mv;
                const unsigned s = it % kStages;
                if (it >= (unsigned)kStages && !mbar_wait(&empty[s], ((it / kStages) - 1) & 1)) { ok = false; break; }
                build_onehot_row(ring + (size_t)s * kStageBytes, r, mv);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor core
                mbar_arrive(&full[s]);
                mv = next;
            }
        }
        if (!ok && r == 0) atomicOr(g.err, kErrTimeout);
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            unsigned it = 0, lt = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++lt) {
                const unsigned acc = lt & 1u;
                if (lt >= 2 && !mbar_wait(&acc_empty[acc], ((lt / 2) - 1) & 1)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + acc * BN;
                for (int kt = 0; kt < KT; ++kt, ++it) {
                    const unsigned s = it % kStages;
                    if (!mbar_wait(&full[s], (it / kStages) & 1)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a = saddr(ring + (size_t)s * kStageBytes), b = a + kTileBytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)
                        umma<BN>(d, sdesc(a + kk * 32), sdesc(b + kk * 32), (kt | kk) ? 1u : 0u);
                    umma_commit(&empty[s]);                // stage s free once these MMAs have read it
                }
                umma_commit(&acc_full[acc]);               // accumulator complete (or abandoned)
            }
            if (!ok) atomicOr(g.err, kErrTimeout);
        }
    } else if (warp < 2 + kEW) {
        // epilogue: warp w drains TMEM lanes 32 (w mod 4).. and part (w - 2) / 4 of the columns
        constexpr int kParts = kEW / 4, kCols = BN / kParts;
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        unsigned lt = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++lt) {
            const unsigned acc = lt & 1u;
            if (!mbar_wait(&acc_full[acc], (lt / 2) & 1)) {
                if (tid == 64) atomicOr(g.err, kErrTimeout);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (tile / tiles_n) * kBM, n0 = (tile % tiles_n) * BN;
            const int row = m0 + quarter * 32 + lane;
            // sixteen-column chunks where sixteen epilogue warps share the register file
            constexpr int CW = kEW > 8 ? 16 : 32;
            for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += CW) {
                uint32_t r[CW];
                tmem_ld<CW>(tmem + ((uint32_t)(quarter * 32) << 16) + acc * BN + (uint32_t)c0, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                epilogue_chunk<CW>(g, r, row, n0 + c0);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acc_empty[acc]);                  // accumulator acc may be overwritten
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
}

template <int BN>
constexpr size_t gemm_smem() { return (size_t)kStages * kTileBytes * (1 + BN / kBM) + 1024; }

// ---- small kernels of the MLP -------------------------------------------

// one-hot encoding of voxel materials: x[b][4 v + m] = (mat[b][v] == m)
__global__ void k_encode(const uint8_t *mats, int B, int nvox, __nv_bfloat16 *x)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)B * nvox;
    if (i >= n) return;
    const int m = mats[i];
    __nv_bfloat16 *o = x + i * 4;
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = __float2bfloat16(m == q ? 1.f : 0.f);
}

__global__ void k_transpose_bf16(const __nv_bfloat16 *in, int R, int Cc, __nv_bfloat16 *out)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + j, c = bx + threadIdx.x;
        if (r < R && c < Cc) t[j][threadIdx.x] = in[(size_t)r * Cc + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = bx + j, c = by + threadIdx.x;
        if (r < Cc && c < R) out[(size_t)r * R + c] = t[threadIdx.x][j];
    }
}

// y[b] = H2[b] . w3 + b3 from the second layer's 16-column partial sums
// hpart [nparts][B], added in a fixed order
__global__ void k_head_sum(const float *hpart, int nparts, int B, const float *b3, float *y)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float s = 0.f;
    for (int j = 0; j < nparts; ++j) s += hpart[(size_t)j * B + b];
    y[b] = s + b3[0];
}

// dy = (y - t)/B; per-row loss terms
__global__ void k_loss(const float *y, const float *t, int B, float *dy, float *lterm)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float d = y[b] - t[b];
    dy[b] = d / (float)B;
    lterm[b] = 0.5f * d * d / (float)B;
}

// dZ2[b][k] = dy[b] w3[k] GELU'(Z2[b][k]); row-major and transposed bf16
__global__ void k_dhead(const float *dy, const float *w3, const __nv_bfloat16 *Z2, int B, int Hd,
                        __nv_bfloat16 *dZ2, __nv_bfloat16 *dZ2t)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)B * Hd) return;
    const int b = (int)(i / Hd), k = (int)(i % Hd);
    const float g = dy[b] * w3[k] * gelu_grad(__bfloat162float(Z2[i]));
    const __nv_bfloat16 gb = __float2bfloat16(g);
    dZ2[i] = gb;
    dZ2t[(size_t)k * B + b] = gb;
}

// column sums over the batch: out[k] = sum_b M[b][k] (bf16 or fp32 source), fixed order
__global__ void k_colsum_bf16(const __nv_bfloat16 *Mx, int B, int Hd, float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Hd) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += __bfloat162float(Mx[(size_t)b * Hd + k]);
    out[k] = s;
}

// dw3[k] = sum_b dy[b] H2[b][k];  db3 = sum_b dy[b]
__global__ void k_dw3(const float *dy, const __nv_bfloat16 *H2, int B, int Hd, float *dw3, float *db3)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < Hd) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dy[b] * __bfloat162float(H2[(size_t)b * Hd + k]);
        dw3[k] = s;
    }
    if (k == 0) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dy[b];
        db3[0] = s;
    }
}

__global__ void k_sum(const float *v, int n, float *out)
{
    if (blockIdx.x || threadIdx.x) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += v[i];
    out[0] = s;
}

// Adam (bias-corrected), fp32 master weights; refresh the bf16 copy
__global__ void k_adam(float *w, const float *g, float *m, float *v, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *wb)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float *w, size_t n, __nv_bfloat16 *wb)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// ---- host side -----------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

// 2-D tensor map of a row-major bf16 matrix [rows][cols], box 64 x 128, 128-byte swizzle
ms_status make_map(CUtensorMap *map, const void *ptr, int rows, int cols)
{
    auto fn = encode_fn();
    if (!fn) return fail(MS_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if (((uintptr_t)ptr & 15) || (cols * 2) % 16) return fail(MS_ERR_ARG, "tensor map: base or row pitch not 16-byte aligned");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return MS_OK;
}

// C = A . B^T with A [M x K] either a bf16 matrix or, when mats is not null,
// the one-hot encoding of materials [M][K/4] built in shared memory.
ms_status gemm_any(const __nv_bfloat16 *A, const uint8_t *mats, const __nv_bfloat16 *B, int M, int N, int K,
                   const GemmArgs &proto, cudaStream_t st)
{
    if (M % kBM || N % kBM || K % kBK || M <= 0 || N <= 0 || K <= 0)
        return fail(MS_ERR_ARG, "gemm: M and N must be multiples of 128 and K of 64");
    CUtensorMap ma, mb;
    ms_status s;
    if ((s = make_map(&mb, B, N, K)) != MS_OK) return s;
    if (mats) ma = mb;                               // unused: the A tiles are built from mats
    else if ((s = make_map(&ma, A, M, K)) != MS_OK) return s;
    static std::once_flag once;
    static int n_sms = 0;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_gemm_tc<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>());
        cudaFuncSetAttribute(k_gemm_tc<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<256>());
        cudaFuncSetAttribute(k_gemm_tc<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<128>());
        cudaFuncSetAttribute(k_gemm_tc<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_smem<256>());
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sms < 1) n_sms = 1;
    });
    GemmArgs g = proto;
    g.M = M; g.N = N; g.K = K;
    g.mats = mats; g.n_vox = K / 4;
    // 128 x 256 tiles halve the A-tile traffic per FLOP; they need N % 256 == 0
    // and enough tiles to give every SM one
    const int t256 = N % 256 == 0 ? (M / kBM) * (N / 256) : 0;
    const int t128 = (M / kBM) * (N / kBM);
    if (t256 >= n_sms) {
        if (mats) k_gemm_tc<256, true><<<std::min(t256, n_sms), gemm_threads<true>(), gemm_smem<256>(), st>>>(ma, mb, g);
        else k_gemm_tc<256, false><<<std::min(t256, n_sms), gemm_threads<false>(), gemm_smem<256>(), st>>>(ma, mb, g);
    } else {
        if (mats) k_gemm_tc<128, true><<<std::min(t128, n_sms), gemm_threads<true>(), gemm_smem<128>(), st>>>(ma, mb, g);
        else k_gemm_tc<128, false><<<std::min(t128, n_sms), gemm_threads<false>(), gemm_smem<128>(), st>>>(ma, mb, g);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return MS_OK;
}

ms_status gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, const GemmArgs &proto,
               cudaStream_t st)
{
    return gemm_any(A, nullptr, B, M, N, K, proto, st);
}

}  // namespace
}  // namespace ms

using namespace ms;

struct mlp_model {
    int n_in = 0, n_h = 0, max_b = 0;
    cudaStream_t stream = nullptr;
    ms_allocator alloc{};
    bool custom_alloc = false;
    std::vector<std::pair<void *, size_t>> allocs;
    // fp32 master parameters and Adam moments (W1 [h][in], b1, W2 [h][h], b2, w3 [h], b3)
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    size_t off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_w3 = 0, off_b3 = 0, n_par = 0;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2tb = nullptr;
    // activations
    __nv_bfloat16 *X = nullptr, *Xt = nullptr, *Z1 = nullptr, *H1 = nullptr, *H1t = nullptr, *Z2 = nullptr, *H2 = nullptr;
    __nv_bfloat16 *dZ2 = nullptr, *dZ2t = nullptr, *dZ1 = nullptr, *dZ1t = nullptr;
    float *y = nullptr, *dy = nullptr, *lterm = nullptr, *loss = nullptr;
    float *hpart = nullptr;            // the head's 16-column partial sums [n_h / 16][max_b]
    int *err = nullptr;
    // materials of the loaded batch (mlp_encode); X holds their one-hot
    // encoding only once a pass needs it (x_pending = not yet written)
    uint8_t *mats = nullptr;
    bool x_pending = false;
    int64_t t = 0;                     // Adam step

    void *dev_alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *ptr = nullptr;
        if (custom_alloc) ptr = alloc.alloc(bytes, stream, alloc.ctx);
        else if (cudaMalloc(&ptr, bytes) != cudaSuccess) { cudaGetLastError(); ptr = nullptr; }
        if (ptr) allocs.push_back({ptr, bytes});
        return ptr;
    }
    void release()
    {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        for (auto &a : allocs) {
            if (custom_alloc) alloc.free(a.first, a.second, stream, alloc.ctx);
            else cudaFree(a.first);
        }
        allocs.clear();
    }
};

namespace {

#define MLP_CUDA_TRY(expr)                                                                     \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return fail(MS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));     \
    } while (0)

template <class T>
T *mal(mlp_model *m, size_t n) { return (T *)m->dev_alloc(sizeof(T) * n); }

inline unsigned nblk(size_t n, unsigned bs = 256) { return (unsigned)((n + bs - 1) / bs); }

ms_status refresh_bf16(mlp_model *m)
{
    const size_t nw1 = (size_t)m->n_h * m->n_in, nw2 = (size_t)m->n_h * m->n_h;
    k_to_bf16<<<nblk(nw1), 256, 0, m->stream>>>(m->P + m->off_W1, nw1, m->W1b);
    k_to_bf16<<<nblk(nw2), 256, 0, m->stream>>>(m->P + m->off_W2, nw2, m->W2b);
    k_transpose_bf16<<<dim3((m->n_h + 31) / 32, (m->n_h + 31) / 32), dim3(32, 8), 0, m->stream>>>(m->W2b, m->n_h, m->n_h, m->W2tb);
    MLP_CUDA_TRY(cudaGetLastError());
    return MS_OK;
}

// X = one-hot(materials) for a batch loaded by mlp_encode, if not yet written
ms_status ensure_x(mlp_model *m, int B)
{
    if (!m->x_pending) return MS_OK;
    k_encode<<<nblk((size_t)B * (m->n_in / 4)), 256, 0, m->stream>>>(m->mats, B, m->n_in / 4, m->X);
    MLP_CUDA_TRY(cudaGetLastError());
    m->x_pending = false;
    return MS_OK;
}

// keep: also store what the backward pass needs (Z1, Z2, H1^T, and X).
// ext_mats (inference only): the caller's device materials [B][n_in/4], read
// in place by the first GEMM instead of the model's copy.
ms_status forward(mlp_model *m, int B, bool keep, const uint8_t *ext_mats = nullptr)
{
    GemmArgs g{};
    g.err = m->err;
    // Z1 = X W1^T + b1, H1 = GELU(Z1) (and H1^T).  An inference pass on a
    // batch of materials builds the one-hot X tiles inside the GEMM instead.
    g.epi = EPI_BIAS_GELU; g.bias = m->P + m->off_b1; g.Z = keep ? m->Z1 : nullptr; g.H = m->H1;
    g.Ht = keep ? m->H1t : nullptr;
    ms_status s;
    if (!keep && (ext_mats || m->x_pending)) {
        s = gemm_any(nullptr, ext_mats ? ext_mats : m->mats, m->W1b, B, m->n_h, m->n_in, g, m->stream);
    } else {
        if ((s = ensure_x(m, B)) != MS_OK) return s;
        s = gemm(m->X, m->W1b, B, m->n_h, m->n_in, g, m->stream);
    }
    if (s != MS_OK) return s;
    // Z2 = H1 W2^T + b2, H2 = GELU(Z2) (stored for training only), and the
    // head y = H2 w3 + b3 from the epilogue's partial sums
    g.bias = m->P + m->off_b2; g.Z = keep ? m->Z2 : nullptr; g.H = keep ? m->H2 : nullptr; g.Ht = nullptr;
    g.w3 = m->P + m->off_w3; g.hpart = m->hpart;
    if ((s = gemm(m->H1, m->W2b, B, m->n_h, m->n_h, g, m->stream)) != MS_OK) return s;
    k_head_sum<<<nblk(B), 256, 0, m->stream>>>(m->hpart, m->n_h / 16, B, m->P + m->off_b3, m->y);
    MLP_CUDA_TRY(cudaGetLastError());
    return MS_OK;
}

ms_status backward(mlp_model *m, const float *target, int B)
{
    const int H = m->n_h;
    k_loss<<<nblk(B), 256, 0, m->stream>>>(m->y, target, B, m->dy, m->lterm);
    k_sum<<<1, 1, 0, m->stream>>>(m->lterm, B, m->loss);
    k_dw3<<<nblk(H), 256, 0, m->stream>>>(m->dy, m->H2, B, H, m->G + m->off_w3, m->G + m->off_b3);
    k_dhead<<<nblk((size_t)B * H), 256, 0, m->stream>>>(m->dy, m->P + m->off_w3, m->Z2, B, H, m->dZ2, m->dZ2t);
    k_colsum_bf16<<<nblk(H), 256, 0, m->stream>>>(m->dZ2, B, H, m->G + m->off_b2);
    MLP_CUDA_TRY(cudaGetLastError());
    GemmArgs g{};
    g.err = m->err;
    // dW2 = dZ2^T H1   (A = dZ2^T [H x B], B-operand = H1^T [H x B])
    g.epi = EPI_F32; g.C = m->G + m->off_W2;
    ms_status s = gemm(m->dZ2t, m->H1t, H, H, B, g, m->stream);
    if (s != MS_OK) return s;
    // dZ1 = (dZ2 W2) * GELU'(Z1)   (B-operand = W2^T)
    g.epi = EPI_DGELU; g.Z = m->Z1; g.H = m->dZ1; g.Ht = m->dZ1t; g.C = nullptr;
    if ((s = gemm(m->dZ2, m->W2tb, B, H, H, g, m->stream)) != MS_OK) return s;
    k_colsum_bf16<<<nblk(H), 256, 0, m->stream>>>(m->dZ1, B, H, m->G + m->off_b1);
    // dW1 = dZ1^T X   (B-operand = X^T [in x B])
    k_transpose_bf16<<<dim3((m->n_in + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, m->stream>>>(m->X, B, m->n_in, m->Xt);
    MLP_CUDA_TRY(cudaGetLastError());
    g.epi = EPI_F32; g.C = m->G + m->off_W1; g.Z = nullptr; g.H = nullptr; g.Ht = nullptr;
    return gemm(m->dZ1t, m->Xt, H, m->n_in, B, g, m->stream);
}

ms_status check_err(mlp_model *m)
{
    int flag = 0;
    MLP_CUDA_TRY(cudaStreamSynchronize(m->stream));
    MLP_CUDA_TRY(cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & kErrTimeout) return fail(MS_ERR_TIMEOUT, "a tensor-core GEMM wait gave up");
    return MS_OK;
}

ms_status check_batch(mlp_model *m, int B)
{
    if (B < kBM || B > m->max_b || B % kBM) return fail(MS_ERR_ARG, "batch must be a multiple of 128 in [128, max_batch]");
    return MS_OK;
}

}  // namespace

extern "C" {

ms_status mlp_create(int32_t n_in, int32_t n_hidden, int32_t max_batch, uint64_t seed, const ms_allocator *alloc,
                     void *stream, mlp_model **out)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_in <= 0 || n_hidden <= 0 || n_in % kBM || n_hidden % kBM || max_batch < kBM || max_batch % kBM)
        return fail(MS_ERR_ARG, "n_in and n_hidden must be multiples of 128, max_batch a multiple of 128");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(MS_ERR_ARG, "allocator needs alloc and free");
    mlp_model *m = new (std::nothrow) mlp_model();
    if (!m) return fail(MS_ERR_OOM, "host allocation failed");
    struct Guard { mlp_model *m; ~Guard() { if (m) { m->release(); delete m; } } } guard{m};
    m->n_in = n_in; m->n_h = n_hidden; m->max_b = max_batch; m->stream = (cudaStream_t)stream;
    if (alloc) { m->alloc = *alloc; m->custom_alloc = true; }
    const size_t H = n_hidden, I = n_in, B = max_batch;
    m->off_W1 = 0; m->off_b1 = H * I; m->off_W2 = m->off_b1 + H; m->off_b2 = m->off_W2 + H * H;
    m->off_w3 = m->off_b2 + H; m->off_b3 = m->off_w3 + H; m->n_par = m->off_b3 + 1;
    m->P = mal<float>(m, m->n_par); m->G = mal<float>(m, m->n_par);
    m->Mo = mal<float>(m, m->n_par); m->Vo = mal<float>(m, m->n_par);
    m->W1b = mal<__nv_bfloat16>(m, H * I); m->W2b = mal<__nv_bfloat16>(m, H * H); m->W2tb = mal<__nv_bfloat16>(m, H * H);
    m->X = mal<__nv_bfloat16>(m, B * I); m->Xt = mal<__nv_bfloat16>(m, B * I);
    m->Z1 = mal<__nv_bfloat16>(m, B * H); m->H1 = mal<__nv_bfloat16>(m, B * H); m->H1t = mal<__nv_bfloat16>(m, B * H);
    m->Z2 = mal<__nv_bfloat16>(m, B * H); m->H2 = mal<__nv_bfloat16>(m, B * H);
    m->dZ2 = mal<__nv_bfloat16>(m, B * H); m->dZ2t = mal<__nv_bfloat16>(m, B * H);
    m->dZ1 = mal<__nv_bfloat16>(m, B * H); m->dZ1t = mal<__nv_bfloat16>(m, B * H);
    m->y = mal<float>(m, B); m->dy = mal<float>(m, B); m->lterm = mal<float>(m, B); m->loss = mal<float>(m, 1);
    m->err = mal<int>(m, 1);
    m->mats = mal<uint8_t>(m, B * (I / 4));
    m->hpart = mal<float>(m, (H / 16) * B);
    if (!m->mats || !m->hpart) return fail(MS_ERR_OOM, "device allocation failed");
    if (!m->P || !m->G || !m->Mo || !m->Vo || !m->W1b || !m->W2b || !m->W2tb || !m->X || !m->Xt || !m->Z1 ||
        !m->H1 || !m->H1t || !m->Z2 || !m->H2 || !m->dZ2 || !m->dZ2t || !m->dZ1 || !m->dZ1t || !m->y || !m->dy ||
        !m->lterm || !m->loss || !m->err)
        return fail(MS_ERR_OOM, "device allocation failed");
    // initialisation: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) from the seed, biases 0
    std::vector<float> hp(m->n_par, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](size_t off, size_t n, double fan) {
        std::uniform_real_distribution<double> u(-1.0 / std::sqrt(fan), 1.0 / std::sqrt(fan));
        for (size_t i = 0; i < n; ++i) hp[off + i] = (float)u(rng);
    };
    fill(m->off_W1, H * I, (double)I); fill(m->off_W2, H * H, (double)H); fill(m->off_w3, H, (double)H);
    MLP_CUDA_TRY(cudaMemcpyAsync(m->P, hp.data(), sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream));
    MLP_CUDA_TRY(cudaMemsetAsync(m->Mo, 0, sizeof(float) * m->n_par, m->stream));
    MLP_CUDA_TRY(cudaMemsetAsync(m->Vo, 0, sizeof(float) * m->n_par, m->stream));
    MLP_CUDA_TRY(cudaMemsetAsync(m->err, 0, sizeof(int), m->stream));
    ms_status s = refresh_bf16(m);
    if (s != MS_OK) return s;
    MLP_CUDA_TRY(cudaStreamSynchronize(m->stream));
    guard.m = nullptr;
    *out = m;
    return MS_OK;
}

ms_status mlp_set_params(mlp_model *m, const float *params)
{
    if (!m || !params) return fail(MS_ERR_ARG, "model and params are required");
    MLP_CUDA_TRY(cudaMemcpyAsync(m->P, params, sizeof(float) * m->n_par, cudaMemcpyHostToDevice, m->stream));
    ms_status s = refresh_bf16(m);
    if (s != MS_OK) return s;
    MLP_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return MS_OK;
}

ms_status mlp_get_params(mlp_model *m, float *params, float *grads)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    if (params) MLP_CUDA_TRY(cudaMemcpyAsync(params, m->P, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream));
    if (grads) MLP_CUDA_TRY(cudaMemcpyAsync(grads, m->G, sizeof(float) * m->n_par, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return MS_OK;
}

int64_t mlp_num_params(const mlp_model *m) { return m ? (int64_t)m->n_par : 0; }

ms_status mlp_encode(mlp_model *m, const uint8_t *materials, int32_t B)
{
    if (!m || !materials) return fail(MS_ERR_ARG, "model and materials are required");
    ms_status s = check_batch(m, B);
    if (s != MS_OK) return s;
    // keep a copy of the materials; X is encoded when a pass needs it
    MLP_CUDA_TRY(cudaMemcpyAsync(m->mats, materials, (size_t)B * (m->n_in / 4), cudaMemcpyDeviceToDevice, m->stream));
    m->x_pending = true;
    return MS_OK;
}

ms_status mlp_set_input(mlp_model *m, const uint16_t *x_bf16, int32_t B)
{
    if (!m || !x_bf16) return fail(MS_ERR_ARG, "model and input are required");
    ms_status s = check_batch(m, B);
    if (s != MS_OK) return s;
    MLP_CUDA_TRY(cudaMemcpyAsync(m->X, x_bf16, sizeof(uint16_t) * (size_t)B * m->n_in, cudaMemcpyDeviceToDevice, m->stream));
    m->x_pending = false;
    return MS_OK;
}

ms_status mlp_forward(mlp_model *m, int32_t B, float *y)
{
    ms::Range range_("mlp_forward");
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    ms_status s = check_batch(m, B);
    if (s != MS_OK) return s;
    if ((s = forward(m, B, false)) != MS_OK) return s;
    if (y) MLP_CUDA_TRY(cudaMemcpyAsync(y, m->y, sizeof(float) * B, cudaMemcpyDeviceToDevice, m->stream));
    return MS_OK;
}

ms_status mlp_forward_materials(mlp_model *m, const uint8_t *materials, int32_t B, float *y)
{
    ms::Range range_("mlp_forward_materials");
    if (!m || !materials) return fail(MS_ERR_ARG, "model and materials are required");
    ms_status s = check_batch(m, B);
    if (s != MS_OK) return s;
    if ((uintptr_t)materials & 15) return fail(MS_ERR_ARG, "materials must be 16-byte aligned");
    if ((s = forward(m, B, false, materials)) != MS_OK) return s;
    if (y) MLP_CUDA_TRY(cudaMemcpyAsync(y, m->y, sizeof(float) * B, cudaMemcpyDeviceToDevice, m->stream));
    return MS_OK;
}

ms_status mlp_backward(mlp_model *m, const float *target, int32_t B, float *loss)
{
    ms::Range range_("mlp_backward");
    if (!m || !target) return fail(MS_ERR_ARG, "model and target are required");
    ms_status s = check_batch(m, B);
    if (s != MS_OK) return s;
    if ((s = forward(m, B, true)) != MS_OK) return s;
    if ((s = backward(m, target, B)) != MS_OK) return s;
    if (loss) MLP_CUDA_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->stream));
    return MS_OK;
}

ms_status mlp_adam(mlp_model *m, float lr, float beta1, float beta2, float eps)
{
    ms::Range range_("mlp_adam");
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    m->t += 1;
    const float c1 = 1.f - (float)std::pow((double)beta1, (double)m->t), c2 = 1.f - (float)std::pow((double)beta2, (double)m->t);
    k_adam<<<nblk(m->n_par), 256, 0, m->stream>>>(m->P, m->G, m->Mo, m->Vo, m->n_par, lr, beta1, beta2, eps, c1, c2, nullptr);
    MLP_CUDA_TRY(cudaGetLastError());
    return refresh_bf16(m);
}

ms_status mlp_sync(mlp_model *m)
{
    if (!m) return fail(MS_ERR_ARG, "model is NULL");
    return check_err(m);
}

ms_status mlp_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int32_t M, int32_t N, int32_t K, void *stream)
{
    if (!A || !B || !C) return fail(MS_ERR_ARG, "A, B and C are required");
    static int *err = nullptr;
    if (!err) {
        if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return fail(MS_ERR_OOM, "device allocation failed");
        cudaMemset(err, 0, sizeof(int));
    }
    GemmArgs g{};
    g.epi = EPI_F32; g.C = C; g.err = err;
    ms_status s = gemm((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, M, N, K, g, (cudaStream_t)stream);
    if (s != MS_OK) return s;
    int flag = 0;
    MLP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    MLP_CUDA_TRY(cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(MS_ERR_TIMEOUT, "a tensor-core GEMM wait gave up");
    return MS_OK;
}

ms_status mlp_destroy(mlp_model *m)
{
    if (!m) return MS_OK;
    m->release();
    delete m;
    return MS_OK;
}

}  // extern "C"
