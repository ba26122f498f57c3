// ms_internal.h -- structures shared by the host builder and the step kernels
// of the mass-spring library (library-internal; not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "cronos_ms.h"

#include <nvtx3/nvToolsExt.h>

namespace ms {

// An NVTX range around one API call, for timeline profilers (Nsight
// Systems).  NVTX is header-only: without an attached tool a range costs a
// check of a function pointer.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Records msg as the calling thread's last error and returns st (ms_api.cu).
ms_status fail(ms_status st, const std::string &msg);

// Device layout of one simulation (all pointers are device memory).
//
// Masses are stored in the library's internal order, double buffered (the
// step reads buffer `cur` and writes `cur ^ 1`), packed as in StepArgs below:
//   sa[i] = (x, y, z, vx), sb[i] = (vy, vz), and the constant w[i] = 1/m for
//   a free mass, -m for an anchored one.
//
// Gather layout (kernel 1): springs are stored once, in the row of their lower-indexed endpoint (the
// "owner"), in a sliced-ELL layout with slices of 32 masses (one warp):
//   record (owner o, slot s) lives at  slice[o/32].fwd_off + 32*s + o%32
// with arrays f_nbr (partner index, -1 = padding), f_kl = (k, L0) and
// optionally f_c (per-record damping) and f_ab = (alpha, beta) (actuation).
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
// Back references of robots, robot-local form: owner o (< 4096 masses) in the low 12 bits, the owner's
// record as an offset from the robot's first record above them (< 2^20
// records per robot), or kBackPad.  One dependent load less than the
// (owner, slot) form, which needs the owner's slice header.
constexpr int kRobotOwnerBits = 12;
constexpr uint32_t kRobotOwnerMask = (1u << kRobotOwnerBits) - 1u;
constexpr uint32_t kBackPad = 0xffffffffu;
constexpr int kMaxFwdDegree = 31;

// Kernels of the single-system step.
constexpr int kKernelGather = 1;   // one thread per mass, sliced-ELL rows + back references
constexpr int kKernelTiled = 2;    // CTA per tile of masses, state + halo in shared memory
constexpr int kKernelPersistent = 3; // small systems: all steps in one cluster launch, state in shared memory
constexpr int kTileMasses = 512;   // masses per tile (= threads per CTA)
constexpr int kTileMaxLocal = 2048; // tile members + halo that fit the CTA's shared memory (24 B each)
constexpr int kTileGroup = 3;      // spring slots per pipeline stage (one bulk copy per array)
constexpr int kTileStages = 2;     // pipeline depth
constexpr int kTileStagesDeep = 9; // small systems (one wave of tiles): one stage per slot group, up to 27 slots
constexpr size_t kTileSmemMax = 226 * 1024;   // dynamic shared memory a tiled CTA opts in to (227 KB less its static part)
constexpr int kErrNonFinite = 1;   // bits of the device error flag
constexpr int kErrTimeout = 2;

// State of a single system, packed per mass: a = (x, y, z, vx), b = (vy, vz)
// (double buffered) and w = 1/m, or -m for an anchored mass (constant):
// 28 bytes read and 24 written per mass and step.
struct StepArgs {
    const float4 *sa;    // state at t_n
    const float2 *sb;
    float4 *oa;          // state at t_{n+1}
    float2 *ob;
    const float *w;
    const float4 *fext;  // or nullptr
    const uint4 *slice;
    const int32_t *f_nbr;
    const float2 *f_kl;  // (k, L0)
    const float *f_c;    // or nullptr (then c_uniform)
    const float2 *f_ab;  // (alpha, beta), or nullptr (passive)
    const uint32_t *b_ent;
    int back_local;      // 1: b_ent in the robot-local form, records from back_base
    uint32_t back_base;
    // tiled layout: tiles[2t] = (first mass, members, halo offset, halo count),
    // tiles[2t+1] = (first record slot, slots per member, 0, 0); slot s of
    // member m of tile t is record rec + s*kTileMasses + m (slot-major, so
    // a group of slots for the whole tile is one contiguous range);
    // t_nbr = tile-local partner index (0xffff = padding)
    const uint16_t *t_nbr;
    const int4 *tiles;
    const int32_t *halo;
    int n_tiles;
    int tile_local;      // max members + halo over the tiles (shared-memory entries)
    int max_slots;       // max slots per member over the tiles
    int n_sms;           // multiprocessors of the device (one wave of tiles when n_tiles <= n_sms)
    int tiled;           // 1: tiled layout
    int *err;            // non-finite flag (sticky)
    int N;
    float c_uniform;
    float dt, gx, gy, gz;
    float k_c, mu, keep; // keep = 1 - vel_damping
    float s_n, c_n;      // sin, cos of 2 pi f t_n
    int contact;
    int integrator;      // 0 symplectic Euler, 1 forward Euler, 2 position Verlet, 3 RK4
    int first_step;      // 1 on the first step since creation (Verlet's eq. 5)
    const float4 *rk_ba;     // RK4: the state Y_n of the step (packed as the state)
    const float2 *rk_bb;
    float4 *rk_acc;          // RK4: weighted sum of the stage slopes (2 float4 per mass)
    int rk_stage;            // RK4: stage 0..3
};

// Lattice layout (kernel 4, ms_lattice.cu).  A network whose masses sit on
// the cells of a box lattice, whose springs join cells of the 26-neighbourhood
// (at most one per pair), with one rest length per lattice direction and one
// dashpot coefficient: topology and rest lengths come from the lattice, and
// only k is stored per spring (4 bytes).
//   * Cells live in a padded lattice of X x Y x Z cells (x fastest): one guard
//     cell on every side, and the interior rounded up to whole bricks of
//     kBrickX x kBrickY x kBrickZ cells.  A cell's internal index is its
//     padded lattice index; the caller's mass c sits at cidx[c].
//   * Each of the 13 forward directions d (lat_dx/dy/dz below) has its own
//     array over the padded cells: kf[d][i] = k of the spring from cell i to
//     cell i + off(d); 0 on a slot that touches a cell without a mass (a
//     hole, the guard band), NaN between two masses that have no spring.
//   * Cells without a mass have w = NaN, the position kLatEmptyPos on every
//     axis and zero velocity; no kernel integrates them.
constexpr int kKernelLattice = 4;
constexpr int kBrickX = 16, kBrickY = 16, kBrickZ = 8;
constexpr int kBrickCells = kBrickX * kBrickY * kBrickZ;        // 2048 cells per brick
constexpr int kLatThreads = kBrickCells / 2;                    // 1024: each thread two cells stacked in z
constexpr int kHaloX = kBrickX + 2, kHaloY = kBrickY + 2, kHaloZ = kBrickZ + 2;
constexpr int kHaloCells = kHaloX * kHaloY * kHaloZ;            // 3240 cells staged per brick
constexpr int kLatDirs = 13;
// forward direction d: (1,0,0); then (dx,1,0) for dx = -1..1; then (dx,dy,1) for
// dy = -1..1, dx = -1..1 -- the 13 offsets that are positive in (z, y, x) order
__host__ __device__ constexpr int lat_dx(int d) { return d == 0 ? 1 : d <= 3 ? d - 2 : (d - 4) % 3 - 1; }
__host__ __device__ constexpr int lat_dy(int d) { return d == 0 ? 0 : d <= 3 ? 1 : (d - 4) / 3 - 1; }
__host__ __device__ constexpr int lat_dz(int d) { return d <= 3 ? 0 : 1; }

struct LatticeArgs {
    const float *kf[kLatDirs];   // kf[d][i]: the spring from cell i in direction d
    const float *kb[kLatDirs];   // kb[d][i] = kf[d][i - off(d)]: the spring reaching cell i from direction -d
    float L[kLatDirs];           // rest length per direction
    float c;                     // dashpot coefficient of every spring
    int X, Y, Z;                 // padded extents (cells)
    int nbx, nby, nbz;           // bricks per axis
    int guard;                   // 1: some neighbouring masses have no spring between them (k = NaN there)
    // actuation (act = 1): (alpha, beta) of the spring from cell i in direction d,
    // abf[d][i], and abb[d][i] = abf[d][i - off(d)] as for k; the rest length is
    // L[d] (1 + alpha sin(2 pi f t) + beta cos(2 pi f t))
    const float2 *abf[kLatDirs];
    const float2 *abb[kLatDirs];
    int act;
};
// Cells without a mass (padding, holes) hold this position and zero velocity,
// and every spring slot that touches one holds k = 0: the squared distance to
// such a cell overflows to +inf, 1/l becomes 0, and the spring term is exactly
// zero without a test.
constexpr float kLatEmptyPos = 1e30f;
// Tensor maps (TMA descriptors) of the lattice layout: one pair per state
// buffer that a step reads -- its (x, y, z, vx) array as a 4-D float box and
// its (vy, vz) array as a 3-D box of 8-byte elements -- and one of the 13
// stiffness arrays as a 4-D float box (for L2 prefetch).
struct LatticeMaps {
    static constexpr int kMax = 8;
    int n = 0;
    const void *sa[kMax] = {};
    const void *sb[kMax] = {};
    CUtensorMap a[kMax];
    CUtensorMap b[kMax];
    CUtensorMap k;
};
// adds the pair of state buffer (sa, sb); the stiffness map on the first call
ms_status lattice_maps_add(LatticeMaps &m, const LatticeArgs &g, const float4 *sa, const float2 *sb);
cudaError_t launch_step_lattice(const StepArgs &a, const LatticeArgs &g, const LatticeMaps &m, int n_sms,
                                cudaStream_t st);

// Persistent grid step (ms_step.cu): nsteps steps of the tiled layout in one
// cooperative launch; buffer n & 1 holds the state at step n of the call.
struct GridArgs {
    float4 *buf_a[2];
    float2 *buf_b[2];
    const float2 *sc;        // (sin, cos)(2 pi f t_n) per step, if actuated
    int nsteps;
    unsigned *bar_count;     // grid barrier: arrivals (zeroed before each launch)
    unsigned *bar_gen;       //               generation
    unsigned expected;       // arrivals that complete the barrier (= CTAs; more only in a timeout test)
    unsigned max_polls;      // polls of a barrier wait before the CTA gives up (MS_ERR_TIMEOUT)
};
constexpr unsigned kGridPollsDefault = 1u << 22;
size_t grid_smem_bytes(int tile_local, int slots, bool has_c, bool has_act);
cudaError_t launch_step_grid(const StepArgs &a, const GridArgs &g, cudaStream_t st);

// Energy reduction (ms_instr.cu) over either record layout.
struct EnergyArgs {
    const float4 *sa;        // packed state, as in StepArgs
    const float2 *sb;
    const float *w;
    const uint4 *slice;      // gather layout
    const int32_t *f_nbr;
    const uint16_t *t_nbr;   // tiled layout
    const int4 *tiles;
    const int32_t *halo;
    const float2 *f_kl;
    const float2 *f_ab;      // or nullptr (passive)
    double *partial;         // 4 doubles per block (energy_blocks)
    int N, n_tiles, tiled;
    float s_n, c_n;          // sin, cos of 2 pi f t_n
    float gx, gy, gz, k_c;
    int contact;
};
// lat: the lattice layout's arrays (nullptr for the gather and tiled layouts)
int energy_blocks(const EnergyArgs &a, const LatticeArgs *lat);
// out (device): kinetic, elastic, gravitational, ground-penalty energy (FP64)
cudaError_t launch_energy(const EnergyArgs &a, const LatticeArgs *lat, double *out, cudaStream_t s);
// out[3 q + c] = x[idx[q]][c] for q < n
cudaError_t launch_trace(const float4 *sa, const int32_t *idx, int n, float *out, cudaStream_t s);

// Launchers (ms_step.cu, ms_state.cu).
cudaError_t launch_step(const StepArgs &a, cudaStream_t st);
// perm: internal -> caller index (or nullptr = identity), or cidx: caller -> internal index
cudaError_t launch_gather_state(const float4 *sa, const float2 *sb, const int32_t *perm, const int32_t *cidx, int N,
                                float *x_out, float *v_out, cudaStream_t stream);
cudaError_t launch_scatter_state(float4 *sa, float2 *sb, const float *w, const int32_t *perm, const int32_t *cidx,
                                 int N, const float *x_in, const float *v_in, cudaStream_t stream);
// the same, after a device-side finiteness check of the inputs: first_bad
// (device int) receives the first caller index with a non-finite value, or
// INT_MAX, and the state is written only when every value is finite
cudaError_t launch_checked_scatter_state(float4 *sa, float2 *sb, const float *w, const int32_t *perm,
                                         const int32_t *cidx, int N, const float *x_in, const float *v_in,
                                         int *first_bad, cudaStream_t stream);
// packed state <-> 2 float4 per mass ((x, w), (v, 0)), for n masses
cudaError_t launch_pack_state(const float4 *pairs, int n, float4 *sa, float2 *sb, float *w, cudaStream_t stream);
cudaError_t launch_unpack_state(const float4 *sa, const float2 *sb, const float *w, int n, float4 *pairs,
                                cudaStream_t stream);

}  // namespace ms
