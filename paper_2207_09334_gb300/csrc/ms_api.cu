// ms_api.cu -- C ABI entry points and the host-side builder of the
// mass-spring library (see include/cronos_ms.h for the contract).
//
// The builder turns a caller's spring list into the device layout described
// in ms_internal.h:
//   1. optional Morton reordering of the masses by initial position, so that
//      springs connect masses that are close in memory;
//   2. each spring is filed in the row of its lower-indexed endpoint; parallel
//      springs (same pair) are merged (summed k and c, stiffness-weighted rest
//      length), which is exact for a force linear in k and k*L;
//   3. rows are laid out sliced-ELL (32 masses per slice), and every record
//      gets a back reference in its partner's row.
// Everything is O(S) except the optional Morton sort (O(N log N)).
#include "cronos_ms.h"
#include "ms_internal.h"
#include "ms_voxel.h"

#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace {
thread_local std::string g_last_error = "no error";
}  // namespace

namespace ms {
ms_status fail(ms_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace ms

namespace {
using ms::fail;

#define MS_CUDA_TRY(expr)                                                                     \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess)                                                                \
            return fail(MS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));    \
    } while (0)

struct Alloc {
    void *ptr;
    size_t bytes;
};

}  // namespace

struct ms_sim {
    ms_params p{};
    int32_t N = 0;
    int64_t S = 0;
    cudaStream_t stream = nullptr;
    ms_allocator alloc{};
    bool custom_alloc = false;
    std::vector<Alloc> allocs;
    int64_t device_bytes = 0;

    // ordering
    bool permuted = false;
    std::vector<int32_t> perm;      // internal -> caller
    std::vector<int32_t> iperm;     // caller -> internal

    // host copies needed to rebuild actuation coefficients
    std::vector<uint32_t> spring_rec;   // caller spring -> merged record (lattice: the cell it leaves forward)
    std::vector<uint8_t> spring_dir;    // lattice: caller spring -> forward direction
    std::vector<uint32_t> rec_slot_a, rec_slot_b;   // merged record -> device slot(s)
    std::vector<float> k_caller, L0_caller;
    std::vector<double> rec_KL;         // per merged record: sum k * L0

    // device layout
    int n_slices = 0;
    int64_t n_slots = 0, n_back_slots = 0, n_records = 0;
    int max_fwd = 0, max_back = 0;
    int n_sms = 0;                      // multiprocessors of the device the system lives on
    // state, packed and double buffered: sa = (x, y, z, vx), sb = (vy, vz);
    // w = 1/m, or -m for an anchored mass (constant)
    float4 *sa[2] = {nullptr, nullptr};
    float2 *sb[2] = {nullptr, nullptr};
    float *w = nullptr;
    int cur = 0;
    float4 *fext = nullptr;
    uint4 *slice = nullptr;
    int32_t *f_nbr = nullptr;
    float2 *f_kl = nullptr, *f_ab = nullptr;
    float *f_c = nullptr;
    uint32_t *b_ent = nullptr;
    // tiled layout
    int kernel = 0;                     // ms::kKernelGather or ms::kKernelTiled (record layout)
    bool persistent = false;            // stepped by the persistent cluster kernel (ms_cluster.cu)
    bool grid_persistent = false;       // tiled layout stepped by the persistent grid kernel (ms_step.cu)
    unsigned *grid_bar = nullptr;       // its barrier: arrivals, generation
    unsigned grid_polls = ms::kGridPollsDefault;   // polls of a barrier wait before it gives up
    unsigned grid_missing = 0;          // arrivals the barrier waits for beyond the CTAs (timeout test hook)
    uint16_t *cl_nbr = nullptr;         // its records (both directions, lane-interleaved per tile)
    float2 *cl_kl = nullptr, *cl_ab = nullptr;
    float *cl_c = nullptr;
    int cl_slots = 0, cl_tm = 0;        // slots per mass (a multiple of the lanes), masses per tile
    int64_t cl_n = 0;
    std::vector<uint32_t> cl_slot_a, cl_slot_b;   // merged record -> its two cluster slots
    float2 *sc = nullptr;               // (sin, cos) table of a persistent multi-step call
    int sc_cap = 0;
    int n_tiles = 0, max_tile_local = 0;
    uint16_t *t_nbr = nullptr;
    int4 *tiles = nullptr;
    int32_t *halo = nullptr;
    int32_t *d_perm = nullptr;          // internal -> caller index (layouts indexed 0..N-1)
    int32_t *d_cidx = nullptr;          // caller -> internal index (the lattice layout)
    ms::LatticeArgs lat{};              // lattice layout (kernel 4): stiffness arrays, rest lengths, extents
    ms::LatticeMaps lat_maps;           // its tensor maps (TMA descriptors) per state buffer
    int64_t lat_cells = 0;              // padded cells of the lattice layout
    float2 *lat_ab = nullptr;           // lattice actuation: (alpha, beta) per forward slot, 13 x cells
    float *stage = nullptr;             // (N,3)*2 floats for host copies
    int *err = nullptr;
    float c_uniform = 0.f;
    // instrumentation
    double *e_partial = nullptr;        // 4 doubles per energy block, then the 4 results
    int32_t *tr_idx = nullptr;          // traced masses (internal order)
    float *tr_buf = nullptr;            // tr_cap steps x tr_n masses x 3
    int tr_n = 0, tr_cap = 0, tr_count = 0;
    // RK4: two stage states (packed as the state) and the slope accumulator (2 float4 per mass)
    float4 *rk_a[2] = {nullptr, nullptr};
    float2 *rk_b[2] = {nullptr, nullptr};
    float4 *rk_acc = nullptr;

    double freq = 0.0;
    bool actuated = false;
    int64_t step_count = 0;
    double stability = 0.0;

    void *dev_alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        void *ptr = nullptr;
        if (custom_alloc) {
            ptr = alloc.alloc(bytes, stream, alloc.ctx);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            ptr = nullptr;
        }
        if (ptr) {
            allocs.push_back({ptr, bytes});
            device_bytes += (int64_t)bytes;
        }
        return ptr;
    }
    void dev_free(void *ptr)
    {
        for (size_t q = 0; q < allocs.size(); ++q)
            if (allocs[q].ptr == ptr) {
                if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
                if (custom_alloc) alloc.free(ptr, allocs[q].bytes, stream, alloc.ctx);
                else cudaFree(ptr);
                device_bytes -= (int64_t)allocs[q].bytes;
                allocs.erase(allocs.begin() + (long)q);
                return;
            }
    }
    void release()
    {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        for (auto &a : allocs) {
            if (custom_alloc) alloc.free(a.ptr, a.bytes, stream, alloc.ctx);
            else cudaFree(a.ptr);
        }
        allocs.clear();
        device_bytes = 0;
    }
};

namespace {

template <class T>
ms_status upload(ms_sim *s, T **dst, const T *src, size_t count)
{
    *dst = (T *)s->dev_alloc(sizeof(T) * count);
    if (!*dst) return fail(MS_ERR_OOM, "device allocation failed");
    if (src && count) {
        cudaError_t e = cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return fail(MS_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    return MS_OK;
}

uint64_t spread3(uint64_t v)
{   // spread the low 21 bits of v to every third bit
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

bool finite3(const float *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

// ---------------------------------------------------------------------------
// Lattice layout (kernel 4; see ms_internal.h).  lattice_shape checks, on the
// host and without allocating device memory, that the network is a box
// lattice of that form, and fills its arrays; build_lattice uploads them.
// ---------------------------------------------------------------------------
constexpr int32_t kLatticeAutoMin = 1 << 18;   // default kernel: lattice layout from 64^3 masses up

struct LatticeShape {
    int nx = 0, ny = 0, nz = 0, nbx = 0, nby = 0, nbz = 0, X = 0, Y = 0, Z = 0;
    int64_t P = 0;                    // padded cells
    std::vector<int32_t> cidx;        // caller mass -> padded index
    std::vector<float> kf;            // [13][P] stiffness; 0 on a slot that touches a cell without a
                                      // mass, NaN between two masses that have no spring
    bool guard = false;               // some slot between two masses is NaN
    std::vector<uint32_t> owner;      // per caller spring: the cell it leaves in a forward direction
    std::vector<uint8_t> dir;         // ... and that direction
    float L[ms::kLatDirs] = {};
    float c = 0.f;
    std::vector<double> sumK;         // per caller mass: sum of the k of its springs
};

bool lattice_shape(int32_t N, const float *x0, int64_t S, const int32_t *ij, const float *k, const float *c,
                   float c_uniform, const float *rest_len, LatticeShape &L, std::string &why)
{
    if (S == 0) { why = "no springs"; return false; }
    // lattice spacing: the shortest spring
    double h = 0.0;
    for (int64_t e = 0; e < S; ++e) {
        const int32_t a = ij[2 * e], b = ij[2 * e + 1];
        const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                     dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
        const double l = std::sqrt(dx * dx + dy * dy + dz * dz);
        if (!(l > 0.0)) { why = "a spring of zero length"; return false; }
        if (h == 0.0 || l < h) h = l;
    }
    double lo[3] = {x0[0], x0[1], x0[2]}, hi[3] = {x0[0], x0[1], x0[2]};
    for (int32_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], (double)x0[3 * i + a]);
            hi[a] = std::max(hi[a], (double)x0[3 * i + a]);
        }
    // every mass on a grid point: cell indices from the shortest spring, then
    // the spacing of each axis from its extent (the shortest spring carries
    // the FP32 rounding of its endpoints, which would add up over many cells)
    std::vector<int32_t> cell(3 * (size_t)N);
    int64_t ext[3] = {0, 0, 0};
    for (int32_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            const double q = ((double)x0[3 * i + a] - lo[a]) / h;
            const double r = std::nearbyint(q);
            if (std::fabs(q - r) > 0.25 || r > 1048575.0) { why = "masses are not on a cubic grid"; return false; }
            cell[3 * (size_t)i + a] = (int32_t)r;
            ext[a] = std::max<int64_t>(ext[a], (int64_t)r + 1);
        }
    for (int a = 0; a < 3; ++a) {
        const double ha = ext[a] > 1 ? (hi[a] - lo[a]) / (double)(ext[a] - 1) : h;
        for (int32_t i = 0; i < N; ++i)
            if (std::fabs(((double)x0[3 * i + a] - lo[a]) / ha - cell[3 * (size_t)i + a]) > 1e-2) {
                why = "masses are not on a cubic grid";
                return false;
            }
    }
    if (ext[0] * ext[1] * ext[2] > 8 * (int64_t)N + 4096) { why = "the grid is mostly empty"; return false; }
    L.nx = (int)ext[0]; L.ny = (int)ext[1]; L.nz = (int)ext[2];
    L.nbx = (L.nx + ms::kBrickX - 1) / ms::kBrickX;
    L.nby = (L.ny + ms::kBrickY - 1) / ms::kBrickY;
    L.nbz = (L.nz + ms::kBrickZ - 1) / ms::kBrickZ;
    // one guard cell below each axis; above, one in y and z and three in x, so
    // that a row of the float arrays is a multiple of 16 bytes (tensor copies)
    L.X = L.nbx * ms::kBrickX + 4; L.Y = L.nby * ms::kBrickY + 2; L.Z = L.nbz * ms::kBrickZ + 2;
    L.P = (int64_t)L.X * L.Y * L.Z;
    if (L.P >= (int64_t)INT32_MAX / 2) { why = "the padded lattice is too large for 32-bit cell indices"; return false; }
    const int64_t XY = (int64_t)L.X * L.Y;
    L.cidx.resize(N);
    std::vector<uint8_t> used((size_t)L.P, 0);
    for (int32_t i = 0; i < N; ++i) {
        const int64_t ci = (cell[3 * (size_t)i] + 1) + L.X * (int64_t)(cell[3 * (size_t)i + 1] + 1) +
                           XY * (cell[3 * (size_t)i + 2] + 1);
        if (used[ci]) { why = "two masses on one grid point"; return false; }
        used[ci] = 1;
        L.cidx[i] = (int32_t)ci;
    }
    // springs: neighbouring cells, one per pair, one rest length per direction, one dashpot value
    L.c = c ? c[0] : c_uniform;
    bool have_L[ms::kLatDirs] = {};
    L.kf.assign((size_t)ms::kLatDirs * (size_t)L.P, std::numeric_limits<float>::quiet_NaN());
    L.sumK.assign(N, 0.0);
    L.owner.resize(S);
    L.dir.resize(S);
    for (int64_t e = 0; e < S; ++e) {
        int32_t a = ij[2 * e], b = ij[2 * e + 1];
        int dd[3];
        for (int q = 0; q < 3; ++q) dd[q] = cell[3 * (size_t)b + q] - cell[3 * (size_t)a + q];
        if (std::abs(dd[0]) > 1 || std::abs(dd[1]) > 1 || std::abs(dd[2]) > 1) {
            why = "spring " + std::to_string(e) + " joins masses that are not lattice neighbours";
            return false;
        }
        const bool fwd = dd[2] > 0 || (dd[2] == 0 && (dd[1] > 0 || (dd[1] == 0 && dd[0] > 0)));
        if (!fwd) { std::swap(a, b); for (int q = 0; q < 3; ++q) dd[q] = -dd[q]; }
        const int d = dd[2] == 0 ? (dd[1] == 0 ? 0 : dd[0] + 2) : 4 + (dd[0] + 1) + 3 * (dd[1] + 1);
        float Lv;
        if (rest_len) Lv = rest_len[e];
        else {
            const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                         dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
            Lv = (float)std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        if (!have_L[d]) { L.L[d] = Lv; have_L[d] = true; }
        else if (L.L[d] != Lv) { why = "rest lengths differ within one lattice direction"; return false; }
        if (c && c[e] != L.c) { why = "the dashpot coefficient differs between springs"; return false; }
        float &slot = L.kf[(size_t)d * (size_t)L.P + (size_t)L.cidx[a]];
        if (slot == slot) { why = "two springs join the same pair of masses"; return false; }
        slot = k[e];
        L.owner[e] = (uint32_t)L.cidx[a];
        L.dir[e] = (uint8_t)d;
        L.sumK[a] += k[e]; L.sumK[b] += k[e];
    }
    // a slot without a spring: k = 0 where it touches a cell without a mass
    // (that cell sits at the sentinel position, and the term vanishes), NaN
    // between two masses (the kernel then tests every term)
    L.guard = false;
    for (int d = 0; d < ms::kLatDirs; ++d) {
        const int64_t off = ms::lat_dx(d) + (int64_t)L.X * ms::lat_dy(d) + XY * ms::lat_dz(d);   // > 0
        float *kd = &L.kf[(size_t)d * (size_t)L.P];
        for (int64_t i = 0; i < L.P; ++i) {
            if (kd[i] == kd[i]) continue;
            if (used[(size_t)i] && i + off < L.P && used[(size_t)(i + off)]) L.guard = true;
            else kd[i] = 0.f;
        }
    }
    return true;
}

}  // namespace

namespace {

// Upload the lattice layout into s (after lattice_shape succeeded).
ms_status build_lattice(ms_sim *s, const ms_params *p, int32_t N, const float *x0, const float *v0,
                        const float *mass, const uint8_t *fixed, const float *fext, LatticeShape &L)
{
    const size_t P = (size_t)L.P;
    s->kernel = ms::kKernelLattice;
    s->lat_cells = L.P;
    s->n_tiles = L.nbx * L.nby * L.nbz;
    s->max_tile_local = ms::kHaloCells;
    s->n_records = s->S;
    s->n_slots = (int64_t)ms::kLatDirs * L.P;
    s->iperm = L.cidx;
    s->perm.clear();
    s->permuted = true;
    // state of the padded cells: w = NaN and the sentinel position (zero
    // velocity) where there is no mass
    std::vector<float4> ha(P, make_float4(ms::kLatEmptyPos, ms::kLatEmptyPos, ms::kLatEmptyPos, 0.f));
    std::vector<float2> hb(P, make_float2(0.f, 0.f));
    std::vector<float> hw(P, std::numeric_limits<float>::quiet_NaN());
    std::vector<float4> hf;
    if (fext) hf.assign(P, make_float4(0.f, 0.f, 0.f, 0.f));
    double bound = 0.0;
    const double dt2 = (double)p->dt * p->dt;
    for (int32_t m = 0; m < N; ++m) {
        const size_t i = (size_t)L.cidx[m];
        const bool anchored = fixed && fixed[m];
        hw[i] = !anchored ? (float)(1.0 / (double)mass[m])
                : (mass[m] > 0.f && std::isfinite(mass[m])) ? -mass[m] : -FLT_MIN;
        ha[i] = make_float4(x0[3 * m], x0[3 * m + 1], x0[3 * m + 2], anchored ? 0.f : v0[3 * m]);
        hb[i] = anchored ? make_float2(0.f, 0.f) : make_float2(v0[3 * m + 1], v0[3 * m + 2]);
        if (fext) hf[i] = make_float4(fext[3 * m], fext[3 * m + 1], fext[3 * m + 2], 0.f);
        if (!anchored) bound = std::max(bound, dt2 * (2.0 * L.sumK[m] + (p->contact_on ? p->k_c : 0.0)) / mass[m]);
    }
    s->stability = bound;
    if (p->strict_stability && bound >= 4.0) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "stability bound dt^2*max(2 sum k + k_c)/m = %.3g >= 4", bound);
        return fail(MS_ERR_UNSTABLE, buf);
    }
    ms_status st;
    for (int q = 0; q < 2; ++q) {
        if ((st = upload(s, &s->sa[q], ha.data(), P)) != MS_OK) return st;
        if ((st = upload(s, &s->sb[q], hb.data(), P)) != MS_OK) return st;
    }
    if ((st = upload(s, &s->w, hw.data(), P)) != MS_OK) return st;
    if (fext && (st = upload(s, &s->fext, hf.data(), P)) != MS_OK) return st;
    float *kdev = nullptr;
    if ((st = upload(s, &kdev, L.kf.data(), L.kf.size())) != MS_OK) return st;
    const int64_t XY = (int64_t)L.X * L.Y;
    for (int d = 0; d < ms::kLatDirs; ++d) {
        s->lat.kf[d] = kdev + (size_t)d * P;
        // kb[d][i] = kf[d][i - off(d)] for every cell with a mass (whose
        // backward neighbours lie in the padded array); formed as an address
        const int64_t off = ms::lat_dx(d) + (int64_t)L.X * ms::lat_dy(d) + XY * ms::lat_dz(d);
        s->lat.kb[d] = reinterpret_cast<const float *>(reinterpret_cast<uintptr_t>(s->lat.kf[d]) -
                                                       (uintptr_t)(off * (int64_t)sizeof(float)));
        s->lat.L[d] = L.L[d];
    }
    s->lat.c = L.c;
    s->lat.guard = L.guard ? 1 : 0;
    s->lat.act = 0;
    s->spring_rec = std::move(L.owner);
    s->spring_dir = std::move(L.dir);
    s->lat.X = L.X; s->lat.Y = L.Y; s->lat.Z = L.Z;
    s->lat.nbx = L.nbx; s->lat.nby = L.nby; s->lat.nbz = L.nbz;
    if ((st = upload(s, &s->d_cidx, L.cidx.data(), (size_t)N)) != MS_OK) return st;
    if ((st = upload<float>(s, &s->stage, nullptr, (size_t)N * 6)) != MS_OK) return st;
    if (p->integrator == 3) {
        // stage states: cells without a mass are never written, and the next
        // stage stages them as partners, so they start (and stay) at the
        // sentinel state
        for (int q = 0; q < 2; ++q) {
            if ((st = upload(s, &s->rk_a[q], ha.data(), P)) != MS_OK) return st;
            if ((st = upload(s, &s->rk_b[q], hb.data(), P)) != MS_OK) return st;
        }
        if ((st = upload<float4>(s, &s->rk_acc, nullptr, 2 * P)) != MS_OK) return st;
    }
    {
        int dev = 0;
        MS_CUDA_TRY(cudaGetDevice(&dev));
        MS_CUDA_TRY(cudaDeviceGetAttribute(&s->n_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    if ((st = upload<int>(s, &s->err, nullptr, 2)) != MS_OK) return st;
    MS_CUDA_TRY(cudaMemsetAsync(s->err, 0, 2 * sizeof(int), s->stream));
    for (int q = 0; q < 2; ++q) {
        if ((st = ms::lattice_maps_add(s->lat_maps, s->lat, s->sa[q], s->sb[q])) != MS_OK) return st;
        if (p->integrator == 3 && (st = ms::lattice_maps_add(s->lat_maps, s->lat, s->rk_a[q], s->rk_b[q])) != MS_OK)
            return st;
    }
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));      // host arrays must outlive the copies
    return MS_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// ms_create for the general layouts (gather, tiled, persistent), in steps:
// check the input, order the masses, merge parallel springs into records,
// lay the records out for the chosen kernel, build and upload the state.
// ---------------------------------------------------------------------------
struct CreateInput {
    const ms_params *p;
    int32_t N;
    const float *x0, *v0, *mass;
    const uint8_t *fixed;
    const float *fext;
    int64_t S;
    const int32_t *ij;
    const float *k, *c;
    float c_uniform;
    const float *rest_len;
};

// merged spring records in internal order: owner o < partner, records of
// owner o in [rec_first[o], rec_first[o + 1])
struct MergedSprings {
    std::vector<int32_t> deg, bdeg;       // records owned / referenced per mass
    std::vector<int64_t> rec_first;
    std::vector<int32_t> rec_partner;
    std::vector<float2> rec_kl;           // (summed k, stiffness-weighted L0)
    std::vector<float> rec_c;             // summed c (per-spring damping only)
    std::vector<double> sumK;             // per mass: sum of the k of its records
    int64_t n_rec = 0;
};

// host image of the general layouts before upload
struct GeneralLayout {
    int n_slices = 0;
    int64_t n_slots = 0;
    std::vector<uint32_t> slot_a, slot_b;
    std::vector<ms::Slice> sl;
    std::vector<int32_t> h_nbr;
    std::vector<uint16_t> h_nbr16;
    std::vector<uint32_t> h_b;
    std::vector<int4> h_tiles;
    std::vector<int32_t> h_halo;
    std::vector<float2> h_kl;
    std::vector<float> h_c;
    std::vector<uint16_t> c_nbr;          // persistent cluster layout
    std::vector<float2> c_kl;
    std::vector<float> c_c;
};

// Every argument check, before any allocation (host only).
ms_status check_create_input(const CreateInput &in, const ms_allocator *alloc)
{
    const ms_params *p = in.p;
    const int32_t N = in.N;
    const float *x0 = in.x0;
    const float *v0 = in.v0;
    const float *mass = in.mass;
    const float *fext = in.fext;
    const uint8_t *fixed = in.fixed;
    const int64_t S = in.S;
    const int32_t *ij = in.ij;
    const float *k = in.k;
    const float *c = in.c;
    const float *rest_len = in.rest_len;
    const float c_uniform = in.c_uniform;
    if (!p || !x0 || !v0 || !mass) return fail(MS_ERR_ARG, "p, x0, v0 and mass are required");
    if (N < 1 || N >= (1 << ms::kOwnerBits)) return fail(MS_ERR_ARG, "N must be in [1, 2^27)");
    if (S < 0 || (S > 0 && (!ij || !k))) return fail(MS_ERR_ARG, "S < 0, or ij / k missing");
    if (!(p->dt > 0.f) || !std::isfinite(p->dt)) return fail(MS_ERR_ARG, "dt must be positive and finite");
    if (p->integrator < 0 || p->integrator > 3)
        return fail(MS_ERR_ARG, "integrator must be 0 (symplectic Euler), 1 (forward Euler), 2 (Verlet) or 3 (RK4)");
    if (p->integrator >= 2 && (p->mu > 0.f || p->vel_damping != 0.f))
        return fail(MS_ERR_ARG, "the Verlet and RK4 integrators take no friction and no global damping");
    if (!(p->vel_damping >= 0.f && p->vel_damping < 1.f)) return fail(MS_ERR_ARG, "vel_damping must be in [0, 1)");
    if (p->contact_on && !(p->k_c >= 0.f && p->mu >= 0.f)) return fail(MS_ERR_ARG, "k_c and mu must be >= 0");
    if (!c && !(c_uniform >= 0.f && std::isfinite(c_uniform))) return fail(MS_ERR_ARG, "c_uniform must be >= 0");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(MS_ERR_ARG, "allocator needs alloc and free");

    for (int32_t i = 0; i < N; ++i) {
        const bool anchored = fixed && fixed[i];
        if (!finite3(x0 + 3 * i) || !finite3(v0 + 3 * i)) return fail(MS_ERR_ARG, "non-finite position or velocity at mass " + std::to_string(i));
        if (!anchored && !(mass[i] > 0.f && std::isfinite(mass[i]))) return fail(MS_ERR_ARG, "mass must be positive and finite at mass " + std::to_string(i));
        if (fext && !finite3(fext + 3 * i)) return fail(MS_ERR_ARG, "non-finite external force at mass " + std::to_string(i));
    }

    for (int64_t e = 0; e < S; ++e) {
        const int32_t a = ij[2 * e], b = ij[2 * e + 1];
        if (a < 0 || a >= N || b < 0 || b >= N) return fail(MS_ERR_ARG, "spring endpoint out of range at spring " + std::to_string(e));
        if (a == b) return fail(MS_ERR_ARG, "spring joins a mass to itself at spring " + std::to_string(e));
        if (!(k[e] >= 0.f && std::isfinite(k[e]))) return fail(MS_ERR_ARG, "k must be >= 0 and finite at spring " + std::to_string(e));
        if (c && !(c[e] >= 0.f && std::isfinite(c[e]))) return fail(MS_ERR_ARG, "c must be >= 0 and finite at spring " + std::to_string(e));
        if (rest_len && !(rest_len[e] >= 0.f && std::isfinite(rest_len[e]))) return fail(MS_ERR_ARG, "rest length must be >= 0 and finite at spring " + std::to_string(e));
    }
    return MS_OK;
}

// Mass order: Morton order by initial position for the tiled and persistent
// kernels (or when asked for), else the caller's.
void order_masses(ms_sim *s, const CreateInput &in, bool persistent)
{
    const ms_params *p = in.p;
    const int32_t N = in.N;
    const float *x0 = in.x0;
    const int64_t S = in.S;
    const int32_t *ij = in.ij;
    // 1. mass order
    s->perm.resize(N); s->iperm.resize(N);
    for (int32_t i = 0; i < N; ++i) s->perm[i] = i;
    const bool morton = p->reorder == 1 || (p->reorder == 0 && (s->kernel == ms::kKernelTiled || persistent));
    if (morton) {
        float lo[3] = {x0[0], x0[1], x0[2]}, hi[3] = {x0[0], x0[1], x0[2]};
        for (int32_t i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], x0[3 * i + a]); hi[a] = std::max(hi[a], x0[3 * i + a]); }
        double ext = 0; for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)hi[a] - lo[a]);
        // quantise by the shortest spring, so a lattice maps to its integer
        // cell coordinates and Morton blocks are aligned cubes of cells
        double h = 0.0;
        for (int64_t e = 0; e < S; ++e) {
            const int32_t a = ij[2 * e], b = ij[2 * e + 1];
            const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                         dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
            const double l = std::sqrt(dx * dx + dy * dy + dz * dz);
            if (l > 0 && (h == 0.0 || l < h)) h = l;
        }
        double scale = h > 0 ? 1.0 / h : 0.0;
        if (ext * scale >= 2097151.0 || scale == 0.0) scale = ext > 0 ? 2097151.0 / ext : 0.0;
        std::vector<std::pair<uint64_t, int32_t>> key(N);
        for (int32_t i = 0; i < N; ++i) {
            uint64_t code = 0;
            for (int a = 0; a < 3; ++a) code |= spread3((uint64_t)(((double)x0[3 * i + a] - lo[a]) * scale + 0.5)) << a;
            key[i] = {code, i};
        }
        std::sort(key.begin(), key.end());
        for (int32_t i = 0; i < N; ++i) s->perm[i] = key[i].second;
        s->permuted = true;
    }
    for (int32_t i = 0; i < N; ++i) s->iperm[s->perm[i]] = i;
}

// File springs by owner and merge parallel springs into records.
ms_status merge_springs(ms_sim *s, const CreateInput &in, MergedSprings &M)
{
    const int32_t N = in.N;
    const float *x0 = in.x0;
    const int64_t S = in.S;
    const int32_t *ij = in.ij;
    const float *k = in.k;
    const float *c = in.c;
    const float *rest_len = in.rest_len;
    // 2. file springs by owner (counting sort), merge parallel springs into
    //    records: (owner < partner) in internal order, grouped by owner.
    std::vector<int64_t> row(N + 1, 0);
    for (int64_t e = 0; e < S; ++e) {
        const int32_t a = ij[2 * e], b = ij[2 * e + 1];
        row[std::min(s->iperm[a], s->iperm[b]) + 1]++;
    }
    for (int32_t i = 0; i < N; ++i) row[i + 1] += row[i];
    std::vector<int32_t> r_other(S), r_spring(S);
    {
        std::vector<int64_t> fill(row.begin(), row.end() - 1);
        for (int64_t e = 0; e < S; ++e) {
            const int32_t a = s->iperm[ij[2 * e]], b = s->iperm[ij[2 * e + 1]];
            const int32_t o = std::min(a, b);
            const int64_t at = fill[o]++;
            r_other[at] = std::max(a, b);
            r_spring[at] = (int32_t)e;
        }
    }
    // sort each row by (partner, spring) and merge equal partners
    std::vector<int32_t> deg(N, 0), bdeg(N, 0);
    std::vector<int64_t> rec_first(N + 1, 0);       // merged records of owner o: [rec_first[o], rec_first[o+1])
    std::vector<int32_t> rec_partner;
    std::vector<float2> rec_kl;
    std::vector<float> rec_c;
    rec_partner.reserve(S); rec_kl.reserve(S); rec_c.reserve(c ? S : 0);
    s->rec_KL.clear(); s->rec_KL.reserve(S);
    s->spring_rec.resize(S);
    std::vector<double> sumK(N, 0.0);
    for (int32_t o = 0; o < N; ++o) {
        const int64_t b0 = row[o], b1 = row[o + 1];
        for (int64_t q = b0 + 1; q < b1; ++q) {      // insertion sort (rows are short)
            const int32_t vo = r_other[q], vs = r_spring[q];
            int64_t t = q - 1;
            while (t >= b0 && (r_other[t] > vo || (r_other[t] == vo && r_spring[t] > vs))) {
                r_other[t + 1] = r_other[t]; r_spring[t + 1] = r_spring[t]; --t;
            }
            r_other[t + 1] = vo; r_spring[t + 1] = vs;
        }
        rec_first[o] = (int64_t)rec_partner.size();
        for (int64_t q = b0; q < b1;) {
            const int32_t j = r_other[q];
            const uint32_t m = (uint32_t)rec_partner.size();
            double K = 0, KL = 0, Lsum = 0, Csum = 0;
            int cnt = 0;
            for (; q < b1 && r_other[q] == j; ++q) {
                const int32_t e = r_spring[q];
                double L;
                if (rest_len) L = rest_len[e];
                else {
                    const int32_t a = ij[2 * e], b = ij[2 * e + 1];
                    const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                                 dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
                    L = (double)(float)std::sqrt(dx * dx + dy * dy + dz * dz);
                }
                K += k[e]; KL += (double)k[e] * L; Lsum += L; Csum += c ? c[e] : 0.0; ++cnt;
                s->spring_rec[e] = m;
            }
            rec_partner.push_back(j);
            rec_kl.push_back(make_float2((float)K, (float)(K > 0 ? KL / K : Lsum / cnt)));
            if (c) rec_c.push_back((float)Csum);
            s->rec_KL.push_back(K > 0 ? KL : 0.0);
            deg[o]++; bdeg[j]++;
            sumK[o] += K; sumK[j] += K;
        }
    }
    rec_first[N] = (int64_t)rec_partner.size();
    const int64_t n_rec = (int64_t)rec_partner.size();
    s->n_records = n_rec;
    r_other.clear(); r_other.shrink_to_fit(); r_spring.clear(); r_spring.shrink_to_fit();
    if (n_rec >= (int64_t)UINT32_MAX / 2) return fail(MS_ERR_ARG, "too many springs for 32-bit record offsets");
    M.deg.swap(deg); M.bdeg.swap(bdeg); M.rec_first.swap(rec_first); M.rec_partner.swap(rec_partner);
    M.rec_kl.swap(rec_kl); M.rec_c.swap(rec_c); M.sumK.swap(sumK);
    M.n_rec = n_rec;
    return MS_OK;
}

// Records laid out for the tiled kernel (falling back to the gather layout
// when a tile does not fit shared memory) or for the gather kernel.
ms_status build_rows(ms_sim *s, const CreateInput &in, const MergedSprings &M, bool persistent, bool cluster_fits,
                     GeneralLayout &G)
{
    const int32_t N = in.N;
    const float *x0 = in.x0;
    const float *c = in.c;
    const auto &deg = M.deg;
    const auto &bdeg = M.bdeg;
    const auto &rec_first = M.rec_first;
    const auto &rec_partner = M.rec_partner;
    const auto &rec_kl = M.rec_kl;
    const auto &rec_c = M.rec_c;
    const int64_t n_rec = M.n_rec;
    // 3. device layout of the chosen kernel
    const int n_slices = (N + 31) / 32;
    s->n_slices = n_slices;
    std::vector<uint32_t> slot_a(n_rec, 0), slot_b(n_rec, UINT32_MAX);   // record -> its slot(s)
    std::vector<ms::Slice> sl;
    std::vector<int32_t> h_nbr;
    std::vector<uint16_t> h_nbr16;
    std::vector<uint32_t> h_b;
    std::vector<int4> h_tiles;
    std::vector<int32_t> h_halo;
    std::vector<float2> h_kl;
    std::vector<float> h_c;
    int64_t n_slots = 0;
    if (s->kernel == ms::kKernelTiled) {
        std::fill(slot_a.begin(), slot_a.end(), UINT32_MAX);
        // every mass lists all of its springs (both directions); partners are
        // tile-local indices: members 0..nb-1, then the tile's halo
        const int B = ms::kTileMasses;
        const int n_tiles = (N + B - 1) / B;
        std::vector<int64_t> inc_first(N + 1, 0);
        for (int32_t i = 0; i < N; ++i) inc_first[i + 1] = inc_first[i] + deg[i] + bdeg[i];
        std::vector<int32_t> inc_p(inc_first[N]);
        std::vector<uint32_t> inc_m(inc_first[N]);
        {
            std::vector<int64_t> fill(inc_first.begin(), inc_first.end() - 1);
            // masses ascending: each mass first sees its lower partners (as j), then its own records
            for (int32_t o = 0; o < N; ++o)
                for (int64_t m = rec_first[o]; m < rec_first[o + 1]; ++m) {
                    const int32_t j = rec_partner[m];
                    inc_p[fill[o]] = j; inc_m[fill[o]++] = (uint32_t)m;
                    inc_p[fill[j]] = o; inc_m[fill[j]++] = (uint32_t)m;
                }
        }
        int max_deg = 0;
        for (int32_t i = 0; i < N; ++i) max_deg = std::max<int>(max_deg, (int)(inc_first[i + 1] - inc_first[i]));
        if (max_deg > 0xffff) return fail(MS_ERR_ARG, "a mass has more than 65535 springs");
        // Slot order inside a row.  When every mass's springs point in
        // distinct directions of the 26-neighbourhood (a lattice), slot q is
        // the direction q for every mass, so the 32 lanes of a warp read
        // partners that are one shifted block of the Morton order (few
        // shared-memory bank conflicts).  Otherwise rows are compact, in
        // partner order.
        std::vector<int8_t> inc_dir(inc_p.size(), -1);
        bool by_dir = true;
        for (int32_t i = 0; i < N && by_dir; ++i) {
            const float *xi = x0 + 3 * (size_t)s->perm[i];
            uint32_t seen = 0;
            for (int64_t q = inc_first[i]; q < inc_first[i + 1]; ++q) {
                const float *xj = x0 + 3 * (size_t)s->perm[inc_p[q]];
                const double d[3] = {(double)xj[0] - xi[0], (double)xj[1] - xi[1], (double)xj[2] - xi[2]};
                const double L = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                int t[3];
                for (int a = 0; a < 3; ++a) t[a] = d[a] > 0.25 * L ? 1 : (d[a] < -0.25 * L ? -1 : 0);
                int code = (t[2] + 1) * 9 + (t[1] + 1) * 3 + (t[0] + 1);
                if (code == 13 || L == 0.0) { by_dir = false; break; }
                if (code > 13) --code;                    // 0..25
                if (seen & (1u << code)) { by_dir = false; break; }
                seen |= 1u << code;
                inc_dir[q] = (int8_t)code;
            }
        }
        sl.assign(n_slices, ms::Slice{0, 0, 0, 0});
        h_tiles.resize(2 * (size_t)n_tiles);
        std::vector<int32_t> halo;
        int max_local = 0;
        for (int t = 0; t < n_tiles; ++t) {
            const int32_t base = t * B, nb = std::min(B, N - base);
            halo.clear();
            int slots = 0;
            for (int32_t i = base; i < base + nb; ++i) {
                if (by_dir) {
                    for (int64_t q = inc_first[i]; q < inc_first[i + 1]; ++q) slots = std::max<int>(slots, inc_dir[q] + 1);
                } else {
                    slots = std::max<int>(slots, (int)(inc_first[i + 1] - inc_first[i]));
                }
                for (int64_t q = inc_first[i]; q < inc_first[i + 1]; ++q)
                    if (inc_p[q] < base || inc_p[q] >= base + nb) halo.push_back(inc_p[q]);
            }
            std::sort(halo.begin(), halo.end());
            halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
            const int nloc = nb + (int)halo.size();
            max_local = std::max(max_local, nloc);
            if (nloc > ms::kTileMaxLocal) {
                if (s->p.kernel == ms::kKernelTiled || s->grid_persistent)
                    return fail(MS_ERR_ARG, "tile " + std::to_string(t) + " needs " + std::to_string(nloc) +
                                                " shared-memory entries (> " + std::to_string(ms::kTileMaxLocal) + ")");
                s->kernel = ms::kKernelGather;       // fall back to the gather layout
                break;
            }
            h_tiles[2 * t] = make_int4(base, nb, (int)h_halo.size(), (int)halo.size());
            h_tiles[2 * t + 1] = make_int4((int)n_slots, slots, 0, 0);
            h_halo.insert(h_halo.end(), halo.begin(), halo.end());
            n_slots += (int64_t)slots * B;
            if (n_slots >= (int64_t)INT32_MAX) return fail(MS_ERR_ARG, "too many spring slots for 32-bit offsets");
            s->max_fwd = std::max(s->max_fwd, slots);
        }
        if (s->kernel == ms::kKernelTiled) {
            s->max_tile_local = max_local;
            s->n_tiles = n_tiles;
            h_nbr16.assign(n_slots, 0xffffu);
            h_kl.assign(n_slots, make_float2(0.f, 0.f));
            if (c) h_c.assign(n_slots, 0.f);
            for (int t = 0; t < n_tiles; ++t) {
                const int4 T = h_tiles[2 * t], R = h_tiles[2 * t + 1];
                const int32_t *hb = h_halo.data() + T.z;
                // a padding slot of a member points at the member itself (zero
                // length, k = 0: no force), so the kernel needs no test for it
                for (int sl2 = 0; sl2 < R.y; ++sl2)
                    for (int m = 0; m < T.y; ++m) h_nbr16[(size_t)R.x + (size_t)sl2 * B + m] = (uint16_t)m;
                for (int32_t i = T.x; i < T.x + T.y; ++i) {
                    int slot = 0;
                    for (int64_t q = inc_first[i]; q < inc_first[i + 1]; ++q, ++slot) {
                        if (by_dir) slot = inc_dir[q];
                        const int32_t pidx = inc_p[q];
                        int loc;
                        if (pidx >= T.x && pidx < T.x + T.y) loc = pidx - T.x;
                        else loc = T.y + (int)(std::lower_bound(hb, hb + T.w, pidx) - hb);
                        const uint32_t r = (uint32_t)R.x + (uint32_t)slot * B + (uint32_t)(i - T.x);
                        const uint32_t m = inc_m[q];
                        h_nbr16[r] = (uint16_t)loc;
                        h_kl[r] = rec_kl[m];
                        if (c) h_c[r] = rec_c[m];
                        if (slot_a[m] == UINT32_MAX) slot_a[m] = r; else slot_b[m] = r;
                    }
                }
            }
        }
    }
    if (s->kernel == ms::kKernelGather) {
        sl.assign(n_slices, ms::Slice{0, 0, 0, 0});
        n_slots = 0;
        for (int b = 0; b < n_slices; ++b) {
            int mx = 0;
            for (int l = 0; l < 32 && 32 * b + l < N; ++l) mx = std::max(mx, deg[32 * b + l]);
            if (mx > ms::kMaxFwdDegree) {
                int who = 0;
                for (int l = 0; l < 32 && 32 * b + l < N; ++l) if (deg[32 * b + l] == mx) who = 32 * b + l;
                return fail(MS_ERR_ARG, "mass " + std::to_string(s->perm[who]) + " owns " + std::to_string(mx) +
                                            " distinct partners after ordering; at most 31 are supported");
            }
            sl[b].fwd_off = (uint32_t)n_slots;
            sl[b].lens = (uint32_t)mx;
            n_slots += 32LL * mx;
            s->max_fwd = std::max(s->max_fwd, mx);
        }
        h_nbr.assign(n_slots, -1);
        h_kl.assign(n_slots, make_float2(0.f, 0.f));
        if (c) h_c.assign(n_slots, 0.f);
        for (int32_t o = 0; o < N; ++o) {
            const uint32_t base = sl[o >> 5].fwd_off + (uint32_t)(o & 31);
            for (int64_t m = rec_first[o]; m < rec_first[o + 1]; ++m) {
                const uint32_t r = base + 32u * (uint32_t)(m - rec_first[o]);
                h_nbr[r] = rec_partner[m];
                h_kl[r] = rec_kl[m];
                if (c) h_c[r] = rec_c[m];
                slot_a[m] = r;
            }
        }
        int64_t boff = 0;
        for (int b = 0; b < n_slices; ++b) {
            int mx = 0;
            for (int l = 0; l < 32 && 32 * b + l < N; ++l) mx = std::max(mx, bdeg[32 * b + l]);
            if (mx > 0xffff) return fail(MS_ERR_ARG, "a mass has more than 65535 lower-indexed partners");
            sl[b].bwd_off = (uint32_t)boff;
            sl[b].lens |= (uint32_t)mx << 16;
            boff += 32LL * mx;
            s->max_back = std::max(s->max_back, mx);
        }
        if (boff >= (int64_t)UINT32_MAX) return fail(MS_ERR_ARG, "too many back-reference slots for 32-bit offsets");
        s->n_back_slots = boff;
        h_b.assign(boff, ms::kBackPad);
        std::vector<int32_t> bfill(N, 0);
        for (int32_t o = 0; o < N; ++o)            // owners ascending: back lists sorted by owner
            for (int64_t m = rec_first[o]; m < rec_first[o + 1]; ++m) {
                const int32_t j = rec_partner[m];
                const int t = bfill[j]++;
                const uint32_t slot = (uint32_t)(m - rec_first[o]);
                h_b[sl[j >> 5].bwd_off + 32u * (uint32_t)t + (uint32_t)(j & 31)] = (uint32_t)o | (slot << ms::kOwnerBits);
            }
    }
    s->n_slots = n_slots;
    s->persistent = persistent && cluster_fits;
    s->rec_slot_a.swap(slot_a);
    s->rec_slot_b.swap(slot_b);
    G.n_slices = n_slices; G.n_slots = n_slots;
    G.sl.swap(sl); G.h_nbr.swap(h_nbr); G.h_nbr16.swap(h_nbr16); G.h_b.swap(h_b);
    G.h_tiles.swap(h_tiles); G.h_halo.swap(h_halo); G.h_kl.swap(h_kl); G.h_c.swap(h_c);
    return MS_OK;
}

// Records of the persistent cluster kernel (small systems).
ms_status build_cluster_rows(ms_sim *s, const CreateInput &in, const MergedSprings &M, GeneralLayout &G)
{
    const int32_t N = in.N;
    const float *c = in.c;
    const auto &rec_first = M.rec_first;
    const auto &rec_partner = M.rec_partner;
    const auto &rec_kl = M.rec_kl;
    const auto &rec_c = M.rec_c;
    const int64_t n_rec = M.n_rec;
    // persistent cluster layout: tiles of CM masses, the smallest of 64, 128,
    // 256, 512 that needs at most kClusterMax tiles; every mass lists all of
    // its springs (both directions), the slots of its L lanes interleaved,
    // the partner coded by its mass index
    std::vector<uint16_t> c_nbr;
    std::vector<float2> c_kl;
    std::vector<float> c_c;
    if (s->persistent) {
        int CM = 64;
        while (CM < ms::kClMassesMax && (int64_t)CM * ms::kClusterMax < N) CM *= 2;
        const int LN = ms::kClThreads / CM;
        const int tiles = (N + CM - 1) / CM;
        std::vector<std::vector<std::pair<int32_t, uint32_t>>> inc(N);   // (partner, record)
        for (int32_t o = 0; o < N; ++o)
            for (int64_t m = rec_first[o]; m < rec_first[o + 1]; ++m) {
                inc[o].push_back({rec_partner[m], (uint32_t)m});
                inc[rec_partner[m]].push_back({o, (uint32_t)m});
            }
        int slots = 1;
        for (int32_t i = 0; i < N; ++i) slots = std::max<int>(slots, (int)inc[i].size());
        slots = (slots + LN - 1) / LN * LN;
        if (ms::cluster_smem_bytes(CM, slots, c != nullptr, false) > 227 * 1024)
            return fail(MS_ERR_ARG, "the persistent kernel's records of " + std::to_string(slots) + " springs per mass over " +
                                        std::to_string(CM) + "-mass tiles do not fit shared memory");
        const size_t per_tile = (size_t)slots * CM;
        c_nbr.assign((size_t)tiles * per_tile, 0);
        c_kl.assign((size_t)tiles * per_tile, make_float2(0.f, 0.f));
        if (c) c_c.assign((size_t)tiles * per_tile, 0.f);
        s->cl_slot_a.assign(n_rec, UINT32_MAX);
        s->cl_slot_b.assign(n_rec, UINT32_MAX);
        for (int32_t i = 0; i < N; ++i) {
            const int t = i / CM, mi = i % CM;
            auto rec_at = [&](int q) {
                return (size_t)t * per_tile + ((size_t)(q / LN) * CM + mi) * LN + (size_t)(q % LN);
            };
            for (int q = 0; q < slots; ++q) c_nbr[rec_at(q)] = (uint16_t)i;   // padding: the mass itself, (k, L0) = 0
            for (size_t q = 0; q < inc[i].size(); ++q) {
                const size_t r = rec_at((int)q);
                const uint32_t m = inc[i][q].second;
                c_nbr[r] = (uint16_t)inc[i][q].first;
                c_kl[r] = rec_kl[m];
                if (c) c_c[r] = rec_c[m];
                if (s->cl_slot_a[m] == UINT32_MAX) s->cl_slot_a[m] = (uint32_t)r; else s->cl_slot_b[m] = (uint32_t)r;
            }
        }
        s->cl_tm = CM;
        s->cl_slots = slots;
        s->cl_n = (int64_t)tiles * per_tile;
    }
    G.c_nbr.swap(c_nbr); G.c_kl.swap(c_kl); G.c_c.swap(c_c);
    return MS_OK;
}

// The masses' state (internal order), the stability bound, and the upload of
// every array of the chosen layout.
ms_status upload_general(ms_sim *s, const CreateInput &in, const MergedSprings &M, GeneralLayout &G)
{
    const ms_params *p = in.p;
    const int32_t N = in.N;
    const float *x0 = in.x0;
    const float *v0 = in.v0;
    const float *mass = in.mass;
    const float *fext = in.fext;
    const uint8_t *fixed = in.fixed;
    const float *c = in.c;
    const auto &sumK = M.sumK;
    const int n_slices = G.n_slices;
    const int64_t n_slots = G.n_slots;
    const auto &sl = G.sl;
    const auto &h_nbr = G.h_nbr;
    const auto &h_nbr16 = G.h_nbr16;
    const auto &h_b = G.h_b;
    const auto &h_tiles = G.h_tiles;
    const auto &h_halo = G.h_halo;
    const auto &h_kl = G.h_kl;
    const auto &h_c = G.h_c;
    const auto &c_nbr = G.c_nbr;
    const auto &c_kl = G.c_kl;
    const auto &c_c = G.c_c;
    // masses
    std::vector<float4> ha(N), hf;
    std::vector<float2> hb(N);
    std::vector<float> hw(N);
    double bound = 0.0;
    const double dt2 = (double)p->dt * p->dt;
    for (int32_t i = 0; i < N; ++i) {
        const int32_t cidx = s->perm[i];
        const bool anchored = fixed && fixed[cidx];
        // free: 1/m; anchored: -m (a mass of zero or less is stored as the
        // smallest negative normal, so the sign still marks the anchor)
        const float w = !anchored ? (float)(1.0 / (double)mass[cidx])
                        : (mass[cidx] > 0.f && std::isfinite(mass[cidx])) ? -mass[cidx] : -FLT_MIN;
        ha[i] = make_float4(x0[3 * cidx], x0[3 * cidx + 1], x0[3 * cidx + 2], anchored ? 0.f : v0[3 * cidx]);
        hb[i] = anchored ? make_float2(0.f, 0.f) : make_float2(v0[3 * cidx + 1], v0[3 * cidx + 2]);
        hw[i] = w;
        if (!anchored) bound = std::max(bound, dt2 * (2.0 * sumK[i] + (p->contact_on ? p->k_c : 0.0)) / mass[cidx]);
    }
    s->stability = bound;
    if (p->strict_stability && bound >= 4.0) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "stability bound dt^2*max(2 sum k + k_c)/m = %.3g >= 4", bound);
        return fail(MS_ERR_UNSTABLE, buf);
    }
    if (fext) {
        hf.resize(N);
        for (int32_t i = 0; i < N; ++i) {
            const int32_t cidx = s->perm[i];
            hf[i] = make_float4(fext[3 * cidx], fext[3 * cidx + 1], fext[3 * cidx + 2], 0.f);
        }
    }

    // 4. device upload
    ms_status st;
    for (int q = 0; q < 2; ++q) {
        if ((st = upload(s, &s->sa[q], ha.data(), N)) != MS_OK) return st;
        if ((st = upload(s, &s->sb[q], hb.data(), N)) != MS_OK) return st;
    }
    if ((st = upload(s, &s->w, hw.data(), N)) != MS_OK) return st;
    if (fext && (st = upload(s, &s->fext, hf.data(), N)) != MS_OK) return st;
    static_assert(sizeof(ms::Slice) == sizeof(uint4), "slice size");
    if ((st = upload(s, &s->slice, (const uint4 *)sl.data(), n_slices)) != MS_OK) return st;
    if ((st = upload(s, &s->f_kl, h_kl.data(), n_slots)) != MS_OK) return st;
    if (c && (st = upload(s, &s->f_c, h_c.data(), n_slots)) != MS_OK) return st;
    if (s->kernel == ms::kKernelGather) {
        if ((st = upload(s, &s->f_nbr, h_nbr.data(), n_slots)) != MS_OK) return st;
        if ((st = upload(s, &s->b_ent, h_b.data(), h_b.size())) != MS_OK) return st;
    } else {
        if ((st = upload(s, &s->t_nbr, h_nbr16.data(), h_nbr16.size())) != MS_OK) return st;
        if ((st = upload(s, &s->tiles, h_tiles.data(), h_tiles.size())) != MS_OK) return st;
        if ((st = upload(s, &s->halo, h_halo.data(), h_halo.size())) != MS_OK) return st;
    }
    if (s->permuted && (st = upload(s, &s->d_perm, s->perm.data(), N)) != MS_OK) return st;
    if ((st = upload<float>(s, &s->stage, nullptr, (size_t)N * 6)) != MS_OK) return st;
    if (s->persistent) {
        if ((st = upload(s, &s->cl_nbr, c_nbr.data(), c_nbr.size())) != MS_OK) return st;
        if ((st = upload(s, &s->cl_kl, c_kl.data(), c_kl.size())) != MS_OK) return st;
        if (c && (st = upload(s, &s->cl_c, c_c.data(), c_c.size())) != MS_OK) return st;
    }
    if (p->integrator == 3) {
        for (int q = 0; q < 2; ++q) {
            if ((st = upload<float4>(s, &s->rk_a[q], nullptr, (size_t)N)) != MS_OK) return st;
            if ((st = upload<float2>(s, &s->rk_b[q], nullptr, (size_t)N)) != MS_OK) return st;
        }
        if ((st = upload<float4>(s, &s->rk_acc, nullptr, 2 * (size_t)N)) != MS_OK) return st;
    }
    {
        int dev = 0;
        MS_CUDA_TRY(cudaGetDevice(&dev));
        MS_CUDA_TRY(cudaDeviceGetAttribute(&s->n_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    if (s->grid_persistent) {
        if (s->n_tiles > s->n_sms)
            return fail(MS_ERR_ARG, "the persistent kernel takes one tile of " + std::to_string(ms::kTileMasses) +
                                        " masses per multiprocessor: " + std::to_string(s->n_tiles) + " tiles > " +
                                        std::to_string(s->n_sms));
        if (ms::grid_smem_bytes(s->max_tile_local, s->max_fwd, c != nullptr, false) > ms::kTileSmemMax)
            return fail(MS_ERR_ARG, "the persistent kernel's tile records do not fit shared memory");
        if ((st = upload<unsigned>(s, &s->grid_bar, nullptr, 2)) != MS_OK) return st;
        MS_CUDA_TRY(cudaMemsetAsync(s->grid_bar, 0, 2 * sizeof(unsigned), s->stream));
    }
    // err[0]: sticky device error flags; err[1]: scratch of ms_set_state's finiteness check
    if ((st = upload<int>(s, &s->err, nullptr, 2)) != MS_OK) return st;
    MS_CUDA_TRY(cudaMemsetAsync(s->err, 0, 2 * sizeof(int), s->stream));
    // host arrays must outlive the asynchronous copies
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return MS_OK;
}

// The caller's k and rest lengths, kept for ms_set_actuation's merge.
void keep_caller_springs(ms_sim *s, const CreateInput &in)
{
    const float *x0 = in.x0;
    const int64_t S = in.S;
    const int32_t *ij = in.ij;
    const float *k = in.k;
    const float *rest_len = in.rest_len;
    s->k_caller.assign(k, k + S);
    s->L0_caller.resize(S);
    for (int64_t e = 0; e < S; ++e) {
        if (rest_len) s->L0_caller[e] = rest_len[e];
        else {
            const int32_t a = ij[2 * e], b = ij[2 * e + 1];
            const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                         dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
            s->L0_caller[e] = (float)std::sqrt(dx * dx + dy * dy + dz * dz);
        }
    }
}

}  // namespace

extern "C" {

const char *ms_last_error(void) { return g_last_error.c_str(); }

const char *ms_version(void) { return "cronos-ms-gb300 0.1 (sm_103a)"; }

ms_status ms_create(const ms_params *p, int32_t N, const float *x0, const float *v0, const float *mass,
                    const uint8_t *fixed, const float *fext, int64_t S, const int32_t *ij, const float *k,
                    const float *c, float c_uniform, const float *rest_len, const ms_allocator *alloc,
                    void *stream, ms_sim **out)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    const CreateInput in{p, N, x0, v0, mass, fixed, fext, S, ij, k, c, c_uniform, rest_len};
    ms_status st = check_create_input(in, alloc);
    if (st != MS_OK) return st;

    ms_sim *s = new (std::nothrow) ms_sim();
    if (!s) return fail(MS_ERR_OOM, "host allocation failed");
    struct Guard { ms_sim *s; ~Guard() { if (s) { s->release(); delete s; } } } guard{s};
    s->p = *p; s->N = N; s->S = S;
    s->stream = (cudaStream_t)stream;
    if (alloc) { s->alloc = *alloc; s->custom_alloc = true; }
    s->c_uniform = c_uniform;

    if (p->kernel < 0 || p->kernel > 4 || p->reorder < 0 || p->reorder > 2) return fail(MS_ERR_ARG, "kernel must be 0..4 and reorder 0..2");
    // lattice layout: when asked for, or by default for a large box lattice
    if (p->kernel == ms::kKernelLattice || (p->kernel == 0 && N >= kLatticeAutoMin)) {
        LatticeShape L;
        std::string why;
        if (lattice_shape(N, x0, S, ij, k, c, c_uniform, rest_len, L, why)) {
            if ((st = build_lattice(s, p, N, x0, v0, mass, fixed, fext, L)) != MS_OK) return st;
            guard.s = nullptr;
            *out = s;
            return MS_OK;
        }
        if (p->kernel == ms::kKernelLattice) return fail(MS_ERR_ARG, "not a lattice for the lattice kernel: " + why);
    }
    if (p->kernel == 3 && p->integrator != 0)
        return fail(MS_ERR_ARG, "the persistent kernel integrates with symplectic Euler only");
    // persistent: up to kClusterMax x kClMassesMax masses one thread-block
    // cluster; above, the tiled layout in one cooperative launch (one wave of tiles)
    const bool cluster_fits = N <= ms::kClMassesMax * ms::kClusterMax;
    s->kernel = p->kernel == 1 ? ms::kKernelGather
              : p->kernel == 2 ? ms::kKernelTiled
              : p->kernel == 3 ? ms::kKernelPersistent
              : ms::kKernelTiled;
    const bool persistent = s->kernel == ms::kKernelPersistent;
    s->grid_persistent = persistent && !cluster_fits;
    // the cluster kernel keeps the gather layout (for the energy kernel); the grid kernel steps the tiled one
    if (persistent) s->kernel = cluster_fits ? ms::kKernelGather : ms::kKernelTiled;

    order_masses(s, in, persistent);
    MergedSprings M;
    if ((st = merge_springs(s, in, M)) != MS_OK) return st;
    GeneralLayout G;
    if ((st = build_rows(s, in, M, persistent, cluster_fits, G)) != MS_OK) return st;
    if ((st = build_cluster_rows(s, in, M, G)) != MS_OK) return st;
    if ((st = upload_general(s, in, M, G)) != MS_OK) return st;
    keep_caller_springs(s, in);
    guard.s = nullptr;
    *out = s;
    return MS_OK;
}

ms_status ms_create_materials(const ms_params *p, int32_t N, const float *x0, const float *v0, const float *mass,
                              const uint8_t *fixed, const float *fext, int64_t S, const int32_t *ij,
                              const uint16_t *mat, int32_t n_mat, const float *mat_k, const float *mat_c,
                              const float *mat_L0scale, const float *rest_len, const ms_allocator *alloc,
                              void *stream, ms_sim **out)
{
    if (!out) return fail(MS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!x0) return fail(MS_ERR_ARG, "x0 is required");
    if (S < 0 || (S > 0 && (!ij || !mat))) return fail(MS_ERR_ARG, "S < 0, or ij / mat missing");
    if (n_mat < 1 || n_mat > 65536 || !mat_k) return fail(MS_ERR_ARG, "need 1 <= n_mat <= 65536 and mat_k");
    for (int32_t q = 0; q < n_mat; ++q) {
        if (!(mat_k[q] >= 0.f && std::isfinite(mat_k[q]))) return fail(MS_ERR_ARG, "mat_k must be >= 0 and finite at material " + std::to_string(q));
        if (mat_c && !(mat_c[q] >= 0.f && std::isfinite(mat_c[q]))) return fail(MS_ERR_ARG, "mat_c must be >= 0 and finite at material " + std::to_string(q));
        if (mat_L0scale && !(mat_L0scale[q] >= 0.f && std::isfinite(mat_L0scale[q])))
            return fail(MS_ERR_ARG, "mat_L0scale must be >= 0 and finite at material " + std::to_string(q));
    }
    // expand the tables into the per-spring form of ms_create
    std::vector<float> k(S), c, L0;
    bool uniform_c = true;
    for (int64_t e = 0; e < S; ++e) {
        if (mat[e] >= (uint32_t)n_mat) return fail(MS_ERR_ARG, "material id out of range at spring " + std::to_string(e));
        k[e] = mat_k[mat[e]];
        if (mat_c && mat_c[mat[e]] != mat_c[mat[0]]) uniform_c = false;
    }
    if (mat_c && !uniform_c) {
        c.resize(S);
        for (int64_t e = 0; e < S; ++e) c[e] = mat_c[mat[e]];
    }
    const float c_uniform = (mat_c && S > 0) ? mat_c[mat[0]] : 0.f;
    if (mat_L0scale) {
        L0.resize(S);
        for (int64_t e = 0; e < S; ++e) {
            const int32_t a = ij[2 * e], b = ij[2 * e + 1];
            if (a < 0 || a >= N || b < 0 || b >= N) return fail(MS_ERR_ARG, "spring endpoint out of range at spring " + std::to_string(e));
            float base;
            if (rest_len) base = rest_len[e];
            else {
                const double dx = (double)x0[3 * b] - x0[3 * a], dy = (double)x0[3 * b + 1] - x0[3 * a + 1],
                             dz = (double)x0[3 * b + 2] - x0[3 * a + 2];
                base = (float)std::sqrt(dx * dx + dy * dy + dz * dz);
            }
            L0[e] = base * mat_L0scale[mat[e]];       // one FP32 rounding
        }
    }
    return ms_create(p, N, x0, v0, mass, fixed, fext, S, ij, S > 0 ? k.data() : nullptr,
                     c.empty() ? nullptr : c.data(), c_uniform, mat_L0scale ? (S > 0 ? L0.data() : nullptr) : rest_len,
                     alloc, stream, out);
}

ms_status ms_set_actuation(ms_sim *s, float freq_hz, const float *amp, const float *phase)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (!amp) { s->actuated = false; s->freq = 0.0; s->lat.act = 0; return MS_OK; }
    if (!phase) return fail(MS_ERR_ARG, "phase is required with amp");
    if (!std::isfinite(freq_hz)) return fail(MS_ERR_ARG, "freq must be finite");
    if (s->kernel == ms::kKernelLattice) {
        // one spring per pair: alpha = A cos(phi), beta = A sin(phi) in the slot of
        // the cell the spring leaves forward (reading R3 of the actuated rest length)
        const size_t P = (size_t)s->lat_cells;
        std::vector<float2> abh((size_t)ms::kLatDirs * P, make_float2(0.f, 0.f));
        for (int64_t e = 0; e < s->S; ++e) {
            if (!std::isfinite(amp[e]) || !std::isfinite(phase[e]))
                return fail(MS_ERR_ARG, "non-finite amp or phase at spring " + std::to_string(e));
            abh[(size_t)s->spring_dir[e] * P + s->spring_rec[e]] =
                make_float2((float)((double)amp[e] * std::cos((double)phase[e])),
                            (float)((double)amp[e] * std::sin((double)phase[e])));
        }
        ms_status st;
        if (!s->lat_ab && (st = upload<float2>(s, &s->lat_ab, nullptr, abh.size())) != MS_OK) return st;
        MS_CUDA_TRY(cudaMemcpyAsync(s->lat_ab, abh.data(), sizeof(float2) * abh.size(), cudaMemcpyHostToDevice, s->stream));
        const int64_t XY = (int64_t)s->lat.X * s->lat.Y;
        for (int d = 0; d < ms::kLatDirs; ++d) {
            s->lat.abf[d] = s->lat_ab + (size_t)d * P;
            const int64_t off = ms::lat_dx(d) + (int64_t)s->lat.X * ms::lat_dy(d) + XY * ms::lat_dz(d);
            s->lat.abb[d] = reinterpret_cast<const float2 *>(reinterpret_cast<uintptr_t>(s->lat.abf[d]) -
                                                             (uintptr_t)(off * (int64_t)sizeof(float2)));
        }
        MS_CUDA_TRY(cudaStreamSynchronize(s->stream));    // the host array must outlive the copy
        s->lat.act = 1;
        s->actuated = true;
        s->freq = freq_hz;
        return MS_OK;
    }
    if ((s->persistent && ms::cluster_smem_bytes(s->cl_tm, s->cl_slots, s->cl_c != nullptr, true) > 227 * 1024) ||
        (s->grid_persistent && ms::grid_smem_bytes(s->max_tile_local, s->max_fwd, s->f_c != nullptr, true) > ms::kTileSmemMax))
        return fail(MS_ERR_ARG, "the persistent kernel cannot hold the actuation coefficients of this system in "
                                "shared memory; create it with the tiled kernel");
    const int64_t S = s->S, nrec = s->n_records, n = s->n_slots;
    std::vector<double> sa(nrec, 0.0), sb(nrec, 0.0);
    for (int64_t e = 0; e < S; ++e) {
        if (!std::isfinite(amp[e]) || !std::isfinite(phase[e])) return fail(MS_ERR_ARG, "non-finite amp or phase at spring " + std::to_string(e));
        const double w = (double)s->k_caller[e] * s->L0_caller[e] * amp[e];
        const uint32_t m = s->spring_rec[e];
        sa[m] += w * std::cos((double)phase[e]);    // coefficient of sin(2 pi f t)
        sb[m] += w * std::sin((double)phase[e]);    // coefficient of cos(2 pi f t)
    }
    std::vector<float2> ab(n, make_float2(0.f, 0.f));
    for (int64_t m = 0; m < nrec; ++m) {
        if (!(s->rec_KL[m] > 0)) continue;
        const float2 v = make_float2((float)(sa[m] / s->rec_KL[m]), (float)(sb[m] / s->rec_KL[m]));
        ab[s->rec_slot_a[m]] = v;
        if (s->rec_slot_b[m] != UINT32_MAX) ab[s->rec_slot_b[m]] = v;
    }
    ms_status st;
    if (!s->f_ab && (st = upload<float2>(s, &s->f_ab, nullptr, n)) != MS_OK) return st;
    MS_CUDA_TRY(cudaMemcpyAsync(s->f_ab, ab.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s->stream));
    std::vector<float2> cab;
    if (s->persistent) {
        cab.assign(s->cl_n, make_float2(0.f, 0.f));
        for (int64_t m = 0; m < nrec; ++m) {
            if (!(s->rec_KL[m] > 0)) continue;
            const float2 v = make_float2((float)(sa[m] / s->rec_KL[m]), (float)(sb[m] / s->rec_KL[m]));
            if (s->cl_slot_a[m] != UINT32_MAX) cab[s->cl_slot_a[m]] = v;
            if (s->cl_slot_b[m] != UINT32_MAX) cab[s->cl_slot_b[m]] = v;
        }
        if (!s->cl_ab && (st = upload<float2>(s, &s->cl_ab, nullptr, (size_t)s->cl_n)) != MS_OK) return st;
        MS_CUDA_TRY(cudaMemcpyAsync(s->cl_ab, cab.data(), sizeof(float2) * (size_t)s->cl_n, cudaMemcpyHostToDevice, s->stream));
    }
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->actuated = true;
    s->freq = freq_hz;
    return MS_OK;
}

ms_status ms_step(ms_sim *s, int32_t nsteps)
{
    ms::Range range_("ms_step");
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (nsteps < 0) return fail(MS_ERR_ARG, "nsteps must be >= 0");
    const double two_pi_f = 2.0 * M_PI * s->freq;
    if (s->persistent) {
        if (nsteps == 0) return MS_OK;
        const float2 *sc = nullptr;
        if (s->actuated) {
            if (nsteps > s->sc_cap) {
                ms_status st = upload<float2>(s, &s->sc, nullptr, (size_t)nsteps);
                if (st != MS_OK) return st;
                s->sc_cap = nsteps;
            }
            ms::launch_sc_table_from(s->step_count, nsteps, (double)s->p.dt, two_pi_f, s->sc, s->stream);
            MS_CUDA_TRY(cudaGetLastError());
            sc = s->sc;
        }
        ms::ClusterArgs ca{};
        ca.sa = s->sa[s->cur]; ca.sb = s->sb[s->cur]; ca.w = s->w; ca.fext = s->fext;
        ca.nbr = s->cl_nbr; ca.kl = s->cl_kl; ca.c = s->cl_c; ca.ab = s->actuated ? s->cl_ab : nullptr;
        ca.c_uniform = s->c_uniform; ca.N = s->N; ca.slots = s->cl_slots; ca.tm = s->cl_tm;
        ca.sc = sc; ca.nsteps = nsteps; ca.env = ms::make_env(s->p); ca.err = s->err;
        MS_CUDA_TRY(ms::launch_cluster(ca, s->stream));
        s->step_count += nsteps;
        return MS_OK;
    }
    ms::StepArgs a{};
    a.w = s->w;
    a.fext = s->fext; a.slice = s->slice; a.f_nbr = s->f_nbr; a.f_kl = s->f_kl;
    a.f_c = s->f_c; a.f_ab = s->actuated ? s->f_ab : nullptr;
    a.b_ent = s->b_ent; a.err = s->err; a.N = s->N; a.c_uniform = s->c_uniform;
    a.t_nbr = s->t_nbr; a.tiles = s->tiles; a.halo = s->halo; a.n_tiles = s->n_tiles;
    a.tile_local = s->max_tile_local; a.tiled = s->kernel == ms::kKernelTiled;
    a.max_slots = s->max_fwd; a.n_sms = s->n_sms;
    a.dt = s->p.dt; a.gx = s->p.g[0]; a.gy = s->p.g[1]; a.gz = s->p.g[2];
    a.k_c = s->p.k_c; a.mu = s->p.mu; a.keep = 1.0f - s->p.vel_damping; a.contact = s->p.contact_on;
    a.integrator = s->p.integrator;
    a.rk_acc = s->rk_acc;
    if (s->grid_persistent) {
        if (nsteps == 0) return MS_OK;
        const float2 *sc = nullptr;
        if (s->actuated) {
            if (nsteps > s->sc_cap) {
                ms_status st = upload<float2>(s, &s->sc, nullptr, (size_t)nsteps);
                if (st != MS_OK) return st;
                s->sc_cap = nsteps;
            }
            ms::launch_sc_table_from(s->step_count, nsteps, (double)s->p.dt, two_pi_f, s->sc, s->stream);
            MS_CUDA_TRY(cudaGetLastError());
            sc = s->sc;
        }
        ms::GridArgs gr{};
        gr.buf_a[0] = s->sa[s->cur]; gr.buf_a[1] = s->sa[s->cur ^ 1];
        gr.buf_b[0] = s->sb[s->cur]; gr.buf_b[1] = s->sb[s->cur ^ 1];
        gr.sc = sc; gr.nsteps = nsteps; gr.bar_count = s->grid_bar; gr.bar_gen = s->grid_bar + 1;
        gr.expected = (unsigned)s->n_tiles + s->grid_missing;
        gr.max_polls = s->grid_polls;
        MS_CUDA_TRY(ms::launch_step_grid(a, gr, s->stream));
        s->cur ^= nsteps & 1;
        s->step_count += nsteps;
        return MS_OK;
    }
    const bool lattice = s->kernel == ms::kKernelLattice;
    for (int32_t n = 0; n < nsteps; ++n) {
        a.first_step = (s->step_count + n == 0) ? 1 : 0;
        const double t = (double)(s->step_count + n) * (double)s->p.dt;
        if (s->p.integrator == 3) {
            // four stage launches: Y_0 = Y_n -> rk stage 0 -> rk stage 1 -> rk stage 0 -> Y_{n+1};
            // stage q sees the actuation at t_n + c_q dt, c = 0, 1/2, 1/2, 1
            static const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};
            a.rk_ba = s->sa[s->cur]; a.rk_bb = s->sb[s->cur];
            for (int q = 0; q < 4; ++q) {
                if (s->actuated) {
                    const double tq = t + c_stage[q] * (double)s->p.dt;
                    a.s_n = (float)std::sin(two_pi_f * tq);
                    a.c_n = (float)std::cos(two_pi_f * tq);
                }
                a.rk_stage = q;
                a.sa = q == 0 ? s->sa[s->cur] : s->rk_a[(q - 1) & 1];
                a.sb = q == 0 ? s->sb[s->cur] : s->rk_b[(q - 1) & 1];
                a.oa = q == 3 ? s->sa[s->cur ^ 1] : s->rk_a[q & 1];
                a.ob = q == 3 ? s->sb[s->cur ^ 1] : s->rk_b[q & 1];
                MS_CUDA_TRY(lattice ? ms::launch_step_lattice(a, s->lat, s->lat_maps, s->n_sms, s->stream)
                                    : ms::launch_step(a, s->stream));
            }
        } else {
            if (s->actuated) {
                a.s_n = (float)std::sin(two_pi_f * t);
                a.c_n = (float)std::cos(two_pi_f * t);
            }
            a.sa = s->sa[s->cur]; a.sb = s->sb[s->cur];
            a.oa = s->sa[s->cur ^ 1]; a.ob = s->sb[s->cur ^ 1];
            MS_CUDA_TRY(lattice ? ms::launch_step_lattice(a, s->lat, s->lat_maps, s->n_sms, s->stream)
                                    : ms::launch_step(a, s->stream));
        }
        s->cur ^= 1;
        if (s->tr_n > 0 && s->tr_count < s->tr_cap) {
            MS_CUDA_TRY(ms::launch_trace(s->sa[s->cur], s->tr_idx, s->tr_n,
                                         s->tr_buf + (size_t)s->tr_count * s->tr_n * 3, s->stream));
            ++s->tr_count;
        }
    }
    s->step_count += nsteps;
    return MS_OK;
}

ms_status ms_get_state(ms_sim *s, float *x, float *v, int32_t on_device)
{
    ms::Range range_("ms_get_state");
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    const int N = s->N;
    if (on_device) {
        MS_CUDA_TRY(ms::launch_gather_state(s->sa[s->cur], s->sb[s->cur], s->d_perm, s->d_cidx, N, x, v, s->stream));
        return MS_OK;
    }
    float *sx = x ? s->stage : nullptr, *sv = v ? s->stage + 3 * (size_t)N : nullptr;
    MS_CUDA_TRY(ms::launch_gather_state(s->sa[s->cur], s->sb[s->cur], s->d_perm, s->d_cidx, N, sx, sv, s->stream));
    if (x) MS_CUDA_TRY(cudaMemcpyAsync(x, sx, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, s->stream));
    if (v) MS_CUDA_TRY(cudaMemcpyAsync(v, sv, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, s->stream));
    return ms_sync(s);
}

ms_status ms_set_state(ms_sim *s, const float *x, const float *v, int32_t on_device)
{
    ms::Range range_("ms_set_state");
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    const int N = s->N;
    if (on_device) {
        MS_CUDA_TRY(ms::launch_scatter_state(s->sa[s->cur], s->sb[s->cur], s->w, s->d_perm, s->d_cidx, N, x, v, s->stream));
        return MS_OK;
    }
    // host input: copy to the staging buffer, check finiteness on the device,
    // and scatter only if every value is finite (the state is untouched otherwise)
    if (x) MS_CUDA_TRY(cudaMemcpyAsync(s->stage, x, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s->stream));
    if (v) MS_CUDA_TRY(cudaMemcpyAsync(s->stage + 3 * (size_t)N, v, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, s->stream));
    MS_CUDA_TRY(ms::launch_checked_scatter_state(s->sa[s->cur], s->sb[s->cur], s->w, s->d_perm, s->d_cidx, N, x ? s->stage : nullptr,
                                                 v ? s->stage + 3 * (size_t)N : nullptr, s->err + 1, s->stream));
    int first_bad = INT_MAX;
    MS_CUDA_TRY(cudaMemcpyAsync(&first_bad, s->err + 1, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (first_bad != INT_MAX) return fail(MS_ERR_ARG, "non-finite state at mass " + std::to_string(first_bad));
    return MS_OK;
}

ms_status ms_sync(ms_sim *s)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    int flag = 0;
    MS_CUDA_TRY(cudaMemcpy(&flag, s->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & ms::kErrTimeout) return fail(MS_ERR_TIMEOUT, "a bounded device-side wait gave up (a bulk copy or a grid barrier never completed)");
    if (flag & ms::kErrNonFinite) return fail(MS_ERR_NONFINITE, "a step produced a non-finite position or velocity");
    return MS_OK;
}

ms_status ms_set_wait_limit(ms_sim *s, int32_t max_polls)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (max_polls < 0) return fail(MS_ERR_ARG, "max_polls must be >= 0");
    s->grid_polls = max_polls == 0 ? ms::kGridPollsDefault : (unsigned)max_polls;
    return MS_OK;
}

ms_status ms_test_barrier_deficit(ms_sim *s, int32_t missing)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (missing < 0 || missing > 1024) return fail(MS_ERR_ARG, "missing must be in [0, 1024]");
    if (missing > 0 && !s->grid_persistent)
        return fail(MS_ERR_ARG, "only the persistent grid kernel has a grid barrier");
    s->grid_missing = (unsigned)missing;
    return MS_OK;
}

ms_status ms_energy(ms_sim *s, double *out, int32_t on_device)
{
    ms::Range range_("ms_energy");
    if (!s || !out) return fail(MS_ERR_ARG, "sim or out is NULL");
    ms::EnergyArgs a{};
    a.sa = s->sa[s->cur]; a.sb = s->sb[s->cur]; a.w = s->w;
    a.slice = s->slice; a.f_nbr = s->f_nbr; a.t_nbr = s->t_nbr;
    a.tiles = s->tiles; a.halo = s->halo; a.f_kl = s->f_kl; a.f_ab = s->actuated ? s->f_ab : nullptr;
    a.N = s->N; a.n_tiles = s->n_tiles; a.tiled = s->kernel == ms::kKernelTiled;
    if (s->actuated) {
        const double t = (double)s->step_count * (double)s->p.dt;
        a.s_n = (float)std::sin(2.0 * M_PI * s->freq * t);
        a.c_n = (float)std::cos(2.0 * M_PI * s->freq * t);
    }
    a.gx = s->p.g[0]; a.gy = s->p.g[1]; a.gz = s->p.g[2]; a.k_c = s->p.k_c; a.contact = s->p.contact_on;
    const ms::LatticeArgs *lat = s->kernel == ms::kKernelLattice ? &s->lat : nullptr;
    if (!s->e_partial) {
        ms_status st = upload<double>(s, &s->e_partial, nullptr, 4 * (size_t)ms::energy_blocks(a, lat) + 4);
        if (st != MS_OK) return st;
    }
    a.partial = s->e_partial;
    double *res = s->e_partial + 4 * (size_t)ms::energy_blocks(a, lat);
    MS_CUDA_TRY(ms::launch_energy(a, lat, on_device ? out : res, s->stream));
    if (on_device) return MS_OK;
    MS_CUDA_TRY(cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return MS_OK;
}

ms_status ms_trace_set(ms_sim *s, const int32_t *masses, int32_t n_masses, int32_t capacity)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (n_masses < 0 || capacity < 0 || (n_masses > 0 && (!masses || capacity < 1)))
        return fail(MS_ERR_ARG, "need n_masses >= 0, and masses and capacity >= 1 when n_masses > 0");
    if (n_masses > 0 && (s->persistent || s->grid_persistent))
        return fail(MS_ERR_ARG, "the persistent kernel records no per-step trace");
    if ((int64_t)n_masses * capacity * 3 >= ((int64_t)1 << 40)) return fail(MS_ERR_ARG, "trace too large");
    std::vector<int32_t> idx(n_masses);
    for (int32_t q = 0; q < n_masses; ++q) {
        if (masses[q] < 0 || masses[q] >= s->N) return fail(MS_ERR_ARG, "trace mass index out of range");
        idx[q] = s->iperm[masses[q]];
    }
    if (s->tr_idx) { s->dev_free(s->tr_idx); s->tr_idx = nullptr; }
    if (s->tr_buf) { s->dev_free(s->tr_buf); s->tr_buf = nullptr; }
    s->tr_n = 0; s->tr_cap = 0; s->tr_count = 0;
    if (n_masses == 0) return MS_OK;
    ms_status st = upload(s, &s->tr_idx, idx.data(), (size_t)n_masses);
    if (st != MS_OK) return st;
    if ((st = upload<float>(s, &s->tr_buf, nullptr, (size_t)n_masses * capacity * 3)) != MS_OK) return st;
    MS_CUDA_TRY(cudaStreamSynchronize(s->stream));      // idx is a host temporary
    s->tr_n = n_masses; s->tr_cap = capacity;
    return MS_OK;
}

ms_status ms_trace_get(ms_sim *s, float *out, int32_t *n_steps, int32_t on_device)
{
    if (!s) return fail(MS_ERR_ARG, "sim is NULL");
    if (n_steps) *n_steps = s->tr_count;
    if (!out || s->tr_count == 0) return MS_OK;
    const size_t bytes = sizeof(float) * 3 * (size_t)s->tr_n * s->tr_count;
    MS_CUDA_TRY(cudaMemcpyAsync(out, s->tr_buf, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                s->stream));
    if (!on_device) MS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return MS_OK;
}

ms_status ms_get_info(const ms_sim *s, ms_info_t *out)
{
    if (!s || !out) return fail(MS_ERR_ARG, "sim or out is NULL");
    out->n_masses = s->N; out->n_springs = s->S; out->n_records = s->n_records;
    out->n_slots = s->n_slots; out->n_back_slots = s->n_back_slots; out->device_bytes = s->device_bytes;
    out->step_count = s->step_count; out->stability_bound = s->stability;
    out->max_fwd_degree = s->max_fwd; out->max_back_degree = s->max_back;
    out->kernel = (s->persistent || s->grid_persistent) ? ms::kKernelPersistent : s->kernel;
    out->n_tiles = s->n_tiles; out->max_tile_local = s->max_tile_local;
    out->lattice_guard = s->kernel == ms::kKernelLattice ? s->lat.guard : 0;
    return MS_OK;
}

ms_status ms_destroy(ms_sim *s)
{
    if (!s) return MS_OK;
    s->release();
    delete s;
    return MS_OK;
}

}  // extern "C"
