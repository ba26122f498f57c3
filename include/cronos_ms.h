/*
 * cronos_ms.h -- C ABI of the GB300 mass-spring step library.
 *
 * The library advances a nonlinear Hookean mass-spring system with an
 * explicit scheme on one GPU (sm_103a).  It implements the method of the
 * Cronos paper (arXiv 2207.09334), section "Method":
 *   eq. 1-3  m_i a_i = f_i,  f_i = m_i g + f_ext_i + sum_j k_ij (|l_ij| - L_ij) l_ij/|l_ij|,
 *            l_ij = x_j - x_i, d/dt [x; v] = [v; f/m];
 *   eq. 4    the explicit time step (read as symplectic Euler: v' = v + dt f/m,
 *            x' = x + dt v', all forces taken at t_n);
 *   Algorithm 1 ("Parallel Simulation Process"): spring forces, a grid-wide
 *            synchronisation, then a per-mass sum and integration.  Here the
 *            sum is a deterministic per-mass gather (no atomics of any kind).
 * together with the features the paper names around it: axial spring
 * damping, actuated ("volumetric") rest lengths, anchored masses, and
 * ground contact planes with friction (Appendix A).
 *
 * Conventions for every entry point:
 *   - Errors are status codes; nothing aborts or throws across the ABI.
 *     ms_last_error() gives a message for the calling thread's last failure.
 *   - All arrays are caller-owned and copied (inputs) or filled (outputs);
 *     the library never keeps a caller pointer.
 *   - Masses and springs are addressed in the caller's index order.  Any
 *     internal reordering is invisible at the ABI.
 *   - Work is enqueued on the CUDA stream given at creation (NULL = legacy
 *     default stream).  ms_step is asynchronous; errors detected on the
 *     device (non-finite state) are reported by the next synchronising call
 *     (ms_sync, ms_get_state to host).
 *   - Vectors are float32 triples, row-major (N,3).
 */
#ifndef CRONOS_MS_H
#define CRONOS_MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MS_OK = 0,
    MS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size or index, non-finite input) */
    MS_ERR_OOM = 2,        /* device or host allocation failed */
    MS_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    MS_ERR_UNSTABLE = 4,   /* strict_stability set and the step-size bound is violated */
    MS_ERR_NONFINITE = 5,  /* the device saw a non-finite position or velocity */
    MS_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
    MS_ERR_STATE = 7       /* call not valid in the object's current state */
} ms_status;

/* Integration and environment parameters (paper: eq. 2-4; Appendix A for
 * contact planes).  Ground plane is z = 0 with normal +z. */
typedef struct {
    float dt;               /* time step [s] */
    float g[3];             /* gravity [m/s^2] */
    float k_c;              /* ground penalty stiffness [N/m]: Fn = k_c max(0, -z), active when z < 0 */
    float mu;               /* Coulomb friction coefficient on the ground (impulse clamp on tangential v) */
    float vel_damping;      /* global damping d: v' *= (1 - d) every step (0 = off) */
    int32_t contact_on;     /* 1 = ground contact active */
    int32_t integrator;     /* 0 = symplectic Euler (default); 1 = forward Euler (eq. 4); 2 = position
                               Verlet (eq. 5-6; no friction, no global damping; the dashpots see
                               v_n = (x_n - x_{n-1})/dt); 3 = classical RK4 (eq. 7-8 with the step
                               size in every stage; no friction, no global damping; four force
                               evaluations per step, stage q at t_n + c_q dt, c = 0, 1/2, 1/2, 1;
                               3 x 32 B per mass of extra device memory).  ms_create only;
                               populations and the adjoint take 0. */
    int32_t strict_stability; /* 1 = ms_create fails with MS_ERR_UNSTABLE if the bound below exceeds 4 */
    int32_t reorder;        /* mass order: 0 = library default (Morton for the tiled kernel, caller
                               order for the gather kernel), 1 = Morton order by initial position,
                               2 = caller order */
    int32_t kernel;         /* 0 = library default: lattice (4) for a box lattice of at least 2^18
                               masses, else tiled (gather when a tile's partners do not fit shared
                               memory); 1 = gather, 2 = tiled (MS_ERR_ARG if a tile does not fit),
                               3 = persistent: all steps of one ms_step call in one launch.  Up to
                               8192 masses: a thread-block cluster (at most 16 CTAs, one per tile
                               of 64 to 512 masses) with the state and the spring records in
                               shared memory, partners in other CTAs read through distributed
                               shared memory.  Above: the tiled layout in one cooperative launch
                               (one CTA per 512-mass tile, at most one per multiprocessor), each
                               tile's records in shared memory, a grid barrier per step.
                               MS_ERR_ARG when the system has more tiles than multiprocessors,
                               when the records do not fit shared memory, or with an integrator
                               other than symplectic Euler; ms_set_actuation returns MS_ERR_ARG
                               when the actuation coefficients do not fit as well.
                               4 = lattice: masses on the points of a cubic grid (spacing = the
                               shortest spring), springs only between grid neighbours of the
                               26-neighbourhood and at most one per pair, one rest length per
                               lattice direction, one dashpot value; topology and rest lengths
                               then come from the grid and only k is stored per spring (the
                               paper's cubic and voxel lattices, "Generating a Lattice"), plus
                               each spring's actuation coefficients once ms_set_actuation is
                               called (8 bytes per spring more).
                               MS_ERR_ARG (with the reason) for any other network */
} ms_params;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc must return device memory aligned to at least 256 bytes usable on
 * `stream`, or NULL on failure; free receives the same pointer and size. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} ms_allocator;

typedef struct ms_sim ms_sim;   /* opaque; owns all of its device memory */

typedef struct {
    int64_t n_masses;          /* N */
    int64_t n_springs;         /* caller springs S */
    int64_t n_records;         /* springs after merging parallel springs (same pair) */
    int64_t n_slots;           /* padded forward record slots (>= n_records); lattice: 13 x padded cells */
    int64_t n_back_slots;      /* padded back-reference slots */
    int64_t device_bytes;      /* device memory held */
    int64_t step_count;        /* steps taken since creation */
    double stability_bound;    /* dt^2 * max_i (2 sum_{springs at i} k + k_c) / m_i  (Gershgorin; stable if < 4) */
    int32_t max_fwd_degree;    /* gather: most springs owned by one mass; tiled: most springs of one mass */
    int32_t max_back_degree;
    int32_t kernel;            /* 1 = gather, 2 = tiled, 3 = persistent, 4 = lattice */
    int32_t n_tiles;           /* tiled: tiles; lattice: bricks of 16 x 16 x 8 cells */
    int32_t max_tile_local;    /* tiled: largest members + halo of a tile; lattice: cells staged per brick */
    int32_t lattice_guard;     /* lattice: 1 when some neighbouring masses have no spring between them
                                  (the kernel then tests every spring term), else 0 */
} ms_info_t;

/*
 * ms_create -- build a simulation object from a general spring network
 * (paper: "Generating a Lattice" final paragraph -- masses from nodes,
 * springs from edges, copied to GPU memory; "GPU Implementation" -- each
 * mass needs the list of springs attached to it).
 *
 *   p        parameters (copied).
 *   N        number of masses, 1 <= N < 2^27.
 *   x0, v0   (N,3) initial positions [m] and velocities [m/s].
 *   mass     (N) masses [kg], > 0 and finite for masses that are not anchored.
 *   fixed    (N) 1 = anchored: position frozen, velocity held at 0, still
 *            exerts spring forces (NULL = none anchored).
 *   fext     (N,3) constant external force [N] (NULL = none).
 *   S        number of springs, >= 0.
 *   ij       (S,2) endpoint indices in [0, N), i != j.
 *   k        (S) stiffness [N/m] >= 0.
 *   c        (S) axial dashpot coefficient [N s/m] >= 0, or NULL to use
 *            c_uniform for every spring.
 *   rest_len (S) rest length [m] >= 0, or NULL = initial distance.
 *   alloc    device allocator, or NULL for cudaMalloc/cudaFree.
 *   stream   cudaStream_t to enqueue all work on (NULL = default stream).
 *   out      receives the new object.
 * Parallel springs (same unordered pair) are merged into one record with
 * summed stiffness and damping and the stiffness-weighted rest length; the
 * merge is exact in real arithmetic because the force is linear in k and in
 * k*L.  A mass may own at most 31 distinct higher-indexed partners after
 * reordering (26 in a lattice).  Returns MS_ERR_ARG on invalid input,
 * MS_ERR_OOM / MS_ERR_CUDA on allocation or copy failure, MS_ERR_UNSTABLE
 * as described for strict_stability.  On failure *out is set to NULL.
 */
ms_status ms_create(const ms_params *p, int32_t N, const float *x0, const float *v0,
                    const float *mass, const uint8_t *fixed, const float *fext,
                    int64_t S, const int32_t *ij, const float *k, const float *c,
                    float c_uniform, const float *rest_len, const ms_allocator *alloc,
                    void *stream, ms_sim **out);

/*
 * ms_create_materials -- ms_create with springs described by material
 * (paper: "Generating a Lattice" final paragraph -- physical material
 * properties derive the spring constants and mass values; Fig. 2 -- robots
 * built from soft, stiff and actuated materials).  Every argument not listed
 * here is as for ms_create.
 *   mat          (S) material id of each spring, in [0, n_mat).
 *   n_mat        entries of the tables, 1 <= n_mat <= 65536.
 *   mat_k        (n_mat) stiffness [N/m] >= 0.
 *   mat_c        (n_mat) axial dashpot [N s/m] >= 0, or NULL = 0.
 *   mat_L0scale  (n_mat) rest-length factor >= 0, or NULL = 1: spring s rests
 *                at base_s * mat_L0scale[mat[s]] (one FP32 rounding), base_s =
 *                rest_len[s], or the initial distance when rest_len is NULL
 *                (computed as ms_create computes it).
 * The tables are expanded on the host into ms_create's per-spring arrays, so
 * the object equals, bit for bit, one made by ms_create from those arrays.
 * Errors: MS_ERR_ARG for an id out of range or a bad table entry, otherwise
 * those of ms_create.
 */
ms_status ms_create_materials(const ms_params *p, int32_t N, const float *x0, const float *v0,
                              const float *mass, const uint8_t *fixed, const float *fext,
                              int64_t S, const int32_t *ij, const uint16_t *mat, int32_t n_mat,
                              const float *mat_k, const float *mat_c, const float *mat_L0scale,
                              const float *rest_len, const ms_allocator *alloc, void *stream,
                              ms_sim **out);

/*
 * ms_set_actuation -- actuated rest lengths (paper: Introduction and
 * Applications -- self-actuation by dynamically modifying volumetric
 * properties; Fig. 2 caption -- springs individually actuated).  Spring s
 * then has rest length L0_s (1 + amp_s sin(2 pi freq t_n + phase_s)) at the
 * start-of-step time t_n = n dt.  amp and phase are (S) arrays in caller
 * spring order; amp = NULL switches actuation off.  Merged parallel springs
 * combine exactly: sum_s k_s L_s(t) = K L0eff (1 + alpha sin(w t) + beta cos(w t)).
 * The sine and cosine of 2 pi freq t_n are evaluated in FP64 on the host.
 */
ms_status ms_set_actuation(ms_sim *sim, float freq_hz, const float *amp, const float *phase);

/*
 * ms_step -- advance nsteps explicit steps (eq. 2-4, Algorithm 1), each
 * reading the state at t_n and writing the state at t_{n+1} (double
 * buffered).  Asynchronous on the object's stream.  nsteps >= 0.
 */
ms_status ms_step(ms_sim *sim, int32_t nsteps);

/*
 * ms_get_state / ms_set_state -- copy positions and velocities ((N,3) float32,
 * caller order) out of / into the object (paper: "GPU Implementation" --
 * syncing the state from GPU to CPU and back; a saved state restores a run,
 * i.e. checkpoint and resume).  on_device = 1: x and v are device
 * pointers (stream-ordered, asynchronous); 0: host pointers (the call
 * synchronises the stream; page-locked memory gives the fastest copies).
 * Either pointer may be NULL to skip it.  ms_get_state to host also reports
 * MS_ERR_NONFINITE if the device flagged a non-finite value.  ms_set_state
 * keeps anchored masses' velocity at 0; with host input it checks every
 * value on the device and returns MS_ERR_ARG (naming the first caller mass
 * with a non-finite value) without modifying the state.
 */
ms_status ms_get_state(ms_sim *sim, float *x, float *v, int32_t on_device);
ms_status ms_set_state(ms_sim *sim, const float *x, const float *v, int32_t on_device);

/* ms_sync -- wait for the object's stream (paper: "GPU Implementation" --
 * the host waits for the device before it reads results back); returns
 * MS_ERR_TIMEOUT if a bounded device-side wait gave up, MS_ERR_NONFINITE if a
 * step produced a non-finite value since creation (both sticky), else MS_OK. */
ms_status ms_sync(ms_sim *sim);

/*
 * ms_set_wait_limit -- polls of each bounded device-side wait of the
 * persistent grid kernel (its grid barrier, Algorithm 1's synchronisation
 * between steps) before the waiting CTA gives up, leaves its step loop and
 * flags MS_ERR_TIMEOUT for the next synchronising call.  0 restores the
 * default, 2^22 polls with a short sleep each (well over a second).  A limit
 * shorter than one step's work reports timeouts on a healthy run; the state
 * is then only partly advanced.
 *
 * ms_test_barrier_deficit -- failure-detection test hook with no counterpart
 * in the paper: the grid barrier of later ms_step calls waits for `missing`
 * arrivals beyond the CTAs that exist (0 = off, at most 1024), so no wait can
 * complete and every CTA gives up after the wait limit.  Only a sim stepped
 * by the persistent grid kernel accepts missing > 0 (MS_ERR_ARG otherwise).
 * Nothing faults or hangs: every wait is bounded and no copy is in flight.
 */
ms_status ms_set_wait_limit(ms_sim *sim, int32_t max_polls);
ms_status ms_test_barrier_deficit(ms_sim *sim, int32_t missing);

/*
 * ms_energy -- energy of the current state at t_n = step_count dt, reduced on
 * the device (paper: Energy Conservation Tests; eq. 2's Hooke term):
 *   out[0] kinetic        sum_i m_i |v_i|^2 / 2
 *   out[1] elastic        sum_s k_s (l_s - L_s(t_n))^2 / 2, L_s actuated as in ms_set_actuation
 *   out[2] gravitational  -sum_i m_i g . x_i           (anchored masses included)
 *   out[3] ground         sum_i k_c z_i^2 / 2 over z_i < 0, when contact is on
 * out: 4 doubles; on_device = 1: a device pointer (8-byte aligned), the call
 * is asynchronous on the object's stream and copies nothing to the host, so
 * a run can record the energy every few steps; 0: host pointer, the call
 * synchronises.  The reduction order is fixed: the result is bit-identical
 * between calls on the same state.  FP32 terms, FP32 warp sums, FP64 sums
 * above.  Parallel springs merged into one record contribute that record's
 * energy, which differs from the sum over the separate springs by
 * sum_v k_v (L_v - L)^2 / 2 (L the merged rest length), a term independent
 * of the positions.  The first call allocates a small reduction buffer
 * (4 doubles per 512 masses).
 */
ms_status ms_energy(ms_sim *sim, double *out, int32_t on_device);

/*
 * ms_trace_set -- record the positions of n_masses chosen masses (caller
 * indices) after every subsequent step, for at most `capacity` steps, into a
 * device buffer of the object (e.g. a cantilever tip; paper: cantilever
 * experiments).  Replaces any previous trace and restarts the count; n_masses
 * = 0 switches tracing off and frees the buffer.  Steps beyond capacity are
 * not recorded.  Not available with the persistent kernel (MS_ERR_ARG).
 * Each recorded step adds one small kernel launch.
 * ms_trace_get -- *n_steps (if not NULL) receives the number of recorded
 * steps; out (if not NULL) receives n_steps x n_masses x 3 floats, step-major,
 * masses in the order given to ms_trace_set.  on_device as for ms_get_state.
 */
ms_status ms_trace_set(ms_sim *sim, const int32_t *masses, int32_t n_masses, int32_t capacity);
ms_status ms_trace_get(ms_sim *sim, float *out, int32_t *n_steps, int32_t on_device);

/* ms_get_info -- sizes and diagnostics of the object's device layout
 * (paper: "GPU Implementation" -- springs and masses stored consecutively,
 * with the springs attached to each mass stored on the mass). */
ms_status ms_get_info(const ms_sim *sim, ms_info_t *out);

/* ms_destroy -- free all memory held by the object (after its stream's work);
 * the end of the lifetime that ms_create starts (paper: "Generating a
 * Lattice" -- the lattice is copied to GPU memory to initialise a run).
 * NULL is a no-op. */
ms_status ms_destroy(ms_sim *sim);

/* Message of the calling thread's last error (static storage, never NULL).
 * ABI plumbing; the paper has no counterpart. */
const char *ms_last_error(void);

/* Library version string (ABI plumbing; the paper has no counterpart). */
const char *ms_version(void);


/* ------------------------------------------------------------------------
 * Batched voxel-robot populations.
 *
 * Many independent voxel robots (each with its own ground plane, no contact
 * between robots) advanced together by ONE persistent kernel launch that is
 * captured in a CUDA graph.  Each robot is built as in the paper's voxel
 * lattice ("Generating a Lattice", Fig. figure1): the corners of its
 * non-empty voxels are masses, and every voxel links all 28 pairs of its 8
 * corners (12 edges, 12 face diagonals, 4 long diagonals); springs that
 * neighbouring voxels share are merged exactly (summed k and c, combined
 * actuation).  Materials set k, c and the actuation amplitude; actuated
 * springs have rest length L0 (1 + amp sin(2 pi freq t_n + phase_voxel)).
 * Masses of a robot are numbered in raster order (x fastest) of its
 * (nx+1)(ny+1)(nz+1) corner grid, keeping only corners of non-empty voxels;
 * corner (cx, cy, cz) starts at (cx a, cy a, cz a), so the robot rests on
 * z = 0, at rest.  Each corner weighs voxel_mass / 8 per non-empty voxel it
 * touches.  A robot may have at most 4096 masses.
 * ---------------------------------------------------------------------- */
typedef struct msb_batch msb_batch;

typedef struct {
    float voxel_edge;        /* voxel edge length a [m] */
    float voxel_mass;        /* mass of one voxel [kg] */
    float freq;              /* actuation frequency [Hz] */
    int32_t n_materials;     /* entries in the tables below; id 0 is always "empty" */
    const float *mat_k;      /* stiffness of each of a voxel's 28 springs [N/m] */
    const float *mat_c;      /* axial dashpot of each spring [N s/m] */
    const float *mat_amp;    /* actuation amplitude (0 = passive) */
} msb_voxel_spec;

typedef struct {
    int32_t n_robots;
    int64_t n_masses;        /* over all robots */
    int64_t n_records;       /* merged springs over all robots */
    int32_t max_robot_masses;
    int32_t n_block_items;   /* robots run block-per-robot by the current schedule */
    int32_t n_warp_items;    /* robots run warp-per-robot */
    int64_t device_bytes;
    int64_t step_count;
    int32_t threads;         /* CTA size of the persistent kernel: 512 or 1024 */
} msb_info_t;

/*
 * msb_create -- build a population.
 *   p          environment and step parameters (contact, friction, dt, g).
 *   spec       voxel material table and geometry.
 *   n_robots   >= 1.
 *   dims       [n_robots][3] = (nx, ny, nz) voxels, each >= 1.
 *   materials  concatenated grids, robot r has nz*ny*nx ids, index
 *              ix + nx*(iy + ny*iz); ids in [0, n_materials).
 *   phase      same layout, actuation phase per voxel [rad] (NULL = 0).
 *   logk       same layout or NULL: per-voxel log-stiffness; when given,
 *              every spring of voxel v uses k = exp(logk[v]) instead of its
 *              material's k (empty voxels stay empty).
 * Robots with no non-empty voxel are rejected (MS_ERR_ARG).
 */
ms_status msb_create(const ms_params *p, const msb_voxel_spec *spec, int32_t n_robots,
                     const int32_t *dims, const uint8_t *materials, const float *phase,
                     const float *logk, const ms_allocator *alloc, void *stream, msb_batch **out);

/*
 * msb_autotune -- for each CTA size of the persistent kernel (512 and 1024
 * threads): start from the default schedules, flip one robot-size bucket at
 * a time ((0,32], (32,64], (64,128], (128,256] masses) between
 * warp-per-robot and block-per-robot, and keep a flip when the whole
 * population, run for sample_steps steps from the same state, gets faster;
 * then keep the faster CTA size.  The robots' state is restored afterwards.
 * Without it, the CTA has 512 threads, robots of up to 64 masses run
 * warp-per-robot and the rest block-per-robot.  Synchronises the stream.
 * policy: 0 = autotune, 1 = force block-per-robot, 2 = force warp-per-robot
 * wherever a robot fits a warp's share of shared memory (policies 1 and 2
 * keep the current CTA size).
 */
ms_status msb_autotune(msb_batch *b, int32_t sample_steps, int32_t policy);

/* msb_set_threads -- CTA size of the persistent kernel, 512 or 1024 (else
 * MS_ERR_ARG); a warp item then holds threads / 32 robots, and a robot whose
 * warp share no longer fits shared memory runs block-per-robot. */
ms_status msb_set_threads(msb_batch *b, int32_t threads);

/*
 * msb_run -- advance every robot nsteps steps in one persistent launch
 * (replayed from a CUDA graph after the first call with the same nsteps).
 * Asynchronous on the batch's stream.
 */
ms_status msb_run(msb_batch *b, int32_t nsteps);

/*
 * msb_run_loop -- the same nsteps advanced robot by robot: one kernel launch
 * per robot per step (the plain per-robot loop the batched launch replaces;
 * kept for comparison).
 */
ms_status msb_run_loop(msb_batch *b, int32_t nsteps);

/* msb_com_travel -- per robot, x-travel of the mass-weighted centre of mass
 * since creation or the last msb_reset ([n_robots] floats; on_device: out is
 * device memory, stream-ordered; else host, synchronising). */
ms_status msb_com_travel(msb_batch *b, float *out, int32_t on_device);

/* msb_robot_info -- number of masses of robot r and its first index in the
 * population-wide mass numbering. */
ms_status msb_robot_info(const msb_batch *b, int32_t robot, int32_t *n_masses, int64_t *first_mass);

/* msb_get_state -- positions and velocities of all masses, robots in order,
 * each robot in its own corner order ((n_masses,3) float32 host arrays;
 * either may be NULL).  Synchronises. */
ms_status msb_get_state(msb_batch *b, float *x, float *v);

/* msb_reset -- restore the initial state and time t = 0. */
ms_status msb_reset(msb_batch *b);

ms_status msb_get_info(const msb_batch *b, msb_info_t *out);
ms_status msb_destroy(msb_batch *b);

/* ------------------------------------------------------------------------
 * Adjoint of voxel-robot rollouts (reverse-mode gradients).
 *
 * The paper notes that differentiability is enabled by the method (Related
 * Work, on ChainQueen).  This is a hand-written reverse pass of the
 * explicit step above (symplectic Euler, ground penalty contact and the
 * Coulomb clamp -- differentiated along the branch the forward pass took --
 * the axial dashpot and the Hooke term with actuated rest length).  The
 * forward pass keeps a checkpoint of the state every `checkpoint_every`
 * steps; the reverse pass recomputes each segment from its checkpoint and
 * walks it backwards.  One CTA per robot; gradients are summed per voxel in
 * a fixed order (deterministic).
 * ---------------------------------------------------------------------- */
typedef struct msa_adjoint msa_adjoint;

/*
 * msa_create -- build the adjoint for a population (same voxel layout and
 * mass numbering as msb_create).  Reserves checkpoint and segment memory for
 * rollouts of up to max_steps steps.  checkpoint_every >= 1.  A robot may
 * have at most 1024 masses and 4096 voxels here.
 */
ms_status msa_create(const ms_params *p, const msb_voxel_spec *spec, int32_t n_robots, const int32_t *dims,
                     const uint8_t *materials, int32_t checkpoint_every, int32_t max_steps,
                     const ms_allocator *alloc, void *stream, msa_adjoint **out);

/*
 * msa_gradients -- run nsteps (<= max_steps) steps from rest and return, per
 * robot r, a scalar loss and its gradient with respect to every voxel's
 * actuation phase and log-stiffness.
 *   phase, logk  [total voxels] parameters (layout of msb_create's grids);
 *                voxel v's 28 springs use k = exp(logk[v]) and rest length
 *                L0 (1 + amp sin(2 pi freq t_n + phase[v])).
 *   seed_x       NULL: loss_r = centre-of-mass x-travel of robot r after
 *                nsteps; else [n_masses][3] weights w and loss_r = sum over
 *                robot r's masses of w_i . x_i(t_end).
 *   loss         [n_robots] out; g_phase, g_logk [total voxels] out (0 for
 *                empty voxels).
 *   on_device    1: every array argument is device memory (stream-ordered);
 *                0: host memory (synchronising).
 */
ms_status msa_gradients(msa_adjoint *a, int32_t nsteps, const float *phase, const float *logk,
                        const float *seed_x, float *loss, float *g_phase, float *g_logk, int32_t on_device);

/* msa_set_threads / msa_threads -- threads per robot of the adjoint kernel
 * (one CTA per robot): 256, 512, 768 or 1024.  msa_create picks the size
 * whose estimated time, waves x ceil(largest robot's masses / threads), is
 * smallest for the population on this GPU; msa_set_threads overrides it
 * (MS_ERR_ARG for another value).  Results agree up to FP32 rounding of the
 * loss's block sum; msa_threads returns the current size (0 for NULL). */
ms_status msa_set_threads(msa_adjoint *a, int32_t threads);
int32_t msa_threads(const msa_adjoint *a);

/* msa_sizes -- total voxels and masses of the population. */
ms_status msa_sizes(const msa_adjoint *a, int64_t *n_voxels, int64_t *n_masses);

ms_status msa_destroy(msa_adjoint *a);

/* ------------------------------------------------------------------------
 * Design surrogate: an MLP n_in -> n_hidden -> n_hidden -> 1 with GELU,
 * bf16 weights and activations, fp32 accumulation on the tensor cores
 * (tcgen05 + TMEM, operands staged by TMA).  It predicts a voxel design's
 * locomotion distance from its one-hot materials so that large candidate
 * populations can be pre-screened before the simulator (above) scores the
 * best.  The paper has no learned component; this serves the optimisation
 * loop the paper motivates (Introduction: simulation for design and
 * optimisation of soft robots).
 *
 * Parameters are one fp32 vector: W1 [n_hidden][n_in], b1 [n_hidden],
 * W2 [n_hidden][n_hidden], b2 [n_hidden], w3 [n_hidden], b3 [1]
 * (mlp_num_params entries).  Batches are multiples of 128 up to max_batch.
 * Loss: 0.5 mean (y - target)^2.  All device-pointer arguments are
 * stream-ordered on the model's stream.
 * ---------------------------------------------------------------------- */
typedef struct mlp_model mlp_model;

/* n_in and n_hidden multiples of 128; weights uniform(+-1/sqrt(fan_in)) from seed, biases 0. */
ms_status mlp_create(int32_t n_in, int32_t n_hidden, int32_t max_batch, uint64_t seed,
                     const ms_allocator *alloc, void *stream, mlp_model **out);
int64_t mlp_num_params(const mlp_model *m);
/* host fp32 parameter vector in / out (grads: last computed gradient, may be NULL) */
ms_status mlp_set_params(mlp_model *m, const float *params);
ms_status mlp_get_params(mlp_model *m, float *params, float *grads);
/* load a batch: device materials [B][n_in/4] (ids 0..3) to be one-hot encoded (the model keeps a
 * copy; an inference pass builds the one-hot tiles of X in shared memory inside the first GEMM,
 * a training pass writes X), or bf16 inputs [B][n_in] (copied) */
ms_status mlp_encode(mlp_model *m, const uint8_t *materials, int32_t B);
ms_status mlp_set_input(mlp_model *m, const uint16_t *x_bf16, int32_t B);
/* predictions of the loaded batch into device y [B] (may be NULL); inference only: the
 * pre-activations and transposed activations that training needs are not stored
 * (mlp_backward runs its own forward pass) */
ms_status mlp_forward(mlp_model *m, int32_t B, float *y);
/* inference on device materials [B][n_in/4] (ids 0..3, 16-byte aligned) read in place by
 * the first GEMM, without the copy mlp_encode makes (the caller keeps them unchanged until
 * the pass has run on the model's stream); predictions into device y [B] (may be NULL).
 * The loaded batch (mlp_encode / mlp_set_input) is left as it was. */
ms_status mlp_forward_materials(mlp_model *m, const uint8_t *materials, int32_t B, float *y);
/* forward + backward of the loaded batch against device target [B]; gradients kept in the model;
 * device loss [1] (may be NULL) */
ms_status mlp_backward(mlp_model *m, const float *target, int32_t B, float *loss);
/* one Adam step (bias-corrected) with the last gradients */
ms_status mlp_adam(mlp_model *m, float lr, float beta1, float beta2, float eps);
/* wait for the model's stream; MS_ERR_TIMEOUT if a bounded tensor-core wait gave up */
ms_status mlp_sync(mlp_model *m);
ms_status mlp_destroy(mlp_model *m);

/* C[M][N] (fp32, device) = A[M][K] . B[N][K]^T with bf16 device inputs on the
 * tensor cores; M, N multiples of 128, K a multiple of 64.  Synchronises. */
ms_status mlp_gemm_bf16(const uint16_t *A, const uint16_t *B, float *C, int32_t M, int32_t N, int32_t K,
                        void *stream);

/* ------------------------------------------------------------------------
 * Stepping without allocating.
 *
 * The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory when they advance a system: plugins
 * inside a host application that owns every device allocation and hands the
 * plugin only the buffers it needs, and real-time loops whose latency budget
 * forbids allocator calls (which may synchronise the device or take a lock).
 * The caller owns every input and output; the only working memory is a
 * fixed array that the library declares in its own device memory, so every
 * GPU that loads the library holds it (16 MiB) until the process exits.
 * ---------------------------------------------------------------------- */
#define MS_NOALLOC_MAX_MASSES 262144

/*
 * ms_step_csr_noalloc -- advance nsteps explicit steps (the same physics as
 * ms_step: Hooke term with axial dashpot, gravity, ground contact and the
 * friction clamp, symplectic Euler, global damping; no actuation, no
 * external force) of a system given directly as device arrays, calling no
 * allocator of any kind.
 *   N            masses, 1 <= N <= MS_NOALLOC_MAX_MASSES (larger N: MS_ERR_ARG).
 *   x_in, v_in   (N,3) device, state at t_0 (read only).
 *   mass         (N) device masses; fixed (N) device 1 = anchored, or NULL.
 *   row_ptr      (N+1) device CSR offsets; the springs of mass i are entries
 *                row_ptr[i] .. row_ptr[i+1]-1 of partner / k / c / rest_len
 *                (device, one entry per spring end: every spring is listed
 *                in the rows of both of its masses, with equal k, c, L0).
 *   x_out, v_out (N,3) device, state after nsteps; must not alias the inputs.
 *   stream       cudaStream_t (NULL = legacy default stream); asynchronous.
 * The intermediate states of a multi-step call live in the library's fixed
 * scratch array, which every call shares and which keeps the last call's
 * contents (each call writes a buffer in full before reading it): calls whose
 * work overlaps on the GPU (on different streams, or from different threads)
 * race on it and must be serialised by the caller.  The first call in a CUDA
 * context (per device, and again after a device reset creates a new
 * context) looks up the array's device address with that device current and
 * caches it; make that first call before any stream capture begins.
 * Preconditions that are NOT checked (the arrays are device memory and are
 * not copied to the host): mass > 0 for masses that are not anchored,
 * 0 <= partner < N, row_ptr non-decreasing with row_ptr[0] = 0 and row_ptr[N]
 * the number of entries, every entry's k, c, rest_len finite.  Non-finite
 * results are not flagged by this entry point.
 */
ms_status ms_step_csr_noalloc(const ms_params *p, int32_t N, const float *x_in, const float *v_in,
                              const float *mass, const uint8_t *fixed, const int32_t *row_ptr,
                              const int32_t *partner, const float *k, const float *c,
                              const float *rest_len, int32_t nsteps, float *x_out, float *v_out,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CRONOS_MS_H */
