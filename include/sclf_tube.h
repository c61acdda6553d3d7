/*
 * sclf_tube.h -- C ABI of the GB300 (sm_103a) library for the 1D
 * particle-in-cell tube of Barzilay, "Full simulation of the open field
 * lines above pulsar's polar cap - Part I" (arXiv:1011.6330).
 *
 * One tube is a conducting cylinder of radius R above the polar cap (Sec. 2).
 * Each step (Sec. 2, Figure A) injects electrons at the base while the
 * Goldreich-Julian charge there is not compensated, weights E_z to every
 * particle (cloud-in-cell), pushes it with Eq. 1, deposits a
 * charge-conserving current and advances Eq. 3 (Maxwell with d/dr -> 1/R)
 * by leap-frog, against the flat (Eq. 5) or frame-dragging (Eq. 6-7)
 * rho_GJ(z). Fields start from Eq. 4 with an empty tube.
 *
 * Units (Sec. 3): c = 1, lengths in R, time in R/c, electron q/m = -1,
 * density in units where omega_p^2 = 4 pi |rho|, i.e. |rho_GJ| =
 * Lambda^2 / 4 pi with Lambda = omega_p R / c.
 *
 * Conventions for every call:
 *   - Return 0 (SCLF_OK) on success or a negative SCLF_E* code; no C++
 *     exception crosses the ABI. tube_strerror() names a code.
 *   - Pointers documented "host" are caller-owned host memory (pageable or
 *     pinned); the library never keeps them after the call returns.
 *   - Device memory is owned by the tube: either a caller-provided device
 *     workspace (tube_create with dev_workspace != NULL; the caller keeps it
 *     alive until tube_destroy) or memory the library allocates itself.
 *   - Work is queued on the CUDA stream given to tube_create and is
 *     asynchronous unless the call says it synchronises. Calls on one tube
 *     must not run concurrently from several host threads.
 */
#ifndef SCLF_TUBE_H
#define SCLF_TUBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define SCLF_OK          0
#define SCLF_EINVAL     -1   /* a parameter or argument is out of range      */
#define SCLF_ENOMEM     -2   /* device or host allocation failed, or the
                                caller's workspace is too small               */
#define SCLF_ECUDA      -3   /* a CUDA runtime call failed                    */
#define SCLF_ECAPACITY  -4   /* particle slots exhausted (injection clipped)  */
#define SCLF_ENONFINITE -5   /* a particle produced NaN/Inf and was dropped   */
#define SCLF_ETIMEOUT   -6   /* a bounded device-side wait gave up            */
#define SCLF_ESTATE     -7   /* call not valid in the tube's current state    */
#define SCLF_EBOUNDS    -8   /* an index failed its bounds check (set only by
                                the bounds-checked build of the library)      */

/* ---- sticky device status flags (tube_stats.flags) ---------------------- */
#define SCLF_FLAG_CAPACITY  0x1u
#define SCLF_FLAG_NONFINITE 0x2u
#define SCLF_FLAG_TIMEOUT   0x4u
#define SCLF_FLAG_BOUNDS    0x8u   /* bounds-checked build only: a particle
                                      kernel met an index outside its array
                                      and skipped the access                */

/* ---- enumerations -------------------------------------------------------- */
#define SCLF_RHO_FLAT 0      /* Eq. 5 with the (R_* / r)^3 factor dropped       */
#define SCLF_RHO_GR   1      /* Eq. 6 with omega from Eq. 7, f = H = alpha = 1 */
#define SCLF_RHO_USER 2      /* caller-supplied rho_GJ at the Nz+1 nodes      */

/* Frame-dragging variants of Eq. 6 (tube_params.gr_variant) */
#define SCLF_GR_COS  0       /* Omega -> Omega - omega on the cos i term only    */
#define SCLF_GR_BOTH 1       /* Omega -> Omega - omega on Eq. 6's prefactor, i.e.
                                (1 - kappa/eta^3) on both terms                 */

#define SCLF_FP32 0          /* particle arithmetic in IEEE float32           */
#define SCLF_FP64 1          /* particle arithmetic in IEEE float64           */
#define SCLF_FIX32 2         /* int32 fixed-point positions X = xi 2^fb with
                                fb = 31 - ceil(log2 Nz) (uniform resolution
                                along the tube), float32 momenta and push, the
                                displacement rounded half-even to 2^-fb cell;
                                requires SCLF_ACC_FIXED64 and Nz >= 16         */

#define SCLF_ACC_FIXED64 0   /* current fractions summed exactly in int64
                                multiples of 2^-32 (order independent)        */
#define SCLF_ACC_FP64    1   /* current fractions summed with FP64 atomics    */

typedef struct sclf_tube* tube_t;   /* opaque, library-owned */

/*
 * Parameters of one tube, as the paper states them (Sec. 3: B, P, R_*, i,
 * M; Sec. 2: R, the rho_GJ profile; plus the grid Nz and the step dt).
 * tube_params_default() fills the "standard pulsar" of Sec. 3.
 */
typedef struct tube_params {
    double B_G;            /* surface magnetic field B_* [G]                  */
    double P_s;            /* rotation period P [s]                           */
    double Rstar_cm;       /* stellar radius R_* [cm]                         */
    double incl_rad;       /* inclination i [rad]                             */
    double mass_g;         /* stellar mass M_* [g]                            */
    double R_cm;           /* tube radius R [cm]; <= 0 -> R_* theta_p,
                              theta_p = sqrt(Omega R_* / c) (Sec. 3)          */
    double L_over_R;       /* tube length in units of R                       */
    int64_t Nz;            /* grid cells, 2 <= Nz <= 2^24                     */
    double dt;             /* time step in R/c; <= 0 -> min(0.4 dz, 0.2/Lambda0);
                              must satisfy 0 < dt < dz                        */
    int32_t rho_gj_mode;   /* SCLF_RHO_*                                      */
    int32_t precision;     /* SCLF_FP32, SCLF_FP64 or SCLF_FIX32 (grids are
                              always FP64)                                   */
    const double* rho_gj_user; /* host, Nz+1 node values in code units, read
                                  by tube_create when mode is SCLF_RHO_USER   */
    double lambda_override;/* > 0: use this Lambda0 = omega_p0 R / c instead of
                              deriving it from B, P, R (the calibration of
                              Sec. 3 picks (R, omega_p) with the pulsar's
                              omega_p R / c)                                  */
    double macro_charge;   /* macro-particle charge s < 0 in code units;
                              0 -> -|rho_GJ(0)| L / target_particles          */
    int64_t target_particles; /* used only to derive macro_charge            */
    int64_t capacity;      /* particle slots (live particles plus holes left
                              by removals until the next compaction)          */
    int32_t accumulate;    /* SCLF_ACC_FIXED64 or SCLF_ACC_FP64               */
    int32_t track_ids;     /* 1: keep an int64 ID per particle                */
    int32_t compact_interval; /* steps between compaction checks; 0 -> 64.
                              A check compacts only when holes exceed 1/64
                              of the slots or would add a quarter to the
                              free slots                                     */
    int32_t use_graphs;    /* 1: tube_run replays captured CUDA graphs        */
    /* Eq. 6 in full (SCLF_RHO_GR only; ignored otherwise):
       rho = -(Omega B / 2 pi c alpha) (f / f(1))
             [(1 - omega/Omega) cos i + 3/2 eta^(1/2) (H / f^(1/2)) theta_* sin i]
       with the (R_* / r)^3 factor dropped.                                   */
    int32_t gr_variant;    /* SCLF_GR_COS (default) or SCLF_GR_BOTH           */
    int32_t gr_alpha;      /* 1: divide by the redshift alpha = (1 - r_g/r)^(1/2);
                              0: alpha = 1                                    */
    const double* gr_f;    /* host, Nz+1 values of f(eta) at the nodes (f > 0),
                              or NULL for f = 1; read by tube_create, kept by
                              the tube (f(1) = the value at node 0)           */
    const double* gr_H;    /* host, Nz+1 values of H(eta) at the nodes, or NULL
                              for H = 1; read by tube_create, kept by the tube */
    int32_t sort_interval; /* > 0: tube_run re-sorts the slots by position
                              (tube_sort) every sort_interval steps or more
                              (between graph chunks); 0: never           */
    int32_t push_stages;   /* particle kernel of a single tube: 0 -> the
                              library's default (1); 1: each thread loads its
                              slots straight into registers; 2..4: the tiles
                              a CTA processes next stream into that many
                              shared-memory stages by bulk asynchronous
                              copies (TMA) while it computes (slower on the
                              benchmarked tubes, whose particle kernel is
                              bound by instruction issue, not by load
                              latency). Results do not depend on it (bit
                              for bit); < 0 or > 4 is EINVAL              */
    int32_t launch_overlap;/* consecutive kernels of a step (particles, fields;
                              in batches and adjoint passes too): 0 -> the
                              library's default (1); 1: programmatic
                              dependent launch, each kernel launched as the
                              CTAs of the one before it exit and waiting for
                              it on the device before its first memory
                              access (hides the launch: +10 % on a 1e6-
                              particle tube, neutral on 1e8); -1: plain
                              stream order. Results do not depend on it
                              (bit for bit); other values are EINVAL. A
                              batch takes its first tube's setting        */
} tube_params;

/* Code-unit quantities derived from tube_params (all FP64). */
typedef struct tube_derived {
    double Omega;          /* 2 pi / P [1/s]                                  */
    double theta_p;        /* sqrt(Omega R_* / c)                             */
    double R_cm;           /* tube radius actually used [cm]                  */
    double n0;             /* Omega B / (2 pi c e) [cm^-3] (n_GJ / cos i)     */
    double omega_p0;       /* sqrt(4 pi n0 e^2 / m) [1/s]                     */
    double Lambda0;        /* omega_p0 R / c (or lambda_override)             */
    double kappa;          /* (2/5) r_g / R_*  (Eq. 7)                        */
    double theta_star;     /* 0.67 theta_p (Eq. 5 text)                       */
    double R_over_Rstar;   /* R / R_*                                         */
    double L;              /* tube length in R                                */
    double dz;             /* L / Nz                                          */
    double dt;             /* time step in R/c                                */
    double s;              /* macro-particle charge (< 0)                     */
    double rho0;           /* rho_GJ at node 0, code units                    */
    double pos_unit;       /* cells per stored position unit: 2^-fb for
                              SCLF_FIX32, 1 otherwise                        */
} tube_derived;

/* Per-tube counters, read back by tube_status (synchronises the stream). */
typedef struct tube_stats {
    int64_t step;              /* completed steps                            */
    int64_t n_particles;       /* live particles                             */
    int64_t n_slots;           /* occupied slots (live + holes)              */
    int64_t total_injected;    /* IDs handed out so far                      */
    int64_t last_injected;     /* injected in the last step                  */
    int64_t last_removed;      /* removed in the last step                   */
    int64_t pending_injection; /* electrons the next step will inject        */
    double surface_field;      /* E_s at the base before that injection      */
    uint32_t flags;            /* SCLF_FLAG_* (sticky)                       */
    uint32_t reserved;
} tube_stats;

/* Kernel timings accumulated while timing is enabled. With a sampling
 * period n > 1 (tube_set_timing) the times cover the sampled steps only;
 * per-launch averages are push_ms / n_steps and particle_slots / steps_run. */
typedef struct tube_timing {
    double push_ms;            /* summed device time of the particle kernel  */
    double field_ms;           /* summed device time of the field kernel     */
    double compact_ms;         /* summed device time of compactions          */
    int64_t n_steps;           /* steps timed                                */
    int64_t n_compactions;     /* compactions timed                          */
    int64_t particle_slots;    /* slots processed by the particle kernel, all
                                  steps since timing was enabled            */
    int64_t steps_run;         /* steps run since timing was enabled (timed
                                  or not)                                    */
    int64_t compactions_run;   /* compaction checks launched since then      */
} tube_timing;

/* Fill p with the standard pulsar of Sec. 3 (P = 1 s, B = 1e12 G,
 * R_* = 1e6 cm, M = 1.4 M_sun, i = 0, flat rho_GJ), L = 8 R, Nz = 1024,
 * FP32 particles, fixed-point current, capacity 2^20. */
int tube_params_default(tube_params* p);

/* Validate p and compute the derived code-unit quantities (host only, no
 * CUDA). Units: Sec. 3 normalisation; rho_GJ(0) from Eq. 5 or Eq. 6. */
int tube_derive(const tube_params* p, tube_derived* d);

/* rho_GJ at the Nz+1 nodes (host only, no CUDA) in code units, as
 * tube_create builds it: Eq. 5 (flat), Eq. 6 with Eq. 7 (frame dragging,
 * gr_variant, gr_alpha, gr_f, gr_H) or the caller's profile. rho: host,
 * Nz+1 doubles. SCLF_EINVAL for invalid parameters. */
int tube_rho_gj_profile(const tube_params* p, double* rho);

/* Chain rule from rho_GJ to the pulsar's parameters (host only, no CUDA):
 * grad (host, 3 doubles) = sum_j d_rho[j] d rho_GJ,j / d(B_G, P_s, R_cm) for
 * d_rho (host, Nz+1 doubles), from the analytic derivatives of Eq. 5 or
 * Eq. 6-7 with the Sec. 3 units (Lambda0^2 is proportional to B R^2 / P,
 * theta_* to P^(-1/2), eta_j = 1 + z_j R / R_*), on the fixed grid z_j = j dz
 * (in R) with R an independent coordinate taken at its derived value (so
 * d/dP is at fixed R). lambda_override > 0 holds Lambda0; the f, H tables
 * stay at their nodes; SCLF_RHO_USER gives 0. SCLF_EINVAL for invalid p. */
int tube_rho_gj_param_gradient(const tube_params* p, const double* d_rho, double* grad);

/* Bytes of device memory a tube with these parameters needs. */
int tube_workspace_bytes(const tube_params* p, int64_t* bytes);

/* Create a tube: validate p, build rho_GJ (Eq. 5/6 or user), solve Eq. 4
 * for the empty tube (phi = 0 at the base, phi' = 0 at the top), set
 * E_z = -phi', E_r = phi / R, B_phi = 0 (Sec. 2), and upload to the device.
 * dev_workspace: device memory of at least tube_workspace_bytes() bytes,
 *   aligned to 256 bytes, or NULL to let the library allocate.
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Synchronises the stream before returning. */
int tube_create(const tube_params* p, void* dev_workspace, int64_t ws_bytes,
                void* stream, tube_t* out);

/* Release the tube (and its own device memory if it allocated any). */
int tube_destroy(tube_t t);

/* Copy the derived quantities of a live tube. */
int tube_get_derived(tube_t t, tube_derived* d);

/* One base injection (step (a1) alone, Sec. 2): append the pending number
 * of electrons at z = 0 with u = 0. *n_injected (host, may be NULL)
 * receives the count. Synchronises. */
int tube_inject(tube_t t, int64_t* n_injected);

/* Append n particles at heights z[i] (host, in R, 0 <= z < L) with
 * u[i] = gamma beta (host); IDs continue the tube's count. Used for
 * synthetic prefilled states and tests. Synchronises. */
int tube_add_particles(tube_t t, int64_t n, const double* z, const double* u);

/* One time step (a1..a6 of Sec. 2, Figure A). Asynchronous. */
int tube_step(tube_t t);

/* nsteps time steps; replays captured CUDA graphs of compact_interval
 * steps when use_graphs is set (with event nodes around every kernel while
 * timing is on). Asynchronous. */
int tube_run(tube_t t, int64_t nsteps);

/* Copy fields to host arrays (any may be NULL): Ez, Bphi, J at the Nz cell
 * centres (Ez at step n, Bphi at n+1/2, J of the last step, code units);
 * Er and rho (cloud-in-cell charge density) at the Nz+1 nodes.
 * Synchronises. */
int tube_read_fields(tube_t t, double* Ez, double* Er, double* Bphi,
                     double* J, double* rho);

/* Copy live particles in slot order (ID order unless the tube was re-sorted
 * by cell: tube_sort, sort_interval) to host arrays of capacity cap: z in R,
 * u = gamma beta, id (any of z, u, id may be NULL). *n receives the number
 * of live particles; min(cap, *n) are written. Synchronises. */
int tube_read_particles(tube_t t, int64_t cap, int64_t* n, double* z,
                        double* u, int64_t* id);

/* Raw particle state in the tube's precision, live particles only, slot
 * order (as tube_read_particles):
 * positions xi = z / dz as float (SCLF_FP32) or double (SCLF_FP64), or as
 * int32 X = xi / pos_unit (SCLF_FIX32); u as float (FP32, FIX32) or double.
 * Host buffers of capacity cap (pinned memory makes the copies fastest);
 * *n receives the live count. The slots are compacted on the device first
 * (the order and every result stay as they were). Synchronises.
 * (Checkpointing.) */
int tube_save_particles(tube_t t, int64_t cap, int64_t* n, void* xi, void* u,
                        int64_t* id);

/* Replace all particles by n raw particles (host, layout as
 * tube_save_particles; id may be NULL to number them 0..n-1, and must be
 * NULL for a tube without IDs). Holes are not allowed: every position must
 * lie in [0, Nz) cells, every u be finite and every ID be >= 0; the arrays
 * are copied to the device and checked there, and on SCLF_EINVAL the tube
 * is left without particles. IDs continue after the largest loaded one.
 * Synchronises. */
int tube_load_particles(tube_t t, int64_t n, const void* xi, const void* u,
                        const int64_t* id);

/* Re-solve Eq. 4 with the tube's current charge: phi'' - phi / R^2 =
 * -4 pi (rho - rho_GJ) with rho the cloud-in-cell density of the live
 * particles at the nodes, phi = 0 at the base and phi' = 0 at the top;
 * then E_z = -phi', E_r = phi / R and B_phi = 0 (Sec. 2 initialisation,
 * generalised from the empty tube to a prefilled one). The next injection
 * count is recomputed. Synchronises. */
int tube_solve_fields(tube_t t);

/* Counters and sticky flags. Synchronises. Returns SCLF_OK even when flags
 * are set; tube_check() turns flags into an error code. */
int tube_status(tube_t t, tube_stats* out);

/* Pipelined status: queue a copy of the counters as they stand after the
 * work queued so far (the same fields tube_status gives) into a pinned ring
 * the tube owns, without waiting; *ticket names it. tube_status_collect
 * synchronises the tube's stream and writes that copy to out (caller-owned
 * host memory). A ticket stays valid for the next 1023 tube_status_async
 * calls on the tube; an older, future or unknown ticket returns SCLF_EINVAL.
 * The ring (256 KB of pinned host memory) is allocated on the first call. */
int tube_status_async(tube_t t, int64_t* ticket);
int tube_status_collect(tube_t t, int64_t ticket, tube_stats* out);

/* SCLF_OK, or the error code of the most severe sticky flag. Synchronises. */
int tube_check(tube_t t);

/* Diagnostics of the current state (code units, per unit cross-section):
 * the live particles' largest and mean gamma and kinetic energy
 * |s| sum (gamma - 1) (a deterministic device reduction), the field energy
 * sum (E_z^2 + B_phi^2) dz / 8 pi over the cells plus sum E_r^2 dz / 8 pi over
 * the nodes (half weight at the two ends), and the residual of Gauss's law
 * (Eq. 2 with d/dr -> 1/R) on the interior nodes,
 * G_j = (E_{j+1/2} - E_{j-1/2}) / dz + E_r,j - 4 pi (rho_j - rho_GJ,j), with the
 * scale max 4 pi |rho_j - rho_GJ,j| to compare it with. Synchronises. */
typedef struct tube_diag {
    int64_t n_particles;
    double gamma_max;
    double gamma_mean;
    double kinetic;
    double field_energy;
    double gauss_max;
    double gauss_scale;
} tube_diag;
int tube_diagnostics(tube_t t, tube_diag* out);

/* Compact the particle slots now, whatever the number of holes (removes
 * holes, keeps ID order). Async. */
int tube_compact(tube_t t);

/* Self-test of the failure path of a bounded device-side wait (no paper
 * counterpart): runs one forced compaction in which the first tile publishes
 * nothing, so the decoupled look-back of the second tile gives up after 4096
 * polls, sets SCLF_FLAG_TIMEOUT and the kernel finishes; nothing faults or
 * hangs and the CUDA context stays usable. Returns SCLF_ETIMEOUT when the
 * device reported the timeout (the expected result), SCLF_EINVAL when the
 * tube has at most one tile of slots. The tube's particle slots and counters
 * are unspecified afterwards and its TIMEOUT flag stays set: use a scratch
 * tube. Synchronises. */
int tube_selftest_wait_timeout(tube_t t);

/* Check of the particle kernels' float32 velocity (Sec. 2, Eq. 1: the push
 * advances z by dt u / gamma with gamma = sqrt(1 + u^2)). The kernels
 * compute v = u / sqrt(1 + u^2) by a Newton step on the hardware reciprocal
 * square root and Markstein's FMA division instead of the general-range
 * square root and division; this runs both on the float32 bit patterns
 * [first, first + count) on the current device and counts the patterns
 * whose results differ in any bit (NaN equals NaN): *n_mismatch, and the
 * smallest such pattern in *first_mismatch (0xffffffff when none).
 * first + count <= 2^32, else SCLF_EINVAL; NULL outputs are EINVAL.
 * Allocates 16 bytes of device memory for the call. Synchronises. */
int tube_selftest_velocity(uint32_t first, uint64_t count, uint64_t* n_mismatch,
                           uint32_t* first_mismatch);

/* Re-sort the particle slots by position, stably (particles in one of 256
 * bins per cell keep their slot order; fewer bins above 2^23 cells), and
 * drop the holes: a radix sort of (position bin, slot) pairs with 8-bit
 * digits and a gather of positions, momenta and IDs. The results
 * of every later step are unchanged (the current and the base-cell weight
 * are exact integer sums, independent of the order); the particle kernel
 * gets back its per-cell runs. Afterwards the slot order, and so the order
 * of tube_read_particles / tube_save_particles, is cell order rather than ID
 * order. The first call allocates scratch of about 24 bytes per slot of
 * capacity (plus 8 with IDs). Synchronises. */
int tube_sort(tube_t t);

/* Per-kernel CUDA-event timing of steps: enable = n >= 1 times every n-th
 * unit of work, a unit being one step launched on its own or one graph
 * replay of a compaction interval's steps (every step: n = 1); 0 disables;
 * < 0 is EINVAL. Enabling clears the accumulated numbers. A timed graph
 * replay carries an event-record node before each kernel (and one after the
 * last); each such node adds a few microseconds to the run, so a sampling
 * period keeps the run's own pace close to the untimed one. Compaction
 * checks are timed whenever timing is enabled. Reading a timed replay back
 * waits for the replay two timed chunks earlier. */
int tube_set_timing(tube_t t, int enable);

/* Accumulated timings since timing was enabled. Synchronises. */
int tube_get_timing(tube_t t, tube_timing* out);

/* ---- one tube split into z-domains ------------------------------------------
 * A tube's cells cut into contiguous ranges ("sub-domains"), each with its own
 * particle slots, stream and copy of the grids, as a multi-GPU run would hold
 * them; here all sub-domains share one GPU. The split follows Sec. 2: Eq. 3
 * couples a cell only to its neighbours (B_phi of the adjacent cells, E_r at
 * the cell's two nodes), the cloud-in-cell gather reads the cell and its
 * neighbour, and a particle moves less than one cell per step (c dt < dz),
 * so each step a sub-domain exchanges with each neighbour: the current its
 * particles deposited in the neighbour's first cell, the neighbour's new
 * B_phi and E_z of that cell (E_r at the shared node is computed on both
 * sides from the same values), and the particles that crossed. Every step
 * runs: particle kernels (one per sub-domain, concurrently) -> current
 * exchange -> field kernels -> particle hand-off and field halos. The
 * current is the exact fixed-point sum, so a decomposed run gives the same
 * fields bit for bit as the same tube stepped whole, and the same particles
 * (compared by ID; their slot order differs). Requires SCLF_ACC_FIXED64;
 * every sub-domain has at least 2 cells. Only the base sub-domain injects. */
typedef struct sclf_dtube* dtube_t;   /* opaque, library-owned */

/* Create a tube of parameters *p split at the cell boundaries cuts[0..n]
 * (host array: cuts[0] = 0 < cuts[1] < ... < cuts[n] = Nz, every range at
 * least 2 cells), or into n near-equal ranges when cuts is NULL; 1 <= n <= 64.
 * Each sub-domain holds the tube's full capacity of slots and its own copy
 * of the grids (only its cells and their neighbours are kept current), plus
 * two outboxes of max(65536, capacity/8) particles for the particles that
 * leave it; an outbox overflow sets SCLF_FLAG_CAPACITY. The fields start as
 * the empty tube's (Eq. 4 without particles). Synchronises. EINVAL for bad
 * cuts, accumulate != SCLF_ACC_FIXED64 or invalid params. */
int dtube_create(const tube_params* p, int32_t n, const int64_t* cuts, dtube_t* out);

/* Free every sub-domain and the exchange buffers. */
int dtube_destroy(dtube_t dt);

/* Number of sub-domains, and sub-domain i's tube and owned cells [lo, hi).
 * The tube is for reading (tube_read_particles, tube_save_particles,
 * tube_status, tube_read_fields: only cells lo-1..hi of its grids are
 * current); stepping it alone returns SCLF_ESTATE. */
int dtube_domains(dtube_t dt, int32_t* n);
int dtube_domain(dtube_t dt, int32_t i, tube_t* tube, int64_t* lo, int64_t* hi);

/* The tube's initial particles (host heights z in [0, L) in units of R, and
 * u = gamma beta; ID k for particle k), each given to the sub-domain of its
 * cell. Only on a tube that has no particles and has not stepped (ESTATE
 * otherwise). Synchronises. */
int dtube_load_particles(dtube_t dt, int64_t n, const double* z, const double* u);

/* Set every sub-domain's fields from host arrays: E_z at the Nz cells, E_r
 * at the Nz+1 nodes, B_phi at the Nz cells (NULL: zero); the next injection
 * count follows from them (Sec. 2). Synchronises. */
int dtube_set_fields(dtube_t dt, const double* Ez, const double* Er, const double* Bphi);

/* Eq. 4 with the charge of every sub-domain's particles (as
 * tube_solve_fields; the density is summed over the sub-domains in FP64, so
 * its last bits can differ from a whole tube's). Synchronises. */
int dtube_solve_fields(dtube_t dt);

/* One step (Figure A) of every sub-domain with its exchanges. Async. */
int dtube_step(dtube_t dt);
/* nsteps such steps. With use_graphs and an even compaction interval, runs of
 * that many steps starting at an even step right after a compaction check
 * replay one CUDA graph captured on first use (the same kernels and
 * exchanges, bit for bit); the other steps are launched one by one. Async. */
int dtube_run(dtube_t dt, int64_t nsteps);

/* The whole tube's counters: live particles, slots, removals and flags
 * summed (flags OR-ed) over the sub-domains, injection counters of the base
 * sub-domain. Synchronises. */
int dtube_status(dtube_t dt, tube_stats* out);

/* The whole tube's fields (caller-owned host arrays, NULL skips): each cell
 * (and node) from the sub-domain that owns it; the last node from the top
 * sub-domain. Synchronises. */
int dtube_read_fields(dtube_t dt, double* Ez, double* Er, double* Bphi, double* J);

/* Data exchanged between sub-domains since creation: *steps, *field_bytes
 * (current, B_phi and E_z halo values), *particles (particles handed to a
 * neighbour) and *particle_bytes (their positions, momenta and IDs).
 * Synchronises. */
int dtube_exchange_stats(dtube_t dt, int64_t* steps, int64_t* field_bytes, int64_t* particles,
                         int64_t* particle_bytes);

/* ---- batches of independent tubes -------------------------------------------
 * Many tubes (each its own pulsar: B, P, R, Nz, rho_GJ profile, particles)
 * advanced together: every step is one particle launch over all tubes'
 * tiles and one field launch over all tubes' cells (plus the per-tube
 * compaction checks), so tubes of uneven Nz and particle count share the
 * GPU. Each tube computes exactly what it would compute alone (Sec. 2 step
 * for every tube). Batched tubes must use SCLF_ACC_FIXED64 and all the
 * same particle format: SCLF_FP32, or SCLF_FIX32 (32-bit fixed-point
 * positions; each tube's fractional bits follow from its own Nz). */
typedef struct sclf_batch* batch_t;   /* opaque, library-owned */

/* Create n tubes from params[0..n-1] (host array) on one stream; the
 * compaction interval and graph flag of params[0] apply to the batch.
 * Synchronises. */
int batch_create(int32_t n, const tube_params* params, void* stream, batch_t* out);

/* Destroy the batch and its tubes. */
int batch_destroy(batch_t b);

/* Number of tubes. */
int batch_size(batch_t b, int32_t* n);

/* The i-th tube: tube_add_particles, tube_solve_fields, tube_read_*,
 * tube_status, tube_save/load_particles, tube_inject and tube_compact work
 * on it; tube_step and tube_run return SCLF_ESTATE (the batch steps it). */
int batch_tube(batch_t b, int32_t i, tube_t* out);

/* The counters of all n tubes (n must equal batch_size) in one call: one
 * gather kernel and one device-to-host copy into out[0..n-1] (caller-owned
 * host memory), the same fields tube_status gives for each tube.
 * Synchronises the batch's stream. */
int batch_status(batch_t b, int32_t n, tube_stats* out);

/* One step of every tube. Asynchronous. */
int batch_step(batch_t b);

/* nsteps steps of every tube (replays a captured graph when timing is off).
 * Asynchronous. */
int batch_run(batch_t b, int64_t nsteps);

/* Per-kernel event timing of the batched launches: enable = n >= 1 times
 * every n-th step (each timed step is launched on its own, with event
 * records around its kernels); with n > 1 the other steps run as graph
 * replays where the step count allows; 0 disables; < 0 is EINVAL. */
int batch_set_timing(batch_t b, int enable);

/* Accumulated timings; particle_slots sums over all tubes. Synchronises. */
int batch_get_timing(batch_t b, tube_timing* out);

/* Shapes of the batched particle kernel (index: particles per thread, CTAs
 * per SM in its launch bounds, per-thread current runs): 0: 8, 4, 1 (the
 * default); 1: 8, 3, 1; 2: 4, 4, 1; 3: 8, 4, 2; 4: 8, 3, 2; 5: 16, 2, 2.
 * Tiles are 256 threads times the particles per thread; a second run sums
 * the current of the particles sharing the cell of a thread's last particle
 * without a branch (for tubes with few particles per cell). Every shape
 * computes the same results bit for bit (the current and W_0 are exact
 * integer sums in any order). */
#define SCLF_BATCH_VARIANTS 6

/* Use shape `variant` from the next step on (SCLF_EINVAL outside
 * [0, SCLF_BATCH_VARIANTS); an SCLF_FIX32 batch has one shape, 0). */
int batch_set_variant(batch_t b, int32_t variant);

/* Autotuner: run 2 + steps ordinary steps of the batch with each shape,
 * timing its particle kernel with CUDA events, and keep the fastest. ms
 * (host, SCLF_BATCH_VARIANTS doubles, may be NULL) receives each shape's
 * mean particle-kernel time per step, chosen (may be NULL) the shape kept.
 * The batch advances by SCLF_BATCH_VARIANTS * (steps + 2) steps; timing is
 * left off and its totals cleared. An SCLF_FIX32 batch times its one shape
 * (steps + 2 steps; ms[1..] = -1). Synchronises. */
int batch_autotune(batch_t b, int32_t steps, double* ms, int32_t* chosen);

/* ---- discrete adjoint of a run: gradients ------------------------------------
 * An adjoint driver owns one tube (SCLF_FP32, SCLF_FP64 or SCLF_FIX32
 * particles, SCLF_ACC_FIXED64 current) and differentiates an N-step run of it (the
 * Sec. 2 step of Figure A) that starts from the particles the tube holds at
 * the first adjoint_forward, with fields solving Eq. 4 for their charge
 * (as tube_solve_fields). The inputs it differentiates are rho_GJ at the
 * nodes (which enters through the t = 0 fields of Eq. 4) and the
 * macro-particle charge s (which enters the current J = (s/dt) sum F and
 * the charge of the particles at t = 0). Held fixed: the number of
 * electrons injected at each step (recorded by the forward pass, or given by
 * adjoint_set_injections), the grid (L, Nz, dt in code units) and the
 * rounding of the particle precision (including SCLF_FIX32's rounding of
 * the displacement to its position grid). The piecewise-linear gather and
 * deposit are differentiated inside their pieces (dF_j/dx = 1 on cell j);
 * adjoints of positions are in cell units.
 * Particles keep their slots for the whole run (no compaction).
 *
 * The forward pass stores the state at every checkpoint_every-th step; the
 * backward pass recomputes each segment from its checkpoint with the
 * recorded injections, keeping every step of that one segment, and sweeps
 * it in reverse (transposed Eq. 3 on the grid in FP64, then per particle
 * the adjoints of the deposit, the Eq. 1 push and the gather, in the
 * particle precision, their grid sums in FP64). */
typedef struct sclf_adjoint* adjoint_t;   /* opaque, library-owned */

#define SCLF_OBJ_GAMMA 0   /* mean gamma = sqrt(1 + u^2) over the live particles
                              after the last step                            */
#define SCLF_OBJ_EZ    1   /* ||E_z||_2 = sqrt(sum_j E_z,j^2 dz) after the last
                              step                                           */
#define SCLF_OBJ_EZ_WEIGHTED 2 /* sum_j w_j E_z,j after the last step, with the
                              cell weights of adjoint_set_weights: any
                              projection of the E_z profile (unit weights give
                              one cell's sensitivity); its value is the dot
                              product of w with tube_read_fields' E_z     */

/* Create a driver for runs of nsteps steps (> 0, even, a multiple of
 * checkpoint_every, which is even and > 0) of a tube with parameters p
 * (track_ids is ignored). checkpoint_every = 0 lets the library choose the
 * longest segment whose arrays fit in 80 % of the free device memory: a
 * single segment (K = nsteps), whose backward pass needs no recompute, when
 * the whole run's snapshots fit (adjoint_checkpoint_every reports the
 * choice; ENOMEM when not even K = 2 fits). Device memory: about checkpoint_every +
 * nsteps / checkpoint_every + 5 copies of the particle arrays
 * (2 * capacity * 4 or 8 bytes each) and checkpoint_every grid copies.
 * SCLF_EINVAL for SCLF_ACC_FP64 (a recompute must reproduce the run bit for
 * bit, which FP64 atomics do not promise), SCLF_ENOMEM when it
 * does not fit. Work goes to the tube's stream (stream, or a stream of its
 * own when NULL). Synchronises. */
int adjoint_create(const tube_params* p, int64_t nsteps, int32_t checkpoint_every,
                   void* stream, adjoint_t* out);

/* The segment length K the driver uses (the caller's checkpoint_every, or
 * the library's choice for checkpoint_every = 0). */
int adjoint_checkpoint_every(adjoint_t a, int32_t* k);

/* Destroy the driver and its tube. */
int adjoint_destroy(adjoint_t a);

/* The driver's tube: fill it (tube_add_particles, tube_load_particles,
 * tube_inject) before the first adjoint_forward; after a forward pass its
 * particles, fields and counters are those at the end of the run (read
 * them with tube_read_*, tube_status). tube_step and tube_run return
 * SCLF_ESTATE on it. The driver keeps ownership. */
int adjoint_tube(adjoint_t a, tube_t* out);

/* n_inj: host, nsteps counts that the forward pass injects instead of the
 * tube's own choice (replaying another run's events), or NULL to return
 * to the tube's own rule. A negative count is SCLF_EINVAL. */
int adjoint_set_injections(adjoint_t a, const int64_t* n_inj);

/* w: host, Nz finite cell weights of SCLF_OBJ_EZ_WEIGHTED (copied). */
int adjoint_set_weights(adjoint_t a, const double* w);

/* Run the nsteps steps from the initial state (the tube's particles at the
 * first call), storing checkpoints and the per-step events. values: host,
 * 2 doubles or NULL, receives the objectives SCLF_OBJ_GAMMA and
 * SCLF_OBJ_EZ. Synchronises. */
int adjoint_forward(adjoint_t a, double* values);

/* Per-step events of the last forward pass into host arrays of nsteps
 * (each may be NULL): electrons injected, particles removed (left the tube
 * or became non-finite) and slots in use before the step. SCLF_ESTATE
 * before the first forward pass. Synchronises. */
int adjoint_events(adjoint_t a, int64_t* n_inj, int64_t* n_removed, int64_t* n_slots);

/* Gradient of one objective (SCLF_OBJ_*) of the last forward pass
 * (SCLF_ESTATE for SCLF_OBJ_EZ_WEIGHTED before adjoint_set_weights): d_rho_gj (host,
 * Nz+1 doubles or NULL) = d objective / d rho_GJ at the nodes (node 0 is
 * 0: it enters only the frozen injection count), d_s (host or NULL) =
 * d objective / d s. SCLF_ESTATE before the first forward pass.
 * Synchronises. */
int adjoint_backward(adjoint_t a, int32_t objective, double* d_rho_gj, double* d_s);

/* Chain a gradient to the pulsar's parameters: grad (host, 4 doubles) =
 * d objective / d(B_G, P_s, R_cm, w), where the macro charge is s = w s_ref.
 * s_ref: the reference charge the weight w multiplies, or 0 to take the
 * tube's own s (w = 1); d/dw = d_s s_ref. The B, P, R entries are
 * tube_rho_gj_param_gradient(d_rho_gj) of the driver's tube (analytic
 * derivatives of Eq. 5 or Eq. 6-7 on the fixed grid, R an independent
 * coordinate taken at its derived value; a SCLF_RHO_USER profile gives 0).
 * SCLF_EINVAL for a non-finite s_ref. */
int adjoint_param_gradient(adjoint_t a, const double* d_rho_gj, double d_s, double s_ref,
                           double* grad);

/* Device time (CUDA events on the driver's stream) of the last forward and
 * backward passes, and the particle slots one pass processes (the sum over
 * steps of the slots in use plus the electrons injected). */
int adjoint_timing(adjoint_t a, double* forward_ms, double* backward_ms,
                   int64_t* particle_steps);

/* Per-kernel CUDA-event timing of the passes that follow: every > 0 times
 * every every-th segment of each kind (recorded forward, recompute,
 * reverse) with a graph that carries event-record nodes around each
 * kernel (about 2-3 us each on this GPU, hence the sampling); 0 turns it
 * off. Clears the totals. SCLF_EINVAL for every < 0. Synchronises. */
int adjoint_set_timing(adjoint_t a, int every);

/* Per-kernel totals of the timed segments since timing was enabled, 6
 * entries each (host, may be NULL): forward particle, forward field,
 * recompute particle, recompute field, reverse field, reverse particle
 * kernels; ms = summed device time, launches = number of timed launches. */
int adjoint_kernel_times(adjoint_t a, double* ms, int64_t* launches);

/* ---- one pass without any device allocation --------------------------------
 * The paper has no counterpart to this call; it is here for users of the
 * library who cannot call cudaMalloc: an application whose own allocator has
 * reserved the device's memory, a plug-in whose host forbids allocation once
 * it runs, or a latency-critical loop that cannot afford the device-wide
 * synchronisation of cudaMalloc/cudaFree. After its first call on a device
 * it allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).
 *
 * One gather-push-deposit pass over n FP32 particles, the same arithmetic
 * as a tube step without injection: cloud-in-cell gather of E_z, the Eq. 1
 * push, the charge-conserving current summed in 2^-32 fixed point, and
 * removal of particles leaving the tube (their xi becomes -1, u 0).
 *   xi, u     device, n floats each, in/out: positions in cell units
 *             (xi = z / dz; entries with xi < 0 are holes and are skipped)
 *             and u = gamma beta
 *   ez        device, nz doubles: E_z at the cell centres (code units)
 *   dt, dz    step and cell size in R/c and R (0 < dt < dz); s < 0 the
 *             macro-particle charge
 *   j_out     device, nz doubles, out: J_{j+1/2} = (s/dt) sum of fractions
 *   n_removed device int64 or NULL, out: particles removed by this pass,
 *             those that left the tube and those whose push gave a NaN or
 *             an infinity (both become holes)
 *   flags     device uint32 or NULL, in/out: SCLF_FLAG_NONFINITE is OR-ed
 *             in when a push gave a NaN or an infinity (other bits are kept)
 *   stream    cudaStream_t; the call is asynchronous on it
 * Returns SCLF_ECUDA without launching anything when a CUDA error is already
 * pending in the calling thread (cudaPeekAtLastError; it stays pending).
 * Its scratch is one fixed file-scope device array of SCLF_STATIC_MAX_NZ
 * cells (about 1 MB), held by every GPU that loads the library until the
 * process exits; nz > SCLF_STATIC_MAX_NZ returns SCLF_EINVAL.
 * The first call on a device, with that device current, does the set-up:
 * CUDA loads modules lazily by default, so it loads this call's kernels and
 * the scratch array (which takes device memory) and looks up the array's
 * device address (cudaGetSymbolAddress). Make that first call before the
 * application reserves the device's memory and before any stream capture
 * (or run with CUDA_MODULE_LOADING=EAGER); later calls allocate nothing.
 * After a cudaDeviceReset the library must be reloaded before this call is
 * used again on that device (the address is cached per device).
 * Every call shares the array and clears it before use, so calls that
 * overlap on the GPU (other streams, other host threads) race with one
 * another: serialise them. */
#define SCLF_STATIC_MAX_NZ 65536
int tube_push_deposit_static(float* xi, float* u, int64_t n, const double* ez,
                             int32_t nz, double dt, double dz, double s,
                             double* j_out, int64_t* n_removed, uint32_t* flags,
                             void* stream);

/* Human-readable name of a return code (static storage). */
const char* tube_strerror(int code);

/* Library version string, e.g. "sclf_tube 0.1.0 sm_103a". */
const char* tube_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SCLF_TUBE_H */
