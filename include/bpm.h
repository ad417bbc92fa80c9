/*
 * bpm.h -- C ABI of the GB300 (sm_103a) bonded-particle magneto-elastic rod
 * library: one timestep of the model of Alkuino, Clemmer, Santangelo and
 * Zhang, "Bonded-particle model for magneto-elastic rods" (arXiv 2603.27279).
 *
 * What one step computes (all on the GPU, FP64 unless `precision` says
 * otherwise):
 *   - co-rotational bond forces and torques between consecutive particles of
 *     a rod (main text, "Bonded-particle model for elastic rods", Eqs.
 *     bpm-fr, bpm-fst, bpm-tst, bpm-tb, bpm-tt, bpm-vector; SI "Symmetric
 *     rotational decomposition", Eq. S-quat-h), spring constants from
 *     (E, nu, d) as in the main text after Eq. bpm-vector;
 *   - Zeeman torque m x B and force grad(m.B) on each particle's body-fixed
 *     dipole m = R m~ (Methods, "Magnetic interactions"; main text,
 *     "Magnetized beams in non-uniform fields");
 *   - all-pairs open-boundary dipole-dipole forces and torques (Methods,
 *     "Magnetic interactions", U_ij);
 *   - global viscous damping and bond-level damping per mode (Methods,
 *     "Damping");
 *   - optional Hertz-Mindlin contact between non-bonded particles
 *     (Methods, "Contact");
 *   - velocity Verlet for x, v, omega and Richardson extrapolation for q
 *     with renormalisation after every substep (SI "Equations of motion").
 *
 * Conventions
 *   - Arrays crossing this ABI are AoS per particle, float64: x[3N],
 *     q[4N] = (w, x, y, z) (Hamilton product; a body vector maps to space
 *     as q v q*), v[3N], omega[3N] (space frame), f[3N], tau[3N].
 *   - Rods are CSR: rod r holds particles rod_offset[r] .. rod_offset[r+1]-1;
 *     a bond joins each pair of consecutive particles of a rod.
 *   - Every call returns BPM_OK (0) or a negative BPM_ERR_* code and never
 *     throws; bpm_last_error() gives the message of the last failure.
 *   - The handle owns every device buffer it allocates; the caller owns the
 *     arrays it passes and may free them as soon as the call returns.
 *   - Work is issued on desc.stream (a cudaStream_t; NULL = a stream the
 *     handle creates).  Calls that return data to the host synchronise that
 *     stream.  A handle is not thread-safe.
 */
#ifndef BPM_H
#define BPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BPM_OK 0
#define BPM_ERR_ARG (-1)       /* invalid argument or description          */
#define BPM_ERR_CUDA (-2)      /* a CUDA call failed (message has details) */
#define BPM_ERR_NONFINITE (-3) /* a force, torque, position or orientation
                                  became non-finite during bpm_step        */
#define BPM_ERR_TIMEOUT (-4)   /* a bounded device-side wait gave up       */
#define BPM_ERR_SINGULAR (-5)  /* zero-length rest bond                    */
#define BPM_ERR_CAPACITY (-6)  /* a particle had more contacts than
                                  bpm_contact.max_contacts                 */

#define BPM_DIPOLE_OFF 0       /* no dipole-dipole interaction             */
#define BPM_DIPOLE_GLOBAL 1    /* all ordered pairs i != j of the system   */
#define BPM_DIPOLE_PER_ROD 2   /* all ordered pairs i != j within each rod */

#define BPM_FP64 0             /* everything in FP64                       */
#define BPM_MIXED 1            /* dipole pair terms in FP32 (positions as
                                  FP32 hi/lo pairs), per-particle sums
                                  flushed to FP64 every j-tile; bonds,
                                  Zeeman and integration stay FP64          */
#define BPM_FF 2               /* dipole pair terms in float-float (pairs of
                                  FP32 joined by error-free transforms, about
                                  48 significant bits; positions as exact
                                  fixed-binade FP32 digits), sums flushed to
                                  FP64 every 32 pairs; symmetric dipole
                                  plans only; the adjoint's dipole VJP in
                                  float-float as well, and the fluid's
                                  collision (FP64 storage).  The finest
                                  position
                                  digit Q is fixed at create: the smallest
                                  power of two with 2^66 Q >= 4 max|x0| + 64
                                  over the initial coordinates.  A particle
                                  with a coordinate of 2^66 Q or more makes
                                  the forces non-finite (BPM_ERR_NONFINITE
                                  from bpm_step).  Bonds, Zeeman and
                                  integration stay FP64                     */

/* Hertz-Mindlin contact between particles that are not bonded neighbours
 * (Methods, "Contact"; the paper names the model, the forms are the
 * textbook ones).  For overlapping particles i, j (d = x_i - x_j,
 * n = d/|d|, delta = R_i + R_j - |d| > 0, R* = R_i R_j/(R_i + R_j),
 * E* = E/(2(1 - nu^2)), G* = G/(2(2 - nu)), G = E/(2(1 + nu)),
 * a = sqrt(R* delta)):
 *   normal force on i     (4/3 E* a delta - gamma_n v_n) n;
 *   contact velocity      v_rel = v_i - v_j - (R_i w_i + R_j w_j) x n,
 *                         v_n = v_rel . n, v_t = v_rel - v_n n;
 *   tangential history    xi = (xi_old in the current tangent plane, its
 *                         length kept) + v_t dt, zero before the contact;
 *   tangential force      F_t = -8 G* a xi - gamma_t v_t, at most
 *                         mu 4/3 E* a delta in length (xi then follows F_t);
 *   torques               (-R_i n) x F_t on i, (-R_j n) x F_t on j.
 * Particles of the same rod at most `exclude` bonds apart do not touch.
 * The histories follow the rule of bpm_desc.bond_damping: the force
 * evaluation of a step advances them, bpm_forces / bpm_energy read the
 * previous state's, bpm_set_state forgets them.  Contact energy is not part
 * of bpm_energy. */
typedef struct bpm_contact {
    double E;                  /* Young's modulus of the particles > 0     */
    double nu;                 /* Poisson ratio, -1 < nu < 0.5             */
    double mu;                 /* Coulomb friction coefficient >= 0        */
    double gamma_n, gamma_t;   /* viscous damping of v_n and v_t, >= 0     */
    int32_t exclude;           /* bonded-neighbour exclusion depth >= 0    */
    int32_t max_contacts;      /* history slots per particle, 1..64 (0: 16);
                                  more simultaneous contacts on a particle
                                  make bpm_step / bpm_forces return
                                  BPM_ERR_CAPACITY                         */
} bpm_contact;

/* Lattice Boltzmann fluid coupled to the particles (Methods, "Lattice
 * Boltzmann method", "Immersed boundary coupling"): a periodic D3Q19 lattice
 * with BGK collision, f_eq = w rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u), and
 * Guo's forcing, the velocity in both taken at the half step,
 * rho u = sum f e + F/2, F = body_force + the particles' reaction.  Lattice
 * units: spacing 1 in the system's length unit, one LBM step = n_sub DEM
 * steps = 1 time unit (desc.dt * n_sub must be 1), density scale 1; node
 * (i, j, k) sits at (i, j, k), index i + nx (j + ny k).
 * Coupling: at the start of each LBM cycle (the first step's force
 * evaluation) the fluid velocity is interpolated at every coupled particle
 * with Peskin's four-point delta; every force evaluation adds the penalty
 * force m_p (U - v_p) (kappa = m_p / dt_LBM, v_p the velocity present at
 * force time); the force evaluations of the time stepping spread -F_p / n_sub
 * onto the lattice with the same weights; after n_sub steps one LBM step
 * runs.  Particles are point forces (no torque exchange).  bpm_set_state
 * restarts the cycle and re-interpolates.  BPM_FP64 handles store the
 * distributions in FP64; BPM_FF handles store them in FP64 and collide in
 * float-float on the deviations f - w (formed in FP64); BPM_MIXED handles
 * store f - w in FP32 and collide in FP32.  The reaction sums use FP64
 * atomics: steps with a fluid are
 * reproducible to rounding, not bit for bit. */
typedef struct bpm_lbm {
    int32_t nx, ny, nz;        /* nodes per axis, >= 1                     */
    int32_t n_sub;             /* DEM steps per LBM step, >= 1             */
    double tau;                /* BGK relaxation time > 0.5; the kinematic
                                  viscosity is (tau - 1/2)/3               */
    double body_force[3];      /* uniform force density on the fluid       */
    const double* rho0;        /* [nodes] initial density (host), or NULL = 1 */
    const double* u0;          /* [3 nodes] initial velocity, AoS (host), or NULL = 0 */
    const uint8_t* coupled;    /* [N] 1 = exchanges momentum with the fluid
                                  (host), or NULL = every particle          */
} bpm_lbm;

/* Description of a system; every pointer is a HOST pointer read during
 * bpm_create only. */
typedef struct bpm_desc {
    int64_t n_particles;       /* N >= 0                                   */
    int64_t n_rods;            /* R >= 1 when N > 0                         */
    const int64_t* rod_offset; /* [R+1], rod_offset[0] = 0, [R] = N,
                                  non-decreasing                            */
    const double* x;           /* [3N] positions                           */
    const double* q;           /* [4N] orientations (normalised on entry)  */
    const double* v;           /* [3N] or NULL (zero)                      */
    const double* omega;       /* [3N] or NULL (zero)                      */
    const double* mass;        /* [N] > 0                                  */
    const double* radius;      /* [N] > 0; I = 2/5 m R^2 (solid sphere)    */
    const double* m_body;      /* [3N] dipole in the body frame, or NULL   */
    const uint8_t* clamped;    /* [N] 1 = excluded from integration, or NULL;
                                  v and omega of clamped particles are set
                                  to zero                                   */
    const double* x_rest;      /* [3N] configuration in which the bonds are
                                  created, or NULL = x                     */
    const double* q_rest;      /* [4N] or NULL = q                         */
    const double* E;           /* [R] Young's modulus per rod              */
    const double* nu;          /* [R] Poisson ratio, G = E / (2 (1 + nu))  */
    const double* d;           /* [R] bond (cylinder) diameter             */
    /* external field B(x,t) = B + B_rod[rod] + Brot_amp (cos(Brot_omega t)
     * e1 + sin(Brot_omega t) e2) + gradB (x - gradB_x0)                    */
    double B[3];
    const double* B_rod;       /* [3R] or NULL                             */
    double Brot_amp, Brot_omega;
    double Brot_e1[3], Brot_e2[3];
    double gradB[9];           /* row-major dB_a/dx_b                      */
    double gradB_x0[3];
    double mu0_over_4pi;       /* prefactor c of U_ij                      */
    int32_t dipole_mode;       /* BPM_DIPOLE_*                             */
    int32_t precision;         /* BPM_FP64, BPM_MIXED or BPM_FF            */
    double damping;            /* global viscous damping coefficient >= 0  */
    double dt;                 /* timestep > 0                             */
    double t0;                 /* initial time                             */
    void* stream;              /* cudaStream_t or NULL                     */
    /* Bond-level damping per mode (Methods, "Damping"): [4R] per rod
     * g_r, g_s, g_t, g_b >= 0 (host), or NULL = none.  Radial: g_r (dv . r^_f)
     * with dv = v_2 - v_1 the velocities present at force time; shear, twist,
     * bend: g_s r_f gamma' along s^ (and 1/2 g_s r_f^2 gamma' along t^ in the
     * torque), g_t psi' about the bond axis, g_b theta' along b^, the rates
     * being backward differences over dt of the measures gamma, psi, theta.
     * The handle keeps each bond's measures of the previous and of the
     * current state: the force evaluation of each step (at a new state)
     * differences against the current state's and then shifts them;
     * bpm_forces and bpm_energy difference against the previous state's, so
     * they reproduce the angular damping the last step ended with, and only
     * fill in the current state's when there is none.  A new handle and
     * bpm_set_state start without measures (zero angular rates). */
    const double* bond_damping;
    /* Contact between non-bonded particles (see bpm_contact), or NULL.
     * Supported for n_particles <= 2^21. */
    const bpm_contact* contact;
    /* Lattice Boltzmann fluid (see bpm_lbm), or NULL. */
    const bpm_lbm* lbm;
} bpm_desc;

typedef struct bpm_handle bpm_handle;

/* Builds a system: validates the description, normalises quaternions,
 * computes each bond's rest vector and K_r = EA/L, K_s = 12EI/L^3,
 * K_t = GJ/L, K_b = EI/L (main text after Eq. bpm-vector), uploads the
 * state to device memory owned by the handle.  *out is NULL on failure.
 * Errors: BPM_ERR_ARG (bad description), BPM_ERR_SINGULAR (zero-length
 * rest bond), BPM_ERR_CUDA (allocation or copy failed). */
int bpm_create(const bpm_desc* d, bpm_handle** out);

/* State arrays owned by the caller for bpm_create_device: DEVICE pointers
 * of the current device, component-major (SoA): x[3][N] holds component k of
 * particle i at x[k N + i] (a contiguous torch tensor of shape (3, N)), and
 * likewise q[4][N] (w, x, y, z), v[3][N], omega[3][N], f[3][N], tau[3][N].
 * All six are required. */
typedef struct bpm_device_state {
    double* x;
    double* q;
    double* v;
    double* omega;
    double* f;
    double* tau;
} bpm_device_state;

/* Builds a system whose state lives in caller-owned device arrays (the same
 * model and validation as bpm_create; main text "Bonded-particle model for
 * elastic rods", spring constants after Eq. bpm-vector).  The handle works on
 * st's arrays in place: bpm_step advances x, q, v, omega there and leaves the
 * forces of the final state in f and tau; bpm_forces and bpm_energy write f
 * and tau there too.  On entry the arrays hold the initial state (f and tau
 * are overwritten); bpm_create_device normalises q in place and sets v and
 * omega of clamped particles to zero.  The caller keeps the arrays alive
 * until bpm_destroy, which never frees them, and changes them between calls
 * only through bpm_set_state (or bpm_set_forces), so that the handle knows
 * its stored forces are stale.
 * d->x, d->q, d->v and d->omega must be NULL (the state comes from st);
 * d->x_rest (host) may give the rest positions, NULL = the initial device
 * positions; d->q_rest must be NULL: rest orientations are the identity, the
 * paper's convention q^i = 1, so q is each particle's rotation since rest.
 * Errors: BPM_ERR_ARG (a pointer that is not device memory of the current
 * device, a state field of d set, d->q_rest set, or a bad description as in
 * bpm_create), BPM_ERR_SINGULAR, BPM_ERR_CUDA. */
int bpm_create_device(const bpm_desc* d, const bpm_device_state* st, bpm_handle** out);

/* Frees every resource of the handle (NULL is ignored).  Arrays given to
 * bpm_create_device stay the caller's. */
void bpm_destroy(bpm_handle* h);

/* Total force and torque at the current state and time (bonds, Zeeman,
 * dipole-dipole, damping with the current velocities).  f and tau ([3N]
 * each, AoS) may be host or device pointers, or NULL to skip the copy;
 * device pointers must be writable by the handle's device.  The handle
 * keeps the result as the forces of the current state.
 * Errors: BPM_ERR_ARG, BPM_ERR_CAPACITY, BPM_ERR_CUDA. */
int bpm_forces(bpm_handle* h, double* f, double* tau);

/* Advances n >= 0 velocity-Verlet steps (SI "Equations of motion"), the
 * step loop replayed from CUDA graphs.  On return x, v, q, omega, t and the
 * stored forces are those at the end of the n steps.  Synchronises the
 * stream once at the end to read the device error word.
 * Errors: BPM_ERR_NONFINITE (the state left the finite range; the message
 * names the first step at which it did), BPM_ERR_CAPACITY, BPM_ERR_ARG,
 * BPM_ERR_CUDA. */
int bpm_step(bpm_handle* h, int32_t n);

/* Energies of the current state: out[5] = {bond (main text Eq.
 * total-energy), Zeeman (-sum m.B), dipole-dipole (sum over pairs i<j of
 * U_ij), translational kinetic, rotational kinetic}; host pointer.
 * Recomputes (and stores) the forces of the current state.
 * Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_energy(bpm_handle* h, double out[5]);

/* Copies the current state out: any pointer may be NULL; each may be host or
 * device.  x[3N], q[4N], v[3N], omega[3N], *t (host).
 * Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_get_state(bpm_handle* h, double* x, double* q, double* v, double* omega, double* t);

/* Replaces the state (NULL pointers leave that part unchanged; host or
 * device pointers); q is normalised; clamped particles keep zero v and
 * omega.  Invalidates the stored forces and forgets the bond-damping
 * measures.
 * Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_set_state(bpm_handle* h, const double* x, const double* q, const double* v,
                  const double* omega, double t);

/* Declares f and tau ([3N] each, AoS, host or device) the forces and torques
 * of the current state, so that the next bpm_step starts from them instead
 * of evaluating them (velocity Verlet carries the forces of the current state
 * from one step to the next, SI "Equations of motion").  For restarting from
 * a saved state: bpm_set_state, then bpm_set_forces with the forces that
 * bpm_get_forces returned for that state.  Bond-damping measures and contact
 * histories are not restored.  On a handle whose dipole plan is not yet
 * fixed, the call first evaluates the forces once (which fixes it).
 * Errors: BPM_ERR_ARG (NULL pointer), BPM_ERR_CUDA. */
int bpm_set_forces(bpm_handle* h, const double* f, const double* tau);

/* Copies out the stored forces and torques of the current state ([3N] each,
 * AoS, host or device; either may be NULL) without evaluating them.
 * Errors: BPM_ERR_ARG (no stored forces: none evaluated since the state was
 * last replaced), BPM_ERR_CUDA. */
int bpm_get_forces(bpm_handle* h, double* f, double* tau);

/* Replaces the uniform part of the external field: B[3] (host, or NULL =
 * unchanged) and, when B_rod is not NULL, the per-rod fields [3R] (host).
 * Invalidates the stored forces.  Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_set_field(bpm_handle* h, const double* B, const double* B_rod);

/* Replaces the body-frame dipoles m~ ([3N], host or device).  Invalidates
 * the stored forces.  Errors: BPM_ERR_ARG, BPM_ERR_CUDA. */
int bpm_set_dipoles(bpm_handle* h, const double* m_body);

/* Work decomposition of the dipole pass.  kind 0: chosen by the library's
 * autotuner at the first force evaluation (default); kind 1: ordered-pair
 * kernel, each i against all j, with the j range split in `param` chunks
 * (global mode) or chunks of `param` particles (per-rod mode); kind 2:
 * symmetric kernel (each unordered pair once, Newton's third law) over pairs
 * of supertiles of `param` tiles (param in 1..8), or, with param 0, over
 * pairs of warp tiles with one warp each (32 particles per tile on BPM_FP64
 * and BPM_FF handles, 64 on BPM_MIXED ones; for systems too small to fill
 * the GPU otherwise and for many short rods; one partial sum per particle
 * and partner tile, at most 2 GB).  Takes
 * effect at the next force evaluation.  Results of different plans agree to
 * rounding.  The adjoint follows the plan kind: kind 1 makes its dipole
 * VJP ordered (j-chunks), otherwise it is symmetric where it can be (see
 * bpm_adjoint_begin).
 * Errors: BPM_ERR_ARG (unknown kind, bad param, or a plan needing more than
 * 255 partial slots per particle). */
#define BPM_PLAN_AUTO 0
#define BPM_PLAN_ORDERED 1
#define BPM_PLAN_SYMMETRIC 2
int bpm_set_dipole_plan(bpm_handle* h, int32_t kind, int32_t param);

/* The plan in use: *kind = BPM_PLAN_ORDERED or BPM_PLAN_SYMMETRIC and its
 * param once the first force evaluation has fixed it, BPM_PLAN_AUTO before.
 * Errors: BPM_ERR_ARG. */
int bpm_get_dipole_plan(bpm_handle* h, int32_t* kind, int32_t* param);

/* Concurrency of the bond and dipole kernels within a force evaluation.
 * The bond kernel is bound by the FP64 pipe and the FP32-pair dipole kernels
 * by the FP32 pipe, so they can share the SMs: m = q m~ q* is then computed
 * first by its own kernel, the dipole kernel runs on the handle's stream
 * with one block per SM fewer than its occupancy, and the bond kernel on a
 * second stream owned by the handle with a few blocks per SM that loop over
 * the particles, so that both stay resident; the streams are joined before
 * the finish kernel.
 * The arithmetic is unchanged, so forces and trajectories are bitwise those
 * of the sequential form.  mode -1 (default): the autotuner times the
 * sequential and concurrent forms on BPM_MIXED and BPM_FF handles with the
 * automatic plan, and keeps the faster; 0: always sequential; 1: concurrent
 * whenever the handle allows it.  Handles with contact or a fluid, and
 * energy evaluations, always run sequentially.  Takes effect at the next
 * force evaluation.  Errors: BPM_ERR_ARG (mode outside -1..1). */
int bpm_set_overlap(bpm_handle* h, int32_t mode);

/* The form in use after the first force evaluation: *on = 1 with the dipole
 * and bond kernels' grids (blocks) in *dipole_blocks and *bond_blocks when
 * the kernels run concurrently, else all three 0.  Errors: BPM_ERR_ARG. */
int bpm_get_overlap(bpm_handle* h, int32_t* on, int32_t* dipole_blocks, int32_t* bond_blocks);

/* Adjoint of the time stepping (the differentiation pattern used for
 * magnetisation-profile design).  bpm_adjoint_begin records the current
 * state, advances n_steps velocity-Verlet steps exactly as bpm_step would
 * and keeps a checkpoint every `checkpoint_every` steps in device memory
 * owned by the handle.  bpm_adjoint_end then returns the gradient of a loss
 * L(x(T)) of the final positions: given dL_dx = dL/dx(T) ([3N], host or
 * device), it writes dL/dm~ ([3N], body-frame dipoles, host or device, may
 * be NULL) and dL/dB ([3], uniform part of the field, host, may be NULL).
 * The reverse sweep recomputes each segment from its checkpoint (the kernels
 * are deterministic, so the recomputed states equal the recorded ones) and
 * applies hand-written vector-Jacobian products of the integrator (SI
 * "Equations of motion"), the bond forces (main text Eqs. bpm-fr ..
 * bpm-vector, differentiated as implemented; the paper notes they are not
 * gradients of its energy), the Zeeman and dipole-dipole terms (Methods,
 * "Magnetic interactions") and the damping.  BPM_FP64 and BPM_FF handles
 * (a BPM_FF handle records its trajectory with float-float dipole pairs and
 * evaluates the symmetric dipole VJP in float-float too; the gradient is
 * that of its own time stepping).  The
 * dipole VJP evaluates each unordered pair once (both of its sides) when the
 * dipoles form one interacting set (global mode, or one rod) and its
 * per-tile partial sums (48 N ceil(N/32) bytes) fit in 512 MB, unless the
 * ordered dipole plan was forced; otherwise it runs over ordered pairs.
 * The forces of the starting state are evaluated from that state (damping
 * with its own velocities), as on a fresh handle.
 * bpm_set_dipoles / bpm_set_field between begin and end discard the record.
 * Errors: BPM_ERR_ARG (bad arguments, BPM_MIXED handle, a handle with bond
 * damping, contact or a fluid, no record), BPM_ERR_NONFINITE, BPM_ERR_CUDA. */
int bpm_adjoint_begin(bpm_handle* h, int32_t n_steps, int32_t checkpoint_every);
int bpm_adjoint_end(bpm_handle* h, const double* dL_dx, double* grad_m_body, double* grad_B);

/* Density and velocity of the fluid's current state (after streaming,
 * rho u = sum f e + body_force / 2): rho[nodes] and u[3 nodes] (AoS), host
 * or device pointers, either may be NULL.
 * Errors: BPM_ERR_ARG (no fluid), BPM_ERR_CUDA. */
int bpm_lbm_fields(bpm_handle* h, double* rho, double* u);

/* Per-kernel timing.  When enabled, bpm_step and bpm_forces launch without
 * CUDA graphs and bracket every kernel with CUDA events on the handle's
 * stream.  bpm_get_timing fills, for kinds k = 0 bond, 1 dipole,
 * 2 integrate (reduce, update, fluid interpolation and penalty), 3 contact
 * (cell list + pairs), 4 LBM step, out[3k] = launches, out[3k+1] = total
 * milliseconds, out[3k+2] = work units (bonds, ordered pairs, particles,
 * particles, lattice nodes)
 * since the last reset; bpm_set_timing(h, 1) resets the counters.  The
 * events are read (with a stream synchronisation) by bpm_get_timing, so
 * timing adds no host round trip to bpm_step and bpm_forces. */
int bpm_set_timing(bpm_handle* h, int32_t enable);
int bpm_get_timing(bpm_handle* h, double out[15]);

/* Message of the last failure on this handle (or, when h is NULL, of the
 * last failed call made without a handle: bpm_create or
 * bpm_dipole_forces_noalloc).  The string lives until the next call. */
const char* bpm_last_error(const bpm_handle* h);

/* Dipole-dipole forces and torques of n free dipoles, for callers that cannot
 * allocate device memory.  The paper has no counterpart: it is a packaging of
 * the library's FP64 all-pairs dipole kernel (every ordered pair i != j, no
 * cutoff, prefactor mu0_over_4pi) for applications that must not call
 * cudaMalloc -- for example a host whose caching allocator has already
 * reserved the device memory, or a fixed-latency control loop in which
 * cudaMalloc's possible device synchronisation is not acceptable.
 *
 * Inputs x[3n] (positions) and m[3n] (space-frame dipoles) and outputs
 * f[3n], tau[3n] are DEVICE pointers of the current device (or managed
 * memory), AoS per particle, each holding at least 3n doubles; f and tau are
 * overwritten.  Before launching, the call rejects with BPM_ERR_ARG any of
 * them that cudaPointerGetAttributes does not report as device memory of the
 * current device or managed memory, and any whose allocation (as the driver
 * reports it) ends before 3n doubles.  Work is issued on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * waiting for it.
 *
 * It allocates nothing: its scratch is a fixed 7.3 MB array inside the
 * library's device image, which every GPU that loads the library holds until
 * the process exits.  n may be at most 32768; larger n is rejected with
 * BPM_ERR_ARG before anything is launched.  The first call on a device looks
 * up that array's device address (with the device current) and caches it
 * with the id of the current context; a later call under another context
 * (after cudaDeviceReset, for instance) looks it up again.  Make the first
 * call on each device, and the first after a reset, before any stream
 * capture.  All calls share the one array: calls whose work overlaps on the
 * GPU (other streams, other threads) race and give wrong results, so
 * serialise them.  Each call overwrites every part of the array that it
 * reads, so nothing needs clearing between calls.
 * Errors: BPM_ERR_ARG, BPM_ERR_CUDA (message via bpm_last_error(NULL)). */
int bpm_dipole_forces_noalloc(int64_t n, const double* x, const double* m, double mu0_over_4pi,
                              double* f, double* tau, void* stream);

/* Throughput probe of the arithmetic pipes that bound the library's kernels
 * (the paper has no counterpart; the results are the denominators of the
 * roofline fractions reported for ALU-bound kernels).  On the current device
 * it runs, for about 50 ms each, eight independent chains per thread of one
 * operation on fully occupied SMs: op 0 FP64 fma, op 1 FP32 fma, op 2 the
 * packed two-lane FP32 fma (each counted as two lane operations), op 3 the
 * FP32 reciprocal square root of the special-function unit, op 4 FP64 add.
 * out[4 op + 0] =
 * lane operations per SM per clock, [4 op + 1] = lane operations per second,
 * [4 op + 2] = SM clock of the run in MHz (cycle counter over global timer),
 * [4 op + 3] = kernel time in ms.  Allocates a few MB of device memory for
 * the run.  Errors: BPM_ERR_ARG (out is NULL), BPM_ERR_CUDA (message via
 * bpm_last_error(NULL)). */
int bpm_measure_pipes(double out[20]);

/* Library version string. */
const char* bpm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BPM_H */
