/*
 * CPU FP64 oracle for the bonded-particle magneto-elastic rod model
 * (Alkuino, Clemmer, Santangelo, Zhang, arXiv 2603.27279).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, scalar C in double precision that
 * restates the paper's steps in the paper's order and notation.  It shares no
 * source with the CUDA library (paper_2603_27279_gb300/csrc) and neither side
 * includes or links the other.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it.
 *
 * Layouts (AoS per particle): x[3N], q[4N] as (w,x,y,z) with v_space =
 * q v_body q*, v[3N], w[3N] (angular velocity, space frame), f[3N], tau[3N].
 * Rods are CSR (rod_offset[n_rods+1]); a bond joins consecutive particles of
 * a rod, particle "1" = k and particle "2" = k+1 of the paper's Fig. 2.
 *
 * Readings of the paper taken where it is silent or singular are listed in
 * the file header of bpm_oracle.c.
 */
#ifndef BPM_ORACLE_H
#define BPM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Hertz-Mindlin contact between non-bonded particles (Methods, "Contact";
 * reading R11).  The history of the tangential displacement xi is kept per
 * particle and contact partner, in two levels like the bond measures. */
typedef struct orc_contact {
    double E, nu;               /* particle Young's modulus and Poisson ratio */
    double mu;                  /* Coulomb friction coefficient */
    double gamma_n, gamma_t;    /* viscous damping of the normal and tangential
                                   relative velocity at the contact point */
    int exclude;                /* same-rod pairs with |i - j| <= exclude are skipped */
    int cap;                    /* capacity of each particle's history list */
    int level;                  /* index (0/1) of the current level */
    int valid[2];               /* 1 when the level holds a record */
    int* count;                 /* [2][N] contacts recorded per particle */
    int64_t* partner;           /* [2][N][cap] */
    double* xi;                 /* [2][N][cap][3] tangential displacement of i w.r.t. partner */
    int overflow;               /* set when a particle had more than cap contacts */
} orc_contact;

/* Lattice Boltzmann fluid (D3Q19, BGK, Guo forcing) on a periodic lattice
 * with penalty immersed-boundary coupling and sub-cycling (Methods,
 * "Lattice Boltzmann method", "Immersed boundary coupling"; reading R12).
 * Lattice units: spacing 1, LBM step 1 = n_sub DEM steps, density scale 1.
 * The stored state is the post-collision distributions. */
typedef struct orc_lbm {
    int nx, ny, nz;             /* nodes per axis; node (i,j,k) sits at (i,j,k) */
    int n_sub;                  /* DEM steps per LBM step */
    double tau;                 /* BGK relaxation time */
    double body_force[3];       /* uniform force density on the fluid */
    double* f;                  /* [19][nodes] post-collision distributions */
    double* f_tmp;              /* [19][nodes] scratch of the same size */
    double* F;                  /* [3][nodes] particle reaction force for the next LBM step */
    double* U;                  /* [3N] fluid velocity interpolated at the particles */
    const uint8_t* coupled;     /* [N] 1 = exchanges momentum with the fluid; NULL = all */
    int phase;                  /* DEM steps done in the current LBM cycle */
    int64_t steps;              /* LBM steps done */
} orc_lbm;

typedef struct orc_system {
    int64_t n;                  /* particles */
    int64_t n_rods;
    const int64_t* rod_offset;  /* [n_rods+1] */
    /* per-bond rest data, filled by orc_init_bonds (caller allocates n-n_rods) */
    int64_t n_bonds;
    int64_t* bond_p1;           /* particle "1" */
    int64_t* bond_p2;           /* particle "2" */
    double* bond_ri;            /* [3 per bond] rest bond vector r_i (rest-relative frame) */
    double* bond_K;             /* [4 per bond] K_r, K_s, K_t, K_b */
    /* particles */
    const double* q_rest;       /* [4N] rest orientations q^i */
    const double* mass;         /* [N] */
    const double* radius;       /* [N] */
    const double* m_body;       /* [3N] dipole in the body frame */
    const uint8_t* clamped;     /* [N] 1 = excluded from integration */
    /* field: B(x,t) = B + B_rod[rod] + amp (cos(wt) e1 + sin(wt) e2) + G (x - x0) */
    double B[3];
    const double* B_rod;        /* [3 n_rods] or NULL */
    double Brot_amp, Brot_omega;
    double Brot_e1[3], Brot_e2[3];
    double gradB[9];            /* row-major dB_a/dx_b */
    double gradB_x0[3];
    double c;                   /* mu0 / (4 pi) */
    int dipole_mode;            /* 0 off, 1 all pairs, 2 pairs within a rod */
    int n_threads;              /* OpenMP threads for the dipole loop (<=0: default) */
    double damping;             /* global viscous damping coefficient */
    double dt;
    /* bond-level damping per mode (Methods, "Damping"; reading R10) */
    const double* bond_g;       /* [4 per bond] g_r, g_s, g_t, g_b, or NULL (none) */
    double* bond_hist;          /* [6 per bond] gamma, psi, theta of the previous
                                   and of the current level; NaN = none.
                                   Written by every force evaluation. */
    orc_contact* contact;       /* NULL: no contact forces */
    orc_lbm* lbm;               /* NULL: no fluid */
} orc_system;

/* D3Q19 velocities e[19][3] and weights w[19] of the oracle */
void orc_lbm_lattice(int e[57], double w[19]);
/* Peskin's four-point regularised delta, one dimension, lattice units */
double orc_ibm_phi(double r);
/* f = equilibrium of (rho, u) at every node: rho[nodes] (NULL: 1),
 * u[3 nodes] AoS (NULL: 0); F = 0, phase = steps = 0 */
void orc_lbm_init(orc_lbm* L, const double* rho, const double* u);
/* density and velocity (AoS) of the current state: after streaming,
 * rho u = sum f e + body_force / 2 */
void orc_lbm_macro(const orc_lbm* L, double* rho, double* u);
/* one LBM step: stream, collide with Guo forcing of body_force + F; F = 0 */
int orc_lbm_step(orc_lbm* L);
/* U[3N] = fluid velocity of the current state at positions x[3N] */
void orc_lbm_interp(const orc_lbm* L, const double* x, int64_t n, double* U);

/* Contact forces and torques (R11) on the particles idx[k] from all other
 * particles, as a fresh state has them (no recorded histories), for checks
 * and timings on sampled particles of large systems.  OpenMP over k. */
int orc_contact_sample(const orc_system* s, const double* x, const double* v, const double* w,
                       const int64_t* idx, int64_t k, double* f, double* tau);

/* One contact pair (reading R11): x, v, w of particles i and j, radii, the
 * tangential displacement xi_old of i w.r.t. j (NULL: new contact), dt.
 * Returns 0 when the particles do not overlap (outputs untouched), else 1
 * with the force on i (f_j = -f_i), the torques on i and j and the updated
 * xi of i w.r.t. j. */
int orc_contact_pair(const orc_contact* c, const double xi_[3], const double xj[3], const double vi[3],
                     const double vj[3], const double wi[3], const double wj[3], double Ri, double Rj,
                     const double* xi_old, double dt, double f_i[3], double tau_i[3], double tau_j[3],
                     double xi_new[3]);

/* Fills bond_p1/p2/ri/K from the rest configuration and per-rod material
 * (E, nu, d).  Returns 0, or -1 on a zero-length rest bond / bad argument. */
int orc_init_bonds(orc_system* s, const double* x_rest, const double* E,
                   const double* nu, const double* d);

/* One bond (main text Eqs. bpm-fr .. bpm-vector).  q1, q2 are orientations
 * relative to the rest state (q_alpha q_alpha^{i*}); ri is the rest bond
 * vector.  Outputs f1, tau1, f2, tau2 (space frame), the energy estimate of
 * Eq. total-energy in *U, and diag[8] = {gamma, psi, theta_b_x, theta_b_y,
 * theta_b_z (in C'), r_f, branch_of_m, 0} for tests (diag may be NULL).
 * m_branch: -1 automatic (paper's form for z >= 0, flipped gauge for z < 0),
 * 0 force the paper's form, 1 force the flipped gauge. */
void orc_bond(const double x1[3], const double x2[3], const double q1[4], const double q2[4],
              const double ri[3], const double K[4], int m_branch,
              double f1[3], double tau1[3], double f2[3], double tau2[3],
              double* U, double* diag);

/* The same bond with damping per mode (Methods, "Damping"): g = {g_r, g_s,
 * g_t, g_b}; v1, v2 the particle velocities (radial term g_r (dv . r^_f));
 * prev = {gamma, psi, theta} of the previous force evaluation or NULL (zero
 * rates); dt the step of the finite-difference rates.  meas (may be NULL)
 * receives this evaluation's {gamma, psi, theta}. */
void orc_bond_damped(const double x1[3], const double x2[3], const double q1[4], const double q2[4],
                     const double ri[3], const double K[4], const double g[4], const double v1[3],
                     const double v2[3], const double prev[3], double dt,
                     double f1[3], double tau1[3], double f2[3], double tau2[3], double* U,
                     double meas[3]);

/* Total force/torque at time t on every particle: bonds (with bond damping
 * when bond_g is set: a stand-alone evaluation in the sense of R10), Zeeman,
 * dipole, global damping.  m_out[3N] (may be NULL)
 * receives the space-frame dipoles.
 * energy[5] (may be NULL) = {bond, zeeman, dipole, kinetic_trans, kinetic_rot}. */
int orc_forces(const orc_system* s, const double* x, const double* q, const double* v,
               const double* w, double t, double* f, double* tau, double* m_out,
               double* energy);

/* Dipole-dipole force and torque on the listed particles only (all partners),
 * given space-frame dipoles m[3N]; H[3*n_idx] (may be NULL) receives the
 * summed dipole field at x_i (without the mu0/4pi factor applied twice). */
int orc_dipole_sample(const orc_system* s, const double* x, const double* m,
                      const int64_t* idx, int64_t n_idx, double* F, double* tau, double* H);

/* Condition scale of each listed particle's force and torque (the
 * denominator of the per-particle error |dF_i| / sum_j |F_ij|): the sum of
 * the magnitudes of every term that the total force (torque) of particle
 * idx[k] adds up -- each elastic bond force (torque) at that end, the Zeeman
 * force G^T m, each dipole pair force F_ij and the global damping force g v
 * (torque g omega).  The magnetic torque m_i x B(x_i) is the cross product
 * of a summed field, so its terms are counted as |m_i| |B| for the external
 * field and |m_i| |B_j(x_i)| for each dipole's field.  Bond
 * damping, contact and fluid terms are not included.  sf[n_idx], st[n_idx].
 * Returns 0, or -1 on allocation failure. */
int orc_term_scales(const orc_system* s, const double* x, const double* q, const double* v,
                    const double* w, double t, const int64_t* idx, int64_t n_idx, double* sf,
                    double* st);

/* n_steps velocity-Verlet steps (SI "Equations of motion") from state
 * (x,q,v,w) at *t.  f/tau hold the forces at *t if forces_valid, else they
 * are computed first.  On return the state, *t, f and tau are at the end.
 * The force evaluations after each step shift the bond-damping history (R10).
 * With a fluid (R12): the velocity is interpolated at the start of each LBM
 * cycle (after the drift of the cycle's first step), every step's force
 * evaluation spreads the particles' reaction forces, and an LBM step follows
 * every n_sub steps. */
int orc_run(const orc_system* s, double* x, double* q, double* v, double* w, double* t,
            int n_steps, double* f, double* tau, int forces_valid);

/* Helpers exposed for tests. */
void orc_quat_mul(const double a[4], const double b[4], double out[4]);
void orc_rotate(const double q[4], const double v[3], double out[3]);
void orc_richardson(const double q[4], const double w[3], double dt, double out[4]);
/* m of reading R4 for a vector r (branch -1 automatic, 0 or 1 forced). */
void orc_align_z(const double r[3], int branch, double m[4]);

#ifdef __cplusplus
}
#endif
#endif
