/*
 * CPU FP64 oracle for the bonded-particle magneto-elastic rod model
 * (arXiv 2603.27279).  TEST INFRASTRUCTURE ONLY: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg load this library.
 * It shares no code with the CUDA path.
 *
 * Every function follows the paper's steps in the paper's order:
 *   - bond model: main text, "Bonded-particle model for elastic rods"
 *     (Eqs. bpm-fr, bpm-fst, bpm-tst, bpm-tb, bpm-tt, bpm-vector, total-energy)
 *     and SI "Symmetric rotational decomposition" (Eq. S-quat-h, the u / t / b
 *     construction);
 *   - spring constants: main text after Eq. bpm-vector and SI "Deriving the
 *     spring constants";
 *   - Zeeman and dipole-dipole: Methods, "Magnetic interactions";
 *   - dipole kinematics: main text, "Magnetized beams" (m = R m~);
 *   - integration: SI "Equations of motion" (velocity Verlet, Richardson
 *     quaternion update, renormalisation after every substep);
 *   - damping: Methods, "Damping" (global viscous damping).
 *
 * Readings where the paper is silent, singular or leaves a choice:
 *   R1 rest orientations: the paper sets q^i = 1 without loss of generality;
 *      for general rest orientations each end uses its rotation since rest,
 *      q'_a = q_a q_a^{i*}, and r_i = x_2^i - x_1^i in the global frame.
 *   R2 central frame: q_C is the slerp midpoint on the shorter arc, computed
 *      as the normalised sum q_1 + s q_2 with s = sign(q_1 . q_2) (s = +1 at
 *      0); u^0 = q_C^* (s q_2).
 *   R3 shear angle: gamma = atan2(|r^_i x r^_f|, r^_i . r^_f) (same value as
 *      the paper's arccos, accurate at small angles); gamma t^ = (gamma/|c|) c
 *      with the limit 1/(r^_i . r^_f) at |c| = 0.
 *   R4 m quaternion: (r+z, -y, x, 0)/sqrt(2r(r+z)) for z >= 0, the paper's
 *      Eq. S-quat-h in a form free of 0/0; for z < 0 the rotation
 *      (-y, r-z, 0, x)/sqrt(2r(r-z)), which also takes z onto r_f[C] (it
 *      differs from the paper's m by a rotation about z, which leaves every
 *      force and torque unchanged) and stays regular at r_f[C] = -z.
 *   R5 swing-twist: u = t_2 b_2 with t_2 = normalise(u_w, 0, 0, u_z),
 *      b_2 = t_2^* u; u^* = t_1 b_1 likewise; psi_a = 2 atan2(t_a,z, t_a,w);
 *      b = b_2 b_1^*, theta b^ its full axis-angle vector (w >= 0 branch).
 *   R6 r_f = |x_2 - x_1| is taken in the global frame (rotation-invariant).
 *   R7 omega is the space-frame angular velocity, q' = 1/2 (0, omega) q.
 *   R8 global damping: f -= g v and tau -= g omega with the half-step
 *      velocities present at force time.
 *   R9 clamped particles: no update of x, q, v, omega.
 *   R10 bond damping (Methods, "Damping"): the radial term uses the relative
 *      velocity v_2 - v_1 (the velocities present at force time) projected on
 *      r^_f.  The rates of gamma, psi, theta are backward differences over dt
 *      against recorded measures; each bond keeps two levels, the measures of
 *      the state before the current one and those of the current state (NaN:
 *      none recorded).  The force evaluation of a time step, at a new state,
 *      differences against the current level and then shifts the levels; a
 *      stand-alone evaluation of the current state differences against the
 *      previous level (so it reproduces the forces the last step ended with)
 *      and only fills in an empty current level.  Rates are zero when the
 *      level differenced against is empty.  Each damping term acts along its
 *      elastic direction (s^ and t^ for shear, z of C' for twist, b^ for
 *      bend); the shear and bend terms vanish at exactly zero angle.
 *   R11 contact (Methods, "Contact": Hertz-Mindlin between non-bonded
 *      particles; the paper gives no formulas, so the textbook forms are
 *      used).  Pairs of the same rod within `exclude` bonds are skipped.
 *      With d = x_i - x_j, n = d/|d|, overlap delta = R_i + R_j - |d| > 0,
 *      R* = R_i R_j/(R_i + R_j), E* = E/(2(1 - nu^2)), G* = G/(2(2 - nu)),
 *      G = E/(2(1 + nu)) and contact radius a = sqrt(R* delta):
 *      normal force on i  (4/3 E* a delta - gamma_n v_n) n  (Hertz);
 *      relative velocity of the contact points
 *      v_rel = v_i - v_j - (R_i w_i + R_j w_j) x n, v_n = v_rel . n,
 *      v_t = v_rel - v_n n;
 *      tangential displacement xi = rot(xi_old) + v_t dt, where rot removes
 *      the normal component of xi_old and restores its length (xi_old = 0
 *      for a new contact); tangential force F_t = -8 G* a xi - gamma_t v_t
 *      (Mindlin's stiffness), limited to mu times the Hertz force
 *      4/3 E* a delta, in which case xi = -(F_t + gamma_t v_t)/(8 G* a);
 *      torques (-R_i n) x F_t on i and (-R_j n) x F_t on j; f_j = -f_i.
 *      The tangential displacements are recorded per particle and partner in
 *      two levels, with the same step / stand-alone rule as R10.
 *   R12 fluid coupling (Methods, "Lattice Boltzmann method", "Immersed
 *      boundary coupling"): a periodic D3Q19 lattice in lattice units
 *      (spacing 1, LBM step 1 = n_sub DEM steps, density scale 1); BGK
 *      collision with the second-order equilibrium and Guo's source, the
 *      velocity in both taken at the half step, rho u = sum f e + F/2;
 *      Peskin's four-point delta as the regularised delta; the fluid
 *      velocity is interpolated once per cycle, at the positions of the
 *      cycle's first force evaluation, from the streamed distributions with
 *      the body-force half step; the penalty force F_p = m_p (U - v_p) (kappa
 *      = m_p / dt_LBM) enters every force evaluation with the velocity
 *      present at force time; each step's force evaluation spreads -F_p /
 *      n_sub with the delta weights (Delta V_p = Delta x^3, so the spread
 *      force sums to -F_p / n_sub); stand-alone evaluations do not spread.
 */
#include "bpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* quaternions (w, x, y, z), Hamilton product                          */
/* ------------------------------------------------------------------ */
typedef struct { double w, x, y, z; } quat;
typedef struct { double x, y, z; } vec3;

static quat qmake(double w, double x, double y, double z) { quat q = {w, x, y, z}; return q; }
static quat qload(const double* p) { return qmake(p[0], p[1], p[2], p[3]); }
static void qstore(quat q, double* p) { p[0] = q.w; p[1] = q.x; p[2] = q.y; p[3] = q.z; }
static vec3 vmake(double x, double y, double z) { vec3 v = {x, y, z}; return v; }
static vec3 vload(const double* p) { return vmake(p[0], p[1], p[2]); }
static void vstore(vec3 v, double* p) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }

static quat qmul(quat a, quat b) {
    return qmake(a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
                 a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
                 a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
                 a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w);
}
static quat qconj(quat a) { return qmake(a.w, -a.x, -a.y, -a.z); }
static quat qscale(quat a, double s) { return qmake(s * a.w, s * a.x, s * a.y, s * a.z); }
static quat qadd(quat a, quat b) { return qmake(a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z); }
static double qdot(quat a, quat b) { return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z; }
static quat qnormalize(quat a) { return qscale(a, 1.0 / sqrt(qdot(a, a))); }

static vec3 vadd(vec3 a, vec3 b) { return vmake(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vsub(vec3 a, vec3 b) { return vmake(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vscale(vec3 a, double s) { return vmake(s * a.x, s * a.y, s * a.z); }
static double vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double vnorm(vec3 a) { return sqrt(vdot(a, a)); }
static vec3 vcross(vec3 a, vec3 b) {
    return vmake(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

/* v expressed in O when given in the frame q: q v q* (SI Fig. S-frames, property 2) */
static vec3 rot(quat q, vec3 v) {
    quat r = qmul(qmul(q, qmake(0.0, v.x, v.y, v.z)), qconj(q));
    return vmake(r.x, r.y, r.z);
}
/* v given in O expressed in the frame q: q* v q */
static vec3 rot_inv(quat q, vec3 v) {
    quat r = qmul(qmul(qconj(q), qmake(0.0, v.x, v.y, v.z)), q);
    return vmake(r.x, r.y, r.z);
}

void orc_quat_mul(const double a[4], const double b[4], double out[4]) {
    qstore(qmul(qload(a), qload(b)), out);
}
void orc_rotate(const double q[4], const double v[3], double out[3]) {
    vstore(rot(qload(q), vload(v)), out);
}

/* ------------------------------------------------------------------ */
/* spring constants (main text; SI "Deriving the spring constants")    */
/* ------------------------------------------------------------------ */
int orc_init_bonds(orc_system* s, const double* x_rest, const double* E, const double* nu,
                   const double* d) {
    if (!s || !x_rest || !E || !nu || !d) return -1;
    int64_t b = 0;
    for (int64_t r = 0; r < s->n_rods; ++r) {
        double G = E[r] / (2.0 * (1.0 + nu[r]));
        double A = M_PI * d[r] * d[r] / 4.0;
        double I = M_PI * pow(d[r], 4) / 64.0;
        double J = M_PI * pow(d[r], 4) / 32.0;
        for (int64_t k = s->rod_offset[r]; k + 1 < s->rod_offset[r + 1]; ++k) {
            vec3 ri = vsub(vload(x_rest + 3 * (k + 1)), vload(x_rest + 3 * k));
            double L = vnorm(ri);
            if (!(L > 0.0)) return -1;
            s->bond_p1[b] = k;
            s->bond_p2[b] = k + 1;
            vstore(ri, s->bond_ri + 3 * b);
            s->bond_K[4 * b + 0] = E[r] * A / L;               /* K_r = EA/L   */
            s->bond_K[4 * b + 1] = 12.0 * E[r] * I / (L * L * L); /* K_s = 12EI/L^3 */
            s->bond_K[4 * b + 2] = G * J / L;                  /* K_t = GJ/L   */
            s->bond_K[4 * b + 3] = E[r] * I / L;               /* K_b = EI/L   */
            ++b;
        }
    }
    s->n_bonds = b;
    return 0;
}

/* ------------------------------------------------------------------ */
/* one bond                                                            */
/* ------------------------------------------------------------------ */
static quat align_z(vec3 rf, double r, int branch) {
    /* R4: rotation m in C taking z onto r_f[C] / r */
    double x = rf.x, y = rf.y, z = rf.z;
    if (branch < 0) branch = (z >= 0.0) ? 0 : 1;
    if (branch == 0) {
        double n = sqrt(2.0 * r * (r + z));
        return qmake((r + z) / n, -y / n, x / n, 0.0);
    }
    double n = sqrt(2.0 * r * (r - z));
    return qmake(-y / n, (r - z) / n, 0.0, x / n);
}

void orc_align_z(const double r[3], int branch, double m[4]) {
    vec3 v = vload(r);
    qstore(align_z(v, vnorm(v), branch), m);
}

static void bond_impl(const double x1[3], const double x2[3], const double q1[4], const double q2[4],
                      const double ri_[3], const double K[4], int m_branch, const double* g,
                      const double* v1, const double* v2, const double* prev, double dt,
                      double f1[3], double tau1[3], double f2[3], double tau2[3], double* U,
                      double* diag, double* meas) {
    const double Kr = K[0], Ks = K[1], Kt = K[2], Kb = K[3];
    quat Q1 = qload(q1), Q2 = qload(q2);

    /* central frame C: slerp midpoint of q_1, q_2 (R2) */
    if (qdot(Q1, Q2) < 0.0) Q2 = qscale(Q2, -1.0);
    quat qC = qnormalize(qadd(Q1, Q2));

    /* current bond vector measured in C: r_f[C] = q_C^* r_f[O] q_C */
    vec3 rfO = vsub(vload(x2), vload(x1));
    vec3 rf = rot_inv(qC, rfO);
    vec3 ri = vload(ri_);
    double rf_len = vnorm(rfO); /* R6 */
    double ri_len = vnorm(ri);
    vec3 rfh = vscale(rf, 1.0 / rf_len);
    vec3 rih = vscale(ri, 1.0 / ri_len);

    /* radial force on particle 1 (Eq. bpm-fr) */
    vec3 fr = vscale(rfh, Kr * (rf_len - ri_len));

    /* shear force and counter torque (Eqs. bpm-fst, bpm-tst; R3) */
    vec3 c = vcross(rih, rfh);
    double sin_g = vnorm(c), cos_g = vdot(rih, rfh);
    double gamma = atan2(sin_g, cos_g);
    double g_over_s = (sin_g > 0.0) ? gamma / sin_g : 1.0 / cos_g;
    vec3 gamma_t = vscale(c, g_over_s);                      /* gamma t^            */
    vec3 gamma_s = vcross(gamma_t, rfh);                     /* gamma s^ = gamma t^ x r^_f */
    vec3 fs = vscale(gamma_s, Ks * rf_len);                  /* K_s r_f gamma s^    */
    vec3 ts = vscale(gamma_t, 0.5 * Ks * rf_len * rf_len);   /* 1/2 K_s r_f^2 gamma t^ */

    /* C' frame: m takes the z axis of C onto r_f[C] (Eq. S-quat-h; R4) */
    double rf_len_C = vnorm(rf);
    if (m_branch < 0) m_branch = (rf.z >= 0.0) ? 0 : 1;
    quat m = align_z(rf, rf_len_C, m_branch);

    /* half rotation u^0 = q_C^* q_2 = q_1^* q_C, and u = m^* u^0 m in C' */
    quat u0 = qmul(qconj(qC), Q2);
    quat u = qmul(qmul(qconj(m), u0), m);

    /* bend before twist: u = t_2 b_2, u^* = t_1 b_1 (R5) */
    quat t2 = qnormalize(qmake(u.w, 0.0, 0.0, u.z));
    quat b2 = qmul(qconj(t2), u);
    quat uc = qconj(u);
    quat t1 = qnormalize(qmake(uc.w, 0.0, 0.0, uc.z));
    quat b1 = qmul(qconj(t1), uc);
    double psi2 = 2.0 * atan2(t2.z, t2.w);
    double psi1 = 2.0 * atan2(t1.z, t1.w);
    double psi = psi2 - psi1;

    /* effective bending b = b_2 b_1^*, its axis-angle vector theta b^ */
    quat b = qmul(b2, qconj(b1));
    if (b.w < 0.0) b = qscale(b, -1.0);
    vec3 bv = vmake(b.x, b.y, b.z);
    double sin_half = vnorm(bv);
    double theta = 2.0 * atan2(sin_half, b.w);
    double th_over_s = (sin_half > 0.0) ? theta / sin_half : 2.0 / b.w;
    vec3 theta_b = vscale(bv, th_over_s);

    /* bending and twisting torques on particle 1 in C' (Eqs. bpm-tb, bpm-tt) */
    vec3 tb = vscale(theta_b, Kb);
    vec3 tt = vmake(0.0, 0.0, Kt * psi);

    /* bond damping per mode (Methods, "Damping"): radial term on the relative
     * velocity along the bond; shear, twist and bend terms on finite-difference
     * rates of the stored measures, added along the elastic directions */
    if (g) {
        vec3 dv = rot_inv(qC, vsub(vload(v2), vload(v1)));
        fr = vadd(fr, vscale(rfh, g[0] * vdot(dv, rfh)));
        if (prev) {
            double gdot = (gamma - prev[0]) / dt;
            double pdot = (psi - prev[1]) / dt;
            double tdot = (theta - prev[2]) / dt;
            if (gamma > 0.0) {
                vec3 t_hat = vscale(gamma_t, 1.0 / gamma);
                fs = vadd(fs, vscale(vcross(t_hat, rfh), g[1] * rf_len * gdot));
                ts = vadd(ts, vscale(t_hat, 0.5 * g[1] * rf_len * rf_len * gdot));
            }
            tt = vadd(tt, vmake(0.0, 0.0, g[2] * pdot));
            if (theta > 0.0) tb = vadd(tb, vscale(theta_b, g[3] * tdot / theta));
        }
    }
    if (meas) {
        meas[0] = gamma;
        meas[1] = psi;
        meas[2] = theta;
    }

    /* back to O: v[O] = q_C v[C] q_C^*, v[O] = q_C m v[C'] m^* q_C^* */
    quat qCm = qmul(qC, m);
    vec3 F = rot(qC, vadd(fr, fs));
    vec3 TS = rot(qC, ts);
    vec3 TBT = rot(qCm, vadd(tb, tt));

    /* superposition (Eq. bpm-vector) */
    vstore(F, f1);
    vstore(vadd(TS, TBT), tau1);
    vstore(vscale(F, -1.0), f2);
    vstore(vsub(TS, TBT), tau2);

    if (U) {
        /* Eq. total-energy */
        *U = 0.5 * Kr * (rf_len - ri_len) * (rf_len - ri_len) +
             0.5 * Ks * rf_len * rf_len * gamma * gamma + 0.5 * Kt * psi * psi +
             0.5 * Kb * theta * theta;
    }
    if (diag) {
        diag[0] = gamma;
        diag[1] = psi;
        diag[2] = theta_b.x;
        diag[3] = theta_b.y;
        diag[4] = theta_b.z;
        diag[5] = rf_len;
        diag[6] = (double)m_branch;
        diag[7] = 0.0;
    }
}

void orc_bond(const double x1[3], const double x2[3], const double q1[4], const double q2[4],
              const double ri[3], const double K[4], int m_branch,
              double f1[3], double tau1[3], double f2[3], double tau2[3], double* U, double* diag) {
    bond_impl(x1, x2, q1, q2, ri, K, m_branch, NULL, NULL, NULL, NULL, 0.0, f1, tau1, f2, tau2, U, diag,
              NULL);
}

void orc_bond_damped(const double x1[3], const double x2[3], const double q1[4], const double q2[4],
                     const double ri[3], const double K[4], const double g[4], const double v1[3],
                     const double v2[3], const double prev[3], double dt,
                     double f1[3], double tau1[3], double f2[3], double tau2[3], double* U,
                     double meas[3]) {
    bond_impl(x1, x2, q1, q2, ri, K, -1, g, v1, v2, prev, dt, f1, tau1, f2, tau2, U, NULL, meas);
}

/* ------------------------------------------------------------------ */
/* external field                                                      */
/* ------------------------------------------------------------------ */
static int n_threads(const orc_system* s) {
#ifdef _OPENMP
    return s->n_threads > 0 ? s->n_threads : omp_get_max_threads();
#else
    (void)s;
    return 1;
#endif
}

static int64_t* rod_index(const orc_system* s) {
    int64_t* rod_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n > 0 ? s->n : 1));
    if (!rod_of) return NULL;
    for (int64_t r = 0; r < s->n_rods; ++r)
        for (int64_t k = s->rod_offset[r]; k < s->rod_offset[r + 1]; ++k) rod_of[k] = r;
    return rod_of;
}

static vec3 field_at(const orc_system* s, vec3 x, int64_t rod, double t) {
    vec3 B = vmake(s->B[0], s->B[1], s->B[2]);
    if (s->B_rod) B = vadd(B, vload(s->B_rod + 3 * rod));
    if (s->Brot_amp != 0.0) {
        double cw = cos(s->Brot_omega * t), sw = sin(s->Brot_omega * t);
        B = vadd(B, vscale(vload(s->Brot_e1), s->Brot_amp * cw));
        B = vadd(B, vscale(vload(s->Brot_e2), s->Brot_amp * sw));
    }
    vec3 dx = vsub(x, vload(s->gradB_x0));
    const double* G = s->gradB;
    B = vadd(B, vmake(G[0] * dx.x + G[1] * dx.y + G[2] * dx.z,
                      G[3] * dx.x + G[4] * dx.y + G[5] * dx.z,
                      G[6] * dx.x + G[7] * dx.y + G[8] * dx.z));
    return B;
}

/* ------------------------------------------------------------------ */
/* dipole-dipole (Methods, "Magnetic interactions"), textbook gradient */
/* ------------------------------------------------------------------ */
static void dipole_on(const orc_system* s, const double* x, const double* m, const int64_t* rod_of,
                      int64_t i, vec3* F_out, vec3* tau_out, vec3* H_out, double* U_half) {
    vec3 F = vmake(0, 0, 0), T = vmake(0, 0, 0), H = vmake(0, 0, 0);
    double U = 0.0;
    const double c = s->c;
    vec3 xi = vload(x + 3 * i), mi = vload(m + 3 * i);
    int64_t j0 = 0, j1 = s->n;
    if (s->dipole_mode == 2) {
        j0 = s->rod_offset[rod_of[i]];
        j1 = s->rod_offset[rod_of[i] + 1];
    }
    for (int64_t j = j0; j < j1; ++j) {
        if (j == i) continue;
        vec3 mj = vload(m + 3 * j);
        vec3 r = vsub(xi, vload(x + 3 * j)); /* r = x_i - x_j */
        double r2 = vdot(r, r);
        double rl = sqrt(r2);
        double r3 = r2 * rl, r5 = r3 * r2, r7 = r5 * r2;
        double a = vdot(mi, r), b = vdot(mj, r), dd = vdot(mi, mj);
        /* F_i = 3c [ (a m_j + b m_i + d r)/r^5 - 5 a b r / r^7 ] */
        vec3 t1 = vadd(vadd(vscale(mj, a), vscale(mi, b)), vscale(r, dd));
        vec3 Fij = vscale(vsub(vscale(t1, 1.0 / r5), vscale(r, 5.0 * a * b / r7)), 3.0 * c);
        /* field of j at x_i: B_j = c [ 3 b r / r^5 - m_j / r^3 ] */
        vec3 Bj = vscale(vsub(vscale(r, 3.0 * b / r5), vscale(mj, 1.0 / r3)), c);
        F = vadd(F, Fij);
        T = vadd(T, vcross(mi, Bj));
        H = vadd(H, Bj);
        /* U_ij = c / r^3 [ m_i.m_j - 3 (m_i.r^)(m_j.r^) ] */
        U += c / r3 * (dd - 3.0 * a * b / r2);
    }
    *F_out = F;
    *tau_out = T;
    if (H_out) *H_out = H;
    if (U_half) *U_half = 0.5 * U;
}

int orc_dipole_sample(const orc_system* s, const double* x, const double* m, const int64_t* idx,
                      int64_t n_idx, double* F, double* tau, double* H) {
    int64_t* rod_of = rod_index(s);
    if (!rod_of) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads(s))
    for (int64_t k = 0; k < n_idx; ++k) {
        vec3 Fi, Ti, Hi;
        dipole_on(s, x, m, rod_of, idx[k], &Fi, &Ti, &Hi, NULL);
        vstore(Fi, F + 3 * k);
        vstore(Ti, tau + 3 * k);
        if (H) vstore(Hi, H + 3 * k);
    }
    free(rod_of);
    return 0;
}

/* ------------------------------------------------------------------ */
/* contact (R11)                                                       */
/* ------------------------------------------------------------------ */
int orc_contact_pair(const orc_contact* c, const double xi_[3], const double xj_[3], const double vi[3],
                     const double vj[3], const double wi[3], const double wj[3], double Ri, double Rj,
                     const double* xi_old, double dt, double f_i[3], double tau_i[3], double tau_j[3],
                     double xi_new[3]) {
    vec3 d = vsub(vload(xi_), vload(xj_));
    double dist = vnorm(d);
    double delta = Ri + Rj - dist;
    if (!(delta > 0.0) || !(dist > 0.0)) return 0;
    vec3 n = vscale(d, 1.0 / dist);
    double Rstar = Ri * Rj / (Ri + Rj);
    double Estar = c->E / (2.0 * (1.0 - c->nu * c->nu));
    double G = c->E / (2.0 * (1.0 + c->nu));
    double Gstar = G / (2.0 * (2.0 - c->nu));
    double a = sqrt(Rstar * delta);
    double Fh = 4.0 / 3.0 * Estar * a * delta; /* Hertz */

    /* relative velocity of the contact points */
    vec3 wsum = vadd(vscale(vload(wi), Ri), vscale(vload(wj), Rj));
    vec3 vrel = vsub(vsub(vload(vi), vload(vj)), vcross(wsum, n));
    double vn = vdot(vrel, n);
    vec3 vt = vsub(vrel, vscale(n, vn));

    /* tangential displacement carried into the current tangent plane */
    vec3 xi = vmake(0.0, 0.0, 0.0);
    if (xi_old) {
        vec3 xo = vload(xi_old);
        vec3 xp = vsub(xo, vscale(n, vdot(xo, n)));
        double lo = vnorm(xo), lp = vnorm(xp);
        xi = (lp > 0.0) ? vscale(xp, lo / lp) : xp;
    }
    xi = vadd(xi, vscale(vt, dt));

    double kt = 8.0 * Gstar * a; /* Mindlin */
    vec3 Ft = vsub(vscale(xi, -kt), vscale(vt, c->gamma_t));
    double ft = vnorm(Ft);
    if (ft > c->mu * Fh) {
        Ft = vscale(Ft, c->mu * Fh / ft);
        xi = vscale(vadd(Ft, vscale(vt, c->gamma_t)), -1.0 / kt);
    }
    vec3 F = vadd(vscale(n, Fh - c->gamma_n * vn), Ft);
    vstore(F, f_i);
    vstore(vcross(vscale(n, -Ri), Ft), tau_i);
    vstore(vcross(vscale(n, -Rj), Ft), tau_j);
    vstore(xi, xi_new);
    return 1;
}

static const double* contact_find(const orc_contact* c, int64_t n, int L, int64_t i, int64_t j) {
    if (!c->valid[L]) return NULL;
    int cnt = c->count[(size_t)L * n + i];
    for (int k = 0; k < cnt; ++k)
        if (c->partner[((size_t)L * n + i) * c->cap + k] == j) return c->xi + (((size_t)L * n + i) * c->cap + k) * 3;
    return NULL;
}

static void contact_record(orc_contact* c, int64_t n, int L, int64_t i, int64_t j, const double xi[3]) {
    int* cnt = c->count + (size_t)L * n + i;
    if (*cnt >= c->cap) {
        c->overflow = 1;
        return;
    }
    size_t slot = ((size_t)L * n + i) * c->cap + *cnt;
    c->partner[slot] = j;
    memcpy(c->xi + slot * 3, xi, 3 * sizeof(double));
    *cnt += 1;
}

/* adds contact forces to f, tau; hist_step as in forces_impl */
static void contact_forces(const orc_system* s, const int64_t* rod_of, const double* x, const double* v,
                           const double* w, double* f, double* tau, int hist_step) {
    orc_contact* c = s->contact;
    const int64_t n = s->n;
    const int cur = c->level, prv = 1 - c->level;
    const int ref = hist_step ? cur : prv;
    int out = -1; /* level written by this evaluation */
    if (hist_step)
        out = prv;
    else if (!c->valid[cur])
        out = cur;
    if (out >= 0)
        for (int64_t i = 0; i < n; ++i) c->count[(size_t)out * n + i] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            int64_t dij = j - i;
            if (rod_of[i] == rod_of[j] && dij <= c->exclude) continue;
            double fi[3], ti[3], tj[3], xin[3];
            const double* xo = contact_find(c, n, ref, i, j);
            if (!orc_contact_pair(c, x + 3 * i, x + 3 * j, v + 3 * i, v + 3 * j, w + 3 * i, w + 3 * j,
                                  s->radius[i], s->radius[j], xo, s->dt, fi, ti, tj, xin))
                continue;
            for (int a = 0; a < 3; ++a) {
                f[3 * i + a] += fi[a];
                f[3 * j + a] -= fi[a];
                tau[3 * i + a] += ti[a];
                tau[3 * j + a] += tj[a];
            }
            if (out >= 0) {
                double xjn[3] = {-xin[0], -xin[1], -xin[2]};
                contact_record(c, n, out, i, j, xin);
                contact_record(c, n, out, j, i, xjn);
            }
        }
    }
    if (out >= 0) c->valid[out] = 1;
    if (hist_step) c->level = prv;
}

int orc_contact_sample(const orc_system* s, const double* x, const double* v, const double* w,
                       const int64_t* idx, int64_t k, double* f, double* tau) {
    if (!s->contact) return -1;
    int64_t* rod_of = rod_index(s);
    if (!rod_of) return -1;
    const orc_contact* c = s->contact;
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads(s))
    for (int64_t a = 0; a < k; ++a) {
        const int64_t i = idx[a];
        double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
        for (int64_t j = 0; j < s->n; ++j) {
            if (j == i) continue;
            int64_t dij = j > i ? j - i : i - j;
            if (rod_of[i] == rod_of[j] && dij <= c->exclude) continue;
            double fi[3], ti[3], tj[3], xin[3];
            if (!orc_contact_pair(c, x + 3 * i, x + 3 * j, v + 3 * i, v + 3 * j, w + 3 * i, w + 3 * j,
                                  s->radius[i], s->radius[j], NULL, s->dt, fi, ti, tj, xin))
                continue;
            for (int e = 0; e < 3; ++e) {
                F[e] += fi[e];
                T[e] += ti[e];
            }
        }
        memcpy(f + 3 * a, F, sizeof(F));
        memcpy(tau + 3 * a, T, sizeof(T));
    }
    free(rod_of);
    return 0;
}

/* ------------------------------------------------------------------ */
/* lattice Boltzmann fluid and immersed boundary (R12)                 */
/* ------------------------------------------------------------------ */
static const int LBM_E[19][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double lbm_w(int i) { return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

void orc_lbm_lattice(int e[57], double w[19]) {
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = LBM_E[i][a];
        w[i] = lbm_w(i);
    }
}

static int64_t lbm_nodes(const orc_lbm* L) { return (int64_t)L->nx * L->ny * L->nz; }

static int wrap(int64_t i, int n) {
    int64_t r = i % n;
    return (int)(r < 0 ? r + n : r);
}

static int64_t lbm_node(const orc_lbm* L, int64_t i, int64_t j, int64_t k) {
    return wrap(i, L->nx) + (int64_t)L->nx * (wrap(j, L->ny) + (int64_t)L->ny * wrap(k, L->nz));
}

/* f_i^eq = w_i rho (1 + e.u / cs^2 + (e.u)^2 / (2 cs^4) - u.u / (2 cs^2)), cs^2 = 1/3 */
static void lbm_feq(double rho, const double u[3], double out[19]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double eu = LBM_E[i][0] * u[0] + LBM_E[i][1] * u[1] + LBM_E[i][2] * u[2];
        out[i] = lbm_w(i) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* distributions arriving at node (i,j,k) by streaming */
static void lbm_pull(const orc_lbm* L, int64_t i, int64_t j, int64_t k, double fi[19]) {
    const int64_t nn = lbm_nodes(L);
    for (int q = 0; q < 19; ++q)
        fi[q] = L->f[q * nn + lbm_node(L, i - LBM_E[q][0], j - LBM_E[q][1], k - LBM_E[q][2])];
}

void orc_lbm_init(orc_lbm* L, const double* rho, const double* u) {
    const int64_t nn = lbm_nodes(L);
    for (int64_t x = 0; x < nn; ++x) {
        double r = rho ? rho[x] : 1.0;
        double uu[3] = {u ? u[3 * x] : 0.0, u ? u[3 * x + 1] : 0.0, u ? u[3 * x + 2] : 0.0};
        double fe[19];
        lbm_feq(r, uu, fe);
        for (int q = 0; q < 19; ++q) L->f[q * nn + x] = fe[q];
        for (int a = 0; a < 3; ++a) L->F[a * nn + x] = 0.0;
    }
    L->phase = 0;
    L->steps = 0;
}

void orc_lbm_macro(const orc_lbm* L, double* rho, double* u) {
    for (int64_t k = 0; k < L->nz; ++k)
        for (int64_t j = 0; j < L->ny; ++j)
            for (int64_t i = 0; i < L->nx; ++i) {
                double fi[19], r = 0.0, m[3] = {0, 0, 0};
                lbm_pull(L, i, j, k, fi);
                for (int q = 0; q < 19; ++q) {
                    r += fi[q];
                    for (int a = 0; a < 3; ++a) m[a] += fi[q] * LBM_E[q][a];
                }
                int64_t x = lbm_node(L, i, j, k);
                if (rho) rho[x] = r;
                for (int a = 0; a < 3; ++a) u[3 * x + a] = (m[a] + 0.5 * L->body_force[a]) / r;
            }
}

int orc_lbm_step(orc_lbm* L) {
    const int64_t nn = lbm_nodes(L);
    const double tau = L->tau;
    for (int64_t k = 0; k < L->nz; ++k)
        for (int64_t j = 0; j < L->ny; ++j)
            for (int64_t i = 0; i < L->nx; ++i) {
                int64_t x = lbm_node(L, i, j, k);
                double fi[19], r = 0.0, m[3] = {0, 0, 0}, F[3], u[3], fe[19];
                lbm_pull(L, i, j, k, fi);
                for (int q = 0; q < 19; ++q) {
                    r += fi[q];
                    for (int a = 0; a < 3; ++a) m[a] += fi[q] * LBM_E[q][a];
                }
                for (int a = 0; a < 3; ++a) {
                    F[a] = L->body_force[a] + L->F[a * nn + x];
                    u[a] = (m[a] + 0.5 * F[a]) / r; /* half-step velocity */
                }
                lbm_feq(r, u, fe);
                double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
                for (int q = 0; q < 19; ++q) {
                    double eF = LBM_E[q][0] * F[0] + LBM_E[q][1] * F[1] + LBM_E[q][2] * F[2];
                    double eu = LBM_E[q][0] * u[0] + LBM_E[q][1] * u[1] + LBM_E[q][2] * u[2];
                    /* Guo's source with cs^2 = 1/3 */
                    double S = (1.0 - 0.5 / tau) * lbm_w(q) * (3.0 * eF + 9.0 * eu * eF - 3.0 * uF);
                    L->f_tmp[q * nn + x] = fi[q] - (fi[q] - fe[q]) / tau + S;
                }
            }
    double* t = L->f;
    L->f = L->f_tmp;
    L->f_tmp = t;
    memset(L->F, 0, sizeof(double) * 3 * (size_t)nn);
    L->steps += 1;
    return 0;
}

double orc_ibm_phi(double r) {
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) / 8.0;
    if (r < 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) / 8.0;
    return 0.0;
}

/* the 4 x 4 x 4 support of the delta at X: node indices and weights */
static void ibm_support(const double X[3], int64_t idx[3][4], double wgt[3][4]) {
    for (int a = 0; a < 3; ++a) {
        int64_t base = (int64_t)floor(X[a]) - 1;
        for (int s = 0; s < 4; ++s) {
            idx[a][s] = base + s;
            wgt[a][s] = orc_ibm_phi(X[a] - (double)(base + s));
        }
    }
}

void orc_lbm_interp(const orc_lbm* L, const double* x, int64_t n, double* U) {
    const int64_t nn = lbm_nodes(L);
    double* rho = (double*)malloc(sizeof(double) * (size_t)nn);
    double* u = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
    orc_lbm_macro(L, rho, u);
    for (int64_t p = 0; p < n; ++p) {
        int64_t idx[3][4];
        double wgt[3][4];
        ibm_support(x + 3 * p, idx, wgt);
        double acc[3] = {0, 0, 0};
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    double wv = wgt[0][a] * wgt[1][b] * wgt[2][c];
                    int64_t node = lbm_node(L, idx[0][a], idx[1][b], idx[2][c]);
                    for (int e = 0; e < 3; ++e) acc[e] += u[3 * node + e] * wv;
                }
        for (int e = 0; e < 3; ++e) U[3 * p + e] = acc[e];
    }
    free(rho);
    free(u);
}

/* penalty force on the coupled particles; spread its reaction when asked */
static void ibm_penalty(const orc_system* s, const double* x, const double* v, double* f, int spread) {
    orc_lbm* L = s->lbm;
    const int64_t nn = lbm_nodes(L);
    for (int64_t p = 0; p < s->n; ++p) {
        if (L->coupled && !L->coupled[p]) continue;
        double Fp[3];
        for (int a = 0; a < 3; ++a) {
            Fp[a] = s->mass[p] * (L->U[3 * p + a] - v[3 * p + a]); /* kappa = m_p / dt_LBM */
            f[3 * p + a] += Fp[a];
        }
        if (!spread) continue;
        int64_t idx[3][4];
        double wgt[3][4];
        ibm_support(x + 3 * p, idx, wgt);
        for (int c = 0; c < 4; ++c)
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    double wv = wgt[0][a] * wgt[1][b] * wgt[2][c];
                    int64_t node = lbm_node(L, idx[0][a], idx[1][b], idx[2][c]);
                    for (int e = 0; e < 3; ++e) L->F[e * nn + node] -= Fp[e] * wv / L->n_sub;
                }
    }
}

/* ------------------------------------------------------------------ */
/* total force and torque                                              */
/* ------------------------------------------------------------------ */
static int has_measures(const double* h) { return !isnan(h[0]) && !isnan(h[1]) && !isnan(h[2]); }

/* hist_step = 0: a stand-alone evaluation (rates against the previous level,
 * the current level filled in when empty); 1: an evaluation of the time
 * stepping at a new state (rates against the current level, then the levels
 * shift) -- reading R10 */
static int forces_impl(const orc_system* s, const double* x, const double* q, const double* v,
                       const double* w, double t, double* f, double* tau, double* m_out,
                       double* energy, int hist_step) {
    const int64_t n = s->n;
    const int damped = s->bond_g != NULL && s->bond_hist != NULL;
    int64_t* rod_of = rod_index(s);
    double* m = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* meas = damped ? (double*)malloc(sizeof(double) * 3 * (size_t)(s->n_bonds > 0 ? s->n_bonds : 1))
                          : NULL;
    if (!rod_of || !m || (damped && !meas)) { free(rod_of); free(m); free(meas); return -1; }
    double E_bond = 0.0, E_zee = 0.0, E_dip = 0.0, E_kt = 0.0, E_kr = 0.0;

    /* dipoles rotate with the particle: m = q m~ q^* */
    for (int64_t i = 0; i < n; ++i) vstore(rot(qload(q + 4 * i), vload(s->m_body + 3 * i)), m + 3 * i);
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    memset(tau, 0, sizeof(double) * 3 * (size_t)n);

    /* bonds */
    for (int64_t b = 0; b < s->n_bonds; ++b) {
        int64_t p1 = s->bond_p1[b], p2 = s->bond_p2[b];
        double q1r[4], q2r[4], f1[3], t1[3], f2[3], t2[3], U;
        /* R1: rotation of each end since the rest state */
        qstore(qmul(qload(q + 4 * p1), qconj(qload(s->q_rest + 4 * p1))), q1r);
        qstore(qmul(qload(q + 4 * p2), qconj(qload(s->q_rest + 4 * p2))), q2r);
        const double* g = damped ? s->bond_g + 4 * b : NULL;
        const double* prev = NULL;
        if (damped) {
            /* the two recorded levels of bond b: [previous | current] */
            const double* ref = s->bond_hist + 6 * b + (hist_step ? 3 : 0);
            if (has_measures(ref)) prev = ref;
        }
        bond_impl(x + 3 * p1, x + 3 * p2, q1r, q2r, s->bond_ri + 3 * b, s->bond_K + 4 * b, -1, g,
                  v + 3 * p1, v + 3 * p2, prev, s->dt, f1, t1, f2, t2, &U, NULL,
                  damped ? meas + 3 * b : NULL);
        for (int a = 0; a < 3; ++a) {
            f[3 * p1 + a] += f1[a];
            tau[3 * p1 + a] += t1[a];
            f[3 * p2 + a] += f2[a];
            tau[3 * p2 + a] += t2[a];
        }
        E_bond += U;
    }

    /* contact between non-bonded particles (R11) */
    if (s->contact) contact_forces(s, rod_of, x, v, w, f, tau, hist_step);

    /* penalty coupling to the fluid (R12): step evaluations spread */
    if (s->lbm) ibm_penalty(s, x, v, f, hist_step);

    /* Zeeman: U = -m.B, tau = m x B, f = grad(m.B) = G^T m */
    for (int64_t i = 0; i < n; ++i) {
        vec3 xi = vload(x + 3 * i), mi = vload(m + 3 * i);
        vec3 B = field_at(s, xi, rod_of[i], t);
        vec3 T = vcross(mi, B);
        const double* G = s->gradB;
        vec3 Fz = vmake(G[0] * mi.x + G[3] * mi.y + G[6] * mi.z,
                        G[1] * mi.x + G[4] * mi.y + G[7] * mi.z,
                        G[2] * mi.x + G[5] * mi.y + G[8] * mi.z);
        f[3 * i + 0] += Fz.x; f[3 * i + 1] += Fz.y; f[3 * i + 2] += Fz.z;
        tau[3 * i + 0] += T.x; tau[3 * i + 1] += T.y; tau[3 * i + 2] += T.z;
        E_zee -= vdot(mi, B);
    }

    /* dipole-dipole */
    if (s->dipole_mode != 0) {
        double Ud = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : Ud) num_threads(n_threads(s))
        for (int64_t i = 0; i < n; ++i) {
            vec3 Fi, Ti;
            double Uh;
            dipole_on(s, x, m, rod_of, i, &Fi, &Ti, NULL, &Uh);
            f[3 * i + 0] += Fi.x; f[3 * i + 1] += Fi.y; f[3 * i + 2] += Fi.z;
            tau[3 * i + 0] += Ti.x; tau[3 * i + 1] += Ti.y; tau[3 * i + 2] += Ti.z;
            Ud += Uh;
        }
        E_dip = Ud;
    }

    /* global viscous damping (R8) and kinetic energy */
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            f[3 * i + a] -= s->damping * v[3 * i + a];
            tau[3 * i + a] -= s->damping * w[3 * i + a];
        }
        double I = 0.4 * s->mass[i] * s->radius[i] * s->radius[i];
        E_kt += 0.5 * s->mass[i] * vdot(vload(v + 3 * i), vload(v + 3 * i));
        E_kr += 0.5 * I * vdot(vload(w + 3 * i), vload(w + 3 * i));
    }

    /* record this evaluation's measures (R10) */
    for (int64_t b = 0; damped && b < s->n_bonds; ++b) {
        double* h = s->bond_hist + 6 * b;
        if (hist_step) {
            memcpy(h, h + 3, 3 * sizeof(double));
            memcpy(h + 3, meas + 3 * b, 3 * sizeof(double));
        } else if (!has_measures(h + 3)) {
            memcpy(h + 3, meas + 3 * b, 3 * sizeof(double));
        }
    }

    if (m_out) memcpy(m_out, m, sizeof(double) * 3 * (size_t)n);
    if (energy) {
        energy[0] = E_bond;
        energy[1] = E_zee;
        energy[2] = E_dip;
        energy[3] = E_kt;
        energy[4] = E_kr;
    }
    free(meas);
    free(m);
    free(rod_of);
    return 0;
}

int orc_forces(const orc_system* s, const double* x, const double* q, const double* v,
               const double* w, double t, double* f, double* tau, double* m_out,
               double* energy) {
    return forces_impl(s, x, q, v, w, t, f, tau, m_out, energy, 0);
}

/* ------------------------------------------------------------------ */
/* per-particle condition scale of the summed force and torque         */
/* ------------------------------------------------------------------ */
int orc_term_scales(const orc_system* s, const double* x, const double* q, const double* v,
                    const double* w, double t, const int64_t* idx, int64_t n_idx, double* sf,
                    double* st) {
    const int64_t n = s->n;
    int64_t* rod_of = rod_index(s);
    double* m = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* bf = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* bt = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!rod_of || !m || !bf || !bt) { free(rod_of); free(m); free(bf); free(bt); return -1; }
    for (int64_t i = 0; i < n; ++i) vstore(rot(qload(q + 4 * i), vload(s->m_body + 3 * i)), m + 3 * i);
    /* elastic bond terms at each end */
    for (int64_t b = 0; b < s->n_bonds; ++b) {
        int64_t p1 = s->bond_p1[b], p2 = s->bond_p2[b];
        double q1r[4], q2r[4], f1[3], t1[3], f2[3], t2[3];
        qstore(qmul(qload(q + 4 * p1), qconj(qload(s->q_rest + 4 * p1))), q1r);
        qstore(qmul(qload(q + 4 * p2), qconj(qload(s->q_rest + 4 * p2))), q2r);
        bond_impl(x + 3 * p1, x + 3 * p2, q1r, q2r, s->bond_ri + 3 * b, s->bond_K + 4 * b, -1, NULL,
                  NULL, NULL, NULL, s->dt, f1, t1, f2, t2, NULL, NULL, NULL);
        bf[p1] += vnorm(vload(f1));
        bt[p1] += vnorm(vload(t1));
        bf[p2] += vnorm(vload(f2));
        bt[p2] += vnorm(vload(t2));
    }
#pragma omp parallel for schedule(dynamic, 4) num_threads(n_threads(s))
    for (int64_t k = 0; k < n_idx; ++k) {
        const int64_t i = idx[k];
        vec3 xi = vload(x + 3 * i), mi = vload(m + 3 * i);
        double SF = bf[i], ST = bt[i];
        /* Zeeman */
        vec3 B = field_at(s, xi, rod_of[i], t);
        const double* G = s->gradB;
        vec3 Fz = vmake(G[0] * mi.x + G[3] * mi.y + G[6] * mi.z, G[1] * mi.x + G[4] * mi.y + G[7] * mi.z,
                        G[2] * mi.x + G[5] * mi.y + G[8] * mi.z);
        SF += vnorm(Fz);
        ST += vnorm(mi) * vnorm(B);
        /* dipole pairs */
        if (s->dipole_mode != 0) {
            int64_t j0 = 0, j1 = n;
            if (s->dipole_mode == 2) {
                j0 = s->rod_offset[rod_of[i]];
                j1 = s->rod_offset[rod_of[i] + 1];
            }
            for (int64_t j = j0; j < j1; ++j) {
                if (j == i) continue;
                vec3 mj = vload(m + 3 * j);
                vec3 r = vsub(xi, vload(x + 3 * j));
                double r2 = vdot(r, r), rl = sqrt(r2);
                double r3 = r2 * rl, r5 = r3 * r2, r7 = r5 * r2;
                double a = vdot(mi, r), bb = vdot(mj, r), dd = vdot(mi, mj);
                vec3 t1 = vadd(vadd(vscale(mj, a), vscale(mi, bb)), vscale(r, dd));
                vec3 Fij = vscale(vsub(vscale(t1, 1.0 / r5), vscale(r, 5.0 * a * bb / r7)), 3.0 * s->c);
                vec3 Bj = vscale(vsub(vscale(r, 3.0 * bb / r5), vscale(mj, 1.0 / r3)), s->c);
                SF += vnorm(Fij);
                ST += vnorm(mi) * vnorm(Bj);
            }
        }
        /* global damping */
        SF += s->damping * vnorm(vload(v + 3 * i));
        ST += s->damping * vnorm(vload(w + 3 * i));
        sf[k] = SF;
        st[k] = ST;
    }
    free(rod_of);
    free(m);
    free(bf);
    free(bt);
    return 0;
}

/* ------------------------------------------------------------------ */
/* integration (SI "Equations of motion")                              */
/* ------------------------------------------------------------------ */
void orc_richardson(const double q_[4], const double w_[3], double dt, double out[4]) {
    quat q = qload(q_);
    quat W = qmake(0.0, w_[0], w_[1], w_[2]);
    /* q' = 1/2 omega q (R7) */
    quat qd = qscale(qmul(W, q), 0.5);
    /* one step of dt */
    quat q1 = qnormalize(qadd(q, qscale(qd, dt)));
    /* two steps of dt/2 */
    quat qh = qnormalize(qadd(q, qscale(qd, 0.5 * dt)));
    quat qhd = qscale(qmul(W, qh), 0.5);
    quat q2 = qnormalize(qadd(qh, qscale(qhd, 0.5 * dt)));
    /* extrapolation: q(t+dt) = 2 q_(2) - q_(1) */
    quat qn = qnormalize(qadd(qscale(q2, 2.0), qscale(q1, -1.0)));
    qstore(qn, out);
}

int orc_run(const orc_system* s, double* x, double* q, double* v, double* w, double* t,
            int n_steps, double* f, double* tau, int forces_valid) {
    const int64_t n = s->n;
    const double dt = s->dt;
    if (!forces_valid && forces_impl(s, x, q, v, w, *t, f, tau, NULL, NULL, 0) != 0) return -1;
    for (int step = 0; step < n_steps; ++step) {
        for (int64_t i = 0; i < n; ++i) {
            if (s->clamped[i]) continue; /* R9 */
            double mass = s->mass[i];
            double I = 0.4 * mass * s->radius[i] * s->radius[i];
            for (int a = 0; a < 3; ++a) {
                v[3 * i + a] += 0.5 * dt * f[3 * i + a] / mass;
                x[3 * i + a] += dt * v[3 * i + a];
                w[3 * i + a] += 0.5 * dt * tau[3 * i + a] / I;
            }
            double qn[4];
            orc_richardson(q + 4 * i, w + 3 * i, dt, qn);
            memcpy(q + 4 * i, qn, sizeof(qn));
        }
        *t += dt;
        /* a new LBM cycle interpolates the fluid velocity once (R12) */
        if (s->lbm && s->lbm->phase == 0) orc_lbm_interp(s->lbm, x, n, s->lbm->U);
        if (forces_impl(s, x, q, v, w, *t, f, tau, NULL, NULL, 1) != 0) return -1;
        for (int64_t i = 0; i < n; ++i) {
            if (s->clamped[i]) continue;
            double mass = s->mass[i];
            double I = 0.4 * mass * s->radius[i] * s->radius[i];
            for (int a = 0; a < 3; ++a) {
                v[3 * i + a] += 0.5 * dt * f[3 * i + a] / mass;
                w[3 * i + a] += 0.5 * dt * tau[3 * i + a] / I;
            }
        }
        if (s->lbm && ++s->lbm->phase == s->lbm->n_sub) {
            orc_lbm_step(s->lbm);
            s->lbm->phase = 0;
        }
    }
    return 0;
}
