// Bond kernel: co-rotational bond forces and torques (main text, "Bonded-
// particle model for elastic rods", Eqs. bpm-fr .. bpm-vector; SI
// "Symmetric rotational decomposition", Eq. S-quat-h), fused with the
// dipole orientation m = q m~ q* ("Magnetized beams"), the Zeeman torque and
// force (Methods, "Magnetic interactions") and global viscous damping
// and bond-level damping per mode (Methods, "Damping").
//
// Work decomposition: a warp loads 32 consecutive particles p = 30w-1+lane
// (one per lane, coalesced SoA loads).  Lanes 0..30 evaluate the bond
// (p, p+1), taking particle p+1 from the next lane with a shuffle; lanes
// 1..30 then own particle p and add bond p (as particle 1) and bond p-1 (as
// particle 2, shuffled up from the previous lane).  Every particle is written
// by exactly one lane, in rod order, with no atomics and no scratch; 31
// bonds are evaluated per 30 particles.
#include "bpm_devmath.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

struct BondOut {
    d3 f1, t1, t2;
    double U;
    double gamma, psi, theta;  // measures (filled when damping)
};

// Bond damping inputs (Methods, "Damping"): factors g, relative velocity
// v_2 - v_1, and the measures (gamma, psi, theta) the rates difference
// against (NaN: none, zero angular rates).
struct BondDamp {
    double gr, gs, gt, gb;
    d3 dv;
    double g0, p0, t0;
    double dt;
};

// Rotation matrix of a unit quaternion, R v = q v q*: built once where q
// rotates several vectors (9 FP64 operations per vector instead of the 18
// of the quaternion form).
struct m33 {
    d3 r0, r1, r2;  // rows
};
__device__ __forceinline__ m33 qmat(dq q) {
    const double x2 = q.x + q.x, y2 = q.y + q.y, z2 = q.z + q.z;
    const double xx = q.x * x2, yy = q.y * y2, zz = q.z * z2;
    const double xy = q.x * y2, xz = q.x * z2, yz = q.y * z2;
    const double wx = q.w * x2, wy = q.w * y2, wz = q.w * z2;
    return m33{mk3(1.0 - (yy + zz), xy - wz, xz + wy), mk3(xy + wz, 1.0 - (xx + zz), yz - wx),
               mk3(xz - wy, yz + wx, 1.0 - (xx + yy))};
}
// matrix products with explicit roundings
__device__ __forceinline__ double dot_rn(d3 a, d3 b) {
    return __fma_rn(a.z, b.z, __fma_rn(a.y, b.y, __dmul_rn(a.x, b.x)));
}
__device__ __forceinline__ d3 mv(const m33& R, d3 v) { return mk3(dot_rn(R.r0, v), dot_rn(R.r1, v), dot_rn(R.r2, v)); }
// Reading of the paper used for the quaternion m of Eq. S-quat-h: for z >= 0
// (r+z, -y, x, 0)/sqrt(2r(r+z)) (the printed m without its 0/0); for z < 0
// the rotation (-y, r-z, 0, x)/sqrt(2r(r-z)), which also takes z onto r_f[C]
// and differs from the printed one by a turn about z, leaving the torques
// unchanged.  Only its rotation matrix is used; with n = r_f / r and
// k = 1 / (1 + |n_z|) it is, written out from the quaternion,
//   n_z >= 0:  [[1 - n_x^2 k, -n_x n_y k, n_x], [-n_x n_y k, 1 - n_y^2 k, n_y], [-n_x, -n_y, n_z]]
//   n_z <  0:  [[1 - n_x^2 k,  n_x n_y k, n_x], [-n_x n_y k, n_z - n_x^2 k, n_y], [ n_x, -n_y, n_z]]
// (7 FP64 operations and a reciprocal instead of the quaternion's square
// root and the 21 operations of its matrix).
__device__ __forceinline__ m33 align_z_mat(d3 n) {
    if (n.z >= 0.0) {
        const double k = rcp_nr(1.0 + n.z);
        const double a = __dmul_rn(n.x, k), b = __dmul_rn(n.y, k);
        const double c = -__dmul_rn(n.y, a);
        return m33{mk3(__fma_rn(-n.x, a, 1.0), c, n.x), mk3(c, __fma_rn(-n.y, b, 1.0), n.y), mk3(-n.x, -n.y, n.z)};
    }
    const double k = rcp_nr(1.0 - n.z);
    const double a = __dmul_rn(n.x, k);
    const double c = __dmul_rn(n.y, a);
    return m33{mk3(__fma_rn(-n.x, a, 1.0), c, n.x), mk3(-c, __fma_rn(-n.x, a, n.z), n.y), mk3(n.x, -n.y, n.z)};
}
// R^T v
__device__ __forceinline__ d3 mtv(const m33& R, d3 v) {
    return mk3(__fma_rn(R.r2.x, v.z, __fma_rn(R.r1.x, v.y, __dmul_rn(R.r0.x, v.x))),
               __fma_rn(R.r2.y, v.z, __fma_rn(R.r1.y, v.y, __dmul_rn(R.r0.y, v.x))),
               __fma_rn(R.r2.z, v.z, __fma_rn(R.r1.z, v.y, __dmul_rn(R.r0.z, v.x))));
}

// Not inlined: the bond kernel's sequential form and its form beside the
// dipole kernel call this one compiled function, so their results are
// bitwise the same (inlined into two differently shaped kernels, the
// compiler may contract the same expression into different fused
// multiply-adds).
template <bool ENERGY, bool DAMP>
__device__ __noinline__ BondOut bond_eval(d3 x1, d3 x2, dq q1, dq q2, d3 rih, double L, double Kr,
                                             double Ks, double Kt, double Kb, const BondDamp& dm) {
    BondOut o;
    // central frame C: slerp midpoint on the shorter arc
    if (qdot(q1, q2) < 0.0) q2 = qscale(q2, -1.0);
    dq qC = qnormalise_nr(dq{q1.w + q2.w, q1.x + q2.x, q1.y + q2.y, q1.z + q2.z});

    // rotation of C (frame C to O), used on r_f and on the results
    const m33 RC = qmat(qC);

    // r_f measured in C; its length in the global frame (an IEEE sqrt of a
    // sum without fused multiply-adds: the stretch below cancels against L)
    d3 rfO = x2 - x1;
    const double rf2 = norm2_rn(rfO);
    const double rf_len = sqrt(rf2);
    d3 rf = mtv(RC, rfO);
    const double rinv = rsqrt_nr(rf2);
    d3 rfh = rf * rinv;

    // radial force on particle 1 (Eq. bpm-fr), with radial damping on the
    // relative velocity along the bond (frame independent: dv . r^_f)
    double stretch = rf_len - L;
    double fr = Kr * stretch;
    if (DAMP) fr += dm.gr * (dot(dm.dv, rfO) * rinv);
    d3 F = rfh * fr;

    // shear (Eqs. bpm-fst, bpm-tst): gamma t^ = (gamma / |c|) c, c = r^_i x r^_f
    d3 c = cross(rih, rfh);
    const double sin2_g = dot(c, c);
    const double g_over_s = atan_over(sin2_g, dot(rih, rfh));
    d3 gt = c * g_over_s;
    F = F + cross(gt, rfh) * (Ks * rf_len);
    d3 TS = gt * (0.5 * Ks * rf_len * rf_len);

    // C' frame (Eq. S-quat-h) and the half rotation u = m* (q_C* q_2) m:
    // the scalar part of u^0, its vector part rotated by m^-1
    const m33 Rm = align_z_mat(rfh);
    const dq u0 = qmul(qconj(qC), q2);
    const d3 uv = mtv(Rm, mk3(u0.x, u0.y, u0.z));
    const dq u = dq{u0.w, uv.x, uv.y, uv.z};

    // bend before twist: u = t2 b2, u* = t1 b1 with t1 = t2*;
    // psi = psi2 - psi1 = 4 atan2(t_z, t_w)
    double tn = rsqrt_nr(u.w * u.w + u.z * u.z);
    double tw = u.w * tn, tz = u.z * tn;
    double psi = 4.0 * tz * atan_over(tz * tz, tw);
    // b = b2 b1* = t2* u u t2*
    // u u and the products with t2* = (tw, 0, 0, -tz), written out for their
    // zero components (the general product would spend 24 more FP64
    // operations on them)
    const double uv2 = u.x * u.x + u.y * u.y + u.z * u.z, uw2 = 2.0 * u.w;
    const dq uu = dq{u.w * u.w - uv2, uw2 * u.x, uw2 * u.y, uw2 * u.z};
    const dq tu = dq{tw * uu.w + tz * uu.z, tw * uu.x + tz * uu.y, tw * uu.y - tz * uu.x, tw * uu.z - tz * uu.w};
    dq b = dq{tw * tu.w + tz * tu.z, tw * tu.x - tz * tu.y, tw * tu.y + tz * tu.x, tw * tu.z - tz * tu.w};
    if (b.w < 0.0) b = qscale(b, -1.0);
    d3 bv = mk3(b.x, b.y, b.z);
    const double sb2 = dot(bv, bv);
    // theta b^ = (theta / |b_v|) b_v, theta = 2 atan2(|b_v|, b_w)
    double th_over_s = 2.0 * atan_over(sb2, b.w);
    // bending and twisting torques on particle 1 in C' (Eqs. bpm-tb, bpm-tt)
    d3 TBT = bv * (Kb * th_over_s);
    TBT.z += Kt * psi;

    if (DAMP) {
        // damping of the angular modes on backward-difference rates, each
        // along its elastic direction; shear and bend vanish at zero angle
        const double sg = sqrt(sin2_g), sbn = sqrt(sb2);
        o.gamma = g_over_s * sg;
        o.psi = psi;
        o.theta = th_over_s * sbn;
        if (!isnan(dm.g0) && !isnan(dm.p0) && !isnan(dm.t0)) {
            const double gdot = (o.gamma - dm.g0) / dm.dt;
            const double pdot = (psi - dm.p0) / dm.dt;
            const double tdot = (o.theta - dm.t0) / dm.dt;
            if (sin2_g > 0.0) {
                const d3 th = c * (1.0 / sg);  // t^
                F = F + cross(th, rfh) * (dm.gs * rf_len * gdot);
                TS = TS + th * (0.5 * dm.gs * rf_len * rf_len * gdot);
            }
            TBT.z += dm.gt * pdot;
            if (sb2 > 0.0) TBT = TBT + bv * (dm.gb * tdot / sbn);
        }
    }

    // back to O (Eq. bpm-vector): f1 = F, tau1 = TS + TBT, tau2 = TS - TBT,
    // with v[O] = q_C v[C] q_C* and v[O] = q_C m v[C'] m* q_C*
    d3 Fo = mv(RC, F);
    d3 TSo = mv(RC, TS);
    d3 TBTo = mv(RC, mv(Rm, TBT));
    o.f1 = Fo;
    o.t1 = TSo + TBTo;
    o.t2 = TSo - TBTo;
    if (ENERGY) {
        // Eq. total-energy, with gamma = (gamma/|c|)|c| and theta likewise
        const double gamma2 = g_over_s * g_over_s * sin2_g;
        const double theta2 = th_over_s * th_over_s * sb2;
        o.U = 0.5 * Kr * stretch * stretch + 0.5 * Ks * rf_len * rf_len * gamma2 + 0.5 * Kt * psi * psi +
              0.5 * Kb * theta2;
    } else {
        o.U = 0.0;
    }
    return o;
}

__device__ __forceinline__ d3 shfl_down3(d3 a) {
    return mk3(__shfl_down_sync(0xffffffffu, a.x, 1), __shfl_down_sync(0xffffffffu, a.y, 1),
               __shfl_down_sync(0xffffffffu, a.z, 1));
}
__device__ __forceinline__ d3 shfl_up3(d3 a) {
    return mk3(__shfl_up_sync(0xffffffffu, a.x, 1), __shfl_up_sync(0xffffffffu, a.y, 1),
               __shfl_up_sync(0xffffffffu, a.z, 1));
}

// The dipole moments in space, m = q m~ q*, and their FP32 copies for the
// FP32-pair dipole kernels (positions as hi + lo, moments rounded).
__device__ __forceinline__ void write_orientation(const Sys& s, int64_t p, d3 x, d3 m, bool copies) {
    const int64_t n = s.n;
    s.m[p] = m.x;
    s.m[n + p] = m.y;
    s.m[2 * n + p] = m.z;
    if (copies) {
        float hx = __double2float_rn(x.x), hy = __double2float_rn(x.y), hz = __double2float_rn(x.z);
        s.xh[p] = hx;
        s.xh[n + p] = hy;
        s.xh[2 * n + p] = hz;
        s.xl[p] = __double2float_rn(x.x - (double)hx);
        s.xl[n + p] = __double2float_rn(x.y - (double)hy);
        s.xl[2 * n + p] = __double2float_rn(x.z - (double)hz);
        s.mf[p] = __double2float_rn(m.x);
        s.mf[n + p] = __double2float_rn(m.y);
        s.mf[2 * n + p] = __double2float_rn(m.z);
    }
}

// MMODE: M_OWN computes m and writes it; M_OWN_COPIES writes the FP32 copies
// too; M_GIVEN reads the m that k_orient wrote (the dipole kernel may then
// run at the same time as this one).
enum { M_OWN = 0, M_OWN_COPIES = 1, M_GIVEN = 2 };

template <bool COPIES>
__global__ void __launch_bounds__(256) k_orient(Sys s) {
    const int64_t n = s.n;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const dq q = dq{s.q[p], s.q[n + p], s.q[2 * n + p], s.q[3 * n + p]};
    const d3 mb = mk3(s.m_body[p], s.m_body[n + p], s.m_body[2 * n + p]);
    const d3 x = mk3(s.x[p], s.x[n + p], s.x[2 * n + p]);
    write_orientation(s, p, x, rot(q, mb), COPIES);
}

// the 31 bonds and 30 particles of warp `warp` (p = 30 warp - 1 + lane)
template <bool ENERGY, int MMODE, bool DAMP>
__device__ __forceinline__ void bond_warp(const Sys& s, int64_t warp, int lane) {
    const int64_t n = s.n;
    const int64_t p = warp * 30 - 1 + lane;
    const bool valid = (p >= 0) && (p < n);
    const int64_t pc = valid ? p : 0;

    d3 x = mk3(s.x[pc], s.x[n + pc], s.x[2 * n + pc]);
    dq q = dq{s.q[pc], s.q[n + pc], s.q[2 * n + pc], s.q[3 * n + pc]};
    uint8_t flags = valid ? s.flags[pc] : 0;

    // neighbour p+1 from the next lane
    d3 xn = shfl_down3(x);
    dq qn = dq{__shfl_down_sync(0xffffffffu, q.w, 1), __shfl_down_sync(0xffffffffu, q.x, 1),
               __shfl_down_sync(0xffffffffu, q.y, 1), __shfl_down_sync(0xffffffffu, q.z, 1)};

    BondDamp dm{};
    double* hist_rate = nullptr;   // level the rates difference against
    double* hist_out = nullptr;    // level this evaluation's measures go to
    if (DAMP) {
        // v of p and p+1; level buffers: a step's evaluation differences
        // against the current level and writes the previous level's buffer
        // (the finish kernel then flips the parity); a stand-alone one
        // differences against the previous level and fills in an empty
        // current level
        const d3 vp = mk3(s.v[pc], s.v[n + pc], s.v[2 * n + pc]);
        dm.dv = shfl_down3(vp) - vp;
        const int gen = *s.hist_gen;
        double* cur = s.hist + (size_t)(gen & 1) * 3 * n;
        double* prv = s.hist + (size_t)((gen + 1) & 1) * 3 * n;
        hist_rate = s.count_step ? cur : prv;
        hist_out = s.count_step ? prv : cur;
        dm.dt = s.dt;
    }

    BondOut b;
    b.f1 = mk3(0, 0, 0);
    b.t1 = mk3(0, 0, 0);
    b.t2 = mk3(0, 0, 0);
    b.U = 0.0;
    const bool has_bond = valid && lane < 31 && (flags & F_BOND_RIGHT);
    if (has_bond) {
        const double* bd = s.bond;
        d3 rih = mk3(bd[pc], bd[n + pc], bd[2 * n + pc]);
        if (DAMP) {
            const int r = s.rod_of[pc];
            const int64_t R = s.field.n_rods;
            dm.gr = s.bond_g[r];
            dm.gs = s.bond_g[R + r];
            dm.gt = s.bond_g[2 * R + r];
            dm.gb = s.bond_g[3 * R + r];
            dm.g0 = hist_rate[pc];
            dm.p0 = hist_rate[n + pc];
            dm.t0 = hist_rate[2 * n + pc];
        }
        b = bond_eval<ENERGY, DAMP>(x, xn, q, qn, rih, bd[3 * n + pc], bd[4 * n + pc], bd[5 * n + pc],
                                    bd[6 * n + pc], bd[7 * n + pc], dm);
        // lane 0 repeats the bond of lane 30 of the previous warp: lanes
        // 1..30 own the record
        if (DAMP && lane >= 1 && (s.count_step || isnan(hist_out[pc]))) {
            hist_out[pc] = b.gamma;
            hist_out[n + pc] = b.psi;
            hist_out[2 * n + pc] = b.theta;
        }
    }
    // bond p-1 acts on p as its particle 2: f2 = -f1, tau2
    d3 f_prev = shfl_up3(b.f1);
    d3 t2_prev = shfl_up3(b.t2);

    if (!valid || lane == 0 || lane == 31) return;

    d3 F = b.f1 - f_prev;
    d3 T = b.t1 + t2_prev;

    // dipole in space: m = q m~ q*
    d3 m;
    if (MMODE == M_GIVEN) {
        m = mk3(s.m[p], s.m[n + p], s.m[2 * n + p]);
    } else {
        const d3 mb = mk3(s.m_body[p], s.m_body[n + p], s.m_body[2 * n + p]);
        m = rot(q, mb);
    }

    // external field at x_p and time t
    const Field& fd = s.field;
    const double tnow = *s.tdev;
    d3 B = mk3(fd.B[0], fd.B[1], fd.B[2]);
    if (fd.B_rod) {
        int r = s.rod_of[p];
        B = B + mk3(fd.B_rod[r], fd.B_rod[fd.n_rods + r], fd.B_rod[2 * fd.n_rods + r]);
    }
    if (fd.rot_amp != 0.0) {
        double sw, cw;
        sincos(fd.rot_omega * tnow, &sw, &cw);
        B = B + mk3(fd.e1[0], fd.e1[1], fd.e1[2]) * (fd.rot_amp * cw) +
            mk3(fd.e2[0], fd.e2[1], fd.e2[2]) * (fd.rot_amp * sw);
    }
    if (fd.has_grad) {
        d3 dx = x - mk3(fd.x0[0], fd.x0[1], fd.x0[2]);
        const double* G = fd.G;
        B = B + mk3(G[0] * dx.x + G[1] * dx.y + G[2] * dx.z, G[3] * dx.x + G[4] * dx.y + G[5] * dx.z,
                    G[6] * dx.x + G[7] * dx.y + G[8] * dx.z);
        // f = grad(m.B) = G^T m
        F = F + mk3(G[0] * m.x + G[3] * m.y + G[6] * m.z, G[1] * m.x + G[4] * m.y + G[7] * m.z,
                    G[2] * m.x + G[5] * m.y + G[8] * m.z);
    }
    T = T + cross(m, B);

    // global viscous damping with the velocities present at force time
    d3 v = mk3(s.v[p], s.v[n + p], s.v[2 * n + p]);
    d3 w = mk3(s.w[p], s.w[n + p], s.w[2 * n + p]);
    F = F - v * s.damping;
    T = T - w * s.damping;

    s.f[p] = F.x;
    s.f[n + p] = F.y;
    s.f[2 * n + p] = F.z;
    s.t[p] = T.x;
    s.t[n + p] = T.y;
    s.t[2 * n + p] = T.z;
    if (MMODE != M_GIVEN) write_orientation(s, p, x, m, MMODE == M_OWN_COPIES);
    if (ENERGY) {
        // bond p's energy is owned by particle p; Zeeman U = -m.B
        s.e_part[p] = b.U;
        s.e_part[n + p] = -dot(m, B);
    }
}

// One warp per 30-particle group.  The form that runs beside the dipole
// kernel (M_GIVEN) takes a smaller grid whose blocks stay resident and loop
// over the groups; the others keep the one-pass form (no loop state to hold
// in registers).
template <bool ENERGY, int MMODE, bool DAMP>
__global__ void __launch_bounds__(256) k_bond(Sys s) {
    const int lane = threadIdx.x & 31;
    if (s.count_step && blockIdx.x == 0 && threadIdx.x == 0) *s.step_counter += 1;
    const int64_t groups = (s.n + 29) / 30;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (MMODE == M_GIVEN) {
        const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t w = w0; w < groups; w += stride) bond_warp<ENERGY, MMODE, DAMP>(s, w, lane);
    } else if (w0 < groups) {
        bond_warp<ENERGY, MMODE, DAMP>(s, w0, lane);
    }
}

// The form beside the dipole kernel (m given, no energy, no bond damping)
// with its registers capped at 112 (24 bytes of spills), so that two of its
// blocks and two of the FP32-pair dipole kernel's capped form fit an SM's
// register file together.  With bond damping the uncapped form runs.
template <bool DAMP>
__global__ void __maxnreg__(112) k_bond_beside(Sys s) {
    const int lane = threadIdx.x & 31;
    if (s.count_step && blockIdx.x == 0 && threadIdx.x == 0) *s.step_counter += 1;
    const int64_t groups = (s.n + 29) / 30;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < groups; w += stride)
        bond_warp<false, M_GIVEN, DAMP>(s, w, lane);
}

}  // namespace

cudaError_t launch_bond(const Sys& s, bool energy, bool mixed_copies, bool m_given, int grid, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    const int threads = 128;
    const int64_t warps = (s.n + 29) / 30;
    const int64_t full = (warps * 32 + threads - 1) / threads;
    const unsigned blocks = (unsigned)(grid > 0 && grid < full ? grid : full);
    const bool damp = s.hist != nullptr;
    if (m_given) {
        // only force evaluations without energy take this form
        if (energy) return cudaErrorInvalidValue;
        if (damp) k_bond<false, M_GIVEN, true><<<blocks, threads, 0, st>>>(s);
        else k_bond_beside<false><<<blocks, threads, 0, st>>>(s);
        return cudaGetLastError();
    }
    const int v = (energy ? 4 : 0) | (mixed_copies ? 2 : 0) | (damp ? 1 : 0);
    switch (v) {
        case 0: k_bond<false, M_OWN, false><<<blocks, threads, 0, st>>>(s); break;
        case 1: k_bond<false, M_OWN, true><<<blocks, threads, 0, st>>>(s); break;
        case 2: k_bond<false, M_OWN_COPIES, false><<<blocks, threads, 0, st>>>(s); break;
        case 3: k_bond<false, M_OWN_COPIES, true><<<blocks, threads, 0, st>>>(s); break;
        case 4: k_bond<true, M_OWN, false><<<blocks, threads, 0, st>>>(s); break;
        case 5: k_bond<true, M_OWN, true><<<blocks, threads, 0, st>>>(s); break;
        case 6: k_bond<true, M_OWN_COPIES, false><<<blocks, threads, 0, st>>>(s); break;
        default: k_bond<true, M_OWN_COPIES, true><<<blocks, threads, 0, st>>>(s); break;
    }
    return cudaGetLastError();
}

BlockRes bond_side_block_res(bool damp) {
    return damp ? block_res_of((const void*)k_bond<false, M_GIVEN, true>, 128, 0)
                : block_res_of((const void*)k_bond_beside<false>, 128, 0);
}

cudaError_t launch_orient(const Sys& s, bool mixed_copies, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((s.n + 255) / 256);
    if (mixed_copies) k_orient<true><<<blocks, 256, 0, st>>>(s);
    else k_orient<false><<<blocks, 256, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace bpm
