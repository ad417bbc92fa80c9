// Adjoint (reverse mode) of K velocity-Verlet steps: gradient of a loss of the
// final positions with respect to the body-frame dipoles m~ and the uniform
// field B.  The forward map is differentiated as implemented (the bond forces
// are not gradients of an energy, so the force function itself is
// differentiated, not an energy).
//
// Notation: the state at the k-th force evaluation is P_k = (x_k, q_k, vh_k,
// wh_k) (positions, orientations, and the half-step velocities that the
// damping uses); P_0 holds the initial velocities.  With F_k = Phi(P_k):
//   vh_{k+1} = vh_k + kick F_k / m,  wh_{k+1} = wh_k + kick T_k / I
//   x_{k+1} = x_k + dt vh_{k+1},     q_{k+1} = R(q_k, wh_{k+1})  (Richardson)
// with kick = dt/2 for the first step (from P_0) and dt afterwards (two half
// kicks).  Reverse step k -> k-1:
//   a(vh_k) += dt a(x_k);  (a(q_{k-1}), a(wh_k)) += VJP_R(a(q_k))
//   a(F_{k-1}) = kick a(vh_k)/m,  a(T_{k-1}) = kick a(wh_k)/I
//   then VJP_Phi at P_{k-1} adds to a(P_{k-1}), a(m~) and a(B).
// VJP_Phi: global damping; Zeeman tau = m x B and f = G^T m; the dipole
// orientation m = q m~ q*; the bond forces (forward-mode dual numbers, one
// pass per input of the bond, 14 passes); the dipole-dipole forces and
// torques (closed-form derivatives of F and H, O(N^2), no scatter).
#include <algorithm>

#include "bpm_devmath.cuh"
#include "bpm_internal.h"

// the double overloads below serve the generic templates' double instances
#pragma nv_diag_suppress 177

namespace bpm {

namespace {

// ------------------------------------------------------------------ duals
// a value and one directional derivative
struct Dual {
    double v, d;
};
__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
    const double q = a / b.v;
    return {q, -q * b.d / b.v};
}
__device__ __forceinline__ Dual tsqrt(Dual a) {
    const double s = sqrt(a.v);
    return {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};
}
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dual tatan2(Dual y, Dual x) {
    const double r2 = x.v * x.v + y.v * y.v;
    return {atan2(y.v, x.v), r2 > 0.0 ? (x.v * y.d - y.v * x.d) / r2 : 0.0};
}
__device__ __forceinline__ double tatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ Dual cst(double v, Dual) { return {v, 0.0}; }
__device__ __forceinline__ double cst(double v, double) { return v; }

template <class T>
struct V3 {
    T x, y, z;
};
template <class T>
struct Q4 {
    T w, x, y, z;
};

template <class T>
__device__ __forceinline__ V3<T> vadd(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
__device__ __forceinline__ V3<T> vsub(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S>
__device__ __forceinline__ V3<T> vscale(V3<T> a, S s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T>
__device__ __forceinline__ T vdot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
__device__ __forceinline__ V3<T> vcross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T>
__device__ __forceinline__ Q4<T> qmul_t(Q4<T> a, Q4<T> b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
template <class T>
__device__ __forceinline__ Q4<T> qconj_t(Q4<T> a) { return {a.w, -a.x, -a.y, -a.z}; }
template <class T, class S>
__device__ __forceinline__ Q4<T> qscale_t(Q4<T> a, S s) { return {a.w * s, a.x * s, a.y * s, a.z * s}; }
template <class T>
__device__ __forceinline__ T qdot_t(Q4<T> a, Q4<T> b) { return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
__device__ __forceinline__ Q4<T> qnorm_t(Q4<T> a) { return qscale_t(a, 1.0 / tsqrt(qdot_t(a, a))); }
// q v q*
template <class T>
__device__ __forceinline__ V3<T> rot_t(Q4<T> q, V3<T> v) {
    const V3<T> u = {q.x, q.y, q.z};
    const V3<T> t = vscale(vcross(u, v), 2.0);
    return vadd(vadd(v, vscale(t, q.w)), vcross(u, t));
}

// atan2(s, c)/s written through t = s^2 so that it stays smooth (and its
// derivative accurate) as s -> 0: (1/c)(1 - z/3 + z^2/5 - z^3/7), z = t/c^2,
// for z < 1e-8 (truncation below 1e-32); the exact ratio otherwise.
template <class T>
__device__ __forceinline__ T atan_ratio(T t, T c) {
    if (val(c) > 0.0 && val(t) < 1e-8 * val(c) * val(c)) {
        const T z = t / (c * c);
        return (1.0 - z * (1.0 / 3.0 - z * (1.0 / 5.0 - z * (1.0 / 7.0)))) / c;
    }
    const T s = tsqrt(t);
    return tatan2(s, c) / s;
}

// The bond model (same steps as the production bond kernel), generic in
// the scalar type: outputs f1, tau1, tau2 (f2 = -f1).
template <class T>
__device__ void bond_t(V3<T> x1, V3<T> x2, Q4<T> q1, Q4<T> q2, d3 rih_, double L, double Kr, double Ks,
                       double Kt, double Kb, V3<T>& f1, V3<T>& t1, V3<T>& t2) {
    const T z0 = cst(0.0, x1.x);
    const V3<T> rih = {cst(rih_.x, z0), cst(rih_.y, z0), cst(rih_.z, z0)};
    if (val(qdot_t(q1, q2)) < 0.0) q2 = qscale_t(q2, -1.0);
    const Q4<T> qC = qnorm_t(Q4<T>{q1.w + q2.w, q1.x + q2.x, q1.y + q2.y, q1.z + q2.z});
    const V3<T> rfO = vsub(x2, x1);
    const T rf_len = tsqrt(vdot(rfO, rfO));
    const V3<T> rf = rot_t(qconj_t(qC), rfO);
    const V3<T> rfh = vscale(rf, 1.0 / rf_len);
    V3<T> F = vscale(rfh, Kr * (rf_len - L));
    const V3<T> c = vcross(rih, rfh);
    const T g_over_s = atan_ratio(vdot(c, c), vdot(rih, rfh));
    const V3<T> gt = vscale(c, g_over_s);
    F = vadd(F, vscale(vcross(gt, rfh), Ks * rf_len));
    const V3<T> TS = vscale(gt, 0.5 * Ks * rf_len * rf_len);
    const T rl = tsqrt(vdot(rf, rf));
    Q4<T> m;
    if (val(rf.z) >= 0.0) {
        const T s = 1.0 / tsqrt(2.0 * rl * (rl + rf.z));
        m = {(rl + rf.z) * s, -rf.y * s, rf.x * s, z0};
    } else {
        const T s = 1.0 / tsqrt(2.0 * rl * (rl - rf.z));
        m = {-rf.y * s, (rl - rf.z) * s, z0, rf.x * s};
    }
    const Q4<T> u0 = qmul_t(qconj_t(qC), q2);
    const Q4<T> u = qmul_t(qmul_t(qconj_t(m), u0), m);
    const T tn = 1.0 / tsqrt(u.w * u.w + u.z * u.z);
    const T tw = u.w * tn, tz = u.z * tn;
    const T psi = 2.0 * tatan2(tz, tw) - 2.0 * tatan2(-tz, tw);
    const Q4<T> uu = qmul_t(u, u);
    const Q4<T> t2c = {tw, z0, z0, -tz};
    Q4<T> b = qmul_t(qmul_t(t2c, uu), t2c);
    if (val(b.w) < 0.0) b = qscale_t(b, -1.0);
    const V3<T> bv = {b.x, b.y, b.z};
    // theta b^ = (theta / |b_v|) b_v with theta = 2 atan2(|b_v|, b_w)
    const T th_over_s = 2.0 * atan_ratio(vdot(bv, bv), b.w);
    V3<T> TBT = vscale(bv, Kb * th_over_s);
    TBT.z = TBT.z + Kt * psi;
    const Q4<T> qCm = qmul_t(qC, m);
    f1 = rot_t(qC, F);
    const V3<T> TSo = rot_t(qC, TS);
    const V3<T> TBTo = rot_t(qCm, TBT);
    t1 = vadd(TSo, TBTo);
    t2 = vsub(TSo, TBTo);
}

template <class T>
__device__ Q4<T> richardson_t(Q4<T> q, V3<T> w, double dt) {
    const T z0 = cst(0.0, q.w);
    const Q4<T> W = {z0, w.x, w.y, w.z};
    const Q4<T> qd = qscale_t(qmul_t(W, q), 0.5);
    const Q4<T> q1 = qnorm_t(Q4<T>{q.w + qd.w * dt, q.x + qd.x * dt, q.y + qd.y * dt, q.z + qd.z * dt});
    const double h = 0.5 * dt;
    const Q4<T> qh = qnorm_t(Q4<T>{q.w + qd.w * h, q.x + qd.x * h, q.y + qd.y * h, q.z + qd.z * h});
    const Q4<T> qhd = qscale_t(qmul_t(W, qh), 0.5);
    const Q4<T> q2 = qnorm_t(Q4<T>{qh.w + qhd.w * h, qh.x + qhd.x * h, qh.y + qhd.y * h, qh.z + qhd.z * h});
    return qnorm_t(Q4<T>{2.0 * q2.w - q1.w, 2.0 * q2.x - q1.x, 2.0 * q2.y - q1.y, 2.0 * q2.z - q1.z});
}

__device__ __forceinline__ Dual dv(double v, bool on) { return {v, on ? 1.0 : 0.0}; }

__device__ __forceinline__ d3 ld3(const double* a, int64_t n, int64_t i) { return mk3(a[i], a[n + i], a[2 * n + i]); }
__device__ __forceinline__ void st3(double* a, int64_t n, int64_t i, d3 v) {
    a[i] = v.x;
    a[n + i] = v.y;
    a[2 * n + i] = v.z;
}
__device__ __forceinline__ void add3(double* a, int64_t n, int64_t i, d3 v) {
    a[i] += v.x;
    a[n + i] += v.y;
    a[2 * n + i] += v.z;
}

// ------------------------------------------------------------------ kernels
// m = q m~ q* at the snapshot and mu = lambda_tau x m
__global__ void k_adj_orient(Sys s, AdjBuf a) {
    const int64_t n = s.n, i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dq q = dq{s.q[i], s.q[n + i], s.q[2 * n + i], s.q[3 * n + i]};
    const d3 m = rot(q, ld3(s.m_body, n, i));
    st3(a.m, n, i, m);
    st3(a.mu, n, i, cross(ld3(a.aT, n, i), m));
}

// gradient of phi = lam.F(r; m1, m2) + mu.H(r; m2) with
// F = 3c[(a m2 + b m1 + d r)/r^5 - 5ab r/r^7], H = c[3b r/r^5 - m2/r^3]
// Powers of 1/r shared by the two sides of a pair
struct RPow {
    double ri2, ri3, ri5, ri7, ri9;
};

__device__ __forceinline__ RPow rpowers(double r2) {
    RPow P;
    const double ri = rsqrt_nr(r2);
    P.ri2 = ri * ri;
    P.ri3 = P.ri2 * ri;
    P.ri5 = P.ri3 * P.ri2;
    P.ri7 = P.ri5 * P.ri2;
    P.ri9 = P.ri7 * P.ri2;
    return P;
}

// Gradient of lam . F_1 + mu . H_1 (F_1, H_1: force and field on dipole 1
// at r = x_1 - x_2 from dipole 2) with respect to r, m1 and m2, given
// a = m1.r, b = m2.r, d = m1.m2; H = the field H_1 itself.
//
// Every gradient is a combination of the vectors m1, m2, lam, mu and r, and
// the three share most of their scalar coefficients.  With k = 3c,
// Lv = lam.v, Mv = mu.v and P = a Lm2 + b Lm1 + d Lr:
//   d/dr  = k [C1 m1 + C2 m2 + (d/r^5 - 5ab/r^7) lam + (b/r^5) mu + Cr r]
//   d/dm1 = k [C1 r + (b/r^5) lam + (Lr/r^5) m2]
//   d/dm2 = k [(a/r^5) lam + C2 r + (Lr/r^5) m1] - (c/r^3) mu
//   H     = k (b/r^5) r - (c/r^3) m2
// with C1 = Lm2/r^5 - 5 b Lr/r^7, C2 = (Lm1 + Mr)/r^5 - 5 a Lr/r^7 and
// Cr = Mm2/r^5 - 5 (P + b Mr)/r^7 + 35 a b Lr/r^9.
__device__ __forceinline__ void dip_grad(d3 r, const RPow& P, double a, double b, double d, d3 m1, d3 m2, d3 lam,
                                         d3 mu, double c, d3& gr, d3& gm1, d3& gm2, d3& H) {
    const double ri3 = P.ri3, ri5 = P.ri5, ri7 = P.ri7, ri9 = P.ri9;
    const double Lm1 = dot(lam, m1), Lm2 = dot(lam, m2), Lr = dot(lam, r);
    const double Mr = dot(mu, r), Mm2 = dot(mu, m2);
    const double k = 3.0 * c;
    const double t5 = 5.0 * ri7;
    const double ab = a * b;
    const double Pl = a * Lm2 + b * Lm1 + d * Lr;
    const double C1 = Lm2 * ri5 - (b * Lr) * t5;
    const double C2 = (Lm1 + Mr) * ri5 - (a * Lr) * t5;
    const double Clam = d * ri5 - ab * t5;
    const double Cmu = b * ri5;
    const double Cr = Mm2 * ri5 - (Pl + b * Mr) * t5 + 35.0 * ab * Lr * ri9;
    const double Lri5 = Lr * ri5;
    const double cri3 = c * ri3;
    gr = (m1 * C1 + m2 * C2 + lam * Clam + mu * Cmu + r * Cr) * k;
    gm1 = (r * C1 + lam * Cmu + m2 * Lri5) * k;
    gm2 = (lam * (a * ri5) + r * C2 + m1 * Lri5) * k - mu * cri3;
    H = r * (k * Cmu) - m2 * cri3;
}

// dipole VJP: for particle p, both ordered pairs (p, j) and (j, p); no
// scatter.  blockIdx.y selects one of gridDim.y chunks of the j range; chunk
// c writes its sums to dpart[c][6][N] (d/dx 3, d/dm 3).
__global__ void __launch_bounds__(128) k_adj_dipole(Sys s, AdjBuf a, int per_rod, const int64_t* rod_off) {
    const int64_t n = s.n, p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t b0 = 0, b1 = n;
    if (per_rod) {
        const int r = s.rod_of[p];
        b0 = rod_off[r];
        b1 = rod_off[r + 1];
    }
    const int64_t S = gridDim.y, chunk = (b1 - b0 + S - 1) / S;
    const int64_t j0 = min(b1, b0 + (int64_t)blockIdx.y * chunk), j1 = min(b1, j0 + chunk);
    const d3 xp = ld3(s.x, n, p), mp = ld3(a.m, n, p);
    const d3 lFp = ld3(a.aF, n, p), mup = ld3(a.mu, n, p), lTp = ld3(a.aT, n, p);
    d3 gx = mk3(0, 0, 0), gm = mk3(0, 0, 0), Hs = mk3(0, 0, 0);
    for (int64_t j = j0; j < j1; ++j) {
        if (j == p) continue;
        const d3 xj = ld3(s.x, n, j), mj = ld3(a.m, n, j);
        const d3 r = xp - xj;
        // shared by both sides: |r|, its powers, m_p.r, m_j.r, m_p.m_j
        const RPow P = rpowers(dot(r, r));
        const double ap = dot(mp, r), bj = dot(mj, r), dd = dot(mp, mj);
        d3 gr, gm1, gm2, H;
        dip_grad(r, P, ap, bj, dd, mp, mj, lFp, mup, s.c, gr, gm1, gm2, H);
        gx = gx + gr;
        gm = gm + gm1;
        Hs = Hs + H;
        // the pair seen from j: r -> -r, so m_j.(-r) = -bj and m_p.(-r) = -ap
        d3 gr2, gm1b, gm2b, H2;
        dip_grad(-r, P, -bj, -ap, dd, mj, mp, ld3(a.aF, n, j), ld3(a.mu, n, j), s.c, gr2, gm1b, gm2b, H2);
        gx = gx - gr2;
        gm = gm + gm2b;
    }
    // torque tau_p = m_p x H_p: d/dm_p = H_p x lambda_tau
    gm = gm + cross(Hs, lTp);
    double* D = a.dpart + (int64_t)blockIdx.y * 6 * n;
    st3(D, n, p, gx);
    st3(D + 3 * n, n, p, gm);
}

// Symmetric dipole VJP: each unordered pair {i, j} evaluated once, both of
// its sides (dipole i in the field of j and dipole j in the field of i):
//   d/dx_i = -d/dx_j = gr - gr',  d/dm_i = gm1 + gm2',  d/dm_j = gm2 + gm1'
// (primes: the side of j, evaluated at -r).  Items are pairs of 32-particle
// tiles I <= J, one warp each; lane l holds i = 32 I + l and, at step s, the
// accumulator of j = 32 J + (l + s) mod 32, which then moves to lane l - 1
// by shuffles, so after 32 steps every j accumulator is home and no
// floating-point reduction is needed.  A diagonal tile evaluates its 32 x 31
// ordered pairs on the i side only.  i-side sums go to slot J and j-side
// sums to slot I: each particle gets exactly one partial per partner tile,
// whatever the schedule.  Missing j of a ragged last tile sit far away with
// zero moment and adjoints, which makes every term they contribute zero.
struct AdjAcc {
    d3 gx, gm, H;
};

__device__ __forceinline__ d3 shfl3(d3 v, int src) {
    return mk3(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
               __shfl_sync(0xffffffffu, v.z, src));
}

// Both sides of the pair (i, j) at once: the two dip_grad evaluations
// (side i: m1 = m_i, m2 = m_j, r; side j: m1 = m_j, m2 = m_i, -r, so
// a' = -b, b' = -a; primes mark lam_j, mu_j) regrouped by vector.  With
// k = 3c, dlam = lam_i - lam_j and the coefficients C1, C2, Clam, Cr of
// dip_grad for each side:
//   d/dx_i = -d/dx_j = K1 m_i + K2 m_j + KL dlam + KMi mu_i + KMj mu_j + KR r
//   d/dm_i += K1 r + KMi dlam + KLr m_j - (c/r^3) mu_j
//   d/dm_j += K2 r + KMj dlam + KLr m_i - (c/r^3) mu_i
//   H_i = KMi r - (c/r^3) m_j,  H_j = KMj r - (c/r^3) m_i
// with K1 = k (C1 - C2'), K2 = k (C2 - C1'), KL = k Clam (the same on both
// sides), KMi = k b/r^5, KMj = k a/r^5, KR = k (Cr + Cr'),
// KLr = k (Lr + Lr')/r^5.  About 180 FP64 operations per pair instead of the
// 262 of two dip_grad calls.  lmi, lmj: lam . m of each particle.
template <bool DIAG>
__device__ __forceinline__ void dip_pair(d3 r, const RPow& P, d3 mi, d3 mj, d3 li, d3 lj, d3 ui, d3 uj, double lmi,
                                         double lmj, double c, AdjAcc& ai, AdjAcc& aj) {
    const double ri3 = P.ri3, ri5 = P.ri5, ri7 = P.ri7, ri9 = P.ri9;
    const double a = dot(mi, r), b = dot(mj, r), d = dot(mi, mj);
    const double k = 3.0 * c;
    const double t5 = 5.0 * ri7;
    const double ab = a * b;
    const double Lm2 = dot(li, mj), Lr = dot(li, r), Mr = dot(ui, r), Mm2 = dot(ui, mj);
    const double Lm2p = dot(lj, mi), Lrp = -dot(lj, r), Mrp = -dot(uj, r), Mm2p = dot(uj, mi);
    const double C1 = Lm2 * ri5 - (b * Lr) * t5;
    const double C2 = (lmi + Mr) * ri5 - (a * Lr) * t5;
    const double C1p = Lm2p * ri5 + (a * Lrp) * t5;
    const double C2p = (lmj + Mrp) * ri5 + (b * Lrp) * t5;
    const double Clam = d * ri5 - ab * t5;
    const double Pl = a * Lm2 + b * lmi + d * Lr;
    const double Plp = -b * Lm2p - a * lmj + d * Lrp;
    const double abr9 = 35.0 * ab * ri9;
    const double Cr = Mm2 * ri5 - (Pl + b * Mr) * t5 + abr9 * Lr;
    const double Crp = Mm2p * ri5 - (Plp - a * Mrp) * t5 + abr9 * Lrp;
    const double K1 = k * (C1 - C2p), K2 = k * (C2 - C1p), KL = k * Clam;
    const double KMi = k * (b * ri5), KMj = k * (a * ri5);
    const double KR = k * (Cr + Crp), KLr = k * ((Lr + Lrp) * ri5), cr3 = c * ri3;
    const d3 dl = li - lj;
    const d3 gd = mi * K1 + mj * K2 + dl * KL + ui * KMi + uj * KMj + r * KR;
    ai.gx = ai.gx + gd;
    ai.gm = ai.gm + r * K1 + dl * KMi + mj * KLr - uj * cr3;
    ai.H = ai.H + r * KMi - mj * cr3;
    if (!DIAG) {
        aj.gx = aj.gx - gd;
        aj.gm = aj.gm + r * K2 + dl * KMj + mi * KLr - ui * cr3;
        aj.H = aj.H + r * KMj - mi * cr3;
    }
}

template <bool DIAG>
__device__ __forceinline__ void adj_tile(double c, d3 xi, d3 mi, d3 li, d3 ui, const double (*sj)[32], int lane,
                                         AdjAcc& ai, AdjAcc& aj) {
    const int from = (lane + 1) & 31;
    const double lmi = dot(li, mi);
    for (int step = DIAG ? 1 : 0; step < 32; ++step) {
        const int o = (lane + step) & 31;
        const d3 xj = mk3(sj[0][o], sj[1][o], sj[2][o]), mj = mk3(sj[3][o], sj[4][o], sj[5][o]);
        const d3 lj = mk3(sj[6][o], sj[7][o], sj[8][o]), uj = mk3(sj[9][o], sj[10][o], sj[11][o]);
        const d3 r = xi - xj;
        const RPow P = rpowers(dot(r, r));
        dip_pair<DIAG>(r, P, mi, mj, li, lj, ui, uj, lmi, sj[12][o], c, ai, aj);
        if (!DIAG) {
            aj.gx = shfl3(aj.gx, from);
            aj.gm = shfl3(aj.gm, from);
            aj.H = shfl3(aj.H, from);
        }
    }
}

__global__ void __launch_bounds__(128) k_adj_dipole_sym(Sys s, AdjBuf a, int64_t n_items) {
    __shared__ double sjw[4][13][32];
    const int64_t n = s.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double(*sj)[32] = sjw[warp];
    const int64_t n_warps = (int64_t)gridDim.x * 4;
    for (int64_t t = (int64_t)blockIdx.x * 4 + warp; t < n_items; t += n_warps) {
        // t = J (J + 1) / 2 + I with 0 <= I <= J
        int64_t J = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (J * (J + 1) / 2 > t) --J;
        while ((J + 1) * (J + 2) / 2 <= t) ++J;
        const int64_t I = t - J * (J + 1) / 2;
        const int64_t i = 32 * I + lane, j = 32 * J + lane;
        const bool iv = i < n, jv = j < n;
        const int64_t ic = iv ? i : 0;
        const d3 xi = ld3(s.x, n, ic), mi = ld3(a.m, n, ic), li = ld3(a.aF, n, ic), ui = ld3(a.mu, n, ic);
        __syncwarp();
        if (jv) {
            const d3 v[4] = {ld3(s.x, n, j), ld3(a.m, n, j), ld3(a.aF, n, j), ld3(a.mu, n, j)};
            for (int k = 0; k < 4; ++k) {
                sj[3 * k][lane] = v[k].x;
                sj[3 * k + 1][lane] = v[k].y;
                sj[3 * k + 2][lane] = v[k].z;
            }
            sj[12][lane] = dot(v[2], v[1]);  // lam . m
        } else {
            for (int k = 0; k < 13; ++k) sj[k][lane] = k < 3 ? 1e15 : 0.0;
        }
        __syncwarp();
        const d3 z = mk3(0, 0, 0);
        AdjAcc ai{z, z, z}, aj{z, z, z};
        if (I == J)
            adj_tile<true>(s.c, xi, mi, li, ui, sj, lane, ai, aj);
        else
            adj_tile<false>(s.c, xi, mi, li, ui, sj, lane, ai, aj);
        // torque tau = m x H: d/dm += H x lambda_tau
        if (iv) {
            double* D = a.dpart + J * 6 * n;
            st3(D, n, i, ai.gx);
            st3(D + 3 * n, n, i, ai.gm + cross(ai.H, ld3(a.aT, n, i)));
        }
        if (I != J && jv) {
            double* D = a.dpart + I * 6 * n;
            st3(D, n, j, aj.gx);
            st3(D + 3 * n, n, j, aj.gm + cross(aj.H, ld3(a.aT, n, j)));
        }
    }
}

// bond VJP: for bond p -> p+1, the gradient of
// (lam_f1 - lam_f2).f1 + lam_t1.tau1 + lam_t2.tau2 with respect to
// (x1, q1) -> bL[.][p] and (x2, q2) -> bR[.][p], by 14 forward-mode passes,
// one thread per (bond, pass): pass k seeds one of x1 (0..2), x2 (3..5),
// q1 (6..9), q2 (10..13).
__global__ void __launch_bounds__(128) k_adj_bond(Sys s, AdjBuf a) {
    const int64_t n = s.n, t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 14 * n) return;
    const int64_t p = t / 14;
    const int k = (int)(t - 14 * p);
    double g = 0.0;
    if ((s.flags[p] & F_BOND_RIGHT) && p + 1 < n) {
        const int64_t p2 = p + 1;
        const d3 x1 = ld3(s.x, n, p), x2 = ld3(s.x, n, p2);
        const double q1[4] = {s.q[p], s.q[n + p], s.q[2 * n + p], s.q[3 * n + p]};
        const double q2[4] = {s.q[p2], s.q[n + p2], s.q[2 * n + p2], s.q[3 * n + p2]};
        const d3 Lf = ld3(a.aF, n, p) - ld3(a.aF, n, p2);
        const d3 Lt1 = ld3(a.aT, n, p), Lt2 = ld3(a.aT, n, p2);
        const double* bd = s.bond;
        const d3 rih = mk3(bd[p], bd[n + p], bd[2 * n + p]);
        const double L = bd[3 * n + p], Kr = bd[4 * n + p], Ks = bd[5 * n + p], Kt = bd[6 * n + p],
                     Kb = bd[7 * n + p];
        const V3<Dual> X1 = {dv(x1.x, k == 0), dv(x1.y, k == 1), dv(x1.z, k == 2)};
        const V3<Dual> X2 = {dv(x2.x, k == 3), dv(x2.y, k == 4), dv(x2.z, k == 5)};
        const Q4<Dual> Q1 = {dv(q1[0], k == 6), dv(q1[1], k == 7), dv(q1[2], k == 8), dv(q1[3], k == 9)};
        const Q4<Dual> Q2 = {dv(q2[0], k == 10), dv(q2[1], k == 11), dv(q2[2], k == 12), dv(q2[3], k == 13)};
        V3<Dual> f1, t1, t2;
        bond_t<Dual>(X1, X2, Q1, Q2, rih, L, Kr, Ks, Kt, Kb, f1, t1, t2);
        g = Lf.x * f1.x.d + Lf.y * f1.y.d + Lf.z * f1.z.d + Lt1.x * t1.x.d + Lt1.y * t1.y.d + Lt1.z * t1.z.d +
            Lt2.x * t2.x.d + Lt2.y * t2.y.d + Lt2.z * t2.z.d;
    }
    // left: x1 -> bL[0..2], q1 -> bL[3..6]; right: x2 -> bR[0..2], q2 -> bR[3..6]
    if (k < 3)
        a.bL[k * n + p] = g;
    else if (k < 6)
        a.bR[(k - 3) * n + p] = g;
    else if (k < 10)
        a.bL[(3 + k - 6) * n + p] = g;
    else
        a.bR[(3 + k - 10) * n + p] = g;
}

__global__ void k_adj_phi(Sys s, AdjBuf a) {
    const int64_t n = s.n, p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double tnow = *s.tdev;
    const d3 lF = ld3(a.aF, n, p), lT = ld3(a.aT, n, p);
    const d3 m = ld3(a.m, n, p);
    const d3 xp = ld3(s.x, n, p);
    d3 gx = ld3(a.bL, n, p);
    d3 gdm = mk3(0, 0, 0);
    for (int c = 0; c < a.S; ++c) {
        const double* D = a.dpart + (int64_t)c * 6 * n;
        gx = gx + ld3(D, n, p);
        gdm = gdm + ld3(D + 3 * n, n, p);
    }
    double gq[4] = {a.bL[3 * n + p], a.bL[4 * n + p], a.bL[5 * n + p], a.bL[6 * n + p]};
    if (p > 0) {
        gx = gx + ld3(a.bR, n, p - 1);
        for (int c = 0; c < 4; ++c) gq[c] += a.bR[(3 + c) * n + p - 1];
    }
    // field at x_p, time tnow
    const Field& fd = s.field;
    d3 B = mk3(fd.B[0], fd.B[1], fd.B[2]);
    if (fd.B_rod) {
        const int r = s.rod_of[p];
        B = B + mk3(fd.B_rod[r], fd.B_rod[fd.n_rods + r], fd.B_rod[2 * fd.n_rods + r]);
    }
    if (fd.rot_amp != 0.0) {
        double sw, cw;
        sincos(fd.rot_omega * tnow, &sw, &cw);
        B = B + mk3(fd.e1[0], fd.e1[1], fd.e1[2]) * (fd.rot_amp * cw) + mk3(fd.e2[0], fd.e2[1], fd.e2[2]) * (fd.rot_amp * sw);
    }
    const double* G = fd.G;
    // a(m) = dipole part + Zeeman: B x lam_tau + G lam_F
    d3 gm = gdm + cross(B, lT);
    const d3 lxm = cross(lT, m);
    if (fd.has_grad) {
        const d3 dx = xp - mk3(fd.x0[0], fd.x0[1], fd.x0[2]);
        B = B + mk3(G[0] * dx.x + G[1] * dx.y + G[2] * dx.z, G[3] * dx.x + G[4] * dx.y + G[5] * dx.z,
                    G[6] * dx.x + G[7] * dx.y + G[8] * dx.z);
        gm = gdm + cross(B, lT) +
             mk3(G[0] * lF.x + G[1] * lF.y + G[2] * lF.z, G[3] * lF.x + G[4] * lF.y + G[5] * lF.z,
                 G[6] * lF.x + G[7] * lF.y + G[8] * lF.z);
        // d/dx of lam_tau.(m x G x) = G^T (lam_tau x m)
        gx = gx + mk3(G[0] * lxm.x + G[3] * lxm.y + G[6] * lxm.z, G[1] * lxm.x + G[4] * lxm.y + G[7] * lxm.z,
                      G[2] * lxm.x + G[5] * lxm.y + G[8] * lxm.z);
    }
    // m = q m~ q*: a(m~) += R(q)^T a(m); a(q) by 4 forward passes
    const double qv[4] = {s.q[p], s.q[n + p], s.q[2 * n + p], s.q[3 * n + p]};
    const d3 mb = ld3(s.m_body, n, p);
    for (int k = 0; k < 4; ++k) {
        const Q4<Dual> Q = {dv(qv[0], k == 0), dv(qv[1], k == 1), dv(qv[2], k == 2), dv(qv[3], k == 3)};
        const V3<Dual> MB = {{mb.x, 0.0}, {mb.y, 0.0}, {mb.z, 0.0}};
        const V3<Dual> mm = rot_t(Q, MB);
        gq[k] += gm.x * mm.x.d + gm.y * mm.y.d + gm.z * mm.z.d;
    }
    const dq q = dq{qv[0], qv[1], qv[2], qv[3]};
    add3(a.amb, n, p, rot_inv(q, gm));
    add3(a.aB, n, p, lxm);
    // state adjoints
    add3(a.ax, n, p, gx);
    for (int c = 0; c < 4; ++c) a.aq[c * n + p] += gq[c];
    // damping f -= g vh, tau -= g wh
    add3(a.av, n, p, lF * (-s.damping));
    add3(a.aw, n, p, lT * (-s.damping));
}

// reverse of the update P_{k-1} -> P_k (Richardson by 7 forward passes);
// leaves a(P_{k-1}) (before VJP_Phi at P_{k-1}) and a(F_{k-1}), a(T_{k-1}).
__global__ void k_adj_update(Sys prev, Sys cur, AdjBuf a, double kick) {
    const int64_t n = prev.n, p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (prev.flags[p] & F_CLAMPED) {
        // x and q are constant; velocities and forces do not act
        for (int c = 0; c < 3; ++c) {
            a.av[c * n + p] = 0.0;
            a.aw[c * n + p] = 0.0;
            a.aF[c * n + p] = 0.0;
            a.aT[c * n + p] = 0.0;
        }
        return;
    }
    const double dt = prev.dt;
    const d3 ax = ld3(a.ax, n, p);
    const d3 avh = ld3(a.av, n, p) + ax * dt;
    const double aqk[4] = {a.aq[p], a.aq[n + p], a.aq[2 * n + p], a.aq[3 * n + p]};
    const double q0[4] = {prev.q[p], prev.q[n + p], prev.q[2 * n + p], prev.q[3 * n + p]};
    const d3 wk = ld3(cur.w, n, p);
    double g[7];
    for (int k = 0; k < 7; ++k) {
        const Q4<Dual> Q = {dv(q0[0], k == 0), dv(q0[1], k == 1), dv(q0[2], k == 2), dv(q0[3], k == 3)};
        const V3<Dual> Wd = {dv(wk.x, k == 4), dv(wk.y, k == 5), dv(wk.z, k == 6)};
        const Q4<Dual> r = richardson_t<Dual>(Q, Wd, dt);
        g[k] = aqk[0] * r.w.d + aqk[1] * r.x.d + aqk[2] * r.y.d + aqk[3] * r.z.d;
    }
    const d3 awh = ld3(a.aw, n, p) + mk3(g[4], g[5], g[6]);
    for (int c = 0; c < 4; ++c) a.aq[c * n + p] = g[c];
    st3(a.av, n, p, avh);
    st3(a.aw, n, p, awh);
    const double mass = prev.mass[p], I = prev.inertia[p];
    st3(a.aF, n, p, avh * (kick / mass));
    st3(a.aT, n, p, awh * (kick / I));
}

// one block: deterministic sum of the per-particle B-gradient pieces
__global__ void __launch_bounds__(1024) k_adj_reduce_B(const double* aB, int64_t n, double* out) {
    __shared__ double red[1024];
    for (int c = 0; c < 3; ++c) {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += aB[c * n + i];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = red[0];
        __syncthreads();
    }
}

inline unsigned grid_of(int64_t n) { return (unsigned)((n + 127) / 128); }

}  // namespace

cudaError_t launch_adj_phi(const Sys& s, const AdjBuf& a, int dipole_mode, const int64_t* rod_off,
                           cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    const unsigned g = grid_of(s.n);
    k_adj_orient<<<g, 128, 0, st>>>(s, a);
    if (dipole_mode != BPM_DIPOLE_OFF && a.sym && a.ffbuf) {
        const int64_t T = (s.n + 31) / 32;
        cudaError_t e = launch_adj_dipole_sym_ff(s, a, T * (T + 1) / 2, st);
        if (e != cudaSuccess) return e;
    } else if (dipole_mode != BPM_DIPOLE_OFF && a.sym) {
        // a static round-robin of the tile pairs over the warps, with the
        // resident block count per SM (4 warps each, one per SM partition)
        // that best evens out the items per warp; ties go to more warps
        const int64_t T = (s.n + 31) / 32, items = T * (T + 1) / 2;
        static int n_sm = 0, per_sm = 0;
        if (n_sm == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_dipole_sym, 128, 0);
            per_sm = std::max(1, per_sm);
        }
        int64_t best = 1;
        double best_eff = -1.0;
        for (int b = 1; b <= per_sm; ++b) {
            const int64_t blocks = std::min<int64_t>((int64_t)n_sm * b, (items + 3) / 4);
            const int64_t rounds = (items + 4 * blocks - 1) / (4 * blocks);
            const double eff = (double)items / (double)(4 * blocks * rounds);
            if (eff >= best_eff - 1e-9) {
                best_eff = eff;
                best = blocks;
            }
        }
        k_adj_dipole_sym<<<(unsigned)best, 128, 0, st>>>(s, a, items);
    } else if (dipole_mode != BPM_DIPOLE_OFF) {
        k_adj_dipole<<<dim3(g, a.S), 128, 0, st>>>(s, a, dipole_mode == BPM_DIPOLE_PER_ROD ? 1 : 0, rod_off);
    } else {
        cudaMemsetAsync(a.dpart, 0, 6 * (size_t)a.S * (size_t)s.n * sizeof(double), st);
    }
    k_adj_bond<<<grid_of(14 * s.n), 128, 0, st>>>(s, a);
    k_adj_phi<<<g, 128, 0, st>>>(s, a);
    return cudaGetLastError();
}

cudaError_t launch_adj_update(const Sys& prev, const Sys& cur, const AdjBuf& a, double kick, cudaStream_t st) {
    if (prev.n == 0) return cudaSuccess;
    k_adj_update<<<grid_of(prev.n), 128, 0, st>>>(prev, cur, a, kick);
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce_B(const double* aB, int64_t n, double* out, cudaStream_t st) {
    k_adj_reduce_B<<<1, 1024, 0, st>>>(aB, n, out);
    return cudaGetLastError();
}

}  // namespace bpm
