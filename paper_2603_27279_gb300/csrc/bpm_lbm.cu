// Lattice Boltzmann fluid (D3Q19, BGK, Guo forcing) on a periodic lattice
// and its penalty immersed-boundary coupling to the particles (Methods,
// "Lattice Boltzmann method", "Immersed boundary coupling").
//
// Lattice units: spacing 1, one LBM step = n_sub DEM steps = 1, density
// scale 1.  Node (i, j, k) sits at (i, j, k), index i + nx (j + ny k).  The
// stored state is the post-collision distributions f*[19][nodes]; a step
// pulls f_q(x) = f*_q(x - e_q) from the neighbours (streaming), takes
// rho = sum f, rho u = sum f e + F/2 with F = body force + particle reaction,
// and writes f*_new = f - (f - f_eq)/tau + S (Guo's source) into the other
// buffer, zeroing the reaction field as it reads it.  One thread per node,
// x fastest, so every pull of a warp is a contiguous (shifted) run.
//
// Storage: FP64 for FP64 handles; for mixed handles the deviation
// f - w_q (w_q = the rest-state equilibrium at rho = 1) in FP32, with the
// collision and the reaction field in FP32 (halving the traffic of an
// HBM-bound kernel, keeping the small deviations at FP32 relative precision,
// and leaving the 1/64-rate FP64 pipe idle).
//
// Coupling: the fluid velocity is interpolated at the particles once per
// cycle with Peskin's four-point delta, from the streamed distributions (the
// interpolation kernel pulls the 19 values of each of the 64 support nodes);
// the penalty force m_p (U - v_p) is added to every force evaluation, and the
// time stepping's evaluations spread -F_p / n_sub onto the reaction field
// with the same weights (atomics: sums are reproducible to rounding, not
// bitwise).
#include "bpm_devmath.cuh"
#include "bpm_ff.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

// D3Q19: rest, 6 faces, 12 edges
__device__ __constant__ int c_E[19][3] = {
    {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

// the same velocities as compile-time functions (fold to constants after
// unrolling over q)
__host__ __device__ constexpr int ex(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
           : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
           : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
           : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}

__host__ __device__ constexpr double wq(int q) { return q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <class T>
struct Store;
template <>
struct Store<double> {
    __device__ static double load(const double* p, int q) { return *p; }
    __device__ static void store(double* p, int q, double v) { *p = v; }
};
template <>
struct Store<float> {
    // deviation from the rest equilibrium w_q
    __device__ static double load(const float* p, int q) { return (double)*p + wq(q); }
    __device__ static void store(float* p, int q, double v) { *p = __double2float_rn(v - wq(q)); }
};

// One step of node n.  The kernel works on the stored values s_q: f_q for
// FP64 storage, f_q - w_q for FP32 storage (DEV).  With sum w = 1 and
// sum w e = 0: rho = sum s (+ 1 when DEV), rho u = sum s e + F/2, and the
// stored equilibrium is s_eq = w (sum s + rho (3 eu + 9/2 eu^2 - 3/2 u.u)),
// so FP32 arithmetic only ever sees the small deviations.
//
// The update s - (s - s_eq) / tau + S is evaluated as
//   (1 - omega) s + A_c + eu (B_c + C_c eu) + eF (G_c + H_c eu),
// with, per weight class c: A_c = w_c (omega (sum s - 3/2 rho u.u) - 3 gfac u.F),
// B_c = 3 omega rho w_c, C_c = 9/2 omega rho w_c, G_c = 3 gfac w_c,
// H_c = 9 gfac w_c (omega = 1/tau, gfac = 1 - 1/(2 tau)): five fused
// multiply-adds per direction on GB300's narrow FP64 pipe.
__host__ __device__ constexpr int wcls(int q) { return q == 0 ? 0 : (q < 7 ? 1 : 2); }

template <class T>
__global__ void __launch_bounds__(256) k_lbm_step(const T* __restrict__ fin, T* __restrict__ fout, T* Fr,
                                                  Lbm L) {
    using R = T;  // arithmetic type = storage type
    constexpr bool DEV = sizeof(T) == 4;
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    const int i = (int)(n % L.nx);
    const int64_t r = n / L.nx;
    const int j = (int)(r % L.ny), k = (int)(r / L.ny);
    R f[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int si = wrapi(i - ex(q), L.nx), sj = wrapi(j - ey(q), L.ny), sk = wrapi(k - ez(q), L.nz);
        f[q] = fin[(int64_t)q * nodes + si + (int64_t)L.nx * (sj + (int64_t)L.ny * sk)];
    }
    R s0 = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        s0 += f[q];
        if (ex(q)) mx += ex(q) > 0 ? f[q] : -f[q];
        if (ey(q)) my += ey(q) > 0 ? f[q] : -f[q];
        if (ez(q)) mz += ez(q) > 0 ? f[q] : -f[q];
    }
    const R rho = DEV ? (R)1 + s0 : s0;
    const R Fr0 = Fr[n], Fr1 = Fr[nodes + n], Fr2 = Fr[2 * nodes + n];
    Fr[n] = 0;
    Fr[nodes + n] = 0;
    Fr[2 * nodes + n] = 0;
    // constants in the storage type, with no FP64 conversion in the FP32 path
    R bx, by, bz, omega, gfac;
    if (DEV) {
        bx = (R)L.bodyf[0], by = (R)L.bodyf[1], bz = (R)L.bodyf[2], omega = (R)L.omegaf, gfac = (R)L.gfacf;
    } else {
        bx = (R)L.body[0], by = (R)L.body[1], bz = (R)L.body[2], omega = (R)L.omega, gfac = (R)L.gfac;
    }
    const R Fx = bx + Fr0, Fy = by + Fr1, Fz = bz + Fr2;
    R irho;
    if (DEV)
        irho = (R)1 / rho;
    else
        irho = (R)rcp_nr((double)rho);
    const R ux = fma((R)0.5, Fx, mx) * irho, uy = fma((R)0.5, Fy, my) * irho, uz = fma((R)0.5, Fz, mz) * irho;
    const R uu = fma(ux, ux, fma(uy, uy, uz * uz));
    const R uF = fma(ux, Fx, fma(uy, Fy, uz * Fz));
    const R om1 = (R)1 - omega;
    const R K = fma(omega, fma((R)-1.5 * rho, uu, s0), (R)-3 * gfac * uF);
    const R orho = omega * rho;
    R A[3], B[3], C[3], G[3], H[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R w = (R)(c == 0 ? 1.0 / 3.0 : (c == 1 ? 1.0 / 18.0 : 1.0 / 36.0));
        A[c] = w * K;
        B[c] = ((R)3 * w) * orho;
        C[c] = ((R)4.5 * w) * orho;
        G[c] = ((R)3 * w) * gfac;
        H[c] = ((R)9 * w) * gfac;
    }
    fout[n] = fma(om1, f[0], A[0]);
#pragma unroll
    for (int q = 1; q < 19; ++q) {
        const int c = wcls(q);
        R eu = 0, eF = 0;
        if (ex(q)) { eu += ex(q) > 0 ? ux : -ux; eF += ex(q) > 0 ? Fx : -Fx; }
        if (ey(q)) { eu += ey(q) > 0 ? uy : -uy; eF += ey(q) > 0 ? Fy : -Fy; }
        if (ez(q)) { eu += ez(q) > 0 ? uz : -uz; eF += ez(q) > 0 ? Fz : -Fz; }
        R o = fma(om1, f[q], A[c]);
        o = fma(eu, fma(C[c], eu, B[c]), o);
        o = fma(eF, fma(H[c], eu, G[c]), o);
        fout[(int64_t)q * nodes + n] = o;
    }
}

// The step of k_lbm_step for FP64 storage with float-float arithmetic
// (BPM_FF handles).  Each pulled f_q gives its deviation s_q = f_q - w_q in
// FP64 (exact while f_q stays within a factor 2 of w_q) and then as a
// float-float value: about 48 significant bits on a number of order 1e-3,
// finer than FP64's rounding of f_q itself.  The deviation form of the
// update above runs in float-float on the FP32 pipe, and the new f_q is
// w_q + s_new in FP64.  The FP64 pipe then carries about 60 operations per
// node instead of about 217.
__device__ __forceinline__ ffm::ffv wff(int c) {
    // 1/3, 1/18, 1/36 as float-float constants
    return c == 0 ? ffm::ffv{3.333333433e-01f, -9.934107759e-09f}
                  : (c == 1 ? ffm::ffv{5.555555597e-02f, -4.139211474e-10f} : ffm::ffv{2.777777798e-02f, -2.069605737e-10f});
}
__global__ void __launch_bounds__(256) k_lbm_step_ff(const double* __restrict__ fin, double* __restrict__ fout,
                                                     double* Fr, Lbm L) {
    using namespace ffm;
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    const int i = (int)(n % L.nx);
    const int64_t r = n / L.nx;
    const int j = (int)(r % L.ny), k = (int)(r / L.ny);
    ffv s[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int si = wrapi(i - ex(q), L.nx), sj = wrapi(j - ey(q), L.ny), sk = wrapi(k - ez(q), L.nz);
        const double fq = fin[(int64_t)q * nodes + si + (int64_t)L.nx * (sj + (int64_t)L.ny * sk)];
        s[q] = split_d(fq - wq(q));
    }
    ffv s0{0.f, 0.f}, mx{0.f, 0.f}, my{0.f, 0.f}, mz{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        s0 = add_ff(s0, s[q]);
        if (ex(q)) mx = add_ff(mx, ex(q) > 0 ? s[q] : neg(s[q]));
        if (ey(q)) my = add_ff(my, ey(q) > 0 ? s[q] : neg(s[q]));
        if (ez(q)) mz = add_ff(mz, ez(q) > 0 ? s[q] : neg(s[q]));
    }
    const ffv rho = add_ff(ffv{1.f, 0.f}, s0);
    const ffv Fr0 = split_d(Fr[n]), Fr1 = split_d(Fr[nodes + n]), Fr2 = split_d(Fr[2 * nodes + n]);
    Fr[n] = 0;
    Fr[nodes + n] = 0;
    Fr[2 * nodes + n] = 0;
    const ffv Fx = add_ff(ffv{L.body2[0][0], L.body2[0][1]}, Fr0);
    const ffv Fy = add_ff(ffv{L.body2[1][0], L.body2[1][1]}, Fr1);
    const ffv Fz = add_ff(ffv{L.body2[2][0], L.body2[2][1]}, Fr2);
    const ffv omega{L.omega2[0], L.omega2[1]}, gfac{L.gfac2[0], L.gfac2[1]};
    const ffv irho = rcp_ff(norm_ff(rho));
    const ffv ux = norm_ff(mul_u(add_ff(mulc(Fx, 0.5f), mx), irho));
    const ffv uy = norm_ff(mul_u(add_ff(mulc(Fy, 0.5f), my), irho));
    const ffv uz = norm_ff(mul_u(add_ff(mulc(Fz, 0.5f), mz), irho));
    const ffv uu = add_ff(add_ff(sqr_u(ux), sqr_u(uy)), sqr_u(uz));
    const ffv uF = add_ff(add_ff(mul_u(ux, Fx), mul_u(uy, Fy)), mul_u(uz, Fz));
    const ffv om1 = add_ff(ffv{1.f, 0.f}, neg(omega));
    // K = omega (sum s - 3/2 rho u.u) - 3 gfac u.F
    const ffv K = add_ff(mul_u(omega, add_ff(s0, neg(mulc(mul_u(rho, uu), 1.5f)))), neg(mulc(mul_u(gfac, uF), 3.0f)));
    const ffv orho = norm_ff(mul_u(omega, rho));
    ffv A[3], B[3], C[3], G[3], H[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const ffv w = wff(c);
        A[c] = mul_u(w, K);
        B[c] = mulc(mul_u(w, orho), 3.0f);
        C[c] = mulc(mul_u(w, orho), 4.5f);
        G[c] = mulc(mul_u(w, gfac), 3.0f);
        H[c] = mulc(mul_u(w, gfac), 9.0f);
    }
    fout[n] = wq(0) + to_double(norm_ff(add_ff(mul_u(om1, s[0]), A[0])));
#pragma unroll
    for (int q = 1; q < 19; ++q) {
        const int c = wcls(q);
        ffv eu{0.f, 0.f}, eF{0.f, 0.f};
        if (ex(q)) { eu = add_ff(eu, ex(q) > 0 ? ux : neg(ux)); eF = add_ff(eF, ex(q) > 0 ? Fx : neg(Fx)); }
        if (ey(q)) { eu = add_ff(eu, ey(q) > 0 ? uy : neg(uy)); eF = add_ff(eF, ey(q) > 0 ? Fy : neg(Fy)); }
        if (ez(q)) { eu = add_ff(eu, ez(q) > 0 ? uz : neg(uz)); eF = add_ff(eF, ez(q) > 0 ? Fz : neg(Fz)); }
        ffv o = add_ff(mul_u(om1, s[q]), A[c]);
        o = add_ff(o, mul_u(eu, add_ff(mul_u(C[c], eu), B[c])));
        o = add_ff(o, mul_u(eF, add_ff(mul_u(H[c], eu), G[c])));
        fout[(int64_t)q * nodes + n] = wq(q) + to_double(norm_ff(o));
    }
}

// density and velocity (AoS) of the current state: streamed distributions,
// rho u = sum f e + body / 2
template <class T>
__global__ void __launch_bounds__(256) k_lbm_macro(const T* __restrict__ fin, double* rho_out, double* u_out, Lbm L) {
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    const int i = (int)(n % L.nx);
    const int64_t r = n / L.nx;
    const int j = (int)(r % L.ny), k = (int)(r / L.ny);
    double rho = 0, m[3] = {0, 0, 0};
    for (int q = 0; q < 19; ++q) {
        const int si = wrapi(i - c_E[q][0], L.nx), sj = wrapi(j - c_E[q][1], L.ny), sk = wrapi(k - c_E[q][2], L.nz);
        const double fq = Store<T>::load(fin + (int64_t)q * nodes + si + (int64_t)L.nx * (sj + (int64_t)L.ny * sk), q);
        rho += fq;
        for (int a = 0; a < 3; ++a) m[a] += c_E[q][a] * fq;
    }
    if (rho_out) rho_out[n] = rho;
    for (int a = 0; a < 3; ++a) u_out[3 * n + a] = (m[a] + 0.5 * L.body[a]) / rho;
}

// Peskin's four-point delta, one dimension
__device__ __forceinline__ double phi4(double r) {
    r = fabs(r);
    if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) * 0.125;
    if (r < 2.0) return (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r)) * 0.125;
    return 0.0;
}

struct Support {
    int base[3];
    double w[3][4];
};

__device__ __forceinline__ Support support_of(d3 X) {
    Support s;
    const double xs[3] = {X.x, X.y, X.z};
    for (int a = 0; a < 3; ++a) {
        const double b = floor(xs[a]) - 1.0;
        s.base[a] = (int)b;
        for (int t = 0; t < 4; ++t) s.w[a][t] = phi4(xs[a] - (b + t));
    }
    return s;
}

__device__ __forceinline__ int wrapn(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// One warp per particle: lane l takes support nodes l and l + 32 of the
// 4 x 4 x 4 support (node t: a = t % 4, b = (t / 4) % 4, c = t / 16), and the
// lanes' partial sums are added in a fixed butterfly order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// U_p = sum over the 4^3 support of u(node) * weights, u from the streamed
// distributions of each support node
template <class T>
__global__ void __launch_bounds__(128) k_ibm_interp(const T* __restrict__ fin, Sys s, Lbm L) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= s.n) return;
    const int64_t n = s.n;
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    // the 12 one-dimensional weights: lane 4 axis + t computes phi(X_axis -
    // (base_axis + t)); every lane reads the three it needs by shuffle
    const double X[3] = {s.x[p], s.x[n + p], s.x[2 * n + p]};
    const double bse[3] = {floor(X[0]) - 1.0, floor(X[1]) - 1.0, floor(X[2]) - 1.0};
    const int my_axis = lane < 12 ? lane >> 2 : 0;
    const double wl = lane < 12 ? phi4(X[my_axis] - (bse[my_axis] + (lane & 3))) : 0.0;
    double U[3] = {0, 0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        const int a = t & 3, b = (t >> 2) & 3, cc = t >> 4;
        const double wa = __shfl_sync(0xffffffffu, wl, a), wb = __shfl_sync(0xffffffffu, wl, 4 + b),
                     wc = __shfl_sync(0xffffffffu, wl, 8 + cc);
        const int i = wrapn((int)bse[0] + a, L.nx), j = wrapn((int)bse[1] + b, L.ny), k = wrapn((int)bse[2] + cc, L.nz);
        // stored values s (f, or f - w for FP32 storage), summed in the
        // storage type: rho = sum s (+ 1), rho u = sum s e + body / 2
        T s0 = 0, mx = 0, my = 0, mz = 0;
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const int si = wrapi(i - ex(q), L.nx), sj = wrapi(j - ey(q), L.ny), sk = wrapi(k - ez(q), L.nz);
            const T sq = fin[(int64_t)q * nodes + si + (int64_t)L.nx * (sj + (int64_t)L.ny * sk)];
            s0 += sq;
            if (ex(q)) mx += ex(q) > 0 ? sq : -sq;
            if (ey(q)) my += ey(q) > 0 ? sq : -sq;
            if (ez(q)) mz += ez(q) > 0 ? sq : -sq;
        }
        const T rho = sizeof(T) == 4 ? (T)1 + s0 : s0;
        const T irho = (T)1 / rho;
        const double wv = wa * wb * wc;
        U[0] += (double)((mx + (T)(0.5 * L.body[0])) * irho) * wv;
        U[1] += (double)((my + (T)(0.5 * L.body[1])) * irho) * wv;
        U[2] += (double)((mz + (T)(0.5 * L.body[2])) * irho) * wv;
    }
    for (int e = 0; e < 3; ++e) U[e] = warp_sum(U[e]);
    if (lane == 0) {
        L.U[p] = U[0];
        L.U[n + p] = U[1];
        L.U[2 * n + p] = U[2];
    }
}

// penalty force of every coupled particle, one thread per particle; the
// time stepping's evaluations spread its reaction (one warp per particle was
// slower: neighbouring particles' warps then hit the same nodes' atomics at
// the same time)
template <class T>
__global__ void __launch_bounds__(128) k_ibm_penalty(Sys s, Lbm L) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= s.n) return;
    if (L.coupled && !L.coupled[p]) return;
    const int64_t n = s.n;
    const double m = s.mass[p];  // kappa = m_p / dt_LBM
    const double Fp[3] = {m * (L.U[p] - s.v[p]), m * (L.U[n + p] - s.v[n + p]), m * (L.U[2 * n + p] - s.v[2 * n + p])};
    s.f[p] += Fp[0];
    s.f[n + p] += Fp[1];
    s.f[2 * n + p] += Fp[2];
    if (!s.count_step) return;
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    const Support sp = support_of(mk3(s.x[p], s.x[n + p], s.x[2 * n + p]));
    const double inv_sub = 1.0 / L.n_sub;
    for (int cc = 0; cc < 4; ++cc)
        for (int b = 0; b < 4; ++b)
            for (int a = 0; a < 4; ++a) {
                const int64_t node = wrapn(sp.base[0] + a, L.nx) +
                                     (int64_t)L.nx * (wrapn(sp.base[1] + b, L.ny) + (int64_t)L.ny * wrapn(sp.base[2] + cc, L.nz));
                const double wv = sp.w[0][a] * sp.w[1][b] * sp.w[2][cc] * inv_sub;
                T* F = (T*)L.F;
                atomicAdd(F + node, (T)(-Fp[0] * wv));
                atomicAdd(F + nodes + node, (T)(-Fp[1] * wv));
                atomicAdd(F + 2 * nodes + node, (T)(-Fp[2] * wv));
            }
}

// f* = f_eq(rho0, u0) (FP64 arguments, either storage)
template <class T>
__global__ void __launch_bounds__(256) k_lbm_init(T* f, const double* rho0, const double* u0, Lbm L) {
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nodes) return;
    const double rho = rho0 ? rho0[n] : 1.0;
    const double u[3] = {u0 ? u0[3 * n] : 0.0, u0 ? u0[3 * n + 1] : 0.0, u0 ? u0[3 * n + 2] : 0.0};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < 19; ++q) {
        const double eu = c_E[q][0] * u[0] + c_E[q][1] * u[1] + c_E[q][2] * u[2];
        Store<T>::store(f + (int64_t)q * nodes + n, q, wq(q) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    }
    T* F = (T*)L.F;
    F[n] = F[nodes + n] = F[2 * nodes + n] = 0;
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_lbm_init(const Lbm& L, const double* rho0, const double* u0, cudaStream_t st) {
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    if (L.fp32)
        k_lbm_init<float><<<blocks_for(nodes, 256), 256, 0, st>>>((float*)L.f[0], rho0, u0, L);
    else
        k_lbm_init<double><<<blocks_for(nodes, 256), 256, 0, st>>>((double*)L.f[0], rho0, u0, L);
    return cudaGetLastError();
}

cudaError_t launch_lbm_step(const Lbm& L, int parity, cudaStream_t st) {
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    if (L.fp32)
        k_lbm_step<float><<<blocks_for(nodes, 256), 256, 0, st>>>((const float*)L.f[parity], (float*)L.f[parity ^ 1],
                                                                   (float*)L.F, L);
    else if (L.ff)
        k_lbm_step_ff<<<blocks_for(nodes, 256), 256, 0, st>>>((const double*)L.f[parity], (double*)L.f[parity ^ 1],
                                                              (double*)L.F, L);
    else
        k_lbm_step<double><<<blocks_for(nodes, 256), 256, 0, st>>>((const double*)L.f[parity],
                                                                    (double*)L.f[parity ^ 1], (double*)L.F, L);
    return cudaGetLastError();
}

cudaError_t launch_lbm_macro(const Lbm& L, int parity, double* rho, double* u, cudaStream_t st) {
    const int64_t nodes = (int64_t)L.nx * L.ny * L.nz;
    if (L.fp32)
        k_lbm_macro<float><<<blocks_for(nodes, 256), 256, 0, st>>>((const float*)L.f[parity], rho, u, L);
    else
        k_lbm_macro<double><<<blocks_for(nodes, 256), 256, 0, st>>>((const double*)L.f[parity], rho, u, L);
    return cudaGetLastError();
}

cudaError_t launch_ibm_interp(const Sys& s, const Lbm& L, int parity, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    if (L.fp32)
        k_ibm_interp<float><<<blocks_for(32 * s.n, 128), 128, 0, st>>>((const float*)L.f[parity], s, L);
    else
        k_ibm_interp<double><<<blocks_for(32 * s.n, 128), 128, 0, st>>>((const double*)L.f[parity], s, L);
    return cudaGetLastError();
}

cudaError_t launch_ibm_penalty(const Sys& s, const Lbm& L, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    if (L.fp32)
        k_ibm_penalty<float><<<blocks_for(s.n, 128), 128, 0, st>>>(s, L);
    else
        k_ibm_penalty<double><<<blocks_for(s.n, 128), 128, 0, st>>>(s, L);
    return cudaGetLastError();
}

}  // namespace bpm
