// Per-particle kernels: reduction of the dipole partial sums into the total
// force/torque, the velocity-Verlet / Richardson update (SI "Equations of
// motion"), energies, and layout conversions.
//
// Time stepping (SI "Equations of motion"), given f, tau at t:
//   v += dt/2 f/m;  x += dt v;  omega += dt/2 tau/I;  q <- Richardson(q, omega)
//   forces at t + dt (damping uses these half-step velocities)
//   v += dt/2 f/m;  omega += dt/2 tau/I
// The closing half kick of step k and the opening half kick of step k+1 run
// in the same kernel (k_finish, FINISH_CONTINUE) as two separate additions,
// so the rounding is that of the two-kick form.
#include "bpm_devmath.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

// (0, a) q for a pure-vector quaternion (0, a): the Hamilton product with
// its zero scalar part left out (12 FP64 operations instead of 16)
__device__ __forceinline__ dq vmul(d3 a, dq q) {
    return dq{-(a.x * q.x + a.y * q.y + a.z * q.z), a.x * q.w + a.y * q.z - a.z * q.y,
              a.y * q.w + a.z * q.x - a.x * q.z, a.z * q.w + a.x * q.y - a.y * q.x};
}

// q' = 1/2 (0, omega) q; one step of dt and two of dt/2, each renormalised;
// result 2 q_(2) - q_(1), renormalised.  With a = (dt/2) omega,
// dt q' = (0, a) q, and the half steps use a/2.
__device__ __forceinline__ dq richardson(dq q, d3 w, double dt) {
    const d3 a = w * (0.5 * dt);
    const dq p = vmul(a, q);  // dt q'(q)
    const dq q1 = qnormalise_nr(dq{q.w + p.w, q.x + p.x, q.y + p.y, q.z + p.z});
    const dq qh = qnormalise_nr(dq{fma(0.5, p.w, q.w), fma(0.5, p.x, q.x), fma(0.5, p.y, q.y), fma(0.5, p.z, q.z)});
    const dq ph = vmul(a * 0.5, qh);  // (dt/2) q'(qh)
    const dq q2 = qnormalise_nr(dq{qh.w + ph.w, qh.x + ph.x, qh.y + ph.y, qh.z + ph.z});
    return qnormalise_nr(dq{2.0 * q2.w - q1.w, 2.0 * q2.x - q1.x, 2.0 * q2.y - q1.y, 2.0 * q2.z - q1.z});
}


// finiteness from the exponent bits of the high word (integer operations, so
// the checks take nothing from the FP64 pipe)
__device__ __forceinline__ bool finite1(double a) { return (__double2hiint(a) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool finite3(d3 a) { return finite1(a.x) && finite1(a.y) && finite1(a.z); }

template <bool DIPOLE, int MODE, bool ENERGY>
__global__ void __launch_bounds__(256) k_finish(Sys s, int* counter) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the step counter is advanced by the bond kernel of each step, so every
    // thread here reads the same value
    if (i == 0) {
        if (counter) *counter = 0;  // dipole work queue for the next launch
        if (MODE == FINISH_CONTINUE) *s.tdev += s.dt;
        // the bond and contact kernels of a step wrote the previous level's
        // buffers: they become the current level; a stand-alone evaluation
        // has filled in the current level if it was empty
        if (s.ct_valid) s.ct_valid[s.count_step ? ((*s.hist_gen + 1) & 1) : (*s.hist_gen & 1)] = 1;
        if (s.count_step && s.hist_gen) *s.hist_gen += 1;
    }
    if (i >= n) return;
    d3 F = mk3(s.f[i], s.f[n + i], s.f[2 * n + i]);
    d3 T = mk3(s.t[i], s.t[n + i], s.t[2 * n + i]);
    if (DIPOLE) {
        const d3 m = mk3(s.m[i], s.m[n + i], s.m[2 * n + i]);
        d3 Fd = mk3(0, 0, 0), Hd = mk3(0, 0, 0);
        double bs = 0.0;
        // after k_reduce_slots the sums sit in slot 0
        const int ns = s.slots_reduced ? min(1, (int)s.nslot[i]) : s.nslot[i];
        for (int k = 0; k < ns; ++k) {
            const double* P = s.part + (int64_t)k * 7 * n;
            Fd = Fd + mk3(P[i], P[n + i], P[2 * n + i]);
            Hd = Hd + mk3(P[3 * n + i], P[4 * n + i], P[5 * n + i]);
            bs += P[6 * n + i];
        }
        const d3 Fdip = (Fd + m * bs) * (3.0 * s.c);
        const d3 H = Hd * s.c;
        F = F + Fdip;
        T = T + cross(m, H);
        if (ENERGY) s.e_part[2 * n + i] = -0.5 * dot(m, H);
    } else if (ENERGY) {
        s.e_part[2 * n + i] = 0.0;
    }
    s.f[i] = F.x;
    s.f[n + i] = F.y;
    s.f[2 * n + i] = F.z;
    s.t[i] = T.x;
    s.t[n + i] = T.y;
    s.t[2 * n + i] = T.z;

    d3 v = mk3(s.v[i], s.v[n + i], s.v[2 * n + i]);
    d3 w = mk3(s.w[i], s.w[n + i], s.w[2 * n + i]);
    const double mass = s.mass[i], I = s.inertia[i];
    if (ENERGY) {
        s.e_part[3 * n + i] = 0.5 * mass * dot(v, v);
        s.e_part[4 * n + i] = 0.5 * I * dot(w, w);
    }
    if (MODE == FINISH_FORCES) {
        if (!(finite3(F) && finite3(T))) atomicCAS(s.err, 0, 1);
        return;
    }
    bool ok = finite3(F) && finite3(T);
    const bool clamped = s.flags[i] & F_CLAMPED;
    if (!clamped) {
        const double h = 0.5 * s.dt;
        const double im = s.inv_mass[i], iI = s.inv_inertia[i];
        // the closing half kick of this step and the opening one of the next
        // add the same increment, formed once
        const d3 dv = (F * h) * im, dw = (T * h) * iI;
        v = v + dv;
        w = w + dw;
        if (MODE == FINISH_CONTINUE) {
            v = v + dv;
            w = w + dw;
            d3 x = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
            x = x + v * s.dt;
            dq q = dq{s.q[i], s.q[n + i], s.q[2 * n + i], s.q[3 * n + i]};
            q = richardson(q, w, s.dt);
            ok = ok && finite3(x) && finite1(q.w) && finite1(q.x) && finite1(q.y) && finite1(q.z);
            s.x[i] = x.x;
            s.x[n + i] = x.y;
            s.x[2 * n + i] = x.z;
            s.q[i] = q.w;
            s.q[n + i] = q.x;
            s.q[2 * n + i] = q.y;
            s.q[3 * n + i] = q.z;
        }
        s.v[i] = v.x;
        s.v[n + i] = v.y;
        s.v[2 * n + i] = v.z;
        s.w[i] = w.x;
        s.w[n + i] = w.y;
        s.w[2 * n + i] = w.z;
    }
    if (!ok) atomicCAS(s.err, 0, *s.step_counter + 1);
}

// Sums the partial slots of each (component, particle) in slot order into
// slot 0: one thread per (c, i), so the reduction of many slots spreads over
// the whole GPU; the order (and so every bit) is that of the finish kernel's
// own loop.
__global__ void __launch_bounds__(256) k_reduce_slots(Sys s) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    const int ns = s.nslot[i];
    if (ns <= 1) return;
    const int64_t stride = 7 * n;
    const double* P = s.part + (int64_t)c * n + i;
    double acc = 0.0;
    for (int k = 0; k < ns; ++k) acc += P[k * stride];
    s.part[(int64_t)c * n + i] = acc;
}

__global__ void __launch_bounds__(256) k_first_half(Sys s) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *s.tdev += s.dt;
    if (i >= n) return;
    if (s.flags[i] & F_CLAMPED) return;
    const double h = 0.5 * s.dt;
    const double im = s.inv_mass[i], iI = s.inv_inertia[i];
    d3 F = mk3(s.f[i], s.f[n + i], s.f[2 * n + i]);
    d3 T = mk3(s.t[i], s.t[n + i], s.t[2 * n + i]);
    d3 v = mk3(s.v[i], s.v[n + i], s.v[2 * n + i]);
    d3 w = mk3(s.w[i], s.w[n + i], s.w[2 * n + i]);
    v = v + (F * h) * im;
    w = w + (T * h) * iI;
    d3 x = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
    x = x + v * s.dt;
    dq q = dq{s.q[i], s.q[n + i], s.q[2 * n + i], s.q[3 * n + i]};
    q = richardson(q, w, s.dt);
    s.x[i] = x.x;
    s.x[n + i] = x.y;
    s.x[2 * n + i] = x.z;
    s.q[i] = q.w;
    s.q[n + i] = q.x;
    s.q[2 * n + i] = q.y;
    s.q[3 * n + i] = q.z;
    s.v[i] = v.x;
    s.v[n + i] = v.y;
    s.v[2 * n + i] = v.z;
    s.w[i] = w.x;
    s.w[n + i] = w.y;
    s.w[2 * n + i] = w.z;
}

// One block; each thread sums a strided range in index order, then a fixed
// shared-memory tree: the result is the same on every run.
__global__ void __launch_bounds__(1024) k_energy_reduce(Sys s, double* out) {
    __shared__ double red[1024];
    const int64_t n = s.n;
    for (int c = 0; c < 5; ++c) {
        double acc = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += s.e_part[c * n + i];
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

__global__ void k_aos_to_soa(const double* __restrict__ aos, double* __restrict__ soa, int64_t n, int nc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nc; ++c) soa[c * n + i] = aos[i * nc + c];
}

__global__ void k_soa_to_aos(const double* __restrict__ soa, double* __restrict__ aos, int64_t n, int nc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < nc; ++c) aos[i * nc + c] = soa[c * n + i];
}

__global__ void k_quat_right_mul(double* q, const double* r, int64_t n, bool conj_r, bool norm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dq a = dq{q[i], q[n + i], q[2 * n + i], q[3 * n + i]};
    dq b = dq{r[i], r[n + i], r[2 * n + i], r[3 * n + i]};
    if (conj_r) b = qconj(b);
    dq c = qmul(a, b);
    if (norm) c = qnormalise(c);
    q[i] = c.w;
    q[n + i] = c.x;
    q[2 * n + i] = c.y;
    q[3 * n + i] = c.z;
}

__global__ void k_rotate_vec(const double* q, double* v, int64_t n, bool inverse) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dq a = dq{q[i], q[n + i], q[2 * n + i], q[3 * n + i]};
    d3 x = mk3(v[i], v[n + i], v[2 * n + i]);
    d3 y = inverse ? rot_inv(a, x) : rot(a, x);
    v[i] = y.x;
    v[n + i] = y.y;
    v[2 * n + i] = y.z;
}

__global__ void k_zero_clamped(Sys s) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !(s.flags[i] & F_CLAMPED)) return;
    for (int c = 0; c < 3; ++c) {
        s.v[c * n + i] = 0.0;
        s.w[c * n + i] = 0.0;
    }
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_finish(const Sys& s, bool dipole, int mode, bool energy, int* counter, cudaStream_t st) {
    const int th = 256;
    const unsigned g = grid_for(s.n > 0 ? s.n : 1, th);
#define BPM_FIN(D, M, E) k_finish<D, M, E><<<g, th, 0, st>>>(s, counter)
    if (dipole) {
        if (energy) {
            BPM_FIN(true, FINISH_FORCES, true);
        } else if (mode == FINISH_FORCES) {
            BPM_FIN(true, FINISH_FORCES, false);
        } else if (mode == FINISH_HALF_KICK) {
            BPM_FIN(true, FINISH_HALF_KICK, false);
        } else {
            BPM_FIN(true, FINISH_CONTINUE, false);
        }
    } else {
        if (energy) {
            BPM_FIN(false, FINISH_FORCES, true);
        } else if (mode == FINISH_FORCES) {
            BPM_FIN(false, FINISH_FORCES, false);
        } else if (mode == FINISH_HALF_KICK) {
            BPM_FIN(false, FINISH_HALF_KICK, false);
        } else {
            BPM_FIN(false, FINISH_CONTINUE, false);
        }
    }
#undef BPM_FIN
    return cudaGetLastError();
}

cudaError_t launch_reduce_slots(const Sys& s, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    k_reduce_slots<<<dim3(grid_for(s.n, 256), 7), 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_first_half(const Sys& s, cudaStream_t st) {
    k_first_half<<<grid_for(s.n > 0 ? s.n : 1, 256), 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(const Sys& s, double* out5, cudaStream_t st) {
    k_energy_reduce<<<1, 1024, 0, st>>>(s, out5);
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double* aos, double* soa, int64_t n, int nc, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_aos_to_soa<<<grid_for(n, 256), 256, 0, st>>>(aos, soa, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double* soa, double* aos, int64_t n, int nc, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_soa_to_aos<<<grid_for(n, 256), 256, 0, st>>>(soa, aos, n, nc);
    return cudaGetLastError();
}

cudaError_t launch_quat_right_mul(double* q, const double* r, int64_t n, bool conj_r, bool norm,
                                  cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_quat_right_mul<<<grid_for(n, 256), 256, 0, st>>>(q, r, n, conj_r, norm);
    return cudaGetLastError();
}

cudaError_t launch_rotate_vec(const double* q, double* v, int64_t n, bool inverse, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_rotate_vec<<<grid_for(n, 256), 256, 0, st>>>(q, v, n, inverse);
    return cudaGetLastError();
}

cudaError_t launch_zero_clamped(const Sys& s, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    k_zero_clamped<<<grid_for(s.n, 256), 256, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace bpm
