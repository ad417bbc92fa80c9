// All-pairs, open-boundary dipole-dipole interaction (Methods, "Magnetic
// interactions": U_ij = c/r^3 [m_i.m_j - 3 (m_i.r^)(m_j.r^)], forces and
// torques by differentiation).  With r = x_i - x_j, a = m_i.r, b = m_j.r,
// d = m_i.m_j:
//   F_i  = 3c sum_j [ (a m_j + (d - 5ab/r^2) r) / r^5 ] + 3c m_i sum_j b/r^5
//   B(x_i) = c sum_j [ 3 b r / r^5 - m_j / r^3 ],   tau_i = m_i x B(x_i).
// The kernels accumulate, per particle i and work item, the three sums
//   F~ = sum (A m_j + S r), A = a/r^5, S = (d - 5ab/r^2)/r^5
//   H~ = sum (3 b r / r^5 - m_j / r^3),   Bs = sum b / r^5
// into a fixed partial slot; the finish kernel applies c, 3c and m_i x .
//
// Work: a persistent grid pulls items (i-tile x j-range) from an atomic
// queue, largest first; j-tiles are staged in shared memory and broadcast
// to the block.  Each (particle, slot) is written by exactly one item, so the
// result does not depend on scheduling.
//
// FP64 path: everything in double; 1/r from an FP32 estimate plus two
// Newton steps (rsqrt_nr).  Mixed path: pair terms in FP32 with positions
// split into FP32 hi/lo parts, r = (hi_i - hi_j) + (lo_i - lo_j), 1/r from
// the FP32 hardware estimate; the FP32 sums of one j-tile are added to FP64
// running sums after every tile.
#include "bpm_devmath.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

constexpr int FP64_BT = 128;   // threads = i per item = j per tile
constexpr int MIX_BT = 128;    // threads
constexpr int MIX_R = 2;       // i particles per thread
constexpr int MIX_TJ = 256;    // j per tile

__device__ __forceinline__ int fetch_item(int* counter, int* s_item) {
    __syncthreads();
    if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
    __syncthreads();
    return *s_item;
}

// ---------------------------------------------------------------- FP64
struct Acc64 {
    double fx, fy, fz, hx, hy, hz, bs;
};

template <bool SELF>
__device__ __forceinline__ void pairs_fp64(Acc64& acc, d3 xi, d3 mi, const double (*sx)[FP64_BT],
                                           const double (*sm)[FP64_BT], int jn, int self) {
#pragma unroll 2
    for (int jj = 0; jj < jn; ++jj) {
        if (SELF && jj == self) continue;
        const double rx = xi.x - sx[0][jj];
        const double ry = xi.y - sx[1][jj];
        const double rz = xi.z - sx[2][jj];
        const double mjx = sm[0][jj], mjy = sm[1][jj], mjz = sm[2][jj];
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double rinv = rsqrt_nr(r2);
        const double rinv2 = rinv * rinv;
        const double rinv3 = rinv2 * rinv;
        const double rinv5 = rinv3 * rinv2;
        const double a = mi.x * rx + mi.y * ry + mi.z * rz;
        const double b = mjx * rx + mjy * ry + mjz * rz;
        const double d = mi.x * mjx + mi.y * mjy + mi.z * mjz;
        const double s = fma(-5.0 * a * b, rinv2, d);
        const double A = rinv5 * a;
        const double S = rinv5 * s;
        acc.fx = fma(A, mjx, fma(S, rx, acc.fx));
        acc.fy = fma(A, mjy, fma(S, ry, acc.fy));
        acc.fz = fma(A, mjz, fma(S, rz, acc.fz));
        const double rb5 = rinv5 * b;
        acc.bs += rb5;
        const double G = 3.0 * rb5;
        acc.hx = fma(-rinv3, mjx, fma(G, rx, acc.hx));
        acc.hy = fma(-rinv3, mjy, fma(G, ry, acc.hy));
        acc.hz = fma(-rinv3, mjz, fma(G, rz, acc.hz));
    }
}

__global__ void __launch_bounds__(FP64_BT) k_dipole_fp64(Sys s, const WorkItem* __restrict__ items,
                                                         int n_items, int* counter) {
    __shared__ double sx[3][FP64_BT];
    __shared__ double sm[3][FP64_BT];
    __shared__ int s_item;
    const int64_t n = s.n;
    for (;;) {
        const int it = fetch_item(counter, &s_item);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const int i = wi.i0 + (int)threadIdx.x;
        const bool iv = (int)threadIdx.x < wi.ni;
        d3 xi = mk3(0, 0, 0), mi = mk3(0, 0, 0);
        if (iv) {
            xi = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
            mi = mk3(s.m[i], s.m[n + i], s.m[2 * n + i]);
        }
        Acc64 acc = {0, 0, 0, 0, 0, 0, 0};
        const int jend = wi.j0 + wi.nj;
        for (int jt = wi.j0; jt < jend; jt += FP64_BT) {
            const int jn = min(FP64_BT, jend - jt);
            __syncthreads();
            if ((int)threadIdx.x < jn) {
                const int j = jt + threadIdx.x;
                sx[0][threadIdx.x] = s.x[j];
                sx[1][threadIdx.x] = s.x[n + j];
                sx[2][threadIdx.x] = s.x[2 * n + j];
                sm[0][threadIdx.x] = s.m[j];
                sm[1][threadIdx.x] = s.m[n + j];
                sm[2][threadIdx.x] = s.m[2 * n + j];
            }
            __syncthreads();
            // tiles that overlap the item's i-range skip the self pair
            const bool diag = (wi.i0 < jt + jn) && (wi.i0 + wi.ni > jt);
            if (iv) {
                if (diag)
                    pairs_fp64<true>(acc, xi, mi, sx, sm, jn, (i >= jt && i < jt + jn) ? i - jt : -1);
                else
                    pairs_fp64<false>(acc, xi, mi, sx, sm, jn, -1);
            }
        }
        if (iv) {
            double* P = s.part + (int64_t)wi.slot * 7 * n;
            P[i] = acc.fx;
            P[n + i] = acc.fy;
            P[2 * n + i] = acc.fz;
            P[3 * n + i] = acc.hx;
            P[4 * n + i] = acc.hy;
            P[5 * n + i] = acc.hz;
            P[6 * n + i] = acc.bs;
        }
    }
}

// ---------------------------------------------------------------- mixed
struct Acc32 {
    float fx, fy, fz, hx, hy, hz, bs;
};

__device__ __forceinline__ void pair_fp32(Acc32& acc, float ihx, float ihy, float ihz, float ilx,
                                          float ily, float ilz, float mix, float miy, float miz,
                                          float4 j0, float4 j1, float mjz) {
    // j0 = (hx, hy, hz, lx), j1 = (ly, lz, mx, my)
    const float rx = (ihx - j0.x) + (ilx - j0.w);
    const float ry = (ihy - j0.y) + (ily - j1.x);
    const float rz = (ihz - j0.z) + (ilz - j1.y);
    const float mjx = j1.z, mjy = j1.w;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    float rinv;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv) : "f"(r2));
    const float rinv2 = rinv * rinv;
    const float rinv3 = rinv2 * rinv;
    const float rinv5 = rinv3 * rinv2;
    const float a = fmaf(mix, rx, fmaf(miy, ry, miz * rz));
    const float b = fmaf(mjx, rx, fmaf(mjy, ry, mjz * rz));
    const float d = fmaf(mix, mjx, fmaf(miy, mjy, miz * mjz));
    const float sfac = fmaf(-5.0f * a * b, rinv2, d);
    const float A = rinv5 * a;
    const float S = rinv5 * sfac;
    acc.fx = fmaf(A, mjx, fmaf(S, rx, acc.fx));
    acc.fy = fmaf(A, mjy, fmaf(S, ry, acc.fy));
    acc.fz = fmaf(A, mjz, fmaf(S, rz, acc.fz));
    const float rb5 = rinv5 * b;
    acc.bs += rb5;
    const float G = 3.0f * rb5;
    acc.hx = fmaf(-rinv3, mjx, fmaf(G, rx, acc.hx));
    acc.hy = fmaf(-rinv3, mjy, fmaf(G, ry, acc.hy));
    acc.hz = fmaf(-rinv3, mjz, fmaf(G, rz, acc.hz));
}

struct IData {
    float hx, hy, hz, lx, ly, lz, mx, my, mz;
};

__device__ __forceinline__ void flush(Acc64& A, Acc32& a) {
    A.fx += (double)a.fx;
    A.fy += (double)a.fy;
    A.fz += (double)a.fz;
    A.hx += (double)a.hx;
    A.hy += (double)a.hy;
    A.hz += (double)a.hz;
    A.bs += (double)a.bs;
    a = Acc32{0, 0, 0, 0, 0, 0, 0};
}

__global__ void __launch_bounds__(MIX_BT) k_dipole_mixed(Sys s, const WorkItem* __restrict__ items,
                                                         int n_items, int* counter) {
    __shared__ float4 sj0[MIX_TJ];
    __shared__ float4 sj1[MIX_TJ];
    __shared__ float sjz[MIX_TJ];
    __shared__ int s_item;
    const int64_t n = s.n;
    for (;;) {
        const int it = fetch_item(counter, &s_item);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        int ii[MIX_R];
        bool iv[MIX_R];
        IData id[MIX_R];
        Acc64 A64[MIX_R];
        Acc32 A32[MIX_R];
#pragma unroll
        for (int r = 0; r < MIX_R; ++r) {
            const int li = (int)threadIdx.x + r * MIX_BT;
            ii[r] = wi.i0 + li;
            iv[r] = li < wi.ni;
            const int i = iv[r] ? ii[r] : wi.i0;
            id[r] = IData{s.xh[i], s.xh[n + i], s.xh[2 * n + i], s.xl[i], s.xl[n + i], s.xl[2 * n + i],
                          s.mf[i], s.mf[n + i], s.mf[2 * n + i]};
            A64[r] = Acc64{0, 0, 0, 0, 0, 0, 0};
            A32[r] = Acc32{0, 0, 0, 0, 0, 0, 0};
        }
        const int jend = wi.j0 + wi.nj;
        for (int jt = wi.j0; jt < jend; jt += MIX_TJ) {
            const int jn = min(MIX_TJ, jend - jt);
            __syncthreads();
            for (int l = threadIdx.x; l < jn; l += MIX_BT) {
                const int j = jt + l;
                sj0[l] = make_float4(s.xh[j], s.xh[n + j], s.xh[2 * n + j], s.xl[j]);
                sj1[l] = make_float4(s.xl[n + j], s.xl[2 * n + j], s.mf[j], s.mf[n + j]);
                sjz[l] = s.mf[2 * n + j];
            }
            __syncthreads();
            const bool self_tile = (wi.i0 < jt + jn) && (wi.i0 + wi.ni > jt);
            if (!self_tile) {
#pragma unroll 2
                for (int jj = 0; jj < jn; ++jj) {
                    const float4 j0 = sj0[jj];
                    const float4 j1 = sj1[jj];
                    const float mjz = sjz[jj];
#pragma unroll
                    for (int r = 0; r < MIX_R; ++r)
                        pair_fp32(A32[r], id[r].hx, id[r].hy, id[r].hz, id[r].lx, id[r].ly, id[r].lz,
                                  id[r].mx, id[r].my, id[r].mz, j0, j1, mjz);
                }
            } else {
                for (int jj = 0; jj < jn; ++jj) {
                    const float4 j0 = sj0[jj];
                    const float4 j1 = sj1[jj];
                    const float mjz = sjz[jj];
#pragma unroll
                    for (int r = 0; r < MIX_R; ++r) {
                        if (jt + jj == ii[r]) continue;
                        pair_fp32(A32[r], id[r].hx, id[r].hy, id[r].hz, id[r].lx, id[r].ly, id[r].lz,
                                  id[r].mx, id[r].my, id[r].mz, j0, j1, mjz);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < MIX_R; ++r) flush(A64[r], A32[r]);
        }
#pragma unroll
        for (int r = 0; r < MIX_R; ++r) {
            if (!iv[r]) continue;
            const int i = ii[r];
            double* P = s.part + (int64_t)wi.slot * 7 * n;
            P[i] = A64[r].fx;
            P[n + i] = A64[r].fy;
            P[2 * n + i] = A64[r].fz;
            P[3 * n + i] = A64[r].hx;
            P[4 * n + i] = A64[r].hy;
            P[5 * n + i] = A64[r].hz;
            P[6 * n + i] = A64[r].bs;
        }
    }
}

}  // namespace

int dipole_tile_i(bool mixed, const DipoleCfg&) { return mixed ? MIX_BT * MIX_R : FP64_BT; }

int dipole_blocks_per_sm(bool mixed) {
    int b = 0;
    if (mixed)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_mixed, MIX_BT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_fp64, FP64_BT, 0);
    return b;
}

cudaError_t launch_dipole(const Sys& s, bool mixed, const WorkItem* items, int n_items, int* counter,
                          const DipoleCfg& cfg, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const int blocks = cfg.blocks > 0 ? cfg.blocks : n_items;
    if (mixed)
        k_dipole_mixed<<<blocks, MIX_BT, 0, st>>>(s, items, n_items, counter);
    else
        k_dipole_fp64<<<blocks, FP64_BT, 0, st>>>(s, items, n_items, counter);
    return cudaGetLastError();
}

}  // namespace bpm
