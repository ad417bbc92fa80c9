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
#include <mutex>

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

// Two j per instruction with Blackwell's packed FP32 arithmetic
// (fma/add/mul .f32x2): the i data broadcast to both halves once per item,
// the j data loaded as (j, j+1) pairs from SoA shared memory, and the sums of
// even and odd j kept in the two halves of each accumulator until the tile
// flush.  Each half evaluates the FP32 pair term: r from the hi and lo
// differences, 1/r from the hardware rsqrt estimate, and the force and field
// sums of the FP64 kernel in FP32.  The packed form halves the instructions
// issued per pair.
// SELF (a j tile that holds the thread's own i): dj = i - j0, where j0 is the
// even j of the packed pair; the half with j = i gets 1/r := 0, and since r
// is then exactly zero, every one of its terms is an exact zero.
struct Acc2 {
    float2 fx, fy, fz, hx, hy, hz, bs;
};
struct IData2 {
    float2 hx, hy, hz, lx, ly, lz, mx, my, mz;
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// The i data of a lane of a packed symmetric kernel.  A lane past the
// item's i range holds a stand-in far from every particle and from the j
// stand-in (at -1e18, the j one at +1e18) with zero moment: its pair terms
// on both sides are exact zeros, so every lane runs the symmetric pair
// without a branch on its validity (which would split the two i of a lane
// into separate blocks of code and serialise their dependency chains).
__device__ __forceinline__ IData2 i_data2(const Sys& s, int64_t n, int i, bool valid) {
    if (!valid) {
        const float2 far = bc2(-1e18f), z = bc2(0.f);
        return IData2{far, far, far, z, z, z, z, z, z};
    }
    return IData2{bc2(s.xh[i]), bc2(s.xh[n + i]), bc2(s.xh[2 * n + i]), bc2(s.xl[i]), bc2(s.xl[n + i]),
                  bc2(s.xl[2 * n + i]), bc2(s.mf[i]), bc2(s.mf[n + i]), bc2(s.mf[2 * n + i])};
}

template <bool SELF>
__device__ __forceinline__ void pair_fp32x2(Acc2& acc, const IData2& I, float2 jhx, float2 jhy, float2 jhz,
                                            float2 jlx, float2 jly, float2 jlz, float2 mjx, float2 mjy,
                                            float2 mjz, int dj) {
    const float2 rx = __fadd2_rn(__fadd2_rn(I.hx, make_float2(-jhx.x, -jhx.y)), __fadd2_rn(I.lx, make_float2(-jlx.x, -jlx.y)));
    const float2 ry = __fadd2_rn(__fadd2_rn(I.hy, make_float2(-jhy.x, -jhy.y)), __fadd2_rn(I.ly, make_float2(-jly.x, -jly.y)));
    const float2 rz = __fadd2_rn(__fadd2_rn(I.hz, make_float2(-jhz.x, -jhz.y)), __fadd2_rn(I.lz, make_float2(-jlz.x, -jlz.y)));
    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
    float2 rinv;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv.x) : "f"(r2.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv.y) : "f"(r2.y));
    if (SELF) {
        if (dj == 0) rinv.x = 0.f;
        if (dj == 1) rinv.y = 0.f;
    }
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 rinv3 = __fmul2_rn(rinv2, rinv);
    const float2 rinv5 = __fmul2_rn(rinv3, rinv2);
    const float2 a = __ffma2_rn(I.mx, rx, __ffma2_rn(I.my, ry, __fmul2_rn(I.mz, rz)));
    const float2 b = __ffma2_rn(mjx, rx, __ffma2_rn(mjy, ry, __fmul2_rn(mjz, rz)));
    const float2 d = __ffma2_rn(I.mx, mjx, __ffma2_rn(I.my, mjy, __fmul2_rn(I.mz, mjz)));
    const float2 sfac = __ffma2_rn(__fmul2_rn(__fmul2_rn(bc2(-5.0f), a), b), rinv2, d);
    const float2 A = __fmul2_rn(rinv5, a);
    const float2 S = __fmul2_rn(rinv5, sfac);
    acc.fx = __ffma2_rn(A, mjx, __ffma2_rn(S, rx, acc.fx));
    acc.fy = __ffma2_rn(A, mjy, __ffma2_rn(S, ry, acc.fy));
    acc.fz = __ffma2_rn(A, mjz, __ffma2_rn(S, rz, acc.fz));
    const float2 rb5 = __fmul2_rn(rinv5, b);
    acc.bs = __fadd2_rn(acc.bs, rb5);
    const float2 G = __fmul2_rn(bc2(3.0f), rb5);
    const float2 nr3 = make_float2(-rinv3.x, -rinv3.y);
    acc.hx = __ffma2_rn(nr3, mjx, __ffma2_rn(G, rx, acc.hx));
    acc.hy = __ffma2_rn(nr3, mjy, __ffma2_rn(G, ry, acc.hy));
    acc.hz = __ffma2_rn(nr3, mjz, __ffma2_rn(G, rz, acc.hz));
}

// the two halves (even and odd j) added into the scalar FP32 tile sums
// the FP32 sums of one tile added to a thread's FP64 i sums kept in shared
// memory ([.][7][128] doubles, slot r), in the order of flush()
__device__ __forceinline__ void flush_smem(double* a64s, int r, int tid, Acc32& a) {
    double* A = a64s + r * 7 * 128 + tid;
    A[0] += (double)a.fx;
    A[128] += (double)a.fy;
    A[2 * 128] += (double)a.fz;
    A[3 * 128] += (double)a.hx;
    A[4 * 128] += (double)a.hy;
    A[5 * 128] += (double)a.hz;
    A[6 * 128] += (double)a.bs;
    a = Acc32{0, 0, 0, 0, 0, 0, 0};
}

__device__ __forceinline__ void fold2(Acc32& a, Acc2& b) {
    a.fx += b.fx.x + b.fx.y;
    a.fy += b.fy.x + b.fy.y;
    a.fz += b.fz.x + b.fz.y;
    a.hx += b.hx.x + b.hx.y;
    a.hy += b.hy.x + b.hy.y;
    a.hz += b.hz.x + b.hz.y;
    a.bs += b.bs.x + b.bs.y;
    const float2 z = make_float2(0.f, 0.f);
    b = Acc2{z, z, z, z, z, z, z};
}

// The i of this thread against the j tile in shared memory (SoA rows: hi x,
// y, z; lo x, y, z; moment x, y, z), two j per packed instruction.  Groups
// of 32 i that hold no particle (gv false, warp-uniform) skip the work.
template <bool SELF, bool ALL>
__device__ __forceinline__ void mix_jloop(Acc2 (&P2)[MIX_R], const IData2 (&id2)[MIX_R], const bool (&gv)[MIX_R],
                                          const int (&ii)[MIX_R], const float (*sj)[MIX_TJ], int jn2, int jt) {
#pragma unroll 2
    for (int jj = 0; jj < jn2; jj += 2) {
        const float2 jhx = *reinterpret_cast<const float2*>(&sj[0][jj]);
        const float2 jhy = *reinterpret_cast<const float2*>(&sj[1][jj]);
        const float2 jhz = *reinterpret_cast<const float2*>(&sj[2][jj]);
        const float2 jlx = *reinterpret_cast<const float2*>(&sj[3][jj]);
        const float2 jly = *reinterpret_cast<const float2*>(&sj[4][jj]);
        const float2 jlz = *reinterpret_cast<const float2*>(&sj[5][jj]);
        const float2 mjx = *reinterpret_cast<const float2*>(&sj[6][jj]);
        const float2 mjy = *reinterpret_cast<const float2*>(&sj[7][jj]);
        const float2 mjz = *reinterpret_cast<const float2*>(&sj[8][jj]);
#pragma unroll
        for (int r = 0; r < MIX_R; ++r)
            if (ALL || gv[r])
                pair_fp32x2<SELF>(P2[r], id2[r], jhx, jhy, jhz, jlx, jly, jlz, mjx, mjy, mjz, ii[r] - (jt + jj));
    }
}

__device__ __forceinline__ void dipole_mixed_items(Sys s, const WorkItem* __restrict__ items, int n_items,
                                                   int* counter) {
    // j tile, SoA: hi x, y, z; lo x, y, z; moment x, y, z (even padded)
    __shared__ __align__(16) float sj[9][MIX_TJ];
    __shared__ int s_item;
    const int64_t n = s.n;
    for (;;) {
        const int it = fetch_item(counter, &s_item);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        int ii[MIX_R];
        bool iv[MIX_R], gv[MIX_R];  // gv: the warp's 32 i of group r hold a particle (warp-uniform)
        IData id[MIX_R];
        Acc64 A64[MIX_R];
        Acc32 A32[MIX_R];
#pragma unroll
        for (int r = 0; r < MIX_R; ++r) {
            const int li = (int)threadIdx.x + r * MIX_BT;
            ii[r] = wi.i0 + li;
            iv[r] = li < wi.ni;
            gv[r] = r * MIX_BT + (int)(threadIdx.x & ~31u) < wi.ni;
            const int i = iv[r] ? ii[r] : wi.i0;
            id[r] = IData{s.xh[i], s.xh[n + i], s.xh[2 * n + i], s.xl[i], s.xl[n + i], s.xl[2 * n + i],
                          s.mf[i], s.mf[n + i], s.mf[2 * n + i]};
            A64[r] = Acc64{0, 0, 0, 0, 0, 0, 0};
            A32[r] = Acc32{0, 0, 0, 0, 0, 0, 0};
        }
        IData2 id2[MIX_R];
#pragma unroll
        for (int r = 0; r < MIX_R; ++r)
            id2[r] = IData2{bc2(id[r].hx), bc2(id[r].hy), bc2(id[r].hz), bc2(id[r].lx), bc2(id[r].ly),
                            bc2(id[r].lz), bc2(id[r].mx), bc2(id[r].my), bc2(id[r].mz)};
        const int jend = wi.j0 + wi.nj;
        for (int jt = wi.j0; jt < jend; jt += MIX_TJ) {
            const int jn = min(MIX_TJ, jend - jt);
            const int jn2 = (jn + 1) & ~1;
            __syncthreads();
            for (int l = threadIdx.x; l < jn2; l += MIX_BT) {
                // a missing j (odd tail): far away with zero moment
                float v[9] = {1e18f, 1e18f, 1e18f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (l < jn) {
                    const int j = jt + l;
                    v[0] = s.xh[j];
                    v[1] = s.xh[n + j];
                    v[2] = s.xh[2 * n + j];
                    v[3] = s.xl[j];
                    v[4] = s.xl[n + j];
                    v[5] = s.xl[2 * n + j];
                    v[6] = s.mf[j];
                    v[7] = s.mf[n + j];
                    v[8] = s.mf[2 * n + j];
                }
#pragma unroll
                for (int c9 = 0; c9 < 9; ++c9) sj[c9][l] = v[c9];
            }
            __syncthreads();
            const bool self_tile = (wi.i0 < jt + jn) && (wi.i0 + wi.ni > jt);
            Acc2 P2[MIX_R];
            const float2 z = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < MIX_R; ++r) P2[r] = Acc2{z, z, z, z, z, z, z};
            // a tile holding the item's own i takes the masked packed form
            // (the pair j = i contributes exact zeros)
            // with every group of 32 i holding particles (warp-uniform), the
            // loop runs without the per-group test, so that the compiler can
            // interleave the groups' dependency chains
            bool all = true;
#pragma unroll
            for (int r = 0; r < MIX_R; ++r) all = all && gv[r];
            if (all) {
                if (!self_tile)
                    mix_jloop<false, true>(P2, id2, gv, ii, sj, jn2, jt);
                else
                    mix_jloop<true, true>(P2, id2, gv, ii, sj, jn2, jt);
            } else {
                if (!self_tile)
                    mix_jloop<false, false>(P2, id2, gv, ii, sj, jn2, jt);
                else
                    mix_jloop<true, false>(P2, id2, gv, ii, sj, jn2, jt);
            }
#pragma unroll
            for (int r = 0; r < MIX_R; ++r) fold2(A32[r], P2[r]);
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

__global__ void __launch_bounds__(MIX_BT) k_dipole_mixed(Sys s, const WorkItem* __restrict__ items,
                                                         int n_items, int* counter) {
    dipole_mixed_items(s, items, n_items, counter);
}
// The same kernel with its registers capped at 144 (no spills), for the
// form beside the bond kernel: two blocks of it and two of the bond kernel
// then fit an SM's register file together (2 x 128 x 144 + 2 x 128 x 112).
__global__ void __maxnreg__(144) k_dipole_mixed_beside(Sys s, const WorkItem* __restrict__ items, int n_items,
                                                       int* counter) {
    dipole_mixed_items(s, items, n_items, counter);
}

// ---------------------------------------------------------------- symmetric FP64
// Each unordered pair evaluated once (Newton's third law): F_j = -F_ij and the
// field of i at x_j, in the accumulator convention of the finish kernel
// (F = 3c (F~ + m Bs), H = c H~):
//   F~_j += -(S r + (b/r^5) m_i),   Bs_j += -a/r^5,   H~_j += 3 (a/r^5) r - m_i/r^3.
// Items are pairs of supertiles (I <= J) of g tiles of SYM_BT particles.  A
// warp owns 32 i (one per lane, registers) and meets the 32 j of a j-subtile
// in 32 steps: at step s lane l takes j = (l + s) mod 32 from shared memory
// and holds that j's accumulator, which then moves to lane l - 1 by a
// shuffle.  After 32 steps every j accumulator is back in its home lane and
// holds the sum over the warp's 32 i, with no floating-point reduction work.
// The 4 warp partials of a j-subtile are summed in a fixed order into a
// shared-memory accumulator of the J supertile.  In a diagonal tile, warp w
// pairs its subtile with subtiles k > w symmetrically and with itself as
// ordered pairs (i side only).  i-side sums go to slot J and j-side sums to
// slot I (slot = partner supertile): each particle gets one partial per
// partner supertile, independent of scheduling.
constexpr int SYM_BT = 128;

// shared memory of k_dipole_sym_fp64, in doubles, for g tiles per supertile
__host__ __device__ constexpr int sym_smem_doubles(int g) { return 7 * g * SYM_BT + 4 * 4 * 7 * 32 + 10 * SYM_BT; }

// The j tile in shared memory, five double2 per particle: (x, y), (z, mx),
// (my, mz), and the moment times -5, (-5 mx, -5 my), (-5 mz, 0).  With -5 m_j
// stored, b5 = -5 m_j.r costs what b = m_j.r did and saves the
// multiplication by -5 in the pair term (GB300's FP64 pipe bounds the
// kernel).
struct JTile {
    const double2 *s01, *s23, *s45, *s67, *s89;
};
__device__ __forceinline__ void stage_j(double2* const (&S)[5], int slot, const Sys& s, int64_t n, int j, bool present) {
    // a missing j (ragged tile) is far away (r^2 within the range of the
    // fast reciprocal square root) with zero moment: it adds exactly zero
    double2 a01 = make_double2(1e15, 1e15), a23 = make_double2(1e15, 0.0), a45 = make_double2(0.0, 0.0);
    double2 a67 = make_double2(0.0, 0.0), a89 = make_double2(0.0, 0.0);
    if (present) {
        a01 = make_double2(s.x[j], s.x[n + j]);
        a23 = make_double2(s.x[2 * n + j], s.m[j]);
        a45 = make_double2(s.m[n + j], s.m[2 * n + j]);
        a67 = make_double2(-5.0 * a23.y, -5.0 * a45.x);
        a89 = make_double2(-5.0 * a45.y, 0.0);
    }
    S[0][slot] = a01;
    S[1][slot] = a23;
    S[2][slot] = a45;
    S[3][slot] = a67;
    S[4][slot] = a89;
}

// Accumulators of the symmetric kernel.  The field sum
// H~ = sum(3 b r / r^5 - m / r^3) is kept as its two parts, hb = sum b r / r^5
// and hm = sum m / r^3, combined once per tile as H~ = 3 hb - hm: this saves
// the two multiplications by 3 per pair on GB300's narrow FP64 pipe.  On the
// i side, hb and bs are kept times -5 (they are sums of -5 b / r^5 terms);
// i_side_h and i_side_bs undo that once per tile.
struct AccS {
    double fx, fy, fz, hbx, hby, hbz, hmx, hmy, hmz, bs;
};

__device__ __forceinline__ void shfl_acc(AccS& a, int src) {
    a.fx = __shfl_sync(0xffffffffu, a.fx, src);
    a.fy = __shfl_sync(0xffffffffu, a.fy, src);
    a.fz = __shfl_sync(0xffffffffu, a.fz, src);
    a.hbx = __shfl_sync(0xffffffffu, a.hbx, src);
    a.hby = __shfl_sync(0xffffffffu, a.hby, src);
    a.hbz = __shfl_sync(0xffffffffu, a.hbz, src);
    a.hmx = __shfl_sync(0xffffffffu, a.hmx, src);
    a.hmy = __shfl_sync(0xffffffffu, a.hmy, src);
    a.hmz = __shfl_sync(0xffffffffu, a.hmz, src);
    a.bs = __shfl_sync(0xffffffffu, a.bs, src);
}

__device__ __forceinline__ double i_side_bs(const AccS& a) { return -0.2 * a.bs; }
__device__ __forceinline__ d3 i_side_h(const AccS& a) {
    return mk3(fma(-0.6, a.hbx, -a.hmx), fma(-0.6, a.hby, -a.hmy), fma(-0.6, a.hbz, -a.hmz));
}

// one pair (i in registers, j from shared memory); SYM adds the j-side terms.
// mi5 = m_i / 5 (the j side's -b m_i / r^5 is then (-5 b / r^5) mi5).
template <bool SYM>
__device__ __forceinline__ void pair_sym(AccS& ai, AccS& aj, d3 xi, d3 mi, d3 mi5, const JTile& T, int jj,
                                         bool iv) {
    const double2 p01 = T.s01[jj], p23 = T.s23[jj], p45 = T.s45[jj], p67 = T.s67[jj], p89 = T.s89[jj];
    const double rx = xi.x - p01.x, ry = xi.y - p01.y, rz = xi.z - p23.x;
    const double mjx = p23.y, mjy = p45.x, mjz = p45.y;
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double rinv = rsqrt_nr(r2);
    const double rinv2 = rinv * rinv;
    const double rinv3 = rinv2 * rinv;
    const double rinv5 = rinv3 * rinv2;
    const double a = mi.x * rx + mi.y * ry + mi.z * rz;
    const double b5 = p67.x * rx + p67.y * ry + p89.x * rz;  // -5 b
    const double d = mi.x * mjx + mi.y * mjy + mi.z * mjz;
    const double sfac = fma(a * b5, rinv2, d);
    const double A = rinv5 * a;
    const double S = rinv5 * sfac;
    const double rb5 = rinv5 * b5;  // -5 b / r^5
    ai.fx = fma(A, mjx, fma(S, rx, ai.fx));
    ai.fy = fma(A, mjy, fma(S, ry, ai.fy));
    ai.fz = fma(A, mjz, fma(S, rz, ai.fz));
    ai.bs += rb5;
    ai.hbx = fma(rb5, rx, ai.hbx);
    ai.hby = fma(rb5, ry, ai.hby);
    ai.hbz = fma(rb5, rz, ai.hbz);
    ai.hmx = fma(rinv3, mjx, ai.hmx);
    ai.hmy = fma(rinv3, mjy, ai.hmy);
    ai.hmz = fma(rinv3, mjz, ai.hmz);
    if (SYM && iv) {
        // j side: r -> -r, a <-> b
        aj.fx = fma(-S, rx, fma(rb5, mi5.x, aj.fx));
        aj.fy = fma(-S, ry, fma(rb5, mi5.y, aj.fy));
        aj.fz = fma(-S, rz, fma(rb5, mi5.z, aj.fz));
        aj.hbx = fma(A, rx, aj.hbx);
        aj.hby = fma(A, ry, aj.hby);
        aj.hbz = fma(A, rz, aj.hbz);
        aj.hmx = fma(rinv3, mi.x, aj.hmx);
        aj.hmy = fma(rinv3, mi.y, aj.hmy);
        aj.hmz = fma(rinv3, mi.z, aj.hmz);
        aj.bs -= A;
    }
}

// RAGGED: the system has tiles that end early (rods of uneven length); warps
// of padding i and subtiles of padding j then skip their work.  Systems of
// whole tiles take the instantiation without those tests.
template <bool RAGGED>
__global__ void __launch_bounds__(SYM_BT, 4) k_dipole_sym_fp64(Sys s, const WorkItem* __restrict__ items,
                                                            int n_items, int* counter, int g) {
    extern __shared__ double sh[];
    const int st = g * SYM_BT;
    double* accJ = sh;                          // [7][st]
    double* wpart = sh + 7 * st;                // [4 warps][4 subtiles][7][32]
    double2* s01 = reinterpret_cast<double2*>(wpart + 4 * 4 * 7 * 32);  // the j tile (JTile) [5][SYM_BT]
    double2* const S5[5] = {s01, s01 + SYM_BT, s01 + 2 * SYM_BT, s01 + 3 * SYM_BT, s01 + 4 * SYM_BT};
    const JTile T{S5[0], S5[1], S5[2], S5[3], S5[4]};
    __shared__ int s_item;
    const int64_t n = s.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int from = (lane + 1) & 31;
    for (;;) {
        const int it = fetch_item(counter, &s_item);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        for (int k = tid; k < 7 * st; k += SYM_BT) accJ[k] = 0.0;
        const int nIt = (wi.ni + SYM_BT - 1) / SYM_BT, nJt = (wi.nj + SYM_BT - 1) / SYM_BT;
        for (int ti = 0; ti < nIt; ++ti) {
            const int li = ti * SYM_BT + tid;
            const bool iv = li < wi.ni;
            const int i = wi.i0 + (iv ? li : 0);
            const d3 xi = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
            const d3 mi = mk3(s.m[i], s.m[n + i], s.m[2 * n + i]);
            const d3 mi5 = mi * 0.2;
            AccS acc = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int tj = diag ? ti : 0; tj < nJt; ++tj) {
                const int jt = wi.j0 + tj * SYM_BT;
                const int jn = min(SYM_BT, wi.nj - tj * SYM_BT);
                const bool same = diag && tj == ti;
                __syncthreads();
                stage_j(S5, tid, s, n, jt + tid, tid < jn);
                __syncthreads();
                // a warp whose 32 i are all padding, or a j subtile beyond a
                // ragged tile's end, has no work (uniform across the warp)
                const bool wv = ti * SYM_BT + warp * 32 < wi.ni;
                for (int k = 0; k < 4; ++k) {
                    AccS aj = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
                    const int base = k * 32;
                    if (RAGGED && (!wv || base >= jn)) {
                    } else if (!same || k > warp) {
                        // symmetric: i-subtile `warp` against j-subtile k
                        for (int step = 0; step < 32; ++step) {
                            pair_sym<true>(acc, aj, xi, mi, mi5, T, base + ((lane + step) & 31), iv);
                            shfl_acc(aj, from);
                        }
                    } else if (k == warp) {
                        // same subtile: ordered pairs, i side only
                        for (int step = 1; step < 32; ++step)
                            pair_sym<false>(acc, aj, xi, mi, mi5, T, base + ((lane + step) & 31), iv);
                    }
                    double* W = wpart + (warp * 4 + k) * 7 * 32;
                    W[lane] = aj.fx;
                    W[32 + lane] = aj.fy;
                    W[64 + lane] = aj.fz;
                    W[96 + lane] = fma(3.0, aj.hbx, -aj.hmx);
                    W[128 + lane] = fma(3.0, aj.hby, -aj.hmy);
                    W[160 + lane] = fma(3.0, aj.hbz, -aj.hmz);
                    W[192 + lane] = aj.bs;
                }
                __syncthreads();
                // the 4 warp partials of every j of this tile, in a fixed order
                for (int idx = tid; idx < 7 * jn; idx += SYM_BT) {
                    const int c = idx / jn, jj = idx - c * jn;
                    const int k = jj >> 5, l = jj & 31;
                    const double* W0 = wpart + k * 7 * 32 + c * 32 + l;
                    const int ws = 4 * 7 * 32;
                    accJ[c * st + tj * SYM_BT + jj] += ((W0[0] + W0[ws]) + W0[2 * ws]) + W0[3 * ws];
                }
            }
            __syncthreads();
            if (iv) {
                const d3 h = i_side_h(acc);
                const double bs = i_side_bs(acc);
                if (diag) {
                    // same supertile: i and j sides share the particle's slot
                    const int l = ti * SYM_BT + tid;
                    accJ[l] += acc.fx;
                    accJ[st + l] += acc.fy;
                    accJ[2 * st + l] += acc.fz;
                    accJ[3 * st + l] += h.x;
                    accJ[4 * st + l] += h.y;
                    accJ[5 * st + l] += h.z;
                    accJ[6 * st + l] += bs;
                } else {
                    double* P = s.part + (int64_t)wi.slot * 7 * n;
                    P[i] = acc.fx;
                    P[n + i] = acc.fy;
                    P[2 * n + i] = acc.fz;
                    P[3 * n + i] = h.x;
                    P[4 * n + i] = h.y;
                    P[5 * n + i] = h.z;
                    P[6 * n + i] = bs;
                }
            }
        }
        __syncthreads();
        double* P = s.part + (int64_t)wi.pad0 * 7 * n;
        for (int l = tid; l < wi.nj; l += SYM_BT) {
            const int j = wi.j0 + l;
#pragma unroll
            for (int c = 0; c < 7; ++c) P[c * n + j] = accJ[c * st + l];
        }
    }
}

// ---------------------------------------------------------------- symmetric FP64, warp tiles
// The symmetric scheme with 32-particle tiles and one warp per pair of tiles
// (I <= J), for systems too small to fill the GPU with supertile pairs of
// 128: lane l holds i = tile I + l, the j of tile J rotate through the warp
// with their accumulators as in k_dipole_sym_fp64, a diagonal pair (I = J)
// evaluates its 32 x 31 ordered pairs on the i side only.  i-side sums go to
// slot `slot` (tile J) and j-side sums to slot `pad0` (tile I), so every
// particle gets one partial per partner tile, whatever the schedule.  Items
// are pulled per warp from the atomic queue.
__global__ void __launch_bounds__(128) k_dipole_symw_fp64(Sys s, const WorkItem* __restrict__ items, int n_items,
                                                           int* counter) {
    __shared__ double2 sjw[4][5][32];
    const int64_t n = s.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int from = (lane + 1) & 31;
    double2* const S5[5] = {sjw[warp][0], sjw[warp][1], sjw[warp][2], sjw[warp][3], sjw[warp][4]};
    const JTile T{S5[0], S5[1], S5[2], S5[3], S5[4]};
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        const bool iv = lane < wi.ni;
        const int i = wi.i0 + (iv ? lane : 0);
        const d3 xi = mk3(s.x[i], s.x[n + i], s.x[2 * n + i]);
        const d3 mi = mk3(s.m[i], s.m[n + i], s.m[2 * n + i]);
        const d3 mi5 = mi * 0.2;
        __syncwarp();
        stage_j(S5, lane, s, n, wi.j0 + lane, lane < wi.nj);
        __syncwarp();
        AccS acc = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, aj = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (diag) {
            for (int step = 1; step < 32; ++step)
                pair_sym<false>(acc, aj, xi, mi, mi5, T, (lane + step) & 31, iv);
        } else {
            for (int step = 0; step < 32; ++step) {
                pair_sym<true>(acc, aj, xi, mi, mi5, T, (lane + step) & 31, iv);
                shfl_acc(aj, from);
            }
        }
        if (iv) {
            double* P = s.part + (int64_t)wi.slot * 7 * n;
            P[i] = acc.fx;
            P[n + i] = acc.fy;
            P[2 * n + i] = acc.fz;
            const d3 h = i_side_h(acc);
            P[3 * n + i] = h.x;
            P[4 * n + i] = h.y;
            P[5 * n + i] = h.z;
            P[6 * n + i] = i_side_bs(acc);
        }
        if (!diag && lane < wi.nj) {
            const int j = wi.j0 + lane;
            double* P = s.part + (int64_t)wi.pad0 * 7 * n;
            P[j] = aj.fx;
            P[n + j] = aj.fy;
            P[2 * n + j] = aj.fz;
            P[3 * n + j] = fma(3.0, aj.hbx, -aj.hmx);
            P[4 * n + j] = fma(3.0, aj.hby, -aj.hmy);
            P[5 * n + j] = fma(3.0, aj.hbz, -aj.hmz);
            P[6 * n + j] = aj.bs;
        }
    }
}

// ---------------------------------------------------------------- symmetric mixed
// The symmetric scheme of k_dipole_sym_fp64 with FP32 pair terms (positions as
// FP32 hi/lo parts, as in k_dipole_mixed).  Tiles hold 256 particles in 8
// groups of 32; warp w owns i-groups w and w + 4 (two i per lane, sharing the
// j data and the rotating j accumulator of every step).  FP32 sums of one j
// tile are added to FP64 registers (i side) and to the FP64 shared-memory
// accumulator of the J supertile (j side) after every tile.
//
// Off-diagonal tiles use the packed FP32 arithmetic (f32x2): subtiles p and
// p + 4 are met together, the two halves of every packed value holding the
// pair with the j of subtile p and the j of subtile p + 4 at the same
// rotation offset, so one instruction does the work of two pairs and the
// rotating accumulator is a packed pair as well.  Each half performs exactly
// the arithmetic of pair_mix.  The FP32 FMA pipe then bounds the kernel
// (57 FMA-pipe operations per unordered pair) instead of instruction issue.
// Diagonal tiles, whose subtile pairs mix symmetric, ordered and skipped
// modes, keep the scalar path.
constexpr int MSYM_T = 256;   // particles per tile
constexpr int MSYM_BT = 128;  // threads
static_assert(MSYM_BT == 128, "flush_smem strides the FP64 i sums by 128 threads");

// SPLIT: the warp partials of two subtiles at a time (7 KB), reduced into
// the J sums as they are made, so that a plan whose shared memory limits the
// blocks per SM fits one more block; otherwise all eight subtiles (28 KB),
// reduced once per tile.  A64S: the FP64 i sums in shared memory (14 KB)
// instead of 28 registers per thread, for a fourth block per SM.
__host__ __device__ constexpr int msym_smem_bytes(int g, bool split, bool a64s = false) {
    return 7 * g * MSYM_T * 8                  // accJ (FP64)
           + (a64s ? 2 * 7 * MSYM_BT * 8 : 0)  // FP64 i sums
           + 4 * (split ? 2 : 8) * 7 * 32 * 4  // warp partials (FP32)
           + MSYM_T * (16 + 16 + 4);           // J tile: float4, float4, float
}



// the factor that restores component c of the j-side sums of pair_mix
// (-f, H/3, -b)
__device__ __forceinline__ double msym_jscale(int c) { return (c >= 3 && c <= 5) ? 3.0 : -1.0; }

// Adds the four warps' FP32 partials of subtile sa (buffer half 0) and, when
// sb >= 0, subtile sb (half 1) to the FP64 accumulator of the J supertile,
// summed in a fixed order in FP32, then one conversion and one FP64 FMA with
// the restoring factor (the FP64 pipe runs at 1/64 of the FP32 rate).  wpart
// is [warp][half][7][32].
__device__ __forceinline__ void msym_reduce(double* accJ, const float* wpart, int st, int col0, int jn, int sa,
                                            int sb, int tid) {
    for (int idx = tid; idx < 7 * 64; idx += MSYM_BT) {
        const int c = idx >> 6, r = idx & 63, h = r >> 5, l = r & 31;
        const int sub = h ? sb : sa;
        const int jj = sub * 32 + l;
        if (sub < 0 || jj >= jn) continue;
        const float* W0 = wpart + h * 224 + c * 32 + l;
        const int ws = 2 * 224;
        double& acc = accJ[c * st + col0 + jj];
        acc = fma(msym_jscale(c), (double)(((W0[0] + W0[ws]) + W0[2 * ws]) + W0[3 * ws]), acc);
    }
}

__device__ __forceinline__ void shfl_acc32(Acc32& a, int src) {
    a.fx = __shfl_sync(0xffffffffu, a.fx, src);
    a.fy = __shfl_sync(0xffffffffu, a.fy, src);
    a.fz = __shfl_sync(0xffffffffu, a.fz, src);
    a.hx = __shfl_sync(0xffffffffu, a.hx, src);
    a.hy = __shfl_sync(0xffffffffu, a.hy, src);
    a.hz = __shfl_sync(0xffffffffu, a.hz, src);
    a.bs = __shfl_sync(0xffffffffu, a.bs, src);
}

// One pair in FP32: i side always, j side when SYM.  The sums are kept in
// scaled forms that need no negation or factor 3 per pair: the i side holds
// f, H/3 and b; the j side -f, H/3 and -b (msym_reduce and the i-side writes
// restore them).  With c = -1/(3 r^3):
//   i: f += A m_j + S r,  H/3 += (m_j.r / r^5) r + c m_j,  b += m_j.r / r^5
//   j: -f += S r + (m_j.r / r^5) m_i,  H/3 += A r + c m_i,  -b += A
// where A = m_i.r / r^5 and S = (m_i.m_j - 5 (m_i.r)(m_j.r) / r^2) / r^5.
template <bool SYM>
__device__ __forceinline__ void pair_mix(Acc32& ai, Acc32& aj, const IData& id, float4 j0, float4 j1, float mjz) {
    const float rx = (id.hx - j0.x) + (id.lx - j0.w);
    const float ry = (id.hy - j0.y) + (id.ly - j1.x);
    const float rz = (id.hz - j0.z) + (id.lz - j1.y);
    const float mjx = j1.z, mjy = j1.w;
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    float rinv;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv) : "f"(r2));
    const float rinv2 = rinv * rinv;
    const float rinv3 = rinv2 * rinv;
    const float rinv5 = rinv3 * rinv2;
    const float a = fmaf(id.mx, rx, fmaf(id.my, ry, id.mz * rz));
    const float b = fmaf(mjx, rx, fmaf(mjy, ry, mjz * rz));
    const float d = fmaf(id.mx, mjx, fmaf(id.my, mjy, id.mz * mjz));
    const float sfac = fmaf(-5.0f * a * b, rinv2, d);
    const float A = rinv5 * a;
    const float S = rinv5 * sfac;
    const float rb5 = rinv5 * b;
    const float c = rinv3 * (-1.0f / 3.0f);
    ai.fx = fmaf(A, mjx, fmaf(S, rx, ai.fx));
    ai.fy = fmaf(A, mjy, fmaf(S, ry, ai.fy));
    ai.fz = fmaf(A, mjz, fmaf(S, rz, ai.fz));
    ai.bs += rb5;
    ai.hx = fmaf(c, mjx, fmaf(rb5, rx, ai.hx));
    ai.hy = fmaf(c, mjy, fmaf(rb5, ry, ai.hy));
    ai.hz = fmaf(c, mjz, fmaf(rb5, rz, ai.hz));
    if (SYM) {
        aj.fx = fmaf(S, rx, fmaf(rb5, id.mx, aj.fx));
        aj.fy = fmaf(S, ry, fmaf(rb5, id.my, aj.fy));
        aj.fz = fmaf(S, rz, fmaf(rb5, id.mz, aj.fz));
        aj.hx = fmaf(A, rx, fmaf(c, id.mx, aj.hx));
        aj.hy = fmaf(A, ry, fmaf(c, id.my, aj.hy));
        aj.hz = fmaf(A, rz, fmaf(c, id.mz, aj.hz));
        aj.bs += A;
    }
}

// one i against two j (packed halves) in FP32, the arithmetic and the scaled
// sums of pair_mix in each half
// (SELF: the half `self` holds the pair of the lane's i with itself, whose
// r is exactly zero; its 1/r := 0 makes every term of that half an exact zero)
template <bool SYM, bool SELF = false>
__device__ __forceinline__ void pair_mix2(Acc2& ai, Acc2& aj, const IData2& I, float2 jhx, float2 jhy,
                                          float2 jhz, float2 jlx, float2 jly, float2 jlz, float2 mjx,
                                          float2 mjy, float2 mjz, int self = -1) {
    const float2 rx = __fadd2_rn(__fadd2_rn(I.hx, make_float2(-jhx.x, -jhx.y)), __fadd2_rn(I.lx, make_float2(-jlx.x, -jlx.y)));
    const float2 ry = __fadd2_rn(__fadd2_rn(I.hy, make_float2(-jhy.x, -jhy.y)), __fadd2_rn(I.ly, make_float2(-jly.x, -jly.y)));
    const float2 rz = __fadd2_rn(__fadd2_rn(I.hz, make_float2(-jhz.x, -jhz.y)), __fadd2_rn(I.lz, make_float2(-jlz.x, -jlz.y)));
    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __fmul2_rn(rz, rz)));
    float2 rinv;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv.x) : "f"(r2.x));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rinv.y) : "f"(r2.y));
    if (SELF) {
        if (self == 0) rinv.x = 0.f;
        if (self == 1) rinv.y = 0.f;
    }
    const float2 rinv2 = __fmul2_rn(rinv, rinv);
    const float2 rinv3 = __fmul2_rn(rinv2, rinv);
    const float2 rinv5 = __fmul2_rn(rinv3, rinv2);
    const float2 a = __ffma2_rn(I.mx, rx, __ffma2_rn(I.my, ry, __fmul2_rn(I.mz, rz)));
    const float2 b = __ffma2_rn(mjx, rx, __ffma2_rn(mjy, ry, __fmul2_rn(mjz, rz)));
    const float2 d = __ffma2_rn(I.mx, mjx, __ffma2_rn(I.my, mjy, __fmul2_rn(I.mz, mjz)));
    const float2 sfac = __ffma2_rn(__fmul2_rn(__fmul2_rn(bc2(-5.0f), a), b), rinv2, d);
    const float2 A = __fmul2_rn(rinv5, a);
    const float2 S = __fmul2_rn(rinv5, sfac);
    const float2 rb5 = __fmul2_rn(rinv5, b);
    const float2 c = __fmul2_rn(rinv3, bc2(-1.0f / 3.0f));
    ai.fx = __ffma2_rn(A, mjx, __ffma2_rn(S, rx, ai.fx));
    ai.fy = __ffma2_rn(A, mjy, __ffma2_rn(S, ry, ai.fy));
    ai.fz = __ffma2_rn(A, mjz, __ffma2_rn(S, rz, ai.fz));
    ai.bs = __fadd2_rn(ai.bs, rb5);
    ai.hx = __ffma2_rn(c, mjx, __ffma2_rn(rb5, rx, ai.hx));
    ai.hy = __ffma2_rn(c, mjy, __ffma2_rn(rb5, ry, ai.hy));
    ai.hz = __ffma2_rn(c, mjz, __ffma2_rn(rb5, rz, ai.hz));
    if (SYM) {
        aj.fx = __ffma2_rn(S, rx, __ffma2_rn(rb5, I.mx, aj.fx));
        aj.fy = __ffma2_rn(S, ry, __ffma2_rn(rb5, I.my, aj.fy));
        aj.fz = __ffma2_rn(S, rz, __ffma2_rn(rb5, I.mz, aj.fz));
        aj.hx = __ffma2_rn(A, rx, __ffma2_rn(c, I.mx, aj.hx));
        aj.hy = __ffma2_rn(A, ry, __ffma2_rn(c, I.my, aj.hy));
        aj.hz = __ffma2_rn(A, rz, __ffma2_rn(c, I.mz, aj.hz));
        aj.bs = __fadd2_rn(aj.bs, A);
    }
}

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ void shfl_acc2(Acc2& a, int src) {
    a.fx = shfl2(a.fx, src);
    a.fy = shfl2(a.fy, src);
    a.fz = shfl2(a.fz, src);
    a.hx = shfl2(a.hx, src);
    a.hy = shfl2(a.hy, src);
    a.hz = shfl2(a.hz, src);
    a.bs = shfl2(a.bs, src);
}

// mode of (i-group a, j-subtile b): 0 skip, 1 symmetric, 2 same group
// (ordered pairs, i side only)
__device__ __forceinline__ int msym_mode(bool same_tile, int a, int b) {
    if (!same_tile) return 1;
    return b > a ? 1 : (b == a ? 2 : 0);
}

// One j subtile of a diagonal tile against the lane's two i, with the
// groups' modes fixed at compile time (M0 for group warp, M1 for group
// warp + 4; 0 skip, 1 symmetric, 2 the group's own subtile: ordered pairs
// without the self pair at step 0), so that no test splits the step loop.
// A lane past the i range holds the far stand-in, whose symmetric terms add
// exact zeros to the j sums.
template <int M0, int M1>
__device__ __forceinline__ void msym_diag_sub(Acc32 (&A32)[2], Acc32& aj, const IData (&id)[2], const float4* sA,
                                              const float4* sB, const float* sZ, int base, int lane, int from) {
    constexpr bool OWN = M0 == 2 || M1 == 2;
    if (OWN) {
        // step 0 of the own subtile is the self pair: the symmetric group only
        const int jj = base + lane;
        const float4 j0 = sA[jj], j1 = sB[jj];
        const float mjz = sZ[jj];
        if (M0 == 1) pair_mix<true>(A32[0], aj, id[0], j0, j1, mjz);
        if (M1 == 1) pair_mix<true>(A32[1], aj, id[1], j0, j1, mjz);
        shfl_acc32(aj, from);
    }
#pragma unroll 2
    for (int step = OWN ? 1 : 0; step < 32; ++step) {
        const int jj = base + ((lane + step) & 31);
        const float4 j0 = sA[jj], j1 = sB[jj];
        const float mjz = sZ[jj];
        if (M0 == 1) pair_mix<true>(A32[0], aj, id[0], j0, j1, mjz);
        if (M0 == 2) pair_mix<false>(A32[0], aj, id[0], j0, j1, mjz);
        if (M1 == 1) pair_mix<true>(A32[1], aj, id[1], j0, j1, mjz);
        if (M1 == 2) pair_mix<false>(A32[1], aj, id[1], j0, j1, mjz);
        shfl_acc32(aj, from);
    }
}

// MINB 4: the SPLIT layout with the FP64 i sums in shared memory and
// registers for 4 blocks per SM; MINB 3: the SPLIT layout with registers for
// 3 blocks per SM; MINB 2: the full layout
template <int MINB>
__global__ void __launch_bounds__(MSYM_BT, MINB) k_dipole_sym_mixed(Sys s, const WorkItem* __restrict__ items,
                                                                 int n_items, int* counter, int g) {
    constexpr bool SPLIT = MINB >= 3;
    constexpr bool A64S = MINB >= 4;
    constexpr int WH = SPLIT ? 2 : 8;  // subtile slots per warp in wpart
    extern __shared__ __align__(16) unsigned char shb[];
    const int st = g * MSYM_T;
    double* accJ = reinterpret_cast<double*>(shb);                       // [7][st]
    double* a64s = accJ + 7 * st;                                        // [2][7][MSYM_BT] when A64S
    float* wpart = reinterpret_cast<float*>(a64s + (A64S ? 2 * 7 * MSYM_BT : 0));  // [4][WH][7][32]
    float4* sA = reinterpret_cast<float4*>(wpart + 4 * WH * 7 * 32);     // [MSYM_T]
    float4* sB = sA + MSYM_T;
    float* sZ = reinterpret_cast<float*>(sB + MSYM_T);
    __shared__ int s_item;
    const int64_t n = s.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int from = (lane + 1) & 31;
    for (;;) {
        const int it = fetch_item(counter, &s_item);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        for (int k = tid; k < 7 * st; k += MSYM_BT) accJ[k] = 0.0;
        const int nIt = (wi.ni + MSYM_T - 1) / MSYM_T, nJt = (wi.nj + MSYM_T - 1) / MSYM_T;
        for (int ti = 0; ti < nIt; ++ti) {
            // the two i of this lane: groups warp and warp + 4
            int li[2];
            bool iv[2];
            int ii[2];
            IData2 id2[2];  // i data broadcast to both halves
            Acc64 A64[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                li[r] = ti * MSYM_T + (warp + 4 * r) * 32 + lane;
                iv[r] = li[r] < wi.ni;
                ii[r] = wi.i0 + (iv[r] ? li[r] : 0);
                id2[r] = i_data2(s, n, ii[r], iv[r]);
                A64[r] = Acc64{0, 0, 0, 0, 0, 0, 0};
                if constexpr (A64S)
                    for (int c = 0; c < 7; ++c) a64s[(r * 7 + c) * MSYM_BT + tid] = 0.0;
            }
            for (int tj = diag ? ti : 0; tj < nJt; ++tj) {
                const int jt = wi.j0 + tj * MSYM_T;
                const int jn = min(MSYM_T, wi.nj - tj * MSYM_T);
                const bool same = diag && tj == ti;
                __syncthreads();
                for (int l = tid; l < MSYM_T; l += MSYM_BT) {
                    // missing j of a ragged tile: far away, zero moment
                    float4 a = make_float4(1e18f, 1e18f, 1e18f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
                    float z = 0.f;
                    if (l < jn) {
                        const int j = jt + l;
                        a = make_float4(s.xh[j], s.xh[n + j], s.xh[2 * n + j], s.xl[j]);
                        b = make_float4(s.xl[n + j], s.xl[2 * n + j], s.mf[j], s.mf[n + j]);
                        z = s.mf[2 * n + j];
                    }
                    if (same) {
                        sA[l] = a;
                        sB[l] = b;
                        sZ[l] = z;
                    } else {
                        // packed layout over the same storage: for subtile
                        // pair p and offset o, Q0 = (hx, hx', hy, hy'),
                        // Q1 = (hz, hz', lx, lx'), Q2 = (ly, ly', lz, lz'),
                        // Q3 = (mx, mx', my, my'), Q4 = (mz, mz'), where '
                        // marks the j of subtile p + 4
                        const int sub = l >> 5, h = sub >> 2, q = (sub & 3) * 32 + (l & 31);
                        float* Q = reinterpret_cast<float*>(sA);
                        Q[4 * q + h] = a.x;
                        Q[4 * q + 2 + h] = a.y;
                        Q[512 + 4 * q + h] = a.z;
                        Q[512 + 4 * q + 2 + h] = a.w;
                        Q[1024 + 4 * q + h] = b.x;
                        Q[1024 + 4 * q + 2 + h] = b.y;
                        Q[1536 + 4 * q + h] = b.z;
                        Q[1536 + 4 * q + 2 + h] = b.w;
                        Q[2048 + 2 * q + h] = z;
                    }
                }
                __syncthreads();
                Acc32 A32[2] = {Acc32{0, 0, 0, 0, 0, 0, 0}, Acc32{0, 0, 0, 0, 0, 0, 0}};
                if (!same) {
                    const float4* Q0 = sA;
                    const float4* Q1 = sA + 128;
                    const float4* Q2 = sA + 256;
                    const float4* Q3 = sA + 384;
                    const float2* Q4 = reinterpret_cast<const float2*>(sA + 512);
                    const float2 z2 = make_float2(0.f, 0.f);
                    Acc2 P2[2] = {Acc2{z2, z2, z2, z2, z2, z2, z2}, Acc2{z2, z2, z2, z2, z2, z2, z2}};
                    for (int p = 0; p < 4; ++p) {
                        Acc2 aj = Acc2{z2, z2, z2, z2, z2, z2, z2};
#pragma unroll 2
                        for (int step = 0; step < 32; ++step) {
                            const int q = p * 32 + ((lane + step) & 31);
                            const float4 q0 = Q0[q], q1 = Q1[q], q2 = Q2[q], q3 = Q3[q];
                            const float2 q4 = Q4[q];
                            const float2 jhx = make_float2(q0.x, q0.y), jhy = make_float2(q0.z, q0.w);
                            const float2 jhz = make_float2(q1.x, q1.y), jlx = make_float2(q1.z, q1.w);
                            const float2 jly = make_float2(q2.x, q2.y), jlz = make_float2(q2.z, q2.w);
                            const float2 mjx = make_float2(q3.x, q3.y), mjy = make_float2(q3.z, q3.w);
#pragma unroll
                            for (int r = 0; r < 2; ++r)
                                pair_mix2<true>(P2[r], aj, id2[r], jhx, jhy, jhz, jlx, jly, jlz, mjx, mjy, q4);
                            shfl_acc2(aj, from);
                        }
                        float* Wa = wpart + (warp * WH + (SPLIT ? 0 : p)) * 7 * 32;
                        float* Wb = wpart + (warp * WH + (SPLIT ? 1 : p + 4)) * 7 * 32;
                        Wa[lane] = aj.fx.x;
                        Wa[32 + lane] = aj.fy.x;
                        Wa[64 + lane] = aj.fz.x;
                        Wa[96 + lane] = aj.hx.x;
                        Wa[128 + lane] = aj.hy.x;
                        Wa[160 + lane] = aj.hz.x;
                        Wa[192 + lane] = aj.bs.x;
                        Wb[lane] = aj.fx.y;
                        Wb[32 + lane] = aj.fy.y;
                        Wb[64 + lane] = aj.fz.y;
                        Wb[96 + lane] = aj.hx.y;
                        Wb[128 + lane] = aj.hy.y;
                        Wb[160 + lane] = aj.hz.y;
                        Wb[192 + lane] = aj.bs.y;
                        if constexpr (SPLIT) {
                            // subtiles p and p + 4 of all warps into the J sums
                            __syncthreads();
                            msym_reduce(accJ, wpart, st, tj * MSYM_T, jn, p, p + 4, tid);
                            __syncthreads();
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 2; ++r) fold2(A32[r], P2[r]);
                } else {
                  const IData id[2] = {
                      IData{id2[0].hx.x, id2[0].hy.x, id2[0].hz.x, id2[0].lx.x, id2[0].ly.x, id2[0].lz.x, id2[0].mx.x,
                            id2[0].my.x, id2[0].mz.x},
                      IData{id2[1].hx.x, id2[1].hy.x, id2[1].hz.x, id2[1].lx.x, id2[1].ly.x, id2[1].lz.x, id2[1].mx.x,
                            id2[1].my.x, id2[1].mz.x}};
                  for (int sub = 0; sub < 8; ++sub) {
                    const int m0 = msym_mode(same, warp, sub), m1 = msym_mode(same, warp + 4, sub);
                    Acc32 aj = {0, 0, 0, 0, 0, 0, 0};
                    const int base = sub * 32;
                    // the combinations a warp meets: sub < warp (0, 0),
                    // sub == warp (2, 0), warp < sub < warp + 4 (1, 0),
                    // sub == warp + 4 (1, 2), sub > warp + 4 (1, 1)
                    if (m0 == 2)
                        msym_diag_sub<2, 0>(A32, aj, id, sA, sB, sZ, base, lane, from);
                    else if (m0 == 1 && m1 == 0)
                        msym_diag_sub<1, 0>(A32, aj, id, sA, sB, sZ, base, lane, from);
                    else if (m0 == 1 && m1 == 2)
                        msym_diag_sub<1, 2>(A32, aj, id, sA, sB, sZ, base, lane, from);
                    else if (m0 == 1 && m1 == 1)
                        msym_diag_sub<1, 1>(A32, aj, id, sA, sB, sZ, base, lane, from);
                    float* W = wpart + (warp * WH + (SPLIT ? 0 : sub)) * 7 * 32;
                    W[lane] = aj.fx;
                    W[32 + lane] = aj.fy;
                    W[64 + lane] = aj.fz;
                    W[96 + lane] = aj.hx;
                    W[128 + lane] = aj.hy;
                    W[160 + lane] = aj.hz;
                    W[192 + lane] = aj.bs;
                    if constexpr (SPLIT) {
                        __syncthreads();
                        msym_reduce(accJ, wpart, st, tj * MSYM_T, jn, sub, -1, tid);
                        __syncthreads();
                    }
                  }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if constexpr (A64S)
                        flush_smem(a64s, r, tid, A32[r]);
                    else
                        flush(A64[r], A32[r]);
                }
                if constexpr (!SPLIT) {
                    __syncthreads();
                    for (int idx = tid; idx < 7 * jn; idx += MSYM_BT) {
                        const int c = idx / jn, jj = idx - c * jn;
                        const int sub = jj >> 5, l = jj & 31;
                        const float* W0 = wpart + sub * 7 * 32 + c * 32 + l;
                        const int ws = 8 * 7 * 32;
                        // the order and arithmetic of msym_reduce
                        double& acc = accJ[c * st + tj * MSYM_T + jj];
                        acc = fma(msym_jscale(c), (double)(((W0[0] + W0[ws]) + W0[2 * ws]) + W0[3 * ws]), acc);
                    }
                }
            }
            __syncthreads();
            if constexpr (A64S) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const double* A = a64s + r * 7 * MSYM_BT + tid;
                    A64[r] = Acc64{A[0], A[MSYM_BT], A[2 * MSYM_BT], A[3 * MSYM_BT], A[4 * MSYM_BT], A[5 * MSYM_BT],
                                   A[6 * MSYM_BT]};
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (!iv[r]) continue;
                // the i side holds H/3
                if (diag) {
                    const int l = li[r];
                    accJ[l] += A64[r].fx;
                    accJ[st + l] += A64[r].fy;
                    accJ[2 * st + l] += A64[r].fz;
                    accJ[3 * st + l] = fma(3.0, A64[r].hx, accJ[3 * st + l]);
                    accJ[4 * st + l] = fma(3.0, A64[r].hy, accJ[4 * st + l]);
                    accJ[5 * st + l] = fma(3.0, A64[r].hz, accJ[5 * st + l]);
                    accJ[6 * st + l] += A64[r].bs;
                } else {
                    const int i = ii[r];
                    double* P = s.part + (int64_t)wi.slot * 7 * n;
                    P[i] = A64[r].fx;
                    P[n + i] = A64[r].fy;
                    P[2 * n + i] = A64[r].fz;
                    P[3 * n + i] = 3.0 * A64[r].hx;
                    P[4 * n + i] = 3.0 * A64[r].hy;
                    P[5 * n + i] = 3.0 * A64[r].hz;
                    P[6 * n + i] = A64[r].bs;
                }
            }
        }
        __syncthreads();
        double* P = s.part + (int64_t)wi.pad0 * 7 * n;
        for (int l = tid; l < wi.nj; l += MSYM_BT) {
            const int j = wi.j0 + l;
#pragma unroll
            for (int c = 0; c < 7; ++c) P[c * n + j] = accJ[c * st + l];
        }
    }
}

}  // namespace

int dipole_tile_i(bool mixed, const DipoleCfg&) { return mixed ? MIX_BT * MIX_R : FP64_BT; }

// The largest dynamic shared memory a kernel may take is an attribute of the
// function, shared by every handle of the process, so it is set once to the
// device's limit and never to one plan's size (a plan with more shared memory,
// tuned for another handle, would otherwise fail to launch).  Also prefers
// all of the SM's unified L1/shared storage as shared memory.  Returns
// whether smem bytes fit.
bool allow_dynamic_smem(const void* fn, size_t smem) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int lim = optin - (int)fa.sharedSizeBytes;
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaGetLastError();
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return smem <= (size_t)lim;
}

int dipole_blocks_per_sm(bool mixed) {
    int b = 0;
    if (mixed)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_mixed, MIX_BT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_fp64, FP64_BT, 0);
    return b;
}

int dipole_sym_tile(bool mixed) { return mixed ? MSYM_T : SYM_BT; }

namespace {
// ---------------------------------------------------------------- symmetric mixed, warp tiles
// The symmetric FP32-pair scheme with 64-particle tiles and one warp per pair
// of tiles (I <= J), for systems of many short rods, which 256-particle tiles
// would mostly pad.  Lane l holds i = I + l and I + 32 + l and meets the j of
// tile J in packed pairs (J + q, J + 32 + q) at rotation offset q, with the
// arithmetic of pair_mix2 and its rotating packed j accumulator.  A diagonal
// pair (I = J) evaluates its ordered pairs on the i side only.  The FP32 sums
// of one item (at most 64 terms per particle and side) become one FP64
// partial: the i side in slot `slot` (tile J), the j side in slot `pad0`
// (tile I), so every particle gets one partial per partner tile, whatever the
// schedule.  Items are pulled per warp from the atomic queue.
constexpr int MSYMW_BT = 128;

__global__ void __launch_bounds__(MSYMW_BT, 4) k_dipole_symw_mixed(Sys s, const WorkItem* __restrict__ items,
                                                                   int n_items, int* counter) {
    // per warp, the packed j tile: Q0 .. Q3 (float4 [32]) and Q4 (float2 [32])
    // in the layout of k_dipole_sym_mixed with one subtile pair
    __shared__ __align__(16) float4 sq[MSYMW_BT / 32][4 * 32 + 16];
    const int64_t n = s.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int from = (lane + 1) & 31;
    const float4* Q0 = sq[warp];
    const float4* Q1 = Q0 + 32;
    const float4* Q2 = Q0 + 64;
    const float4* Q3 = Q0 + 96;
    const float2* Q4 = reinterpret_cast<const float2*>(Q0 + 128);
    float* Q = reinterpret_cast<float*>(sq[warp]);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        bool iv[2];
        int ii[2];
        IData2 id2[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int li = r * 32 + lane;
            iv[r] = li < wi.ni;
            ii[r] = wi.i0 + (iv[r] ? li : 0);
            id2[r] = i_data2(s, n, ii[r], iv[r]);
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // a missing j of a ragged tile: far away, zero moment
            const int l = h * 32 + lane;
            float v[9] = {1e18f, 1e18f, 1e18f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (l < wi.nj) {
                const int j = wi.j0 + l;
                v[0] = s.xh[j];
                v[1] = s.xh[n + j];
                v[2] = s.xh[2 * n + j];
                v[3] = s.xl[j];
                v[4] = s.xl[n + j];
                v[5] = s.xl[2 * n + j];
                v[6] = s.mf[j];
                v[7] = s.mf[n + j];
                v[8] = s.mf[2 * n + j];
            }
            for (int k = 0; k < 4; ++k) {
                Q[128 * k + 4 * lane + h] = v[2 * k];
                Q[128 * k + 4 * lane + 2 + h] = v[2 * k + 1];
            }
            Q[512 + 2 * lane + h] = v[8];
        }
        __syncwarp();
        const float2 z2 = make_float2(0.f, 0.f);
        Acc2 P2[2] = {Acc2{z2, z2, z2, z2, z2, z2, z2}, Acc2{z2, z2, z2, z2, z2, z2, z2}};
        Acc2 aj = Acc2{z2, z2, z2, z2, z2, z2, z2};
        auto pass = [&](auto diag_c) {
            constexpr bool DIAG = decltype(diag_c)::value;
#pragma unroll 2
            for (int step = 0; step < 32; ++step) {
                const int q = (lane + step) & 31;
                const float4 q0 = Q0[q], q1 = Q1[q], q2 = Q2[q], q3 = Q3[q];
                const float2 q4 = Q4[q];
                const float2 jhx = make_float2(q0.x, q0.y), jhy = make_float2(q0.z, q0.w);
                const float2 jhz = make_float2(q1.x, q1.y), jlx = make_float2(q1.z, q1.w);
                const float2 jly = make_float2(q2.x, q2.y), jlz = make_float2(q2.z, q2.w);
                const float2 mjx = make_float2(q3.x, q3.y), mjy = make_float2(q3.z, q3.w);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (DIAG) {
                        // i = I + 32 r + lane meets itself in half r at step 0
                        pair_mix2<false, true>(P2[r], aj, id2[r], jhx, jhy, jhz, jlx, jly, jlz, mjx, mjy, q4,
                                               step == 0 ? r : -1);
                    } else {
                        pair_mix2<true>(P2[r], aj, id2[r], jhx, jhy, jhz, jlx, jly, jlz, mjx, mjy, q4);
                    }
                }
                if (!DIAG) shfl_acc2(aj, from);
            }
        };
        if (diag) pass(std::integral_constant<bool, true>{});
        else pass(std::integral_constant<bool, false>{});
        // i side (the field held over 3, as in pair_mix)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!iv[r]) continue;
            const int i = ii[r];
            double* P = s.part + (int64_t)wi.slot * 7 * n;
            P[i] = (double)(P2[r].fx.x + P2[r].fx.y);
            P[n + i] = (double)(P2[r].fy.x + P2[r].fy.y);
            P[2 * n + i] = (double)(P2[r].fz.x + P2[r].fz.y);
            P[3 * n + i] = 3.0 * (double)(P2[r].hx.x + P2[r].hx.y);
            P[4 * n + i] = 3.0 * (double)(P2[r].hy.x + P2[r].hy.y);
            P[5 * n + i] = 3.0 * (double)(P2[r].hz.x + P2[r].hz.y);
            P[6 * n + i] = (double)(P2[r].bs.x + P2[r].bs.y);
        }
        if (!diag) {
            // j side, back at lane l after 32 rotations: half h is j = J + 32 h + l
            // (held as -f, H/3 and -b)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int l = h * 32 + lane;
                if (l >= wi.nj) continue;
                const int j = wi.j0 + l;
                double* P = s.part + (int64_t)wi.pad0 * 7 * n;
                P[j] = -(double)(h ? aj.fx.y : aj.fx.x);
                P[n + j] = -(double)(h ? aj.fy.y : aj.fy.x);
                P[2 * n + j] = -(double)(h ? aj.fz.y : aj.fz.x);
                P[3 * n + j] = 3.0 * (double)(h ? aj.hx.y : aj.hx.x);
                P[4 * n + j] = 3.0 * (double)(h ? aj.hy.y : aj.hy.x);
                P[5 * n + j] = 3.0 * (double)(h ? aj.hz.y : aj.hz.x);
                P[6 * n + j] = -(double)(h ? aj.bs.y : aj.bs.x);
            }
        }
    }
}

template <int MINB>
int msym_occupancy(int smem) {
    if (!allow_dynamic_smem((const void*)k_dipole_sym_mixed<MINB>, (size_t)smem)) return 0;  // not runnable
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_sym_mixed<MINB>, MSYM_BT, smem);
    return b;
}
// the layout of each g: the one with more blocks per SM; on a tie the full
// layout (more registers, one reduction per tile)
struct MsymVariant {
    int minb, b;
};
MsymVariant msym_variant(int g) {
    static MsymVariant cache[9] = {};
    static std::once_flag once[9];
    std::call_once(once[g], [g] {
        const int b2 = msym_occupancy<2>(msym_smem_bytes(g, false)), b3 = msym_occupancy<3>(msym_smem_bytes(g, true)),
                  b4 = msym_occupancy<4>(msym_smem_bytes(g, true, true));
        cache[g] = b4 > b3 && b4 > b2 ? MsymVariant{4, b4} : (b3 > b2 ? MsymVariant{3, b3} : MsymVariant{2, b2});
    });
    return cache[g];
}
}  // namespace

int dipole_sym_blocks_per_sm(bool mixed, int g) {
    int b = 0;
    if (g < 1 || g > 8) return 0;
    if (mixed) return msym_variant(g).b;
    const size_t smem = (size_t)sym_smem_doubles(g) * sizeof(double);
    for (auto k : {k_dipole_sym_fp64<false>, k_dipole_sym_fp64<true>})
        if (!allow_dynamic_smem((const void*)k, smem)) return 0;  // the plan is not runnable
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_sym_fp64<false>, SYM_BT, smem);
    return b;
}

cudaError_t launch_dipole_sym(const Sys& s, bool mixed, const WorkItem* items, int n_items, int* counter,
                              int g, int blocks, bool ragged, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (mixed) {
        if (g < 1 || g > 8) return cudaErrorInvalidValue;
        const int grid = blocks > 0 ? blocks : n_items;
        switch (msym_variant(g).minb) {
            case 4: k_dipole_sym_mixed<4><<<grid, MSYM_BT, msym_smem_bytes(g, true, true), st>>>(s, items, n_items, counter, g); break;
            case 3: k_dipole_sym_mixed<3><<<grid, MSYM_BT, msym_smem_bytes(g, true), st>>>(s, items, n_items, counter, g); break;
            case 2: k_dipole_sym_mixed<2><<<grid, MSYM_BT, msym_smem_bytes(g, false), st>>>(s, items, n_items, counter, g); break;
            default: return cudaErrorInvalidConfiguration;  // no variant fits this g
        }
        return cudaGetLastError();
    }
    const size_t smem = (size_t)sym_smem_doubles(g) * sizeof(double);
    if (ragged)
        k_dipole_sym_fp64<true><<<blocks > 0 ? blocks : n_items, SYM_BT, smem, st>>>(s, items, n_items, counter, g);
    else
        k_dipole_sym_fp64<false><<<blocks > 0 ? blocks : n_items, SYM_BT, smem, st>>>(s, items, n_items, counter, g);
    return cudaGetLastError();
}

BlockRes block_res_of(const void* fn, int threads, int dyn_smem) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return BlockRes{};
    }
    return BlockRes{(fa.numRegs + 7) & ~7, threads, (int)fa.sharedSizeBytes + dyn_smem};
}

BlockRes dipole_block_res(bool mixed, bool sym, int g, bool beside) {
    if (!sym)
        return mixed ? block_res_of(beside ? (const void*)k_dipole_mixed_beside : (const void*)k_dipole_mixed, MIX_BT, 0)
                     : block_res_of((const void*)k_dipole_fp64, FP64_BT, 0);
    if (g == 0)
        return mixed ? block_res_of((const void*)k_dipole_symw_mixed, MSYMW_BT, 0)
                     : block_res_of((const void*)k_dipole_symw_fp64, 128, 0);
    if (g < 1 || g > 8) return BlockRes{};
    if (!mixed)
        return block_res_of((const void*)k_dipole_sym_fp64<false>, SYM_BT, (int)(sym_smem_doubles(g) * sizeof(double)));
    switch (msym_variant(g).minb) {
        case 4: return block_res_of((const void*)k_dipole_sym_mixed<4>, MSYM_BT, msym_smem_bytes(g, true, true));
        case 3: return block_res_of((const void*)k_dipole_sym_mixed<3>, MSYM_BT, msym_smem_bytes(g, true));
        case 2: return block_res_of((const void*)k_dipole_sym_mixed<2>, MSYM_BT, msym_smem_bytes(g, false));
        default: return BlockRes{};
    }
}

int dipole_symw_mixed_blocks_per_sm() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_symw_mixed, MSYMW_BT, 0);
    return b;
}

cudaError_t launch_dipole_symw_mixed(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                     cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    constexpr int warps = MSYMW_BT / 32;
    k_dipole_symw_mixed<<<blocks > 0 ? blocks : (n_items + warps - 1) / warps, MSYMW_BT, 0, st>>>(s, items, n_items,
                                                                                                  counter);
    return cudaGetLastError();
}

int dipole_symw_blocks_per_sm() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_symw_fp64, 128, 0);
    return b;
}

cudaError_t launch_dipole_symw_fp64(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                    cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    k_dipole_symw_fp64<<<blocks > 0 ? blocks : (n_items + 3) / 4, 128, 0, st>>>(s, items, n_items, counter);
    return cudaGetLastError();
}

cudaError_t launch_dipole(const Sys& s, bool mixed, const WorkItem* items, int n_items, int* counter,
                          const DipoleCfg& cfg, cudaStream_t st, bool beside) {
    if (n_items == 0) return cudaSuccess;
    const int blocks = cfg.blocks > 0 ? cfg.blocks : n_items;
    if (mixed && beside)
        k_dipole_mixed_beside<<<blocks, MIX_BT, 0, st>>>(s, items, n_items, counter);
    else if (mixed)
        k_dipole_mixed<<<blocks, MIX_BT, 0, st>>>(s, items, n_items, counter);
    else
        k_dipole_fp64<<<blocks, FP64_BT, 0, st>>>(s, items, n_items, counter);
    return cudaGetLastError();
}

}  // namespace bpm

// ===========================================================================
// bpm_dipole_forces_noalloc: the FP64 all-pairs dipole kernel for callers that
// cannot allocate device memory.  Its partial sums go to a fixed array in the
// library's device image instead of a cudaMalloc'd buffer.
// ===========================================================================
#include <mutex>
#include <string>

namespace bpm {
void set_handleless_error(const std::string& msg);

namespace {

constexpr int kNoAllocMaxN = 32768;  // largest n accepted
constexpr int kNoAllocSlots = 4;     // j-chunks per call

// Partial sums [slot][7][kNoAllocMaxN] (7.3 MB).  It belongs to the module
// image, so every GPU that loads the library holds it until the process
// exits.  In host code this name is only a stand-in for the device array: the
// kernels receive the device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_part[(size_t)kNoAllocSlots * 7 * kNoAllocMaxN];

// One block per (i-tile, j-chunk).  Every slot s < kNoAllocSlots of every
// i < n is written by exactly one block (zeros when its j-chunk is empty), so
// a call never reads what an earlier call left in the array and nothing needs
// clearing.  x and m are AoS [3n].
__global__ void __launch_bounds__(FP64_BT) k_dipole_noalloc_partial(int n, const double* __restrict__ x,
                                                                    const double* __restrict__ m,
                                                                    double* __restrict__ part) {
    __shared__ double sx[3][FP64_BT];
    __shared__ double sm[3][FP64_BT];
    const int S = gridDim.y, s = blockIdx.y;
    const int chunk = (n + S - 1) / S;
    const int j0 = min(n, s * chunk), j1 = min(n, j0 + chunk);
    const int i0 = blockIdx.x * FP64_BT;
    const int i = i0 + (int)threadIdx.x;
    const bool iv = i < n;
    d3 xi = mk3(0, 0, 0), mi = mk3(0, 0, 0);
    if (iv) {
        xi = mk3(x[3 * i], x[3 * i + 1], x[3 * i + 2]);
        mi = mk3(m[3 * i], m[3 * i + 1], m[3 * i + 2]);
    }
    Acc64 acc = {0, 0, 0, 0, 0, 0, 0};
    const int ni = min(FP64_BT, n - i0);
    for (int jt = j0; jt < j1; jt += FP64_BT) {
        const int jn = min(FP64_BT, j1 - jt);
        __syncthreads();
        if ((int)threadIdx.x < jn) {
            const int j = jt + threadIdx.x;
            for (int c = 0; c < 3; ++c) {
                sx[c][threadIdx.x] = x[3 * j + c];
                sm[c][threadIdx.x] = m[3 * j + c];
            }
        }
        __syncthreads();
        const bool diag = (i0 < jt + jn) && (i0 + ni > jt);
        if (iv) {
            if (diag)
                pairs_fp64<true>(acc, xi, mi, sx, sm, jn, (i >= jt && i < jt + jn) ? i - jt : -1);
            else
                pairs_fp64<false>(acc, xi, mi, sx, sm, jn, -1);
        }
    }
    if (iv) {
        double* P = part + (size_t)s * 7 * kNoAllocMaxN;
        P[i] = acc.fx;
        P[kNoAllocMaxN + i] = acc.fy;
        P[2 * kNoAllocMaxN + i] = acc.fz;
        P[3 * kNoAllocMaxN + i] = acc.hx;
        P[4 * kNoAllocMaxN + i] = acc.hy;
        P[5 * kNoAllocMaxN + i] = acc.hz;
        P[6 * kNoAllocMaxN + i] = acc.bs;
    }
}

// Sums the slots of particle i in a fixed order and writes f and tau (AoS).
__global__ void k_dipole_noalloc_finish(int n, int S, double c, const double* __restrict__ m,
                                        const double* __restrict__ part, double* __restrict__ f,
                                        double* __restrict__ tau) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    d3 Fd = mk3(0, 0, 0), Hd = mk3(0, 0, 0);
    double bs = 0.0;
    for (int s = 0; s < S; ++s) {
        const double* P = part + (size_t)s * 7 * kNoAllocMaxN;
        Fd = Fd + mk3(P[i], P[kNoAllocMaxN + i], P[2 * kNoAllocMaxN + i]);
        Hd = Hd + mk3(P[3 * kNoAllocMaxN + i], P[4 * kNoAllocMaxN + i], P[5 * kNoAllocMaxN + i]);
        bs += P[6 * kNoAllocMaxN + i];
    }
    const d3 mi = mk3(m[3 * i], m[3 * i + 1], m[3 * i + 2]);
    const d3 F = (Fd + mi * bs) * (3.0 * c);
    const d3 T = cross(mi, Hd * c);
    f[3 * i] = F.x;
    f[3 * i + 1] = F.y;
    f[3 * i + 2] = F.z;
    tau[3 * i] = T.x;
    tau[3 * i + 1] = T.y;
    tau[3 * i + 2] = T.z;
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

// Driver functions reached through the runtime (no link against libcuda):
// the current context's unique id, and the allocation that holds a device
// address.  Either may be missing on an old driver; the checks that use them
// are then skipped.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
typedef int (*MemGetAddressRangeFn)(unsigned long long*, size_t*, unsigned long long);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
MemGetAddressRangeFn g_mem_range = nullptr;
bool g_driver_fns_looked_up = false;

void lookup_driver_fns() {
    if (g_driver_fns_looked_up) return;
    g_driver_fns_looked_up = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_current = (CtxGetCurrentFn)fn;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_ctx_get_id = (CtxGetIdFn)fn;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_mem_range = (MemGetAddressRangeFn)fn;
    cudaGetLastError();
}

// Unique id of the current context (0 when it cannot be read).  A device
// reset or a context created anew gets a new id.
unsigned long long current_context_id() {
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_noalloc_part on the current device.  The set-up, with
// the device current, runs at the first call on each device and again
// whenever the current context is not the one the address was taken in (after
// cudaDeviceReset, for instance); otherwise the cached address is used.
cudaError_t noalloc_scratch(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    lookup_driver_fns();
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_ptr[dev] || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_part);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double*)p;
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Checks that p is device (or managed) memory that the current device dev can
// use and, where the driver tells the allocation's extent, that
// [p, p + bytes) lies inside one allocation.  Returns an empty string when
// the buffer is usable, else the reason.
std::string check_buffer(const char* name, const void* p, size_t bytes, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return std::string(name) + " is not a CUDA pointer";
    }
    if (a.type == cudaMemoryTypeDevice) {
        if (a.device != dev)
            return std::string(name) + " is memory of device " + std::to_string(a.device) +
                   ", not of the current device " + std::to_string(dev);
    } else if (a.type != cudaMemoryTypeManaged) {
        return std::string(name) + " is not device memory (host or unregistered pointer)";
    }
    if (g_mem_range) {
        unsigned long long base = 0;
        size_t size = 0;
        if (g_mem_range(&base, &size, (unsigned long long)(uintptr_t)p) == 0) {
            const unsigned long long end = (unsigned long long)(uintptr_t)p + bytes;
            if (end > base + size)
                return std::string(name) + " is shorter than 3n doubles (its allocation ends " +
                       std::to_string(base + size - (unsigned long long)(uintptr_t)p) + " bytes after it)";
        }
    }
    return std::string();
}

int noalloc_fail(int code, const std::string& msg) {
    set_handleless_error("bpm_dipole_forces_noalloc: " + msg);
    return code;
}

}  // namespace

}  // namespace bpm

extern "C" int bpm_dipole_forces_noalloc(int64_t n, const double* x, const double* m, double mu0_over_4pi,
                                         double* f, double* tau, void* stream) {
    using namespace bpm;
    if (n < 0 || n > kNoAllocMaxN)
        return noalloc_fail(BPM_ERR_ARG, "n = " + std::to_string(n) + " outside [0, " +
                                             std::to_string(kNoAllocMaxN) + "]");
    if (n == 0) return BPM_OK;
    if (!x || !m || !f || !tau) return noalloc_fail(BPM_ERR_ARG, "x, m, f and tau are required");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(BPM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(BPM_ERR_ARG, "device index out of range");
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mutex);
        lookup_driver_fns();
    }
    const size_t bytes = (size_t)n * 3 * sizeof(double);
    const char* names[4] = {"x", "m", "f", "tau"};
    const void* ptrs[4] = {x, m, f, tau};
    for (int k = 0; k < 4; ++k) {
        const std::string why = check_buffer(names[k], ptrs[k], bytes, dev);
        if (!why.empty()) return noalloc_fail(BPM_ERR_ARG, why);
    }
    double* part = nullptr;
    e = noalloc_scratch(dev, &part);
    if (e != cudaSuccess) return noalloc_fail(BPM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    const int ni = (int)n;
    const dim3 grid((unsigned)((ni + FP64_BT - 1) / FP64_BT), kNoAllocSlots);
    k_dipole_noalloc_partial<<<grid, FP64_BT, 0, st>>>(ni, x, m, part);
    k_dipole_noalloc_finish<<<(unsigned)((ni + 255) / 256), 256, 0, st>>>(ni, kNoAllocSlots, mu0_over_4pi, m, part, f, tau);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(BPM_ERR_CUDA, cudaGetErrorString(e));
    return BPM_OK;
}
