// Float-float (FP32 pair) form of the all-pairs dipole-dipole sums (Methods,
// "Magnetic interactions": U_ij = c/r^3 [m_i.m_j - 3 (m_i.r^)(m_j.r^)],
// forces and torques by differentiation), for BPM_FF handles.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so an all-pairs sum that needs
// near-FP64 accuracy is cheaper in unevaluated sums of two floats (h + l,
// |l| <= ulp(h)/2, about 48 significant bits) built from error-free
// transforms (Knuth's TwoSum, Dekker's Fast2Sum, the FMA product error) than
// in FP64 itself.  The sums are those of bpm_dipole.cu: per particle i,
//   F~ = sum (A m_j + S r),  H~ = sum (3 b r / r^5 - m_j / r^3),  Bs = sum b / r^5
// with r = x_i - x_j, a = m_i.r, b = m_j.r, d = m_i.m_j, A = a/r^5,
// S = (d - 5ab/r^2)/r^5, written to the partial slots the finish kernel
// reads.
//
// Exact differences of positions.  The encoder writes each position
// component x as three floats of fixed binades (digits of the 69-bit integer
// U = round(x / Q) + 2^68, Q = 2^q):
//   da = (2^23 + U>>46) 2^(46+q),  db = (2^23 + (U>>23 & M)) 2^(23+q),
//   dc = (2^23 + (U & M)) 2^q,  M = 2^23 - 1.
// Two floats of one binade differ exactly (Sterbenz), so r = (a_i - a_j) +
// (b_i - b_j) + (c_i - c_j) is formed without error, Fast2Sum makes it a
// float-float value, and a neighbour 1 apart at |x| = 650 keeps all its
// digits (an FP32 hi/lo split would lose 2^-48 |x|).  Q is picked per
// handle from the initial positions; a position with |x| >= 2^(66+q) gets NaN
// digits, so its forces become non-finite and the step reports it.
//
// Accuracy: every float-float operation carries a relative error of a few
// 2^-48; the accumulators are renormalised every fourth pair (the ordered
// sums every second) and flushed to FP64 after every 32 pairs.
//
// Work decomposition: that of k_dipole_sym_fp64 (each unordered pair once;
// items are pairs of supertiles of g tiles of 128; a warp holds 32 i and
// meets the 32 j of a subtile in 32 steps with the j-side sums rotating
// around the warp by shuffles; warp partials summed in a fixed order), so the
// result is bitwise reproducible.
#include <algorithm>
#include <mutex>

#include "bpm_devmath.cuh"
#include "bpm_ff.cuh"
#include "bpm_internal.h"

namespace bpm {

namespace {

constexpr int FF_BT = 128;  // threads = particles per tile

using namespace ffm;

// 1/sqrt(r2): the FP32 hardware estimate, one FP32 Newton step (error a few
// ulp), then one third-order float-float correction y (1 + e/2 + 3e^2/8)
// with e = 1 - r2 y^2 formed from exact products.
__device__ __forceinline__ ffv rsqrt_ff(ffv r2) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r2.h));
    const float hy = __fmul_rn(__fmul_rn(0.5f, r2.h), y);
    y = __fmul_rn(y, __fmaf_rn(-hy, y, 1.5f));
    const float th = __fmul_rn(y, y);
    const float tl = __fmaf_rn(y, y, -th);
    const float uh = __fmul_rn(r2.h, th);
    float ul = __fmaf_rn(r2.h, th, -uh);
    ul = __fmaf_rn(r2.h, tl, ul);
    ul = __fmaf_rn(r2.l, th, ul);
    const float e = __fsub_rn(__fsub_rn(1.0f, uh), ul);  // 1 - uh is exact
    const float corr = __fmul_rn(e, __fmaf_rn(0.375f, e, 0.5f));
    return ffv{y, __fmul_rn(y, corr)};  // the low part is about 2^-24 of y
}

// --- accumulators: hi part summed with TwoSum, errors gathered in lo
struct acc {
    float h, l;
};
__device__ __forceinline__ void acc_prod(acc& A, ffv x, ffv y) {  // A += x y
    const float p = __fmul_rn(x.h, y.h);
    const float ep = __fmaf_rn(x.h, y.h, -p);
    const ffv s = two_sum(A.h, p);
    A.h = s.h;
    float l = __fadd_rn(A.l, __fadd_rn(s.l, ep));
    l = __fmaf_rn(x.h, y.l, l);
    A.l = __fmaf_rn(x.l, y.h, l);
}
__device__ __forceinline__ void acc_add(acc& A, ffv x) {  // A += x
    const ffv s = two_sum(A.h, x.h);
    A.h = s.h;
    A.l = __fadd_rn(A.l, __fadd_rn(s.l, x.l));
}
__device__ __forceinline__ void acc_norm(acc& A) {
    const ffv s = fast_two_sum(A.h, A.l);
    A.h = s.h;
    A.l = s.l;
}
__device__ __forceinline__ double acc_d(const acc& A) { return widen(A.h) + widen(A.l); }

// --- x and y components side by side: Blackwell's packed FP32 arithmetic
// (add/mul/fma .rn.f32x2) does the same operation on both halves, so every
// half performs exactly the scalar arithmetic above in half the instructions
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

struct ff2 {
    float2 h, l;
};
__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return ff2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return ff2{s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ ff2 mul_u2(ff2 a, ff2 b) {
    const float2 p = mul2(a.h, b.h);
    float2 e = fma2(a.h, b.h, neg2(p));
    e = fma2(a.h, b.l, e);
    e = fma2(a.l, b.h, e);
    return ff2{p, e};
}
__device__ __forceinline__ ff2 sqr_u2(ff2 a) {
    const float2 p = mul2(a.h, a.h);
    float2 e = fma2(a.h, a.h, neg2(p));
    e = fma2(add2(a.h, a.h), a.l, e);
    return ff2{p, e};
}
__device__ __forceinline__ ff2 bcf(ffv a) { return ff2{bc(a.h), bc(a.l)}; }

struct acc2 {
    float2 h, l;
};
__device__ __forceinline__ void acc_prod2(acc2& A, ffv x, ff2 y) {  // A += x y (x the same in both halves)
    const float2 xh = bc(x.h);
    const float2 p = mul2(xh, y.h);
    const float2 ep = fma2(xh, y.h, neg2(p));
    const ff2 s = two_sum2(A.h, p);
    A.h = s.h;
    float2 l = add2(A.l, add2(s.l, ep));
    l = fma2(xh, y.l, l);
    A.l = fma2(bc(x.l), y.h, l);
}
__device__ __forceinline__ void acc_add2(acc2& A, ff2 x) {
    const ff2 s = two_sum2(A.h, x.h);
    A.h = s.h;
    A.l = add2(A.l, add2(s.l, x.l));
}
__device__ __forceinline__ void acc_norm2(acc2& A) {
    const ff2 s = fast_two_sum2(A.h, A.l);
    A.h = s.h;
    A.l = s.l;
}

// the accumulators of one side: F~, hb = sum b r / r^5, hm = sum m / r^3 as
// (x, y) pairs and z, and Bs
struct AccF {
    acc2 f, hb, hm;
    acc fz, hbz, hmz, bs;
};
__device__ __forceinline__ void accf_zero(AccF& a) {
    const float2 z = make_float2(0.f, 0.f);
    a.f = a.hb = a.hm = acc2{z, z};
    a.fz = a.hbz = a.hmz = a.bs = acc{0.f, 0.f};
}
__device__ __forceinline__ void accf_norm(AccF& a) {
    acc_norm2(a.f);
    acc_norm2(a.hb);
    acc_norm2(a.hm);
    acc_norm(a.fz);
    acc_norm(a.hbz);
    acc_norm(a.hmz);
    acc_norm(a.bs);
}
__device__ __forceinline__ float shfl1(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl2(float2 v, int src) { return make_float2(shfl1(v.x, src), shfl1(v.y, src)); }
__device__ __forceinline__ void accf_shfl(AccF& a, int src) {
    a.f.h = shfl2(a.f.h, src);
    a.f.l = shfl2(a.f.l, src);
    a.hb.h = shfl2(a.hb.h, src);
    a.hb.l = shfl2(a.hb.l, src);
    a.hm.h = shfl2(a.hm.h, src);
    a.hm.l = shfl2(a.hm.l, src);
    a.fz.h = shfl1(a.fz.h, src);
    a.fz.l = shfl1(a.fz.l, src);
    a.hbz.h = shfl1(a.hbz.h, src);
    a.hbz.l = shfl1(a.hbz.l, src);
    a.hmz.h = shfl1(a.hmz.h, src);
    a.hmz.l = shfl1(a.hmz.l, src);
    a.bs.h = shfl1(a.bs.h, src);
    a.bs.l = shfl1(a.bs.l, src);
}
// component c (0, 1, 2) of a packed-plus-z accumulator as a double
__device__ __forceinline__ double acc_dc(const acc2& xy, const acc& z, int c) {
    return c == 0 ? widen(xy.h.x) + widen(xy.l.x) : (c == 1 ? widen(xy.h.y) + widen(xy.l.y) : acc_d(z));
}

// a particle: position digits (a, b, c) and the moment, x and y packed
struct PF {
    float2 axy, bxy, cxy;
    float az, bz, cz;
    ff2 mxy;
    ffv mz;
};

// FP64 sums of the i side: F~ (3), H~ = 3 hb - hm (3), Bs
struct Acc7 {
    double v[7];
};
__device__ __forceinline__ void flush7(Acc7& D, const AccF& a) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        D.v[c] += acc_dc(a.f, a.fz, c);
        D.v[3 + c] += fma(3.0, acc_dc(a.hb, a.hbz, c), -acc_dc(a.hm, a.hmz, c));
    }
    D.v[6] += acc_d(a.bs);
}

// x.y for vectors given as a packed (x, y) part and z: exact hi products,
// TwoSum on the hi parts; the result is left unnormalised (it only feeds
// products and sums that take its low part as it is)
__device__ __forceinline__ ffv dot3p(ff2 xxy, ffv xz, ff2 yxy, ffv yz) {
    const ff2 p = mul_u2(xxy, yxy);
    const ffv pz = mul_u(xz, yz);
    const ffv s = two_sum(p.h.x, p.h.y);
    const ffv t = two_sum(s.h, pz.h);
    return ffv{t.h, __fadd_rn(__fadd_rn(__fadd_rn(p.l.x, p.l.y), __fadd_rn(pz.l, s.l)), t.l)};
}

// One pair: i side always; j side when SYM (the j sums with r -> -r,
// a <-> b).  A lane past the item's i range holds the stand-in of
// i_standin, whose j-side terms are exact zeros, so the j side needs no
// branch on the lane's validity (a branch would keep the compiler from
// interleaving the two sides' dependency chains).
template <bool SYM>
__device__ __forceinline__ void pair_ff(AccF& ai, AccF& aj, const PF& I, const PF& J) {
    // r, exact digit differences (same binade), joined by Fast2Sum (|db| is
    // below the unit of da)
    ff2 rxy;
    {
        const ff2 t = fast_two_sum2(sub2(I.axy, J.axy), sub2(I.bxy, J.bxy));
        rxy = ff2{t.h, add2(t.l, sub2(I.cxy, J.cxy))};
    }
    ffv rz;
    {
        const ffv t = fast_two_sum(__fsub_rn(I.az, J.az), __fsub_rn(I.bz, J.bz));
        rz = ffv{t.h, __fadd_rn(t.l, __fsub_rn(I.cz, J.cz))};
    }
    ffv r2;
    {
        const ff2 pxy = sqr_u2(rxy);
        const ffv pz = sqr_u(rz);
        const ffv s = two_sum(pxy.h.x, pxy.h.y);
        const ffv t = two_sum(s.h, pz.h);
        // a sum of squares: t.h dominates; left unnormalised
        r2 = ffv{t.h, __fadd_rn(__fadd_rn(__fadd_rn(pxy.l.x, pxy.l.y), __fadd_rn(pz.l, s.l)), t.l)};
    }
    // products that only feed further products stay unnormalised: their low
    // parts are at most about 2^-23 of the high parts
    const ffv ri = rsqrt_ff(r2);
    const ffv i2 = mul_u(ri, ri);
    const ffv i3 = mul_u(i2, ri);
    const ffv i5 = mul_u(i3, i2);
    const ffv a = dot3p(I.mxy, I.mz, rxy, rz);
    const ffv b = dot3p(J.mxy, J.mz, rxy, rz);
    const ffv d = dot3p(I.mxy, I.mz, J.mxy, J.mz);
    // sfac = d - 5 a b / r^2
    ffv sfac;
    {
        const ffv w = mul_u(mul_u(a, b), i2);
        const float p5 = __fmul_rn(-5.0f, w.h);
        const float e5 = __fmaf_rn(-5.0f, w.l, __fmaf_rn(-5.0f, w.h, -p5));
        // renormalised: d and 5ab/r^2 can nearly cancel, leaving the low
        // part as large as the high part
        const ffv s = two_sum(d.h, p5);
        sfac = two_sum(s.h, __fadd_rn(__fadd_rn(d.l, e5), s.l));
    }
    const ffv A = mul_u(i5, a);
    const ffv S = mul_u(i5, sfac);
    const ffv rb5 = mul_u(i5, b);
    // S r, shared by both sides (unnormalised product)
    const ff2 Srxy = mul_u2(bcf(S), rxy);
    const ffv Srz = mul_u(S, rz);
    acc_prod2(ai.f, A, J.mxy);
    acc_add2(ai.f, Srxy);
    acc_prod2(ai.hb, rb5, rxy);
    acc_prod2(ai.hm, i3, J.mxy);
    acc_prod(ai.fz, A, J.mz);
    acc_add(ai.fz, Srz);
    acc_prod(ai.hbz, rb5, rz);
    acc_prod(ai.hmz, i3, J.mz);
    acc_add(ai.bs, rb5);
    if (SYM) {
        acc_add2(aj.f, ff2{neg2(Srxy.h), neg2(Srxy.l)});
        acc_prod2(aj.f, neg(rb5), I.mxy);
        acc_prod2(aj.hb, A, rxy);
        acc_prod2(aj.hm, i3, I.mxy);
        acc_add(aj.fz, neg(Srz));
        acc_prod(aj.fz, neg(rb5), I.mz);
        acc_prod(aj.hbz, A, rz);
        acc_prod(aj.hmz, i3, I.mz);
        acc_add(aj.bs, neg(A));
    }
}

// j tile in shared memory, 4 float4 per particle:
//   (ax, ay, bx, by), (cx, cy, mhx, mhy), (mlx, mly, az, bz), (cz, mhz, mlz, 0)
__device__ __forceinline__ PF load_j(const float4* __restrict__ T, int jj) {
    const float4 q0 = T[4 * jj], q1 = T[4 * jj + 1], q2 = T[4 * jj + 2], q3 = T[4 * jj + 3];
    PF p;
    p.axy = make_float2(q0.x, q0.y);
    p.bxy = make_float2(q0.z, q0.w);
    p.cxy = make_float2(q1.x, q1.y);
    p.mxy = ff2{make_float2(q1.z, q1.w), make_float2(q2.x, q2.y)};
    p.az = q2.z;
    p.bz = q2.w;
    p.cz = q3.x;
    p.mz = ffv{q3.y, q3.z};
    return p;
}
__device__ __forceinline__ void store_j(float4* __restrict__ T, int jj, const PF& p) {
    T[4 * jj] = make_float4(p.axy.x, p.axy.y, p.bxy.x, p.bxy.y);
    T[4 * jj + 1] = make_float4(p.cxy.x, p.cxy.y, p.mxy.h.x, p.mxy.h.y);
    T[4 * jj + 2] = make_float4(p.mxy.l.x, p.mxy.l.y, p.az, p.bz);
    T[4 * jj + 3] = make_float4(p.cz, p.mz.h, p.mz.l, 0.f);
}

__device__ __forceinline__ PF load_global(const Sys& s, int64_t i) {
    const int64_t n = s.n;
    const float* x = s.xq;
    const float* m = s.mq;
    PF p;
    p.axy = make_float2(x[i], x[n + i]);
    p.az = x[2 * n + i];
    p.bxy = make_float2(x[3 * n + i], x[4 * n + i]);
    p.bz = x[5 * n + i];
    p.cxy = make_float2(x[6 * n + i], x[7 * n + i]);
    p.cz = x[8 * n + i];
    p.mxy = ff2{make_float2(m[i], m[n + i]), make_float2(m[3 * n + i], m[4 * n + i])};
    p.mz = ffv{m[2 * n + i], m[5 * n + i]};
    return p;
}

// The i of a lane past the item's i range: position digits (sa, sb, sc) in x
// and zero in y and z (exact differences with any digit), zero moment.  It
// coincides neither with a particle nor with the j stand-in of a ragged
// tile, which holds (sa, sb, sc) in all three components; with m_i = 0 every
// j-side term of its pairs (S r, (b/r^5) m_i, A r with A = (m_i.r)/r^5,
// m_i/r^3, A) is an exact zero.
__device__ __forceinline__ PF i_standin(float sa, float sb, float sc) {
    PF p;
    p.axy = make_float2(sa, 0.f);
    p.bxy = make_float2(sb, 0.f);
    p.cxy = make_float2(sc, 0.f);
    p.az = p.bz = p.cz = 0.f;
    p.mxy = ff2{bc(0.f), bc(0.f)};
    p.mz = ffv{0.f, 0.f};
    return p;
}

// shared memory of k_dipole_sym_ff in bytes for g tiles per supertile.
// SPLIT: the warp partials of one subtile at a time (7 KB instead of 28 KB),
// reduced into the J sums after each subtile, so that a plan whose shared
// memory limits the blocks per SM fits one more
__host__ __device__ constexpr int ff_smem_bytes(int g, bool split = false) {
    return 7 * g * FF_BT * 8                 // accJ (FP64)
           + 4 * (split ? 1 : 4) * 7 * 32 * 8  // warp partials (FP64)
           + FF_BT * 4 * 16;                 // j tile
}

// 32 rotation steps of one warp against j-subtile `base`, both sides (SYM;
// lanes without a valid i add exact zeros to the j sums and pass them on),
// or the 31 ordered steps of the warp's own subtile, i side only (s0 = 1).
// BY4: four pairs per iteration of the symmetric loop, which leaves no test
// in its body (1.3 % faster in the supertile kernel; the warp-tile kernel,
// at 128 registers, keeps two pairs per iteration, 2.8 % faster there).
template <bool SYM, bool BY4 = true>
__device__ __forceinline__ void run_subtile(AccF& ai, AccF& aj, const PF& I, const float4* __restrict__ T, int base,
                                            int lane, int from, int s0) {
    if constexpr (!SYM) {
        pair_ff<false>(ai, aj, I, load_j(T, base + ((lane + s0) & 31)));
        for (int step = s0 + 1; step < 32; step += 2) {
            pair_ff<false>(ai, aj, I, load_j(T, base + ((lane + step) & 31)));
            pair_ff<false>(ai, aj, I, load_j(T, base + ((lane + step + 1) & 31)));
            accf_norm(ai);
        }
    } else {
        // the i and j sums are renormalised in turn: each every fourth pair
      if constexpr (BY4) {
        for (int step = 0; step < 32; step += 4) {
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step) & 31)));
            accf_shfl(aj, from);
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step + 1) & 31)));
            accf_shfl(aj, from);
            accf_norm(ai);
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step + 2) & 31)));
            accf_shfl(aj, from);
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step + 3) & 31)));
            accf_shfl(aj, from);
            accf_norm(aj);
        }
      } else {
        for (int step = 0; step < 32; step += 2) {
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step) & 31)));
            accf_shfl(aj, from);
            pair_ff<true>(ai, aj, I, load_j(T, base + ((lane + step + 1) & 31)));
            accf_shfl(aj, from);
            if (step & 2)
                accf_norm(aj);
            else
                accf_norm(ai);
        }
      }
    }
}

// MINB: blocks per SM the register allocation is made for (4: 128
// registers per thread, 3: 167, 2: the full 187); the launcher takes the
// largest block count the plan's shared memory allows.
// RAGGED: the system has tiles that end early (rods of uneven length); warps
// of padding i and subtiles of padding j then skip their work.  Systems of
// whole tiles take the instantiation without those tests.
template <int MINB, bool RAGGED, bool SPLIT>
__global__ void __launch_bounds__(FF_BT, MINB) k_dipole_sym_ff(Sys s, const WorkItem* __restrict__ items, int n_items,
                                                              int* counter, int g) {
    constexpr int WK = SPLIT ? 1 : 4;  // subtile slots per warp in wpart
    extern __shared__ __align__(16) unsigned char shb[];
    const int st = g * FF_BT;
    double* accJ = reinterpret_cast<double*>(shb);                   // [7][st]
    double* wpart = accJ + 7 * st;                                   // [4 warps][WK subtiles][7][32]
    float4* T = reinterpret_cast<float4*>(wpart + 4 * WK * 7 * 32);  // [FF_BT][4]
    __shared__ int s_item;
    const int64_t n = s.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int from = (lane + 1) & 31;
    // a missing j of a ragged tile: U = 0 (x = -2^(68+q), outside the range
    // the encoder accepts) and zero moment, so it adds exactly zero to the
    // i side; its own j-side sums are never written
    const float sa = __int_as_float((196 + s.q_exp) << 23), sb = __int_as_float((173 + s.q_exp) << 23),
                sc = __int_as_float((150 + s.q_exp) << 23);
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        for (int k = tid; k < 7 * st; k += FF_BT) accJ[k] = 0.0;
        const int nIt = (wi.ni + FF_BT - 1) / FF_BT, nJt = (wi.nj + FF_BT - 1) / FF_BT;
        for (int ti = 0; ti < nIt; ++ti) {
            const int li = ti * FF_BT + tid;
            const bool iv = li < wi.ni;
            const int i = wi.i0 + (iv ? li : 0);
            const PF I = iv ? load_global(s, i) : i_standin(sa, sb, sc);
            Acc7 D = {{0, 0, 0, 0, 0, 0, 0}};
            for (int tj = diag ? ti : 0; tj < nJt; ++tj) {
                const int jt = wi.j0 + tj * FF_BT;
                const int jn = min(FF_BT, wi.nj - tj * FF_BT);
                const bool same = diag && tj == ti;
                __syncthreads();
                {
                    PF J;
                    if (tid < jn) {
                        J = load_global(s, jt + tid);
                    } else {
                        J.axy = bc(sa);
                        J.bxy = bc(sb);
                        J.cxy = bc(sc);
                        J.az = sa;
                        J.bz = sb;
                        J.cz = sc;
                        J.mxy = ff2{bc(0.f), bc(0.f)};
                        J.mz = ffv{0.f, 0.f};
                    }
                    store_j(T, tid, J);
                }
                __syncthreads();
                // a warp whose 32 i are all padding, or a j subtile beyond a
                // ragged tile's end, has no work (uniform across the warp)
                const bool wv = ti * FF_BT + warp * 32 < wi.ni;
                for (int k = 0; k < 4; ++k) {
                    AccF ai, aj;
                    accf_zero(ai);
                    accf_zero(aj);
                    const int base = k * 32;
                    if (RAGGED && (!wv || base >= jn)) {
                    } else if (!same || k > warp) {
                        run_subtile<true>(ai, aj, I, T, base, lane, from, 0);
                    } else if (k == warp) {
                        run_subtile<false>(ai, aj, I, T, base, lane, from, 1);
                    }
                    flush7(D, ai);
                    double* W = wpart + (warp * WK + (SPLIT ? 0 : k)) * 7 * 32;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        W[c * 32 + lane] = acc_dc(aj.f, aj.fz, c);
                        W[(3 + c) * 32 + lane] = fma(3.0, acc_dc(aj.hb, aj.hbz, c), -acc_dc(aj.hm, aj.hmz, c));
                    }
                    W[6 * 32 + lane] = acc_d(aj.bs);
                    if constexpr (SPLIT) {
                        // the 4 warp partials of subtile k, in the fixed order
                        __syncthreads();
                        const int jk = min(32, jn - base);
                        for (int idx = tid; idx < 7 * 32; idx += FF_BT) {
                            const int c = idx >> 5, l = idx & 31;
                            if (l >= jk) continue;
                            const double* W0 = wpart + c * 32 + l;
                            const int ws = 7 * 32;
                            accJ[c * st + tj * FF_BT + base + l] += ((W0[0] + W0[ws]) + W0[2 * ws]) + W0[3 * ws];
                        }
                        __syncthreads();
                    }
                }
                if constexpr (!SPLIT) {
                    __syncthreads();
                    // the 4 warp partials of every j of this tile, in a fixed order
                    for (int idx = tid; idx < 7 * jn; idx += FF_BT) {
                        const int c = idx / jn, jj = idx - c * jn;
                        const int k = jj >> 5, l = jj & 31;
                        const double* W0 = wpart + k * 7 * 32 + c * 32 + l;
                        const int ws = 4 * 7 * 32;
                        accJ[c * st + tj * FF_BT + jj] += ((W0[0] + W0[ws]) + W0[2 * ws]) + W0[3 * ws];
                    }
                }
            }
            __syncthreads();
            if (iv) {
                if (diag) {
                    const int l = ti * FF_BT + tid;
#pragma unroll
                    for (int c = 0; c < 7; ++c) accJ[c * st + l] += D.v[c];
                } else {
                    double* P = s.part + (int64_t)wi.slot * 7 * n;
#pragma unroll
                    for (int c = 0; c < 7; ++c) P[c * n + i] = D.v[c];
                }
            }
        }
        __syncthreads();
        double* P = s.part + (int64_t)wi.pad0 * 7 * n;
        for (int l = tid; l < wi.nj; l += FF_BT) {
            const int j = wi.j0 + l;
#pragma unroll
            for (int c = 0; c < 7; ++c) P[c * n + j] = accJ[c * st + l];
        }
    }
}

// The same sums with 32-particle tiles and one warp per pair of tiles (the
// decomposition of k_dipole_symw_fp64 in bpm_dipole.cu), for systems too
// small to fill the GPU with supertile pairs: the j tile sits in the warp's
// shared memory, the j sums rotate through the warp, a diagonal pair takes
// its 32 x 31 ordered pairs on the i side only; i-side sums go to slot
// `slot`, j-side sums to slot `pad0`.
template <int MINB>
__global__ void __launch_bounds__(FF_BT, MINB) k_dipole_symw_ff(Sys s, const WorkItem* __restrict__ items,
                                                               int n_items, int* counter) {
    __shared__ float4 Tw[4][32 * 4];
    const int64_t n = s.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int from = (lane + 1) & 31;
    float4* T = Tw[warp];
    const float sa = __int_as_float((196 + s.q_exp) << 23), sb = __int_as_float((173 + s.q_exp) << 23),
                sc = __int_as_float((150 + s.q_exp) << 23);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) return;
        const WorkItem wi = items[it];
        const bool diag = wi.pad1 != 0;
        const bool iv = lane < wi.ni;
        const int i = wi.i0 + (iv ? lane : 0);
        const PF I = iv ? load_global(s, i) : i_standin(sa, sb, sc);
        __syncwarp();
        {
            PF J;
            if (lane < wi.nj) {
                J = load_global(s, wi.j0 + lane);
            } else {
                J.axy = bc(sa);
                J.bxy = bc(sb);
                J.cxy = bc(sc);
                J.az = sa;
                J.bz = sb;
                J.cz = sc;
                J.mxy = ff2{bc(0.f), bc(0.f)};
                J.mz = ffv{0.f, 0.f};
            }
            store_j(T, lane, J);
        }
        __syncwarp();
        AccF ai, aj;
        accf_zero(ai);
        accf_zero(aj);
        if (diag)
            run_subtile<false>(ai, aj, I, T, 0, lane, from, 1);
        else
            run_subtile<true, false>(ai, aj, I, T, 0, lane, from, 0);
        if (iv) {
            Acc7 D = {{0, 0, 0, 0, 0, 0, 0}};
            flush7(D, ai);
            double* P = s.part + (int64_t)wi.slot * 7 * n;
#pragma unroll
            for (int c = 0; c < 7; ++c) P[c * n + i] = D.v[c];
        }
        if (!diag && lane < wi.nj) {
            const int j = wi.j0 + lane;
            double* P = s.part + (int64_t)wi.pad0 * 7 * n;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                P[c * n + j] = acc_dc(aj.f, aj.fz, c);
                P[(3 + c) * n + j] = fma(3.0, acc_dc(aj.hb, aj.hbz, c), -acc_dc(aj.hm, aj.hmz, c));
            }
            P[6 * n + j] = acc_d(aj.bs);
        }
    }
}

// Position digits and moment pairs of every particle (see the file comment).
__global__ void __launch_bounds__(256) k_ff_encode(Sys s) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double lim = ldexp(1.0, 66 + s.q_exp);
    const double inv_q = ldexp(1.0, -s.q_exp);
    const int ea = 196 + s.q_exp, eb = 173 + s.q_exp, ec = 150 + s.q_exp;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double x = s.x[c * n + i];
        float fa, fb, fc;
        if (fabs(x) < lim) {  // false for NaN
            // Y = round(x / Q), |Y| < 2^66: x / Q is exact (power-of-two
            // scale), rint is exact, and Y = Yh 2^23 + Yl splits exactly
            const double Y = rint(x * inv_q);
            const double Yh = floor(Y * 0x1p-23);
            const double Yl = fma(Yh, -0x1p23, Y);                  // in [0, 2^23)
            const long long Uh = __double2ll_rn(Yh) + (1ll << 45);  // U >> 23, U = Y + 2^68
            const unsigned A = (unsigned)(Uh >> 23), B = (unsigned)(Uh & 0x7fffff),
                           C = (unsigned)__double2int_rn(Yl);
            fa = __int_as_float((ea << 23) | (int)A);
            fb = __int_as_float((eb << 23) | (int)B);
            fc = __int_as_float((ec << 23) | (int)C);
        } else {
            // NaN digits: the forces of this particle become non-finite
            fa = fb = fc = __int_as_float(0x7fc00000);
        }
        s.xq[c * n + i] = fa;
        s.xq[(3 + c) * n + i] = fb;
        s.xq[(6 + c) * n + i] = fc;
        const double m = s.m[c * n + i];
        const float mh = __double2float_rn(m);
        s.mq[c * n + i] = mh;
        s.mq[(3 + c) * n + i] = __double2float_rn(m - (double)mh);
    }
}

// ============================================================================
// Dipole VJP of the adjoint (BPM_FF handles) in float-float.  For the pair
// (i, j), with lam the adjoint of the force, mu = lam_tau x m that of the
// field, k = 3c, and the coefficients of the two sides (the side of j has
// r -> -r, a' = -b, b' = -a; primes mark its lam, mu):
//   C1 = Lm2/r^5 - 5 b Lr/r^7,  C2 = (Lm1 + Mr)/r^5 - 5 a Lr/r^7,
//   Clam = d/r^5 - 5ab/r^7 (the same on both sides),
//   Cr = Mm2/r^5 - 5 (P + b Mr)/r^7 + 35 ab Lr/r^9,  P = a Lm2 + b Lm1 + d Lr
// (Lv = lam.v, Mv = mu.v with m1 the own and m2 the partner moment), the
// gradients of lam.F + mu.H of both sides combine into
//   d/dx_i = -d/dx_j = K1 m_i + K2 m_j + KL dlam + KMi mu_i + KMj mu_j + KR r
//   d/dm_i += K1 r + KMi dlam + KLr m_j - (c/r^3) mu_j
//   d/dm_j += K2 r + KMj dlam + KLr m_i - (c/r^3) mu_i
//   H_i = KMi r - (c/r^3) m_j,  H_j = KMj r - (c/r^3) m_i
// with dlam = lam_i - lam_j, K1 = k (C1 - C2'), K2 = k (C2 - C1'),
// KL = k Clam, KMi = k b/r^5, KMj = k a/r^5, KR = k (Cr + Cr'),
// KLr = k (Lr + Lr')/r^5.  These are the two dip_grad evaluations of the
// FP64 VJP (bpm_adjoint.cu) regrouped by vector.  The decomposition is that
// of k_adj_dipole_sym: one warp per pair of 32-particle tiles, j sums
// rotating around the warp, one partial per partner tile.

// per-particle inputs, SoA [29][N] floats: position digits a, b, c (9), m, lam,
// mu hi (3 each) and lo (3 each) (18), lam.m hi and lo (2)
constexpr int FFA_COMP = 29;

// a vector as a packed (x, y) float-float pair and z
struct fv3 {
    ff2 xy;
    ffv z;
};
struct acc3 {
    acc2 xy;
    acc z;
};
__device__ __forceinline__ ffv dotv(const fv3& a, const fv3& b) { return dot3p(a.xy, a.z, b.xy, b.z); }
__device__ __forceinline__ void acc3_prod(acc3& A, ffv s, const fv3& v) {
    acc_prod2(A.xy, s, v.xy);
    acc_prod(A.z, s, v.z);
}
__device__ __forceinline__ void acc3_add(acc3& A, const acc3& t, bool negate) {
    const float sg = negate ? -1.f : 1.f;
    acc_add2(A.xy, ff2{mul2(bc(sg), t.xy.h), mul2(bc(sg), t.xy.l)});
    acc_add(A.z, ffv{sg * t.z.h, sg * t.z.l});
}
__device__ __forceinline__ void acc3_zero(acc3& A) {
    A.xy = acc2{bc(0.f), bc(0.f)};
    A.z = acc{0.f, 0.f};
}
__device__ __forceinline__ void acc3_norm(acc3& A) {
    acc_norm2(A.xy);
    acc_norm(A.z);
}
__device__ __forceinline__ void acc3_shfl(acc3& A, int src) {
    A.xy.h = shfl2(A.xy.h, src);
    A.xy.l = shfl2(A.xy.l, src);
    A.z.h = shfl1(A.z.h, src);
    A.z.l = shfl1(A.z.l, src);
}
__device__ __forceinline__ d3 acc3_d(const acc3& A) {
    return mk3(widen(A.xy.h.x) + widen(A.xy.l.x), widen(A.xy.h.y) + widen(A.xy.l.y), acc_d(A.z));
}

struct AdjF {
    acc3 gx, gm, H;
};
__device__ __forceinline__ void adjf_zero(AdjF& a) {
    acc3_zero(a.gx);
    acc3_zero(a.gm);
    acc3_zero(a.H);
}
__device__ __forceinline__ void adjf_norm(AdjF& a) {
    acc3_norm(a.gx);
    acc3_norm(a.gm);
    acc3_norm(a.H);
}
__device__ __forceinline__ void adjf_shfl(AdjF& a, int src) {
    acc3_shfl(a.gx, src);
    acc3_shfl(a.gm, src);
    acc3_shfl(a.H, src);
}

struct PAdj {
    float2 axy, bxy, cxy;
    float az, bz, cz;
    fv3 m, lam, mu;
    ffv lm;  // lam . m
};

__device__ __forceinline__ fv3 ld_fv3(const float* p, int64_t n, int64_t i, int c0) {
    return fv3{ff2{make_float2(p[c0 * n + i], p[(c0 + 1) * n + i]), make_float2(p[(c0 + 3) * n + i], p[(c0 + 4) * n + i])},
               ffv{p[(c0 + 2) * n + i], p[(c0 + 5) * n + i]}};
}
__device__ __forceinline__ PAdj load_adj(const float* p, int64_t n, int64_t i) {
    PAdj q;
    q.axy = make_float2(p[i], p[n + i]);
    q.az = p[2 * n + i];
    q.bxy = make_float2(p[3 * n + i], p[4 * n + i]);
    q.bz = p[5 * n + i];
    q.cxy = make_float2(p[6 * n + i], p[7 * n + i]);
    q.cz = p[8 * n + i];
    q.m = ld_fv3(p, n, i, 9);
    q.lam = ld_fv3(p, n, i, 15);
    q.mu = ld_fv3(p, n, i, 21);
    q.lm = ffv{p[27 * n + i], p[28 * n + i]};
    return q;
}

// both sides of the pair (i, j); SYM: the j sums as well (lanes without a
// valid i add nothing but still pass them on)
template <bool SYM>
__device__ __forceinline__ void adj_pair_ff(AdjF& ai, AdjF& aj, const PAdj& I, const PAdj& J, ffv kk, ffv cc,
                                            bool jside) {
    fv3 r;
    {
        const ff2 t = fast_two_sum2(sub2(I.axy, J.axy), sub2(I.bxy, J.bxy));
        r.xy = ff2{t.h, add2(t.l, sub2(I.cxy, J.cxy))};
        const ffv u = fast_two_sum(__fsub_rn(I.az, J.az), __fsub_rn(I.bz, J.bz));
        r.z = ffv{u.h, __fadd_rn(u.l, __fsub_rn(I.cz, J.cz))};
    }
    ffv r2;
    {
        const ff2 pxy = sqr_u2(r.xy);
        const ffv pz = sqr_u(r.z);
        const ffv s = two_sum(pxy.h.x, pxy.h.y);
        const ffv t = two_sum(s.h, pz.h);
        r2 = ffv{t.h, __fadd_rn(__fadd_rn(__fadd_rn(pxy.l.x, pxy.l.y), __fadd_rn(pz.l, s.l)), t.l)};
    }
    const ffv ri = rsqrt_ff(r2);
    const ffv ri2 = mul_u(ri, ri), ri3 = mul_u(ri2, ri), ri5 = mul_u(ri3, ri2), ri7 = mul_u(ri5, ri2),
              ri9 = mul_u(ri7, ri2);
    const ffv a = dotv(I.m, r), b = dotv(J.m, r), d = dotv(I.m, J.m);
    const ffv ab = mul_u(a, b), t5 = mulc(ri7, 5.0f), abr9 = mulc(mul_u(ab, ri9), 35.0f);
    // side i (m1 = m_i, m2 = m_j)
    const ffv Lm2 = dotv(I.lam, J.m), Lr = dotv(I.lam, r), Mr = dotv(I.mu, r), Mm2 = dotv(I.mu, J.m);
    // side j (m1 = m_j, m2 = m_i, r -> -r): Lr', Mr' carry the sign flip
    const ffv Lm2p = dotv(J.lam, I.m), Lrp = neg(dotv(J.lam, r)), Mrp = neg(dotv(J.mu, r)), Mm2p = dotv(J.mu, I.m);
    const ffv aLrt5 = mul_u(mul_u(a, Lr), t5), bLrt5 = mul_u(mul_u(b, Lr), t5);
    const ffv aLrpt5 = mul_u(mul_u(a, Lrp), t5), bLrpt5 = mul_u(mul_u(b, Lrp), t5);
    // C1 - C2' and C2 - C1' (the 5 a Lr'/r^7 and 5 b Lr'/r^7 terms of the side
    // of j enter with a' = -b, b' = -a)
    const ffv C1 = add_ff(mul_u(Lm2, ri5), neg(bLrt5));
    const ffv C2 = add_ff(mul_u(add_ff(I.lm, Mr), ri5), neg(aLrt5));
    const ffv C1p = add_ff(mul_u(Lm2p, ri5), aLrpt5);
    const ffv C2p = add_ff(mul_u(add_ff(J.lm, Mrp), ri5), bLrpt5);
    const ffv Clam = add_ff(mul_u(d, ri5), neg(mul_u(ab, t5)));
    // Cr and Cr'
    const ffv Pl = add_ff(add_ff(mul_u(a, Lm2), mul_u(b, I.lm)), mul_u(d, Lr));
    const ffv Plp = add_ff(add_ff(neg(mul_u(b, Lm2p)), neg(mul_u(a, J.lm))), mul_u(d, Lrp));
    const ffv Cr = add_ff(add_ff(mul_u(Mm2, ri5), neg(mul_u(add_ff(Pl, mul_u(b, Mr)), t5))), mul_u(abr9, Lr));
    const ffv Crp = add_ff(add_ff(mul_u(Mm2p, ri5), neg(mul_u(add_ff(Plp, neg(mul_u(a, Mrp))), t5))),
                           mul_u(abr9, Lrp));
    // the k-scaled coefficients, renormalised (differences can cancel)
    const ffv K1 = mul_u(kk, norm_ff(add_ff(C1, neg(C2p))));
    const ffv K2 = mul_u(kk, norm_ff(add_ff(C2, neg(C1p))));
    const ffv KL = mul_u(kk, norm_ff(Clam));
    const ffv KMi = mul_u(kk, mul_u(b, ri5));
    const ffv KMj = mul_u(kk, mul_u(a, ri5));
    const ffv KR = mul_u(kk, norm_ff(add_ff(Cr, Crp)));
    const ffv KLr = mul_u(kk, norm_ff(mul_u(add_ff(Lr, Lrp), ri5)));
    const ffv cr3 = mul_u(cc, ri3);
    const ffv ncr3 = neg(cr3);
    // dlam = lam_i - lam_j
    fv3 dl;
    {
        const ff2 s = two_sum2(I.lam.xy.h, neg2(J.lam.xy.h));
        dl.xy = ff2{s.h, add2(add2(I.lam.xy.l, neg2(J.lam.xy.l)), s.l)};
        dl.z = add_ff(I.lam.z, neg(J.lam.z));
    }
    // d/dx: one sum, added to i and subtracted from j
    acc3 gd;
    acc3_zero(gd);
    acc3_prod(gd, K1, I.m);
    acc3_prod(gd, K2, J.m);
    acc3_prod(gd, KL, dl);
    acc3_prod(gd, KMi, I.mu);
    acc3_prod(gd, KMj, J.mu);
    acc3_prod(gd, KR, r);
    acc3_add(ai.gx, gd, false);
    acc3_prod(ai.gm, K1, r);
    acc3_prod(ai.gm, KMi, dl);
    acc3_prod(ai.gm, KLr, J.m);
    acc3_prod(ai.gm, ncr3, J.mu);
    acc3_prod(ai.H, KMi, r);
    acc3_prod(ai.H, ncr3, J.m);
    if (SYM && jside) {
        acc3_add(aj.gx, gd, true);
        acc3_prod(aj.gm, K2, r);
        acc3_prod(aj.gm, KMj, dl);
        acc3_prod(aj.gm, KLr, I.m);
        acc3_prod(aj.gm, ncr3, I.mu);
        acc3_prod(aj.H, KMj, r);
        acc3_prod(aj.H, ncr3, I.m);
    }
}

template <bool DIAG>
__device__ __forceinline__ void adj_tile_ff(AdjF& ai, AdjF& aj, const PAdj& I, const float (*sj)[32], int lane,
                                            bool iv, ffv kk, ffv cc) {
    const int from = (lane + 1) & 31;
    for (int step = DIAG ? 1 : 0; step < 32; ++step) {
        const int o = (lane + step) & 31;
        PAdj J;
        J.axy = make_float2(sj[0][o], sj[1][o]);
        J.az = sj[2][o];
        J.bxy = make_float2(sj[3][o], sj[4][o]);
        J.bz = sj[5][o];
        J.cxy = make_float2(sj[6][o], sj[7][o]);
        J.cz = sj[8][o];
        J.m = fv3{ff2{make_float2(sj[9][o], sj[10][o]), make_float2(sj[12][o], sj[13][o])}, ffv{sj[11][o], sj[14][o]}};
        J.lam = fv3{ff2{make_float2(sj[15][o], sj[16][o]), make_float2(sj[18][o], sj[19][o])}, ffv{sj[17][o], sj[20][o]}};
        J.mu = fv3{ff2{make_float2(sj[21][o], sj[22][o]), make_float2(sj[24][o], sj[25][o])}, ffv{sj[23][o], sj[26][o]}};
        J.lm = ffv{sj[27][o], sj[28][o]};
        if (DIAG) {
            adj_pair_ff<false>(ai, aj, I, J, kk, cc, false);
        } else {
            adj_pair_ff<true>(ai, aj, I, J, kk, cc, iv);
            adjf_shfl(aj, from);
        }
        if ((step & 3) == 3) {
            adjf_norm(ai);
            if (!DIAG) adjf_norm(aj);
        }
    }
}

__global__ void __launch_bounds__(128) k_adj_dipole_sym_ff(Sys s, AdjBuf a, int64_t n_items) {
    __shared__ float sjw[4][FFA_COMP][32];
    const int64_t n = s.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float(*sj)[32] = sjw[warp];
    const float* F = a.ffbuf;
    // k = 3c and c as float-float
    const float kh = __double2float_rn(3.0 * s.c), ch = __double2float_rn(s.c);
    const ffv kk{kh, __double2float_rn(3.0 * s.c - (double)kh)}, cc{ch, __double2float_rn(s.c - (double)ch)};
    // a missing j of a ragged last tile: outside the encoder's range, with
    // zero moment and adjoints, so every term it contributes is zero
    const float sa = __int_as_float((196 + s.q_exp) << 23), sb = __int_as_float((173 + s.q_exp) << 23),
                sc = __int_as_float((150 + s.q_exp) << 23);
    const int64_t n_warps = (int64_t)gridDim.x * 4;
    for (int64_t t = (int64_t)blockIdx.x * 4 + warp; t < n_items; t += n_warps) {
        // t = J (J + 1) / 2 + I with 0 <= I <= J
        int64_t J = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
        while (J * (J + 1) / 2 > t) --J;
        while ((J + 1) * (J + 2) / 2 <= t) ++J;
        const int64_t I = t - J * (J + 1) / 2;
        const int64_t i = 32 * I + lane, j = 32 * J + lane;
        const bool iv = i < n, jv = j < n;
        const PAdj Pi = load_adj(F, n, iv ? i : 0);
        __syncwarp();
        for (int k = 0; k < FFA_COMP; ++k) {
            float v;
            if (jv)
                v = F[k * n + j];
            else
                v = k < 3 ? sa : (k < 6 ? sb : (k < 9 ? sc : 0.f));
            sj[k][lane] = v;
        }
        __syncwarp();
        AdjF ai, aj;
        adjf_zero(ai);
        adjf_zero(aj);
        if (I == J)
            adj_tile_ff<true>(ai, aj, Pi, sj, lane, iv, kk, cc);
        else
            adj_tile_ff<false>(ai, aj, Pi, sj, lane, iv, kk, cc);
        // torque tau = m x H: d/dm += H x lambda_tau
        if (iv) {
            double* D = a.dpart + J * 6 * n;
            const d3 gx = acc3_d(ai.gx), gm = acc3_d(ai.gm), H = acc3_d(ai.H);
            const d3 lt = mk3(a.aT[i], a.aT[n + i], a.aT[2 * n + i]);
            const d3 g2 = gm + cross(H, lt);
            D[i] = gx.x;
            D[n + i] = gx.y;
            D[2 * n + i] = gx.z;
            D[3 * n + i] = g2.x;
            D[4 * n + i] = g2.y;
            D[5 * n + i] = g2.z;
        }
        if (I != J && jv) {
            double* D = a.dpart + I * 6 * n;
            const d3 gx = acc3_d(aj.gx), gm = acc3_d(aj.gm), H = acc3_d(aj.H);
            const d3 lt = mk3(a.aT[j], a.aT[n + j], a.aT[2 * n + j]);
            const d3 g2 = gm + cross(H, lt);
            D[j] = gx.x;
            D[n + j] = gx.y;
            D[2 * n + j] = gx.z;
            D[3 * n + j] = g2.x;
            D[4 * n + j] = g2.y;
            D[5 * n + j] = g2.z;
        }
    }
}

// the float-float inputs of the VJP at a snapshot: position digits (as
// k_ff_encode), m, lam = the force adjoint, mu and lam . m as hi/lo pairs
__global__ void __launch_bounds__(256) k_adj_ff_encode(Sys s, AdjBuf a) {
    const int64_t n = s.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* F = a.ffbuf;
    const double lim = ldexp(1.0, 66 + s.q_exp), inv_q = ldexp(1.0, -s.q_exp);
    const int ea = 196 + s.q_exp, eb = 173 + s.q_exp, ec = 150 + s.q_exp;
    double lm = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double x = s.x[c * n + i];
        float fa, fb, fc;
        if (fabs(x) < lim) {
            const double Y = rint(x * inv_q);
            const double Yh = floor(Y * 0x1p-23);
            const double Yl = fma(Yh, -0x1p23, Y);
            const long long Uh = __double2ll_rn(Yh) + (1ll << 45);
            fa = __int_as_float((ea << 23) | (int)(unsigned)(Uh >> 23));
            fb = __int_as_float((eb << 23) | (int)(unsigned)(Uh & 0x7fffff));
            fc = __int_as_float((ec << 23) | (int)(unsigned)__double2int_rn(Yl));
        } else {
            fa = fb = fc = __int_as_float(0x7fc00000);
        }
        F[c * n + i] = fa;
        F[(3 + c) * n + i] = fb;
        F[(6 + c) * n + i] = fc;
        const double v3[3] = {a.m[c * n + i], a.aF[c * n + i], a.mu[c * n + i]};
        for (int k = 0; k < 3; ++k) {
            const float h = __double2float_rn(v3[k]);
            F[(9 + 6 * k + c) * n + i] = h;
            F[(12 + 6 * k + c) * n + i] = __double2float_rn(v3[k] - (double)h);
        }
        lm = fma(v3[1], v3[0], lm);
    }
    const float h = __double2float_rn(lm);
    F[27 * n + i] = h;
    F[28 * n + i] = __double2float_rn(lm - (double)h);
}

}  // namespace

int dipole_ff_tile() { return FF_BT; }

namespace {
template <int MINB, bool SPLIT>
int ff_occupancy(int smem) {
    for (auto k : {k_dipole_sym_ff<MINB, false, SPLIT>, k_dipole_sym_ff<MINB, true, SPLIT>})
        if (!allow_dynamic_smem((const void*)k, (size_t)smem)) return 0;  // the variant is not runnable
    int b = 0, br = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_sym_ff<MINB, false, SPLIT>, FF_BT, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&br, k_dipole_sym_ff<MINB, true, SPLIT>, FF_BT, smem);
    return b < br ? b : br;
}

// the variant of each g: the most blocks per SM; among equals the most
// registers per thread, and the full partials (one reduction per tile) before
// the split ones; b = its blocks per SM
struct FFVariant {
    int minb, b;
    bool split;
};
FFVariant ff_variant(int g) {
    static FFVariant cache[9] = {};
    static std::once_flag once[9];
    std::call_once(once[g], [g] {
        const int smem = ff_smem_bytes(g), smem_s = ff_smem_bytes(g, true);
        FFVariant best{0, 0, false};
        const int b2 = ff_occupancy<2, false>(smem), b3 = ff_occupancy<3, false>(smem),
                  b4 = ff_occupancy<4, false>(smem), b4s = ff_occupancy<4, true>(smem_s);
        if (b2 > best.b) best = FFVariant{2, b2, false};
        if (b3 > best.b) best = FFVariant{3, b3, false};
        if (b4 > best.b) best = FFVariant{4, b4, false};
        if (b4s > best.b) best = FFVariant{4, b4s, true};
        cache[g] = best;
    });
    return cache[g];
}
}  // namespace

int dipole_ff_blocks_per_sm(int g) {
    if (g < 1 || g > 8) return 0;
    return ff_variant(g).b;
}

template <bool RAGGED>
void launch_sym_ff_variant(const FFVariant& v, int grid, int g, cudaStream_t st, const Sys& s,
                           const WorkItem* items, int n_items, int* counter) {
    const int smem = ff_smem_bytes(g, v.split);
    if (v.split) {
        k_dipole_sym_ff<4, RAGGED, true><<<grid, FF_BT, smem, st>>>(s, items, n_items, counter, g);
        return;
    }
    switch (v.minb) {
        case 4: k_dipole_sym_ff<4, RAGGED, false><<<grid, FF_BT, smem, st>>>(s, items, n_items, counter, g); break;
        case 3: k_dipole_sym_ff<3, RAGGED, false><<<grid, FF_BT, smem, st>>>(s, items, n_items, counter, g); break;
        default: k_dipole_sym_ff<2, RAGGED, false><<<grid, FF_BT, smem, st>>>(s, items, n_items, counter, g); break;
    }
}

cudaError_t launch_dipole_sym_ff(const Sys& s, const WorkItem* items, int n_items, int* counter, int g, int blocks,
                                 bool ragged, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (g < 1 || g > 8) return cudaErrorInvalidValue;
    const int grid = blocks > 0 ? blocks : n_items;
    const FFVariant v = ff_variant(g);
    if (v.minb < 2 || v.minb > 4) return cudaErrorInvalidConfiguration;  // no variant fits this g
    if (ragged)
        launch_sym_ff_variant<true>(v, grid, g, st, s, items, n_items, counter);
    else
        launch_sym_ff_variant<false>(v, grid, g, st, s, items, n_items, counter);
    return cudaGetLastError();
}

BlockRes dipole_ff_block_res(int g) {
    if (g == 0) return block_res_of((const void*)k_dipole_symw_ff<4>, FF_BT, 0);
    if (g < 1 || g > 8) return BlockRes{};
    const FFVariant v = ff_variant(g);
    const int smem = ff_smem_bytes(g, v.split);
    // the ragged form: registers at least those of the dense one
    if (v.split) return block_res_of((const void*)k_dipole_sym_ff<4, true, true>, FF_BT, smem);
    switch (v.minb) {
        case 4: return block_res_of((const void*)k_dipole_sym_ff<4, true, false>, FF_BT, smem);
        case 3: return block_res_of((const void*)k_dipole_sym_ff<3, true, false>, FF_BT, smem);
        case 2: return block_res_of((const void*)k_dipole_sym_ff<2, true, false>, FF_BT, smem);
        default: return BlockRes{};
    }
}

int dipole_symw_ff_blocks_per_sm() {
    // 128 registers: 4 blocks of 4 warps per SM
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dipole_symw_ff<4>, FF_BT, 0);
    return b;
}

cudaError_t launch_dipole_symw_ff(const Sys& s, const WorkItem* items, int n_items, int* counter, int blocks,
                                  cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    k_dipole_symw_ff<4><<<blocks > 0 ? blocks : (n_items + 3) / 4, FF_BT, 0, st>>>(s, items, n_items, counter);
    return cudaGetLastError();
}

int adj_ff_comp() { return FFA_COMP; }

cudaError_t launch_adj_dipole_sym_ff(const Sys& s, const AdjBuf& a, int64_t n_items, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    k_adj_ff_encode<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, a);
    // a static round-robin of the tile pairs over the warps, with the
    // resident block count per SM that best evens out the items per warp
    static int n_sm = 0, per_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adj_dipole_sym_ff, 128, 0);
        per_sm = per_sm > 0 ? per_sm : 1;
    }
    int64_t best = 1;
    double best_eff = -1.0;
    for (int b = 1; b <= per_sm; ++b) {
        const int64_t blocks = std::min<int64_t>((int64_t)n_sm * b, (n_items + 3) / 4);
        const int64_t rounds = (n_items + 4 * blocks - 1) / (4 * blocks);
        const double eff = (double)n_items / (double)(4 * blocks * rounds);
        if (eff >= best_eff - 1e-9) {
            best_eff = eff;
            best = blocks;
        }
    }
    k_adj_dipole_sym_ff<<<(unsigned)best, 128, 0, st>>>(s, a, n_items);
    return cudaGetLastError();
}

cudaError_t launch_ff_encode(const Sys& s, cudaStream_t st) {
    if (s.n == 0) return cudaSuccess;
    k_ff_encode<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace bpm
