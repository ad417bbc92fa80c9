// FP64 vector / quaternion helpers for the device code.  Quaternions are
// (w, x, y, z) with the Hamilton product; rot(q, v) = q v q*.
#pragma once

#include <cuda_runtime.h>

namespace bpm {

struct d3 {
    double x, y, z;
};
struct dq {
    double w, x, y, z;
};

__device__ __forceinline__ d3 mk3(double x, double y, double z) { return d3{x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator-(d3 a) { return d3{-a.x, -a.y, -a.z}; }
__device__ __forceinline__ d3 operator*(d3 a, double s) { return d3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// |a|^2 summed left to right without fused multiply-adds (matches a plain
// C evaluation bit for bit; used where a difference of lengths cancels).
__device__ __forceinline__ double norm2_rn(d3 a) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)), __dmul_rn(a.z, a.z));
}

__device__ __forceinline__ dq qmul(dq a, dq b) {
    return dq{a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
              a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
              a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
              a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
__device__ __forceinline__ dq qconj(dq a) { return dq{a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ dq qscale(dq a, double s) { return dq{a.w * s, a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ double qdot(dq a, dq b) { return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ dq qnormalise(dq a) { return qscale(a, 1.0 / sqrt(qdot(a, a))); }

// q v q* for unit q: v + w t + u x t with t = 2 u x v
__device__ __forceinline__ d3 rot(dq q, d3 v) {
    d3 u = mk3(q.x, q.y, q.z);
    d3 t = cross(u, v) * 2.0;
    return v + t * q.w + cross(u, t);
}
// q* v q
__device__ __forceinline__ d3 rot_inv(dq q, d3 v) { return rot(qconj(q), v); }

// 1/sqrt(a).  For 2^-125 <= a < 2^126: the FP32 hardware estimate y of a
// float made from a's high word by integer operations (exponent rebias and
// shift: the leading 20 mantissa bits), widened the same way, so no FP64
// conversion instruction is issued (relative seed error below 2^-20).  Then
// one third-order step with e = 1 - a y^2:
//   1/sqrt(a) = y (1 + e/2 + 3 e^2/8) + O(e^3) = (y + c) + (y/2) e,
// where c = 3 y e^2 / 8 is below 2^-38 y and needs only a few correct bits:
// it is formed in FP32 from e's leading bits and widened by integer
// operations, and y/2 is y with its exponent lowered.  The error, about
// (5/16) e^3 < 2^-61 plus the roundings of a y, e and the two last FP64
// operations, is within an ulp or so: 4 FP64 instructions instead of the 8
// of two Newton steps.  Other inputs (zero, tiny, huge, negative,
// non-finite) take the IEEE 1/sqrt.
__device__ __forceinline__ double rsqrt_nr(double a) {
    const int hi = __double2hiint(a);
    if (hi < 0x38200000 || hi >= 0x47D00000) return 1.0 / sqrt(a);
    const float af = __uint_as_float(((unsigned)hi - 0x38000000u) << 3);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(af));
    const int yb = __float_as_int(yf);
    const int yhi = (yb >> 3) + 0x38000000, ylo = (int)((unsigned)yb << 29);
    const double y = __hiloint2double(yhi, ylo);
    const double yh = __hiloint2double(yhi - 0x00100000, ylo);  // y / 2
    const double e = fma(-a * y, y, 1.0);
    // |e| as a float (leading bits; 0 when |e| < 2^-126: c is then far
    // below an ulp of y)
    const unsigned eb = (unsigned)__double2hiint(e) & 0x7fffffffu;
    const float ef = eb < 0x38100000u ? 0.0f : __uint_as_float((eb - 0x38000000u) << 3);
    const float cf = (0.375f * yf) * (ef * ef);
    const int cb = __float_as_int(cf);
    const double c = (cb & 0x7f800000) == 0 ? 0.0 : __hiloint2double((cb >> 3) + 0x38000000, (int)((unsigned)cb << 29));
    return fma(yh, e, y + c);
}

// 1/a for a > 0.  For 2^-125 <= a < 2^126: the FP32 hardware estimate y of
// a float made from a's high word by integer operations (the leading 20
// mantissa bits), widened the same way (relative error below 2^-19), then
// 1/a = y / (1 - e) = y (1 + e + e^2) + O(e^3) with e = 1 - a y: 3 FP64
// instructions and no conversion instruction, the truncation error about
// e^3 < 2^-57.  Other inputs take the IEEE division.
__device__ __forceinline__ double rcp_nr(double a) {
    const int hi = __double2hiint(a);
    if (hi < 0x38200000 || hi >= 0x47D00000) return 1.0 / a;
    const float af = __uint_as_float(((unsigned)hi - 0x38000000u) << 3);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(af));
    const int yb = __float_as_int(yf);
    const double y = __hiloint2double((yb >> 3) + 0x38000000, (int)((unsigned)yb << 29));
    const double e = fma(-a, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// q / |q| with the reciprocal square root above
__device__ __forceinline__ dq qnormalise_nr(dq a) { return qscale(a, rsqrt_nr(qdot(a, a))); }

// atan2(sqrt(t), c) / sqrt(t) for t >= 0: for t < 1e-2 c^2 and c > 0 the
// Taylor series of atan(u)/u = sum_k (-u^2)^k / (2k + 1), u^2 = t/c^2,
// truncated after 8 terms (remainder below 6e-18 relative), or after 4 terms
// when u^2 < 1e-4 (remainder u^8/9 below 1.2e-17 relative), the usual case
// of the bond angles; otherwise the library atan2.  The limit 1/c is
// returned at t = 0.  Used for the small angles of the bond model, where it
// replaces a sqrt, an atan2 and a division (1/c from rcp_nr).
__device__ __forceinline__ double atan_over(double t, double c) {
    if (c > 0.0 && t < 1e-2 * c * c) {
        const double ic = rcp_nr(c);
        const double z = t * ic * ic;
        double p;
        if (z < 1e-4) {
            p = 1.0 / 7.0;
        } else {
            p = 1.0 / 15.0;
            p = fma(p, -z, 1.0 / 13.0);
            p = fma(p, -z, 1.0 / 11.0);
            p = fma(p, -z, 1.0 / 9.0);
            p = fma(p, -z, 1.0 / 7.0);
        }
        p = fma(p, -z, 1.0 / 5.0);
        p = fma(p, -z, 1.0 / 3.0);
        p = fma(p, -z, 1.0);
        return p * ic;
    }
    const double s = sqrt(t);
    return s > 0.0 ? atan2(s, c) / s : 1.0 / c;
}

}  // namespace bpm
