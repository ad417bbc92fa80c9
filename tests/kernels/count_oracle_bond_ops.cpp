// Counts the FP64 operations of the oracle's single-bond evaluation (the
// force and torque of one bond, no energy) by compiling the oracle's C source
// with a number type that counts every +, -, x and / (and, apart, the square
// roots and atan2).  Test code only: it pins the per-bond operation count
// that bench.py uses as the bond kernel's unit of work.  Prints
// "<operations> <square roots> <atan2>".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
struct OpCount { static inline long ops = 0, sqrts = 0, atan2s = 0; };
struct cd {
    double v;
    cd() : v(0) {}
    cd(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator long() const { return (long)v; }
    explicit operator int() const { return (int)v; }
    explicit operator bool() const { return v != 0.0; }
};
#define CD_BIN(op) \
    inline cd operator op(cd a, cd b) { OpCount::ops++; return cd(a.v op b.v); } \
    inline cd operator op(cd a, double b) { OpCount::ops++; return cd(a.v op b); } \
    inline cd operator op(double a, cd b) { OpCount::ops++; return cd(a op b.v); } \
    inline cd operator op(cd a, int b) { OpCount::ops++; return cd(a.v op b); }
CD_BIN(+)
CD_BIN(-)
CD_BIN(*)
CD_BIN(/)
inline cd operator-(cd a) { return cd(-a.v); }
#define CD_CMP(op) \
    inline bool operator op(cd a, cd b) { return a.v op b.v; } \
    inline bool operator op(cd a, double b) { return a.v op b; } \
    inline bool operator op(double a, cd b) { return a op b.v; }
CD_CMP(<)
CD_CMP(>)
CD_CMP(<=)
CD_CMP(>=)
CD_CMP(==)
CD_CMP(!=)
inline cd& operator+=(cd& a, cd b) { a = a + b; return a; }
inline cd& operator-=(cd& a, cd b) { a = a - b; return a; }
inline cd& operator*=(cd& a, cd b) { a = a * b; return a; }
inline cd& operator/=(cd& a, cd b) { a = a / b; return a; }
inline cd sqrt(cd a) { OpCount::sqrts++; return cd(std::sqrt(a.v)); }
inline cd atan2(cd a, cd b) { OpCount::atan2s++; return cd(std::atan2(a.v, b.v)); }
inline cd fabs(cd a) { return cd(std::fabs(a.v)); }
inline cd floor(cd a) { return cd(std::floor(a.v)); }
inline cd cos(cd a) { return cd(std::cos(a.v)); }
inline cd sin(cd a) { return cd(std::sin(a.v)); }
inline cd pow(cd a, int b) { return cd(std::pow(a.v, b)); }
inline bool isnan(cd a) { return std::isnan(a.v); }
#define double cd
extern "C" {
#include "bpm_oracle.c"
}
#undef double
int main() {
    cd x1[3] = {0.0, 0.0, 0.0}, x2[3] = {0.98, 0.05, 0.03};
    cd q1[4] = {0.9999, 0.01, 0.005, 0.0}, q2[4] = {0.9998, -0.01, 0.012, 0.011};
    cd ri[3] = {1.0, 0.0, 0.0}, K[4] = {7854.0, 9817.0, 377.0, 490.9};
    cd f1[3], t1[3], f2[3], t2[3], U, diag[8];
    OpCount::ops = OpCount::sqrts = OpCount::atan2s = 0;
    orc_bond(x1, x2, q1, q2, ri, K, -1, f1, t1, f2, t2, nullptr, nullptr);
    std::printf("%ld %ld %ld\n", OpCount::ops, OpCount::sqrts, OpCount::atan2s);
    return 0;
}
