// orc_types.hpp -- scalar types the oracle's scheme is instantiated with.
//
//   double  : plain values.
//   Dual    : value + directional derivative (forward tangent mode); every
//             branch (min, max, sign, limiter switch) is decided on the value,
//             so the derivative is the one of the branch taken.
//   Counted : a double that counts the arithmetic performed on it
//             (add/sub/mul/div/sqrt = 1 flop each, exp/expm1/log = 1 each,
//             tallied apart; negation, comparisons, min/max/abs are free).
//             Used to fix the algorithmic flop count.
//
// Test infrastructure only; shares nothing with the CUDA library.
#pragma once
#include <cmath>

namespace orc {

// ------------------------------------------------------------------ Dual ---
struct Dual {
    double v, d;
    Dual() : v(0.0), d(0.0) {}
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(const Dual &a, const Dual &b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual &a, const Dual &b) {
    double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
inline Dual sqrt(const Dual &a) {
    double s = std::sqrt(a.v);
    return Dual(s, a.d / (2.0 * s));
}
inline Dual exp(const Dual &a) {
    double e = std::exp(a.v);
    return Dual(e, e * a.d);
}
inline Dual expm1(const Dual &a) { return Dual(std::expm1(a.v), std::exp(a.v) * a.d); }
inline Dual log(const Dual &a) { return Dual(std::log(a.v), a.d / a.v); }

// --------------------------------------------------------------- Counted ---
struct FlopTally {
    long long add = 0, mul = 0, div = 0, sqrt = 0, trans = 0;
    long long total() const { return add + mul + div + sqrt + trans; }
};
// One global tally: counting runs are single-threaded.
FlopTally &tally();

struct Counted {
    double v;
    Counted() : v(0.0) {}
    Counted(double x) : v(x) {}
};
inline Counted operator+(const Counted &a, const Counted &b) { tally().add++; return Counted(a.v + b.v); }
inline Counted operator-(const Counted &a, const Counted &b) { tally().add++; return Counted(a.v - b.v); }
inline Counted operator*(const Counted &a, const Counted &b) { tally().mul++; return Counted(a.v * b.v); }
inline Counted operator/(const Counted &a, const Counted &b) { tally().div++; return Counted(a.v / b.v); }
inline Counted operator-(const Counted &a) { return Counted(-a.v); }
inline Counted sqrt(const Counted &a) { tally().sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted exp(const Counted &a) { tally().trans++; return Counted(std::exp(a.v)); }
inline Counted expm1(const Counted &a) { tally().trans++; return Counted(std::expm1(a.v)); }
inline Counted log(const Counted &a) { tally().trans++; return Counted(std::log(a.v)); }

// ------------------------------------------------------- generic helpers ---
inline double val(double x) { return x; }
inline double val(const Dual &x) { return x.v; }
inline double val(const Counted &x) { return x.v; }

inline double sqrt_(double x) { return std::sqrt(x); }
inline Dual sqrt_(const Dual &x) { return sqrt(x); }
inline Counted sqrt_(const Counted &x) { return sqrt(x); }
inline double exp_(double x) { return std::exp(x); }
inline Dual exp_(const Dual &x) { return exp(x); }
inline Counted exp_(const Counted &x) { return exp(x); }
inline double expm1_(double x) { return std::expm1(x); }
inline Dual expm1_(const Dual &x) { return expm1(x); }
inline Counted expm1_(const Counted &x) { return expm1(x); }
inline double log_(double x) { return std::log(x); }
inline Dual log_(const Dual &x) { return log(x); }
inline Counted log_(const Counted &x) { return log(x); }

// min/max/abs pick one operand by value (ties keep the first operand).
template <class T> inline T tmin(const T &a, const T &b) { return val(b) < val(a) ? b : a; }
template <class T> inline T tmax(const T &a, const T &b) { return val(b) > val(a) ? b : a; }
template <class T> inline T tabs(const T &a) { return val(a) < 0.0 ? -a : a; }

template <class T> inline void from_double(T &dst, double x) { dst = T(x); }

}  // namespace orc
