// Scalar types the oracle's right-hand side is instantiated on.
//
// TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h).
//
//   double  - the plain FP64 oracle.
//   Dual    - forward-mode dual number a + b*eps, eps^2 = 0; gives exact
//             directional derivatives R'(U)dU for adjoint dot-product tests.
//   Counted - a double that counts the floating-point operations performed
//             on it, to state the algorithmic flop count per degree of freedom.
#ifndef DGFV_ORACLE_SCALAR_TYPES_HPP
#define DGFV_ORACLE_SCALAR_TYPES_HPP

#include <cmath>

namespace ora {

// ---------------------------------------------------------------- double
inline double val(double a) { return a; }
inline double sqrt_(double a) { return std::sqrt(a); }
inline double abs_(double a) { return std::fabs(a); }

// ---------------------------------------------------------------- long double
// (extended precision: a rounding-error reference for the double instantiation)
inline double val(long double a) { return (double)a; }
inline long double sqrt_(long double a) { return std::sqrt(a); }
inline long double abs_(long double a) { return std::fabs(a); }

// ---------------------------------------------------------------- Dual
struct Dual {
    double v = 0.0, d = 0.0;
    Dual() = default;
    Dual(double x) : v(x), d(0.0) {}
    Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
    return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline double val(Dual a) { return a.v; }
inline Dual sqrt_(Dual a) {
    double s = std::sqrt(a.v);
    return {s, a.d / (2.0 * s)};
}
inline Dual abs_(Dual a) { return a.v < 0.0 ? -a : a; }

// ---------------------------------------------------------------- Counted
struct FlopCounter {
    double add = 0, mul = 0, div = 0, sqrt = 0;
    int phase = 0;            // step of the right-hand side being counted (0..7)
    double by_phase[8][4] = {};  // add, mul, div, sqrt per step
};
// The counting run is single threaded; one global counter suffices.
inline FlopCounter& flop_counter() {
    static FlopCounter c;
    return c;
}
struct Counted {
    double v = 0.0;
    Counted() = default;
    Counted(double x) : v(x) {}
};
inline void count_op(int cat) {
    FlopCounter& c = flop_counter();
    (&c.add)[cat] += 1;
    c.by_phase[c.phase][cat] += 1;
}
inline Counted operator+(Counted a, Counted b) { count_op(0); return {a.v + b.v}; }
inline Counted operator-(Counted a, Counted b) { count_op(0); return {a.v - b.v}; }
inline Counted operator-(Counted a) { return {-a.v}; }
inline Counted operator*(Counted a, Counted b) { count_op(1); return {a.v * b.v}; }
inline Counted operator/(Counted a, Counted b) { count_op(2); return {a.v / b.v}; }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline double val(Counted a) { return a.v; }
inline Counted sqrt_(Counted a) { count_op(3); return {std::sqrt(a.v)}; }
inline Counted abs_(Counted a) { return {std::fabs(a.v)}; }

}  // namespace ora

#endif
