// Scalar types the oracle's right-hand side is instantiated on.
//
// TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h).
//
//   double  - the plain FP64 oracle.
//   Dual    - forward-mode dual number a + b*eps, eps^2 = 0; gives exact
//             directional derivatives R'(U)dU for adjoint dot-product tests
//             (DualL: the same in long double, the tangent's rounding reference).
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
// DualT<R> carries value and derivative in R: Dual (double) for the FP64
// tangent, DualL (long double) for its rounding-error reference.  The
// operators are hidden friends so that a double converts implicitly.
template <class R>
struct DualT {
    R v = 0, d = 0;
    DualT() = default;
    DualT(R x) : v(x), d(0) {}
    DualT(R x, R dx) : v(x), d(dx) {}
    friend DualT operator+(DualT a, DualT b) { return {a.v + b.v, a.d + b.d}; }
    friend DualT operator-(DualT a, DualT b) { return {a.v - b.v, a.d - b.d}; }
    friend DualT operator-(DualT a) { return {-a.v, -a.d}; }
    friend DualT operator*(DualT a, DualT b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
    friend DualT operator/(DualT a, DualT b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
    friend DualT& operator+=(DualT& a, DualT b) { a = a + b; return a; }
    friend DualT& operator-=(DualT& a, DualT b) { a = a - b; return a; }
    friend DualT& operator*=(DualT& a, DualT b) { a = a * b; return a; }
    friend bool operator<(DualT a, DualT b) { return a.v < b.v; }
    friend bool operator>(DualT a, DualT b) { return a.v > b.v; }
    friend bool operator<=(DualT a, DualT b) { return a.v <= b.v; }
    friend bool operator>=(DualT a, DualT b) { return a.v >= b.v; }
    friend double val(DualT a) { return (double)a.v; }
    friend DualT sqrt_(DualT a) {
        R s = std::sqrt(a.v);
        return {s, a.d / (2 * s)};
    }
    friend DualT abs_(DualT a) { return a.v < 0 ? -a : a; }
};
using Dual = DualT<double>;
using DualL = DualT<long double>;

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
