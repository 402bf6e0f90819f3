// Double-double arithmetic for the host set-up (about 106 significant
// bits), built on the error-free transformations TwoSum and TwoProd (the
// latter via a fused multiply-add).  Used so that the operator matrices,
// whose construction involves ill-conditioned sums and solves, round
// correctly to double.  Portable: only IEEE double operations and fma.
#pragma once

#include <cmath>

namespace fr {

struct DD {
    double hi = 0.0, lo = 0.0;
    DD() {}
    DD(double h) : hi(h), lo(0.0) {}
    DD(double h, double l) : hi(h), lo(l) {}
    double to_double() const { return hi + lo; }
};

inline DD two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return DD(s, e);
}

inline DD quick_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return DD(s, e);
}

inline DD two_prod(double a, double b) {
    double p = a * b;
    double e = std::fma(a, b, -p);
    return DD(p, e);
}

inline DD operator+(const DD &a, const DD &b) {
    DD s = two_sum(a.hi, b.hi);
    DD t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

inline DD operator-(const DD &a) { return DD(-a.hi, -a.lo); }
inline DD operator-(const DD &a, const DD &b) { return a + (-b); }

inline DD operator*(const DD &a, const DD &b) {
    DD p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

inline DD operator/(const DD &a, const DD &b) {
    // long division: q1 = a/b, r = a - q1 b, q2 = r/b, ...
    double q1 = a.hi / b.hi;
    DD r = a - b * DD(q1);
    double q2 = r.hi / b.hi;
    r = r - b * DD(q2);
    double q3 = r.hi / b.hi;
    DD q = quick_two_sum(q1, q2);
    return q + DD(q3);
}

inline DD &operator+=(DD &a, const DD &b) { return a = a + b; }
inline DD &operator-=(DD &a, const DD &b) { return a = a - b; }
inline DD &operator*=(DD &a, const DD &b) { return a = a * b; }
inline DD &operator/=(DD &a, const DD &b) { return a = a / b; }

inline bool operator<(const DD &a, const DD &b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline bool operator>(const DD &a, const DD &b) { return b < a; }
inline bool operator==(const DD &a, const DD &b) { return a.hi == b.hi && a.lo == b.lo; }
inline bool operator!=(const DD &a, const DD &b) { return !(a == b); }

inline DD dd_abs(const DD &a) { return a.hi < 0.0 ? -a : a; }

inline DD dd_sqrt(const DD &a) {
    if (a.hi <= 0.0) return DD(0.0);
    double x = 1.0 / std::sqrt(a.hi);
    double ax = a.hi * x;
    DD d = a - two_prod(ax, ax);
    return two_sum(ax, d.hi * (x * 0.5));
}

}  // namespace fr
