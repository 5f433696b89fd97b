// Forward-mode dual numbers for the adjoint kernels: a value of base type B
// with K directional derivatives.  Instantiating the per-node step code with
// this type gives K columns of the node's Jacobian per evaluation; the
// adjoint kernels contract them with the adjoint populations (one
// vector-Jacobian product per K input directions).
#pragma once

#include <type_traits>

#include "lbm_device.cuh"

namespace lbm {

template <class B, int K>
struct Dual {
  B v;
  B d[K];
  LBM_HD Dual() {}
  template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
  LBM_HD Dual(T x) : v(B(x)) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = B(0);
  }
  // the value (only the FP64 condition-bound branch of the diffusion solve,
  // never taken for dual numbers, converts)
  LBM_HD explicit operator double() const { return (double)v; }
  LBM_HD Dual& operator+=(const Dual& b) {
    v += b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] += b.d[k];
    return *this;
  }
  LBM_HD Dual& operator-=(const Dual& b) {
    v -= b.v;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] -= b.d[k];
    return *this;
  }
  LBM_HD Dual& operator*=(const Dual& b) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = d[k] * b.v + v * b.d[k];
    v *= b.v;
    return *this;
  }
  LBM_HD Dual& operator/=(const Dual& b) {
    const B inv = B(1) / b.v;
    const B q = v * inv;
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = (d[k] - q * b.d[k]) * inv;
    v = q;
    return *this;
  }
};

template <class B, int K> LBM_HD Dual<B, K> operator+(Dual<B, K> a, const Dual<B, K>& b) { return a += b; }
template <class B, int K> LBM_HD Dual<B, K> operator-(Dual<B, K> a, const Dual<B, K>& b) { return a -= b; }
template <class B, int K> LBM_HD Dual<B, K> operator*(Dual<B, K> a, const Dual<B, K>& b) { return a *= b; }
template <class B, int K> LBM_HD Dual<B, K> operator/(Dual<B, K> a, const Dual<B, K>& b) { return a /= b; }
template <class B, int K> LBM_HD Dual<B, K> operator-(const Dual<B, K>& a) {
  Dual<B, K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
// mixed operands: a constant of the base type carries no derivative
template <class B, int K> LBM_HD Dual<B, K> operator*(B a, Dual<B, K> b) {
  b.v *= a;
#pragma unroll
  for (int k = 0; k < K; ++k) b.d[k] *= a;
  return b;
}
template <class B, int K> LBM_HD Dual<B, K> operator*(Dual<B, K> b, B a) { return a * b; }
template <class B, int K> LBM_HD Dual<B, K> operator+(B a, Dual<B, K> b) { b.v += a; return b; }
template <class B, int K> LBM_HD Dual<B, K> operator+(Dual<B, K> b, B a) { b.v += a; return b; }
template <class B, int K> LBM_HD Dual<B, K> operator-(Dual<B, K> b, B a) { b.v -= a; return b; }
template <class B, int K> LBM_HD Dual<B, K> operator-(B a, const Dual<B, K>& b) { return Dual<B, K>(a) - b; }
template <class B, int K> LBM_HD Dual<B, K> operator/(Dual<B, K> b, B a) { return b / Dual<B, K>(a); }
template <class B, int K> LBM_HD Dual<B, K> operator/(B a, const Dual<B, K>& b) { return Dual<B, K>(a) / b; }

template <class B, int K> LBM_HD bool operator<(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v < b.v; }
template <class B, int K> LBM_HD bool operator>(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v > b.v; }
template <class B, int K> LBM_HD bool operator<=(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v <= b.v; }
template <class B, int K> LBM_HD bool operator>=(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v >= b.v; }
template <class B, int K> LBM_HD bool operator==(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v == b.v; }
template <class B, int K> LBM_HD bool operator!=(const Dual<B, K>& a, const Dual<B, K>& b) { return a.v != b.v; }

// f(x) with f'(x) given: the chain rule on every lane
template <class B, int K>
LBM_HD Dual<B, K> chain(const Dual<B, K>& x, B fx, B dfx) {
  Dual<B, K> r;
  r.v = fx;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = dfx * x.d[k];
  return r;
}

using ::fabs;    // keep the scalar overloads visible next to the dual one
template <class B, int K>
LBM_HD Dual<B, K> fabs(const Dual<B, K>& x) {
  return x.v < B(0) ? -x : x;
}

template <class B, int K>
struct ScalarTraits<Dual<B, K>> {
  static constexpr bool single = ScalarTraits<B>::single;
};

template <class B, int K>
struct MathOps<Dual<B, K>> {
  static LBM_HD Dual<B, K> sqrt(const Dual<B, K>& x) {
    const B s = MathOps<B>::sqrt(x.v);
    return chain(x, s, B(0.5) / s);
  }
  static LBM_HD Dual<B, K> pow(const Dual<B, K>& x, const Dual<B, K>& e) {
    // exponents are parameters of the transport model: no derivative
    const B p = MathOps<B>::pow(x.v, e.v);
    return chain(x, p, e.v * p / x.v);
  }
};

}  // namespace lbm
