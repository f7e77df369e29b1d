// gks_dual.cuh -- forward-mode derivative numbers for the adjoint of the
// face flux.  Dual<N> carries a value and N directional derivatives; the
// arithmetic and the few elementary functions the kinetic flux uses (exp,
// erfc, sqrt, |x|) propagate them by the chain rule, so the templated flux
// code of gks_device.cuh, instantiated with T = Dual<N>, returns N columns of
// its Jacobian alongside its value.
#pragma once

namespace gks {

template <int N>
struct Dual {
    double v;
    double d[N];
    __device__ __forceinline__ Dual() : v(0.0) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = 0.0;
    }
    __device__ __forceinline__ Dual(double x) : v(x) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = 0.0;
    }
};

#define GKS_DUAL_BINOP(OP, VAL, DER)                                                             \
    template <int N>                                                                             \
    __device__ __forceinline__ Dual<N> operator OP(const Dual<N>& a, const Dual<N>& b) {         \
        Dual<N> r;                                                                               \
        r.v = VAL;                                                                               \
        _Pragma("unroll") for (int i = 0; i < N; ++i) r.d[i] = DER;                              \
        return r;                                                                                \
    }
GKS_DUAL_BINOP(+, a.v + b.v, a.d[i] + b.d[i])
GKS_DUAL_BINOP(-, a.v - b.v, a.d[i] - b.d[i])
GKS_DUAL_BINOP(*, a.v * b.v, a.d[i] * b.v + a.v * b.d[i])
#undef GKS_DUAL_BINOP

template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
    Dual<N> r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
    Dual<N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}

// mixed forms with plain numbers (constants carry no derivative)
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, double b) {
    Dual<N> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(double a, const Dual<N>& b) { return b * a; }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }

template <int N>
__device__ __forceinline__ Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { return a = a + b; }
template <int N>
__device__ __forceinline__ Dual<N>& operator-=(Dual<N>& a, const Dual<N>& b) { return a = a - b; }
template <int N>
__device__ __forceinline__ Dual<N>& operator*=(Dual<N>& a, const Dual<N>& b) { return a = a * b; }

template <int N>
__device__ __forceinline__ bool operator==(const Dual<N>& a, const Dual<N>& b) { return a.v == b.v; }
template <int N>
__device__ __forceinline__ bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N>
__device__ __forceinline__ bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }

// f(a) with f(a.v) = fv and f'(a.v) = fp
template <int N>
__device__ __forceinline__ Dual<N> chain(const Dual<N>& a, double fv, double fp) {
    Dual<N> r;
    r.v = fv;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = fp * a.d[i];
    return r;
}

template <int N>
__device__ __forceinline__ Dual<N> d_exp(const Dual<N>& a) {
    const double e = exp(a.v);
    return chain(a, e, e);
}
// d/dx erfc(x) = -2/sqrt(pi) exp(-x^2)
template <int N>
__device__ __forceinline__ Dual<N> d_erfc(const Dual<N>& a) {
    return chain(a, erfc(a.v), -1.12837916709551257390 * exp(-a.v * a.v));
}
template <int N>
__device__ __forceinline__ Dual<N> d_sqrt(const Dual<N>& a) {
    const double s = sqrt(a.v);
    return chain(a, s, 0.5 / s);
}
// |x|' = sign(x), taken as 0 at 0
template <int N>
__device__ __forceinline__ Dual<N> d_abs(const Dual<N>& a) {
    return chain(a, fabs(a.v), a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0));
}

}  // namespace gks
