// k_scalar.cuh -- scalar types of the kernels: double and float (Laplace, FP64 and mixed) and
// cplx<double> / cplx<float> (Helmholtz, complex128 and complex64), with the few generic
// operations the kernels need, so one template body serves all four.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

namespace rs {

template <class R>
struct cplx {
    R re, im;
    cplx() = default;
    __host__ __device__ constexpr cplx(R r, R i = R(0)) : re(r), im(i) {}
    template <class Q>
    __host__ __device__ explicit constexpr cplx(const cplx<Q>& o) : re(R(o.re)), im(R(o.im)) {}
};

template <class R> __host__ __device__ inline cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __host__ __device__ inline cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <class R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, cplx<R> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> __host__ __device__ inline cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ inline cplx<R> operator*(cplx<R> a, R s) { return {s * a.re, s * a.im}; }
template <class R> __host__ __device__ inline cplx<R> operator/(cplx<R> a, cplx<R> b)
{
    // scaled division (Smith's method) to avoid overflow in |b|^2
    if (fabs(b.re) >= fabs(b.im)) {
        const R t = b.im / b.re, den = b.re + b.im * t;
        return {(a.re + a.im * t) / den, (a.im - a.re * t) / den};
    }
    const R t = b.re / b.im, den = b.re * t + b.im;
    return {(a.re * t + a.im) / den, (a.im * t - a.re) / den};
}
template <class R> __host__ __device__ inline cplx<R>& operator+=(cplx<R>& a, cplx<R> b) { a = a + b; return a; }
template <class R> __host__ __device__ inline cplx<R>& operator-=(cplx<R>& a, cplx<R> b) { a = a - b; return a; }

template <class S> struct is_cplx : std::false_type {};
template <class R> struct is_cplx<cplx<R>> : std::true_type {};

// real part type, the FP64 "wide" type of the Gauss-Jordan panel, and the FP64 I/O type
template <class S> struct sc_traits;
template <> struct sc_traits<double> { using real = double; using wide = double; using io = double; };
template <> struct sc_traits<float> { using real = float; using wide = double; using io = double; };
template <> struct sc_traits<cplx<double>> { using real = double; using wide = cplx<double>; using io = cplx<double>; };
template <> struct sc_traits<cplx<float>> { using real = float; using wide = cplx<double>; using io = cplx<double>; };

// a * b + c
__host__ __device__ inline double fma_(double a, double b, double c) { return fma(a, b, c); }
__host__ __device__ inline float fma_(float a, float b, float c) { return fmaf(a, b, c); }
template <class R>
__host__ __device__ inline cplx<R> fma_(cplx<R> a, cplx<R> b, cplx<R> c)
{
    return {fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im))};
}
__host__ __device__ inline double conj_(double a) { return a; }
__host__ __device__ inline float conj_(float a) { return a; }
template <class R> __host__ __device__ inline cplx<R> conj_(cplx<R> a) { return {a.re, -a.im}; }
// |a|^2 and |a| in FP64
__host__ __device__ inline double abs2d(double a) { return a * a; }
__host__ __device__ inline double abs2d(float a) { return (double)a * (double)a; }
template <class R> __host__ __device__ inline double abs2d(cplx<R> a)
{
    return (double)a.re * (double)a.re + (double)a.im * (double)a.im;
}
template <class S> __host__ __device__ inline double absd(S a) { return sqrt(abs2d(a)); }
__host__ __device__ inline double absd(double a) { return fabs(a); }
__host__ __device__ inline double absd(float a) { return fabs((double)a); }
__host__ __device__ inline bool finite_(double a) { return isfinite(a); }
template <class R> __host__ __device__ inline bool finite_(cplx<R> a) { return isfinite((double)a.re) && isfinite((double)a.im); }

// conversions between scalar types (real -> complex puts the value in the real part)
template <class To, class Ti>
__host__ __device__ inline To cast_(Ti v)
{
    if constexpr (is_cplx<To>::value) {
        if constexpr (is_cplx<Ti>::value) return To(v);
        else return To(typename sc_traits<To>::real(v));
    } else {
        return To(v);
    }
}

// scale by a real number
template <class S> __host__ __device__ inline S rscale(double s, S a)
{
    if constexpr (is_cplx<S>::value) return S(typename sc_traits<S>::real(s) * a.re, typename sc_traits<S>::real(s) * a.im);
    else return S(s) * a;
}

#ifdef __CUDACC__
__device__ inline double shfl_xor_(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ inline float shfl_xor_(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <class R> __device__ inline cplx<R> shfl_xor_(cplx<R> v, int o)
{
    return {__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}
__device__ inline double shfl_(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ inline float shfl_(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
template <class R> __device__ inline cplx<R> shfl_(cplx<R> v, int l)
{
    return {__shfl_sync(0xffffffffu, v.re, l), __shfl_sync(0xffffffffu, v.im, l)};
}

// L2-only load of a scalar written by another CTA
__device__ inline double ldcg_(const double* p) { return __ldcg(p); }
__device__ inline float ldcg_(const float* p) { return __ldcg(p); }
template <class R> __device__ inline cplx<R> ldcg_(const cplx<R>* p)
{
    return {__ldcg(&p->re), __ldcg(&p->im)};
}

#endif  // __CUDACC__

}  // namespace rs
