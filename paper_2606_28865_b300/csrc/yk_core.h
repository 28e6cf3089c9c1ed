/*
 * yk_core.h — per-item arithmetic of the long-range evaluator, shared by the CUDA kernels.
 *
 * Everything here is a pure function of its arguments (no threads, no shared memory), marked
 * host+device so that host code (plan set-up) can use the same statements.  The kernels in
 * yk_kernels.cu decide which thread runs which item.
 */
#ifndef YK_CORE_H
#define YK_CORE_H

#include <stdint.h>
#include <math.h>
#include <string.h>

#if defined(__CUDACC__)
#define YK_HD __host__ __device__ __forceinline__
#else
#define YK_HD static inline
#endif

namespace yk {

/* ---------------------------------------------------------------------------------------- */
/* complex arithmetic on (re, im) pairs                                                      */
template <typename R> struct cpx {
    R re, im;
};
template <typename R> YK_HD cpx<R> mk(R a, R b) { cpx<R> z; z.re = a; z.im = b; return z; }
template <typename R> YK_HD cpx<R> add(cpx<R> a, cpx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <typename R> YK_HD cpx<R> sub(cpx<R> a, cpx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <typename R> YK_HD cpx<R> mul(cpx<R> a, cpx<R> b)
{
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
/* a * conj(b) */
template <typename R> YK_HD cpx<R> mulc(cpx<R> a, cpx<R> b)
{
    return mk<R>(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <typename R> YK_HD cpx<R> conj(cpx<R> a) { return mk<R>(a.re, -a.im); }
template <typename R> YK_HD cpx<R> scale(cpx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
/* multiply by -i (SIGN = -1) or +i (SIGN = +1) */
template <int SIGN, typename R> YK_HD cpx<R> mul_i(cpx<R> a)
{
    return SIGN > 0 ? mk<R>(-a.im, a.re) : mk<R>(a.im, -a.re);
}

/* ---------------------------------------------------------------------------------------- */
/* double-float: a real number held as an unevaluated sum hi + lo of two FP32 values, |lo| <=   */
/* ulp(hi)/2 (about 48 significant bits).  B300 runs FP32 at 64 times its FP64 rate, so FFT    */
/* arithmetic of FP64 accuracy (relative error ~1e-14, far below the 1e-10 target) is cheaper  */
/* in FP32 pairs than in FP64.  Addition uses the two-sum error-free transformation (Knuth),   */
/* multiplication the FMA two-product; both renormalise with a fast two-sum.  Intrinsics with   */
/* explicit rounding keep the compiler from contracting or reordering the error terms.         */
#if defined(__CUDA_ARCH__)
#define YK_FADD(a, b) __fadd_rn(a, b)
#define YK_FSUB(a, b) __fsub_rn(a, b)
#define YK_FMUL(a, b) __fmul_rn(a, b)
#define YK_FFMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define YK_FADD(a, b) ((a) + (b))
#define YK_FSUB(a, b) ((a) - (b))
#define YK_FMUL(a, b) ((a) * (b))
#define YK_FFMA(a, b, c) fmaf(a, b, c)
#endif

struct alignas(8) df32 { /* 8-byte aligned: one 64-bit shared-memory access per value */
    float hi, lo;
    df32() = default;
    YK_HD df32(float h, float l) : hi(h), lo(l) {}
    /* from a double: hi = round(d), lo = round(d - hi) (constant-folded for literals) */
    YK_HD explicit df32(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    YK_HD double to_double() const { return (double)hi + (double)lo; }
};

YK_HD df32 df_fast_two_sum(float a, float b)
{
    const float s = YK_FADD(a, b);
    return df32(s, YK_FSUB(b, YK_FSUB(s, a)));
}
/* a + b exactly as a normalised pair, whatever their magnitudes (Knuth's two-sum) */
YK_HD df32 df_two_sum(float a, float b)
{
    const float s = YK_FADD(a, b);
    const float bb = YK_FSUB(s, a);
    return df32(s, YK_FADD(YK_FSUB(a, YK_FSUB(s, bb)), YK_FSUB(b, bb)));
}
YK_HD df32 operator+(df32 a, df32 b)
{
    const float s = YK_FADD(a.hi, b.hi);
    const float bb = YK_FSUB(s, a.hi);
    float e = YK_FADD(YK_FSUB(a.hi, YK_FSUB(s, bb)), YK_FSUB(b.hi, bb));
    e = YK_FADD(e, YK_FADD(a.lo, b.lo));
    return df_fast_two_sum(s, e);
}
YK_HD df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
YK_HD df32 operator-(df32 a, df32 b) { return a + (-b); }
YK_HD df32 operator*(df32 a, df32 b)
{
    const float p = YK_FMUL(a.hi, b.hi);
    float e = YK_FFMA(a.hi, b.hi, -p);
    e = YK_FFMA(a.hi, b.lo, e);
    e = YK_FFMA(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
/* acc + a * b with the product left unnormalised: its (p, e) pair goes straight into the sum */
YK_HD df32 df_mul_add(df32 acc, df32 a, df32 b)
{
    const float p = YK_FMUL(a.hi, b.hi);
    float e = YK_FFMA(a.hi, b.hi, -p);
    e = YK_FFMA(a.hi, b.lo, e);
    e = YK_FFMA(a.lo, b.hi, e);
    const float s = YK_FADD(acc.hi, p);
    const float bb = YK_FSUB(s, acc.hi);
    float t = YK_FADD(YK_FSUB(acc.hi, YK_FSUB(s, bb)), YK_FSUB(p, bb));
    t = YK_FADD(t, YK_FADD(acc.lo, e));
    return df_fast_two_sum(s, t);
}

/* acc + a * b for an accumulator that is only summed further (the spread's tile cells): the same
 * exact two-sum of the high words, but the pair (s, t) is kept unnormalised (no final fast
 * two-sum).  The low word then gathers the N additions' rounding errors (each below half an ulp of
 * the high word), so the pair stays exact to ~N 2^-48 of the cell, ~4e-12 for 1,000 additions;
 * the pair is normalised when the tiles are summed. */
YK_HD df32 df_mul_add_lazy(df32 acc, df32 a, df32 b)
{
    const float p = YK_FMUL(a.hi, b.hi);
    float e = YK_FFMA(a.hi, b.hi, -p);
    e = YK_FFMA(a.hi, b.lo, e);
    e = YK_FFMA(a.lo, b.hi, e);
    const float s = YK_FADD(acc.hi, p);
    const float bb = YK_FSUB(s, acc.hi);
    const float t = YK_FADD(YK_FSUB(acc.hi, YK_FSUB(s, bb)), YK_FSUB(p, bb));
    return df32(s, YK_FADD(t, YK_FADD(acc.lo, e)));
}

/* acc + a * b for an FP32 a (the two-product needs one FMA less), the pair left unnormalised as
 * in df_mul_add_lazy */
YK_HD df32 df_mul_add_lazy(df32 acc, float a, df32 b)
{
    const float p = YK_FMUL(a, b.hi);
    float e = YK_FFMA(a, b.hi, -p);
    e = YK_FFMA(a, b.lo, e);
    const float s = YK_FADD(acc.hi, p);
    const float bb = YK_FSUB(s, acc.hi);
    const float t = YK_FADD(YK_FSUB(acc.hi, YK_FSUB(s, bb)), YK_FSUB(p, bb));
    return df32(s, YK_FADD(t, YK_FADD(acc.lo, e)));
}

/* Double-float with lazy normalisation, for the FFT butterflies: sums and products keep their
 * (hi, lo) pair as computed (the exact two-sum of the high words with the low words added, or the
 * FMA two-product), without the final fast two-sum that makes |lo| <= ulp(hi)/2.  Every operation
 * still carries the exact rounding error of its high words, so a value keeps ~48 bits relative to
 * the magnitudes it was formed from; where high words cancel, the low word may exceed the high one
 * and the value then keeps 24 bits of itself, i.e. ~2^-48 of the operands (the FFT's error is
 * relative to the transform's norm, so this costs nothing).  A stage's values are normalised
 * once, when they are stored (df_norm).  8 FP32 operations per sum instead of 11, 4 per product
 * instead of 7. */
struct alignas(8) df32l {
    float hi, lo;
    df32l() = default;
    YK_HD df32l(float h, float l) : hi(h), lo(l) {}
    YK_HD explicit df32l(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    YK_HD explicit df32l(df32 v) : hi(v.hi), lo(v.lo) {}
};
YK_HD df32 df_norm(df32l v) { return df_fast_two_sum(v.hi, v.lo); }
YK_HD df32l operator+(df32l a, df32l b)
{
    const float s = YK_FADD(a.hi, b.hi);
    const float bb = YK_FSUB(s, a.hi);
    const float e = YK_FADD(YK_FSUB(a.hi, YK_FSUB(s, bb)), YK_FSUB(b.hi, bb));
    return df32l(s, YK_FADD(e, YK_FADD(a.lo, b.lo)));
}
YK_HD df32l operator-(df32l a) { return df32l(-a.hi, -a.lo); }
YK_HD df32l operator-(df32l a, df32l b) { return a + (-b); }
YK_HD df32l operator*(df32l a, df32l b)
{
    const float p = YK_FMUL(a.hi, b.hi);
    float e = YK_FFMA(a.hi, b.hi, -p);
    e = YK_FFMA(a.hi, b.lo, e);
    e = YK_FFMA(a.lo, b.hi, e);
    return df32l(p, e);
}

/* r rounded to the nearest int64, ties to even (as llrint in the default rounding mode), on the
 * IEEE bits with integer operations: |r| = m 2^(e - 52) with the 53-bit significand m; for
 * e >= 52 it is the integer m << (e - 52), below that m is shifted right and the dropped bits
 * decide the rounding.  Magnitudes of 2^63 and more (and infinities, NaN) give +-LLONG_MAX. */
YK_HD long long round_even_ll(double r)
{
#if defined(__CUDA_ARCH__)
    const long long b = __double_as_longlong(r);
#else
    long long b;
    memcpy(&b, &r, sizeof b);
#endif
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const long long m = (b & 0xfffffffffffffll) | (1ll << 52);
    long long v;
    if (e >= 52) {
        v = e > 62 ? 0x7fffffffffffffffll : (m << (e - 52));
    } else if (e < -1) {
        v = 0; /* |r| < 1/2, zero and subnormals included */
    } else {
        const int s = 52 - e; /* 1 .. 53 */
        const long long q = m >> s, rem = m & ((1ll << s) - 1), half = 1ll << (s - 1);
        v = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
    return b < 0 ? -v : v;
}

/* ---------------------------------------------------------------------------------------- */
/* exponential-of-semicircle window phi(z) = exp(beta (sqrt(1 - (2z/w)^2) - 1)), |z| <= w/2    */
/* (the spreading kernel of the NUFFT that evaluates eqs. disrete_sigma_hat and sh_fourier)  */
template <typename R> YK_HD R es_window(R z, R beta, R c /* = 4/w^2 */)
{
    R s = (R)1 - c * z * z;
    return s >= (R)0 ? exp(beta * (sqrt(s) - (R)1)) : (R)0;
}

/* the same window with the exponent written as -beta c z^2 / (1 + sqrt(1 - c z^2)): no
 * cancellation in sqrt(.) - 1, so in FP32 the relative error of phi stays a few ulp instead of
 * beta ulp (used by the FP32 path, where it decides whether 1e-6 is reachable) */
template <typename R> YK_HD R es_window_stable(R z, R beta, R c)
{
    const R u = c * z * z;
    return u <= (R)1 ? exp(-beta * u / ((R)1 + sqrt((R)1 - u))) : (R)0;
}

#if defined(__CUDACC__)
/* es_window_stable in FP32 with CUDA's fast exponential and division intrinsics, for the FP32C
 * kernels (target 1e-6): __expf is within 2 + 1.2 |x| ulp for the exponent x in [-beta, 0] and
 * __fdividef within 2 ulp, so a window value is within ~1.6e-7 of the window's peak (the IEEE
 * functions: a few ulp of the value) */
__device__ __forceinline__ float es_window32(float z, float beta, float c)
{
    const float u = c * z * z;
    return u <= 1.0f ? __expf(__fdividef(-beta * u, 1.0f + sqrtf(1.0f - u))) : 0.0f;
}
#endif

/* first tap l0 = ceil(t - w/2) of a point at grid coordinate t; taps l0 .. l0+w-1, and the
 * window arguments z_a = l0 + a - t lie in [-w/2, w/2) */
template <int W> YK_HD int first_tap(double t) { return (int)ceil(t - 0.5 * W); }

/* non-negative residue of a mod n for |a| < 2n */
YK_HD int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

/* ---------------------------------------------------------------------------------------- */
/* FFT: in-place mixed-radix decimation-in-frequency (Sande-Tukey) on L points.               */
/*                                                                                           */
/* Stage s has radix r_s, block length B_s = L / (r_1 ... r_{s-1}) and span_s = B_s / r_s.   */
/* Butterfly t in [0, L / r_s) of stage s: block b = t / span_s, k = t % span_s, elements     */
/* x[b B_s + k + q span_s] (q < r_s) -> length-r_s DFT -> output p multiplied by W_{B_s}^{pk}  */
/* and stored back at x[b B_s + k + p span_s] (fft_stage in yk_stages.cuh).  After all stages position                     */
/* sum_s p_s span_s holds frequency p_1 + r_1 (p_2 + r_2 (p_3 + ...)) (digit-reversed order). */
/* The inverse (natural order out, unnormalised, e^{+}) runs the stages in reverse order and   */
/* for each butterfly multiplies by conj(W_{B_s}^{pk}) before the inverse length-r_s DFT.     */
/*                                                                                           */
/* Twiddles come from a table tw[j] = exp(-2 pi i j / n_tab) with W_B^e = tw[e * (n_tab / B)]. */
#define YK_MAX_STAGES 24

struct FftStages {
    int L;                     /* transform length */
    int n;                     /* number of stages */
    int r[YK_MAX_STAGES];      /* radix of stage s */
    int B[YK_MAX_STAGES];      /* block length of stage s */
    int tw_step[YK_MAX_STAGES]; /* twiddle table stride n_tab / B_s */
    /* division by span_s = B_s / r_s and by nb_s = L / r_s (butterflies per row) as a multiply:
     * q = umulhi(x, ceil(2^32 / d)) equals floor(x / d) for x d < 2^32 (all sizes here are far
     * below 2^16); d = 1 is handled apart */
    unsigned span_m[YK_MAX_STAGES], nb_m[YK_MAX_STAGES];
};

/* host side: fill the division multipliers of st (after r and B) */
static inline void fft_fill_magic(FftStages &st)
{
    for (int s = 0; s < st.n; ++s) {
        const unsigned long long span = (unsigned long long)(st.B[s] / st.r[s]);
        const unsigned long long nb = (unsigned long long)(st.L / st.r[s]);
        st.span_m[s] = span > 1 ? (unsigned)(((1ull << 32) + span - 1) / span) : 0u;
        st.nb_m[s] = nb > 1 ? (unsigned)(((1ull << 32) + nb - 1) / nb) : 0u;
    }
}

/* length-r DFT in place on v[0..r-1]; SIGN = -1 forward (e^{-2 pi i pq/r}), +1 inverse */
template <int SIGN, typename R> YK_HD void dft2(cpx<R> *v)
{
    cpx<R> a = v[0], b = v[1];
    v[0] = add(a, b);
    v[1] = sub(a, b);
}
template <int SIGN, typename R> YK_HD void dft3(cpx<R> *v)
{
    const R h = (R)0.86602540378443864676; /* sqrt(3)/2 */
    cpx<R> s = add(v[1], v[2]), d = sub(v[1], v[2]);
    cpx<R> m = mk<R>(v[0].re - (R)0.5 * s.re, v[0].im - (R)0.5 * s.im);
    cpx<R> t = mul_i<SIGN>(scale(d, h)); /* SIGN i h (x1 - x2) */
    v[0] = add(v[0], s);
    v[1] = add(m, t);
    v[2] = sub(m, t);
}
template <int SIGN, typename R> YK_HD void dft4(cpx<R> *v)
{
    cpx<R> s02 = add(v[0], v[2]), d02 = sub(v[0], v[2]);
    cpx<R> s13 = add(v[1], v[3]), d13 = mul_i<SIGN>(sub(v[1], v[3]));
    v[0] = add(s02, s13);
    v[2] = sub(s02, s13);
    v[1] = add(d02, d13);
    v[3] = sub(d02, d13);
}
template <int SIGN, typename R> YK_HD void dft5(cpx<R> *v)
{
    const R c1 = (R)0.30901699437494742410;  /* cos(2 pi/5) */
    const R c2 = (R)-0.80901699437494742410; /* cos(4 pi/5) */
    const R s1 = (R)0.95105651629515357212;  /* sin(2 pi/5) */
    const R s2 = (R)0.58778525229247312917;  /* sin(4 pi/5) */
    cpx<R> a1 = add(v[1], v[4]), b1 = sub(v[1], v[4]);
    cpx<R> a2 = add(v[2], v[3]), b2 = sub(v[2], v[3]);
    cpx<R> x0 = v[0];
    cpx<R> m1 = mk<R>(x0.re + c1 * a1.re + c2 * a2.re, x0.im + c1 * a1.im + c2 * a2.im);
    cpx<R> m2 = mk<R>(x0.re + c2 * a1.re + c1 * a2.re, x0.im + c2 * a1.im + c1 * a2.im);
    /* SIGN i (s1 b1 + s2 b2) and SIGN i (s2 b1 - s1 b2) */
    cpx<R> t1 = mul_i<SIGN>(mk<R>(s1 * b1.re + s2 * b2.re, s1 * b1.im + s2 * b2.im));
    cpx<R> t2 = mul_i<SIGN>(mk<R>(s2 * b1.re - s1 * b2.re, s2 * b1.im - s1 * b2.im));
    v[0] = mk<R>(x0.re + a1.re + a2.re, x0.im + a1.im + a2.im);
    v[1] = add(m1, t1);
    v[4] = sub(m1, t1);
    v[2] = add(m2, t2);
    v[3] = sub(m2, t2);
}

/* ---------------------------------------------------------------------------------------- */
/* real <-> complex packing: a real row x[0..n) is transformed as z[l] = x[2l] + i x[2l+1]     */
/* with an L = n/2 point complex FFT Z; then for m in [0, L]                                  */
/*   X[m] = (Z[m] + conj Z[L-m]) / 2 + W_n^m (Z[m] - conj Z[L-m]) / (2i)                      */
/* and back: Z'[m] = (X[m] + conj X[L-m]) + i conj(W_n^m) (X[m] - conj X[L-m]), whose          */
/* unnormalised inverse FFT is x[2l] + i x[2l+1] (times 1: the full inverse of X).            */
template <typename R> YK_HD cpx<R> r2c_post(cpx<R> Zm, cpx<R> Zc, cpx<R> Wm)
{
    cpx<R> e = mk<R>((R)0.5 * (Zm.re + Zc.re), (R)0.5 * (Zm.im - Zc.im));
    /* (Zm - conj Zc) / (2i) = -i/2 (Zm - conj Zc) */
    cpx<R> d = mk<R>(Zm.re - Zc.re, Zm.im + Zc.im);
    cpx<R> o = mk<R>((R)0.5 * d.im, (R)-0.5 * d.re);
    return add(e, mul(Wm, o));
}
template <typename R> YK_HD cpx<R> c2r_pre(cpx<R> Xm, cpx<R> Xc, cpx<R> Wm)
{
    cpx<R> s = mk<R>(Xm.re + Xc.re, Xm.im - Xc.im);
    cpx<R> d = mk<R>(Xm.re - Xc.re, Xm.im + Xc.im);
    cpx<R> t = mulc(d, Wm);          /* d conj(W) */
    return add(s, mk<R>(-t.im, t.re)); /* s + i t */
}

} /* namespace yk */

#endif /* YK_CORE_H */
