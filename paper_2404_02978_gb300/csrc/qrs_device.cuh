// qrs_device.cuh -- device-side method of libqrs: counter RNG, R2 placement,
// domain maps, PSD weights, coefficients, phase reduction.
//
// Method: Berdja et al., "Quasi-Random Frequency Sampling for Optical
// Turbulence Simulations" (arXiv 2404.02978): Eq. 3 (direct sum and its
// weights), Eq. 4 (jittered grid), Eq. 5 (square map), Eq. 6 (R2 sequence),
// Sec. 3.2 (seed, continuation across realisations, square-to-disc map),
// Eq. 7 (von Karman PSD and aperture filter).
//
// Precision contract of a drawn term (the CPU reference computes the same in
// FP64): the placement s is exact (integer fixed point, FP64 with 53 bits);
// the map to f runs in FP64 and is rounded once to FP32; the weight
// F = sqrt(W(f) J / N_f) and the coefficients (a, b) are FP32 from that FP32
// f, within a few FP32 ulp of the FP64 values.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qrs {

// ------------------------------------------------------------- constants ---
// Philox4x32-10 round multipliers and Weyl key increments (Salmon et al. SC'11).
constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

// Eq. 6 increments in 0.64 fixed point: 2^64/psi and 2^64/psi^2 rounded,
// psi = 1.3247179572447460259609... the real root of x^3 = x + 1.
constexpr uint64_t kR2StepX = 0xC13FA9A902A6328FULL;
constexpr uint64_t kR2StepY = 0x91E10DA5C79E7B1DULL;

// Counter stream ids (third counter word).
constexpr uint32_t kStreamTerm = 0u;  // per-term words
constexpr uint32_t kStreamSeed = 1u;  // random R2 seed
constexpr uint32_t kStreamEq3 = 2u;   // R_u of the literal Eq. 3 coefficients

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

enum { kPsdVonKarman = 0, kPsdKolmogorov = 1 };
enum { kDomSquare = 0, kDomDisc = 1, kDomLogPolar = 2 };
enum { kSmpR2 = 0, kSmpJitter = 1, kSmpUniform = 2, kSmpImportance = 3 };
enum { kCoefGauss = 0, kCoefEq3 = 1 };

// ---------------------------------------------------------------- Philox ---
struct Words {
    uint32_t w0, w1, w2, w3;
};

__host__ __device__ __forceinline__ Words philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                        uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
        const uint32_t hiA = __umulhi(kPhiloxMulA, c0), loA = kPhiloxMulA * c0;
        const uint32_t hiB = __umulhi(kPhiloxMulB, c2), loB = kPhiloxMulB * c2;
#else
        const uint64_t pA = (uint64_t)kPhiloxMulA * c0, pB = (uint64_t)kPhiloxMulB * c2;
        const uint32_t hiA = (uint32_t)(pA >> 32), loA = (uint32_t)pA;
        const uint32_t hiB = (uint32_t)(pB >> 32), loB = (uint32_t)pB;
#endif
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0; c1 = loB; c2 = n2; c3 = loA;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return Words{c0, c1, c2, c3};
}

// ------------------------------------------------------------ parameters ---
// Everything a kernel needs to draw term k of realisation r.  Built on the host
// from the public structs; plain data, passed by value.
struct DrawParams {
    double fmin, fmax;      // cycles/m
    double log_ratio;       // ln(fmax/fmin), LOGPOLAR and IMPORTANCE
    uint64_t s0x, s0y;      // R2 seed, 0.64 fixed point
    const uint32_t* cdf;    // IMPORTANCE cell starts (device)
    int64_t n_f;            // terms per realisation
    int64_t real_offset;    // first realisation of the call
    float psd_c;            // c r0^(-5/3)
    float psd_a;            // L0^-2 (0 for Kolmogorov)
    float jac_c;            // SQUARE 4 fmax^2, DISC pi fmax^2, LOGPOLAR 2 pi ln(fmax/fmin) (x rho^2)
    float inv_nf;           // 1 / N_f
    uint32_t key0, key1;    // Philox key = seed
    int32_t dom, smp, coef; // enums above
    int32_t n_rho, n_theta;
    float ap_D, ap_d;       // Eq. 7 aperture filter of the PSD (ap_D = 0: none)
    float l2_hi, l2_lo;     // log2(fmax/fmin) as a double-float (LOGPOLAR)
    float fmin_hi, fmin_lo; // fmin as a double-float (LOGPOLAR)
    int32_t fold_sh;        // IMPORTANCE: log2 of the sector count (0, 1, 2)
    double frame;           // IMPORTANCE: angle of the cell frame, turns
};

// One drawn term.  J is the cell factor of the weight (w = W J / N_f).
struct Term {
    float fx, fy;  // cycles/m (FP32)
    float F;       // sqrt(W J / N_f), times A(|f|) when the PSD is filtered
    float J;
    float var;     // W J / N_f, the term's variance before the aperture filter
    float A;       // the aperture filter A(|f|) (1 without filter)
    float a, b;    // coefficients
    int32_t cell;
};

// ------------------------------------------------------------------- PSD ---
// W(f) = c r0^(-5/3) (|f|^2 + L0^-2)^(-11/6)  (Eq. 7, first factor), FP32.
__device__ __forceinline__ float psd_w(float psd_c, float psd_a, float f2)
{
    return psd_c * powf(f2 + psd_a, -11.0f / 6.0f);
}

// g(x) = 2 J1(x) / x.  For x < 4 its Taylor series
//   g(x) = sum_m c_m u^m,  u = x^2/4,  c_m = (-1)^m / (m! (m+1)!)
// (m = 0..10: the first omitted term is below 3e-10 at x = 4), by Horner in u
// with an absolute error near 2e-7; beyond, the large-argument form below
// (absolute error of g below 1e-8 from the approximation, a few 1e-8 from
// FP32 evaluation, where |g| < 0.2).
struct AiryCoef {
    float c[11];
    constexpr AiryCoef() : c()
    {
        double v = 1.0;
        for (int m = 0; m < 11; ++m) {
            c[m] = (float)v;
            v = -v / ((double)(m + 1) * (double)(m + 2));
        }
    }
};

// Taylor coefficients of g in v = x^2 through v^M: c_m 4^-m (the series in
// u = x^2/4 with the power of two folded in, which rounds every Horner step
// exactly as the series in u does).  The first omitted term is below 1.1e-11
// for M = 4 at x <= 0.5, 8.9e-11 for M = 6 at x <= 1.5, 3e-10 for M = 10 at
// x <= 4.
template <int M>
struct AirySeriesK {
    float c[M + 1];
    constexpr AirySeriesK() : c()
    {
        constexpr AiryCoef K;
        float s = 1.0f;
        for (int m = 0; m <= M; ++m) {
            c[m] = K.c[m] * s;
            s *= 0.25f;
        }
    }
};

template <int M>
__device__ __forceinline__ float airy_series_v(float v)
{
    constexpr AirySeriesK<M> K;
    float s = K.c[M];
#pragma unroll
    for (int m = M - 1; m >= 0; --m) s = fmaf(s, v, K.c[m]);
    return s;
}

template <int M>
__device__ __forceinline__ float2 airy_series_v2(float2 v)
{
    constexpr AirySeriesK<M> K;
    float2 s = make_float2(K.c[M], K.c[M]);
#pragma unroll
    for (int m = M - 1; m >= 0; --m) s = __ffma2_rn(s, v, make_float2(K.c[m], K.c[m]));
    return s;
}

// The large-argument form from x0 on: J1 in modulus-phase form,
//   g(x) = A(w) x^(-3/2) cos(2 pi [x / (2 pi) - 3/8 + u P(w)]),  u = 1/x, w = u^2,
// with A = 2 sqrt(2/pi) M and P = T / (2 pi) polynomials in w fitted to the
// modulus M and phase correction T of J1 + i Y1 (csrc/airy_fit.py, FP64
// reference values); largest error of g with these FP32 coefficients, in
// FP64: 1.5e-8 (x0 = 4, degree 4), 9.2e-9 (x0 = 8, degree 2), 1.3e-8
// (x0 = 16, degree 1).  The cosine is taken in turns reduced to [-1/2, 1/2],
// so arguments in the hundreds keep their accuracy; x^(-1/2) comes from one
// reciprocal square root and 1/x = its square.
template <int DEG>
struct AiryLargeK;
template <>
struct AiryLargeK<4> {
    float a[5] = {1.595769125e+00f, 2.991877180e-01f, -3.046086143e-01f, 1.014835449e+00f, -3.288978495e+00f};
    float p[5] = {5.968310219e-02f, -2.610418597e-02f, 5.752221473e-02f, -2.702766955e-01f, 1.007727345e+00f};
};
template <>
struct AiryLargeK<2> {
    float a[3] = {1.595769132e+00f, 2.991233879e-01f, -2.871321887e-01f};
    float p[3] = {5.968310043e-02f, -2.608808403e-02f, 5.298583715e-02f};
};
template <>
struct AiryLargeK<1> {
    float a[2] = {1.595769185e+00f, 2.983803074e-01f};
    float p[2] = {5.968309142e-02f, -2.595410740e-02f};
};

template <int DEG>
__device__ __forceinline__ float airy_large(float x)
{
    constexpr AiryLargeK<DEG> K;
    const float rs = rsqrtf(x);
    const float u = __fmul_rn(rs, rs), w = __fmul_rn(u, u), s = __fmul_rn(u, rs);
    float a = K.a[DEG], p = K.p[DEG];
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i) {
        a = __fmaf_rn(a, w, K.a[i]);
        p = __fmaf_rn(p, w, K.p[i]);
    }
    const float turns = __fmaf_rn(x, 0.159154943091895f, __fmaf_rn(u, p, -0.375f));
    const float r = __fsub_rn(__fadd_rn(turns, 12582912.0f), 12582912.0f);  // rint (|turns| < 2^22)
    const float c = __cosf(__fmul_rn(__fsub_rn(turns, r), 6.28318530717958648f));
    return __fmul_rn(__fmul_rn(a, s), c);
}

// airy_large of two arguments in paired FP32 instructions, each element
// rounded exactly as in airy_large.
template <int DEG>
__device__ __forceinline__ float2 airy_large2(float2 x)
{
    constexpr AiryLargeK<DEG> K;
    auto C = [](float c) { return make_float2(c, c); };
    const float2 rs = make_float2(rsqrtf(x.x), rsqrtf(x.y));
    const float2 u = __fmul2_rn(rs, rs), w = __fmul2_rn(u, u), s = __fmul2_rn(u, rs);
    float2 a = C(K.a[DEG]), p = C(K.p[DEG]);
#pragma unroll
    for (int i = DEG - 1; i >= 0; --i) {
        a = __ffma2_rn(a, w, C(K.a[i]));
        p = __ffma2_rn(p, w, C(K.p[i]));
    }
    const float2 turns = __ffma2_rn(x, C(0.159154943091895f), __ffma2_rn(u, p, C(-0.375f)));
    const float2 r = __fadd2_rn(__fadd2_rn(turns, C(12582912.0f)), C(-12582912.0f));
    const float2 ang = __fmul2_rn(__ffma2_rn(r, C(-1.0f), turns), C(6.28318530717958648f));
    return __fmul2_rn(__fmul2_rn(a, s), make_float2(__cosf(ang.x), __cosf(ang.y)));
}

// g(x) = 2 J1(x) / x: below x = 4 its Taylor series (11 terms), from x = 4 on
// the degree-4 large-argument form.  Absolute error near 2e-7 (FP32
// evaluation of the series near x = 4), below 1e-7 beyond.
__device__ __forceinline__ float airy_g_large(float x) { return airy_large<4>(x); }

__device__ __forceinline__ float airy_g(float x)
{
    if (x < 4.0f) return airy_series_v<10>(__fmul_rn(x, x));
    return airy_g_large(x);
}

__device__ __forceinline__ float2 airy_g_large2(float2 x) { return airy_large2<4>(x); }

// Eq. 7 aperture filter A(f) = 2 (D J1(pi D f) - d J1(pi d f)) / (pi (D^2 - d^2) f)
//                            = (D^2 g(pi D f) - d^2 g(pi d f)) / (D^2 - d^2),  A(0) = 1.
__device__ __forceinline__ float airy_filter(float f, float D, float d)
{
    const float piF = 3.14159265358979f * f;
    if (d <= 0.0f) return airy_g(piF * D);
    const float D2 = D * D, d2 = d * d;
    return (D2 * airy_g(piF * D) - d2 * airy_g(piF * d)) / (D2 - d2);
}

// The same with the aperture's weights wD = D^2 / (D^2 - d^2), wd = d^2 /
// (D^2 - d^2) computed once per aperture (no division per term).
__device__ __forceinline__ float airy_filter_w(float f, float D, float d, float wD, float wd)
{
    const float piF = 3.14159265358979f * f;
    if (d <= 0.0f) return airy_g(piF * D);
    return fmaf(wD, airy_g(piF * D), -wd * airy_g(piF * d));
}

// --------------------------------------------------------------- domains ---
// Unit square -> frequency plane in FP64, op for op as the CPU reference
// (explicit _rn intrinsics: no contraction, identical rounding).
__device__ __forceinline__ void map_square(double fmax, double sx, double sy, double& fx, double& fy)
{
    // Eq. 5: f = delta_f N (s - 1/2) with delta_f N = 2 max f
    fx = __dmul_rn(fmax, __dsub_rn(__dmul_rn(2.0, sx), 1.0));
    fy = __dmul_rn(fmax, __dsub_rn(__dmul_rn(2.0, sy), 1.0));
}

__device__ __forceinline__ void map_disc(double fmax, double sx, double sy, double& fx, double& fy)
{
    // Shirley-Chiu concentric map (area ratios preserved), radius fmax.
    const double a = __dsub_rn(__dmul_rn(2.0, sx), 1.0);
    const double b = __dsub_rn(__dmul_rn(2.0, sy), 1.0);
    if (a == 0.0 && b == 0.0) { fx = 0.0; fy = 0.0; return; }
    double r, phi;
    if (fabs(a) > fabs(b)) {
        r = a;
        phi = __dmul_rn(kPi / 4.0, __ddiv_rn(b, a));
    } else {
        r = b;
        phi = __dsub_rn(kPi / 2.0, __dmul_rn(kPi / 4.0, __ddiv_rn(a, b)));
    }
    double s, c;
    sincos(phi, &s, &c);
    const double R = __dmul_rn(fmax, r);
    fx = __dmul_rn(R, c);
    fy = __dmul_rn(R, s);
}

__device__ __forceinline__ void map_logpolar(double fmin, double log_ratio, double sx, double sy, double& fx,
                                             double& fy)
{
    // rho = fmin (fmax/fmin)^s_x, theta = 2 pi s_y
    const double rho = __dmul_rn(fmin, exp(__dmul_rn(sx, log_ratio)));
    const double th = __dmul_rn(kTwoPi, sy);
    double s, c;
    sincos(th, &s, &c);
    fx = __dmul_rn(rho, c);
    fy = __dmul_rn(rho, s);
}

__device__ __forceinline__ double fix_to_unit(uint64_t S) { return (double)(S >> 11) * 0x1p-53; }

// ------------------------------------------- double-float log-polar map ---
// The LOGPOLAR map of an R2 or uniform point without FP64 arithmetic (the
// FP64 pipe runs at 1/64 of the FP32 rate): values carried as unevaluated
// sums hi + lo of two floats (about 48 significant bits) with the classical
// error-free transformations -- Knuth's two-sum, the FMA-based exact product
// -- in explicit round-to-nearest intrinsics, so that no contraction or
// reassociation alters them.  The point is the exact 53-bit fraction
// s = (S >> 11) 2^-53 of the FP64 path, and
//   rho = fmin 2^(s log2(fmax/fmin)),  (cos, sin)(2 pi s_y),
// are evaluated to a relative error near 2^-46 before the one rounding to
// FP32, which therefore agrees with the FP64 map's except when the exact
// value lies within about 2^-46 of a rounding boundary.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_fast_two_sum(float a, float b)  // |a| >= |b| (or a = 0)
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF t = df_two_sum(a.hi, b.hi);
    t.lo = __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(t.hi, t.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}
// a 2^k, exactly: one multiply by the power of two built from its exponent
// field where 2^k and the scaled low part stay normal, ldexpf otherwise.
__device__ __forceinline__ DF df_scale(DF a, int k)
{
    if (k >= -100 && k <= 100) {
        const float s = __int_as_float((k + 127) << 23);
        return DF{__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
    }
    return DF{ldexpf(a.hi, k), ldexpf(a.lo, k)};
}

// Compile-time tables in double, split into (hi, lo) floats:
//   e2[j] = 2^(j/64), j < 64;  sc[j] = (sin, cos)(2 pi j / 256), j < 256,
// from Taylor series summed to convergence (first octant) and the circle's
// symmetries.
struct DfTables {
    float e2[64][2];
    float sc[256][4];
    static constexpr double exp_series(double x)
    {
        double term = 1.0, sum = 1.0;
        for (int n = 1; n < 40; ++n) {
            term = term * x / n;
            sum += term;
        }
        return sum;
    }
    static constexpr double sin_series(double x)
    {
        double term = x, sum = x;
        for (int n = 1; n < 30; ++n) {
            term = -term * x * x / ((2.0 * n) * (2.0 * n + 1.0));
            sum += term;
        }
        return sum;
    }
    static constexpr double cos_series(double x)
    {
        double term = 1.0, sum = 1.0;
        for (int n = 1; n < 30; ++n) {
            term = -term * x * x / ((2.0 * n - 1.0) * (2.0 * n));
            sum += term;
        }
        return sum;
    }
    constexpr DfTables() : e2(), sc()
    {
        const double ln2 = 0.69314718055994530942;
        for (int j = 0; j < 64; ++j) {
            const double v = exp_series(ln2 * j / 64.0);
            e2[j][0] = (float)v;
            e2[j][1] = (float)(v - (double)(float)v);
        }
        for (int j = 0; j < 256; ++j) {
            // angle 2 pi j / 256 = (j mod 64) steps into quadrant q = j / 64
            const int q = j / 64, m = j % 64;
            const double a = kPi * m / 128.0;
            double sn = sin_series(a), cs = cos_series(a);
            for (int r = 0; r < q; ++r) {  // rotate by a quarter turn
                const double t = sn;
                sn = cs;
                cs = -t;
            }
            sc[j][0] = (float)sn;
            sc[j][1] = (float)(sn - (double)(float)sn);
            sc[j][2] = (float)cs;
            sc[j][3] = (float)(cs - (double)(float)cs);
        }
    }
};
static __device__ const DfTables kDfTab{};

// rho = fmin 2^(L2 s): u = L2 s = k + v, v = j/64 + w (w < 1/64),
// 2^w = exp(w ln 2) by its Taylor series (t = w ln 2 < 0.011: the t^2 term in
// double-float, t^3 onwards in float, the first omitted term below 1e-17).
__device__ __forceinline__ DF df_logpolar_rho(uint64_t S, float l2_hi, float l2_lo, float fmin_hi, float fmin_lo)
{
    const uint64_t i = S >> 11;  // 53 bits
    const float s0 = (float)(uint32_t)(i >> 29) * 0x1p-24f;
    const float s1 = __fadd_rn((float)(uint32_t)((i >> 5) & 0xFFFFFFu) * 0x1p-48f, (float)(uint32_t)(i & 31u) * 0x1p-53f);
    const DF s = df_fast_two_sum(s0, s1);
    const DF u = df_mul(DF{l2_hi, l2_lo}, s);
    float k = floorf(u.hi);
    float vh = __fsub_rn(u.hi, k);  // exact
    if (vh == 0.0f && u.lo < 0.0f) {
        k = __fsub_rn(k, 1.0f);
        vh = 1.0f;
    }
    int j = (int)(vh * 64.0f);
    j = j > 63 ? 63 : j;
    const DF w = df_fast_two_sum(__fsub_rn(vh, (float)j * 0.015625f), u.lo);  // first part exact
    const DF t = df_mul(w, DF{0.693147182464599609375f, -1.9046542121259336e-09f});  // ln 2
    const DF t2 = df_mul(t, t);
    const float th = t.hi;
    const float tail = __fmul_rn(__fmul_rn(th, t2.hi),
                                 __fmaf_rn(th, __fmaf_rn(th, __fmaf_rn(th, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f),
                                           1.0f / 6.0f));
    DF e = df_add(t, DF{__fmul_rn(t2.hi, 0.5f), __fmul_rn(t2.lo, 0.5f)});
    e = df_add(e, DF{tail, 0.0f});
    e = df_add(DF{1.0f, 0.0f}, e);  // 2^w
    const DF tj{__ldg(&kDfTab.e2[j][0]), __ldg(&kDfTab.e2[j][1])};
    const DF r = df_mul(df_mul(DF{fmin_hi, fmin_lo}, tj), e);
    return df_scale(r, (int)k);
}

// (sin, cos)(2 pi s): s = j/256 + r (r < 1/256 turns, exact from the 53-bit
// integer), a = 2 pi r < 0.0246; sin a = a - a^3/6 + ..., cos a = 1 - a^2/2 +
// ... (the leading corrections in double-float, the rest in float, the first
// omitted terms below 1e-17), then the angle-sum rotation by the table.
__device__ __forceinline__ void df_sincos_2pi(uint64_t S, DF& sn, DF& cs)
{
    const uint64_t i = S >> 11;  // 53 bits
    const int j = (int)(i >> 45);
    const uint64_t r = i & ((1ull << 45) - 1);
    const DF rr = df_fast_two_sum((float)(uint32_t)(r >> 21) * 0x1p-32f, (float)(uint32_t)(r & 0x1FFFFFu) * 0x1p-53f);
    const DF a = df_mul(rr, DF{6.283185482025146484375f, -1.7484555314695172e-7f});  // 2 pi
    const DF a2 = df_mul(a, a);
    const DF a3 = df_mul(a2, a);
    const float x2 = a2.hi;
    const DF s3 = df_mul(a3, DF{0.16666667163372039795f, -4.967053879312289e-9f});  // 1/6
    const float s_tail = __fmul_rn(__fmul_rn(a3.hi, x2), __fmaf_rn(x2, -1.0f / 5040.0f, 1.0f / 120.0f));
    DF sa = df_add(a, DF{-s3.hi, -s3.lo});
    sa = df_add(sa, DF{s_tail, 0.0f});
    const float c_tail = __fmul_rn(__fmul_rn(x2, x2), __fmaf_rn(x2, __fmaf_rn(x2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f));
    DF ca = df_add(DF{1.0f, 0.0f}, DF{__fmul_rn(a2.hi, -0.5f), __fmul_rn(a2.lo, -0.5f)});
    ca = df_add(ca, DF{c_tail, 0.0f});
    const DF sj{__ldg(&kDfTab.sc[j][0]), __ldg(&kDfTab.sc[j][1])};
    const DF cj{__ldg(&kDfTab.sc[j][2]), __ldg(&kDfTab.sc[j][3])};
    sn = df_add(df_mul(sj, ca), df_mul(cj, sa));
    const DF m = df_mul(sj, sa);
    cs = df_add(df_mul(cj, ca), DF{-m.hi, -m.lo});
}

__device__ __forceinline__ void map_logpolar_df(uint64_t Sx, uint64_t Sy, float l2_hi, float l2_lo, float fmin_hi,
                                                float fmin_lo, float& fx, float& fy)
{
    const DF rho = df_logpolar_rho(Sx, l2_hi, l2_lo, fmin_hi, fmin_lo);
    DF sn, cs;
    df_sincos_2pi(Sy, sn, cs);
    const DF x = df_mul(rho, cs), y = df_mul(rho, sn);
    fx = __fadd_rn(x.hi, x.lo);
    fy = __fadd_rn(y.hi, y.lo);
}

// Coefficients of Eq. 3 from the term's Philox words: Box-Muller from 24-bit
// uniforms (exact in FP32 and FP64 alike), and for the literal Eq. 3 form the
// extra uniform R_u of stream 2.
__device__ __forceinline__ void coef_from_words(const DrawParams& p, uint64_t n, const Words& w, float& a, float& b)
{
    const float U1 = (float)((w.w2 >> 8) + 1u) * 0x1p-24f;
    const float U2 = (float)(w.w3 >> 8) * 0x1p-24f;
    const float rad = sqrtf(-2.0f * logf(U1));
    float sb, cb;
    sincospif(2.0f * U2, &sb, &cb);
    a = rad * cb;
    b = rad * sb;
    if (p.coef == kCoefEq3) {
        // literal Eq. 3: sqrt2 R_n cos(2 pi (f.x + R_u)) = a cos - b sin with
        // a = sqrt2 R_n cos 2 pi R_u, b = sqrt2 R_n sin 2 pi R_u
        const Words v = philox4x32_10((uint32_t)n, (uint32_t)(n >> 32), kStreamEq3, 0u, p.key0, p.key1);
        const float Ru = (float)(v.w0 >> 8) * 0x1p-24f;
        const float Rn = a;
        float su, cu;
        sincospif(2.0f * Ru, &su, &cu);
        a = 1.41421356237309515f * Rn * cu;
        b = 1.41421356237309515f * Rn * su;
    }
}

// The same coefficients in amplitude-phase form: a cos t - b sin t =
// amp cos(t + 2 pi u 2^-24), so that a sum over terms takes one cosine each.
// GAUSS: (a, b) = rad (cos, sin)(2 pi U2), hence amp = rad, u = the 24-bit
// integer of U2; literal Eq. 3: amp = sqrt2 R_n (signed), u = the 24-bit
// integer of R_u.  The top bit of u (half a turn) then moves into the sign of
// amp (cos(t + pi) = -cos t), leaving u < 2^23 (an offset in [0, 0.5) turns,
// exact): the sign of amp is thereby independent of the angle, so that angle
// errors odd in the angle (the FP32 rounding of 2 pi in the turn-to-radian
// step, the cosine's own reduction) average out over the terms instead of
// adding up with the always-positive Box-Muller radius.
__device__ __forceinline__ void coef_polar_from_words(const DrawParams& p, uint64_t n, const Words& w, float& amp,
                                                      uint32_t& u)
{
    const float U1 = (float)((w.w2 >> 8) + 1u) * 0x1p-24f;
    const float rad = sqrtf(-2.0f * logf(U1));
    if (p.coef == kCoefEq3) {
        const float U2 = (float)(w.w3 >> 8) * 0x1p-24f;
        const float Rn = rad * cospif(2.0f * U2);
        const Words v = philox4x32_10((uint32_t)n, (uint32_t)(n >> 32), kStreamEq3, 0u, p.key0, p.key1);
        amp = 1.41421356237309515f * Rn;
        u = v.w0 >> 8;
    } else {
        amp = rad;
        u = w.w3 >> 8;
    }
    if (u & 0x800000u) {
        amp = -amp;
        u &= 0x7FFFFFu;
    }
}

// F amp of coef_polar_from_words for an unfiltered term, as one square root:
// GAUSS amp = sqrt(-2 ln U1) (sign from the top bit of u), so F amp =
// +-sqrt(var (-2 ln U1)), within an FP32 rounding of F amp; the literal Eq. 3
// form takes F amp itself.  u as in coef_polar_from_words.
__device__ __forceinline__ void term_amp_polar(const DrawParams& p, uint64_t n, const Words& w, float var, float F,
                                               float& Fa, uint32_t& u)
{
    if (p.coef == kCoefEq3) {
        float amp;
        coef_polar_from_words(p, n, w, amp, u);
        Fa = F * amp;
        return;
    }
    const float U1 = (float)((w.w2 >> 8) + 1u) * 0x1p-24f;
    Fa = sqrtf(var * (-2.0f * logf(U1)));
    u = w.w3 >> 8;
    if (u & 0x800000u) {
        Fa = -Fa;
        u &= 0x7FFFFFu;
    }
}

// |f| from |f|^2 by one reciprocal square root (within 2 FP32 ulp; 0 at 0).
__device__ __forceinline__ float fast_abs_f(float f2) { return f2 > 0.0f ? f2 * rsqrtf(f2) : 0.0f; }

// Coefficients of stream point n alone (no placement, no FP64).
__device__ __forceinline__ float2 draw_coef(const DrawParams& p, uint64_t n)
{
    const Words w = philox4x32_10((uint32_t)n, (uint32_t)(n >> 32), kStreamTerm, 0u, p.key0, p.key1);
    float a, b;
    coef_from_words(p, n, w, a, b);
    return make_float2(a, b);
}

// --------------------------------------------------------------- the draw ---
// Term k of realisation r: global stream index n = (real_offset + r) N_f + k.
// Optionally returns the Philox words and the R2 state (exact, for parity).
// The filter as an out-of-line call for the draw: kernels whose draw never
// filters keep their register allocation (an inlined filter enlarges it).
static __device__ __noinline__ float airy_filter_call(float f, float D, float d) { return airy_filter(f, D, d); }

// CELL = false skips the cell index (FP64 work the synthesis and piston
// kernels do not use); COEF = false skips the coefficients (a, b) for callers
// that take them in amplitude-phase form from the returned words.
template <bool CELL = true, bool COEF = true>
__device__ __forceinline__ Term draw_term(const DrawParams& p, uint64_t n, int64_t k, Words* words_out = nullptr,
                                          uint64_t* Sx_out = nullptr, uint64_t* Sy_out = nullptr)
{
    const Words w = philox4x32_10((uint32_t)n, (uint32_t)(n >> 32), kStreamTerm, 0u, p.key0, p.key1);
    uint64_t Sx = 0, Sy = 0;
    double sx = 0.0, sy = 0.0, fx = 0.0, fy = 0.0;
    Term t;
    t.cell = -1;
    float J = 0.0f, p_cell = 1.0f;
    if (p.smp == kSmpImportance) {
        // R2 point; the radial band from the marginal CDF with the top 32 bits
        // of x, the angular cell from that band's conditional CDF with the top
        // 32 bits of y; the remainders place the frequency inside the cell by
        // the cell's own log-polar map.  With 2^fold_sh sectors the top
        // fold_sh bits of y pick the sector and the rest, complemented in the
        // mirrored (odd) sectors, takes y's place.
        Sx = p.s0x + n * kR2StepX;
        Sy = p.s0y + n * kR2StepY;
        const uint64_t sec = p.fold_sh ? (Sy >> (64 - p.fold_sh)) : 0ull;
        uint64_t Y = Sy << p.fold_sh;
        if (sec & 1ull) Y = ~Y;
        const uint32_t ux = (uint32_t)(Sx >> 32), uy = (uint32_t)(Y >> 32);
        const uint32_t* cr = p.cdf;
        int lo = 0, hi = p.n_rho;  // largest band with cr[band] <= ux (cr[0] = 0)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(cr + mid) <= ux) lo = mid; else hi = mid;
        }
        const int ir = lo;
        const uint32_t* ct = p.cdf + p.n_rho + (int64_t)ir * p.n_theta;
        lo = 0;
        hi = p.n_theta;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(ct + mid) <= uy) lo = mid; else hi = mid;
        }
        const int it = lo;
        const uint64_t r_start = (uint64_t)__ldg(cr + ir);
        const uint64_t r_end = (ir + 1 < p.n_rho) ? (uint64_t)__ldg(cr + ir + 1) : (1ull << 32);
        const uint64_t t_start = (uint64_t)__ldg(ct + it);
        const uint64_t t_end = (it + 1 < p.n_theta) ? (uint64_t)__ldg(ct + it + 1) : (1ull << 32);
        const double tx = __ddiv_rn((double)(Sx - (r_start << 32)), __dmul_rn((double)(r_end - r_start), 0x1p32));
        const double ty = __ddiv_rn((double)(Y - (t_start << 32)), __dmul_rn((double)(t_end - t_start), 0x1p32));
        const int c = ir * p.n_theta + it;
        const double rho =
            __dmul_rn(p.fmin, exp(__ddiv_rn(__dmul_rn(p.log_ratio, __dadd_rn((double)ir, tx)), (double)p.n_rho)));
        const double v = __ddiv_rn(__dadd_rn((double)it, ty), (double)p.n_theta);  // place in the sector
        const double turn = (sec & 1ull) ? __dsub_rn(__dadd_rn((double)sec, 1.0), v) : __dadd_rn((double)sec, v);
        const double th = __dmul_rn(kTwoPi, __dadd_rn(p.frame, __ddiv_rn(turn, (double)(1 << p.fold_sh))));
        double s, co;
        sincos(th, &s, &co);
        fx = __dmul_rn(rho, co);
        fy = __dmul_rn(rho, s);
        p_cell = (float)__dmul_rn(__dmul_rn((double)(r_end - r_start), 0x1p-32),
                                  __dmul_rn((double)(t_end - t_start), 0x1p-32));
        t.cell = c;
    } else {
        const bool df_map = p.dom == kDomLogPolar && p.smp != kSmpJitter;
        if (p.smp == kSmpR2 || p.smp == kSmpUniform) {
            if (p.smp == kSmpR2) {
                Sx = p.s0x + n * kR2StepX;  // Eq. 6, mod 2^64
                Sy = p.s0y + n * kR2StepY;
            } else {
                Sx = (uint64_t)w.w0 << 32;  // s = w 2^-32
                Sy = (uint64_t)w.w1 << 32;
            }
            if (CELL || !df_map) {
                sx = fix_to_unit(Sx);
                sy = fix_to_unit(Sy);
            }
        } else {  // Eq. 4 jittered grid: cell (i, j), k = j n_rho + i
            const int64_t i = k % p.n_rho, j = k / p.n_rho;
            sx = __ddiv_rn(__dadd_rn((double)i, (double)w.w0 * 0x1p-32), (double)p.n_rho);
            sy = __ddiv_rn(__dadd_rn((double)j, (double)w.w1 * 0x1p-32), (double)p.n_theta);
        }
        if (df_map) {
            // the same point, map in double-float: one rounding to FP32
            map_logpolar_df(Sx, Sy, p.l2_hi, p.l2_lo, p.fmin_hi, p.fmin_lo, t.fx, t.fy);
        } else {
            if (p.dom == kDomSquare) map_square(p.fmax, sx, sy, fx, fy);
            else if (p.dom == kDomDisc) map_disc(p.fmax, sx, sy, fx, fy);
            else map_logpolar(p.fmin, p.log_ratio, sx, sy, fx, fy);
            t.fx = (float)fx;  // the one FP64 -> FP32 rounding of the method
            t.fy = (float)fy;
        }
        if (CELL) {
            int ir = (int)floor(__dmul_rn(sx, (double)p.n_rho));
            int it = (int)floor(__dmul_rn(sy, (double)p.n_theta));
            ir = ir > p.n_rho - 1 ? p.n_rho - 1 : ir;
            it = it > p.n_theta - 1 ? p.n_theta - 1 : it;
            t.cell = ir * p.n_theta + it;
        }
    }
    if (p.smp == kSmpImportance) {
        t.fx = (float)fx;  // the one FP64 -> FP32 rounding of the method
        t.fy = (float)fy;
    }
    const float f2 = t.fx * t.fx + t.fy * t.fy;
    if (p.smp != kSmpImportance) J = (p.dom == kDomLogPolar) ? p.jac_c * f2 : p.jac_c;
    else J = p.jac_c * f2 / ((float)(p.n_rho * p.n_theta) * p_cell);  // log-polar Jacobian / (cells x p_c)
    t.J = J;
    t.A = (p.ap_D > 0.0f) ? airy_filter_call(sqrtf(f2), p.ap_D, p.ap_d) : 1.0f;
    t.var = psd_w(p.psd_c, p.psd_a, f2) * J * p.inv_nf;
    t.F = sqrtf(t.var) * t.A;
    if (COEF) {
        coef_from_words(p, n, w, t.a, t.b);
    } else {
        t.a = 0.0f;
        t.b = 0.0f;
    }
    if (words_out) *words_out = w;
    if (Sx_out) *Sx_out = Sx;
    if (Sy_out) *Sy_out = Sy;
    return t;
}

// ------------------------------------------------------- phase reduction ---
// Double-float reduction of phi = fx x + fy y mod 1 (cycles): each product is
// split error-free (p = fl(f x), e = fma(f, x, -p)), the integer parts of the
// products are removed exactly (magic-number rint, valid for |p| < 2^22), and
// the small remainders are summed.  Result in [-1 - eps, 1 + eps].
__device__ __forceinline__ float phase_df(float fx, float fy, float x, float y)
{
    const float p1 = __fmul_rn(fx, x);
    const float e1 = __fmaf_rn(fx, x, -p1);
    const float p2 = __fmul_rn(fy, y);
    const float e2 = __fmaf_rn(fy, y, -p2);
    const float M = 12582912.0f;  // 1.5 * 2^23
    const float n1 = __fsub_rn(__fadd_rn(p1, M), M);
    const float n2 = __fsub_rn(__fadd_rn(p2, M), M);
    const float r = __fadd_rn(__fsub_rn(p1, n1), __fsub_rn(p2, n2));
    return __fadd_rn(r, __fadd_rn(e1, e2));
}

// phase_df with a per-term phase offset psi (turns, |psi| <= 0.5) taken into
// the small parts: r + (psi + (e1 + e2)) (the scalar form of phase_df2_psi).
__device__ __forceinline__ float phase_df_psi(float fx, float fy, float x, float y, float psi)
{
    const float p1 = __fmul_rn(fx, x);
    const float e1 = __fmaf_rn(fx, x, -p1);
    const float p2 = __fmul_rn(fy, y);
    const float e2 = __fmaf_rn(fy, y, -p2);
    const float M = 12582912.0f;  // 1.5 * 2^23
    const float n1 = __fsub_rn(__fadd_rn(p1, M), M);
    const float n2 = __fsub_rn(__fadd_rn(p2, M), M);
    const float r = __fadd_rn(__fsub_rn(p1, n1), __fsub_rn(p2, n2));
    return __fadd_rn(r, __fadd_rn(psi, __fadd_rn(e1, e2)));
}

// phase_df_psi for two positions at once (x.x, y.x) and (x.y, y.y), in paired
// FP32 instructions: r + (psi + (e1 + e2)), |result| <= 1.5 + eps turns for
// |psi| <= 0.5.  No pair is negated: the product errors are formed negated
// (fma(-f, x, p) = -fma(f, x, -p) exactly, rounding being symmetric) and the
// differences a - b as fma(b, -1, a); each element is rounded exactly as in
// phase_df_psi.
__device__ __forceinline__ float2 phase_df2_psi(float fx, float fy, float2 x, float2 y, float psi)
{
    const float2 FX = make_float2(fx, fx), FY = make_float2(fy, fy);
    const float2 NFX = make_float2(-fx, -fx), NFY = make_float2(-fy, -fy);
    const float2 M = make_float2(12582912.0f, 12582912.0f), NM = make_float2(-12582912.0f, -12582912.0f);
    const float2 MINUS1 = make_float2(-1.0f, -1.0f);
    const float2 p1 = __fmul2_rn(FX, x);
    const float2 ne1 = __ffma2_rn(NFX, x, p1);  // -e1
    const float2 p2 = __fmul2_rn(FY, y);
    const float2 ne2 = __ffma2_rn(NFY, y, p2);  // -e2
    const float2 n1 = __fadd2_rn(__fadd2_rn(p1, M), NM);
    const float2 n2 = __fadd2_rn(__fadd2_rn(p2, M), NM);
    const float2 r = __fadd2_rn(__ffma2_rn(n1, MINUS1, p1), __ffma2_rn(n2, MINUS1, p2));
    const float2 sm = __ffma2_rn(__fadd2_rn(ne1, ne2), MINUS1, make_float2(psi, psi));  // psi + (e1 + e2)
    return __fadd2_rn(r, sm);
}

// phase_df of two frequencies (fx.x, fy.x), (fx.y, fy.y) at one position, in
// paired FP32 instructions; each element is rounded exactly as in phase_df.
__device__ __forceinline__ float2 phase_df2f(float2 fx, float2 fy, float x, float y)
{
    const float2 X = make_float2(x, x), Y = make_float2(y, y), NX = make_float2(-x, -x), NY = make_float2(-y, -y);
    const float2 M = make_float2(12582912.0f, 12582912.0f), NM = make_float2(-12582912.0f, -12582912.0f);
    const float2 MINUS1 = make_float2(-1.0f, -1.0f);
    const float2 p1 = __fmul2_rn(fx, X);
    const float2 ne1 = __ffma2_rn(fx, NX, p1);  // -e1
    const float2 p2 = __fmul2_rn(fy, Y);
    const float2 ne2 = __ffma2_rn(fy, NY, p2);  // -e2
    const float2 n1 = __fadd2_rn(__fadd2_rn(p1, M), NM);
    const float2 n2 = __fadd2_rn(__fadd2_rn(p2, M), NM);
    const float2 r = __fadd2_rn(__ffma2_rn(n1, MINUS1, p1), __ffma2_rn(n2, MINUS1, p2));
    return __ffma2_rn(__fadd2_rn(ne1, ne2), MINUS1, r);  // r + (e1 + e2)
}

// Fixed-point reduction: f and x quantised to int32 at per-launch binary
// scales 2^a and 2^b (|F|, |X| < 2^31), phi 2^(a+b) = Fx X + Fy Y computed
// exactly in 64-bit wraparound arithmetic (the integer part falls off the
// top), 23 fraction bits extracted into a float mantissa.  `bias` adds half a
// revolution and half an output ulp so that the result is the rounded phase
// in [-0.5, 0.5).  Two IMAD.WIDE + SHF + LOP3 + FADD per (point, term).
__device__ __forceinline__ float phase_fx(int32_t Fx, int32_t Fy, int32_t X, int32_t Y, uint64_t bias, uint32_t shift)
{
    uint64_t acc = bias + (uint64_t)((int64_t)Fy * (int64_t)Y);
    acc += (uint64_t)((int64_t)Fx * (int64_t)X);
    const uint32_t m = __funnelshift_rc((uint32_t)acc, (uint32_t)(acc >> 32), shift);
    return __int_as_float((m & 0x007FFFFFu) | 0x3F800000u) - 1.5f;
}

// The same fixed-point phase returned in radians in [0, 2 pi): with `bias`
// holding only the half-ulp rounding term (no half revolution), the mantissa
// m in [1, 2) holds 1 + frac(turns), and one FFMA forms m 2pi - 2pi =
// (m - 1) 2pi with the rounded constant cancelling exactly; error: the
// 2^-24-turn extraction rounding plus one FP32 rounding of the angle.
// The 32-bit word whose low 23 bits are frac(f.x) in units of 2^-23 turn
// (rounded by `bias`): the extraction step of phase_fx_rad.
__device__ __forceinline__ uint32_t phase_fx_word(int32_t Fx, int32_t Fy, int32_t X, int32_t Y, uint64_t bias,
                                                  uint32_t shift)
{
    uint64_t acc = bias + (uint64_t)((int64_t)Fy * (int64_t)Y);
    acc += (uint64_t)((int64_t)Fx * (int64_t)X);
    return __funnelshift_rc((uint32_t)acc, (uint32_t)(acc >> 32), shift);
}

// phase_fx_word at a + b = 55: the 23 fraction bits are the low bits of the
// high word of the phase word, taken without a shift.
__device__ __forceinline__ uint32_t phase_fx_word_hi(int32_t Fx, int32_t Fy, int32_t X, int32_t Y, uint64_t bias)
{
    uint64_t acc = bias + (uint64_t)((int64_t)Fy * (int64_t)Y);
    acc += (uint64_t)((int64_t)Fx * (int64_t)X);
    return (uint32_t)(acc >> 32);
}

__device__ __forceinline__ float phase_fx_rad(int32_t Fx, int32_t Fy, int32_t X, int32_t Y, uint64_t bias,
                                              uint32_t shift)
{
    const uint32_t m = phase_fx_word(Fx, Fy, X, Y, bias, shift);
    return fmaf(__int_as_float((m & 0x007FFFFFu) | 0x3F800000u), 6.28318530717958648f, -6.28318530717958648f);
}

__device__ __forceinline__ void sincos_turns(float turns, float& s, float& c)
{
    const float ang = turns * 6.28318530717958648f;
    s = __sinf(ang);
    c = __cosf(ang);
}

// ceil(log2(v)) for v > 0 (exact for powers of two).
__device__ __host__ __forceinline__ int ceil_log2(double v)
{
    int e;
    const double m = frexp(v, &e);  // v = m 2^e, m in [0.5, 1)
    return (m == 0.5) ? e - 1 : e;
}

// Per-launch scales of the fixed-point phase (phase_fx / phase_fx_rad) from
// the frequency bound and the point bound: a = 31 - ceil(log2 fbound),
// b = 31 - ceil(log2 xbound), b lowered so that a + b <= max_ab (54 for the
// funnel-shift extraction, whose shift a + b - 23 is at most 31; 55 for a
// caller that takes the high word when shift = 32), use_fixed when
// fbound xbound <= 128 (then the quantisation error, <= fbound xbound 2^-30
// turns, is below the double-float path's).  `radians`: bias for
// phase_fx_rad ([0, 1) turns) instead of phase_fx ([-0.5, 0.5) turns).
struct FixedScales {
    bool use_fixed;
    float fscale, xscale;  // 2^a, 2^b
    uint64_t bias;
    uint32_t shift;
    uint32_t psi_mul;      // 2^(a+b-24): a 24-bit phase offset u 2^-24 turns is u psi_mul in the phase word
};

__device__ __forceinline__ FixedScales fixed_scales(float fbound, float xbound, bool radians, int max_ab = 54)
{
    FixedScales z;
    const double fb = (double)fbound * (1.0 + 0x1p-20);
    const double xb = (double)xbound * (1.0 + 0x1p-20);
    z.use_fixed = (fb * xb <= 128.0);
    const int a = 31 - ceil_log2(fb);
    int b = (xb > 0.0) ? 31 - ceil_log2(xb) : max_ab - a;
    if (a + b > max_ab) b = max_ab - a;
    if (a + b < 24) z.use_fixed = false;
    const int ab = a + b;
    z.fscale = ldexpf(1.0f, a);
    z.xscale = ldexpf(1.0f, b);
    z.shift = (uint32_t)(ab - 23);
    z.psi_mul = (ab >= 24 && ab <= 55) ? (1u << (ab - 24)) : 0u;
    // half an output ulp (rounding), plus half a revolution for [-0.5, 0.5) turns
    const uint64_t half_ulp = (ab >= 24 && ab <= 64) ? (1ull << (ab - 24)) : 0ull;
    z.bias = radians ? half_ulp : ((ab >= 1 && ab <= 64) ? ((1ull << (ab - 1)) + half_ulp) : 0ull);
    return z;
}

}  // namespace qrs
