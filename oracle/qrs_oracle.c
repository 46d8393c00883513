/*
 * qrs_oracle.c -- plain, slow, FP64 CPU oracle for quasi-random frequency
 * sampling turbulence synthesis (Berdja et al., "Quasi-Random Frequency
 * Sampling for Optical Turbulence Simulations", arXiv 2404.02978).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark use it.  It shares no source, header, table or
 * constant generator with the CUDA library: every constant below is written
 * out here from its definition and pinned by the tests in tests/.
 *
 * Every routine is the plain definition written out in the paper's order:
 * no blocking, no fusion, no reordering.  Floating point is FP64 throughout;
 * the only FP32 step is the one the method defines: a sampled frequency is
 * rounded to FP32 once, and everything downstream uses that FP32 value
 * promoted exactly to FP64.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so qrs_oracle.c -lm
 * (-ffp-contract=off: no silent a*b+c -> fma contraction, so x86 and aarch64
 * hosts give identical results.)
 *
 * Readings of the paper that this oracle encodes (each is listed in the
 * design notes, with its reason):
 *   - Eq. 3 coefficients: two modes.  GAUSS: a,b ~ N(0,1) i.i.d., the term is
 *     F*(a cos 2 pi phi - b sin 2 pi phi); EQ3: the paper's literal
 *     sqrt(2) R_n cos(2 pi (f.r + R_u)) written as a = sqrt2 R_n cos 2piR_u,
 *     b = sqrt2 R_n sin 2piR_u.  Both give each term variance F^2 (Eq. 3 with
 *     its 2/sqrt(2) factor, Sec. 3).
 *   - Eq. 6 in exact 0.64 fixed point: S_n = S_0 + n*alpha mod 2^64, with
 *     alpha = round(2^64/psi), round(2^64/psi^2); point n of the stream is
 *     S_0 + n*alpha (the first point is the seed itself).  The stream is never
 *     re-initialised across realisations (Sec. 3.2): term k of realisation r
 *     is stream point n = (real_offset + r)*N_f + k.
 *   - Eq. 5: f = delta_f * N * (s - 1/2) with delta_f * N = 2 max f, i.e.
 *     f = f_max (2 s - 1).  Cell weight generalises Eq. 3's delta_fx delta_fy
 *     to J(s)/N_f, J the Jacobian of the unit square -> domain map.
 *   - Eq. 7: piston filter A(f) = 2 (D J1(pi D f) - d J1(pi d f)) /
 *     (pi (D^2 - d^2) f), A(0) = 1; the piston PSD is W A^2, so a piston term
 *     is the phase term times A(|f|) (signed: the aperture average of the
 *     harmonic).  The von Karman constant is the exact value of which the
 *     paper's 0.02289 is a truncation.
 *   - Structure function (Sec. 4.4): the difference reading
 *     <|x(t+tau) - x(t)|^2>; lag 0 means the value itself (the spatial
 *     structure function over a baseline is the variance of the
 *     differential piston).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846264338327950288

/* ---------------------------------------------------------------- Philox ---
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * Weyl key schedule.  Round multipliers and Weyl increments as published. */
static const uint32_t OR_PHILOX_M0 = 0xD2511F53u;
static const uint32_t OR_PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t OR_PHILOX_W0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t OR_PHILOX_W1 = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += OR_PHILOX_W0; k1 += OR_PHILOX_W1; }
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Stream ids in the third counter word. */
#define OR_STREAM_TERM 0u  /* per-term words: placement (0,1) + Box-Muller (2,3) */
#define OR_STREAM_SEED 1u  /* random R2 seed s_0 */
#define OR_STREAM_EQ3  2u  /* the extra uniform R_u of the literal Eq. 3 mode */

static void or_words(uint64_t seed, uint64_t n, uint32_t stream, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), stream, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------ R2 (Eq. 6) ---
 * alpha_1 = round(2^64 / psi), alpha_2 = round(2^64 / psi^2), psi the plastic
 * number (real root of x^3 = x + 1).  Written out here; a test re-derives
 * them from a 50-digit psi. */
static const uint64_t OR_R2_ALPHA1 = 0xC13FA9A902A6328FULL;
static const uint64_t OR_R2_ALPHA2 = 0x91E10DA5C79E7B1DULL;

void oracle_r2_seed(uint64_t seed, int use_fixed, uint64_t fx0, uint64_t fy0, uint64_t s0[2])
{
    if (use_fixed) { s0[0] = fx0; s0[1] = fy0; return; }
    uint32_t w[4];
    or_words(seed, 0, OR_STREAM_SEED, w);
    s0[0] = ((uint64_t)w[1] << 32) | w[0];
    s0[1] = ((uint64_t)w[3] << 32) | w[2];
}

/* Point n of the additive recurrence of Eq. 6 in 0.64 fixed point. */
void oracle_r2_point(const uint64_t s0[2], uint64_t n, uint64_t S[2])
{
    S[0] = s0[0] + n * OR_R2_ALPHA1;  /* mod 2^64 */
    S[1] = s0[1] + n * OR_R2_ALPHA2;
}

/* Fixed point -> [0,1) with 53 significant bits (exact in FP64). */
static double or_fix_to_unit(uint64_t S) { return (double)(S >> 11) * 0x1p-53; }

/* ------------------------------------------------------------------ PSD ---
 * von Karman phase PSD (first factor of Eq. 7):
 *   W(f) = c r0^(-5/3) (f^2 + L0^-2)^(-11/6),
 *   c = Gamma(11/6)^2 / (2 pi^(11/3)) * (24/5 Gamma(6/5))^(5/6) = 0.0228955871...
 * Kolmogorov: L0 -> infinity. */
#define OR_VK_C 0.022895587108555180776
enum { OR_PSD_VK = 0, OR_PSD_KOLMO = 1 };
double oracle_psd(int kind, double r0, double L0, double f2)
{
    double a = (kind == OR_PSD_KOLMO) ? 0.0 : 1.0 / (L0 * L0);
    return OR_VK_C * pow(r0, -5.0 / 3.0) * pow(f2 + a, -11.0 / 6.0);
}

/* ------------------------------------------------------- Eq. 7 filter ---
 * A(f) = 2 (D J1(pi D f) - d J1(pi d f)) / (pi (D^2 - d^2) f), A(0) = 1.
 * For pi D f < 1e-3 the Taylor series of J1 (x/2 - x^3/16 + x^5/384) is used
 * term by term, which removes the 0/0 at the origin. */
double oracle_airy(double f, double D, double d)
{
    if (f == 0.0) return 1.0;
    double xD = OR_PI * D * f;
    if (xD < 1e-3) {
        /* J1(x) = x/2 - x^3/16 + x^5/384 - ..., divided through by
         * pi (D^2 - d^2) f / 2:
         * A = 1 - (pi f)^2 (D^2 + d^2)/8 + (pi f)^4 (D^4 + D^2 d^2 + d^4)/192 */
        double u2 = (OR_PI * f) * (OR_PI * f);
        return 1.0 - u2 * (D * D + d * d) / 8.0
                   + u2 * u2 * (D * D * D * D + D * D * d * d + d * d * d * d) / 192.0;
    }
    double num = D * j1(xD) - ((d > 0.0) ? d * j1(OR_PI * d * f) : 0.0);
    return 2.0 * num / (OR_PI * (D * D - d * d) * f);
}

/* ------------------------------------------------------------- domains ---
 * Unit square -> frequency plane, with the Jacobian J of the map.
 *   SQUARE   (Eq. 5):      f = f_max (2 s - 1) per axis; J = (2 f_max)^2.
 *   DISC     (Sec. 3.2, Shirley-Chiu concentric square-to-disc map);
 *                          J = pi f_max^2 (the map preserves area ratios).
 *   LOGPOLAR (log-radial polar map over [f_min, f_max]):
 *                          rho = f_min (f_max/f_min)^s_x, theta = 2 pi s_y,
 *                          J = 2 pi ln(f_max/f_min) rho^2.
 * Returns the FP64 frequency; the caller rounds it to FP32. */
enum { OR_DOM_SQUARE = 0, OR_DOM_DISC = 1, OR_DOM_LOGPOLAR = 2 };
void oracle_domain_map(int kind, double fmin, double fmax, double sx, double sy, double f[2])
{
    if (kind == OR_DOM_SQUARE) {
        f[0] = fmax * (2.0 * sx - 1.0);
        f[1] = fmax * (2.0 * sy - 1.0);
    } else if (kind == OR_DOM_DISC) {
        double a = 2.0 * sx - 1.0, b = 2.0 * sy - 1.0, r, phi;
        if (a == 0.0 && b == 0.0) { f[0] = 0.0; f[1] = 0.0; return; }
        if (fabs(a) > fabs(b)) { r = a; phi = (OR_PI / 4.0) * (b / a); }
        else { r = b; phi = OR_PI / 2.0 - (OR_PI / 4.0) * (a / b); }
        f[0] = fmax * r * cos(phi);
        f[1] = fmax * r * sin(phi);
    } else {
        double L = log(fmax / fmin);
        double rho = fmin * exp(sx * L);
        double th = 2.0 * OR_PI * sy;
        f[0] = rho * cos(th);
        f[1] = rho * sin(th);
    }
}

/* Jacobian J of the map above, from the FP32-rounded frequency. */
double oracle_domain_jacobian(int kind, double fmin, double fmax, double fx, double fy)
{
    if (kind == OR_DOM_SQUARE) return 4.0 * fmax * fmax;
    if (kind == OR_DOM_DISC) return OR_PI * fmax * fmax;
    return 2.0 * OR_PI * log(fmax / fmin) * (fx * fx + fy * fy);
}

/* -------------------------------------------------------------- samplers --- */
enum { OR_SMP_R2 = 0, OR_SMP_JITTER = 1, OR_SMP_UNIFORM = 2, OR_SMP_IMPORTANCE = 3 };
enum { OR_COEF_GAUSS = 0, OR_COEF_EQ3 = 1 };

typedef struct {
    int psd_kind; double r0, L0;
    double ap_D, ap_d;  /* Eq. 7 aperture filter of the PSD (piston PSD); ap_D = 0: none */
    int dom_kind; double fmin, fmax;
    int smp_kind; uint64_t seed; int use_fixed_s0; uint64_t s0x, s0y;
    int coef_kind; int n_rho, n_theta;
    const uint32_t* cdf;  /* IMPORTANCE: n_rho*n_theta cell starts, cdf[0]=0, implicit end 2^32 */
    int fold;             /* IMPORTANCE: 0/1 cells over the whole turn; 2, 4: over one mirrored sector */
    double frame;         /* IMPORTANCE: angle of the cell frame, turns */
} or_params;

/* Box-Muller (1958) from two 24-bit uniforms:
 *   U1 = (hi24(u2) + 1) 2^-24 in (0,1], U2 = hi24(u3) 2^-24 in [0,1),
 *   a = sqrt(-2 ln U1) cos(2 pi U2), b = sqrt(-2 ln U1) sin(2 pi U2). */
static void or_box_muller(uint32_t u2, uint32_t u3, double* a, double* b)
{
    double U1 = (double)((u2 >> 8) + 1u) * 0x1p-24;
    double U2 = (double)(u3 >> 8) * 0x1p-24;
    double rad = sqrt(-2.0 * log(U1));
    *a = rad * cos(2.0 * OR_PI * U2);
    *b = rad * sin(2.0 * OR_PI * U2);
}

/* One term of the draw (Sec. 3 + Eq. 3, 5, 6, 7 of the paper).
 * Outputs: FP32 frequency, F = sqrt(W J / N_f) in FP64 from the FP32
 * frequency, coefficients (a, b), cell id, Philox words, R2 state. */
static void or_draw_term(const or_params* p, const uint64_t s0[2], int64_t n_f, uint64_t n, int64_t k,
                         float f32[2], double* F, double* Jo, double* ca, double* cb, int32_t* cell,
                         uint32_t w_out[4], uint64_t S_out[2])
{
    uint32_t w[4];
    or_words(p->seed, n, OR_STREAM_TERM, w);
    uint64_t S[2] = {0, 0};
    double sx, sy, J = 0.0, p_cell = 1.0;
    int32_t c = -1;
    double fd[2];
    if (p->smp_kind == OR_SMP_R2) {
        oracle_r2_point(s0, n, S);
        sx = or_fix_to_unit(S[0]);
        sy = or_fix_to_unit(S[1]);
    } else if (p->smp_kind == OR_SMP_UNIFORM) {
        S[0] = (uint64_t)w[0] << 32; S[1] = (uint64_t)w[1] << 32;
        sx = (double)w[0] * 0x1p-32;
        sy = (double)w[1] * 0x1p-32;
    } else if (p->smp_kind == OR_SMP_JITTER) {
        /* Eq. 4: cell (i, j) of an n_rho x n_theta grid on the unit square,
         * one uniformly jittered point per cell, N_f = n_rho * n_theta. */
        int64_t i = k % p->n_rho, j = k / p->n_rho;
        sx = ((double)i + (double)w[0] * 0x1p-32) / (double)p->n_rho;
        sy = ((double)j + (double)w[1] * 0x1p-32) / (double)p->n_theta;
    } else { /* IMPORTANCE: two-level integer inversion over log-polar cells */
        oracle_r2_point(s0, n, S);
        /* radial band from the marginal CDF with the x coordinate,
         * angular cell from that band's conditional CDF with the y coordinate.
         * Folded (F = 2^sh sectors of 1/F turn): the top sh bits of y name the
         * sector q, the remaining bits (complemented in odd sectors, which are
         * mirror images) are inverted by the same conditional CDF. */
        const int sh = (p->fold == 4) ? 2 : (p->fold == 2) ? 1 : 0;
        const uint64_t q = sh ? (S[1] >> (64 - sh)) : 0;
        uint64_t Y = S[1] << sh;
        if (q & 1) Y = ~Y;
        const uint32_t* cr = p->cdf;
        const uint32_t* ct;
        uint32_t ux = (uint32_t)(S[0] >> 32), uy = (uint32_t)(Y >> 32);
        int ir = 0, it = 0;
        for (int q = 1; q < p->n_rho; ++q)  /* plain linear scans */
            if (cr[q] <= ux) ir = q;
        ct = p->cdf + p->n_rho + (size_t)ir * p->n_theta;
        for (int q = 1; q < p->n_theta; ++q)
            if (ct[q] <= uy) it = q;
        uint64_t r_start = (uint64_t)cr[ir];
        uint64_t r_end = (ir + 1 < p->n_rho) ? (uint64_t)cr[ir + 1] : ((uint64_t)1 << 32);
        uint64_t t_start = (uint64_t)ct[it];
        uint64_t t_end = (it + 1 < p->n_theta) ? (uint64_t)ct[it + 1] : ((uint64_t)1 << 32);
        double tx = (double)(S[0] - (r_start << 32)) / ((double)(r_end - r_start) * 0x1p32);
        double ty = (double)(Y - (t_start << 32)) / ((double)(t_end - t_start) * 0x1p32);
        c = ir * p->n_theta + it;
        /* inside the cell, the log-polar map of the cell's own square */
        double L = log(p->fmax / p->fmin);
        double rho = p->fmin * exp(L * ((double)ir + tx) / (double)p->n_rho);
        double v = ((double)it + ty) / (double)p->n_theta;           /* place in the sector */
        double turn = (q & 1) ? ((double)q + 1.0 - v) : ((double)q + v);  /* sectors of the turn */
        double th = 2.0 * OR_PI * (p->frame + turn / (double)(1 << sh));
        fd[0] = rho * cos(th);
        fd[1] = rho * sin(th);
        p_cell = ((double)(r_end - r_start) * 0x1p-32) * ((double)(t_end - t_start) * 0x1p-32);
        sx = sy = 0.0;
    }
    if (p->smp_kind != OR_SMP_IMPORTANCE) {
        oracle_domain_map(p->dom_kind, p->fmin, p->fmax, sx, sy, fd);
        int ir = (int)floor(sx * (double)p->n_rho);
        int it = (int)floor(sy * (double)p->n_theta);
        if (ir > p->n_rho - 1) ir = p->n_rho - 1;
        if (it > p->n_theta - 1) it = p->n_theta - 1;
        c = ir * p->n_theta + it;
    }
    f32[0] = (float)fd[0];
    f32[1] = (float)fd[1];
    double fx = (double)f32[0], fy = (double)f32[1];
    if (p->smp_kind != OR_SMP_IMPORTANCE)
        J = oracle_domain_jacobian(p->dom_kind, p->fmin, p->fmax, fx, fy);
    else  /* the log-polar Jacobian 2 pi L rho^2, divided by n_rho n_theta p_c */
        J = 2.0 * OR_PI * log(p->fmax / p->fmin) * (fx * fx + fy * fy) / ((double)p->n_rho * (double)p->n_theta * p_cell);
    double W = oracle_psd(p->psd_kind, p->r0, p->L0, fx * fx + fy * fy);
    *F = sqrt(W * J / (double)n_f);
    /* Eq. 7: the piston PSD is W times the squared aperture filter; the
     * amplitude carries the signed filter, so that the sum at a point is the
     * piston of an aperture centred there (Sec. 4.1) */
    if (p->ap_D > 0.0) *F *= oracle_airy(sqrt(fx * fx + fy * fy), p->ap_D, p->ap_d);
    *Jo = J;
    double a, b;
    or_box_muller(w[2], w[3], &a, &b);
    if (p->coef_kind == OR_COEF_EQ3) {
        uint32_t v[4];
        or_words(p->seed, n, OR_STREAM_EQ3, v);
        double Ru = (double)(v[0] >> 8) * 0x1p-24;
        double Rn = a;
        a = sqrt(2.0) * Rn * cos(2.0 * OR_PI * Ru);
        b = sqrt(2.0) * Rn * sin(2.0 * OR_PI * Ru);
    }
    *ca = a; *cb = b; *cell = c;
    if (w_out) memcpy(w_out, w, sizeof(w));
    if (S_out) { S_out[0] = S[0]; S_out[1] = S[1]; }
}

static or_params or_pack(int psd_kind, double r0, double L0, double ap_D, double ap_d, int dom_kind,
                         double fmin, double fmax,
                         int smp_kind, uint64_t seed, int use_fixed_s0, uint64_t s0x, uint64_t s0y,
                         int coef_kind, int n_rho, int n_theta, const uint32_t* cdf, int fold, double frame)
{
    or_params p;
    p.psd_kind = psd_kind; p.r0 = r0; p.L0 = L0; p.ap_D = ap_D; p.ap_d = ap_d;
    p.dom_kind = dom_kind; p.fmin = fmin; p.fmax = fmax;
    p.smp_kind = smp_kind; p.seed = seed; p.use_fixed_s0 = use_fixed_s0; p.s0x = s0x; p.s0y = s0y;
    p.coef_kind = coef_kind; p.n_rho = n_rho; p.n_theta = n_theta; p.cdf = cdf;
    p.fold = fold; p.frame = frame;
    return p;
}

#define OR_PARAMS_DECL int psd_kind, double r0, double L0, double psd_apD, double psd_apd, int dom_kind, \
    double fmin, double fmax, \
    int smp_kind, uint64_t seed, int use_fixed_s0, uint64_t s0x, uint64_t s0y, int coef_kind, \
    int n_rho, int n_theta, const uint32_t* cdf, int fold, double frame
#define OR_PARAMS_PASS psd_kind, r0, L0, psd_apD, psd_apd, dom_kind, fmin, fmax, smp_kind, seed, use_fixed_s0, s0x, \
    s0y, \
    coef_kind, n_rho, n_theta, cdf, fold, frame

/* The draw of n_real realisations of n_f terms.  Any output may be NULL.
 *   f_xy [n_real][n_f][2] float, F [n_real][n_f], J [n_real][n_f] (the
 *   cell-area factor of the weight), coef [n_real][n_f][2], cell [n_real][n_f],
 *   words [n_real][n_f][4], r2 [n_real][n_f][2]. */
int oracle_draw(OR_PARAMS_DECL, int64_t n_f, int64_t n_real, int64_t real_offset,
                float* f_xy, double* F, double* Jout, double* coef, int32_t* cell, uint32_t* words,
                uint64_t* r2)
{
    or_params p = or_pack(OR_PARAMS_PASS);
    uint64_t s0[2];
    oracle_r2_seed(seed, use_fixed_s0, s0x, s0y, s0);
    for (int64_t r = 0; r < n_real; ++r)
        for (int64_t k = 0; k < n_f; ++k) {
            uint64_t n = (uint64_t)(real_offset + r) * (uint64_t)n_f + (uint64_t)k;
            int64_t i = r * n_f + k;
            float f32[2]; double Fk, Jk, a, b; int32_t c; uint32_t w[4]; uint64_t S[2];
            or_draw_term(&p, s0, n_f, n, k, f32, &Fk, &Jk, &a, &b, &c, w, S);
            if (f_xy) { f_xy[2 * i] = f32[0]; f_xy[2 * i + 1] = f32[1]; }
            if (F) F[i] = Fk;
            if (Jout) Jout[i] = Jk;
            if (coef) { coef[2 * i] = a; coef[2 * i + 1] = b; }
            if (cell) cell[i] = c;
            if (words) memcpy(words + 4 * i, w, sizeof(w));
            if (r2) { r2[2 * i] = S[0]; r2[2 * i + 1] = S[1]; }
        }
    return 0;
}

/* ------------------------------------------------------------- Eq. 3 sum ---
 * chi(x_m) = sum_k F_k (a_k cos 2 pi phi_mk - b_k sin 2 pi phi_mk),
 * phi_mk = fx_k x_m + fy_k y_m formed in FP64 (each FP32 x FP32 product is
 * exact in FP64), reduced by phi - rint(phi).  Explicit terms in, so tests can
 * feed frequencies chosen by hand (an FFT grid, a single term). */
int oracle_synth_terms(const float* f_xy, const double* F, const double* coef, int64_t n_terms,
                       const float* xy, int64_t n_points, double* out)
{
    for (int64_t m = 0; m < n_points; ++m) {
        double x = (double)xy[2 * m], y = (double)xy[2 * m + 1];
        double acc = 0.0;
        for (int64_t k = 0; k < n_terms; ++k) {
            double phi = (double)f_xy[2 * k] * x + (double)f_xy[2 * k + 1] * y;
            phi = phi - rint(phi);
            acc += F[k] * (coef[2 * k] * cos(2.0 * OR_PI * phi) - coef[2 * k + 1] * sin(2.0 * OR_PI * phi));
        }
        out[m] = acc;
    }
    return 0;
}

/* Draw + Eq. 3 at arbitrary points: out [n_real][n_points]. */
int oracle_synthesize(OR_PARAMS_DECL, int64_t n_f, int64_t n_real, int64_t real_offset,
                      const float* xy, int64_t n_points, double* out)
{
    float* f = (float*)malloc(sizeof(float) * 2 * n_f);
    double* F = (double*)malloc(sizeof(double) * n_f);
    double* c = (double*)malloc(sizeof(double) * 2 * n_f);
    if (!f || !F || !c) { free(f); free(F); free(c); return -5; }
    for (int64_t r = 0; r < n_real; ++r) {
        oracle_draw(OR_PARAMS_PASS, n_f, 1, real_offset + r, f, F, NULL, c, NULL, NULL, NULL);
        oracle_synth_terms(f, F, c, n_f, xy, n_points, out + r * n_points);
    }
    free(f); free(F); free(c);
    return 0;
}

/* Shared-draw form: one frequency draw (that of realisation real_offset)
 * for all n_real columns; column r takes its coefficients from stream point
 * (real_offset + r) N_f + k, and optionally its own (r0, L0) for the weight.
 * col_psd: NULL or [n_real][2] (r0, L0).  out [n_real][n_points]. */
int oracle_synthesize_shared(OR_PARAMS_DECL, int64_t n_f, int64_t n_real, int64_t real_offset,
                             const double* col_psd, const float* xy, int64_t n_points, double* out)
{
    float* f = (float*)malloc(sizeof(float) * 2 * n_f);
    double* J = (double*)malloc(sizeof(double) * n_f);
    float* fr = (float*)malloc(sizeof(float) * 2 * n_f);
    double* Fr = (double*)malloc(sizeof(double) * n_f);
    double* cr = (double*)malloc(sizeof(double) * 2 * n_f);
    if (!f || !J || !fr || !Fr || !cr) { free(f); free(J); free(fr); free(Fr); free(cr); return -5; }
    /* the shared frequencies and their cell factors J: realisation real_offset */
    oracle_draw(OR_PARAMS_PASS, n_f, 1, real_offset, f, NULL, J, NULL, NULL, NULL, NULL);
    for (int64_t r = 0; r < n_real; ++r) {
        /* coefficients of column r come from its own stream points */
        oracle_draw(OR_PARAMS_PASS, n_f, 1, real_offset + r, fr, NULL, NULL, cr, NULL, NULL, NULL);
        double cr0 = col_psd ? col_psd[2 * r] : r0;
        double cL0 = col_psd ? col_psd[2 * r + 1] : L0;
        for (int64_t k = 0; k < n_f; ++k) {
            double fx = (double)f[2 * k], fy = (double)f[2 * k + 1];
            double W = oracle_psd(psd_kind, cr0, cL0, fx * fx + fy * fy);
            Fr[k] = sqrt(W * J[k] / (double)n_f);
            if (psd_apD > 0.0) Fr[k] *= oracle_airy(sqrt(fx * fx + fy * fy), psd_apD, psd_apd);
        }
        oracle_synth_terms(f, Fr, cr, n_f, xy, n_points, out + r * n_points);
    }
    free(f); free(J); free(fr); free(Fr); free(cr);
    return 0;
}

/* ------------------------------------------------------------- pistons ---
 * Piston of aperture a (centre p_a, diameter D_a, obstruction d_a):
 *   piston_r(a) = sum_k F_k A_a(|f_k|) (a_k cos 2 pi f_k.p_a - b_k sin 2 pi f_k.p_a)
 * i.e. Eq. 3 evaluated at the aperture centre with the piston PSD W A^2 of
 * Eq. 7.  Pair differences (Sec. 4.4): delta_r(i,j) = piston(i) - piston(j).
 * piston [n_real][n_ap] (may be NULL), out [n_real][n_pairs] (may be NULL). */
int oracle_diff_piston(OR_PARAMS_DECL, int64_t n_f, int64_t n_real, int64_t real_offset,
                       const float* ap_xy, const float* ap_D, const float* ap_d, int n_ap,
                       const int32_t* pairs, int n_pairs, double* piston, double* out)
{
    if (psd_apD > 0.0) return -2;  /* the apertures filter here: a filtered PSD would filter twice */
    float* f = (float*)malloc(sizeof(float) * 2 * n_f);
    double* F = (double*)malloc(sizeof(double) * n_f);
    double* c = (double*)malloc(sizeof(double) * 2 * n_f);
    double* pis = (double*)malloc(sizeof(double) * (n_ap > 0 ? n_ap : 1));
    if (!f || !F || !c || !pis) { free(f); free(F); free(c); free(pis); return -5; }
    for (int64_t r = 0; r < n_real; ++r) {
        oracle_draw(OR_PARAMS_PASS, n_f, 1, real_offset + r, f, F, NULL, c, NULL, NULL, NULL);
        for (int a = 0; a < n_ap; ++a) {
            double x = (double)ap_xy[2 * a], y = (double)ap_xy[2 * a + 1];
            double acc = 0.0;
            for (int64_t k = 0; k < n_f; ++k) {
                double fx = (double)f[2 * k], fy = (double)f[2 * k + 1];
                double A = oracle_airy(sqrt(fx * fx + fy * fy), (double)ap_D[a], (double)ap_d[a]);
                double phi = fx * x + fy * y;
                phi = phi - rint(phi);
                acc += F[k] * A * (c[2 * k] * cos(2.0 * OR_PI * phi) - c[2 * k + 1] * sin(2.0 * OR_PI * phi));
            }
            pis[a] = acc;
            if (piston) piston[r * n_ap + a] = acc;
        }
        if (out)
            for (int q = 0; q < n_pairs; ++q)
                out[r * n_pairs + q] = pis[pairs[2 * q]] - pis[pairs[2 * q + 1]];
    }
    free(f); free(F); free(c); free(pis);
    return 0;
}

/* ------------------------------------------------------ structure function ---
 * For each series s and lag L (Sec. 4.4):
 *   L >= 1: x = v[t+L] - v[t], t in [0, T-L);  L = 0: x = v[t], t in [0, T)
 * acc[s][l] += (sum x^2, sum x^4, count), summed over realisations and t in
 * FP64 (plain running sums).  delta [n_real][n_series][T] FP32. */
int oracle_structure_fn(const float* delta, int64_t n_real, int64_t n_series, int64_t T,
                        const int32_t* lags, int n_lags, double* acc)
{
    for (int64_t s = 0; s < n_series; ++s)
        for (int l = 0; l < n_lags; ++l) {
            int64_t L = lags[l];
            double s2 = 0.0, s4 = 0.0, cnt = 0.0;
            for (int64_t r = 0; r < n_real; ++r) {
                const float* v = delta + (r * n_series + s) * T;
                if (L == 0) {
                    for (int64_t t = 0; t < T; ++t) {
                        double x = (double)v[t];
                        s2 += x * x; s4 += x * x * x * x; cnt += 1.0;
                    }
                } else {
                    for (int64_t t = 0; t + L < T; ++t) {
                        double x = (double)v[t + L] - (double)v[t];
                        s2 += x * x; s4 += x * x * x * x; cnt += 1.0;
                    }
                }
            }
            double* o = acc + (s * n_lags + l) * 3;
            o[0] += s2; o[1] += s4; o[2] += cnt;
        }
    return 0;
}

/* ------------------------------------------------ normals for MLP init ---
 * out[i] = N(0,1) by Box-Muller from the Philox words of counter
 * (i_lo, i_hi, stream, 0) and key seed: U1 = (hi24(w0) + 1) 2^-24,
 * U2 = hi24(w1) 2^-24, out = sqrt(-2 ln U1) cos(2 pi U2). */
int oracle_normals(uint64_t seed, uint32_t stream, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        or_words(seed, (uint64_t)i, stream, w);
        double U1 = (double)((w[0] >> 8) + 1u) * 0x1p-24;
        double U2 = (double)(w[1] >> 8) * 0x1p-24;
        out[i] = sqrt(-2.0 * log(U1)) * cos(2.0 * OR_PI * U2);
    }
    return 0;
}

/* ------------------------------------------------- sampling statistics ---
 * Clusters and gaps of a frequency draw (Sec. 2.3, 3.2, Figs. 2-3): per set of
 * n points, the distance from each point to its nearest other point
 * (Euclidean, FP64 from the FP32 coordinates, brute force; 0 for n = 1), and
 * the star discrepancy of points in [0,1]^2,
 *   D* = sup over boxes B = [0,u) x [0,v) of | #(points in B) / n - u v |,
 * written out from its definition: the supremum is approached at corners
 * u in {x_i} U {1}, v in {y_j} U {1}, from above (closed box, count with <=,
 * |C/n - uv| with C the closed count) and from below (open box, count with
 * <, |uv - O/n|).  Both counts are integers and u v is one FP64 product of
 * FP32 values. */
int oracle_nearest_neighbour(const float* pts, int64_t n_sets, int64_t n, double* out)
{
    for (int64_t s = 0; s < n_sets; ++s) {
        const float* p = pts + s * n * 2;
        for (int64_t i = 0; i < n; ++i) {
            double best = -1.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double dx = (double)p[2 * j] - (double)p[2 * i];
                double dy = (double)p[2 * j + 1] - (double)p[2 * i + 1];
                double d = sqrt(dx * dx + dy * dy);
                if (best < 0.0 || d < best) best = d;
            }
            out[s * n + i] = best < 0.0 ? 0.0 : best;
        }
    }
    return 0;
}

int oracle_star_discrepancy(const float* pts, int64_t n_sets, int64_t n, double* out)
{
    for (int64_t s = 0; s < n_sets; ++s) {
        const float* p = pts + s * n * 2;
        double D = 0.0;
        for (int64_t i = 0; i <= n; ++i) {
            double u = (i < n) ? (double)p[2 * i] : 1.0;
            for (int64_t j = 0; j <= n; ++j) {
                double v = (j < n) ? (double)p[2 * j + 1] : 1.0;
                int64_t closed = 0, open = 0;
                for (int64_t k = 0; k < n; ++k) {
                    double x = (double)p[2 * k], y = (double)p[2 * k + 1];
                    if (x <= u && y <= v) ++closed;
                    if (x < u && y < v) ++open;
                }
                double uv = u * v;
                double a = (double)closed / (double)n - uv;
                double b = uv - (double)open / (double)n;
                if (a > D) D = a;
                if (b > D) D = b;
            }
        }
        out[s] = D;
    }
    return 0;
}

/* ------------------------------------------------- FFT screen (Eq. 2) ---
 * The comparison method of Sec. 2.2: frequencies on the FFT grid of an n x n
 * screen of pitch dx, f = (j', i') df with df = 1 / (n dx) and the signed
 * index j' = j for j < (n + 1) / 2, j - n otherwise (the order of an FFT);
 * the spectrum of realisation r is
 *   S[r][i][j] = (a + i b) sqrt(W(f)) A(|f|) df,
 * a, b ~ N(0,1) by Box-Muller from words 2 and 3 of counter
 * ((real_offset + r) n^2 + i n + j, stream 4), A the Eq. 7 filter when
 * ap_D > 0 (else 1), and S = 0 at f = 0 (the screen's mean, which no
 * structure function sees).  The screen is n^2 times the inverse DFT of S
 * (taken with numpy in oracle/__init__.py): sum_f S e^{2 pi i f.x}, whose
 * real and imaginary parts are two screens.  spec [n_real][n][n][2]. */
#define OR_STREAM_FFT 4u
int oracle_fft_spectrum(int psd_kind, double r0, double L0, double ap_D, double ap_d, int64_t n, double dx,
                        uint64_t seed, int64_t n_real, int64_t real_offset, double* spec)
{
    const double df = 1.0 / ((double)n * dx);
    const int64_t half = (n + 1) / 2;
    for (int64_t r = 0; r < n_real; ++r)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double* s = spec + 2 * ((r * n + i) * n + j);
                if (i == 0 && j == 0) { s[0] = 0.0; s[1] = 0.0; continue; }
                const uint64_t idx = (uint64_t)(real_offset + r) * (uint64_t)(n * n) + (uint64_t)(i * n + j);
                uint32_t w[4];
                or_words(seed, idx, OR_STREAM_FFT, w);
                double a, b;
                or_box_muller(w[2], w[3], &a, &b);
                const double fx = (double)(j < half ? j : j - n) * df;
                const double fy = (double)(i < half ? i : i - n) * df;
                const double f2 = fx * fx + fy * fy;
                double F = sqrt(oracle_psd(psd_kind, r0, L0, f2)) * df;
                if (ap_D > 0.0) F *= oracle_airy(sqrt(f2), ap_D, ap_d);
                s[0] = a * F;
                s[1] = b * F;
            }
    return 0;
}
