/*
 * qrs.h -- C ABI of libqrs, quasi-random frequency-sampling synthesis of
 * optical-turbulence fields on one GB300 (sm_103a).
 *
 * Method: Berdja, Hadjara, Carbillet, Bernardi, Petrov, "Quasi-Random
 * Frequency Sampling for Optical Turbulence Simulations" (arXiv 2404.02978).
 * A realisation of a field with phase PSD W is the direct sum of Eq. 3,
 *     chi(x) = sum_k F_k (a_k cos 2 pi f_k.x - b_k sin 2 pi f_k.x),
 * F_k = sqrt(W(f_k) J_k / N_f), over N_f frequencies f_k placed by the R2
 * low-discrepancy sequence of Eq. 6 (mapped by Eq. 5 to a square, by the
 * square-to-disc map of Sec. 3.2 to a disc, or log-radially to an annulus),
 * the sequence continuing across realisations (Sec. 3.2).  Pistons filter the
 * PSD by the aperture factor of Eq. 7 (Sec. 4.1); their pair differences and
 * structure functions are the statistics of Sec. 4.4.
 *
 * Conventions shared by every entry point
 *   - Array arguments are DEVICE pointers on the handle's device unless the
 *     comment says "host".  The caller owns them; the library never frees or
 *     retains them after the call returns.  Parameter structs are host memory,
 *     read during the call only.
 *   - Layouts are C order (last index fastest), FP32 unless stated.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and the call returns without synchronising.  Argument errors are
 *     detected on the host before anything is enqueued and return a negative
 *     qrs_status with nothing launched; qrs_last_error() gives the reason.
 *   - Errors detected on the device (a bounded wait that ran out, a caller
 *     index out of range) set a device error word that qrs_sync() reports and
 *     clears.  The library never aborts, traps or prints.
 *   - Results are a pure function of the inputs, the seed and real_offset:
 *     one call over realisations [0, R) equals two calls over [0, R1) and
 *     [R1, R) with real_offset 0 and R1 (checkpoint / resume by counter).
 *   - Not thread-safe per handle: one host thread drives one handle.  The
 *     handle's device workspaces (shared-draw coefficients, grid draw records
 *     and accumulators, piston job tables) serve one call at a time: calls on
 *     one handle must not run concurrently on the GPU (issue them on one
 *     stream, or use one handle per stream).
 *   - Environment: QRS_AUTOTUNE_CACHE (a file of the piston kernel-shape
 *     choices, read and written by the autotuner), QRS_FAULT (read at
 *     qrs_create; "alloc", "launch", "timeout", comma-separated: host-side
 *     fault injection -- workspace allocations fail with QRS_ERR_NOMEM,
 *     compute calls fail with QRS_ERR_CUDA before launching anything; the
 *     next GEMM-form launch of the handle first waits on a barrier that no
 *     thread arrives at, with a limit of about 1 ms, and unwinds through its
 *     time-out path: QRS_ERR_TIMEOUT at the next qrs_sync, later calls run
 *     normally), QRS_GRID_PAIR=0 and QRS_GEMM_PAIR=0 (read at qrs_create:
 *     the grid form and the split-precision GEMM form then run every
 *     128-point tile on its own CTA instead of on pairs of CTAs sharing one
 *     tensor-core product across two SMs; results are identical),
 *     QRS_SYNTH_ANCHOR=0 (read at qrs_create, and by
 *     qrs_synthesize_points_noalloc at each call: the fused form keeps its
 *     exact per-point phase paths instead of the anchored one, see
 *     qrs_synthesize_points; results agree within the stated tolerance),
 *     QRS_CHECKED=1 (read by the Python binding: it loads the bounds-checked
 *     build, see below).
 */
#ifndef QRS_H
#define QRS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QRS_OK = 0,
    QRS_ERR_ARG = -1,          /* invalid argument (size, pointer, enum, alignment) */
    QRS_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    QRS_ERR_TIMEOUT = -3,      /* a bounded device wait ran out (device error word) */
    QRS_ERR_UNSUPPORTED = -4,  /* valid request this build does not provide */
    QRS_ERR_NOMEM = -5,        /* workspace allocation failed */
    QRS_ERR_DEVICE_CHECK = -6  /* a device-side check failed (device error word) */
} qrs_status;

/* PSD of the phase (Eq. 7, first factor): W(f) = c r0^(-5/3) (f^2 + L0^-2)^(-11/6),
 * c = Gamma(11/6)^2/(2 pi^(11/3)) (24/5 Gamma(6/5))^(5/6) = 0.0228955871...
 * (the paper prints its truncation 0.02289).  KOLMOGOROV drops L0^-2. */
#define QRS_PSD_VON_KARMAN 0
#define QRS_PSD_KOLMOGOROV 1

/* Frequency domains (unit square [0,1)^2 -> frequency plane, cycles/m):
 *   SQUARE   f = fmax (2 s - 1) per axis, the map of Eq. 5 with
 *            delta_f N = 2 max f; cell factor J = (2 fmax)^2.
 *   DISC     Shirley-Chiu concentric square-to-disc map of radius fmax
 *            (Sec. 3.2 remark); J = pi fmax^2.
 *   LOGPOLAR rho = fmin (fmax/fmin)^s_x, theta = 2 pi s_y; J = 2 pi ln(fmax/fmin) rho^2.
 * The weight of a term is w = W(f) J / N_f (Eq. 3's delta_fx delta_fy for a
 * cell of the square), F = sqrt(w). */
#define QRS_DOMAIN_SQUARE 0
#define QRS_DOMAIN_DISC 1
#define QRS_DOMAIN_LOGPOLAR 2

/* Placement of the N_f terms of a realisation:
 *   R2         the R2 sequence of Eq. 6 in exact 0.64 fixed point, point
 *              n = (real_offset + r) N_f + k of one stream (Sec. 3.2: never
 *              re-initialised); seed s0 = Philox(seed) or the fixed s0 given.
 *   JITTER     Eq. 4: one uniformly jittered point per cell of an
 *              n_rho x n_theta grid on the unit square (N_f = n_rho n_theta).
 *   UNIFORM    independent uniform points (Sec. 2.3 "fully random").
 *   IMPORTANCE cells of an n_rho (log-radial) x n_theta (angular) grid over
 *              [fmin, fmax] by two-level inversion of the R2 point: the radial
 *              band from the marginal CDF with the x coordinate's top 32 bits,
 *              the angular cell from that band's conditional CDF with the y
 *              coordinate's top 32 bits (so the point keeps its 2-D
 *              stratification); the remainders (t_x, t_y) place it by the
 *              cell's log-polar map, rho = fmin (fmax/fmin)^((i_rho + t_x)/n_rho),
 *              theta = 2 pi (i_theta + t_y)/n_theta; J = 2 pi ln(fmax/fmin)
 *              rho^2 / (n_rho n_theta p_c), p_c = p_band p_cell|band, which
 *              keeps the sum unbiased (learned proposal; uniform CDFs give the
 *              plain log-polar weights).  Domain must be LOGPOLAR. */
#define QRS_SAMPLER_R2 0
#define QRS_SAMPLER_JITTER 1
#define QRS_SAMPLER_UNIFORM 2
#define QRS_SAMPLER_IMPORTANCE 3

/* Coefficients of Eq. 3 (from Philox4x32-10 words, counter (n, stream)):
 *   GAUSS  a, b ~ N(0,1) i.i.d. by Box-Muller from 24-bit uniforms
 *          U1 = (w2>>8 + 1) 2^-24, U2 = (w3>>8) 2^-24.
 *   EQ3    the paper's literal sqrt(2) R_n cos(2 pi (f.x + R_u)):
 *          a = sqrt2 R_n cos 2 pi R_u, b = sqrt2 R_n sin 2 pi R_u,
 *          R_n the GAUSS a, R_u = (v0>>8) 2^-24 from stream 2.
 * Both give every term variance F^2 (Eq. 3's 2/sqrt(2) factor). */
#define QRS_COEF_GAUSS 0
#define QRS_COEF_EQ3 1

/* Aperture filter (Eq. 7): with ap_D_m > 0 the PSD is W(f) A(|f|)^2, the
 * piston PSD of a circular aperture of diameter ap_D_m with a central
 * obstruction of diameter ap_d_m, A(f) = 2 (D J1(pi D f) - d J1(pi d f)) /
 * (pi (D^2 - d^2) f), A(0) = 1; every term's amplitude carries the signed A,
 * so the Eq. 3 sum at a point is the piston of such an aperture centred there
 * (Sec. 4.1: pistons simulated at arbitrary positions, e.g. a telescope's
 * track through a frozen-flow layer).  ap_D_m = 0: no filter (ap_d_m = 0).
 * 0 <= ap_d_m < ap_D_m.  qrs_diff_piston jobs and qrs_proposal_targets filter
 * per aperture themselves and take ap_D_m = 0. */
typedef struct qrs_psd {
    double r0_m;   /* Fried parameter at the simulated wavelength, m (> 0) */
    double L0_m;   /* outer scale, m (> 0; ignored for KOLMOGOROV) */
    int32_t kind;  /* QRS_PSD_* */
    int32_t reserved;
    double ap_D_m; /* aperture filter diameter, m (0: none) */
    double ap_d_m; /* its central obstruction diameter, m */
} qrs_psd;

typedef struct qrs_domain {
    double fmin;   /* cycles/m; LOGPOLAR only (> 0) */
    double fmax;   /* cycles/m (> 0) */
    int32_t kind;  /* QRS_DOMAIN_* */
    int32_t reserved;
} qrs_domain;

typedef struct qrs_sampler {
    uint64_t seed;             /* Philox key (low word, high word) */
    uint64_t s0[2];            /* fixed R2 seed in 0.64 fixed point, if use_fixed_s0 */
    const uint32_t* cell_cdf;  /* device uint32 [n_rho + n_rho*n_theta]: the marginal CDF
                                  over radial bands (start points, [0] = 0, strictly
                                  increasing, implicit end 2^32), then for each band
                                  the conditional CDF over its angular cells (same
                                  form).  IMPORTANCE only, else NULL. */
    int32_t kind;              /* QRS_SAMPLER_* */
    int32_t coef_kind;         /* QRS_COEF_* */
    int32_t use_fixed_s0;      /* 0: s0 = Philox(key=seed, ctr=(0,0,1,0)); 1: s0 above */
    int32_t n_rho;             /* cell grid (cell ids, JITTER grid, IMPORTANCE cells) >= 1 */
    int32_t n_theta;           /* >= 1 */
    int32_t fold;              /* IMPORTANCE only (else 0 or 1): 0 or 1, the angular
                                  cells cover the whole turn; 2 or 4, they cover one
                                  sector of 1/fold turn, repeated over the fold
                                  sectors with every other sector mirrored (the top
                                  log2(fold) bits of the R2 y coordinate pick the
                                  sector, the rest, complemented in odd sectors, is
                                  inverted by the band's conditional CDF).  The density
                                  still covers the whole annulus and the weights stay
                                  unbiased; it suits integrands that depend on the
                                  angle only through |cos(angle - frame)|, such as
                                  the structure function at a baseline along frame. */
    double frame;              /* IMPORTANCE only (else 0): angle of the cells' frame
                                  in turns (cell angles are frame + turn, the turn
                                  made of sectors as above); finite */
} qrs_sampler;

typedef struct qrs_handle qrs_handle;

/* Create a handle on CUDA device `device` (makes it current for the calling
 * thread).  The handle owns small device workspaces (error word, launch
 * descriptors) and its autotune cache.  *h = NULL on failure. */
qrs_status qrs_create(qrs_handle** h, int32_t device);
void qrs_destroy(qrs_handle* h);
/* Last error message of this handle ("" if none); valid until the next call. */
const char* qrs_last_error(const qrs_handle* h);
/* Synchronise `stream`, then read and clear the device error word:
 * QRS_OK, QRS_ERR_TIMEOUT or QRS_ERR_DEVICE_CHECK. */
qrs_status qrs_sync(qrs_handle* h, void* stream);
/* Number of kernel launches this handle has enqueued since creation. */
int64_t qrs_launch_count(const qrs_handle* h);

/* --------------------------------------------------- bounds-checked build ---
 * libqrs_checked.so is the same library compiled with QRS_CHECKED=1: in its
 * kernels the computed index of every global- and shared-memory access the
 * kernels make through their checked accessors (inputs, outputs, draw
 * records, shared-memory term tables and operand tiles, bulk copies) is
 * tested against the extent of its buffer before use.  An index out of range
 * is not used (the access goes to a scratch sink) and QRS_ERR_DEVICE_CHECK
 * is recorded in the device error word of the handle created last, reported
 * by qrs_sync.  It is slower; results of valid calls are those of the
 * default build.
 * qrs_checked_build: 1 in the checked library, 0 in libqrs.so.
 * qrs_check_selftest: checked library only (QRS_ERR_ARG in the default build,
 * nothing launched): one thread stores through the checked accessor into an
 * 8-float scratch of the handle at index i; i outside [0, 8) must record
 * QRS_ERR_DEVICE_CHECK (seen at the next qrs_sync) and leave the scratch
 * untouched -- a test of the checking machinery, not of a kernel. */
int32_t qrs_checked_build(void);
qrs_status qrs_check_selftest(qrs_handle* h, int64_t i, void* stream);

/* ---------------------------------------------------------------- draw ---
 * The frequency draw of n_real realisations x n_f terms (Eq. 3 weights, Eq. 5/6
 * placement, Sec. 3.2 continuation), realisations real_offset .. +n_real-1.
 * Every output may be NULL; sizes in elements:
 *   f_xy  [n_real][n_f][2]  FP32 frequency (cycles/m), the round-to-nearest of
 *                           the FP64 map (within 1 ulp where FP64 exp/sin differ)
 *   amp   [n_real][n_f]     F_k = sqrt(W(f_k) J_k / N_f), FP32
 *   coef  [n_real][n_f][2]  (a_k, b_k), FP32
 *   cell  [n_real][n_f]     cell id i_rho n_theta + i_theta (exact)
 *   words [n_real][n_f][4]  Philox4x32-10 words of counter (n, 0) (exact)
 *   r2    [n_real][n_f][2]  R2 state in 0.64 fixed point (exact; 0 if not R2/IMPORTANCE)
 * n_f in [1, 2^31), n_real >= 0 (0 is a no-op), real_offset >= 0. */
typedef struct qrs_draw_out {
    float* f_xy;
    float* amp;
    float* coef;
    int32_t* cell;
    uint32_t* words;
    uint64_t* r2;
} qrs_draw_out;

qrs_status qrs_draw(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                    int64_t n_f, int64_t n_real, int64_t real_offset, const qrs_draw_out* out,
                    void* stream);

/* ---------------------------------------------------------- synthesis ---
 * Eq. 3 at arbitrary points (Sec. 3: "simulate at specific areas of
 * interest"): out[r][m] = sum_k F_k (a_k cos 2 pi phi_mk - b_k sin 2 pi phi_mk),
 * phi_mk = f_k . x_m reduced mod 1 exactly (64-bit fixed point when
 * f_max max|x| <= 128, else double-float error-free products), FP32
 * accumulation.
 *   xy   [n_points][2]  FP32 point coordinates, m
 *   out  [n_real][n_points]  FP32
 * mode:
 *   QRS_SYNTH_FUSED       per-realisation draw (realisation r uses stream points
 *                         (real_offset + r) N_f + k), draw and accumulate fused
 *                         in one persistent kernel, each term as one cosine in
 *                         Eq. 3's amplitude-phase form F amp cos 2 pi (phi + psi)
 *                         (amp, psi: the polar form of (a, b)); col_psd must be
 *                         NULL.  Where each group of 16 consecutive points lies
 *                         within d of the group's first or last point with
 *                         f_max d <= 8, the exact phase is formed at those
 *                         two anchors
 *                         only and each point adds its FP32 offset
 *                         2 pi f . (x_m - x_anchor) (the anchored path; within
 *                         1e-5 of the field standard deviation per value, as
 *                         the exact paths); QRS_SYNTH_ANCHOR=0 turns it off.
 *   QRS_SYNTH_GEMM_*      shared draw: all n_real columns use the frequencies of
 *                         realisation real_offset; column r takes its coefficients
 *                         from stream points (real_offset + r) N_f + k and, if
 *                         col_psd != NULL, its own (r0, L0) = col_psd[r][0..1]
 *                         (device FP64 [n_real][2]) in the weight.  The sum is the
 *                         product of the [n_points x 2 n_f] cos/sin basis and the
 *                         [2 n_f x n_real] coefficient matrix on the tensor cores:
 *                         3XTF32 (split TF32, ~FP32 accuracy: within 1e-5 of the
 *                         column's field standard deviation per value), BF16X3
 *                         (split BF16, ~2^-17 per product: within 5e-5), or
 *                         TF32 (single pass, each operand rounded once to TF32,
 *                         ~2^-11 per product: within 2e-3, about 3e-4 rms).
 * Column 0 of a GEMM-mode call equals realisation real_offset of a FUSED call. */
#define QRS_SYNTH_FUSED 0
#define QRS_SYNTH_GEMM_3XTF32 1
#define QRS_SYNTH_GEMM_BF16X3 2
#define QRS_SYNTH_GEMM_TF32 3

qrs_status qrs_synthesize_points(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom,
                                 const qrs_sampler* smp, int64_t n_f, int64_t n_real,
                                 int64_t real_offset, const float* xy, int64_t n_points,
                                 int32_t mode, const double* col_psd, float* out, void* stream);

/* ------------------------------------------------ synthesis on a grid ---
 * Eq. 3 on a tensor-product point set {x_i} x {y_j} (a pupil sampled on a
 * grid, Sec. 3 and 4): the same field as qrs_synthesize_points in FUSED mode
 * at the points (x_i, y_j) -- realisation r uses stream points
 * (real_offset + r) N_f + k -- computed through the factorisation
 * e^{i 2 pi f.x} = e^{i 2 pi fx x} e^{i 2 pi fy y} as one matrix product per
 * realisation on the tensor cores (cos/sin of fx x_i against the
 * coefficient-weighted cos/sin of fy y_j; (n_x + n_y) N_f sin/cos pairs per
 * realisation instead of n_x n_y N_f).  The paper has no such form: it is the
 * Eq. 3 sum regrouped, exact up to rounding.
 *   x [nx], y [ny]   FP32 coordinates, m (any values; a uniform grid is not needed)
 *   index            NULL: out [n_real][ny][nx] (x fastest);
 *                    else int32 [ny][nx]: node (i, j) goes to out[r][index[j][i]]
 *                    when index[j][i] >= 0 (each point at most once), out
 *                    [n_real][n_points] -- e.g. the interior of a pupil; an
 *                    index >= n_points is not written and records
 *                    QRS_ERR_DEVICE_CHECK in the device error word.
 *   mode             QRS_SYNTH_GEMM_3XTF32 (split TF32, ~FP32 accuracy) or
 *                    QRS_SYNTH_GEMM_BF16X3 (split BF16, ~2^-16 relative).
 * Workspace: draw records of up to 256 MB of realisations at a time, owned by
 * the handle; calls on one handle must not overlap in time.
 * nx, ny in [0, 2^24], n_real >= 0 (an empty grid or n_real = 0 is a no-op). */
qrs_status qrs_synthesize_grid(qrs_handle* h, const qrs_psd* psd, const qrs_domain* dom,
                               const qrs_sampler* smp, int64_t n_f, int64_t n_real, int64_t real_offset,
                               const float* x, int64_t nx, const float* y, int64_t ny, const int32_t* index,
                               int64_t n_points, int32_t mode, float* out, void* stream);

/* ------------------------------------------------------------- pistons ---
 * Differential pistons (Sec. 4.1, 4.4; PSD and filter of Eq. 7):
 *   piston[r][a] = sum_k F_k A_a(|f_k|) (a_k cos 2 pi f_k.p_a - b_k sin 2 pi f_k.p_a),
 *   A_a(f) = 2 (D_a J1(pi D_a f) - d_a J1(pi d_a f)) / (pi (D_a^2 - d_a^2) f), A(0) = 1,
 *   delta[r][q] = piston[r][i_q] - piston[r][j_q]  for pairs[q] = (i_q, j_q).
 * One job is one interferometer (its own PSD, domain, sampler, N_f, R).
 *   ap_xy [n_ap][2] aperture centres (m), ap_D, ap_d [n_ap] outer and
 *   obstruction diameters (m, 0 <= d < D), pairs [n_pairs][2] int32 in [0, n_ap),
 *   piston [n_real][n_ap] or NULL, delta [n_real][n_pairs] or NULL.
 * n_ap in [1, 64].  flags: QRS_PISTON_PERSISTENT runs all jobs in one
 * persistent launch over a cost-sorted work queue (bounded waits); with
 * QRS_PISTON_GRAPH the launch sequence is captured once per job set into a
 * CUDA graph and replayed.  Without flags, one launch per job. */
#define QRS_PISTON_PERSISTENT 1
#define QRS_PISTON_GRAPH 2

typedef struct qrs_piston_job {
    qrs_psd psd;
    qrs_domain dom;
    qrs_sampler smp;
    int64_t n_f;
    int64_t n_real;
    int64_t real_offset;
    const float* ap_xy;
    const float* ap_D;
    const float* ap_d;
    const int32_t* pairs;
    float* piston;
    float* delta;
    int32_t n_ap;
    int32_t n_pairs;
} qrs_piston_job;

qrs_status qrs_diff_piston(qrs_handle* h, const qrs_piston_job* jobs, int32_t n_jobs, int32_t flags,
                           void* stream);

/* ------------------------------------------------------ pair differences ---
 * Differential pistons of synthesised values (Sec. 4.4):
 *   out[r][q] = values[r][pairs[q][0]] - values[r][pairs[q][1]]
 *   values [n_real][n_points] FP32 (e.g. the output of qrs_synthesize_points
 *   with an aperture-filtered PSD), pairs [n_pairs][2] int32, out
 *   [n_real][n_pairs] FP32.  A pair index outside [0, n_points) gives NaN and
 *   records QRS_ERR_DEVICE_CHECK in the device error word (no out-of-bounds
 *   read). */
qrs_status qrs_pair_diff(qrs_handle* h, const float* values, int64_t n_real, int64_t n_points,
                         const int32_t* pairs, int64_t n_pairs, float* out, void* stream);

/* -------------------------------------------------- sampling statistics ---
 * Clusters and gaps of frequency draws (Sec. 2.3, 3.2, Figs. 2-3: jittered
 * and random sampling leave clusters and gaps, quasi-random sampling does
 * not).  pts [n_sets][n][2] FP32 (e.g. one realisation's frequencies per set,
 * from qrs_draw; for the discrepancy, points in [0,1]^2 such as a SQUARE draw
 * with fmax = 0.5 shifted by 0.5).
 *   qrs_nearest_neighbour: out [n_sets][n] FP32, each point's distance to its
 *     nearest other point (0 when n = 1).
 *   qrs_star_discrepancy:  out [n_sets] FP64, D* = sup over boxes [0,u)x[0,v)
 *     of |#points in the box / n - u v|, exact (integer counts at the
 *     (n+1)^2 corner candidates, exact FP64 products); O(n^3) work per set.
 * 1 <= n <= 65536, 0 <= n_sets <= 65535. */
qrs_status qrs_nearest_neighbour(qrs_handle* h, const float* pts, int64_t n_sets, int64_t n, float* out,
                                 void* stream);
qrs_status qrs_star_discrepancy(qrs_handle* h, const float* pts, int64_t n_sets, int64_t n, double* out,
                                void* stream);

/* ------------------------------------------------------ hyper-parameters ---
 * Sec. 4.2 choice of N for a square domain with cell delta_f: with the
 * isotropic PSD W (von Karman; times A^2 when psd->ap_D_m > 0),
 *   g(x) = int_0^x f W(f) df
 * saturates at g_inf = sigma^2 / (2 pi); the criterion stops at the first
 * m past the largest panel increment (where g saturates) with
 * g(m delta_f) - g((m-1) delta_f) < eps_rel g_inf, and N = 2 m
 * (2 max f = N delta_f, Eq. 5).  Host computation (composite Simpson
 * per delta_f panel), no handle and no GPU.  g_out (may be NULL) receives
 * {g(m delta_f), g_inf, the stopping increment}.  Errors: QRS_ERR_ARG for a
 * non-positive delta_f or eps_rel, a KOLMOGOROV PSD (g diverges at f = 0), or
 * no m <= n_max / 2 meeting the criterion. */
qrs_status qrs_choose_n(const qrs_psd* psd, double delta_f, double eps_rel, int32_t n_max, int32_t* n_out,
                        double* g_out);

/* --------------------------------------------------- structure function ---
 * Sec. 4.4: for series s and lag L = lags[l],
 *   L >= 1: x = v[t+L] - v[t], t in [0, T-L)   (temporal structure function)
 *   L == 0: x = v[t], t in [0, T)              (the value itself: over a baseline
 *                                               this is the spatial structure function)
 * acc[s][l][0..2] += (sum x^2, sum x^4, count) over all realisations and t:
 * x formed exactly from the FP32 inputs, per-thread partial sums in
 * double-float (FP32 pairs, about 48 significant bits; |x| >= 1e9 and NaN in
 * FP64), combined in FP64.
 * The caller zeroes acc once; calls accumulate, so the sums of a chunked run
 * equal those of one run up to rounding order.
 *   delta [n_real][n_series][T] FP32, lags [n_lags] int32 in [0, T), acc FP64. */
qrs_status qrs_structure_fn(qrs_handle* h, const float* delta, int64_t n_real, int64_t n_series,
                            int64_t T, const int32_t* lags, int32_t n_lags, double* acc, void* stream);

/* ----------------------------------------- FFT screen spectrum (Eq. 2) ---
 * The comparison method of Sec. 2.2 (static sampling of the frequency plane;
 * not the paper's method, which is the direct sum above): the spectrum of
 * n_real screens of n x n points at pitch dx (m),
 *   spec[r][i][j] = (a + i b) sqrt(W(f)) A(|f|) df,  f = (j', i') df,
 *   df = 1 / (n dx),  j' = j for j < (n + 1) / 2, j - n otherwise,
 * a, b ~ N(0,1) by Box-Muller from words 2 and 3 of the Philox4x32-10
 * counter ((real_offset + r) n^2 + i n + j, stream 4) with key seed, A the
 * Eq. 7 filter when psd->ap_D_m > 0 (else 1), and spec = 0 at f = 0.  The
 * screens are n^2 times its inverse DFT, sum_f spec(f) e^{2 pi i f.x} at
 * x = (j dx, i dx): the real and the imaginary part are two screens, each of
 * variance sum_f W df^2.  The caller takes that inverse transform (e.g.
 * cuFFT); the static grid is what biases their structure function (Sec. 2.3).
 *   spec [n_real][n][n][2] FP32 (interleaved complex), 8-byte aligned.
 * n in [2, 32768], dx > 0, n_real >= 0 (0 is a no-op), real_offset >= 0;
 * a KOLMOGOROV PSD is allowed (its f = 0 sample is the 0 above). */
qrs_status qrs_fft_spectrum(qrs_handle* h, const qrs_psd* psd, int64_t n, double dx, uint64_t seed, int64_t n_real,
                            int64_t real_offset, float* spec, void* stream);

/* ------------------------------------------------- no-allocation variant ---
 * The paper has no counterpart: this is a deployment variant of
 * qrs_synthesize_points (mode QRS_SYNTH_FUSED) for callers that cannot
 * allocate device memory -- e.g. code running inside a framework that owns all
 * device memory through its own pool, or a latency-bound loop where an
 * allocation could block or synchronise the device.  It takes no handle and
 * never calls cudaMalloc / cudaFree or any allocating routine.
 *   Scratch: a file-scope device array of QRS_NOALLOC_SCRATCH_BYTES per GPU,
 *   held by every GPU that loads the library until the process exits.  The
 *   fused path keeps two floats in it (the point and anchor bounds that select
 *   the phase path), whatever the problem size, so no size outgrows it; requests outside
 *   the limits of qrs_synthesize_points return QRS_ERR_ARG.  The bound is
 *   rewritten by every call, so nothing needs clearing between calls.
 *   Device: the calling thread's current device (at most 64 devices).  The
 *   first call on each device resolves the scratch's device address
 *   (cudaGetSymbolAddress, with that device current); make that first call
 *   before any stream capture.  A call that finds the device's context
 *   replaced since then (after cudaDeviceReset, which reloads the library's
 *   device code) resolves the address again, so the first call after a reset
 *   must also come before any stream capture.
 *   Concurrency: every call on a device shares the one scratch array, so calls
 *   that overlap on the GPU (e.g. on two streams at once) race; serialise them.
 *   Errors: status codes only (there is no handle to hold a message).
 * Arguments, layouts and results are those of qrs_synthesize_points with
 * mode = QRS_SYNTH_FUSED and col_psd = NULL; the output is identical. */
#define QRS_NOALLOC_SCRATCH_BYTES 256

qrs_status qrs_synthesize_points_noalloc(const qrs_psd* psd, const qrs_domain* dom, const qrs_sampler* smp,
                                         int64_t n_f, int64_t n_real, int64_t real_offset, const float* xy,
                                         int64_t n_points, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QRS_H */
