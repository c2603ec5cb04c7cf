/*
 * plsqr_oracle.c -- plain FP64 CPU oracle for the priorconditioned lagged-diffusivity
 * solver of Arridge, Betcke & Harhanen, "A priorconditioned LSQR algorithm for linear
 * ill-posed problems with edge-preserving regularization" (arXiv 1308.6634).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  It shares no code, header, table or helper with
 * the CUDA library: every formula below is written out again from the paper.
 *
 * Everything is double precision, single threaded, written for readability rather than
 * speed.  Loops follow the paper's notation: f (image), g (data), A (forward map),
 * kappa = r'(t)/t (diffusivity, eq. 1.13), M = sum_d D_d^T diag(kappa) D_d (the
 * regulariser operator, eqs. 1.12-1.13), P (the fixed V-cycle approximation of M^{-1},
 * Sec. 4.2), and the MLSQR recurrences of Algorithm 2 with the orthogonal transformation
 * of Algorithm 1 (steps 10-16) and Paige-Saunders damping (eq. 3.6, Sec. 3.3).
 *
 * Readings of points where the paper is silent (each is also listed in the design notes):
 *  - gradient: forward differences, unit spacing, a ghost value 0 beyond the high end of
 *    each axis (so D_d is square and invertible and M is SPD for kappa > 0);
 *  - one kappa per cell, weighting every forward edge of that cell;
 *  - kappa is floored at kfloor * kappa(0);
 *  - damping parameter sqrt(tau) (eqs. 2.3, 3.6);
 *  - Algorithm 2's initialisation also divides p~ by alpha_1 (it must equal M v~_1 for
 *    step 11 of the first iteration, as the derivation in Sec. 3.2 requires);
 *  - Algorithm 3 runs k = 1..n_outer with kappa taken from f^{k-1}, f^0 = 0, and every
 *    inner solve restarts from f = 0 (Sec. 4.3);
 *  - the blur is the tensor product of 1D Gaussian taps exp(-k^2/(2 sigma^2)) normalised
 *    to unit sum, truncated at a radius, with zero boundary;
 *  - the Joseph projector: pixel centres at (j-(n-1)/2, i-(n-1)/2), bin centres at
 *    (k-(nb-1)/2)*ds, angle a*pi/na, rows stepped when 4a < na or 4a > 3na;
 *  - multigrid: cell-centred coarsening by two per axis, piecewise-constant
 *    prolongation P, restriction R = P^T (sum of the 2^d children), Galerkin coarse
 *    operators (edge conductances summed over the fine faces of a coarse face),
 *    red-black Gauss-Seidel (red = even index sum) with nu sweeps red-then-black before
 *    and nu sweeps black-then-red after the coarse correction, zero initial guess, and
 *    an exact dense Cholesky solve on the coarsest level.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846;

/* Allocation that stops the test process with a message instead of returning NULL. */
static void* xmalloc(size_t bytes) {
    void* p = malloc(bytes ? bytes : 1);
    if (!p) {
        fprintf(stderr, "oracle: out of host memory (%zu bytes)\n", bytes);
        abort();
    }
    return p;
}

static void* xcalloc(size_t n, size_t size) {
    void* p = calloc(n ? n : 1, size ? size : 1);
    if (!p) {
        fprintf(stderr, "oracle: out of host memory (%zu x %zu bytes)\n", n, size);
        abort();
    }
    return p;
}

/* ------------------------------------------------------------------------------------ */
/* grid helpers                                                                          */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int ndim;       /* 1, 2 or 3 */
    int64_t n[3];   /* extents; n[0] is the fastest axis (x); unused axes are 1 */
} grid_t;

static int64_t grid_size(const grid_t* G) { return G->n[0] * G->n[1] * G->n[2]; }

static int64_t grid_stride(const grid_t* G, int d) {
    return d == 0 ? 1 : (d == 1 ? G->n[0] : G->n[0] * G->n[1]);
}

static void grid_coords(const grid_t* G, int64_t idx, int64_t c[3]) {
    c[0] = idx % G->n[0];
    c[1] = (idx / G->n[0]) % G->n[1];
    c[2] = idx / (G->n[0] * G->n[1]);
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* regulariser r(t) and diffusivity kappa(t) = r'(t)/t, eqs. (1.3)-(1.5), (1.13)          */
/* ------------------------------------------------------------------------------------ */

enum { REG_TIKHONOV = 0, REG_TV = 1, REG_PM_LOG = 2, REG_PM_EXP = 3 };

/* r(t): (1.3) 1/2 t^2; (1.4) smoothed TV T sqrt(1+(t/T)^2); (1.5) Perona-Malik
 * 1/2 T^2 log(1+(t/T)^2) and 1/2 T^2 (1 - exp(-t^2/T^2)). */
double oracle_r_of(int reg, double T, double t) {
    double q = t / T;
    switch (reg) {
        case REG_TIKHONOV: return 0.5 * t * t;
        case REG_TV: return T * sqrt(1.0 + q * q);
        case REG_PM_LOG: return 0.5 * T * T * log1p(q * q);
        case REG_PM_EXP: return -0.5 * T * T * expm1(-q * q);
    }
    return NAN;
}

/* kappa(t) = r'(t)/t, the diffusivity c_f of (1.13). Derivatives of the r above:
 * Tikhonov r' = t; TV r' = t / sqrt(1+(t/T)^2) / T ... i.e. kappa = 1/sqrt(T^2+t^2);
 * PM-log r' = t/(1+(t/T)^2); PM-exp r' = t exp(-t^2/T^2). */
double oracle_kappa_of(int reg, double T, double t) {
    double q = t / T;
    switch (reg) {
        case REG_TIKHONOV: return 1.0;
        case REG_TV: return 1.0 / sqrt(T * T + t * t);
        case REG_PM_LOG: return 1.0 / (1.0 + q * q);
        case REG_PM_EXP: return exp(-q * q);
    }
    return NAN;
}

/* Forward difference (D_d f)_i = f(i+e_d) - f(i), with f = 0 beyond the high end. */
static double fwd_diff(const grid_t* G, const double* f, int64_t idx, const int64_t c[3], int d) {
    double nb = (c[d] + 1 < G->n[d]) ? f[idx + grid_stride(G, d)] : 0.0;
    return nb - f[idx];
}

/* Diffusivity (Algorithm 3 step 3, eqs. 1.12-1.13): t_i = |(D f)_i|, kappa_i =
 * max(kappa(t_i), kfloor*kappa(0)); returns R(f) = sum_i r(t_i) (discrete eq. 1.2). */
/* Storage rounding of kappa, for the variant that keeps kappa in bfloat16: 0 none; 1 the value
 * rounded to single precision and then to bfloat16 (8 significant bits), both to nearest with
 * ties to even.  The second rounding is the usual bit form: add 0x7fff plus the lowest kept bit
 * to the single-precision pattern and clear the 16 low bits. */
static int kappa_rounding = 0;

void oracle_set_kappa_rounding(int mode) { kappa_rounding = mode; }

double oracle_round_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf, nan */
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&f, &u, sizeof f);
    return (double)f;
}

double oracle_diffusivity(int ndim, const int64_t* n, int reg, double T, double kfloor,
                          const double* f, double* kappa) {
    grid_t G = {ndim, {n[0], ndim > 1 ? n[1] : 1, ndim > 2 ? n[2] : 1}};
    int64_t N = grid_size(&G);
    double kmin = kfloor * oracle_kappa_of(reg, T, 0.0);
    double R = 0.0;
    for (int64_t idx = 0; idx < N; ++idx) {
        int64_t c[3];
        grid_coords(&G, idx, c);
        double t2 = 0.0;
        for (int d = 0; d < ndim; ++d) {
            double g = fwd_diff(&G, f, idx, c, d);
            t2 += g * g;
        }
        double t = sqrt(t2);
        double k = oracle_kappa_of(reg, T, t);
        k = k > kmin ? k : kmin;
        kappa[idx] = kappa_rounding == 1 ? oracle_round_bf16(k) : k;
        R += oracle_r_of(reg, T, t);
    }
    return R;
}

/* ------------------------------------------------------------------------------------ */
/* weighted diffusion operator on a level: edge conductances c[d][i] on the edge i->i+e_d */
/* (the edge leaving the high end goes to the ghost value 0)                              */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    grid_t G;
    double* c[3]; /* conductances per axis, N each */
} level_t;

static double level_diag(const level_t* L, int64_t idx, const int64_t c[3]) {
    double s = 0.0;
    for (int d = 0; d < L->G.ndim; ++d) {
        s += L->c[d][idx];
        if (c[d] > 0) s += L->c[d][idx - grid_stride(&L->G, d)];
    }
    return s;
}

/* sum over neighbours j of c_ij x_j (ghost neighbours contribute 0) */
static double level_offdiag_sum(const level_t* L, const double* x, int64_t idx, const int64_t c[3]) {
    double s = 0.0;
    for (int d = 0; d < L->G.ndim; ++d) {
        int64_t st = grid_stride(&L->G, d);
        if (c[d] + 1 < L->G.n[d]) s += L->c[d][idx] * x[idx + st];
        if (c[d] > 0) s += L->c[d][idx - st] * x[idx - st];
    }
    return s;
}

/* y = M_level x: (M x)_i = sum_d c_d(i)(x_i - x_{i+e_d}) + c_d(i-e_d)(x_i - x_{i-e_d}). */
static void level_apply(const level_t* L, const double* x, double* y) {
    int64_t N = grid_size(&L->G);
    for (int64_t idx = 0; idx < N; ++idx) {
        int64_t c[3];
        grid_coords(&L->G, idx, c);
        y[idx] = level_diag(L, idx, c) * x[idx] - level_offdiag_sum(L, x, idx, c);
    }
}

/* M_f x with M_f = sum_d D_d^T diag(kappa) D_d, eq. (1.13) on the tensor grid. */
void oracle_apply_M(int ndim, const int64_t* n, const double* kappa, const double* x, double* y) {
    level_t L;
    L.G.ndim = ndim;
    L.G.n[0] = n[0];
    L.G.n[1] = ndim > 1 ? n[1] : 1;
    L.G.n[2] = ndim > 2 ? n[2] : 1;
    for (int d = 0; d < 3; ++d) L.c[d] = (double*)kappa;
    level_apply(&L, x, y);
}

/* ------------------------------------------------------------------------------------ */
/* geometric multigrid V-cycle: a fixed symmetric approximation of M^{-1} (Sec. 4.2)     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int levels, nu, cycles;
    level_t lv[16];
    double* chol;      /* dense lower Cholesky factor of the coarsest operator, nc x nc */
    int64_t nc;
    double *tmp_r, *tmp_e; /* scratch for apply (fine-level size) */
    double* work[16][3];   /* per level: rhs, x, residual */
} mg_t;

/* Galerkin coarsening with piecewise-constant prolongation: the coarse conductance of the
 * face between coarse cells I and I+e_d is the sum of the fine conductances of the 2^(d-1)
 * fine edges crossing it (fine cells with i_d = 2 I_d + 1 and i_e in {2I_e, 2I_e+1}). */
static void coarsen(const level_t* F, level_t* C) {
    C->G.ndim = F->G.ndim;
    for (int d = 0; d < 3; ++d) C->G.n[d] = (d < F->G.ndim) ? F->G.n[d] / 2 : 1;
    int64_t NC = grid_size(&C->G);
    for (int d = 0; d < F->G.ndim; ++d) {
        C->c[d] = (double*)xcalloc((size_t)NC, sizeof(double));
        for (int64_t I = 0; I < NC; ++I) {
            int64_t cc[3];
            grid_coords(&C->G, I, cc);
            double s = 0.0;
            /* children on the high face of I in direction d */
            int64_t lo[3], hi[3];
            for (int e = 0; e < 3; ++e) {
                if (e >= F->G.ndim) { lo[e] = hi[e] = 0; continue; }
                if (e == d) { lo[e] = hi[e] = 2 * cc[e] + 1; }
                else { lo[e] = 2 * cc[e]; hi[e] = 2 * cc[e] + 1; }
            }
            for (int64_t z = lo[2]; z <= hi[2]; ++z)
                for (int64_t y = lo[1]; y <= hi[1]; ++y)
                    for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                        int64_t fi = x + F->G.n[0] * (y + F->G.n[1] * z);
                        s += F->c[d][fi];
                    }
            C->c[d][I] = s;
        }
    }
    for (int d = F->G.ndim; d < 3; ++d) C->c[d] = NULL;
}

/* R = P^T: coarse value = sum of the 2^d children. */
static void restrict_sum(const grid_t* F, const grid_t* C, const double* r, double* rc) {
    int64_t NC = grid_size(C);
    for (int64_t I = 0; I < NC; ++I) rc[I] = 0.0;
    int64_t NF = grid_size(F);
    for (int64_t i = 0; i < NF; ++i) {
        int64_t c[3];
        grid_coords(F, i, c);
        int64_t I = (c[0] / 2) + C->n[0] * ((F->ndim > 1 ? c[1] / 2 : 0) + C->n[1] * (F->ndim > 2 ? c[2] / 2 : 0));
        rc[I] += r[i];
    }
}

/* x += P e: every fine cell takes the value of its parent. */
static void prolong_add(const grid_t* F, const grid_t* C, const double* e, double* x) {
    int64_t NF = grid_size(F);
    for (int64_t i = 0; i < NF; ++i) {
        int64_t c[3];
        grid_coords(F, i, c);
        int64_t I = (c[0] / 2) + C->n[0] * ((F->ndim > 1 ? c[1] / 2 : 0) + C->n[1] * (F->ndim > 2 ? c[2] / 2 : 0));
        x[i] += e[I];
    }
}

/* One Gauss-Seidel half sweep over the cells of one colour (colour = parity of the index
 * sum), lexicographic order within the colour. */
static void gs_colour(const level_t* L, int colour, const double* b, double* x) {
    int64_t N = grid_size(&L->G);
    for (int64_t idx = 0; idx < N; ++idx) {
        int64_t c[3];
        grid_coords(&L->G, idx, c);
        if (((c[0] + c[1] + c[2]) & 1) != colour) continue;
        x[idx] = (b[idx] + level_offdiag_sum(L, x, idx, c)) / level_diag(L, idx, c);
    }
}

static int dense_cholesky(int64_t n, double* a) {
    /* in place, lower triangle, row-major a[i*n+j] */
    for (int64_t j = 0; j < n; ++j) {
        double s = a[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= a[j * n + k] * a[j * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        a[j * n + j] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = a[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = t / d;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) a[i * n + j] = 0.0;
    return 0;
}

static void dense_cholesky_solve(int64_t n, const double* l, const double* b, double* x) {
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= l[i * n + k] * x[k];
        x[i] = s / l[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t k = i + 1; k < n; ++k) s -= l[k * n + i] * x[k];
        x[i] = s / l[i * n + i];
    }
}

static void vcycle(const mg_t* mg, int l, const double* b, double* x) {
    const level_t* L = &mg->lv[l];
    int64_t N = grid_size(&L->G);
    if (l == mg->levels - 1) {
        dense_cholesky_solve(mg->nc, mg->chol, b, x);
        return;
    }
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    for (int s = 0; s < mg->nu; ++s) {
        gs_colour(L, 0, b, x);
        gs_colour(L, 1, b, x);
    }
    double* r = mg->work[l][2];
    level_apply(L, x, r);
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - r[i];
    const level_t* C = &mg->lv[l + 1];
    double* bc = mg->work[l + 1][0];
    double* xc = mg->work[l + 1][1];
    restrict_sum(&L->G, &C->G, r, bc);
    vcycle(mg, l + 1, bc, xc);
    prolong_add(&L->G, &C->G, xc, x);
    for (int s = 0; s < mg->nu; ++s) {
        gs_colour(L, 1, b, x);
        gs_colour(L, 0, b, x);
    }
}

/* Build the hierarchy from kappa. Returns NULL on invalid sizes or a failed factorisation. */
void* oracle_mg_create(int ndim, const int64_t* n, const double* kappa, int levels, int nu, int cycles) {
    if (levels < 1 || levels > 16 || ndim < 1 || ndim > 3) return NULL;
    for (int d = 0; d < ndim; ++d)
        if (n[d] % ((int64_t)1 << (levels - 1)) != 0) return NULL;
    mg_t* mg = (mg_t*)xcalloc(1, sizeof(mg_t));
    mg->levels = levels;
    mg->nu = nu;
    mg->cycles = cycles;
    level_t* L0 = &mg->lv[0];
    L0->G.ndim = ndim;
    for (int d = 0; d < 3; ++d) L0->G.n[d] = d < ndim ? n[d] : 1;
    int64_t N = grid_size(&L0->G);
    for (int d = 0; d < ndim; ++d) {
        L0->c[d] = (double*)xmalloc((size_t)N * sizeof(double));
        memcpy(L0->c[d], kappa, (size_t)N * sizeof(double));
    }
    for (int l = 1; l < levels; ++l) coarsen(&mg->lv[l - 1], &mg->lv[l]);
    for (int l = 0; l < levels; ++l) {
        int64_t Nl = grid_size(&mg->lv[l].G);
        for (int k = 0; k < 3; ++k) mg->work[l][k] = (double*)xcalloc((size_t)Nl, sizeof(double));
    }
    mg->tmp_r = (double*)xcalloc((size_t)N, sizeof(double));
    mg->tmp_e = (double*)xcalloc((size_t)N, sizeof(double));
    /* dense coarsest operator, assembled column by column from the stencil */
    level_t* LC = &mg->lv[levels - 1];
    int64_t nc = grid_size(&LC->G);
    mg->nc = nc;
    mg->chol = (double*)xcalloc((size_t)(nc * nc), sizeof(double));
    double* e = (double*)xcalloc((size_t)nc, sizeof(double));
    double* col = (double*)xcalloc((size_t)nc, sizeof(double));
    for (int64_t j = 0; j < nc; ++j) {
        e[j] = 1.0;
        level_apply(LC, e, col);
        e[j] = 0.0;
        for (int64_t i = 0; i < nc; ++i) mg->chol[i * nc + j] = col[i];
    }
    free(e);
    free(col);
    if (dense_cholesky(nc, mg->chol) != 0) {
        /* not SPD: caller sees NULL */
        for (int l = 0; l < levels; ++l) {
            for (int d = 0; d < ndim; ++d) free(mg->lv[l].c[d]);
            for (int k = 0; k < 3; ++k) free(mg->work[l][k]);
        }
        free(mg->tmp_r); free(mg->tmp_e); free(mg->chol); free(mg);
        return NULL;
    }
    return mg;
}

void oracle_mg_free(void* h) {
    mg_t* mg = (mg_t*)h;
    if (!mg) return;
    for (int l = 0; l < mg->levels; ++l) {
        for (int d = 0; d < mg->lv[l].G.ndim; ++d) free(mg->lv[l].c[d]);
        for (int k = 0; k < 3; ++k) free(mg->work[l][k]);
    }
    free(mg->tmp_r); free(mg->tmp_e); free(mg->chol); free(mg);
}

/* x = P b: `cycles` V-cycles from a zero initial guess, x <- x + V(b - M x). */
void oracle_mg_apply(void* h, const double* b, double* x) {
    mg_t* mg = (mg_t*)h;
    const level_t* L0 = &mg->lv[0];
    int64_t N = grid_size(&L0->G);
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    for (int k = 0; k < mg->cycles; ++k) {
        if (k == 0) {
            memcpy(mg->tmp_r, b, (size_t)N * sizeof(double));
        } else {
            level_apply(L0, x, mg->tmp_r);
            for (int64_t i = 0; i < N; ++i) mg->tmp_r[i] = b[i] - mg->tmp_r[i];
        }
        vcycle(mg, 0, mg->tmp_r, mg->tmp_e);
        for (int64_t i = 0; i < N; ++i) x[i] += mg->tmp_e[i];
    }
}

/* y = M_l x on level l of the hierarchy (level 0 is M_f itself). */
void oracle_mg_level_apply(void* h, int l, const double* x, double* y) {
    mg_t* mg = (mg_t*)h;
    level_apply(&mg->lv[l], x, y);
}

int64_t oracle_mg_level_size(void* h, int l) {
    mg_t* mg = (mg_t*)h;
    return grid_size(&mg->lv[l].G);
}

/* ------------------------------------------------------------------------------------ */
/* forward maps A and adjoints A^T                                                        */
/* ------------------------------------------------------------------------------------ */

enum { OP_BLUR = 0, OP_BLUR_MASK = 1, OP_JOSEPH = 2, OP_IDENTITY = 3 };

typedef struct {
    int32_t kind;
    int32_t ndim;
    int64_t n[3];
    double sigma[3];
    int32_t radius[3];
    int32_t n_angles;
    int32_t n_bins;
    int32_t pad_;
    double bin_spacing;
    const uint8_t* mask; /* N bytes, nonzero = observed */
} op_t;

/* Gaussian taps w_k = exp(-k^2/(2 sigma^2)) / sum_{|j|<=R} exp(-j^2/(2 sigma^2)). */
void oracle_blur_taps(double sigma, int R, double* w) {
    double s = 0.0;
    for (int k = -R; k <= R; ++k) {
        w[k + R] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        s += w[k + R];
    }
    for (int k = -R; k <= R; ++k) w[k + R] /= s;
}

/* y = conv_d(x): 1D convolution along axis d with zero boundary. */
static void conv_axis(const grid_t* G, int d, const double* w, int R, const double* x, double* y) {
    int64_t N = grid_size(G), st = grid_stride(G, d);
    for (int64_t idx = 0; idx < N; ++idx) {
        int64_t c[3];
        grid_coords(G, idx, c);
        double acc = 0.0;
        for (int k = -R; k <= R; ++k) {
            int64_t j = c[d] + k;
            if (j < 0 || j >= G->n[d]) continue;
            acc += w[k + R] * x[idx + k * st];
        }
        y[idx] = acc;
    }
}

/* Separable Gaussian blur B (symmetric, so B^T = B). */
static void blur(const op_t* op, const double* x, double* y) {
    grid_t G = {op->ndim, {op->n[0], op->ndim > 1 ? op->n[1] : 1, op->ndim > 2 ? op->n[2] : 1}};
    int64_t N = grid_size(&G);
    double* t = (double*)xmalloc((size_t)N * sizeof(double));
    memcpy(t, x, (size_t)N * sizeof(double));
    for (int d = 0; d < op->ndim; ++d) {
        int R = op->radius[d];
        double* w = (double*)xmalloc((size_t)(2 * R + 1) * sizeof(double));
        oracle_blur_taps(op->sigma[d], R, w);
        conv_axis(&G, d, w, R, t, y);
        memcpy(t, y, (size_t)N * sizeof(double));
        free(w);
    }
    free(t);
}

/* Joseph projector, parallel beam. Ray (a,k): x cos(th) + y sin(th) = s_k. One pass with
 * a flag: adjoint = 0 gathers image -> sinogram, adjoint = 1 scatters sinogram -> image
 * through the same weights (exact transpose). */
static void joseph(const op_t* op, const double* in, double* out, int adjoint) {
    int64_t n = op->n[0]; /* square n x n image, row i = y, column j = x */
    int na = op->n_angles, nb = op->n_bins;
    double ds = op->bin_spacing;
    double cimg = 0.5 * (double)(n - 1), cdet = 0.5 * (double)(nb - 1);
    if (adjoint) memset(out, 0, (size_t)(n * n) * sizeof(double));
    for (int a = 0; a < na; ++a) {
        double th = PI * (double)a / (double)na;
        double ct = cos(th), st = sin(th);
        int rows = (4 * a < na) || (4 * a > 3 * na);
        for (int k = 0; k < nb; ++k) {
            double s = ((double)k - cdet) * ds;
            double acc = 0.0;
            if (rows) {
                double wgt = 1.0 / fabs(ct);
                for (int64_t i = 0; i < n; ++i) {
                    double y = (double)i - cimg;
                    double u = (s - y * st) / ct + cimg;
                    double j0f = floor(u);
                    double fr = u - j0f;
                    int64_t j0 = (int64_t)j0f;
                    if (j0 >= 0 && j0 < n) {
                        if (adjoint) out[i * n + j0] += wgt * (1.0 - fr) * in[(int64_t)a * nb + k];
                        else acc += (1.0 - fr) * in[i * n + j0];
                    }
                    if (j0 + 1 >= 0 && j0 + 1 < n) {
                        if (adjoint) out[i * n + j0 + 1] += wgt * fr * in[(int64_t)a * nb + k];
                        else acc += fr * in[i * n + j0 + 1];
                    }
                }
                if (!adjoint) out[(int64_t)a * nb + k] = wgt * acc;
            } else {
                double wgt = 1.0 / fabs(st);
                for (int64_t j = 0; j < n; ++j) {
                    double x = (double)j - cimg;
                    double v = (s - x * ct) / st + cimg;
                    double i0f = floor(v);
                    double fr = v - i0f;
                    int64_t i0 = (int64_t)i0f;
                    if (i0 >= 0 && i0 < n) {
                        if (adjoint) out[i0 * n + j] += wgt * (1.0 - fr) * in[(int64_t)a * nb + k];
                        else acc += (1.0 - fr) * in[i0 * n + j];
                    }
                    if (i0 + 1 >= 0 && i0 + 1 < n) {
                        if (adjoint) out[(i0 + 1) * n + j] += wgt * fr * in[(int64_t)a * nb + k];
                        else acc += fr * in[(i0 + 1) * n + j];
                    }
                }
                if (!adjoint) out[(int64_t)a * nb + k] = wgt * acc;
            }
        }
    }
}

static int64_t op_unknowns(const op_t* op) {
    int64_t N = 1;
    for (int d = 0; d < op->ndim; ++d) N *= op->n[d];
    return N;
}

int64_t oracle_op_data_len(const op_t* op) {
    if (op->kind == OP_JOSEPH) return (int64_t)op->n_angles * op->n_bins;
    return op_unknowns(op);
}

/* y = A x */
void oracle_apply_A(const op_t* op, const double* x, double* y) {
    int64_t N = op_unknowns(op);
    switch (op->kind) {
        case OP_BLUR: blur(op, x, y); break;
        case OP_BLUR_MASK:
            blur(op, x, y);
            for (int64_t i = 0; i < N; ++i) if (!op->mask[i]) y[i] = 0.0;
            break;
        case OP_JOSEPH: joseph(op, x, y, 0); break;
        case OP_IDENTITY: memcpy(y, x, (size_t)N * sizeof(double)); break;
    }
}

/* x = A^T y */
void oracle_apply_At(const op_t* op, const double* y, double* x) {
    int64_t N = op_unknowns(op);
    switch (op->kind) {
        case OP_BLUR: blur(op, y, x); break;
        case OP_BLUR_MASK: {
            double* t = (double*)xmalloc((size_t)N * sizeof(double));
            for (int64_t i = 0; i < N; ++i) t[i] = op->mask[i] ? y[i] : 0.0;
            blur(op, t, x);
            free(t);
            break;
        }
        case OP_JOSEPH: joseph(op, y, x, 1); break;
        case OP_IDENTITY: memcpy(x, y, (size_t)N * sizeof(double)); break;
    }
}

/* ------------------------------------------------------------------------------------ */
/* MLSQR, Algorithm 2, with the damped orthogonal transformation                          */
/* ------------------------------------------------------------------------------------ */

enum { PREC_MG = 0, PREC_IDENTITY = 1 };

/* Returns the number of iterations completed; *status = 0 ok, 4 breakdown.
 * rbar_hist[i-1] = ||rbar_i|| = sqrt(phibar_{i+1}^2 + sum psi^2) (the LSQR estimate of
 * the residual of the damped problem, Sec. 3.4). prec = NULL applies P = I. */
/* Algorithm 2; with eta_delta > 0 it stops after the first iteration i whose residual estimate
 * ||rbar_i|| = sqrt(phibar_{i+1}^2 + sum psi^2) is <= eta_delta (the discrepancy principle S4,
 * Sec. 3.4, with eta delta given; at tau = 0 the estimate equals ||g - A f_i||), keeping f_i. */
static int mlsqr_impl(const op_t* op, void* prec, double tau, int n_inner, const double* g, double* f,
                      double* rbar_hist, int* status, double eta_delta);

int oracle_mlsqr(const op_t* op, void* prec, double tau, int n_inner, const double* g,
                 double* f, double* rbar_hist, int* status) {
    return mlsqr_impl(op, prec, tau, n_inner, g, f, rbar_hist, status, 0.0);
}

int oracle_mlsqr_s4(const op_t* op, void* prec, double tau, int n_inner, const double* g, double* f,
                    double* rbar_hist, int* status, double eta_delta) {
    return mlsqr_impl(op, prec, tau, n_inner, g, f, rbar_hist, status, eta_delta);
}

static int mlsqr_impl(const op_t* op, void* prec, double tau, int n_inner, const double* g, double* f,
                      double* rbar_hist, int* status, double eta_delta) {
    mg_t* mg = (mg_t*)prec;
    int64_t N = op_unknowns(op), m = oracle_op_data_len(op);
    double* u = (double*)xmalloc((size_t)m * sizeof(double));
    double* Av = (double*)xmalloc((size_t)m * sizeof(double));
    double* p = (double*)xmalloc((size_t)N * sizeof(double));
    double* Atu = (double*)xmalloc((size_t)N * sizeof(double));
    double* v = (double*)xmalloc((size_t)N * sizeof(double));
    double* w = (double*)xmalloc((size_t)N * sizeof(double));
    int done = 0;
    *status = 0;
    for (int64_t i = 0; i < N; ++i) f[i] = 0.0;
    /* initialisation, steps 2-7 */
    memcpy(u, g, (size_t)m * sizeof(double));
    double beta = sqrt(dot(m, u, u));
    double beta1 = beta;
    if (!(beta > 0.0) || !isfinite(beta)) { *status = 4; goto out; }
    for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    oracle_apply_At(op, u, p);
    if (mg) oracle_mg_apply(mg, p, v); else memcpy(v, p, (size_t)N * sizeof(double));
    double alpha = sqrt(dot(N, v, p));
    if (!(alpha > 0.0) || !isfinite(alpha)) { *status = 4; goto out; }
    for (int64_t i = 0; i < N; ++i) { v[i] /= alpha; p[i] /= alpha; }
    memcpy(w, v, (size_t)N * sizeof(double));
    double phibar = beta, rhobar = alpha, res2 = 0.0;
    double damp = sqrt(tau);
    for (int it = 1; it <= n_inner; ++it) {
        /* bidiagonalisation, steps 10-15 */
        oracle_apply_A(op, v, Av);
        for (int64_t i = 0; i < m; ++i) u[i] = Av[i] - alpha * u[i];
        beta = sqrt(dot(m, u, u));
        if (!(beta > 1e-30 * beta1) || !isfinite(beta)) { *status = 4; break; }
        for (int64_t i = 0; i < m; ++i) u[i] /= beta;
        oracle_apply_At(op, u, Atu);
        for (int64_t i = 0; i < N; ++i) p[i] = Atu[i] - beta * p[i];
        if (mg) oracle_mg_apply(mg, p, v); else memcpy(v, p, (size_t)N * sizeof(double));
        double a2 = dot(N, v, p);
        double alpha_new = sqrt(a2);
        if (!(alpha_new > 1e-30 * beta1) || !isfinite(alpha_new)) { *status = 4; break; }
        for (int64_t i = 0; i < N; ++i) { p[i] /= alpha_new; v[i] /= alpha_new; }
        /* orthogonal transformation, Algorithm 1 steps 10-16, damping rotation first */
        double rhohat = rhobar, psi = 0.0;
        if (tau > 0.0) {
            rhohat = sqrt(rhobar * rhobar + tau);
            double c1 = rhobar / rhohat, s1 = damp / rhohat;
            psi = s1 * phibar;
            phibar = c1 * phibar;
        }
        double rho = sqrt(rhohat * rhohat + beta * beta);
        double c = rhohat / rho, s = beta / rho;
        double theta = s * alpha_new;
        rhobar = -c * alpha_new;
        double phi = c * phibar;
        phibar = s * phibar;
        res2 += psi * psi;
        /* update, steps 19-20 */
        for (int64_t i = 0; i < N; ++i) {
            f[i] += (phi / rho) * w[i];
            w[i] = v[i] - (theta / rho) * w[i];
        }
        alpha = alpha_new;
        const double rbar = sqrt(phibar * phibar + res2);
        if (rbar_hist) rbar_hist[it - 1] = rbar;
        done = it;
        if (eta_delta > 0.0 && rbar <= eta_delta) break; /* S4 */
    }
out:
    free(u); free(Av); free(p); free(Atu); free(v); free(w);
    return done;
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 3: lagged-diffusivity fixed point with MLSQR inner solves                   */
/* ------------------------------------------------------------------------------------ */

/* Runs n_outer steps. Outputs: f (N), rbar_hist (n_outer*n_inner; entries after a
 * breakdown stay as given), R_hist (n_outer+1: R(f^0..f^n_outer)), resid_hist (n_outer:
 * ||g - A f^k||). Returns 0, 4 (breakdown in some inner solve; the loop continues with
 * the iterate reached) or 1 (invalid multigrid sizes / factorisation failure). */
/* Algorithm 3 with its stopping rules (Sec. 4.1): each MLSQR solve stops by S4 with eta_delta
 * (0: never) within the cap of n_inner iterations, and the fixed point stops at f^j (j >= 2) when
 * R(f^j) did not decrease by more than the fraction r_rel of R(f^{j-1}) (r_rel <= 0: never).
 * *outer_done receives the number of MLSQR solves run.  Histories as oracle_solve; entries of
 * iterations and steps not run stay as given. */
int oracle_solve_stop(const op_t* op, int reg, double T, double tau, double kfloor, int levels, int nu,
                      int cycles, int n_outer, int n_inner, double eta_delta, double r_rel, const double* g,
                      double* f, double* rbar_hist, double* R_hist, double* resid_hist, int* outer_done) {
    int64_t N = op_unknowns(op), m = oracle_op_data_len(op);
    double* kappa = (double*)xmalloc((size_t)N * sizeof(double));
    double* Af = (double*)xmalloc((size_t)m * sizeof(double));
    int ret = 0, k = 1, stopped = 0;
    double R_prev = 0.0;
    for (int64_t i = 0; i < N; ++i) f[i] = 0.0;
    *outer_done = 0;
    for (; k <= n_outer; ++k) {
        double R = oracle_diffusivity(op->ndim, op->n, reg, T, kfloor, f, kappa); /* R(f^{k-1}) */
        if (R_hist) R_hist[k - 1] = R;
        if (r_rel > 0.0 && k - 1 >= 2 && R_prev > 0.0 && (R - R_prev) / R_prev > -r_rel) { stopped = 1; break; }
        R_prev = R;
        void* mg = oracle_mg_create(op->ndim, op->n, kappa, levels, nu, cycles);
        if (!mg) { ret = 1; break; }
        int st = 0;
        mlsqr_impl(op, mg, tau, n_inner, g, f, rbar_hist ? rbar_hist + (int64_t)(k - 1) * n_inner : NULL, &st,
                   eta_delta);
        if (st) ret = st;
        oracle_mg_free(mg);
        *outer_done = k;
        if (resid_hist) {
            oracle_apply_A(op, f, Af);
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) s += (g[i] - Af[i]) * (g[i] - Af[i]);
            resid_hist[k - 1] = sqrt(s);
        }
    }
    if (R_hist && ret != 1 && !stopped) R_hist[n_outer] = oracle_diffusivity(op->ndim, op->n, reg, T, kfloor, f, kappa);
    free(kappa);
    free(Af);
    return ret;
}

int oracle_solve(const op_t* op, int reg, double T, double tau, double kfloor, int levels,
                 int nu, int cycles, int n_outer, int n_inner, const double* g, double* f,
                 double* rbar_hist, double* R_hist, double* resid_hist) {
    int64_t N = op_unknowns(op), m = oracle_op_data_len(op);
    double* kappa = (double*)xmalloc((size_t)N * sizeof(double));
    double* Af = (double*)xmalloc((size_t)m * sizeof(double));
    int ret = 0;
    for (int64_t i = 0; i < N; ++i) f[i] = 0.0;
    for (int k = 1; k <= n_outer; ++k) {
        double R = oracle_diffusivity(op->ndim, op->n, reg, T, kfloor, f, kappa);
        if (R_hist) R_hist[k - 1] = R;
        void* mg = oracle_mg_create(op->ndim, op->n, kappa, levels, nu, cycles);
        if (!mg) { ret = 1; break; }
        int st = 0;
        oracle_mlsqr(op, mg, tau, n_inner, g, f, rbar_hist ? rbar_hist + (int64_t)(k - 1) * n_inner : NULL, &st);
        if (st) ret = st;
        oracle_mg_free(mg);
        if (resid_hist) {
            oracle_apply_A(op, f, Af);
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) s += (g[i] - Af[i]) * (g[i] - Af[i]);
            resid_hist[k - 1] = sqrt(s);
        }
    }
    if (R_hist && ret != 1) R_hist[n_outer] = oracle_diffusivity(op->ndim, op->n, reg, T, kfloor, f, kappa);
    free(kappa);
    free(Af);
    return ret;
}
