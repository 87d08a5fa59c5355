/*
 * REANN FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct reference for what the GPU library computes.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load it.  It shares no code with the CUDA path (no headers, helpers or
 * tables); the only common input is the flat parameter vector written by
 * synth/model.py and the structures written by synth/structures.py.
 *
 * What it computes (paper Sec. 2.1, Eqs. 1-2; Sec. 2.2, Eqs. 3-5):
 *
 *   neighbours  all (i, j, n) with d = |r_j + n.H - r_i| < r_cut, excluding
 *               only the zero-shift self term (brute force over all pairs and
 *               all image shifts; periodic self-images count).
 *   layer t     b_{i,a,m} = sum_{(j,n), d<r_c} c^t_{j,m} phi_m(d) A_a(r_ij)
 *               g_{i,a,k} = sum_m b_{i,a,m} W^t_{l(a),m,k}
 *               rho^t_{i,l,k} = sum_{a: l(a)=l} l!/(lx! ly! lz!) g_{i,a,k}^2   (Eq. 1)
 *               c^{t+1}_i = M^t_{Z_i}(rho^t_i)  for t < T-1                    (Eq. 2)
 *               eps_i     = M^{T-1}_{Z_i}(rho^{T-1}_i)                          (Sec. 2.1)
 *   energy      E = sum_i eps_i
 *   forces      F = -dE/dr by a hand-derived reverse pass through the layers
 *               (chain rule of Eqs. 3-5; the paper's vector-Jacobian products
 *               are the adjoints cbar, rhobar below).
 *
 * with phi_m(d) = exp(-alpha (d - mu_m)^2) f_c(d), mu_m = m r_c / (N_phi - 1),
 * f_c(d) = (cos(pi d / r_c)/2 + 1/2)^2 and A_a(r) = x^lx y^ly z^lz in A.
 *
 * Readings of points the paper leaves open (cutoff form, Gaussian centres,
 * coefficient shape, self-images, initial coefficients) are the ones listed in
 * the repository's design notes; the parity of the numbers themselves is pinned
 * by closed forms, invariants and finite differences in tests/test_oracle_*.py.
 *
 * Floating-point contract for the neighbour test (so that both sides take the
 * integer decision "is (i,j,n) a neighbour" in the same FP64 arithmetic):
 *   Hinv = adj(H)/det(H) (formula below), frac_k = (x0 Hinv[0][k] + x1
 *   Hinv[1][k]) + x2 Hinv[2][k], m = floor(frac), S(n)_d = (n0 H[0][d] +
 *   n1 H[1][d]) + n2 H[2][d], wrapped x_w = x - S(m), r = (x_w,j - x_w,i) +
 *   S(n), d^2 = (r0 r0 + r1 r1) + r2 r2, compiled without FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_E_ARG (-1)
#define OR_E_NOMEM (-3)
#define OR_E_GEOM (-4)
#define OR_E_CAP (-7)

#define MAX_ANG 64 /* (L+1)(L+2)(L+3)/6 for L <= 6 */

/* ------------------------------------------------------------------ cell --- */

static int cell_inverse(const double *h, double *hinv) {
    double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                 h[2] * (h[3] * h[7] - h[4] * h[6]);
    if (!(fabs(det) > 1e-12) || !isfinite(det)) return OR_E_GEOM;
    hinv[0] = (h[4] * h[8] - h[5] * h[7]) / det;
    hinv[1] = (h[2] * h[7] - h[1] * h[8]) / det;
    hinv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    hinv[3] = (h[5] * h[6] - h[3] * h[8]) / det;
    hinv[4] = (h[0] * h[8] - h[2] * h[6]) / det;
    hinv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    hinv[6] = (h[3] * h[7] - h[4] * h[6]) / det;
    hinv[7] = (h[1] * h[6] - h[0] * h[7]) / det;
    hinv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    return OR_OK;
}

/* perpendicular width of the cell along lattice direction k: |det| / |h_{k+1} x h_{k+2}| */
static double cell_width(const double *h, int k) {
    const double *u = h + 3 * ((k + 1) % 3), *v = h + 3 * ((k + 2) % 3);
    double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    double det = h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6]) +
                 h[2] * (h[3] * h[7] - h[4] * h[6]);
    return fabs(det) / sqrt(cx * cx + cy * cy + cz * cz);
}

static void shift_vec(const double *h, int n0, int n1, int n2, double *s) {
    for (int d = 0; d < 3; ++d) s[d] = ((double)n0 * h[d] + (double)n1 * h[3 + d]) + (double)n2 * h[6 + d];
}

/* Wrap positions into the cell: xw = x - S(m), m = floor(x . Hinv); also the
 * fractional coordinates of xw (for the image-range pruning only). */
static int wrap_positions(int64_t n, const double *pos, const double *h, double *xw, double *fw, int32_t *m) {
    double hinv[9];
    int rc = cell_inverse(h, hinv);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        const double *x = pos + 3 * i;
        int mi[3];
        double fr[3];
        for (int k = 0; k < 3; ++k) {
            fr[k] = (x[0] * hinv[k] + x[1] * hinv[3 + k]) + x[2] * hinv[6 + k];
            if (!isfinite(fr[k])) return OR_E_GEOM;
            mi[k] = (int)floor(fr[k]);
        }
        double s[3];
        shift_vec(h, mi[0], mi[1], mi[2], s);
        for (int d = 0; d < 3; ++d) xw[3 * i + d] = x[d] - s[d];
        for (int k = 0; k < 3; ++k) {
            fw[3 * i + k] = fr[k] - (double)mi[k];
            m[3 * i + k] = mi[k];
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------ neighbour search --- */

typedef struct {
    int64_t n_edges;
    int64_t *off;   /* n+1 */
    int32_t *j;     /* owner index of the neighbour */
    int32_t *shift; /* 3 per edge: image shift relative to the wrapped positions */
    double *r;      /* 3 per edge: r_ij = r_j + S(n) - r_i */
    double *d;      /* |r_ij| */
} edges_t;

static void edges_free(edges_t *e) {
    free(e->off);
    free(e->j);
    free(e->shift);
    free(e->r);
    free(e->d);
    memset(e, 0, sizeof(*e));
}

/* Visit every (j, n) of centre i with d^2 < r_cut^2 (brute force).  When
 * `fill` is non-zero the hits are written at position `o`; returns the count. */
static int64_t scan_centre(int64_t i, int64_t n, const double *xw, const double *fw, const double *h, int periodic,
                           const int *nmax, const double *reach, double rcut2, int fill, int64_t o, edges_t *e) {
    int64_t cnt = 0;
    for (int64_t j = 0; j < n; ++j) {
        int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        if (periodic) {
            for (int k = 0; k < 3; ++k) {
                /* |df + n_k| * w_k <= d is necessary; widen by `reach` margin */
                double df = fw[3 * j + k] - fw[3 * i + k];
                int a = (int)ceil(-reach[k] - df), b = (int)floor(reach[k] - df);
                lo[k] = a < -nmax[k] ? -nmax[k] : a;
                hi[k] = b > nmax[k] ? nmax[k] : b;
            }
        }
        for (int n0 = lo[0]; n0 <= hi[0]; ++n0)
            for (int n1 = lo[1]; n1 <= hi[1]; ++n1)
                for (int n2 = lo[2]; n2 <= hi[2]; ++n2) {
                    if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
                    double s[3] = {0.0, 0.0, 0.0}, r[3];
                    if (periodic) shift_vec(h, n0, n1, n2, s);
                    for (int d = 0; d < 3; ++d) r[d] = (xw[3 * j + d] - xw[3 * i + d]) + s[d];
                    double d2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
                    if (d2 < rcut2) {
                        if (fill) {
                            int64_t q = o + cnt;
                            e->j[q] = (int32_t)j;
                            e->shift[3 * q + 0] = n0;
                            e->shift[3 * q + 1] = n1;
                            e->shift[3 * q + 2] = n2;
                            for (int d = 0; d < 3; ++d) e->r[3 * q + d] = r[d];
                            e->d[q] = sqrt(d2);
                        }
                        ++cnt;
                    }
                }
    }
    return cnt;
}

static int build_edges(int64_t n, const double *xw, const double *fw, const double *h, double r_cut, edges_t *e) {
    int periodic = h != NULL;
    int nmax[3] = {0, 0, 0};
    double reach[3] = {0, 0, 0};
    if (periodic) {
        for (int k = 0; k < 3; ++k) {
            double w = cell_width(h, k);
            nmax[k] = (int)ceil(r_cut / w);
            reach[k] = r_cut / w + 1e-6;
        }
    }
    double rcut2 = r_cut * r_cut;
    memset(e, 0, sizeof(*e));
    e->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!e->off) return OR_E_NOMEM;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        e->off[i + 1] = scan_centre(i, n, xw, fw, h, periodic, nmax, reach, rcut2, 0, 0, e);
    for (int64_t i = 0; i < n; ++i) e->off[i + 1] += e->off[i];
    int64_t ne = e->off[n];
    e->n_edges = ne;
    size_t cap = ne > 0 ? (size_t)ne : 1;
    e->j = (int32_t *)malloc(cap * sizeof(int32_t));
    e->shift = (int32_t *)malloc(3 * cap * sizeof(int32_t));
    e->r = (double *)malloc(3 * cap * sizeof(double));
    e->d = (double *)malloc(cap * sizeof(double));
    if (!e->j || !e->shift || !e->r || !e->d) {
        edges_free(e);
        return OR_E_NOMEM;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) scan_centre(i, n, xw, fw, h, periodic, nmax, reach, rcut2, 1, e->off[i], e);
    return OR_OK;
}

static int prepare(int64_t n, const double *pos, const double *cell, double **xw, double **fw, int32_t **m) {
    *xw = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    *fw = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    *m = (int32_t *)calloc((size_t)(n > 0 ? n : 1) * 3, sizeof(int32_t));
    if (!*xw || !*fw || !*m) return OR_E_NOMEM;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(pos[i])) return OR_E_GEOM;
    if (cell) return wrap_positions(n, pos, cell, *xw, *fw, *m);
    memcpy(*xw, pos, (size_t)n * 3 * sizeof(double));
    memset(*fw, 0, (size_t)n * 3 * sizeof(double));
    return OR_OK;
}

static void set_threads(int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
}

/* All (i, j, n_caller) with d < r_cut, shifts relative to the caller's
 * (unwrapped) positions: r_j + S(n_caller) - r_i.  Order: i, then j, then the
 * shift lexicographically in the wrapped frame.  Returns the total count in
 * *count; writes at most `cap` entries; OR_E_CAP when cap is too small. */
int oracle_neighbors(int64_t n, const double *pos, const double *cell, double r_cut, int64_t cap, int32_t *out_i,
                     int32_t *out_j, int32_t *out_shift, int64_t *count, int n_threads) {
    if (n < 0 || !(r_cut > 0) || !count) return OR_E_ARG;
    set_threads(n_threads);
    double *xw = NULL, *fw = NULL;
    int32_t *m = NULL;
    int rc = prepare(n, pos, cell, &xw, &fw, &m);
    edges_t e;
    memset(&e, 0, sizeof(e));
    if (!rc) rc = build_edges(n, xw, fw, cell, r_cut, &e);
    if (!rc) {
        *count = e.n_edges;
        if (e.n_edges > cap) {
            rc = OR_E_CAP;
        } else {
            for (int64_t i = 0; i < n; ++i)
                for (int64_t q = e.off[i]; q < e.off[i + 1]; ++q) {
                    int32_t j = e.j[q];
                    out_i[q] = (int32_t)i;
                    out_j[q] = j;
                    for (int k = 0; k < 3; ++k) out_shift[3 * q + k] = e.shift[3 * q + k] - m[3 * j + k] + m[3 * i + k];
                }
        }
    }
    edges_free(&e);
    free(xw);
    free(fw);
    free(m);
    return rc;
}

/* ------------------------------------------------------------- the model --- */

typedef struct {
    int n_elem, T, n_phi, l_max, n_orb, h1, h2, n_feat, n_ang;
    int pairs;            /* 0: Eq. 1's squares; 1: products of orbital pairs k <= k' */
    double r_c, alpha;
    int lx[MAX_ANG], ly[MAX_ANG], lz[MAX_ANG], l_of[MAX_ANG];
    double wmul[MAX_ANG]; /* l! / (lx! ly! lz!) */
    double *mu;           /* n_phi Gaussian centres */
    double *c0;           /* [n_elem][n_phi] */
    double *W;            /* [T][L+1][n_phi][n_orb] */
    double **mlp;         /* [T*n_elem] -> W1 b1 W2 b2 W3 b3 packed */
} model_t;

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

static int model_init(model_t *M, int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c,
                      double alpha, int pairs, const float *params) {
    memset(M, 0, sizeof(*M));
    if (n_elem < 1 || T < 1 || n_phi < 2 || l_max < 0 || l_max > 6 || n_orb < 1 || n_orb > 64 || h1 < 1 || h2 < 1 ||
        !(r_c > 0) || !(alpha > 0) || !params || (pairs != 0 && pairs != 1))
        return OR_E_ARG;
    M->n_elem = n_elem;
    M->T = T;
    M->n_phi = n_phi;
    M->l_max = l_max;
    M->n_orb = n_orb;
    M->h1 = h1;
    M->h2 = h2;
    M->r_c = r_c;
    M->alpha = alpha;
    M->pairs = pairs;
    /* one feature per (l, orbital) for Eq. 1's squares; per (l, orbital pair k <= k') for the
       pair products, (L+1) n_orb (n_orb+1)/2 features (the count Sec. 2.1 states) */
    M->n_feat = (l_max + 1) * (pairs ? n_orb * (n_orb + 1) / 2 : n_orb);
    int a = 0;
    for (int l = 0; l <= l_max; ++l)
        for (int lx = l; lx >= 0; --lx)
            for (int ly = l - lx; ly >= 0; --ly) {
                int lz = l - lx - ly;
                M->lx[a] = lx;
                M->ly[a] = ly;
                M->lz[a] = lz;
                M->l_of[a] = l;
                M->wmul[a] = factorial(l) / (factorial(lx) * factorial(ly) * factorial(lz));
                ++a;
            }
    M->n_ang = a;
    M->mu = (double *)malloc(sizeof(double) * n_phi);
    for (int m = 0; m < n_phi; ++m) M->mu[m] = (double)m * r_c / (double)(n_phi - 1);
    size_t o = 0;
    M->c0 = (double *)malloc(sizeof(double) * n_elem * n_phi);
    for (int i = 0; i < n_elem * n_phi; ++i) M->c0[i] = (double)params[o++];
    size_t nw = (size_t)T * (l_max + 1) * n_phi * n_orb;
    M->W = (double *)malloc(sizeof(double) * nw);
    for (size_t i = 0; i < nw; ++i) M->W[i] = (double)params[o++];
    M->mlp = (double **)calloc((size_t)T * n_elem, sizeof(double *));
    for (int t = 0; t < T; ++t) {
        int out = (t == T - 1) ? 1 : n_phi;
        size_t sz = (size_t)M->n_feat * h1 + h1 + (size_t)h1 * h2 + h2 + (size_t)h2 * out + out;
        for (int e = 0; e < n_elem; ++e) {
            double *p = (double *)malloc(sizeof(double) * sz);
            for (size_t i = 0; i < sz; ++i) p[i] = (double)params[o++];
            M->mlp[t * n_elem + e] = p;
        }
    }
    return OR_OK;
}

static void model_free(model_t *M) {
    if (M->mlp)
        for (int i = 0; i < M->T * M->n_elem; ++i) free(M->mlp[i]);
    free(M->mlp);
    free(M->mu);
    free(M->c0);
    free(M->W);
}

static double ipow(double x, int p) {
    double r = 1.0;
    for (int i = 0; i < p; ++i) r *= x;
    return r;
}

/* A_a(r) = x^lx y^ly z^lz and its gradient */
static double monomial(const model_t *M, int a, const double *r) {
    return ipow(r[0], M->lx[a]) * ipow(r[1], M->ly[a]) * ipow(r[2], M->lz[a]);
}

static void monomial_grad(const model_t *M, int a, const double *r, double *g) {
    int px = M->lx[a], py = M->ly[a], pz = M->lz[a];
    g[0] = px ? px * ipow(r[0], px - 1) * ipow(r[1], py) * ipow(r[2], pz) : 0.0;
    g[1] = py ? py * ipow(r[0], px) * ipow(r[1], py - 1) * ipow(r[2], pz) : 0.0;
    g[2] = pz ? pz * ipow(r[0], px) * ipow(r[1], py) * ipow(r[2], pz - 1) : 0.0;
}

/* phi_m(d) = exp(-alpha (d-mu_m)^2) f_c(d) and d phi_m / d d */
static void radial(const model_t *M, double d, double *phi, double *dphi) {
    const double pi = 3.14159265358979323846;
    double fc = 0.0, dfc = 0.0;
    if (d < M->r_c) {
        double u = 0.5 * cos(pi * d / M->r_c) + 0.5;
        fc = u * u;
        dfc = 2.0 * u * (-0.5 * sin(pi * d / M->r_c) * pi / M->r_c);
    }
    for (int m = 0; m < M->n_phi; ++m) {
        double x = d - M->mu[m];
        double gs = exp(-M->alpha * x * x);
        phi[m] = gs * fc;
        if (dphi) dphi[m] = gs * (-2.0 * M->alpha * x) * fc + gs * dfc;
    }
}

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double dsilu(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* y = W3^T silu(W2^T silu(W1^T x + b1) + b2) + b3 ; keeps z1, z2 for the backward */
static void mlp_forward(const model_t *M, const double *p, int out, const double *x, double *z1, double *z2,
                        double *y) {
    int F = M->n_feat, H1 = M->h1, H2 = M->h2;
    const double *W1 = p, *b1 = W1 + (size_t)F * H1, *W2 = b1 + H1, *b2 = W2 + (size_t)H1 * H2, *W3 = b2 + H2,
                 *b3 = W3 + (size_t)H2 * out;
    for (int q = 0; q < H1; ++q) {
        double s = b1[q];
        for (int f = 0; f < F; ++f) s += x[f] * W1[(size_t)f * H1 + q];
        z1[q] = s;
    }
    for (int q = 0; q < H2; ++q) {
        double s = b2[q];
        for (int u = 0; u < H1; ++u) s += silu(z1[u]) * W2[(size_t)u * H2 + q];
        z2[q] = s;
    }
    for (int o = 0; o < out; ++o) {
        double s = b3[o];
        for (int u = 0; u < H2; ++u) s += silu(z2[u]) * W3[(size_t)u * out + o];
        y[o] = s;
    }
}

/* xbar = J^T ybar for the network above, at the point whose z1, z2 are given */
static void mlp_backward(const model_t *M, const double *p, int out, const double *z1, const double *z2,
                         const double *ybar, double *xbar) {
    int F = M->n_feat, H1 = M->h1, H2 = M->h2;
    const double *W1 = p, *b1 = W1 + (size_t)F * H1, *W2 = b1 + H1, *b2 = W2 + (size_t)H1 * H2, *W3 = b2 + H2;
    double z2bar[512], z1bar[512];
    for (int u = 0; u < H2; ++u) {
        double s = 0.0;
        for (int o = 0; o < out; ++o) s += W3[(size_t)u * out + o] * ybar[o];
        z2bar[u] = s * dsilu(z2[u]);
    }
    for (int u = 0; u < H1; ++u) {
        double s = 0.0;
        for (int q = 0; q < H2; ++q) s += W2[(size_t)u * H2 + q] * z2bar[q];
        z1bar[u] = s * dsilu(z1[u]);
    }
    for (int f = 0; f < F; ++f) {
        double s = 0.0;
        for (int q = 0; q < H1; ++q) s += W1[(size_t)f * H1 + q] * z1bar[q];
        xbar[f] = s;
    }
}

/* ------------------------------------------------------ energy + forces --- */

/*
 * E, F = -dE/dr, per-atom energies and (optionally) every layer's features
 * rho^t [T][n][F] and coefficients c^t [T][n][N_phi] for the model whose flat
 * parameters are `params` (layout of synth/model.py).  feature_pairs selects
 * the features: 0 for Eq. 1 (the squares of the contracted orbitals, F =
 * (L+1) n_orb), 1 for the products of orbital pairs k <= k' summed the same
 * way (F = (L+1) n_orb (n_orb+1)/2, the feature count Sec. 2.1 states).  cell == NULL means a
 * free (non-periodic) cluster.  `virial` (nullable, 3 x 3 row-major) receives
 * W_ab = -sum over edges e and layers of (dE/dr_e)_a (r_e)_b, minus the
 * derivative of E with respect to a homogeneous strain eps_ab applied to
 * positions and cell alike: E depends on positions only through the edge
 * vectors r_e of Eq. 1.  Returns OR_E_GEOM on non-finite positions, a
 * singular cell, or two atoms closer than 1e-8 A.
 */
int oracle_energy_forces(int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c,
                         double alpha, int feature_pairs, const float *params, int64_t n, const double *pos,
                         const int32_t *species, const double *cell, double *energy, double *forces,
                         double *atom_energy, double *rho_out, double *coef_out, double *virial, int n_threads) {
    if (n < 0 || !pos || !species || !energy || (n > 0 && !forces)) return OR_E_ARG;
    if (h1 > 512 || h2 > 512) return OR_E_ARG;
    set_threads(n_threads);
    model_t M;
    int rc = model_init(&M, n_elem, T, n_phi, l_max, n_orb, h1, h2, r_c, alpha, feature_pairs, params);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i)
        if (species[i] < 0 || species[i] >= n_elem) {
            model_free(&M);
            return OR_E_ARG;
        }
    double *xw = NULL, *fw = NULL;
    int32_t *mm = NULL;
    edges_t e;
    memset(&e, 0, sizeof(e));
    rc = prepare(n, pos, cell, &xw, &fw, &mm);
    if (!rc) rc = build_edges(n, xw, fw, cell, r_c, &e);
    if (!rc)
        for (int64_t q = 0; q < e.n_edges; ++q)
            if (e.d[q] < 1e-8) rc = OR_E_GEOM;
    if (rc) {
        edges_free(&e);
        free(xw);
        free(fw);
        free(mm);
        model_free(&M);
        return rc;
    }

    const int P = n_phi, A = M.n_ang, F = M.n_feat, K = n_orb;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *c = (double *)calloc((size_t)T * nn * P, sizeof(double));       /* c^t */
    double *b = (double *)calloc((size_t)T * nn * A * P, sizeof(double));   /* b^t */
    double *rho = (double *)calloc((size_t)T * nn * F, sizeof(double));     /* rho^t */
    double *z1 = (double *)calloc((size_t)T * nn * h1, sizeof(double));     /* MLP pre-activations */
    double *z2 = (double *)calloc((size_t)T * nn * h2, sizeof(double));
    double *eps = (double *)calloc(nn, sizeof(double));
    double *rhobar = (double *)calloc(nn * F, sizeof(double));
    double *bbar = (double *)calloc(nn * A * P, sizeof(double));
    double *cbar = (double *)calloc(nn * P, sizeof(double));
    double *grad = (double *)calloc(nn * 3, sizeof(double));
    if (!c || !b || !rho || !z1 || !z2 || !eps || !rhobar || !bbar || !cbar || !grad) rc = OR_E_NOMEM;

    if (virial)
        for (int k = 0; k < 9; ++k) virial[k] = 0.0;
    if (!rc) {
        /* c^0_i = c0[Z_i] */
        for (int64_t i = 0; i < n; ++i)
            for (int m = 0; m < P; ++m) c[(size_t)i * P + m] = M.c0[species[i] * P + m];

        /* forward: Eq. 1 then Eq. 2 (or the energy network at the last layer) */
        for (int t = 0; t < T; ++t) {
            double *ct = c + (size_t)t * nn * P, *bt = b + (size_t)t * nn * A * P, *rt = rho + (size_t)t * nn * F;
            const double *Wt = M.W + (size_t)t * (l_max + 1) * P * K;
#pragma omp parallel for schedule(dynamic, 16)
            for (int64_t i = 0; i < n; ++i) {
                double *bi = bt + (size_t)i * A * P;
                double phi[64];
                for (int64_t q = e.off[i]; q < e.off[i + 1]; ++q) {
                    const double *r = e.r + 3 * q;
                    int64_t j = e.j[q];
                    radial(&M, e.d[q], phi, NULL);
                    for (int a = 0; a < A; ++a) {
                        double Aa = monomial(&M, a, r);
                        for (int m = 0; m < P; ++m) bi[a * P + m] += ct[(size_t)j * P + m] * phi[m] * Aa;
                    }
                }
                double *ri = rt + (size_t)i * F;
                for (int a = 0; a < A; ++a) {
                    int l = M.l_of[a];
                    double g[64];
                    for (int k = 0; k < K; ++k) {
                        g[k] = 0.0;
                        for (int m = 0; m < P; ++m) g[k] += bi[a * P + m] * Wt[((size_t)l * P + m) * K + k];
                    }
                    if (!M.pairs) {
                        for (int k = 0; k < K; ++k) ri[l * K + k] += M.wmul[a] * g[k] * g[k];
                    } else {
                        const int KP = K * (K + 1) / 2;
                        int q = 0;
                        for (int k = 0; k < K; ++k)
                            for (int k2 = k; k2 < K; ++k2, ++q) ri[l * KP + q] += M.wmul[a] * g[k] * g[k2];
                    }
                }
                int out = (t == T - 1) ? 1 : P;
                const double *p = M.mlp[t * n_elem + species[i]];
                double y[64];
                mlp_forward(&M, p, out, ri, z1 + ((size_t)t * nn + i) * h1, z2 + ((size_t)t * nn + i) * h2, y);
                if (t < T - 1)
                    for (int m = 0; m < P; ++m) c[((size_t)(t + 1) * nn + i) * P + m] = y[m];
                else
                    eps[i] = y[0];
            }
        }
        double E = 0.0;
        for (int64_t i = 0; i < n; ++i) E += eps[i];
        *energy = E;
        if (atom_energy)
            for (int64_t i = 0; i < n; ++i) atom_energy[i] = eps[i];
        if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)T * n * F);
        if (coef_out)
            for (int t = 0; t < T; ++t) memcpy(coef_out + (size_t)t * n * P, c + (size_t)t * nn * P, sizeof(double) * n * P);

        /* reverse pass: epsbar_i = 1, rhobar^{T-1} from the energy network */
        {
            int t = T - 1;
            double one = 1.0;
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i)
                mlp_backward(&M, M.mlp[t * n_elem + species[i]], 1, z1 + ((size_t)t * nn + i) * h1,
                             z2 + ((size_t)t * nn + i) * h2, &one, rhobar + (size_t)i * F);
        }
        for (int t = T - 1; t >= 0; --t) {
            const double *ct = c + (size_t)t * nn * P, *bt = b + (size_t)t * nn * A * P;
            const double *Wt = M.W + (size_t)t * (l_max + 1) * P * K;
            /* gbar = 2 w_a g rhobar ; bbar_{a,m} = sum_k gbar_{a,k} W_{l(a),m,k} */
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                const double *bi = bt + (size_t)i * A * P;
                double *bbi = bbar + (size_t)i * A * P;
                for (int a = 0; a < A; ++a) {
                    int l = M.l_of[a];
                    double g[64];
                    for (int k = 0; k < K; ++k) {
                        g[k] = 0.0;
                        for (int m = 0; m < P; ++m) g[k] += bi[a * P + m] * Wt[((size_t)l * P + m) * K + k];
                    }
                    for (int m = 0; m < P; ++m) bbi[a * P + m] = 0.0;
                    for (int k = 0; k < K; ++k) {
                        double gbar;
                        if (!M.pairs) {
                            gbar = 2.0 * M.wmul[a] * g[k] * rhobar[(size_t)i * F + l * K + k];
                        } else {
                            /* d rho_(p,q) / d g_k = w_a (g_q [p = k] + g_p [q = k]) */
                            const int KP = K * (K + 1) / 2;
                            gbar = 0.0;
                            int q = 0;
                            for (int k1 = 0; k1 < K; ++k1)
                                for (int k2 = k1; k2 < K; ++k2, ++q) {
                                    const double rb = rhobar[(size_t)i * F + l * KP + q];
                                    if (k1 == k) gbar += rb * g[k2];
                                    if (k2 == k) gbar += rb * g[k1];
                                }
                            gbar *= M.wmul[a];
                        }
                        for (int m = 0; m < P; ++m) bbi[a * P + m] += gbar * Wt[((size_t)l * P + m) * K + k];
                    }
                }
            }
            /* edge terms: cbar_j += bbar_i phi A ; grad_j += T_ij ; grad_i -= T_ij */
            memset(cbar, 0, sizeof(double) * nn * P);
            for (int64_t i = 0; i < n; ++i) {
                const double *bbi = bbar + (size_t)i * A * P;
                double phi[64], dphi[64];
                for (int64_t q = e.off[i]; q < e.off[i + 1]; ++q) {
                    const double *r = e.r + 3 * q;
                    double d = e.d[q];
                    int64_t j = e.j[q];
                    radial(&M, d, phi, dphi);
                    double tg[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < A; ++a) {
                        double Aa = monomial(&M, a, r), gA[3];
                        monomial_grad(&M, a, r, gA);
                        for (int m = 0; m < P; ++m) {
                            double bb = bbi[a * P + m];
                            cbar[(size_t)j * P + m] += bb * phi[m] * Aa;
                            double coef = bb * ct[(size_t)j * P + m];
                            for (int k = 0; k < 3; ++k) tg[k] += coef * (dphi[m] * Aa * r[k] / d + phi[m] * gA[k]);
                        }
                    }
                    for (int k = 0; k < 3; ++k) {
                        grad[3 * j + k] += tg[k];
                        grad[3 * i + k] -= tg[k];
                    }
                    if (virial)
                        for (int a = 0; a < 3; ++a)
                            for (int bb = 0; bb < 3; ++bb) virial[3 * a + bb] -= tg[a] * r[bb];
                }
            }
            /* rhobar^{t-1} = J_{M^{t-1}}^T cbar^t (Eq. 5); c^0 is a constant */
            if (t >= 1) {
                int tp = t - 1;
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < n; ++i)
                    mlp_backward(&M, M.mlp[tp * n_elem + species[i]], P, z1 + ((size_t)tp * nn + i) * h1,
                                 z2 + ((size_t)tp * nn + i) * h2, cbar + (size_t)i * P, rhobar + (size_t)i * F);
            }
        }
        for (int64_t i = 0; i < 3 * n; ++i) forces[i] = -grad[i];
    }
    free(c);
    free(b);
    free(rho);
    free(z1);
    free(z2);
    free(eps);
    free(rhobar);
    free(bbar);
    free(cbar);
    free(grad);
    edges_free(&e);
    free(xw);
    free(fw);
    free(mm);
    model_free(&M);
    return rc;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
