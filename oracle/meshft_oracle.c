/*
 * FP64 CPU oracle for the mesh Fourier transform and its vertex adjoint.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code with the CUDA path.
 *
 * What it computes (paper: "Inverse 3D Microscopy Rendering for Cell Shape
 * Inference with Active Mesh", Sections 4.1.1-4.1.3):
 *
 *  - Triangle transform, Eq. 7-8:  u_T(xi) = int_T exp(-i x.xi) dS
 *      = 2 A_T f_T(xi),  f_T = sum_p exp(-i v_p.xi) / ((e_{p-}.xi)(e_{p+}.xi)).
 *    f_T is the second divided difference of F(x) = -exp(-i x) at the vertex
 *    phases phi_p = v_p.xi (Hermite-Genocchi: DD_m[F](x_0..x_m) =
 *    int_{simplex} F^(m)(sum lambda_k x_k) d lambda, and F'' = exp(-i x)).
 *    Eq. 8 is exactly the generic expansion of that divided difference; the
 *    paper's special cases (Eq. 12a, 12b) are its confluent limits.
 *  - Divided differences are evaluated without the paper's unstated epsilon:
 *    nodes are sorted; if their spread is below TAU_SERIES the convergent
 *    Taylor series about the node mean is summed to 1e-18 relative, otherwise
 *    the standard recursion DD[x0..xm] = (DD[x1..xm] - DD[x0..x_{m-1}]) / (xm - x0)
 *    is applied, with first-order differences in the cancellation-free form
 *    DD_1(a, b) = i exp(-i (a+b)/2) sin(d)/d, d = (a-b)/2.
 *  - Triangle gradient, Eq. 9-10: d u_T / d v_p = -f_T w_p + 2 A_T xi df/dphi_p,
 *    with df/dphi_p = DD_3[F](phi_p, phi_p, phi_q, phi_r) (the derivative of a
 *    divided difference in one node repeats that node; this equals the bracket
 *    of Eq. 10).
 *  - Volume-labelled transform (the paper names volumes as an extension,
 *    Section 3.3): int_V exp(-i x.xi) dV as a sum over signed tetrahedra
 *    (c0, v1, v2, v3) of 6 Vol_T DD_3[G](phi_c0, phi_1, phi_2, phi_3) with
 *    G = -i exp(-i x) (G''' = exp(-i x)), i.e. G = i F.
 *
 * Every routine works in plain FP64 complex arithmetic on the raw phases
 * v.xi; there is no argument reduction, blocking or reordering.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define TAU_SERIES 0.5
#define MAX_NODES 8
#define MAX_TERMS 60

/* (-i)^k */
static cplx pow_minus_i(int k) {
    switch (k & 3) {
        case 0: return 1.0;
        case 1: return -I;
        case 2: return -1.0;
        default: return I;
    }
}

static void sort_nodes(double* z, int n) {
    for (int i = 1; i < n; ++i) {
        double t = z[i];
        int j = i - 1;
        while (j >= 0 && z[j] > t) { z[j + 1] = z[j]; --j; }
        z[j + 1] = t;
    }
}

/* Series about the mean c of the m+1 nodes:
 * DD_m[F] = sum_k F^(m+k)(c) h_k(z - c) / (m+k)!,  F^(j)(c) = -(-i)^j exp(-i c),
 * h_k the complete homogeneous symmetric polynomial of degree k. */
static cplx dd_series(const double* z, int m) {
    double c = 0.0;
    for (int i = 0; i <= m; ++i) c += z[i];
    c /= (double)(m + 1);
    double y[MAX_NODES];
    for (int i = 0; i <= m; ++i) y[i] = z[i] - c;
    /* h[k] for the variables seen so far: start with y0^k, then fold in the rest. */
    double h[MAX_TERMS];
    h[0] = 1.0;
    for (int k = 1; k < MAX_TERMS; ++k) h[k] = h[k - 1] * y[0];
    for (int i = 1; i <= m; ++i)
        for (int k = 1; k < MAX_TERMS; ++k) h[k] += y[i] * h[k - 1];
    cplx sum = 0.0;
    double inv_fact = 1.0; /* 1/(m+k)! */
    for (int j = 2; j <= m; ++j) inv_fact /= (double)j;
    int small = 0;
    for (int k = 0; k < MAX_TERMS; ++k) {
        if (k > 0) inv_fact /= (double)(m + k);
        cplx term = pow_minus_i(m + k) * (h[k] * inv_fact);
        sum += term;
        if (cabs(term) < 1e-18 * cabs(sum)) {
            if (++small >= 2) break;
        } else {
            small = 0;
        }
    }
    return -cexp(-I * c) * sum;
}

/* divided difference of order m of F over sorted nodes z[0..m] */
static cplx dd_sorted(const double* z, int m) {
    if (m == 0) return -cexp(-I * z[0]);
    double spread = z[m] - z[0];
    if (spread < TAU_SERIES) return dd_series(z, m);
    if (m == 1) {
        double d = 0.5 * (z[0] - z[1]);
        return I * cexp(-I * 0.5 * (z[0] + z[1])) * (sin(d) / d);
    }
    return (dd_sorted(z + 1, m - 1) - dd_sorted(z, m - 1)) / spread;
}

/* Public: divided difference of F(x) = -exp(-i x) of order m over m+1 nodes. */
void oracle_dd(const double* nodes, int m, double* out_re, double* out_im) {
    double z[MAX_NODES];
    memcpy(z, nodes, sizeof(double) * (size_t)(m + 1));
    sort_nodes(z, m + 1);
    cplx r = dd_sorted(z, m);
    *out_re = creal(r);
    *out_im = cimag(r);
}

static cplx dd(const double* nodes, int m) {
    double z[MAX_NODES];
    memcpy(z, nodes, sizeof(double) * (size_t)(m + 1));
    sort_nodes(z, m + 1);
    return dd_sorted(z, m);
}

static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static inline void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Section 4.1.2 notation: v4 = v1, v0 = v3; e_p = v_{p-1} - v_{p+1};
 * A = |e3 x e1| / 2; N = (e3 x e1) / 2A; w_p = e_p x N (w := 0 when A = 0). */
typedef struct {
    const double* v[3];
    double e[3][3];
    double A;
    double N[3];
    double w[3][3];
} tri_geom;

static void make_geom(const double* v1, const double* v2, const double* v3, tri_geom* g) {
    g->v[0] = v1; g->v[1] = v2; g->v[2] = v3;
    sub3(v3, v2, g->e[0]); /* e1 = v0 - v2 = v3 - v2 */
    sub3(v1, v3, g->e[1]); /* e2 = v1 - v3 */
    sub3(v2, v1, g->e[2]); /* e3 = v2 - v4 = v2 - v1 */
    double n[3];
    cross3(g->e[2], g->e[0], n);
    double nn = sqrt(dot3(n, n));
    g->A = 0.5 * nn;
    for (int a = 0; a < 3; ++a) g->N[a] = nn > 0 ? n[a] / nn : 0.0;
    for (int p = 0; p < 3; ++p) {
        if (nn > 0) cross3(g->e[p], g->N, g->w[p]);
        else g->w[p][0] = g->w[p][1] = g->w[p][2] = 0.0;
    }
}

/* Eq. 7-8: u_T(xi) = 2 A_T DD_2[F](phi_1, phi_2, phi_3) */
static cplx tri_ft_surface(const tri_geom* g, const double* xi) {
    double phi[3];
    for (int p = 0; p < 3; ++p) phi[p] = dot3(g->v[p], xi);
    return 2.0 * g->A * dd(phi, 2);
}

/* signed tetrahedron (c0, v1, v2, v3): 6 Vol_T * DD_3[G], G = i F */
static cplx tet_ft(const double* c0, const tri_geom* g, const double* xi, double* vol6_out) {
    double a[3], b[3], c[3], bc[3];
    sub3(g->v[0], c0, a); sub3(g->v[1], c0, b); sub3(g->v[2], c0, c);
    cross3(b, c, bc);
    double vol6 = dot3(a, bc);
    if (vol6_out) *vol6_out = vol6;
    double nodes[4] = {dot3(c0, xi), dot3(g->v[0], xi), dot3(g->v[1], xi), dot3(g->v[2], xi)};
    return vol6 * I * dd(nodes, 3);
}

void oracle_tri_ft(const double* v1, const double* v2, const double* v3, const double* xi,
                   double* out_re, double* out_im) {
    tri_geom g;
    make_geom(v1, v2, v3, &g);
    cplx r = tri_ft_surface(&g, xi);
    *out_re = creal(r);
    *out_im = cimag(r);
}

/* Eq. 9-10: d u_T / d v_p (three complex 3-vectors, layout grad[p][axis][re,im]) */
void oracle_tri_grad(const double* v1, const double* v2, const double* v3, const double* xi, double* grad) {
    tri_geom g;
    make_geom(v1, v2, v3, &g);
    double phi[3];
    for (int p = 0; p < 3; ++p) phi[p] = dot3(g.v[p], xi);
    cplx f = dd(phi, 2);
    for (int p = 0; p < 3; ++p) {
        double nodes[4] = {phi[p], phi[p], phi[(p + 1) % 3], phi[(p + 2) % 3]};
        cplx D = dd(nodes, 3);
        for (int a = 0; a < 3; ++a) {
            cplx v = -f * g.w[p][a] + 2.0 * g.A * xi[a] * D;
            grad[(p * 3 + a) * 2 + 0] = creal(v);
            grad[(p * 3 + a) * 2 + 1] = cimag(v);
        }
    }
}

/*
 * Mesh spectrum S(xi_m) = sum_T rho_T u_T(xi_m) (mode 0, surface; Eq. 5 numerator with the
 * per-triangle fluorophore density rho_T of Section 3.3, wts == NULL meaning 1) or
 * sum_T of the signed tetrahedra (mode 1, volume), at M wavevectors xi[M][3].
 * V[n_v][3], F[n_t][3] (0-based), c0 the tetrahedra apex. Output S[M][2].
 */
void oracle_mesh_ft(int mode, const double* V, int64_t n_v, const int32_t* F, int64_t n_t,
                    const double* xi, int64_t M, const double* c0, const double* wts, double* S) {
    (void)n_v;
    tri_geom* G = (tri_geom*)malloc(sizeof(tri_geom) * (size_t)(n_t > 0 ? n_t : 1));
    for (int64_t t = 0; t < n_t; ++t)
        make_geom(V + 3 * F[3 * t], V + 3 * F[3 * t + 1], V + 3 * F[3 * t + 2], &G[t]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        cplx acc = 0.0;
        for (int64_t t = 0; t < n_t; ++t)
            acc += mode == 0 ? (wts ? wts[t] : 1.0) * tri_ft_surface(&G[t], xi + 3 * m)
                             : tet_ft(c0, &G[t], xi + 3 * m, NULL);
        S[2 * m] = creal(acc);
        S[2 * m + 1] = cimag(acc);
    }
    free(G);
}

/*
 * Vertex adjoint of the mesh spectrum: dV[v][a] = sum_m Re(conj(Gs_m) dS_m / dv_a)
 * for the same modes as oracle_mesh_ft. Gs[M][2]. Output dV[n_v][3] (overwritten).
 * Per-triangle sums run in parallel over triangles, then scatter serially, so the
 * result is independent of the thread count.
 */
void oracle_mesh_ft_adjoint(int mode, const double* V, int64_t n_v, const int32_t* F, int64_t n_t,
                            const double* xi, int64_t M, const double* Gs, const double* c0, const double* wts,
                            double* dV) {
    double* acc = (double*)calloc((size_t)(n_t > 0 ? n_t : 1) * 9, sizeof(double));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_t; ++t) {
        tri_geom g;
        make_geom(V + 3 * F[3 * t], V + 3 * F[3 * t + 1], V + 3 * F[3 * t + 2], &g);
        double loc[9] = {0};
        for (int64_t m = 0; m < M; ++m) {
            const double* x = xi + 3 * m;
            cplx Gc = conj(Gs[2 * m] + I * Gs[2 * m + 1]);
            if (mode == 0) {
                double phi[3];
                for (int p = 0; p < 3; ++p) phi[p] = dot3(g.v[p], x);
                cplx f = dd(phi, 2);
                for (int p = 0; p < 3; ++p) {
                    double nodes[4] = {phi[p], phi[p], phi[(p + 1) % 3], phi[(p + 2) % 3]};
                    cplx D = dd(nodes, 3);
                    for (int a = 0; a < 3; ++a)
                        loc[3 * p + a] += creal(Gc * (-f * g.w[p][a] + 2.0 * g.A * x[a] * D));
                }
            } else {
                /* d/dv_p of 6 Vol_T i DD_3[F](phi_c0, phi_1, phi_2, phi_3):
                 * 6 dVol_T/dv_p i DD_3 + 6 Vol_T i xi DD_4(..., phi_p repeated). */
                double a[3], b[3], c[3], tmp[3];
                sub3(g.v[0], c0, a); sub3(g.v[1], c0, b); sub3(g.v[2], c0, c);
                cross3(b, c, tmp);
                double vol6 = dot3(a, tmp);
                double dvol6[3][3];
                cross3(b, c, dvol6[0]);
                cross3(c, a, dvol6[1]);
                cross3(a, b, dvol6[2]);
                double nodes[5] = {dot3(c0, x), dot3(g.v[0], x), dot3(g.v[1], x), dot3(g.v[2], x), 0.0};
                cplx d3 = I * dd(nodes, 3);
                for (int p = 0; p < 3; ++p) {
                    nodes[4] = nodes[1 + p];
                    cplx d4 = I * dd(nodes, 4);
                    for (int k = 0; k < 3; ++k)
                        loc[3 * p + k] += creal(Gc * (dvol6[p][k] * d3 + vol6 * x[k] * d4));
                }
            }
        }
        const double rho = (mode == 0 && wts) ? wts[t] : 1.0;
        for (int k = 0; k < 9; ++k) acc[9 * t + k] = rho * loc[k];
    }
    memset(dV, 0, sizeof(double) * (size_t)n_v * 3);
    for (int64_t t = 0; t < n_t; ++t)
        for (int p = 0; p < 3; ++p)
            for (int a = 0; a < 3; ++a) dV[3 * F[3 * t + p] + a] += acc[9 * t + 3 * p + a];
    free(acc);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
