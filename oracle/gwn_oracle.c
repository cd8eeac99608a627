/*
 * gwn_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU evaluation of the exact generalized winding number
 * (GWN) of a collection of NURBS curves in 2D or trimmed NURBS patches in 3D,
 * summed directly over every input primitive without subdivision.  This is
 * the "direct" evaluation against which the paper measures the precision of
 * its accelerated method (Section 4.2), and it follows the GWN definition of
 * Eq. 1 / Eq. 2 (Section 2.1).  Only the test-suite, the package smoke check
 * and the benchmark's CPU-baseline leg load this library; the product path
 * (the CUDA library) never does, and the two share no code.
 *
 * Conventions (the paper fixes only the normalisation through Eq. 2):
 *   2D  w_C(q) = (1/2pi) * (signed angle swept by C(t) - q); a counter-
 *       clockwise loop gives +1 inside.
 *   3D  w_S(q) = (1/4pi) * integral over the visible surface of
 *       (x - q) . (S_u x S_v) / |x - q|^3 du dv; outward normals give +1
 *       inside a closed shell.  The visible part of a trimmed patch is counted
 *       with the winding number of its trimming loops in (u, v).
 *
 * 2D algorithm (per rational Bezier piece after Bezier extraction):
 *   w_piece = phi / 2pi + k, phi = principal angle of the chord P0 -> Pp seen
 *   from q, k = winding number of the closed loop "piece followed by the
 *   reversed chord", counted by signed crossings of a ray from q.  Curve
 *   crossings are the roots of a Bernstein polynomial, isolated by de
 *   Casteljau halving and refined by bisection.
 *
 * 3D algorithm (per trimmed patch), a Stokes reduction of Eq. 2:
 *   choose a unit vector s; A_s(r) = (s x r) / (|r| (|r| + s . r)) has
 *   curl A_s = r / |r|^3 away from the half line {q - t s, t > 0}.  Then
 *     w_S(q) = (1/4pi) oint_{dS} A_s(x - q) . dx  -  sum_hits wind(u,v) sign(s . n)
 *   where the hits are the crossings of that half line with the surface.  The
 *   line integral runs over the trimming curves mapped through S (adaptive
 *   Gauss-Legendre); hits are found by recursive subdivision of the Bezier
 *   sub-patches and Newton's method.  When q is outside the control-net
 *   bounding box, s is taken from q towards the box centre, so the half line
 *   cannot meet the patch (it points away from a convex set containing it).
 *
 * Results for queries closer than `near_thr` to the geometry are flagged; a
 * query lying on the geometry returns NaN.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXDEG 9
#define OR_PI 3.14159265358979323846

enum { ORF_NEAR = 1, ORF_ON_BOUNDARY = 2, ORF_DEGENERATE = 4, ORF_NOT_CONVERGED = 8 };

/* ------------------------------------------------------------------ basics */

static void bernstein(int p, double s, double* B) {
    /* all degree-p Bernstein polynomials at s (triangular recurrence) */
    B[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        double saved = 0.0;
        for (int k = 0; k < j; ++k) {
            double tmp = B[k];
            B[k] = saved + (1.0 - s) * tmp;
            saved = s * tmp;
        }
        B[j] = saved;
    }
}

static void bernstein_d(int p, double s, double* B, double* dB) {
    /* values and first derivatives of the degree-p Bernstein polynomials */
    double Bm[OR_MAXDEG + 1];
    bernstein(p, s, B);
    if (p == 0) { dB[0] = 0.0; return; }
    bernstein(p - 1, s, Bm);
    for (int i = 0; i <= p; ++i) {
        double a = (i > 0) ? Bm[i - 1] : 0.0;
        double b = (i < p) ? Bm[i] : 0.0;
        dB[i] = p * (a - b);
    }
}

/* Gauss-Legendre nodes/weights on [0, 1] computed by Newton's method on P_n. */
#define OR_GLN 16
static double g_glx[OR_GLN], g_glw[OR_GLN];
static int g_gl_ready = 0;

static void gauss_legendre(int n, double* x01, double* w01) {
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x01[i] = 0.5 * (1.0 - z);
        w01[i] = 1.0 / ((1.0 - z * z) * pp * pp);  /* = 2/((1-z^2)p'^2) / 2 */
    }
}

static void gl_init(void) {
    if (!g_gl_ready) {
        gauss_legendre(OR_GLN, g_glx, g_glw);
        g_gl_ready = 1;
    }
}

/* ------------------------------------------------------------------ records */

typedef struct {               /* rational Bezier piece in homogeneous 2D */
    int p;
    double h[OR_MAXDEG + 1][3];  /* (w x, w y, w) */
} bez2;

typedef struct {               /* rational Bezier sub-patch in homogeneous 3D */
    int du, dv;
    double u0, u1, v0, v1;       /* global parameter rectangle */
    double h[OR_MAXDEG + 1][OR_MAXDEG + 1][4];
} bez3;

typedef struct {
    int nsu, nsv;                /* grid of Bezier sub-patches */
    double* ub;                  /* nsu + 1 breakpoints */
    double* vb;                  /* nsv + 1 breakpoints */
    bez3* sub;                   /* nsu * nsv, index iu * nsv + iv */
    int n_tp;                    /* boundary pieces in (u, v) */
    bez2* tp;
    int untrimmed;
    double lo[3], hi[3], diag;   /* control-net box */
} opatch;

/* Boehm knot insertion on points of dimension `dim`.  P has n points, U has
 * n + p + 1 knots; on return both have one more entry. */
static void insert_knot(int p, int* n, double* U, int dim, double* P, double t) {
    int nn = *n;
    int k = p;
    while (k + 1 < nn && U[k + 1] <= t) ++k;
    double* Q = (double*)malloc(sizeof(double) * (size_t)(nn + 1) * dim);
    for (int i = 0; i <= k - p; ++i) memcpy(Q + (size_t)i * dim, P + (size_t)i * dim, sizeof(double) * dim);
    for (int i = k - p + 1; i <= k; ++i) {
        double den = U[i + p] - U[i];
        double a = den > 0 ? (t - U[i]) / den : 0.0;
        for (int d = 0; d < dim; ++d)
            Q[(size_t)i * dim + d] = (1.0 - a) * P[(size_t)(i - 1) * dim + d] + a * P[(size_t)i * dim + d];
    }
    for (int i = k + 1; i <= nn; ++i) memcpy(Q + (size_t)i * dim, P + (size_t)(i - 1) * dim, sizeof(double) * dim);
    memcpy(P, Q, sizeof(double) * (size_t)(nn + 1) * dim);
    free(Q);
    for (int j = nn + p; j > k; --j) U[j + 1] = U[j];
    U[k + 1] = t;
    *n = nn + 1;
}

/* Bezier extraction of a clamped B-spline with points of dimension dim.
 * Returns the number of pieces; *pts receives (pieces * p + 1) points and
 * *brk the pieces + 1 breakpoints.  Returns -1 if the knots are not clamped
 * or not non-decreasing. */
static int extract(int p, int n, const double* Uin, int dim, const double* Pin, double** pts, double** brk) {
    int m = n + p + 1;
    for (int i = 0; i + 1 < m; ++i)
        if (Uin[i + 1] < Uin[i]) return -1;
    for (int i = 1; i <= p; ++i)
        if (Uin[i] != Uin[0] || Uin[m - 1 - i] != Uin[m - 1]) return -1;
    if (!(Uin[m - 1] > Uin[0])) return -1;
    /* worst case: every interior knot raised to multiplicity p */
    int cap = n + (n + 1) * p + 4;
    double* U = (double*)malloc(sizeof(double) * (size_t)(cap + p + 2));
    double* P = (double*)malloc(sizeof(double) * (size_t)cap * dim);
    memcpy(U, Uin, sizeof(double) * m);
    memcpy(P, Pin, sizeof(double) * (size_t)n * dim);
    int nn = n;
    int i = p + 1;
    while (i < nn) {
        double t = U[i];
        int mult = 0;
        while (i + mult < nn && U[i + mult] == t) ++mult;
        if (mult > p) { free(U); free(P); return -1; }  /* discontinuous: not supported */
        for (int r = mult; r < p; ++r) insert_knot(p, &nn, U, dim, P, t);
        /* skip the (now p-fold) knot */
        i += (mult < p ? p : mult);
    }
    int pieces = (nn - 1) / p;
    double* b = (double*)malloc(sizeof(double) * (pieces + 1));
    b[0] = U[p];
    for (int j = 1; j <= pieces; ++j) b[j] = U[p + j * p];
    *pts = P;
    *brk = b;
    free(U);
    return pieces;
}

/* ------------------------------------------------------------------ parsing */

typedef struct {
    int n_pieces;
    bez2* pieces;
} ocurve;

static const double* parse_curve(const double* r, const double* end, ocurve* out, int* err) {
    if (end - r < 2) { *err = 1; return end; }
    int p = (int)r[0], n = (int)r[1];
    r += 2;
    if (p < 1 || p > OR_MAXDEG || n < p + 1 || end - r < (long)(2 * n + n + n + p + 1)) { *err = 1; return end; }
    const double* ctrl = r;
    const double* w = r + 2 * n;
    const double* U = w + n;
    double* H = (double*)malloc(sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i) {
        if (!(w[i] > 0)) *err = 1;
        H[3 * i + 0] = w[i] * ctrl[2 * i];
        H[3 * i + 1] = w[i] * ctrl[2 * i + 1];
        H[3 * i + 2] = w[i];
    }
    double *pts = NULL, *brk = NULL;
    int pieces = extract(p, n, U, 3, H, &pts, &brk);
    free(H);
    if (pieces < 1) { *err = 1; out->n_pieces = 0; out->pieces = NULL; return U + n + p + 1; }
    out->n_pieces = pieces;
    out->pieces = (bez2*)calloc(pieces, sizeof(bez2));
    for (int j = 0; j < pieces; ++j) {
        out->pieces[j].p = p;
        for (int i = 0; i <= p; ++i)
            for (int d = 0; d < 3; ++d) out->pieces[j].h[i][d] = pts[(size_t)(j * p + i) * 3 + d];
    }
    free(pts);
    free(brk);
    return U + n + p + 1;
}

static void free_patch(opatch* P) {
    free(P->ub); free(P->vb); free(P->sub); free(P->tp);
}

static const double* parse_patch(const double* r, const double* end, opatch* P, int* err) {
    memset(P, 0, sizeof(*P));
    if (end - r < 4) { *err = 1; return end; }
    int du = (int)r[0], dv = (int)r[1], nu = (int)r[2], nv = (int)r[3];
    r += 4;
    if (du < 1 || dv < 1 || du > OR_MAXDEG || dv > OR_MAXDEG || nu < du + 1 || nv < dv + 1) { *err = 1; return end; }
    const double* ctrl = r;
    const double* w = ctrl + 3 * nu * nv;
    const double* Ku = w + nu * nv;
    const double* Kv = Ku + nu + du + 1;
    r = Kv + nv + dv + 1;
    if (r > end) { *err = 1; return end; }
    /* extraction in u: each point is a whole v-row of homogeneous 4-vectors */
    int dimu = 4 * nv;
    double* H = (double*)malloc(sizeof(double) * (size_t)nu * dimu);
    for (int i = 0; i < nu; ++i)
        for (int j = 0; j < nv; ++j) {
            double ww = w[i * nv + j];
            if (!(ww > 0)) *err = 1;
            for (int d = 0; d < 3; ++d) H[(size_t)i * dimu + 4 * j + d] = ww * ctrl[3 * (i * nv + j) + d];
            H[(size_t)i * dimu + 4 * j + 3] = ww;
        }
    double *pu = NULL, *bu = NULL;
    int su = extract(du, nu, Ku, dimu, H, &pu, &bu);
    free(H);
    if (su < 1) { *err = 1; return end; }
    int nu2 = su * du + 1;
    /* extraction in v of every u-control row */
    double *pv0 = NULL, *bv = NULL;
    int sv = -1;
    double* all = NULL;
    for (int i = 0; i < nu2; ++i) {
        double *pv = NULL, *b = NULL;
        int s = extract(dv, nv, Kv, 4, pu + (size_t)i * dimu, &pv, &b);
        if (s < 1) { *err = 1; free(pu); free(bu); free(all); return end; }
        if (sv < 0) {
            sv = s;
            bv = b;
            all = (double*)malloc(sizeof(double) * (size_t)nu2 * (sv * dv + 1) * 4);
        } else {
            free(b);
        }
        memcpy(all + (size_t)i * (sv * dv + 1) * 4, pv, sizeof(double) * (size_t)(sv * dv + 1) * 4);
        free(pv);
    }
    (void)pv0;
    int nv2 = sv * dv + 1;
    P->nsu = su;
    P->nsv = sv;
    P->ub = bu;
    P->vb = bv;
    P->sub = (bez3*)calloc((size_t)su * sv, sizeof(bez3));
    for (int a = 0; a < su; ++a)
        for (int b = 0; b < sv; ++b) {
            bez3* S = &P->sub[a * sv + b];
            S->du = du; S->dv = dv;
            S->u0 = bu[a]; S->u1 = bu[a + 1]; S->v0 = bv[b]; S->v1 = bv[b + 1];
            for (int i = 0; i <= du; ++i)
                for (int j = 0; j <= dv; ++j)
                    for (int d = 0; d < 4; ++d)
                        S->h[i][j][d] = all[((size_t)(a * du + i) * nv2 + (b * dv + j)) * 4 + d];
        }
    free(all);
    free(pu);
    /* control-net bounding box */
    for (int d = 0; d < 3; ++d) { P->lo[d] = 1e300; P->hi[d] = -1e300; }
    for (int i = 0; i < nu * nv; ++i)
        for (int d = 0; d < 3; ++d) {
            double x = ctrl[3 * i + d];
            if (x < P->lo[d]) P->lo[d] = x;
            if (x > P->hi[d]) P->hi[d] = x;
        }
    P->diag = sqrt((P->hi[0] - P->lo[0]) * (P->hi[0] - P->lo[0]) + (P->hi[1] - P->lo[1]) * (P->hi[1] - P->lo[1]) +
                   (P->hi[2] - P->lo[2]) * (P->hi[2] - P->lo[2]));
    /* trimming curves */
    if (r >= end) { *err = 1; return end; }
    int nt = (int)r[0];
    r += 1;
    if (nt == 0) {
        /* untrimmed: the parameter rectangle, counter-clockwise */
        double U0 = Ku[0], U1 = Ku[nu + du], V0 = Kv[0], V1 = Kv[nv + dv];
        double c[5][2] = {{U0, V0}, {U1, V0}, {U1, V1}, {U0, V1}, {U0, V0}};
        P->untrimmed = 1;
        P->n_tp = 4;
        P->tp = (bez2*)calloc(4, sizeof(bez2));
        for (int e = 0; e < 4; ++e) {
            P->tp[e].p = 1;
            for (int k = 0; k < 2; ++k) {
                P->tp[e].h[k][0] = c[e + k][0];
                P->tp[e].h[k][1] = c[e + k][1];
                P->tp[e].h[k][2] = 1.0;
            }
        }
        return r;
    }
    int cap = 0, cnt = 0;
    bez2* tp = NULL;
    for (int t = 0; t < nt; ++t) {
        ocurve oc;
        r = parse_curve(r, end, &oc, err);
        if (*err) { free(tp); free(oc.pieces); return end; }
        if (cnt + oc.n_pieces > cap) {
            cap = 2 * (cnt + oc.n_pieces) + 8;
            tp = (bez2*)realloc(tp, sizeof(bez2) * cap);
        }
        memcpy(tp + cnt, oc.pieces, sizeof(bez2) * oc.n_pieces);
        cnt += oc.n_pieces;
        free(oc.pieces);
    }
    P->n_tp = cnt;
    P->tp = tp;
    return r;
}

/* ------------------------------------------------------------------ 2D */

static void bez2_eval(const bez2* c, double s, double* x, double* dx) {
    double B[OR_MAXDEG + 1], dB[OR_MAXDEG + 1];
    bernstein_d(c->p, s, B, dB);
    double H[3] = {0, 0, 0}, D[3] = {0, 0, 0};
    for (int i = 0; i <= c->p; ++i)
        for (int d = 0; d < 3; ++d) {
            H[d] += B[i] * c->h[i][d];
            D[d] += dB[i] * c->h[i][d];
        }
    x[0] = H[0] / H[2];
    x[1] = H[1] / H[2];
    if (dx) {
        dx[0] = (D[0] - x[0] * D[2]) / H[2];
        dx[1] = (D[1] - x[1] * D[2]) / H[2];
    }
}

static void bez2_split(const bez2* c, double s, bez2* L, bez2* R) {
    /* de Casteljau split of the homogeneous control polygon at s */
    double T[OR_MAXDEG + 1][3];
    int p = c->p;
    memcpy(T, c->h, sizeof(T));
    L->p = R->p = p;
    for (int d = 0; d < 3; ++d) { L->h[0][d] = T[0][d]; R->h[p][d] = T[p][d]; }
    for (int j = 1; j <= p; ++j) {
        for (int i = 0; i <= p - j; ++i)
            for (int d = 0; d < 3; ++d) T[i][d] = (1.0 - s) * T[i][d] + s * T[i + 1][d];
        for (int d = 0; d < 3; ++d) { L->h[j][d] = T[0][d]; R->h[p - j][d] = T[p - j][d]; }
    }
}

/* Real roots in (0,1) of a Bernstein polynomial with coefficients c[0..p]
 * located on global sub-interval [a,b].  Each isolated simple root is
 * reported with the sign of the polynomial's slope there.  Returns -1 if a
 * root could not be isolated (tangency / root at a subdivision point). */
static int bern_roots(int p, const double* c, double a, double b, int depth, double* roots, int* signs, int cap,
                      int* count) {
    int var = 0, nz = 0;
    double scale = 0;
    for (int i = 0; i <= p; ++i) scale = fmax(scale, fabs(c[i]));
    if (scale == 0.0) return -1;
    for (int i = 0; i <= p; ++i) if (c[i] == 0.0) ++nz;
    if (nz) return -1;
    for (int i = 0; i < p; ++i)
        if ((c[i] < 0) != (c[i + 1] < 0)) ++var;
    if (var == 0) return 0;
    if (var == 1 && ((c[0] < 0) != (c[p] < 0))) {
        /* exactly one simple root: bisection on the polynomial value */
        double lo = 0.0, hi = 1.0, flo = c[0];
        double B[OR_MAXDEG + 1];
        for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
            double m = 0.5 * (lo + hi), f = 0;
            bernstein(p, m, B);
            for (int i = 0; i <= p; ++i) f += B[i] * c[i];
            if (f == 0.0) { lo = hi = m; break; }
            if ((f < 0) == (flo < 0)) { lo = m; flo = f; } else hi = m;
        }
        if (*count >= cap) return -1;
        roots[*count] = a + (b - a) * 0.5 * (lo + hi);
        signs[*count] = (c[p] > 0) ? 1 : -1;
        ++*count;
        return 0;
    }
    if (depth > 60 || b - a < 1e-14) return -1;
    /* split at the middle */
    double T[OR_MAXDEG + 1], Lc[OR_MAXDEG + 1], Rc[OR_MAXDEG + 1];
    memcpy(T, c, sizeof(double) * (p + 1));
    Lc[0] = T[0];
    Rc[p] = T[p];
    for (int j = 1; j <= p; ++j) {
        for (int i = 0; i <= p - j; ++i) T[i] = 0.5 * (T[i] + T[i + 1]);
        Lc[j] = T[0];
        Rc[p - j] = T[p - j];
    }
    double m = 0.5 * (a + b);
    if (Lc[p] == 0.0) return -1;  /* root exactly at the split point */
    if (bern_roots(p, Lc, a, m, depth + 1, roots, signs, cap, count) < 0) return -1;
    return bern_roots(p, Rc, m, b, depth + 1, roots, signs, cap, count);
}

/* GWN of one rational Bezier piece, ray direction d.  Return codes: 0 ok,
 * 1 degenerate ray (try another d), 2 q on the curve, 3 q on the chord. */
static int piece_gwn_ray(const bez2* c, const double* q, const double* d, double* out) {
    int p = c->p;
    double P0[2] = {c->h[0][0] / c->h[0][2], c->h[0][1] / c->h[0][2]};
    double Pp[2] = {c->h[p][0] / c->h[p][2], c->h[p][1] / c->h[p][2]};
    double a[2] = {P0[0] - q[0], P0[1] - q[1]};
    double b[2] = {Pp[0] - q[0], Pp[1] - q[1]};
    double cr = a[0] * b[1] - a[1] * b[0], dt = a[0] * b[0] + a[1] * b[1];
    double la = hypot(a[0], a[1]), lb = hypot(b[0], b[1]);
    if (la == 0.0 || lb == 0.0) return 2;
    if (fabs(cr) <= 1e-12 * la * lb && dt < 0) return 3;
    double phi = atan2(cr, dt);
    double dp[2] = {-d[1], d[0]};
    double coef[OR_MAXDEG + 1];
    for (int i = 0; i <= p; ++i)
        coef[i] = dp[0] * (c->h[i][0] - c->h[i][2] * q[0]) + dp[1] * (c->h[i][1] - c->h[i][2] * q[1]);
    double roots[4 * OR_MAXDEG + 4];
    int signs[4 * OR_MAXDEG + 4], nr = 0;
    if (bern_roots(p, coef, 0.0, 1.0, 0, roots, signs, 4 * OR_MAXDEG + 4, &nr) < 0) return 1;
    int k = 0;
    double scale = la + lb;
    for (int r = 0; r < nr; ++r) {
        if (roots[r] < 1e-12 || roots[r] > 1.0 - 1e-12) return 1;
        double x[2];
        bez2_eval(c, roots[r], x, NULL);
        double along = d[0] * (x[0] - q[0]) + d[1] * (x[1] - q[1]);
        if (fabs(along) < 1e-14 * scale) return 2;
        if (along > 0) k += signs[r];
    }
    /* the closing chord, from Pp back to P0 */
    double g0 = dp[0] * b[0] + dp[1] * b[1];
    double g1 = dp[0] * a[0] + dp[1] * a[1];
    if (g0 == 0.0 || g1 == 0.0) return 1;
    if ((g0 < 0) != (g1 < 0)) {
        double lam = g0 / (g0 - g1);
        double X[2] = {b[0] + lam * (a[0] - b[0]), b[1] + lam * (a[1] - b[1])};
        double along = d[0] * X[0] + d[1] * X[1];
        if (fabs(along) < 1e-14 * scale) return 1;
        if (along > 0) k += (g1 > g0) ? 1 : -1;
    }
    *out = phi / (2.0 * OR_PI) + (double)k;
    return 0;
}

/* GWN of a piece, retrying ray directions and splitting when q sits on the chord. */
static double piece_gwn(const bez2* c, const double* q, int depth, int* flags) {
    double val = 0.0;
    for (int attempt = 0; attempt < 64; ++attempt) {
        double ang = 0.3 + 2.399963229728653 * attempt;  /* golden-angle sequence */
        double d[2] = {cos(ang), sin(ang)};
        int st = piece_gwn_ray(c, q, d, &val);
        if (st == 0) return val;
        if (st == 2) { *flags |= ORF_ON_BOUNDARY; return NAN; }
        if (st == 3) {
            if (depth > 50) { *flags |= ORF_ON_BOUNDARY; return NAN; }
            bez2 L, R;
            bez2_split(c, 0.5, &L, &R);
            return piece_gwn(&L, q, depth + 1, flags) + piece_gwn(&R, q, depth + 1, flags);
        }
    }
    *flags |= ORF_DEGENERATE;
    return NAN;
}

static int piece_near(const bez2* c, const double* q, double thr, int depth) {
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    for (int i = 0; i <= c->p; ++i)
        for (int d = 0; d < 2; ++d) {
            double x = c->h[i][d] / c->h[i][2];
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
    for (int d = 0; d < 2; ++d)
        if (q[d] < lo[d] - thr || q[d] > hi[d] + thr) return 0;
    if (hypot(hi[0] - lo[0], hi[1] - lo[1]) < thr || depth > 60) return 1;
    bez2 L, R;
    bez2_split(c, 0.5, &L, &R);
    return piece_near(&L, q, thr, depth + 1) || piece_near(&R, q, thr, depth + 1);
}

/* ------------------------------------------------------------------ 3D surface */

static const bez3* find_sub(const opatch* P, double u, double v) {
    int a = 0, b = 0;
    while (a + 1 < P->nsu && u >= P->ub[a + 1]) ++a;
    while (b + 1 < P->nsv && v >= P->vb[b + 1]) ++b;
    return &P->sub[a * P->nsv + b];
}

/* S, S_u, S_v at global (u, v). */
static void surf_eval(const opatch* P, double u, double v, double* S, double* Su, double* Sv) {
    const bez3* B = find_sub(P, u, v);
    double hu = B->u1 - B->u0, hv = B->v1 - B->v0;
    double s = (u - B->u0) / hu, t = (v - B->v0) / hv;
    double Bu[OR_MAXDEG + 1], dBu[OR_MAXDEG + 1], Bv[OR_MAXDEG + 1], dBv[OR_MAXDEG + 1];
    bernstein_d(B->du, s, Bu, dBu);
    bernstein_d(B->dv, t, Bv, dBv);
    double H[4] = {0, 0, 0, 0}, Hs[4] = {0, 0, 0, 0}, Ht[4] = {0, 0, 0, 0};
    for (int i = 0; i <= B->du; ++i)
        for (int j = 0; j <= B->dv; ++j)
            for (int d = 0; d < 4; ++d) {
                double h = B->h[i][j][d];
                H[d] += Bu[i] * Bv[j] * h;
                Hs[d] += dBu[i] * Bv[j] * h;
                Ht[d] += Bu[i] * dBv[j] * h;
            }
    for (int d = 0; d < 3; ++d) S[d] = H[d] / H[3];
    if (Su) {
        for (int d = 0; d < 3; ++d) {
            Su[d] = (Hs[d] - S[d] * Hs[3]) / H[3] / hu;
            Sv[d] = (Ht[d] - S[d] * Ht[3]) / H[3] / hv;
        }
    }
}

static void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* integrand of the Stokes line integral at parameter tau of trim piece c */
static double stokes_integrand(const opatch* P, const bez2* c, double tau, const double* q, const double* s) {
    double uv[2], duv[2], S[3], Su[3], Sv[3];
    bez2_eval(c, tau, uv, duv);
    surf_eval(P, uv[0], uv[1], S, Su, Sv);
    double r[3] = {S[0] - q[0], S[1] - q[1], S[2] - q[2]};
    double dx[3] = {Su[0] * duv[0] + Sv[0] * duv[1], Su[1] * duv[0] + Sv[1] * duv[1], Su[2] * duv[0] + Sv[2] * duv[1]};
    double rn = norm3(r);
    double sr[3];
    cross3(s, r, sr);
    double den = rn * (rn + dot3(s, r));
    return dot3(sr, dx) / den;
}

static double gl_panel(const opatch* P, const bez2* c, double a, double b, const double* q, const double* s) {
    double acc = 0.0;
    for (int i = 0; i < OR_GLN; ++i) acc += g_glw[i] * stokes_integrand(P, c, a + (b - a) * g_glx[i], q, s);
    return acc * (b - a);
}

static double adapt(const opatch* P, const bez2* c, double a, double b, double whole, const double* q,
                    const double* s, double tol, int depth, int* flags) {
    double m = 0.5 * (a + b);
    double L = gl_panel(P, c, a, m, q, s), R = gl_panel(P, c, m, b, q, s);
    double err = fabs(L + R - whole);
    /* accept at the requested tolerance, or once the difference is at roundoff level */
    if (err <= tol || err <= 1e-14 * (fabs(L) + fabs(R))) return L + R;
    if (depth >= 40) { *flags |= ORF_NOT_CONVERGED; return L + R; }
    double t2 = fmax(0.5 * tol, 1e-17);
    return adapt(P, c, a, m, L, q, s, t2, depth + 1, flags) + adapt(P, c, m, b, R, q, s, t2, depth + 1, flags);
}

static double line_integral(const opatch* P, const double* q, const double* s, int* flags) {
    double acc = 0.0;
    for (int k = 0; k < P->n_tp; ++k) {
        double whole = gl_panel(P, &P->tp[k], 0.0, 1.0, q, s);
        acc += adapt(P, &P->tp[k], 0.0, 1.0, whole, q, s, 1e-13, 0, flags);
    }
    return acc;
}

/* winding number (integer) of the trimming loops at (u, v); -1000 if (u, v) is on a loop */
static int trim_winding(const opatch* P, double u, double v) {
    double q[2] = {u, v};
    if (P->untrimmed) {
        double U0 = P->ub[0], U1 = P->ub[P->nsu], V0 = P->vb[0], V1 = P->vb[P->nsv];
        double e = 1e-10 * (U1 - U0 + V1 - V0);
        if (u < U0 - e || u > U1 + e || v < V0 - e || v > V1 + e) return 0;
        if (fabs(u - U0) < e || fabs(u - U1) < e || fabs(v - V0) < e || fabs(v - V1) < e) return -1000;
        return 1;
    }
    double acc = 0.0;
    int fl = 0;
    for (int k = 0; k < P->n_tp; ++k) {
        if (piece_near(&P->tp[k], q, 1e-10, 0)) return -1000;
        acc += piece_gwn(&P->tp[k], q, 0, &fl);
    }
    if (fl) return -1000;
    return (int)lround(acc);
}

/* solve the 3x3 system [a b c] x = r by Cramer's rule */
static int solve3(const double* a, const double* b, const double* c, const double* r, double* x) {
    double bc[3], ca[3], ab[3];
    cross3(b, c, bc);
    cross3(c, a, ca);
    cross3(a, b, ab);
    double det = dot3(a, bc);
    if (det == 0.0 || !isfinite(det)) return -1;
    x[0] = dot3(r, bc) / det;
    x[1] = dot3(r, ca) / det;
    x[2] = dot3(r, ab) / det;
    return 0;
}

typedef struct {
    double u, v, t, x[3], n[3];
} ohit;

static void bez3_split(const bez3* B, int dir, bez3* L, bez3* R) {
    *L = *B;
    *R = *B;
    if (dir == 0) {
        double m = 0.5 * (B->u0 + B->u1);
        L->u1 = m; R->u0 = m;
        for (int j = 0; j <= B->dv; ++j) {
            double T[OR_MAXDEG + 1][4];
            for (int i = 0; i <= B->du; ++i) memcpy(T[i], B->h[i][j], sizeof(double) * 4);
            for (int d = 0; d < 4; ++d) { L->h[0][j][d] = T[0][d]; R->h[B->du][j][d] = T[B->du][d]; }
            for (int k = 1; k <= B->du; ++k) {
                for (int i = 0; i <= B->du - k; ++i)
                    for (int d = 0; d < 4; ++d) T[i][d] = 0.5 * (T[i][d] + T[i + 1][d]);
                for (int d = 0; d < 4; ++d) { L->h[k][j][d] = T[0][d]; R->h[B->du - k][j][d] = T[B->du - k][d]; }
            }
        }
    } else {
        double m = 0.5 * (B->v0 + B->v1);
        L->v1 = m; R->v0 = m;
        for (int i = 0; i <= B->du; ++i) {
            double T[OR_MAXDEG + 1][4];
            for (int j = 0; j <= B->dv; ++j) memcpy(T[j], B->h[i][j], sizeof(double) * 4);
            for (int d = 0; d < 4; ++d) { L->h[i][0][d] = T[0][d]; R->h[i][B->dv][d] = T[B->dv][d]; }
            for (int k = 1; k <= B->dv; ++k) {
                for (int j = 0; j <= B->dv - k; ++j)
                    for (int d = 0; d < 4; ++d) T[j][d] = 0.5 * (T[j][d] + T[j + 1][d]);
                for (int d = 0; d < 4; ++d) { L->h[i][k][d] = T[0][d]; R->h[i][B->dv - k][d] = T[B->dv - k][d]; }
            }
        }
    }
}

static void bez3_box(const bez3* B, double* lo, double* hi) {
    for (int d = 0; d < 3; ++d) { lo[d] = 1e300; hi[d] = -1e300; }
    for (int i = 0; i <= B->du; ++i)
        for (int j = 0; j <= B->dv; ++j)
            for (int d = 0; d < 3; ++d) {
                double x = B->h[i][j][d] / B->h[i][j][3];
                lo[d] = fmin(lo[d], x);
                hi[d] = fmax(hi[d], x);
            }
}

/* does the half line q - t s, t > 0, meet the box [lo - e, hi + e]? */
static int ray_box(const double* q, const double* s, const double* lo, const double* hi, double e) {
    double t0 = 0.0, t1 = 1e300;
    for (int d = 0; d < 3; ++d) {
        double dir = -s[d];
        double a = lo[d] - e, b = hi[d] + e;
        if (fabs(dir) < 1e-300) {
            if (q[d] < a || q[d] > b) return 0;
        } else {
            double ta = (a - q[d]) / dir, tb = (b - q[d]) / dir;
            if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
            if (t0 > t1) return 0;
        }
    }
    return 1;
}

typedef struct {
    ohit h[64];
    int n;
    int bad;
} hitlist;

static void newton_hit(const opatch* P, const bez3* B, const double* q, const double* s, hitlist* H) {
    double u = 0.5 * (B->u0 + B->u1), v = 0.5 * (B->v0 + B->v1);
    double U0 = P->ub[0], U1 = P->ub[P->nsu], V0 = P->vb[0], V1 = P->vb[P->nsv];
    double S[3], Su[3], Sv[3];
    surf_eval(P, u, v, S, Su, Sv);
    double qs[3] = {q[0] - S[0], q[1] - S[1], q[2] - S[2]};
    double t = dot3(s, qs);
    int ok = 0;
    for (int it = 0; it < 60; ++it) {
        surf_eval(P, u, v, S, Su, Sv);
        double F[3] = {S[0] + t * s[0] - q[0], S[1] + t * s[1] - q[1], S[2] + t * s[2] - q[2]};
        double mF[3] = {-F[0], -F[1], -F[2]}, dx[3];
        if (solve3(Su, Sv, s, mF, dx) < 0) return;
        u += dx[0];
        v += dx[1];
        t += dx[2];
        if (u < U0) u = U0;
        if (u > U1) u = U1;
        if (v < V0) v = V0;
        if (v > V1) v = V1;
        if (fabs(dx[0]) < 1e-15 * (U1 - U0) && fabs(dx[1]) < 1e-15 * (V1 - V0) && fabs(dx[2]) < 1e-15 * P->diag) {
            ok = 1;
            break;
        }
    }
    surf_eval(P, u, v, S, Su, Sv);
    double F[3] = {S[0] + t * s[0] - q[0], S[1] + t * s[1] - q[1], S[2] + t * s[2] - q[2]};
    if (!ok && norm3(F) > 1e-12 * P->diag) return;
    if (norm3(F) > 1e-10 * P->diag) return;
    double eu = 1e-12 * (U1 - U0), ev = 1e-12 * (V1 - V0);
    if (u < B->u0 - eu || u > B->u1 + eu || v < B->v0 - ev || v > B->v1 + ev) return;
    for (int k = 0; k < H->n; ++k) {
        double dd[3] = {H->h[k].x[0] - S[0], H->h[k].x[1] - S[1], H->h[k].x[2] - S[2]};
        if (norm3(dd) < 1e-9 * P->diag) return;  /* duplicate from a neighbouring sub-patch */
    }
    if (H->n >= 64) { H->bad = 1; return; }
    ohit* o = &H->h[H->n++];
    o->u = u; o->v = v; o->t = t;
    memcpy(o->x, S, sizeof(S));
    cross3(Su, Sv, o->n);
}

static void hits_rec(const opatch* P, const bez3* B, const double* q, const double* s, int depth, hitlist* H) {
    double lo[3], hi[3];
    bez3_box(B, lo, hi);
    double e = 1e-9 * P->diag;
    if (!ray_box(q, s, lo, hi, e)) return;
    double dg = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) + (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (dg < 2e-3 * P->diag || depth >= 22) {
        newton_hit(P, B, q, s, H);
        return;
    }
    bez3 L, R;
    double eu = B->u1 - B->u0, ev = B->v1 - B->v0;
    /* split across the longer physical direction */
    double pu = 0, pv = 0;
    for (int d = 0; d < 3; ++d) {
        double a = B->h[B->du][0][d] / B->h[B->du][0][3] - B->h[0][0][d] / B->h[0][0][3];
        double b = B->h[0][B->dv][d] / B->h[0][B->dv][3] - B->h[0][0][d] / B->h[0][0][3];
        pu += a * a;
        pv += b * b;
    }
    (void)eu; (void)ev;
    bez3_split(B, pu >= pv ? 0 : 1, &L, &R);
    hits_rec(P, &L, q, s, depth + 1, H);
    hits_rec(P, &R, q, s, depth + 1, H);
}

static void fib_dir(int k, int n, double* s) {
    double z = 1.0 - (2.0 * k + 1.0) / n;
    double r = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = 2.399963229728653 * k + 0.1;
    s[0] = r * cos(ph);
    s[1] = r * sin(ph);
    s[2] = z;
}

#define OR_NCAND 96
#define OR_NSAMP 24

static double patch_gwn(const opatch* P, const double* q, double near_thr, int* flags) {
    int inside = 1, inside_near = 1;
    for (int d = 0; d < 3; ++d) {
        if (q[d] < P->lo[d] || q[d] > P->hi[d]) inside = 0;
        if (q[d] < P->lo[d] - near_thr || q[d] > P->hi[d] + near_thr) inside_near = 0;
    }
    if (near_thr > 0 && inside_near) {
        /* distance to the untrimmed surface, a conservative proxy */
        for (int k = 0; k < P->nsu * P->nsv; ++k) {
            bez3 stack[64];
            int sp = 0, near = 0;
            stack[sp++] = P->sub[k];
            while (sp > 0 && !near) {
                bez3 B = stack[--sp];
                double lo[3], hi[3];
                bez3_box(&B, lo, hi);
                int in = 1;
                for (int d = 0; d < 3; ++d)
                    if (q[d] < lo[d] - near_thr || q[d] > hi[d] + near_thr) in = 0;
                if (!in) continue;
                double dg = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                 (hi[2] - lo[2]) * (hi[2] - lo[2]));
                if (dg < near_thr || sp + 2 >= 64) { near = 1; break; }
                bez3 L, R;
                double eu = 0, ev = 0;
                for (int d = 0; d < 3; ++d) {
                    double a = B.h[B.du][0][d] / B.h[B.du][0][3] - B.h[0][0][d] / B.h[0][0][3];
                    double b = B.h[0][B.dv][d] / B.h[0][B.dv][3] - B.h[0][0][d] / B.h[0][0][3];
                    eu += a * a;
                    ev += b * b;
                }
                bez3_split(&B, eu >= ev ? 0 : 1, &L, &R);
                stack[sp++] = L;
                stack[sp++] = R;
            }
            if (near) *flags |= ORF_NEAR;
        }
    }
    /* string from q pointing away from the box centre: it cannot meet the
     * patch (convexity of the box); used directly when q is far from the box */
    double c0[3], s0[3], gap = 0.0;
    for (int d = 0; d < 3; ++d) {
        c0[d] = 0.5 * (P->lo[d] + P->hi[d]);
        s0[d] = c0[d] - q[d];
        double e = fmax(P->lo[d] - q[d], q[d] - P->hi[d]);
        if (e > 0) gap += e * e;
    }
    gap = sqrt(gap);
    if (!inside) {
        double ln = norm3(s0);
        for (int d = 0; d < 3; ++d) s0[d] /= ln;
        if (gap > P->diag) return line_integral(P, q, s0, flags) / (4.0 * OR_PI);
    }
    /* boundary samples for choosing the string direction */
    int ns = P->n_tp * OR_NSAMP;
    double* X = (double*)malloc(sizeof(double) * 3 * ns);
    for (int k = 0; k < P->n_tp; ++k)
        for (int j = 0; j < OR_NSAMP; ++j) {
            double uv[2], S[3];
            bez2_eval(&P->tp[k], (j + 0.5) / OR_NSAMP, uv, NULL);
            surf_eval(P, uv[0], uv[1], S, NULL, NULL);
            double r[3] = {S[0] - q[0], S[1] - q[1], S[2] - q[2]};
            double ln = norm3(r);
            for (int d = 0; d < 3; ++d) X[3 * (k * OR_NSAMP + j) + d] = ln > 0 ? r[d] / ln : 0.0;
        }
    double score[OR_NCAND + 1];
    int order[OR_NCAND + 1];
    int ncand = inside ? OR_NCAND : OR_NCAND + 1;   /* candidate OR_NCAND is s0 */
    for (int c = 0; c < ncand; ++c) {
        double s[3];
        if (c == OR_NCAND) memcpy(s, s0, sizeof(s)); else fib_dir(c, OR_NCAND, s);
        double best = 2.0;
        for (int j = 0; j < ns; ++j) {
            /* 1 - cos(angle between the string direction -s and the boundary direction) */
            best = fmin(best, 1.0 + dot3(s, &X[3 * j]));
        }
        score[c] = best;  /* larger is better */
        order[c] = c;
    }
    free(X);
    for (int i = 1; i < ncand; ++i) {
        int o = order[i];
        int j = i - 1;
        while (j >= 0 && score[order[j]] < score[o]) { order[j + 1] = order[j]; --j; }
        order[j + 1] = o;
    }
    for (int attempt = 0; attempt < ncand; ++attempt) {
        double s[3];
        if (order[attempt] == OR_NCAND) memcpy(s, s0, sizeof(s)); else fib_dir(order[attempt], OR_NCAND, s);
        if (!ray_box(q, s, P->lo, P->hi, 1e-12 * P->diag))
            return line_integral(P, q, s, flags) / (4.0 * OR_PI);   /* no crossings possible */
        hitlist H;
        H.n = 0;
        H.bad = 0;
        for (int k = 0; k < P->nsu * P->nsv; ++k) hits_rec(P, &P->sub[k], q, s, 0, &H);
        if (H.bad) continue;
        int degenerate = 0;
        double hsum = 0.0;
        for (int k = 0; k < H.n && !degenerate; ++k) {
            double nl = norm3(H.h[k].n);
            int on = fabs(H.h[k].t) < 1e-13 * P->diag;
            if (H.h[k].t < 0 && !on) continue;
            int wind = trim_winding(P, H.h[k].u, H.h[k].v);
            if (wind == -1000) { degenerate = 1; break; }
            if (wind == 0) continue;           /* crossing of the invisible (trimmed-away) part */
            if (on) { *flags |= ORF_ON_BOUNDARY; return NAN; }
            if (nl < 1e-14 || fabs(dot3(H.h[k].n, s)) < 1e-6 * nl) { degenerate = 1; break; }
            hsum += wind * (dot3(H.h[k].n, s) > 0 ? 1.0 : -1.0);
        }
        if (degenerate) continue;
        return line_integral(P, q, s, flags) / (4.0 * OR_PI) - hsum;
    }
    *flags |= ORF_DEGENERATE;
    return NAN;
}

/* ------------------------------------------------------------------ exported API */

typedef struct {
    int n;
    ocurve* c;
} curveset;

/* Parse a flat record stream of `n_curves` curves.  Returns 0 on success. */
static int parse_curves(const double* rec, long len, int n_curves, curveset* cs) {
    cs->n = n_curves;
    cs->c = (ocurve*)calloc(n_curves > 0 ? n_curves : 1, sizeof(ocurve));
    const double* r = rec;
    const double* end = rec + len;
    int err = 0;
    for (int i = 0; i < n_curves && !err; ++i) r = parse_curve(r, end, &cs->c[i], &err);
    return err;
}

static void free_curves(curveset* cs) {
    for (int i = 0; i < cs->n; ++i) free(cs->c[i].pieces);
    free(cs->c);
}

int or_gwn2d(const double* rec, long len, int n_curves, const double* q, long n_q, double near_thr, int n_threads,
             double* out_w, int* out_flags) {
    curveset cs;
    if (parse_curves(rec, len, n_curves, &cs)) { free_curves(&cs); return 1; }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (long i = 0; i < n_q; ++i) {
        const double* qi = q + 2 * i;
        int flags = 0;
        double acc = 0.0;
        for (int c = 0; c < cs.n; ++c)
            for (int k = 0; k < cs.c[c].n_pieces; ++k) {
                if (near_thr > 0 && piece_near(&cs.c[c].pieces[k], qi, near_thr, 0)) flags |= ORF_NEAR;
                acc += piece_gwn(&cs.c[c].pieces[k], qi, 0, &flags);
            }
        out_w[i] = acc;
        out_flags[i] = flags;
    }
    free_curves(&cs);
    return 0;
}

typedef struct {
    int n;
    opatch* p;
} patchset;

static int parse_patches(const double* rec, long len, int n_patches, patchset* ps) {
    ps->n = n_patches;
    ps->p = (opatch*)calloc(n_patches > 0 ? n_patches : 1, sizeof(opatch));
    const double* r = rec;
    const double* end = rec + len;
    int err = 0;
    for (int i = 0; i < n_patches && !err; ++i) r = parse_patch(r, end, &ps->p[i], &err);
    return err;
}

static void free_patches(patchset* ps) {
    for (int i = 0; i < ps->n; ++i) free_patch(&ps->p[i]);
    free(ps->p);
}

int or_gwn3d(const double* rec, long len, int n_patches, const double* q, long n_q, double near_thr, int n_threads,
             double* out_w, int* out_flags) {
    gl_init();
    patchset ps;
    if (parse_patches(rec, len, n_patches, &ps)) { free_patches(&ps); return 1; }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long i = 0; i < n_q; ++i) {
        int flags = 0;
        double acc = 0.0;
        for (int k = 0; k < ps.n; ++k) acc += patch_gwn(&ps.p[k], q + 3 * i, near_thr, &flags);
        out_w[i] = acc;
        out_flags[i] = flags;
    }
    free_patches(&ps);
    return 0;
}

/* Per-primitive contributions (for additivity and reversal tests): out is n_q x n_prim. */
int or_gwn2d_each(const double* rec, long len, int n_curves, const double* q, long n_q, double* out) {
    curveset cs;
    if (parse_curves(rec, len, n_curves, &cs)) { free_curves(&cs); return 1; }
    for (long i = 0; i < n_q; ++i)
        for (int c = 0; c < cs.n; ++c) {
            int fl = 0;
            double acc = 0.0;
            for (int k = 0; k < cs.c[c].n_pieces; ++k) acc += piece_gwn(&cs.c[c].pieces[k], q + 2 * i, 0, &fl);
            out[i * cs.n + c] = acc;
        }
    free_curves(&cs);
    return 0;
}

int or_gwn3d_each(const double* rec, long len, int n_patches, const double* q, long n_q, double* out) {
    gl_init();
    patchset ps;
    if (parse_patches(rec, len, n_patches, &ps)) { free_patches(&ps); return 1; }
    for (long i = 0; i < n_q; ++i)
        for (int k = 0; k < ps.n; ++k) {
            int fl = 0;
            out[i * ps.n + k] = patch_gwn(&ps.p[k], q + 3 * i, 0.0, &fl);
        }
    free_patches(&ps);
    return 0;
}

/* Evaluate curve c (of the record stream) at global parameters t: out n_t x 2. */
int or_curve_eval(const double* rec, long len, int n_curves, int which, const double* t, long n_t, double* out) {
    if (which < 0 || which >= n_curves) return 1;
    const double* r = rec;
    const double* end = rec + len;
    for (int i = 0; i < which; ++i) {
        int p = (int)r[0], n = (int)r[1];
        r += 2 + 2 * n + n + n + p + 1;
        if (r > end) return 1;
    }
    int p = (int)r[0], n = (int)r[1];
    const double* ctrl = r + 2;
    const double* w = ctrl + 2 * n;
    const double* U = w + n;
    /* de Boor recurrence in homogeneous coordinates */
    for (long j = 0; j < n_t; ++j) {
        double x = t[j];
        int k = p;
        while (k + 1 < n && U[k + 1] <= x) ++k;
        double D[OR_MAXDEG + 1][3];
        for (int i = 0; i <= p; ++i) {
            int idx = k - p + i;
            D[i][0] = w[idx] * ctrl[2 * idx];
            D[i][1] = w[idx] * ctrl[2 * idx + 1];
            D[i][2] = w[idx];
        }
        for (int rr = 1; rr <= p; ++rr)
            for (int i = p; i >= rr; --i) {
                int idx = k - p + i;
                double den = U[idx + p - rr + 1] - U[idx];
                double a = den > 0 ? (x - U[idx]) / den : 0.0;
                for (int d = 0; d < 3; ++d) D[i][d] = (1.0 - a) * D[i - 1][d] + a * D[i][d];
            }
        out[2 * j] = D[p][0] / D[p][2];
        out[2 * j + 1] = D[p][1] / D[p][2];
    }
    return 0;
}

/* Evaluate patch `which` at global (u, v) pairs: out n x 9 = S, S_u, S_v. */
int or_patch_eval(const double* rec, long len, int n_patches, int which, const double* uv, long n, double* out) {
    patchset ps;
    if (parse_patches(rec, len, n_patches, &ps)) { free_patches(&ps); return 1; }
    if (which < 0 || which >= n_patches) { free_patches(&ps); return 1; }
    for (long j = 0; j < n; ++j) surf_eval(&ps.p[which], uv[2 * j], uv[2 * j + 1], out + 9 * j, out + 9 * j + 3, out + 9 * j + 6);
    free_patches(&ps);
    return 0;
}

/* ------------------------------------------------------------------ moments (plain definitions)
 *
 * Uncentred moments of Section 3.1 about a given point x0, integrated
 * directly from their definitions:
 *   m0 = int n dA, m1_ij = int (x - x0)_i n_j dA, m2_ijk = int (x - x0)_i (x - x0)_j n_k dA,
 * plus area = int |n| dA and c_i = int (x - x0)_i |n| dA.
 * 2D: the integrals are taken over straight segments a -> b (the paper's chord
 * substitution, Section 3.1), with n dA = (dy, -dx).
 * 3D: over a patch.  Untrimmed patches use tensor Gauss-Legendre rules on
 * every Bezier sub-patch.  For trimmed patches the winding-weighted region is
 * decomposed as a fan from the centre c of the parameter domain: for each boundary piece gamma(tau) the
 * curved triangle c + sigma (gamma(tau) - c) has Jacobian
 * sigma * cross(gamma - c, gamma'), and the triangles' signed sum is the
 * region counted with its winding number. */

static void acc_moments(int dim, const double* x, const double* x0, const double* nv, double wgt, double* out) {
    /* out layout: m0[dim], m1[dim*dim], m2[dim^3], area, c[dim] */
    double r[3];
    for (int i = 0; i < dim; ++i) r[i] = x[i] - x0[i];
    double nl = 0;
    for (int i = 0; i < dim; ++i) nl += nv[i] * nv[i];
    nl = sqrt(nl);
    double* m0 = out;
    double* m1 = m0 + dim;
    double* m2 = m1 + dim * dim;
    double* ar = m2 + dim * dim * dim;
    double* cc = ar + 1;
    for (int k = 0; k < dim; ++k) m0[k] += wgt * nv[k];
    for (int i = 0; i < dim; ++i)
        for (int k = 0; k < dim; ++k) m1[i * dim + k] += wgt * r[i] * nv[k];
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j)
            for (int k = 0; k < dim; ++k) m2[(i * dim + j) * dim + k] += wgt * r[i] * r[j] * nv[k];
    ar[0] += wgt * nl;
    for (int i = 0; i < dim; ++i) cc[i] += wgt * r[i] * nl;
}

int or_segment_moments(const double* seg /* n x 4: ax ay bx by */, long n, const double* x0, double* out /* 2+4+8+1+2 */) {
    gl_init();
    memset(out, 0, sizeof(double) * 17);
    for (long s = 0; s < n; ++s) {
        const double* a = seg + 4 * s;
        double e[2] = {a[2] - a[0], a[3] - a[1]};
        double nv[2] = {e[1], -e[0]};
        double len = hypot(e[0], e[1]);
        if (len == 0) continue;
        for (int g = 0; g < OR_GLN; ++g) {
            double x[2] = {a[0] + g_glx[g] * e[0], a[1] + g_glx[g] * e[1]};
            /* n ds = (dy, -dx): with the unit normal times the length element */
            acc_moments(2, x, x0, nv, g_glw[g], out);
        }
    }
    return 0;
}

int or_patch_moments(const double* rec, long len, int n_patches, int which, const double* x0, int nsub,
                     double* out /* 3+9+27+1+3 */) {
    gl_init();
    patchset ps;
    if (parse_patches(rec, len, n_patches, &ps)) { free_patches(&ps); return 1; }
    if (which < 0 || which >= n_patches) { free_patches(&ps); return 1; }
    const opatch* P = &ps.p[which];
    memset(out, 0, sizeof(double) * 43);
    if (nsub < 1) nsub = 1;
    if (P->untrimmed) {
        /* tensor Gauss-Legendre over every Bezier sub-patch rectangle */
        for (int k = 0; k < P->nsu * P->nsv; ++k) {
            const bez3* B = &P->sub[k];
            double hu = (B->u1 - B->u0) / nsub, hv = (B->v1 - B->v0) / nsub;
            for (int a = 0; a < nsub; ++a)
                for (int b = 0; b < nsub; ++b)
                    for (int gi = 0; gi < OR_GLN; ++gi)
                        for (int gj = 0; gj < OR_GLN; ++gj) {
                            double u = B->u0 + (a + g_glx[gi]) * hu, v = B->v0 + (b + g_glx[gj]) * hv;
                            double S[3], Su[3], Sv[3], nv[3];
                            surf_eval(P, u, v, S, Su, Sv);
                            cross3(Su, Sv, nv);
                            acc_moments(3, S, x0, nv, g_glw[gi] * g_glw[gj] * hu * hv, out);
                        }
        }
        free_patches(&ps);
        return 0;
    }
    double c[2] = {0.5 * (P->ub[0] + P->ub[P->nsu]), 0.5 * (P->vb[0] + P->vb[P->nsv])};
    for (int k = 0; k < P->n_tp; ++k)
        for (int a = 0; a < nsub; ++a)
            for (int gi = 0; gi < OR_GLN; ++gi) {
                double tau = (a + g_glx[gi]) / nsub;
                double wt = g_glw[gi] / nsub;
                double g[2], dg[2];
                bez2_eval(&P->tp[k], tau, g, dg);
                double jac = (g[0] - c[0]) * dg[1] - (g[1] - c[1]) * dg[0];
                for (int b = 0; b < nsub; ++b)
                    for (int gj = 0; gj < OR_GLN; ++gj) {
                        double sg = (b + g_glx[gj]) / nsub;
                        double ws = g_glw[gj] / nsub;
                        double u = c[0] + sg * (g[0] - c[0]), v = c[1] + sg * (g[1] - c[1]);
                        double S[3], Su[3], Sv[3], nv[3];
                        surf_eval(P, u, v, S, Su, Sv);
                        cross3(Su, Sv, nv);
                        acc_moments(3, S, x0, nv, wt * ws * sg * jac, out);
                    }
            }
    free_patches(&ps);
    return 0;
}

/* ------------------------------------------------------------------ Taylor approximation (Eq. 3)
 *
 * Evaluates, with full derivative tensors of the Green's function of Eq. 2,
 *   w ~ m0 . dG(x0) + m1 : d2G(x0) + 1/2 m2 : d3G(x0)
 * where the m are the moments centred at x0 (m1_ij = int (x - x0)_i n_j,
 * m2_ijk = int (x - x0)_i (x - x0)_j n_k) and the derivatives are taken with
 * respect to x at x = x0, r = x0 - q.  order selects how many terms are kept. */
int or_taylor(int dim, int order, const double* x0, const double* m0, const double* m1, const double* m2,
              const double* q, double* out) {
    if (dim != 2 && dim != 3) return 1;
    double r[3] = {0, 0, 0};
    for (int i = 0; i < dim; ++i) r[i] = x0[i] - q[i];
    double rho2 = 0;
    for (int i = 0; i < dim; ++i) rho2 += r[i] * r[i];
    double rho = sqrt(rho2);
    double g1[3], g2[3][3], g3[3][3][3];
    if (dim == 2) {
        /* G = (1/2pi) ln rho */
        double c = 1.0 / (2.0 * OR_PI);
        for (int i = 0; i < 2; ++i) g1[i] = c * r[i] / rho2;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) g2[i][j] = c * ((i == j) / rho2 - 2.0 * r[i] * r[j] / (rho2 * rho2));
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int k = 0; k < 2; ++k)
                    g3[i][j][k] = c * (-2.0 * ((i == j) * r[k] + (i == k) * r[j] + (j == k) * r[i]) / (rho2 * rho2) +
                                       8.0 * r[i] * r[j] * r[k] / (rho2 * rho2 * rho2));
    } else {
        /* G = -1/(4pi rho) */
        double c = 1.0 / (4.0 * OR_PI);
        double r3 = rho2 * rho, r5 = r3 * rho2, r7 = r5 * rho2;
        for (int i = 0; i < 3; ++i) g1[i] = c * r[i] / r3;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) g2[i][j] = c * ((i == j) / r3 - 3.0 * r[i] * r[j] / r5);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    g3[i][j][k] = c * (-3.0 * ((i == j) * r[k] + (i == k) * r[j] + (j == k) * r[i]) / r5 +
                                       15.0 * r[i] * r[j] * r[k] / r7);
    }
    double w = 0;
    for (int k = 0; k < dim; ++k) w += m0[k] * g1[k];
    if (order >= 1)
        for (int i = 0; i < dim; ++i)
            for (int k = 0; k < dim; ++k) w += m1[i * dim + k] * g2[i][k];
    if (order >= 2)
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j)
                for (int k = 0; k < dim; ++k) w += 0.5 * m2[(i * dim + j) * dim + k] * g3[i][j][k];
    *out = w;
    return 0;
}
