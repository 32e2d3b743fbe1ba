/*
 * oracle.c -- plain FP64 CPU reference of the MOT-JVIE operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code with the CUDA product path.
 *
 * Everything is in voxel units: lengths in h, time in h/c0, so the time step
 * is rho = c0*dt/h = alpha/sqrt(3) (Eq. 9 with dt_CFL = h/(c0 sqrt 3)).
 *
 * What is computed (paper Sec. II, Eq. 1, Eq. 3, Eq. 10):
 *   temporal basis   T(t) = B2(t/dt + 1), quadratic B-spline (p = 2, Sec. II)
 *   lag kernel       K_k(R) = B2(k + 1 - R/rho) / (4 pi R)   (retarded 1/(4 pi R)
 *                    sampled by Dirac testing at t_n, source basis shifted by k)
 *   Galerkin weight  W_d(s) = prod_i Lambda(s_i - d_i), Lambda(x) = max(1-|x|,0)
 *                    (piecewise-constant voxel basis and testing)
 *   A_k(d)_pq        = int K_k(s) d_p d_q W_d(s) ds   (distributional)
 *   g_k(d)_pq        = A_k(d)_pq - delta_pq sum_r A_k(d)_rr   (curl curl = grad div - lap)
 *   Z_k              = eps_r T(k dt) I - (eps_r - 1) g_k       (Eq. 10 at every lag)
 *
 * Quadrature: every A entry is reduced to a 1-D radial integral whose angular
 * part is exact (arcs of circles clipped by the unit-cell lines).  Radial
 * panels are split at every radius where the integrand is not analytic
 * (kernel knots, line tangencies, cell corners); panels that start at a line
 * tangency use t = sqrt(t0^2 + tau^2), panels that end where a kernel knot
 * enters the z-line use t = sqrt(t1^2 - tau^2), and the single logarithmic
 * case (d_r = 0 near t = 0) uses geometric panels.  Gauss-Legendre nodes are
 * computed here by Newton iteration on the Legendre recurrence.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_TWO_PI (2.0 * OR_PI)

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1, 1]                                      */
/* ------------------------------------------------------------------ */
#define GL_MAXN 64
static double gl_x[GL_MAXN + 1][GL_MAXN];
static double gl_w[GL_MAXN + 1][GL_MAXN];
static int gl_ready = 0;

static void gl_compute(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        /* recompute derivative at the converged root */
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void oracle_init(void) {
    if (gl_ready) return;
    for (int n = 1; n <= GL_MAXN; ++n) gl_compute(n, gl_x[n], gl_w[n]);
    gl_ready = 1;
}

/* exported for the node/weight pin against a library routine */
int oracle_gauss_legendre(int n, double *x, double *w) {
    if (n < 1 || n > GL_MAXN) return -1;
    oracle_init();
    memcpy(x, gl_x[n], sizeof(double) * n);
    memcpy(w, gl_w[n], sizeof(double) * n);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Temporal basis: quadratic B-spline (Sec. II: p = 2)                 */
/* ------------------------------------------------------------------ */
double oracle_bspline2(double u) {
    if (u <= 0.0 || u >= 3.0) return 0.0;
    if (u < 1.0) return 0.5 * u * u;
    if (u < 2.0) return 0.5 * (-2.0 * u * u + 6.0 * u - 3.0);
    return 0.5 * (3.0 - u) * (3.0 - u);
}

/* T(k dt) = B2(k + 1) */
double oracle_temporal(int k) { return oracle_bspline2(k + 1.0); }

/* K_k(R) = B2(k + 1 - R/rho) / (4 pi R) */
static double lag_kernel(int k, double rho, double R) {
    return oracle_bspline2(k + 1.0 - R / rho) / (4.0 * OR_PI * R);
}

/* knot radii of K_k: (k-2)rho .. (k+1)rho, positive ones only */
static int lag_knots(int k, double rho, double *Rj) {
    int m = 0;
    for (int i = -2; i <= 1; ++i) {
        double r = (k + i) * rho;
        if (r > 0.0) Rj[m++] = r;
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* exact angular integrals over circles of radius t                    */
/* ------------------------------------------------------------------ */
static void sort_small(double *a, int n) {
    for (int i = 1; i < n; ++i) {
        double v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

/* crossing angles of the circle |(u,v)| = t with lines u = lo..lo+2, v = lo2..lo2+2 */
static int circle_breaks(double t, double a, double b, double *th) {
    int m = 0;
    th[m++] = 0.0;
    th[m++] = OR_TWO_PI;
    for (int e = -1; e <= 1; ++e) {
        double x = a + e;
        if (fabs(x) < t) {
            double q = acos(x / t);
            th[m++] = q;
            th[m++] = OR_TWO_PI - q;
        }
        double y = b + e;
        if (fabs(y) < t) {
            double q = asin(y / t);
            th[m++] = q < 0.0 ? q + OR_TWO_PI : q;
            th[m++] = OR_PI - q;
        }
    }
    sort_small(th, m);
    return m;
}

/* int_0^{2pi} Lambda(t cos th - a) Lambda(t sin th - b) dth */
double oracle_ang_tent(double t, double a, double b) {
    double th[16];
    int m = circle_breaks(t, a, b, th);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double t1 = th[i], t2 = th[i + 1];
        if (t2 - t1 <= 0.0) continue;
        double tm = 0.5 * (t1 + t2);
        double u = t * cos(tm) - a, v = t * sin(tm) - b;
        if (fabs(u) >= 1.0 || fabs(v) >= 1.0) continue;
        double su = u > 0.0 ? 1.0 : -1.0, sv = v > 0.0 ? 1.0 : -1.0;
        /* Lambda(U - a) = (1 + su a) - su U on this piece, U = t cos th */
        double au = 1.0 + su * a, bu = -su;
        double av = 1.0 + sv * b, bv = -sv;
        double c1 = cos(t1), c2 = cos(t2), s1 = sin(t1), s2 = sin(t2);
        acc += au * av * (t2 - t1)
             + au * bv * t * (c1 - c2)
             + bu * av * t * (s2 - s1)
             + bu * bv * t * t * 0.5 * (s2 * s2 - s1 * s1);
    }
    return acc;
}

static double dlambda(double x) {
    if (x > -1.0 && x < 0.0) return 1.0;
    if (x > 0.0 && x < 1.0) return -1.0;
    return 0.0;
}

/* int_0^{2pi} Lambda'(t cos th - a) Lambda'(t sin th - b) dth */
double oracle_ang_quad(double t, double a, double b) {
    double th[16];
    int m = circle_breaks(t, a, b, th);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double t1 = th[i], t2 = th[i + 1];
        if (t2 - t1 <= 0.0) continue;
        double tm = 0.5 * (t1 + t2);
        double u = t * cos(tm) - a, v = t * sin(tm) - b;
        acc += dlambda(u) * dlambda(v) * (t2 - t1);
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* panel machinery                                                      */
/* ------------------------------------------------------------------ */
#ifndef QN
#define QN 20 /* Gauss-Legendre points per panel */
#endif
#ifndef PANEL_MAX
#define PANEL_MAX 0.75 /* longest panel, in voxel units */
#endif

typedef double (*radial_fn)(double t, const void *ctx);

static int near(double a, double b) { return fabs(a - b) <= 1e-13 * (1.0 + fabs(a)); }

static int in_set(double v, const double *s, int n) {
    for (int i = 0; i < n; ++i)
        if (near(v, s[i])) return 1;
    return 0;
}

/* plain GL over [x0, x1] (split into pieces of at most PANEL_MAX) */
static double gl_plain(radial_fn f, const void *ctx, double x0, double x1) {
    if (x1 <= x0) return 0.0;
    int np = (int)ceil((x1 - x0) / PANEL_MAX);
    if (np < 1) np = 1;
    double h = (x1 - x0) / np, acc = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = x0 + p * h, c = 0.5 * h, m = a + c;
        for (int i = 0; i < QN; ++i) acc += gl_w[QN][i] * c * f(m + c * gl_x[QN][i], ctx);
    }
    return acc;
}

/* panel with a square-root singularity at its left end t0 (line tangency):
 * t = sqrt(t0^2 + tau^2), dt = tau/t dtau */
static double gl_left_sqrt(radial_fn f, const void *ctx, double t0, double t1) {
    double tmax = sqrt(t1 * t1 - t0 * t0);
    int np = (int)ceil(tmax / PANEL_MAX);
    if (np < 1) np = 1;
    double h = tmax / np, acc = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = p * h, c = 0.5 * h, m = a + c;
        for (int i = 0; i < QN; ++i) {
            double tau = m + c * gl_x[QN][i];
            double t = sqrt(t0 * t0 + tau * tau);
            acc += gl_w[QN][i] * c * f(t, ctx) * tau / t;
        }
    }
    return acc;
}

/* panel with a square-root singularity at its right end t1 (kernel knot
 * entering the z-line): t = sqrt(t1^2 - tau^2), dt = -tau/t dtau */
static double gl_right_sqrt(radial_fn f, const void *ctx, double t0, double t1) {
    double tmax = sqrt(t1 * t1 - t0 * t0);
    int np = (int)ceil(tmax / PANEL_MAX);
    if (np < 1) np = 1;
    double h = tmax / np, acc = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = p * h, c = 0.5 * h, m = a + c;
        for (int i = 0; i < QN; ++i) {
            double tau = m + c * gl_x[QN][i];
            double t = sqrt(t1 * t1 - tau * tau);
            acc += gl_w[QN][i] * c * f(t, ctx) * tau / t;
        }
    }
    return acc;
}

/* panel [0, t1] with a logarithmic end at 0: geometric panels t1*q^j */
static double gl_log_left(radial_fn f, const void *ctx, double t1) {
    const double q = 0.25;
    double acc = 0.0, hi = t1;
    for (int j = 0; j < 40; ++j) {
        double lo = hi * q;
        double c = 0.5 * (hi - lo), m = lo + c;
        for (int i = 0; i < QN; ++i) acc += gl_w[QN][i] * c * f(m + c * gl_x[QN][i], ctx);
        hi = lo;
    }
    return acc;
}

/* integrate f over [lo, hi] split at the sorted break list; flags decide the
 * substitution used on each panel */
typedef struct {
    const double *tang; int ntang;   /* radii with a left-end sqrt singularity  */
    const double *rsq; int nrsq;     /* radii with a right-end sqrt singularity */
    int log_at_zero;                 /* logarithmic behaviour at t = 0          */
} panel_flags;

static double radial_integral(radial_fn f, const void *ctx, double *brk, int nb, double lo,
                              double hi, const panel_flags *fl) {
    if (hi <= lo) return 0.0;
    double pts[128];
    int m = 0;
    pts[m++] = lo;
    pts[m++] = hi;
    for (int i = 0; i < nb; ++i)
        if (brk[i] > lo && brk[i] < hi) pts[m++] = brk[i];
    sort_small(pts, m);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double t0 = pts[i], t1 = pts[i + 1];
        if (t1 - t0 <= 1e-14 * (1.0 + t1)) continue;
        int lt = t0 > 0.0 && in_set(t0, fl->tang, fl->ntang);
        int rs = in_set(t1, fl->rsq, fl->nrsq);
        int ltype = (t0 == 0.0 && fl->log_at_zero) ? 2 : (lt ? 1 : 0);
        /* a panel with a special right end is split at its midpoint so that
         * each substitution acts on one end only */
        double tr = rs ? 0.5 * (t0 + t1) : t1;
        if (ltype == 2) acc += gl_log_left(f, ctx, tr);
        else if (ltype == 1) acc += gl_left_sqrt(f, ctx, t0, tr);
        else acc += gl_plain(f, ctx, t0, tr);
        if (rs) acc += gl_right_sqrt(f, ctx, tr, t1);
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* face integral (diagonal A_pp):                                      */
/*   F(c; a, b) = int int K_k(sqrt(c^2+u^2+v^2)) Lambda(u-a) Lambda(v-b)  */
/*             = int_0^inf K_k(sqrt(c^2+t^2)) angT(t; a, b) t dt          */
/* ------------------------------------------------------------------ */
typedef struct { int k; double rho, c, a, b; } face_ctx;

static double face_integrand(double t, const void *vp) {
    const face_ctx *p = (const face_ctx *)vp;
    double R = sqrt(p->c * p->c + t * t);
    return lag_kernel(p->k, p->rho, R) * oracle_ang_tent(t, p->a, p->b) * t;
}

double oracle_face(int k, double rho, double c, double a, double b) {
    oracle_init();
    face_ctx ctx = {k, rho, c, a, b};
    double Rj[4];
    int nk = lag_knots(k, rho, Rj);
    double brk[64], tang[6];
    int nb = 0, nt = 0;
    double tcorner_max = 0.0;
    for (int e = -1; e <= 1; ++e) {
        tang[nt++] = fabs(a + e);
        tang[nt++] = fabs(b + e);
    }
    for (int i = 0; i < nt; ++i) brk[nb++] = tang[i];
    for (int e1 = -1; e1 <= 1; ++e1)
        for (int e2 = -1; e2 <= 1; ++e2) {
            double r = sqrt((a + e1) * (a + e1) + (b + e2) * (b + e2));
            brk[nb++] = r;
            if (r > tcorner_max) tcorner_max = r;
        }
    double c2 = c * c;
    for (int j = 0; j < nk; ++j)
        if (Rj[j] > fabs(c)) brk[nb++] = sqrt(Rj[j] * Rj[j] - c2);
    /* support: t below the block distance or outside the kernel shell is zero */
    double da = fabs(a) > 1.0 ? fabs(a) - 1.0 : 0.0, db = fabs(b) > 1.0 ? fabs(b) - 1.0 : 0.0;
    double lo = sqrt(da * da + db * db);
    double Rout = (k + 1) * rho, Rin = (k - 2) * rho;
    if (Rout <= fabs(c)) return 0.0;
    double hi = sqrt(Rout * Rout - c2);
    if (hi > tcorner_max) hi = tcorner_max;
    if (Rin > fabs(c)) {
        double tin = sqrt(Rin * Rin - c2);
        if (tin > lo) lo = tin;
    }
    panel_flags fl = {tang, nt, NULL, 0, 0};
    return radial_integral(face_integrand, &ctx, brk, nb, lo, hi, &fl);
}

/* ------------------------------------------------------------------ */
/* z-line integral  G(t) = int Lambda(z - dr) K_k(sqrt(t^2 + z^2)) dz   */
/* ------------------------------------------------------------------ */
static double zline(int k, double rho, double t, double dr) {
    double pts[96];
    int m = 0;
    double z0 = dr - 1.0, z1 = dr + 1.0;
    pts[m++] = z0;
    pts[m++] = dr;
    pts[m++] = z1;
    double Rj[4];
    int nk = lag_knots(k, rho, Rj);
    for (int j = 0; j < nk; ++j)
        if (Rj[j] > t) {
            double zk = sqrt(Rj[j] * Rj[j] - t * t);
            if (zk > z0 && zk < z1) pts[m++] = zk;
            if (-zk > z0 && -zk < z1) pts[m++] = -zk;
        }
    if (t < 1.0 && z0 <= 0.0 && z1 >= 0.0) {
        /* 1/R is nearly singular at z = 0 when t is small: geometric panels */
        if (z0 < 0.0 && z1 > 0.0) pts[m++] = 0.0;
        for (double s = t; s < 2.0 && m < 90; s *= 4.0) {
            if (s > z0 && s < z1) pts[m++] = s;
            if (-s > z0 && -s < z1) pts[m++] = -s;
        }
    }
    sort_small(pts, m);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double a = pts[i], b = pts[i + 1];
        if (b - a <= 1e-15) continue;
        int np = (int)ceil((b - a) / PANEL_MAX);
        double h = (b - a) / np;
        for (int p = 0; p < np; ++p) {
            double c = 0.5 * h, mid = a + p * h + c;
            for (int q = 0; q < QN; ++q) {
                double z = mid + c * gl_x[QN][q];
                double w = 1.0 - fabs(z - dr);
                if (w <= 0.0) continue;
                double R = sqrt(t * t + z * z);
                acc += gl_w[QN][q] * c * w * lag_kernel(k, rho, R);
            }
        }
    }
    return acc;
}

/* box integral (off-diagonal A_pq):
 *   int K_k(s) Lambda'(s_p-dp) Lambda'(s_q-dq) Lambda(s_r-dr) ds
 * = int_0^inf G(t; dr) angQ(t; dp, dq) t dt                         */
typedef struct { int k; double rho, dp, dq, dr; } box_ctx;

static double box_integrand(double t, const void *vp) {
    const box_ctx *p = (const box_ctx *)vp;
    double aq = oracle_ang_quad(t, p->dp, p->dq);
    if (aq == 0.0) return 0.0;
    return zline(p->k, p->rho, t, p->dr) * aq * t;
}

double oracle_box(int k, double rho, double dp, double dq, double dr) {
    oracle_init();
    box_ctx ctx = {k, rho, dp, dq, dr};
    double Rj[4];
    int nk = lag_knots(k, rho, Rj);
    double brk[96], tang[6], rsq[4];
    int nb = 0, nt = 0, nr = 0;
    double tcorner_max = 0.0;
    for (int e = -1; e <= 1; ++e) {
        tang[nt++] = fabs(dp + e);
        tang[nt++] = fabs(dq + e);
    }
    for (int i = 0; i < nt; ++i) brk[nb++] = tang[i];
    for (int e1 = -1; e1 <= 1; ++e1)
        for (int e2 = -1; e2 <= 1; ++e2) {
            double r = sqrt((dp + e1) * (dp + e1) + (dq + e2) * (dq + e2));
            brk[nb++] = r;
            if (r > tcorner_max) tcorner_max = r;
        }
    int zero_in = (dr - 1.0 <= 0.0 && dr + 1.0 >= 0.0);
    for (int j = 0; j < nk; ++j) {
        for (int e = -1; e <= 1; ++e) {
            double ze = dr + e;
            if (Rj[j] > fabs(ze)) brk[nb++] = sqrt(Rj[j] * Rj[j] - ze * ze);
        }
        if (zero_in) {
            brk[nb++] = Rj[j];
            rsq[nr++] = Rj[j];
        }
    }
    double dpp = fabs(dp) > 1.0 ? fabs(dp) - 1.0 : 0.0, dqq = fabs(dq) > 1.0 ? fabs(dq) - 1.0 : 0.0;
    double lo = sqrt(dpp * dpp + dqq * dqq);
    double zmin = fabs(dr) > 1.0 ? fabs(dr) - 1.0 : 0.0, zmax = fabs(dr) + 1.0;
    double Rout = (k + 1) * rho, Rin = (k - 2) * rho;
    if (Rout <= zmin) return 0.0;
    double hi = sqrt(Rout * Rout - zmin * zmin);
    if (hi > tcorner_max) hi = tcorner_max;
    if (Rin > zmax) {
        double tin = sqrt(Rin * Rin - zmax * zmax);
        if (tin > lo) lo = tin;
    }
    panel_flags fl = {tang, nt, rsq, nr, (dr == 0.0 && lo == 0.0)};
    return radial_integral(box_integrand, &ctx, brk, nb, lo, hi, &fl);
}

/* ------------------------------------------------------------------ */
/* Galerkin Green tensor of one lag at one offset                       */
/* ------------------------------------------------------------------ */
/* causal support of lag k at offset d (cube-cube distance range)        */
int oracle_in_support(int k, double rho, int dx, int dy, int dz) {
    int d[3] = {dx, dy, dz};
    double mn = 0.0, mx = 0.0;
    for (int i = 0; i < 3; ++i) {
        double a = fabs((double)d[i]);
        double lo = a > 1.0 ? a - 1.0 : 0.0, hi = a + 1.0;
        mn += lo * lo;
        mx += hi * hi;
    }
    mn = sqrt(mn);
    mx = sqrt(mx);
    return (mn < (k + 1) * rho) && (mx > (k - 2) * rho);
}

/* A[3][3] (raw, no symmetry use) at integer offset d */
void oracle_A_raw(int k, double rho, int dx, int dy, int dz, double *A) {
    oracle_init();
    double d[3] = {dx, dy, dz};
    for (int i = 0; i < 9; ++i) A[i] = 0.0;
    if (!oracle_in_support(k, rho, dx, dy, dz)) return;
    for (int p = 0; p < 3; ++p) {
        int q = (p + 1) % 3, r = (p + 2) % 3;
        double acc = 0.0;
        const double w[3] = {1.0, -2.0, 1.0};
        for (int e = -1; e <= 1; ++e) acc += w[e + 1] * oracle_face(k, rho, d[p] + e, d[q], d[r]);
        A[p * 3 + p] = acc;
    }
    for (int p = 0; p < 3; ++p)
        for (int q = p + 1; q < 3; ++q) {
            int r = 3 - p - q;
            double v = oracle_box(k, rho, d[p], d[q], d[r]);
            A[p * 3 + q] = v;
            A[q * 3 + p] = v;
        }
}

/* g = A - I tr(A), returned as 6 components (xx, yy, zz, xy, xz, yz) */
void oracle_g_raw(int k, double rho, int dx, int dy, int dz, double *g6) {
    double A[9];
    oracle_A_raw(k, rho, dx, dy, dz, A);
    double tr = A[0] + A[4] + A[8];
    g6[0] = A[0] - tr;
    g6[1] = A[4] - tr;
    g6[2] = A[8] - tr;
    g6[3] = A[1];
    g6[4] = A[2];
    g6[5] = A[5];
}

static int comp6(int p, int q) {
    if (p == q) return p;
    int a = p < q ? p : q, b = p < q ? q : p;
    if (a == 0 && b == 1) return 3;
    if (a == 0 && b == 2) return 4;
    return 5;
}

/*
 * Full lag table g_k(d) for |d_x| <= Rx, |d_y| <= Ry, |d_z| <= Rz.
 * Layout: g[c][dz+Rz][dy+Ry][dx+Rx], c in (xx, yy, zz, xy, xz, yz).
 * Entries are computed once per sorted |d| (0 <= a <= b <= c) and spread
 * with the reflection / permutation covariance of the Galerkin kernel:
 *   g_pq(d) = s_p s_q g_{pos(p) pos(q)}(sorted |d|)
 * (the covariance itself is checked directly against oracle_g_raw in tests).
 */
void oracle_lag_table(int k, double rho, int Rx, int Ry, int Rz, double *g) {
    oracle_init();
    int nx = 2 * Rx + 1, ny = 2 * Ry + 1, nz = 2 * Rz + 1;
    long n3 = (long)nx * ny * nz;
    memset(g, 0, sizeof(double) * 6 * n3);
    int Rm = Rx > Ry ? Rx : Ry;
    Rm = Rm > Rz ? Rm : Rz;
    int lo3 = Rx < Ry ? Rx : Ry;
    lo3 = lo3 < Rz ? lo3 : Rz;
    /* enumerate sorted triples a <= b <= c that occur in the box */
    long ncan = 0;
    int *can = (int *)malloc(sizeof(int) * 3 * (size_t)(Rm + 1) * (Rm + 1) * (Rm + 1));
    for (int a = 0; a <= Rm; ++a)
        for (int b = a; b <= Rm; ++b)
            for (int c = b; c <= Rm; ++c) {
                if (!oracle_in_support(k, rho, a, b, c)) continue;
                /* does some axis assignment fit in the box? */
                int v[3] = {a, b, c}, ok = 0;
                int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                for (int p = 0; p < 6 && !ok; ++p)
                    if (v[perms[p][0]] <= Rx && v[perms[p][1]] <= Ry && v[perms[p][2]] <= Rz) ok = 1;
                if (!ok) continue;
                can[3 * ncan + 0] = a;
                can[3 * ncan + 1] = b;
                can[3 * ncan + 2] = c;
                ++ncan;
            }
    (void)lo3;
    double *val = (double *)malloc(sizeof(double) * 9 * (ncan > 0 ? ncan : 1));
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < ncan; ++i)
        oracle_A_raw(k, rho, can[3 * i], can[3 * i + 1], can[3 * i + 2], val + 9 * i);
    /* index of sorted triple -> position in can[] via a dense map */
    long *map = (long *)malloc(sizeof(long) * (size_t)(Rm + 1) * (Rm + 1) * (Rm + 1));
    for (long i = 0; i < (long)(Rm + 1) * (Rm + 1) * (Rm + 1); ++i) map[i] = -1;
    for (long i = 0; i < ncan; ++i)
        map[((long)can[3 * i] * (Rm + 1) + can[3 * i + 1]) * (Rm + 1) + can[3 * i + 2]] = i;
    for (int dz = -Rz; dz <= Rz; ++dz)
        for (int dy = -Ry; dy <= Ry; ++dy)
            for (int dx = -Rx; dx <= Rx; ++dx) {
                int d[3] = {dx, dy, dz}, ad[3], ax[3] = {0, 1, 2};
                for (int i = 0; i < 3; ++i) ad[i] = abs(d[i]);
                /* stable sort of axes by |d| */
                for (int i = 1; i < 3; ++i) {
                    int j = i;
                    while (j > 0 && ad[ax[j - 1]] > ad[ax[j]]) {
                        int t = ax[j]; ax[j] = ax[j - 1]; ax[j - 1] = t;
                        --j;
                    }
                }
                long id = map[((long)ad[ax[0]] * (Rm + 1) + ad[ax[1]]) * (Rm + 1) + ad[ax[2]]];
                if (id < 0) continue;
                int pos[3];
                for (int j = 0; j < 3; ++j) pos[ax[j]] = j;
                const double *A = val + 9 * id;
                double tr = A[0] + A[4] + A[8];
                long off = ((long)(dz + Rz) * ny + (dy + Ry)) * nx + (dx + Rx);
                for (int p = 0; p < 3; ++p)
                    for (int q = p; q < 3; ++q) {
                        double s = 1.0;
                        if (p != q) s = (d[p] < 0 ? -1.0 : 1.0) * (d[q] < 0 ? -1.0 : 1.0);
                        double v = s * A[pos[p] * 3 + pos[q]];
                        if (p == q) v -= tr;
                        g[comp6(p, q) * n3 + off] = v;
                    }
            }
    free(map);
    free(val);
    free(can);
}

/* ------------------------------------------------------------------ */
/* direct products                                                      */
/* ------------------------------------------------------------------ */
/*
 * y = (G x) for one lag table, by direct summation (Eq. 11 without the FFT):
 *   y_p(m) = sum_q sum_d g(d)_pq x_q(m - d),  m - d inside the grid.
 * x, y: [3][Nz][Ny][Nx], x fastest.  Table as oracle_lag_table.
 */
void oracle_green_apply(int Nx, int Ny, int Nz, int Rx, int Ry, int Rz, const double *g,
                        const double *x, double *y) {
    long n = (long)Nx * Ny * Nz;
    int tx = 2 * Rx + 1, ty = 2 * Ry + 1, tz = 2 * Rz + 1;
    long t3 = (long)tx * ty * tz;
    /* list of nonzero offsets */
    long nnz = 0;
    int *off = (int *)malloc(sizeof(int) * 3 * t3);
    double *gv = (double *)malloc(sizeof(double) * 6 * t3);
    for (int dz = -Rz; dz <= Rz; ++dz)
        for (int dy = -Ry; dy <= Ry; ++dy)
            for (int dx = -Rx; dx <= Rx; ++dx) {
                long o = ((long)(dz + Rz) * ty + (dy + Ry)) * tx + (dx + Rx);
                int any = 0;
                for (int c = 0; c < 6; ++c)
                    if (g[c * t3 + o] != 0.0) any = 1;
                if (!any) continue;
                off[3 * nnz] = dx;
                off[3 * nnz + 1] = dy;
                off[3 * nnz + 2] = dz;
                for (int c = 0; c < 6; ++c) gv[6 * nnz + c] = g[c * t3 + o];
                ++nnz;
            }
#pragma omp parallel for schedule(static)
    for (long m = 0; m < n; ++m) {
        int mx = (int)(m % Nx), my = (int)((m / Nx) % Ny), mz = (int)(m / ((long)Nx * Ny));
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (long i = 0; i < nnz; ++i) {
            int sx = mx - off[3 * i], sy = my - off[3 * i + 1], sz = mz - off[3 * i + 2];
            if (sx < 0 || sx >= Nx || sy < 0 || sy >= Ny || sz < 0 || sz >= Nz) continue;
            long s = ((long)sz * Ny + sy) * Nx + sx;
            double x0 = x[s], x1 = x[n + s], x2 = x[2 * n + s];
            const double *c = gv + 6 * i;
            a0 += c[0] * x0 + c[3] * x1 + c[4] * x2;
            a1 += c[3] * x0 + c[1] * x1 + c[5] * x2;
            a2 += c[4] * x0 + c[5] * x1 + c[2] * x2;
        }
        y[m] = a0;
        y[n + m] = a1;
        y[2 * n + m] = a2;
    }
    free(off);
    free(gv);
}

/*
 * y = Z_k x = eps_r T(k dt) x - (eps_r - 1) G_k x   (Eq. 10 / Eq. 12 form).
 */
void oracle_Zk_apply(int k, int Nx, int Ny, int Nz, const double *eps, int Rx, int Ry, int Rz,
                     const double *g, const double *x, double *y) {
    long n = (long)Nx * Ny * Nz;
    double *gx = (double *)malloc(sizeof(double) * 3 * n);
    oracle_green_apply(Nx, Ny, Nz, Rx, Ry, Rz, g, x, gx);
    double Tk = oracle_temporal(k);
    for (int p = 0; p < 3; ++p)
        for (long m = 0; m < n; ++m)
            y[p * n + m] = eps[m] * Tk * x[p * n + m] - (eps[m] - 1.0) * gx[p * n + m];
    free(gx);
}

/* ------------------------------------------------------------------ */
/* incident field (Eq. 7-8)                                            */
/* ------------------------------------------------------------------ */
/*
 * b(p, m) = (eps_r(m) - 1) eps0 <d/dt E^i_p(., t)>_m, voxel average by the
 * 2x2x2 Gauss-Legendre rule.  SI units: h [m], t [s], sigma/t0 [s], f0 [Hz].
 * E^i = E0 e (1/(sigma sqrt(2 pi))) exp(-tau^2/(2 sigma^2)) cos(2 pi f0 tau),
 * tau = t - t0 - khat.(r - r_ref)/c0, r_ref the grid corner minimising khat.r.
 * pw: E0, sigma, t0, f0, khat[3], pol[3] (10 doubles).
 */
void oracle_incident(int Nx, int Ny, int Nz, double h, const double *eps, const double *pw,
                     double t, double *b) {
    const double c0 = 299792458.0, eps0 = 8.8541878128e-12;
    double E0 = pw[0], sig = pw[1], t0 = pw[2], f0 = pw[3];
    const double *kh = pw + 4, *e = pw + 7;
    double rref[3] = {kh[0] < 0 ? Nx * h : 0.0, kh[1] < 0 ? Ny * h : 0.0, kh[2] < 0 ? Nz * h : 0.0};
    double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    long n = (long)Nx * Ny * Nz;
    double amp = E0 / (sig * sqrt(2.0 * OR_PI));
#pragma omp parallel for schedule(static)
    for (long m = 0; m < n; ++m) {
        int mx = (int)(m % Nx), my = (int)((m / Nx) % Ny), mz = (int)(m / ((long)Nx * Ny));
        double acc = 0.0;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 2; ++l) {
                    double r[3] = {(mx + gp[i]) * h, (my + gp[j]) * h, (mz + gp[l]) * h};
                    double kr = kh[0] * (r[0] - rref[0]) + kh[1] * (r[1] - rref[1]) + kh[2] * (r[2] - rref[2]);
                    double tau = t - t0 - kr / c0;
                    double env = exp(-tau * tau / (2.0 * sig * sig));
                    double ph = 2.0 * OR_PI * f0 * tau;
                    double dg = amp * env * (-(tau / (sig * sig)) * cos(ph) - 2.0 * OR_PI * f0 * sin(ph));
                    acc += 0.125 * dg;
                }
        double s = (eps[m] - 1.0) * eps0 * acc;
        b[m] = s * e[0];
        b[n + m] = s * e[1];
        b[2 * n + m] = s * e[2];
    }
}

/*
 * Selected rows of y = Z_k x (same definition as oracle_Zk_apply), for
 * parity checks on grids where the full product is too slow:
 * out[i] = (Z_k x)(p_i, m_i) with m_i = (mz*Ny + my)*Nx + mx.
 */
void oracle_Zk_rows(int k, int Nx, int Ny, int Nz, const double *eps, int Rx, int Ry, int Rz, const double *g,
                    const double *x, int nrows, const int *rp, const long *rm, double *out) {
    long n = (long)Nx * Ny * Nz;
    int tx = 2 * Rx + 1, ty = 2 * Ry + 1, tz = 2 * Rz + 1;
    long t3 = (long)tx * ty * tz;
    double Tk = oracle_temporal(k);
    int cmap[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nrows; ++i) {
        int p = rp[i];
        long m = rm[i];
        int mx = (int)(m % Nx), my = (int)((m / Nx) % Ny), mz = (int)(m / ((long)Nx * Ny));
        double acc = 0.0;
        for (int dz = -Rz; dz <= Rz; ++dz)
            for (int dy = -Ry; dy <= Ry; ++dy)
                for (int dx = -Rx; dx <= Rx; ++dx) {
                    int sx = mx - dx, sy = my - dy, sz = mz - dz;
                    if (sx < 0 || sx >= Nx || sy < 0 || sy >= Ny || sz < 0 || sz >= Nz) continue;
                    long o = ((long)(dz + Rz) * ty + (dy + Ry)) * tx + (dx + Rx);
                    long s = ((long)sz * Ny + sy) * Nx + sx;
                    for (int q = 0; q < 3; ++q) acc += g[cmap[p][q] * t3 + o] * x[q * n + s];
                }
        out[i] = eps[m] * Tk * x[p * n + m] - (eps[m] - 1.0) * acc;
    }
}
