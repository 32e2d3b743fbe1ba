// galerkin.cuh -- Galerkin interaction tables g_k(d) of the MOT-JVIE operators.
//
// Space-time discretization of Sec. II: piecewise-constant voxel basis and
// testing per Cartesian component, quadratic-spline (p = 2) temporal basis,
// Dirac temporal testing.  In voxel units (lengths in h, time in h/c0, time
// step rho = c0 dt / h = alpha/sqrt 3, Eq. 9):
//
//   K_k(R)      = B2(k + 1 - R/rho) / (4 pi R)              retarded kernel at lag k
//   W_d(s)      = prod_i L(s_i - d_i),  L(x) = max(1 - |x|, 0)  voxel-voxel weight
//   A_k(d)_pq   = int K_k(s) d_p d_q W_d(s) ds                (distributional)
//   g_k(d)_pq   = A_k(d)_pq - delta_pq sum_r A_k(d)_rr         (curl curl of Eq. 1)
//   Z_k         = eps_r T(k dt) I - (eps_r - 1) g_k            (Eq. 10 at lag k)
//
// Diagonal entries are three plane integrals (d_p^2 L = delta(.+1) - 2 delta(.) +
// delta(.-1)); mixed entries are box integrals with L'(x) = -sign(x) on (-1,1).
// Both are reduced to 1-D radial integrals in the plane normal to one axis:
// the angular factor is integrated exactly cell by cell, the radial one by
// Gauss-Legendre on panels that end at every non-analytic radius.  Singular
// panel ends are mapped away: t = t0 + s^2 at a line tangency, t = t1 - s^2
// where a kernel knot enters the z-line, t = t1 s^8 at a logarithmic origin.
// Line integrals along z use z = t sinh(u), which removes the 1/R near-singularity.
//
// All functions are __host__ __device__ so the same code fills tables on the
// GPU (one thread per lag/offset item) and on the host.
#pragma once

#include <math.h>

#include "common.cuh"

namespace mot {
namespace gk {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr int kMaxN = 32;  // largest Gauss-Legendre rule held

struct Rule {
    const double *x;  // nodes on [-1, 1]
    const double *w;  // weights
    int n;
};

MOT_HD inline double bspline2(double u) {
    if (u <= 0.0 || u >= 3.0) return 0.0;
    if (u < 1.0) return 0.5 * u * u;
    if (u < 2.0) return 0.5 * (-2.0 * u * u + 6.0 * u - 3.0);
    double v = 3.0 - u;
    return 0.5 * v * v;
}

MOT_HD inline double kernel(int k, double rho, double R) {
    return bspline2(k + 1.0 - R / rho) / (4.0 * kPi * R);
}

MOT_HD inline void sort_inplace(double *a, int n) {
    for (int i = 1; i < n; ++i) {
        double v = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

MOT_HD inline bool same(double a, double b) { return fabs(a - b) <= 1e-13 * (1.0 + fabs(a)); }

// ---------------------------------------------------------------------------
// angular factors: circle of radius t about the origin against the unit cells
// [i, i+1] x [j, j+1] of the 2x2 block centred at (a, b)
// ---------------------------------------------------------------------------
// angles in [0, 2 pi) where the circle meets u = x or v = y
MOT_HD inline int cell_angles(double t, double u0, double v0, double *th) {
    int m = 0;
    th[m++] = 0.0;
    th[m++] = 2.0 * kPi;
    for (int e = 0; e < 2; ++e) {
        double x = u0 + e;
        if (fabs(x) < t) {
            double q = acos(x / t);
            th[m++] = q;
            th[m++] = 2.0 * kPi - q;
        }
        double y = v0 + e;
        if (fabs(y) < t) {
            double q = asin(y / t);
            th[m++] = q < 0.0 ? q + 2.0 * kPi : q;
            th[m++] = kPi - q;
        }
    }
    sort_inplace(th, m);
    return m;
}

// exact integral over the arcs inside cell [u0,u0+1]x[v0,v0+1] of
// (cu0 + cu1 * t cos th) (cv0 + cv1 * t sin th)
MOT_HD inline double cell_arc_bilinear(double t, double u0, double v0, double cu0, double cu1,
                                       double cv0, double cv1) {
    double th[10];
    int m = cell_angles(t, u0, v0, th);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double a = th[i], b = th[i + 1];
        if (!(b > a)) continue;
        double mid = 0.5 * (a + b);
        double u = t * cos(mid), v = t * sin(mid);
        if (u <= u0 || u >= u0 + 1.0 || v <= v0 || v >= v0 + 1.0) continue;
        double ca = cos(a), cb = cos(b), sa = sin(a), sb = sin(b);
        acc += cu0 * cv0 * (b - a) + cu0 * cv1 * t * (ca - cb) + cu1 * cv0 * t * (sb - sa) +
               cu1 * cv1 * t * t * 0.5 * (sb * sb - sa * sa);
    }
    return acc;
}

// int_0^{2pi} L(t cos th - a) L(t sin th - b) dth
MOT_HD inline double arc_tent(double t, double a, double b) {
    double acc = 0.0;
    for (int ci = 0; ci < 2; ++ci)
        for (int cj = 0; cj < 2; ++cj) {
            double u0 = a - 1.0 + ci, v0 = b - 1.0 + cj;
            // on [a-1, a]: L = 1 - a + u ; on [a, a+1]: L = 1 + a - u
            double cu0 = ci == 0 ? 1.0 - a : 1.0 + a, cu1 = ci == 0 ? 1.0 : -1.0;
            double cv0 = cj == 0 ? 1.0 - b : 1.0 + b, cv1 = cj == 0 ? 1.0 : -1.0;
            acc += cell_arc_bilinear(t, u0, v0, cu0, cu1, cv0, cv1);
        }
    return acc;
}

// int_0^{2pi} L'(t cos th - a) L'(t sin th - b) dth,  L' = +1 on (-1,0), -1 on (0,1)
MOT_HD inline double arc_sign(double t, double a, double b) {
    double acc = 0.0;
    for (int ci = 0; ci < 2; ++ci)
        for (int cj = 0; cj < 2; ++cj) {
            double s = (ci == 0 ? 1.0 : -1.0) * (cj == 0 ? 1.0 : -1.0);
            acc += s * cell_arc_bilinear(t, a - 1.0 + ci, b - 1.0 + cj, 1.0, 0.0, 1.0, 0.0);
        }
    return acc;
}

// ---------------------------------------------------------------------------
// radial engine
// ---------------------------------------------------------------------------
enum EndKind { kSmooth = 0, kSqrt = 1, kLog = 2 };

constexpr double kPanelLen = 0.7;

struct FaceArgs {
    int k;
    double rho, c, a, b;
};
struct BoxArgs {
    int k;
    double rho, dp, dq, dr;
};

// z-line integral  int L(z - dr) K_k(sqrt(t^2 + z^2)) dz  with z = t sinh(u)
MOT_HD inline double zline(const Rule &q, int k, double rho, double t, double dr) {
    double zs[12];
    int m = 0;
    double z0 = dr - 1.0, z1 = dr + 1.0;
    zs[m++] = z0;
    zs[m++] = dr;
    zs[m++] = z1;
    for (int i = -2; i <= 1; ++i) {
        double R = (k + i) * rho;
        if (R > t) {
            double zk = sqrt(R * R - t * t);
            if (zk > z0 && zk < z1) zs[m++] = zk;
            if (-zk > z0 && -zk < z1) zs[m++] = -zk;
        }
    }
    sort_inplace(zs, m);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double za = zs[i], zb = zs[i + 1];
        if (!(zb > za)) continue;
        double ua = asinh(za / t), ub = asinh(zb / t);
        int np = (int)ceil((ub - ua) / kPanelLen);
        if (np < 1) np = 1;
        double hu = (ub - ua) / np;
        for (int p = 0; p < np; ++p) {
            double c = 0.5 * hu, mid = ua + p * hu + c;
            for (int j = 0; j < q.n; ++j) {
                double u = mid + c * q.x[j];
                double z = t * sinh(u), R = t * cosh(u);
                double w = 1.0 - fabs(z - dr);
                if (w <= 0.0) continue;
                // K(R) dz = B2(.)/(4 pi R) * t cosh(u) du = B2(.)/(4 pi) du
                acc += q.w[j] * c * w * bspline2(k + 1.0 - R / rho) * (0.25 / kPi);
            }
        }
    }
    return acc;
}

template <bool IS_FACE>
MOT_HD inline double radial_value(const Rule &q, const void *args, double t) {
    if (IS_FACE) {
        const FaceArgs *f = (const FaceArgs *)args;
        double R = sqrt(f->c * f->c + t * t);
        return kernel(f->k, f->rho, R) * arc_tent(t, f->a, f->b) * t;
    } else {
        const BoxArgs *f = (const BoxArgs *)args;
        double s = arc_sign(t, f->dp, f->dq);
        if (s == 0.0) return 0.0;
        return zline(q, f->k, f->rho, t, f->dr) * s * t;
    }
}

// one panel [t0, t1] with the given end kinds
template <bool IS_FACE>
MOT_HD inline double panel(const Rule &q, const void *args, double t0, double t1, int left, int right) {
    double acc = 0.0;
    if (left != kSmooth && right != kSmooth) {
        double tm = 0.5 * (t0 + t1);
        return panel<IS_FACE>(q, args, t0, tm, left, kSmooth) + panel<IS_FACE>(q, args, tm, t1, kSmooth, right);
    }
    if (left == kLog) {
        // t = t0 + (t1 - t0) s^8, s in [0, 1]
        double L = t1 - t0;
        for (int p = 0; p < 4; ++p) {
            double sa = p * 0.25, c = 0.125, mid = sa + c;
            for (int j = 0; j < q.n; ++j) {
                double s = mid + c * q.x[j];
                double s7 = s * s * s * s * s * s * s;
                double t = t0 + L * s7 * s;
                acc += q.w[j] * c * radial_value<IS_FACE>(q, args, t) * 8.0 * L * s7;
            }
        }
        return acc;
    }
    if (left == kSqrt || right == kSqrt) {
        // t = t0 + s^2 (left) or t = t1 - s^2 (right), s in [0, sqrt(t1 - t0)]
        double S = sqrt(t1 - t0);
        int np = (int)ceil(S / kPanelLen);
        if (np < 1) np = 1;
        double hs = S / np;
        for (int p = 0; p < np; ++p) {
            double c = 0.5 * hs, mid = p * hs + c;
            for (int j = 0; j < q.n; ++j) {
                double s = mid + c * q.x[j];
                double t = left == kSqrt ? t0 + s * s : t1 - s * s;
                acc += q.w[j] * c * radial_value<IS_FACE>(q, args, t) * 2.0 * s;
            }
        }
        return acc;
    }
    int np = (int)ceil((t1 - t0) / kPanelLen);
    if (np < 1) np = 1;
    double ht = (t1 - t0) / np;
    for (int p = 0; p < np; ++p) {
        double c = 0.5 * ht, mid = t0 + p * ht + c;
        for (int j = 0; j < q.n; ++j) acc += q.w[j] * c * radial_value<IS_FACE>(q, args, mid + c * q.x[j]);
    }
    return acc;
}

// breakpoints shared by both integral kinds: line tangencies and cell corners
// of the 2x2 block centred at (a, b)
MOT_HD inline int block_radii(double a, double b, double *br, double *tang, int *ntang, double *rmax) {
    int m = 0, nt = 0;
    *rmax = 0.0;
    for (int e = -1; e <= 1; ++e) {
        tang[nt++] = fabs(a + e);
        tang[nt++] = fabs(b + e);
    }
    for (int i = 0; i < nt; ++i) br[m++] = tang[i];
    for (int e1 = -1; e1 <= 1; ++e1)
        for (int e2 = -1; e2 <= 1; ++e2) {
            double r = sqrt((a + e1) * (a + e1) + (b + e2) * (b + e2));
            br[m++] = r;
            if (r > *rmax) *rmax = r;
        }
    *ntang = nt;
    return m;
}

MOT_HD inline bool in_list(double v, const double *s, int n) {
    for (int i = 0; i < n; ++i)
        if (same(v, s[i])) return true;
    return false;
}

// plane integral  int int K_k(sqrt(c^2 + u^2 + v^2)) L(u - a) L(v - b) du dv
MOT_HD inline double face_integral(const Rule &q, int k, double rho, double c, double a, double b) {
    double br[48], tang[6], rmax;
    int nt;
    int m = block_radii(a, b, br, tang, &nt, &rmax);
    double ac = fabs(c);
    for (int i = -2; i <= 1; ++i) {
        double R = (k + i) * rho;
        if (R > ac) br[m++] = sqrt(R * R - c * c);
    }
    double da = fmax(fabs(a) - 1.0, 0.0), db = fmax(fabs(b) - 1.0, 0.0);
    double lo = sqrt(da * da + db * db), hi = rmax;
    double Rout = (k + 1) * rho, Rin = (k - 2) * rho;
    if (Rout <= ac) return 0.0;
    hi = fmin(hi, sqrt(Rout * Rout - c * c));
    if (Rin > ac) lo = fmax(lo, sqrt(Rin * Rin - c * c));
    if (!(hi > lo)) return 0.0;
    br[m++] = lo;
    br[m++] = hi;
    sort_inplace(br, m);
    FaceArgs args = {k, rho, c, a, b};
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double t0 = br[i], t1 = br[i + 1];
        if (t0 < lo || t1 > hi || !(t1 - t0 > 1e-14 * (1.0 + t1))) continue;
        int left = (t0 > 0.0 && in_list(t0, tang, nt)) ? kSqrt : kSmooth;
        acc += panel<true>(q, &args, t0, t1, left, kSmooth);
    }
    return acc;
}

// box integral  int K_k(s) L'(s_p - dp) L'(s_q - dq) L(s_r - dr) ds
MOT_HD inline double box_integral(const Rule &q, int k, double rho, double dp, double dq, double dr) {
    double br[64], tang[6], rmax, knot_sq[4];
    int nt, nks = 0;
    int m = block_radii(dp, dq, br, tang, &nt, &rmax);
    bool zero_in = (dr - 1.0 <= 0.0) && (dr + 1.0 >= 0.0);
    for (int i = -2; i <= 1; ++i) {
        double R = (k + i) * rho;
        if (R <= 0.0) continue;
        for (int e = -1; e <= 1; ++e) {
            double ze = dr + e;
            if (R > fabs(ze)) br[m++] = sqrt(R * R - ze * ze);
        }
        if (zero_in) {
            br[m++] = R;
            knot_sq[nks++] = R;
        }
    }
    double dpp = fmax(fabs(dp) - 1.0, 0.0), dqq = fmax(fabs(dq) - 1.0, 0.0);
    double lo = sqrt(dpp * dpp + dqq * dqq), hi = rmax;
    double zmin = fmax(fabs(dr) - 1.0, 0.0), zmax = fabs(dr) + 1.0;
    double Rout = (k + 1) * rho, Rin = (k - 2) * rho;
    if (Rout <= zmin) return 0.0;
    hi = fmin(hi, sqrt(Rout * Rout - zmin * zmin));
    if (Rin > zmax) lo = fmax(lo, sqrt(Rin * Rin - zmax * zmax));
    if (!(hi > lo)) return 0.0;
    br[m++] = lo;
    br[m++] = hi;
    sort_inplace(br, m);
    BoxArgs args = {k, rho, dp, dq, dr};
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        double t0 = br[i], t1 = br[i + 1];
        if (t0 < lo || t1 > hi || !(t1 - t0 > 1e-14 * (1.0 + t1))) continue;
        int left = kSmooth, right = kSmooth;
        if (t0 == 0.0 && dr == 0.0) left = kLog;
        else if (t0 > 0.0 && in_list(t0, tang, nt)) left = kSqrt;
        if (in_list(t1, knot_sq, nks)) right = kSqrt;
        acc += panel<false>(q, &args, t0, t1, left, right);
    }
    return acc;
}

// causal support of lag k at offset d: the cube-cube distance range meets
// the shell ((k-2) rho, (k+1) rho)
MOT_HD inline bool support(int k, double rho, int dx, int dy, int dz) {
    int d[3] = {dx, dy, dz};
    double lo = 0.0, hi = 0.0;
    for (int i = 0; i < 3; ++i) {
        double a = fabs((double)d[i]);
        double l = fmax(a - 1.0, 0.0), h = a + 1.0;
        lo += l * l;
        hi += h * h;
    }
    return sqrt(lo) < (k + 1) * rho && sqrt(hi) > (k - 2) * rho;
}

// A_k(d) for d = (d0, d1, d2); out: A00, A11, A22, A01, A02, A12
MOT_HD inline void galerkin_A(const Rule &q, int k, double rho, int d0, int d1, int d2, double *out) {
    for (int i = 0; i < 6; ++i) out[i] = 0.0;
    if (!support(k, rho, d0, d1, d2)) return;
    double d[3] = {(double)d0, (double)d1, (double)d2};
    for (int p = 0; p < 3; ++p) {
        double o1 = d[(p + 1) % 3], o2 = d[(p + 2) % 3];
        out[p] = face_integral(q, k, rho, d[p] - 1.0, o1, o2) - 2.0 * face_integral(q, k, rho, d[p], o1, o2) +
                 face_integral(q, k, rho, d[p] + 1.0, o1, o2);
    }
    out[3] = box_integral(q, k, rho, d[0], d[1], d[2]);
    out[4] = box_integral(q, k, rho, d[0], d[2], d[1]);
    out[5] = box_integral(q, k, rho, d[1], d[2], d[0]);
}

// largest |d_i| with a nonzero lag-k entry (d - 1 < (k + 1) rho)
inline int reach(int k, double rho) { return (int)ceil((k + 1) * rho + 1.0 - 1e-12) - 1; }

}  // namespace gk
}  // namespace mot
