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
// Diagonal entries are second differences of plane ("face") integrals
// (d_p^2 L = delta(.+1) - 2 delta(.) + delta(.-1)); mixed entries are box
// integrals with L'(x) = -sign(x) on (-1,1).  Both are reduced to 1-D radial
// integrals in the plane normal to one axis: the angular factor is integrated
// exactly cell by cell, the radial one by Gauss-Legendre on panels that end at
// every non-analytic radius (singular ends mapped away: t = t0 + s^2 at a line
// tangency, t = t1 - s^2 where a kernel knot enters the z-line, t = t1 s^8 at a
// logarithmic origin).  The line integrals along the box axis are elementary
// and taken in closed form.
//
// All lags at once: between two knots of the B-spline (R in [j rho, (j+1) rho])
// every lag's kernel is a quadratic in s = (j+1) - R/rho divided by 4 pi R, so
// each face and box integral is computed once as three moments per knot
// interval, and the lag-k entries are fixed combinations of them.
//
// All functions are __host__ __device__ so the same code fills tables on the
// GPU (one thread per face or offset) and on the host.
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
// angular factors: circle of radius t about the origin against the 2x2 block
// of unit cells [a-1, a+1] x [b-1, b+1]
// ---------------------------------------------------------------------------
// the circle's crossings of the block's six lines u = a-1, a, a+1 and
// v = b-1, b, b+1, with cos / sin of each angle taken from the line itself
struct ArcPt {
    double th, c, s;
};

MOT_HD inline int block_crossings(double t, double a, double b, ArcPt *pt) {
    int m = 0;
    pt[m++] = {0.0, 1.0, 0.0};
    pt[m++] = {2.0 * kPi, 1.0, 0.0};
    for (int e = -1; e <= 1; ++e) {
        const double x = a + e;
        if (fabs(x) < t) {
            const double c = x / t, sn = sqrt(fmax(0.0, (1.0 - c) * (1.0 + c))), q = acos(c);
            pt[m++] = {q, c, sn};
            pt[m++] = {2.0 * kPi - q, c, -sn};
        }
        const double y = b + e;
        if (fabs(y) < t) {
            const double sn = y / t, c = sqrt(fmax(0.0, (1.0 - sn) * (1.0 + sn))), q = asin(sn);
            pt[m++] = {q < 0.0 ? q + 2.0 * kPi : q, c, sn};
            pt[m++] = {kPi - q, -c, sn};
        }
    }
    for (int i = 1; i < m; ++i) {
        ArcPt v = pt[i];
        int j = i - 1;
        while (j >= 0 && pt[j].th > v.th) {
            pt[j + 1] = pt[j];
            --j;
        }
        pt[j + 1] = v;
    }
    return m;
}

// Exact integral over the circle's arcs inside the block of the cell-wise
// function f: TENT -> L(u - a) L(v - b) (bilinear on each cell),
// otherwise L'(u - a) L'(v - b) (+-1 on each cell), u = t cos th, v = t sin th.
// Each arc between consecutive crossings lies in one cell, found from the
// arc's midpoint direction (the normalised sum of its end directions).
template <bool TENT>
MOT_HD inline double arc_block(double t, double a, double b) {
    ArcPt pt[14];
    const int m = block_crossings(t, a, b, pt);
    double acc = 0.0;
    for (int i = 0; i + 1 < m; ++i) {
        const ArcPt &A = pt[i], &B = pt[i + 1];
        const double dth = B.th - A.th;
        if (!(dth > 0.0)) continue;
        double mc = A.c + B.c, ms = A.s + B.s;
        const double nrm = sqrt(mc * mc + ms * ms);
        if (dth > 3.0 || nrm < 1e-3) {  // long arc: midpoint from the angle itself
            const double mid = 0.5 * (A.th + B.th);
            mc = cos(mid);
            ms = sin(mid);
        } else {
            mc /= nrm;
            ms /= nrm;
        }
        const double u = t * mc, v = t * ms;
        if (u <= a - 1.0 || u >= a + 1.0 || v <= b - 1.0 || v >= b + 1.0) continue;
        const bool lu = u < a, lv = v < b;
        if (TENT) {
            // on [a-1, a]: L = 1 - a + u ; on [a, a+1]: L = 1 + a - u
            const double cu0 = lu ? 1.0 - a : 1.0 + a, cu1 = lu ? 1.0 : -1.0;
            const double cv0 = lv ? 1.0 - b : 1.0 + b, cv1 = lv ? 1.0 : -1.0;
            acc += cu0 * cv0 * dth + cu0 * cv1 * t * (A.c - B.c) + cu1 * cv0 * t * (B.s - A.s) +
                   cu1 * cv1 * t * t * 0.5 * (B.s * B.s - A.s * A.s);
        } else {
            acc += (lu == lv ? dth : -dth);
        }
    }
    return acc;
}

// int_0^{2pi} L(t cos th - a) L(t sin th - b) dth
MOT_HD inline double arc_tent(double t, double a, double b) { return arc_block<true>(t, a, b); }

// int_0^{2pi} L'(t cos th - a) L'(t sin th - b) dth,  L' = +1 on (-1,0), -1 on (0,1)
MOT_HD inline double arc_sign(double t, double a, double b) { return arc_block<false>(t, a, b); }

// ---------------------------------------------------------------------------
// knot-interval moments
// ---------------------------------------------------------------------------
// On the radial interval j (R in [j rho, (j+1) rho]) the lag-k kernel is a
// quadratic in s = (j+1) - R/rho:  B2(k+1-R/rho) = sum_m b2coef(k-j, m) s^m for
// k - j in {0, 1, 2}.  Every lag's integral is therefore a combination of the
// three moments  int s^m / (4 pi R) (geometric weight)  over the intervals the
// offset's support meets, and one quadrature pass per offset serves every lag.
constexpr int kMaxIntervals = 16;  // knot intervals one support may meet (rho >= 0.25)

MOT_HD inline double b2coef(int i, int m) {
    // B2 on [i, i+1] as a polynomial in s = u - i:  s^2/2,  (1 + 2s - 2s^2)/2,  (1 - s)^2/2
    switch (3 * i + m) {
        case 2: return 0.5;
        case 3: return 0.5;
        case 4: return 1.0;
        case 5: return -1.0;
        case 6: return 0.5;
        case 7: return -1.0;
        case 8: return 0.5;
        default: return 0.0;
    }
}

enum EndKind { kSmooth = 0, kSqrt = 1, kLog = 2 };

constexpr double kPanelLen = 0.7;

// Gauss-Legendre over one panel [t0, t1] with at most one singular end:
// f(t, w) is called with each node and its weight (Jacobian included).
// Singular ends are mapped away: t = t0 + s^2 at a line tangency (left),
// t = t1 - s^2 where a kernel knot enters the z-line (right), t = t1 s^8 at a
// logarithmic origin (left).
template <class F>
MOT_HD inline void panel_one(const Rule &q, double t0, double t1, int left, int right, F &f) {
    if (left == kLog) {
        const double L = t1 - t0;
        for (int p = 0; p < 4; ++p) {
            const double c = 0.125, mid = p * 0.25 + c;
            for (int j = 0; j < q.n; ++j) {
                const double s = mid + c * q.x[j];
                const double s7 = s * s * s * s * s * s * s;
                f(t0 + L * s7 * s, q.w[j] * c * 8.0 * L * s7);
            }
        }
        return;
    }
    if (left == kSqrt || right == kSqrt) {
        const double S = sqrt(t1 - t0);
        int np = (int)ceil(S / kPanelLen);
        if (np < 1) np = 1;
        const double hs = S / np;
        for (int p = 0; p < np; ++p) {
            const double c = 0.5 * hs, mid = p * hs + c;
            for (int j = 0; j < q.n; ++j) {
                const double s = mid + c * q.x[j];
                f(left == kSqrt ? t0 + s * s : t1 - s * s, q.w[j] * c * 2.0 * s);
            }
        }
        return;
    }
    int np = (int)ceil((t1 - t0) / kPanelLen);
    if (np < 1) np = 1;
    const double ht = (t1 - t0) / np;
    for (int p = 0; p < np; ++p) {
        const double c = 0.5 * ht, mid = t0 + p * ht + c;
        for (int j = 0; j < q.n; ++j) f(mid + c * q.x[j], q.w[j] * c);
    }
}

template <class F>
MOT_HD inline void panel_acc(const Rule &q, double t0, double t1, int left, int right, F &f) {
    if (left != kSmooth && right != kSmooth) {
        const double tm = 0.5 * (t0 + t1);
        panel_one(q, t0, tm, left, kSmooth, f);
        panel_one(q, tm, t1, kSmooth, right, f);
    } else {
        panel_one(q, t0, t1, left, right, f);
    }
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

// face moments: out[3 (j - jlo) + m] += int_{R in interval j} s^m / (4 pi R)
// L(u - a) L(v - b) du dv over the plane at distance c, R = sqrt(c^2 + u^2 + v^2),
// for the intervals jlo .. jlo + nj - 1 (polar coordinates about the foot of the
// origin: exact angular factor, Gauss-Legendre in the radius t)
struct FaceNode {
    double c2, a, b, rho;
    int j;
    double *out;
    MOT_HD void operator()(double t, double w) {
        const double R = sqrt(c2 + t * t);
        const double s = (j + 1) - R / rho;
        const double v = w * arc_tent(t, a, b) * t * (0.25 / kPi) / R;
        out[0] += v;
        out[1] += v * s;
        out[2] += v * s * s;
    }
};

MOT_HD inline void face_moments(const Rule &q, double rho, double c, double a, double b, int jlo, int nj, double *out) {
    double br[24 + kMaxIntervals], tang[6], rmax;
    int nt;
    int m = block_radii(a, b, br, tang, &nt, &rmax);
    const double ac = fabs(c);
    for (int j = jlo; j <= jlo + nj; ++j) {
        const double R = j * rho;
        if (R > ac) br[m++] = sqrt(R * R - c * c);
    }
    const double da = fmax(fabs(a) - 1.0, 0.0), db = fmax(fabs(b) - 1.0, 0.0);
    double lo = sqrt(da * da + db * db), hi = rmax;
    const double Rout = (jlo + nj) * rho, Rin = jlo * rho;
    if (Rout <= ac) return;
    hi = fmin(hi, sqrt(Rout * Rout - c * c));
    if (Rin > ac) lo = fmax(lo, sqrt(Rin * Rin - c * c));
    if (!(hi > lo)) return;
    br[m++] = lo;
    br[m++] = hi;
    sort_inplace(br, m);
    FaceNode f = {c * c, a, b, rho, 0, nullptr};
    for (int i = 0; i + 1 < m; ++i) {
        const double t0 = br[i], t1 = br[i + 1];
        if (t0 < lo || t1 > hi || !(t1 - t0 > 1e-14 * (1.0 + t1))) continue;
        const double tm = 0.5 * (t0 + t1);
        int j = (int)floor(sqrt(c * c + tm * tm) / rho);
        if (j < jlo || j >= jlo + nj) continue;
        f.j = j;
        f.out = out + 3 * (j - jlo);
        const int left = (t0 > 0.0 && in_list(t0, tang, nt)) ? kSqrt : kSmooth;
        panel_acc(q, t0, t1, left, kSmooth, f);
    }
}

// asinh(zb/t) - asinh(za/t) for za <= zb without cancellation (Ra, Rb = sqrt(t^2 + z^2))
MOT_HD inline double asinh_diff(double zb, double za, double t, double Rb, double Ra) {
    if (za >= 0.0) return log1p((zb - za) * (1.0 + (zb + za) / (Rb + Ra)) / (za + Ra));
    if (zb <= 0.0) return log1p((zb - za) * (1.0 - (zb + za) / (Rb + Ra)) / (Rb - zb));
    return asinh(zb / t) + asinh(-za / t);
}

// z-line moments:  scale * int_{R in interval j} L(z - dr) s^m / (4 pi R) dz,
// R = sqrt(t^2 + z^2), added to out[3 (j - jlo) + m].  On each piece between the
// tent's kinks and the knot crossings, L = alpha + beta z and s^m / R is a
// combination of 1/R, 1 and R, whose z-antiderivatives are elementary: that
// closed form is used near the origin.  Far from it (nearest R at least four
// piece lengths) the combination cancels digits (terms ~ (j+1)^2 times the
// result), while the integrand is analytic well beyond the piece, so a short
// Gauss-Legendre rule q8 is used there instead.
MOT_HD inline void zline_moments(const Rule &q8, double t, double dr, double rho, int jlo, int nj, double scale,
                                 double *out) {
    double zs[3 + 2 * (kMaxIntervals + 1)];
    int m = 0;
    const double z0 = dr - 1.0, z1 = dr + 1.0;
    zs[m++] = z0;
    zs[m++] = dr;
    zs[m++] = z1;
    for (int j = jlo; j <= jlo + nj; ++j) {
        const double R = j * rho;
        if (R > t) {
            const double zk = sqrt(R * R - t * t);
            if (zk > z0 && zk < z1) zs[m++] = zk;
            if (-zk > z0 && -zk < z1) zs[m++] = -zk;
        }
    }
    sort_inplace(zs, m);
    const double irho = 1.0 / rho, t2 = t * t, s4 = scale * (0.25 / kPi);
    double Ra = sqrt(t2 + zs[0] * zs[0]);
    for (int i = 0; i + 1 < m; ++i) {
        const double za = zs[i], zb = zs[i + 1];
        const double Rb = sqrt(t2 + zb * zb);
        if (zb > za) {
            const double zm = 0.5 * (za + zb);
            const int j = (int)floor(sqrt(t2 + zm * zm) * irho);
            const double rmin = (za <= 0.0 && zb >= 0.0) ? t : fmin(Ra, Rb);
            if (j >= jlo && j < jlo + nj && rmin >= 4.0 * (zb - za)) {
                const double al = zm < dr ? 1.0 - dr : 1.0 + dr, be = zm < dr ? 1.0 : -1.0;
                const double c = 0.5 * (zb - za), J1 = j + 1.0;
                double m0 = 0.0, m1 = 0.0, m2 = 0.0;
                for (int g = 0; g < q8.n; ++g) {
                    const double z = zm + c * q8.x[g];
                    const double R = sqrt(t2 + z * z);
                    const double sj = J1 - R * irho;
                    const double f = q8.w[g] * (al + be * z) / R;
                    m0 += f;
                    m1 += f * sj;
                    m2 += f * sj * sj;
                }
                double *o = out + 3 * (j - jlo);
                o[0] += s4 * c * m0;
                o[1] += s4 * c * m1;
                o[2] += s4 * c * m2;
            } else if (j >= jlo && j < jlo + nj) {
                const double al = zm < dr ? 1.0 - dr : 1.0 + dr, be = zm < dr ? 1.0 : -1.0;
                const double ash = asinh_diff(zb, za, t, Rb, Ra);
                const double dz = zb - za, sz = zb + za;
                const double dR = dz * sz / (Rb + Ra);
                const double dP = al * ash + be * dR;
                const double dQ = al * dz + be * 0.5 * dz * sz;
                const double dS = al * 0.5 * ((zb * Rb - za * Ra) + t2 * ash) + be * dR * (Rb * Rb + Rb * Ra + Ra * Ra) / 3.0;
                const double J1 = j + 1.0;
                double *o = out + 3 * (j - jlo);
                o[0] += s4 * dP;
                o[1] += s4 * (J1 * dP - irho * dQ);
                o[2] += s4 * (J1 * J1 * dP - 2.0 * J1 * irho * dQ + irho * irho * dS);
            }
        }
        Ra = Rb;
    }
}

struct BoxNode {
    const Rule *q8;
    double dp, dq, dr, rho;
    int jlo, nj;
    double *out;
    MOT_HD void operator()(double t, double w) {
        const double sg = arc_sign(t, dp, dq);
        if (sg == 0.0) return;
        zline_moments(*q8, t, dr, rho, jlo, nj, w * sg * t, out);
    }
};

// box moments of int K L'(s_p - dp) L'(s_q - dq) L(s_r - dr) ds: cylindrical
// coordinates about axis r, exact angular factor, closed-form z-line, Gauss-
// Legendre in the radius t
MOT_HD inline void box_moments(const Rule &q, const Rule &q8, double rho, double dp, double dq, double dr, int jlo, int nj,
                               double *out) {
    double br[32 + 4 * (kMaxIntervals + 1)], tang[6], rmax, knot_sq[kMaxIntervals + 1];
    int nt, nks = 0;
    int m = block_radii(dp, dq, br, tang, &nt, &rmax);
    const bool zero_in = (dr - 1.0 <= 0.0) && (dr + 1.0 >= 0.0);
    for (int j = jlo; j <= jlo + nj; ++j) {
        const double R = j * rho;
        if (R <= 0.0) continue;
        for (int e = -1; e <= 1; ++e) {
            const double ze = dr + e;
            if (R > fabs(ze)) br[m++] = sqrt(R * R - ze * ze);
        }
        if (zero_in) {
            br[m++] = R;
            knot_sq[nks++] = R;
        }
    }
    const double dpp = fmax(fabs(dp) - 1.0, 0.0), dqq = fmax(fabs(dq) - 1.0, 0.0);
    double lo = sqrt(dpp * dpp + dqq * dqq), hi = rmax;
    const double zmin = fmax(fabs(dr) - 1.0, 0.0), zmax = fabs(dr) + 1.0;
    const double Rout = (jlo + nj) * rho, Rin = jlo * rho;
    if (Rout <= zmin) return;
    hi = fmin(hi, sqrt(Rout * Rout - zmin * zmin));
    if (Rin > zmax) lo = fmax(lo, sqrt(Rin * Rin - zmax * zmax));
    if (!(hi > lo)) return;
    br[m++] = lo;
    br[m++] = hi;
    sort_inplace(br, m);
    BoxNode f = {&q8, dp, dq, dr, rho, jlo, nj, out};
    for (int i = 0; i + 1 < m; ++i) {
        const double t0 = br[i], t1 = br[i + 1];
        if (t0 < lo || t1 > hi || !(t1 - t0 > 1e-14 * (1.0 + t1))) continue;
        int left = kSmooth, right = kSmooth;
        if (t0 == 0.0 && dr == 0.0) left = kLog;
        else if (t0 > 0.0 && in_list(t0, tang, nt)) left = kSqrt;
        if (in_list(t1, knot_sq, nks)) right = kSqrt;
        panel_acc(q, t0, t1, left, right, f);
    }
}

// knot intervals j (R in [j rho, (j+1) rho]) met by radii [Rmin, Rmax], within
// the intervals [jg0, jg1] that the requested lags use; false if none
MOT_HD inline bool interval_range(double rho, double Rmin, double Rmax, int jg0, int jg1, int *jlo, int *nj) {
    int a = (int)floor(Rmin / rho), b = (int)floor(Rmax / rho);
    if (a < jg0) a = jg0;
    if (b > jg1) b = jg1;
    if (a < 0) a = 0;
    if (b < a) return false;
    *jlo = a;
    *nj = b - a + 1;
    return true;
}

// lag-k value of one moment record (intervals jlo .. jlo + nj - 1, 3 moments each)
MOT_HD inline double lag_from_moments(const double *mom, int jlo, int nj, int k) {
    double acc = 0.0;
    for (int i = 0; i < 3; ++i) {
        const int j = k - i;
        if (j < jlo || j >= jlo + nj) continue;
        const double *o = mom + 3 * (j - jlo);
        acc += b2coef(i, 0) * o[0] + b2coef(i, 1) * o[1] + b2coef(i, 2) * o[2];
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

// largest |d_i| with a nonzero lag-k entry (d - 1 < (k + 1) rho)
inline int reach(int k, double rho) { return (int)ceil((k + 1) * rho + 1.0 - 1e-12) - 1; }

}  // namespace gk
}  // namespace mot
