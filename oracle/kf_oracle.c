/*
 * kf_oracle.c -- FP64 CPU oracle for the per-track Kalman step (p2z / p2r).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product path.  Plain scalar double
 * arithmetic, full 6x6 matrices, no blocking, no fusion, no use of the
 * sparsity of the Jacobian: a reader should be able to check every line
 * against the definitions in kf_oracle.h.
 *
 * Paper basis: section 2 ("The p2r and p2z program") names the two kernels
 * propagateToZ / propagateToR followed by KalmanUpdate and nothing more; the
 * arithmetic below is the plain physics and the textbook filter (see the
 * header for every convention this file fixes).
 *
 * Parity pins live in tests/test_oracle_pins.py (closed forms, an
 * independent Runge-Kutta integration of the Lorentz force, finite
 * differences, the information form and generalised least squares).
 */
#include "kf_oracle.h"

#include <math.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* GeV per (cm * T) for a unit charge: pT = ALPHA * B * rho. */
static const double ALPHA = 0.299792458e-2;

/* ---------------------------------------------------------------- helpers */

static int packed_index(int i, int j)
{
    if (i < j) {
        int t = i;
        i = j;
        j = t;
    }
    return i * (i + 1) / 2 + j;
}

static void unpack6(const double *c21, double C[6][6])
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            C[i][j] = c21[packed_index(i, j)];
}

static void pack6(double C[6][6], double *c21)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j)
            c21[packed_index(i, j)] = C[i][j];
}

static void unpack3(const double *c6, double C[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[i][j] = c6[packed_index(i, j)];
}

static void identity6(double J[6][6])
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            J[i][j] = (i == j) ? 1.0 : 0.0;
}

/* Azimuth wrapped to (-pi, pi]. */
static double wrap_phi(double phi)
{
    double w = fmod(phi + M_PI, 2.0 * M_PI); /* (-2pi, 2pi) */
    if (w <= 0.0)
        w += 2.0 * M_PI; /* (0, 2pi] */
    return w - M_PI;
}

/* S(h) = sin(h) / h, with S(0) = 1 (Taylor series where sin(h)/h would
 * lose digits; the next term is below 1e-26 there). */
static double sinc(double h)
{
    if (fabs(h) < 1e-4)
        return 1.0 - h * h / 6.0 + h * h * h * h / 120.0;
    return sin(h) / h;
}

/* dS/dh = (cos(h) - S(h)) / h.  Near 0 the difference cancels, so the
 * Taylor series sum_{n>=1} (-1)^n 2n h^(2n-1) / (2n+1)! is used there. */
static double dsinc(double h)
{
    if (fabs(h) < 0.05) {
        double h2 = h * h;
        return h * (-1.0 / 3.0 + h2 * (1.0 / 30.0 +
                    h2 * (-1.0 / 840.0 + h2 * (1.0 / 45360.0))));
    }
    return (cos(h) - sinc(h)) / h;
}

static void matmul6(double A[6][6], double B[6][6], double out[6][6])
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l)
                acc += A[i][l] * B[l][j];
            out[i][j] = acc;
        }
}

static void transpose6(double A[6][6], double out[6][6])
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            out[i][j] = A[j][i];
}

/* ------------------------------------------------------------ helix motion */

/* Signed curvature in 1/cm.  The Lorentz force on a positive charge in +z
 * field turns the momentum clockwise seen from +z, hence the minus sign. */
static double curvature(int q, double bz, double k)
{
    return -(double)q * ALPHA * bz * k;
}

/* Exact circle in the transverse plane, half-angle form:
 *   a = omega s (turning angle), h = a / 2,
 *   x' = x + s S(h) cos(phi + h),  y' = y + s S(h) sin(phi + h),
 *   z' = z + s cot(theta),  phi' = phi + a,  k and theta unchanged.
 * (s S(h) = 2 sin(h) / omega is the chord; at omega = 0 a straight line.) */
static void helix_point(const double p[6], double omega, double s,
                        double out[6])
{
    double h = 0.5 * omega * s;
    double chord = s * sinc(h);
    double phim = p[4] + h;
    out[0] = p[0] + chord * cos(phim);
    out[1] = p[1] + chord * sin(phim);
    out[2] = p[2] + s * cos(p[5]) / sin(p[5]);
    out[3] = p[3];
    out[4] = p[4] + omega * s; /* not wrapped here */
    out[5] = p[5];
}

void kfo_helix_at(const double p[6], int q, double bz, double s,
                  double pout[6])
{
    helix_point(p, curvature(q, bz, p[3]), s, pout);
    pout[4] = wrap_phi(pout[4]);
}

/* Partial derivatives of the helix point with respect to the start state at
 * FIXED transverse path s (6x6, row = output, column = input). */
static void helix_jacobian_fixed_s(const double p[6], int q, double bz,
                                   double s, double Js[6][6])
{
    double omega = curvature(q, bz, p[3]);
    double h = 0.5 * omega * s;
    double S = sinc(h);
    double dS = dsinc(h);
    double phim = p[4] + h;
    double domega_dk = -(double)q * ALPHA * bz;

    identity6(Js);
    /* d(chord * cos(phim)) / d omega with dh/domega = s / 2 */
    double dx_domega = 0.5 * s * s * (dS * cos(phim) - S * sin(phim));
    double dy_domega = 0.5 * s * s * (dS * sin(phim) + S * cos(phim));
    Js[0][3] = dx_domega * domega_dk;
    Js[1][3] = dy_domega * domega_dk;
    Js[4][3] = s * domega_dk;
    /* d/dphi of (x' - x, y' - y) = (-(y' - y), x' - x) */
    Js[0][4] = -s * S * sin(phim);
    Js[1][4] = s * S * cos(phim);
    /* z' = z + s cot(theta) */
    Js[2][5] = -s / (sin(p[5]) * sin(p[5]));
}

/* Derivative of the helix point with respect to s at fixed start state. */
static void helix_dpds(const double p[6], double omega, double s,
                       double dpds[6])
{
    double phi1 = p[4] + omega * s;
    dpds[0] = cos(phi1);
    dpds[1] = sin(phi1);
    dpds[2] = cos(p[5]) / sin(p[5]);
    dpds[3] = 0.0;
    dpds[4] = omega;
    dpds[5] = 0.0;
}

/* --------------------------------------------------------- path to surface */

int kfo_path_to_z(const double p[6], double zt, double *s)
{
    double c = cos(p[5]);
    /* Parallel to the plane: |cos(theta)| <= 1e-4 (|eta| below ~1e-4) is
     * treated as no intersection (the path would be > 1e4 |zt - z|). */
    if (!(fabs(c) > 1e-4) || !isfinite(p[5]))
        return 0;
    /* dz/ds = cot(theta)  =>  s = (zt - z) tan(theta) */
    *s = (zt - p[2]) * sin(p[5]) / c;
    return isfinite(*s);
}

/* g(s) = x(s)^2 + y(s)^2 - R^2 along the helix, and dg/ds. */
static void radial_residual(const double p[6], double omega, double R,
                            double s, double *g, double *dg)
{
    double pt[6];
    helix_point(p, omega, s, pt);
    *g = pt[0] * pt[0] + pt[1] * pt[1] - R * R;
    *dg = 2.0 * (pt[0] * cos(pt[4]) + pt[1] * sin(pt[4]));
}

/* Forward path length s > 0 from the start point to the point P on the
 * track circle (centre c): P - c = (sin(phi + a), -cos(phi + a)) / omega. */
static double path_to_circle_point(double phi, double omega, double cx,
                                   double cy, double px, double py)
{
    double psi = atan2(omega * (px - cx), -omega * (py - cy)); /* phi + a */
    double a = (psi - phi) * (omega > 0.0 ? 1.0 : -1.0);      /* |omega| s */
    a = fmod(a, 2.0 * M_PI);
    if (a < 0.0)
        a += 2.0 * M_PI;
    return a / fabs(omega);
}

int kfo_path_to_r(const double p[6], int q, double bz, double R, double *s)
{
    double x0 = p[0], y0 = p[1], phi = p[4];
    double r0sq = x0 * x0 + y0 * y0;
    double omega = curvature(q, bz, p[3]);
    double sol;

    if (!(r0sq < R * R) || !(R > 0.0))
        return 0; /* only outward crossings from inside the cylinder */

    if (fabs(omega) * (R + sqrt(r0sq)) < 1e-6) {
        /* Nearly straight: the positive root of |P0 + s t|^2 = R^2
         * (one root is negative because the start is inside). */
        double b = x0 * cos(phi) + y0 * sin(phi);
        double c = r0sq - R * R;
        sol = -b + sqrt(b * b - c);
    } else {
        /* Intersection of the track circle (centre c, radius rho) with the
         * circle of radius R about the origin, then the nearer of the two
         * intersection points along the direction of motion. */
        double rho = 1.0 / fabs(omega);
        double cx = x0 - sin(phi) / omega;
        double cy = y0 + cos(phi) / omega;
        double d = sqrt(cx * cx + cy * cy);
        if (d == 0.0)
            return 0; /* concentric: never crosses */
        double m = (d * d + R * R - rho * rho) / (2.0 * d);
        double hh2 = R * R - m * m;
        if (hh2 < 0.0)
            return 0; /* the circles do not meet */
        double hh = sqrt(hh2);
        double ux = cx / d, uy = cy / d;
        double p1x = m * ux - hh * uy, p1y = m * uy + hh * ux;
        double p2x = m * ux + hh * uy, p2y = m * uy - hh * ux;
        double s1 = path_to_circle_point(phi, omega, cx, cy, p1x, p1y);
        double s2 = path_to_circle_point(phi, omega, cx, cy, p2x, p2y);
        sol = (s1 < s2) ? s1 : s2;
    }

    /* Newton polish on g(s) = |P(s)|^2 - R^2 using the exact helix. */
    for (int it = 0; it < 20; ++it) {
        double g, dg;
        radial_residual(p, omega, R, sol, &g, &dg);
        if (dg == 0.0)
            break;
        double ds = g / dg;
        sol -= ds;
        if (fabs(ds) <= 1e-15 * (1.0 + fabs(sol)))
            break;
    }
    *s = sol;
    return isfinite(sol) && sol > 0.0;
}

/* ------------------------------------------------------------- propagation */

static void copy_identity_result(const double p[6], double pout[6],
                                 double *J)
{
    memcpy(pout, p, 6 * sizeof(double));
    if (J) {
        double I[6][6];
        identity6(I);
        memcpy(J, I, sizeof(I));
    }
}

unsigned kfo_propagate_to_z(const double p[6], int q, double bz, double zt,
                            double pout[6], double J[36])
{
    double s;
    if (!kfo_path_to_z(p, zt, &s)) {
        copy_identity_result(p, pout, J);
        return KFO_NO_INTERSECT;
    }
    double omega = curvature(q, bz, p[3]);
    helix_point(p, omega, s, pout);
    pout[2] = zt; /* on the plane by construction */

    if (J) {
        double Js[6][6], dpds[6], dsdp[6], Jm[6][6];
        helix_jacobian_fixed_s(p, q, bz, s, Js);
        helix_dpds(p, omega, s, dpds);
        /* s = (zt - z) tan(theta) */
        double c = cos(p[5]);
        for (int j = 0; j < 6; ++j)
            dsdp[j] = 0.0;
        dsdp[2] = -sin(p[5]) / c;
        dsdp[5] = (zt - p[2]) / (c * c);
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j)
                Jm[i][j] = Js[i][j] + dpds[i] * dsdp[j];
        /* z' = zt for every start state: its row is exactly zero (the two
         * terms above cancel analytically). */
        for (int j = 0; j < 6; ++j)
            Jm[2][j] = 0.0;
        memcpy(J, Jm, sizeof(Jm));
    }
    pout[4] = wrap_phi(pout[4]);
    return 0;
}

unsigned kfo_propagate_to_r(const double p[6], int q, double bz, double R,
                            double pout[6], double J[36])
{
    double s;
    if (!kfo_path_to_r(p, q, bz, R, &s)) {
        copy_identity_result(p, pout, J);
        return KFO_NO_INTERSECT;
    }
    double omega = curvature(q, bz, p[3]);
    helix_point(p, omega, s, pout);

    if (J) {
        double Js[6][6], dpds[6], dsdp[6], Jm[6][6];
        helix_jacobian_fixed_s(p, q, bz, s, Js);
        helix_dpds(p, omega, s, dpds);
        /* g(p, s) = x'^2 + y'^2 - R^2 = 0 defines s(p):
         * ds/dp = -(dg/dp at fixed s) / (dg/ds). */
        double dgds = 2.0 * (pout[0] * dpds[0] + pout[1] * dpds[1]);
        for (int j = 0; j < 6; ++j) {
            double dgdp = 2.0 * pout[0] * Js[0][j] + 2.0 * pout[1] * Js[1][j];
            dsdp[j] = -dgdp / dgds;
        }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j)
                Jm[i][j] = Js[i][j] + dpds[i] * dsdp[j];
        memcpy(J, Jm, sizeof(Jm));
    }
    pout[4] = wrap_phi(pout[4]);
    return 0;
}

/* ----------------------------------------------------------------- update */

static unsigned finite_check(const double p[6], const double c21[21])
{
    for (int i = 0; i < 6; ++i)
        if (!isfinite(p[i]))
            return KFO_NONFINITE;
    for (int i = 0; i < 21; ++i)
        if (!isfinite(c21[i]))
            return KFO_NONFINITE;
    return 0;
}

unsigned kfo_kalman_update(const double p[6], const double C21[21],
                           const double H[12], const double V[3],
                           const double r[2], int form,
                           double pout[6], double C21out[21], double *chi2)
{
    double C[6][6];
    unpack6(C21, C);

    /* PHt = C H^T (6x2) */
    double PHt[6][2];
    for (int i = 0; i < 6; ++i)
        for (int a = 0; a < 2; ++a) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l)
                acc += C[i][l] * H[a * 6 + l];
            PHt[i][a] = acc;
        }
    /* S = H C H^T + V (2x2) */
    double S[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0.0;
            for (int l = 0; l < 6; ++l)
                acc += H[a * 6 + l] * PHt[l][b];
            S[a][b] = acc;
        }
    S[0][0] += V[0];
    S[0][1] += V[1];
    S[1][0] += V[1];
    S[1][1] += V[2];

    double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    if (!(S[0][0] > 0.0) || !(det > 0.0)) {
        memcpy(pout, p, 6 * sizeof(double));
        memcpy(C21out, C21, 21 * sizeof(double));
        if (chi2)
            *chi2 = NAN;
        return KFO_S_NOT_PD;
    }
    double Si[2][2] = {{S[1][1] / det, -S[0][1] / det},
                       {-S[1][0] / det, S[0][0] / det}};

    /* K = C H^T S^-1 (6x2) */
    double K[6][2];
    for (int i = 0; i < 6; ++i)
        for (int b = 0; b < 2; ++b)
            K[i][b] = PHt[i][0] * Si[0][b] + PHt[i][1] * Si[1][b];

    for (int i = 0; i < 6; ++i)
        pout[i] = p[i] + K[i][0] * r[0] + K[i][1] * r[1];
    pout[4] = wrap_phi(pout[4]);

    double Cn[6][6];
    if (form == KFO_FORM_JOSEPH) {
        /* (I - K H) C (I - K H)^T + K V K^T */
        double A[6][6], AC[6][6], At[6][6], ACAt[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j)
                A[i][j] = ((i == j) ? 1.0 : 0.0) -
                          (K[i][0] * H[j] + K[i][1] * H[6 + j]);
        matmul6(A, C, AC);
        transpose6(A, At);
        matmul6(AC, At, ACAt);
        double Vm[2][2] = {{V[0], V[1]}, {V[1], V[2]}};
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double kvk = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        kvk += K[i][a] * Vm[a][b] * K[j][b];
                Cn[i][j] = ACAt[i][j] + kvk;
            }
    } else {
        /* C - K H C = C - K (C H^T)^T */
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j)
                Cn[i][j] = C[i][j] - (K[i][0] * PHt[j][0] + K[i][1] * PHt[j][1]);
    }
    pack6(Cn, C21out);

    if (chi2)
        *chi2 = r[0] * (Si[0][0] * r[0] + Si[0][1] * r[1]) +
                r[1] * (Si[1][0] * r[0] + Si[1][1] * r[1]);

    unsigned st = 0;
    if (!(pout[3] > 0.0))
        st |= KFO_BAD_K;
    return st;
}

/* -------------------------------------------------------------- full steps */

/* C' = J C J^T with full matrices. */
static void transport_covariance(const double J[36], const double C21[21],
                                 double C21out[21])
{
    double Jm[6][6], C[6][6], JC[6][6], Jt[6][6], out[6][6];
    memcpy(Jm, J, sizeof(Jm));
    unpack6(C21, C);
    matmul6(Jm, C, JC);
    transpose6(Jm, Jt);
    matmul6(JC, Jt, out);
    pack6(out, C21out);
}

unsigned kfo_p2z_step(const double p[6], const double C21[21], int q,
                      const double hit[3], const double hitcov[6],
                      double bz, double zt, int form,
                      double pout[6], double C21out[21], double *chi2)
{
    double pp[6], J[36], Cp[21];
    unsigned st = kfo_propagate_to_z(p, q, bz, zt, pp, J);
    if (st & KFO_NO_INTERSECT) {
        memcpy(pout, p, 6 * sizeof(double));
        memcpy(C21out, C21, 21 * sizeof(double));
        if (chi2)
            *chi2 = NAN;
        return st | finite_check(pout, C21out);
    }
    transport_covariance(J, C21, Cp);

    /* measurement (x, y): H = [e_x; e_y], V = top-left 2x2 of the hit
     * covariance, residual = hit - predicted position */
    double H[12] = {1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0};
    double V[3] = {hitcov[0], hitcov[1], hitcov[2]};
    double r[2] = {hit[0] - pp[0], hit[1] - pp[1]};
    st |= kfo_kalman_update(pp, Cp, H, V, r, form, pout, C21out, chi2);
    return st | finite_check(pout, C21out);
}

unsigned kfo_p2r_step(const double p[6], const double C21[21], int q,
                      const double hit[3], const double hitcov[6],
                      double bz, double R, int form,
                      double pout[6], double C21out[21], double *chi2)
{
    double pp[6], J[36], Cp[21];
    unsigned st = kfo_propagate_to_r(p, q, bz, R, pp, J);
    if (st & KFO_NO_INTERSECT) {
        memcpy(pout, p, 6 * sizeof(double));
        memcpy(C21out, C21, 21 * sizeof(double));
        if (chi2)
            *chi2 = NAN;
        return st | finite_check(pout, C21out);
    }
    transport_covariance(J, C21, Cp);

    /* measurement on the cylinder: the r*phi direction at the hit,
     * u = (-sin phi_h, cos phi_h), and z.  P projects a 3-vector onto
     * (u, e_z); H = P restricted to the position part of the state. */
    double phih = atan2(hit[1], hit[0]);
    double sh = sin(phih), ch = cos(phih);
    double P[2][3] = {{-sh, ch, 0.0}, {0.0, 0.0, 1.0}};
    double H[12] = {-sh, ch, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0};
    double Vh[3][3];
    unpack3(hitcov, Vh);
    double Vm[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    acc += P[a][i] * Vh[i][j] * P[b][j];
            Vm[a][b] = acc;
        }
    double V[3] = {Vm[0][0], Vm[0][1], Vm[1][1]};
    double d[3] = {hit[0] - pp[0], hit[1] - pp[1], hit[2] - pp[2]};
    double r[2] = {P[0][0] * d[0] + P[0][1] * d[1] + P[0][2] * d[2],
                   P[1][0] * d[0] + P[1][1] * d[1] + P[1][2] * d[2]};
    st |= kfo_kalman_update(pp, Cp, H, V, r, form, pout, C21out, chi2);
    return st | finite_check(pout, C21out);
}

void kfo_step_batch(int kind, int64_t n, const double *state,
                    const double *cov, const int8_t *charge,
                    const double *hit, const double *hitcov,
                    const double *surf, double bz, int form,
                    double *state_out, double *cov_out, uint8_t *status,
                    double *chi2)
{
    for (int64_t i = 0; i < n; ++i) {
        unsigned st;
        double c2;
        if (kind == 0)
            st = kfo_p2z_step(state + 6 * i, cov + 21 * i, charge[i],
                              hit + 3 * i, hitcov + 6 * i, bz, surf[i], form,
                              state_out + 6 * i, cov_out + 21 * i, &c2);
        else
            st = kfo_p2r_step(state + 6 * i, cov + 21 * i, charge[i],
                              hit + 3 * i, hitcov + 6 * i, bz, surf[i], form,
                              state_out + 6 * i, cov_out + 21 * i, &c2);
        status[i] = (uint8_t)st;
        if (chi2)
            chi2[i] = c2;
    }
}

void kfo_chain_batch(int64_t n, int L, const int *kinds, const double *pos,
                     double *state, double *cov, const int8_t *charge,
                     const double *hit, const double *hitcov, double bz,
                     int form, uint8_t *status)
{
    for (int64_t i = 0; i < n; ++i) {
        unsigned st = 0;
        double p[6], c[21];
        memcpy(p, state + 6 * i, sizeof(p));
        memcpy(c, cov + 21 * i, sizeof(c));
        for (int l = 0; l < L; ++l) {
            double pn[6], cn[21];
            const double *h = hit + 3 * ((int64_t)l * n + i);
            const double *hc = hitcov + 6 * ((int64_t)l * n + i);
            if (kinds[l] == 0)
                st |= kfo_p2z_step(p, c, charge[i], h, hc, bz, pos[l], form,
                                   pn, cn, NULL);
            else
                st |= kfo_p2r_step(p, c, charge[i], h, hc, bz, pos[l], form,
                                   pn, cn, NULL);
            memcpy(p, pn, sizeof(p));
            memcpy(c, cn, sizeof(c));
        }
        memcpy(state + 6 * i, p, sizeof(p));
        memcpy(cov + 21 * i, c, sizeof(c));
        status[i] = (uint8_t)st;
    }
}
