/*
 * kf_oracle.h -- FP64 CPU oracle for the per-track Kalman step of the p2z / p2r
 * track-fitting mini-apps (paper section 2, "The p2r and p2z program": each
 * track is propagated to a detector surface at fixed z (propagateToZ) or fixed
 * r (propagateToR) and then Kalman-updated against its hit (KalmanUpdate)).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that the tests, the smoke
 * check and the CPU baseline of the benchmark have an independent, plain,
 * slow and obviously correct answer to compare the CUDA path against.  The
 * product path never calls it, includes it or links it, and it shares no
 * header, helper or constant table with the CUDA sources.
 *
 * The paper prints no formulas (section 2 only names the kernels).  Every
 * function below is therefore the plain definition from first principles:
 *   - exact helix motion of a charged particle in a uniform field B = (0,0,bz)
 *     (Lorentz force F = q v x B), in the half-angle form of the circle;
 *   - the transport Jacobian by differentiating that motion, with the path
 *     length eliminated through the surface constraint;
 *   - the textbook linear Kalman update (Kalman 1960; Fruhwirth 1987,
 *     NIM A262 444), standard form, plus the Joseph form.
 *
 * Conventions (readings of what the paper leaves open):
 *   state p = (x, y, z, k, phi, theta): cm, cm, cm, 1/pT in 1/GeV (k > 0),
 *   azimuth of the momentum (rad, wrapped to (-pi, pi]), polar angle (rad).
 *   charge q = +1 or -1 is held separately.
 *   signed curvature omega = -q * ALPHA * bz * k [1/cm],
 *   ALPHA = 0.299792458e-2 GeV / (cm T).
 *   symmetric 6x6 matrices are packed lower-triangular, 21 values in the order
 *   (00, 10, 11, 20, 21, 22, 30, ...); the 3x3 hit covariance is packed the
 *   same way, 6 values (xx, xy, yy, xz, yz, zz).
 *
 * Status bits (per track, OR-ed):
 *   1  no intersection with the target surface (track left unchanged)
 *   2  innovation covariance S not positive definite (update skipped)
 *   4  updated 1/pT not positive
 *   8  a non-finite value in the result
 */
#ifndef KF_ORACLE_H
#define KF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KFO_NO_INTERSECT 1u
#define KFO_S_NOT_PD     2u
#define KFO_BAD_K        4u
#define KFO_NONFINITE    8u

/* Update forms accepted by the step functions. */
#define KFO_FORM_STANDARD 0
#define KFO_FORM_JOSEPH   1

/* Propagate one track to the plane z = zt.
 * p[6] in, pout[6] out, J[36] row-major dp'/dp out (may be NULL).
 * Returns status bits: KFO_NO_INTERSECT when the track is parallel to the
 * plane, read as |cos(theta)| <= 1e-4.  On KFO_NO_INTERSECT pout = p and
 * J = identity. */
unsigned kfo_propagate_to_z(const double p[6], int q, double bz, double zt,
                            double pout[6], double J[36]);

/* Propagate one track to the cylinder x^2 + y^2 = R^2: the first outward
 * crossing of a track that starts strictly inside the cylinder.  Returns
 * KFO_NO_INTERSECT (pout = p, J = identity) when the track starts on or
 * outside the cylinder or its helix never reaches radius R. */
unsigned kfo_propagate_to_r(const double p[6], int q, double bz, double R,
                            double pout[6], double J[36]);

/* Path length helpers exposed for the tests (transverse arc length s). */
int kfo_path_to_z(const double p[6], double zt, double *s);
int kfo_path_to_r(const double p[6], int q, double bz, double R, double *s);

/* Point on the helix after transverse path s (pout[4] wrapped). */
void kfo_helix_at(const double p[6], int q, double bz, double s,
                  double pout[6]);

/* Kalman update with a 2-row linear measurement m = H p + noise.
 * p[6], C21[21] are the predicted state and covariance, H[12] row-major
 * (2x6), V[3] packed 2x2 measurement covariance, r[2] the residual m - H p.
 * form: KFO_FORM_STANDARD or KFO_FORM_JOSEPH.  Writes pout, C21out and the
 * chi-square r^T S^-1 r (chi2 may be NULL).  Returns status bits; on
 * KFO_S_NOT_PD the prediction is returned unchanged. */
unsigned kfo_kalman_update(const double p[6], const double C21[21],
                           const double H[12], const double V[3],
                           const double r[2], int form,
                           double pout[6], double C21out[21], double *chi2);

/* One full p2z step (propagate to z = zt, update against the hit with the
 * measurement (x, y)) for a single track. hit[3], hitcov[6] packed 3x3. */
unsigned kfo_p2z_step(const double p[6], const double C21[21], int q,
                      const double hit[3], const double hitcov[6],
                      double bz, double zt, int form,
                      double pout[6], double C21out[21], double *chi2);

/* One full p2r step (propagate to r = R, update against the hit with the
 * measurement (r*phi direction, z)) for a single track. */
unsigned kfo_p2r_step(const double p[6], const double C21[21], int q,
                      const double hit[3], const double hitcov[6],
                      double bz, double R, int form,
                      double pout[6], double C21out[21], double *chi2);

/* Batched forms over n tracks in AoS double arrays:
 * state[n][6], cov[n][21], charge[n], hit[n][3], hitcov[n][6],
 * surf[n] (z of the plane or r of the cylinder), outputs
 * state_out[n][6], cov_out[n][21], status[n], chi2[n] (chi2 may be NULL).
 * kind: 0 = p2z, 1 = p2r. */
void kfo_step_batch(int kind, int64_t n, const double *state,
                    const double *cov, const int8_t *charge,
                    const double *hit, const double *hitcov,
                    const double *surf, double bz, int form,
                    double *state_out, double *cov_out, uint8_t *status,
                    double *chi2);

/* Multi-layer chain: for each track, for each layer l < L in order, a p2z
 * (kinds[l] == 0) or p2r (kinds[l] == 1) step to surface pos[l] against
 * hit[l][n][3], hitcov[l][n][6].  A layer whose surface the track does not
 * reach is skipped (status bit KFO_NO_INTERSECT is set, the track is left as
 * it was) and the chain goes on with the next layer.  state/cov are updated
 * in place; status[n] is the OR over layers. */
void kfo_chain_batch(int64_t n, int L, const int *kinds, const double *pos,
                     double *state, double *cov, const int8_t *charge,
                     const double *hit, const double *hitcov, double bz,
                     int form, uint8_t *status);

#ifdef __cplusplus
}
#endif

#endif /* KF_ORACLE_H */
