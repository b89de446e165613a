// Host-side scattering post-processing: the direction set and weights for
// averages over scattering angle, the amplitude and Mueller matrices, and the
// orientation samples of the guide (all FP64, no device work).
//
//  * directions: Sec. "Averaging over Scattering Directions" -- theta values at
//    equal steps of s(theta) = theta + theta/(theta + theta0), theta0 =
//    2 pi/(1 + x), N_theta = nint(1 + 2(3 + x)/eta [1 + 1/(pi + theta0)] /
//    [1 + theta0/(pi + theta0)^2]); N_phi(j) = max(3, nint(4 pi sin theta_j /
//    (theta_{j+1} - theta_{j-1}))) equally spaced azimuths from 0 (one at the
//    poles); solid-angle weights Omega_jk of eq. (average).
//  * S_1..S_4 from f_ml: eq. (fml_rel_S_v4) and the four equations after it,
//    with a, b, c, d the y/z Lab-Frame components of e01^*, e02^*.
//  * S_ij from S_1..S_4: Sec. "Relation Between Stokes Parameters of Incident
//    and Scattered Radiation" (Bohren & Huffman's definitions).
//  * orientations: Sec. "Sampling in Theta, Phi, and beta" -- midpoints in
//    beta and Phi, uniform in cos(Theta) (midpoints for even NTHETA; end points
//    and Simpson weights, normalised to unit sum, for odd NTHETA).
#include <cmath>
#include <complex>
#include <vector>

#include "dda.h"
#include "scattering.h"

namespace dda {

using cplx = std::complex<double>;

static int nint_pos(double v) { return (int)std::floor(v + 0.5); }

void scattering_directions(double x, double eta, std::vector<double>& theta,
                           std::vector<double>& phi, std::vector<double>& omega) {
  const double pi = 3.14159265358979323846;
  const double th0 = 2.0 * pi / (1.0 + x);
  int nt = nint_pos(1.0 + 2.0 * (3.0 + x) / eta * (1.0 + 1.0 / (pi + th0)) /
                             (1.0 + th0 / ((pi + th0) * (pi + th0))));
  if (nt < 3) nt = 3;
  const double ds = (pi + pi / (pi + th0)) / (nt - 1);
  std::vector<double> th(nt);
  for (int j = 0; j < nt; ++j) {
    // the positive root of theta^2 + (1 + theta0 - s) theta - theta0 s = 0
    const double s = j * ds;
    const double bq = 1.0 + th0 - s;
    th[j] = 0.5 * (-bq + std::sqrt(bq * bq + 4.0 * th0 * s));
  }
  th[0] = 0.0;
  th[nt - 1] = pi;
  theta.clear(); phi.clear(); omega.clear();
  for (int j = 0; j < nt; ++j) {
    int np = 1;
    double om;
    if (j == 0) {
      om = 2.0 * pi * (1.0 - 0.5 * (std::cos(th[0]) + std::cos(th[1])));
    } else if (j == nt - 1) {
      om = 2.0 * pi * (0.5 * (std::cos(th[nt - 2]) + std::cos(th[nt - 1])) + 1.0);
    } else {
      np = nint_pos(4.0 * pi * std::sin(th[j]) / (th[j + 1] - th[j - 1]));
      if (np < 3) np = 3;
      om = pi * (std::cos(th[j - 1]) - std::cos(th[j + 1]));
    }
    for (int k = 0; k < np; ++k) {
      theta.push_back(th[j]);
      phi.push_back(2.0 * pi * k / np);
      omega.push_back(om / np);
    }
  }
}

void amplitude_matrix(const cplx f[2][2], const cplx e01[3], double phi_s, cplx S[4]) {
  // e02 = x_LF x e01^* has Lab-Frame components (0, -e01_z^*, e01_y^*)
  const cplx a = std::conj(e01[1]), b = std::conj(e01[2]);
  const cplx c = -e01[2], d = e01[1];  // e02^* . y, e02^* . z
  const double cp = std::cos(phi_s), sp = std::sin(phi_s);
  const cplx I(0.0, 1.0);
  const cplx u1 = a * cp + b * sp, v1 = b * cp - a * sp;  // e01 combinations
  const cplx u2 = c * cp + d * sp, v2 = d * cp - c * sp;  // e02 combinations
  S[0] = -I * (f[1][0] * v1 + f[1][1] * v2);  // S1
  S[1] = -I * (f[0][0] * u1 + f[0][1] * u2);  // S2
  S[2] = I * (f[0][0] * v1 + f[0][1] * v2);   // S3
  S[3] = I * (f[1][0] * u1 + f[1][1] * u2);   // S4
}

void mueller_matrix(const cplx S[4], double M[16]) {
  const cplx S1 = S[0], S2 = S[1], S3 = S[2], S4 = S[3];
  const double q1 = std::norm(S1), q2 = std::norm(S2), q3 = std::norm(S3), q4 = std::norm(S4);
  const cplx s23 = S2 * std::conj(S3), s14 = S1 * std::conj(S4);
  const cplx s24 = S2 * std::conj(S4), s13 = S1 * std::conj(S3);
  const cplx s12 = S1 * std::conj(S2), s34 = S3 * std::conj(S4);
  M[0] = 0.5 * (q1 + q2 + q3 + q4);
  M[1] = 0.5 * (q2 - q1 + q4 - q3);
  M[2] = (s23 + s14).real();
  M[3] = (s23 - s14).imag();
  M[4] = 0.5 * (q2 - q1 + q3 - q4);
  M[5] = 0.5 * (q1 + q2 - q3 - q4);
  M[6] = (s23 - s14).real();
  M[7] = (s23 + s14).imag();
  M[8] = (s24 + s13).real();
  M[9] = (s24 - s13).real();
  M[10] = (s12 + s34).real();
  M[11] = (std::conj(s12) + std::conj(s34)).imag();  // Im(S2 S1^* + S4 S3^*)
  M[12] = (std::conj(s24) + s13).imag();             // Im(S4 S2^* + S1 S3^*)
  M[13] = (std::conj(s24) - s13).imag();             // Im(S4 S2^* - S1 S3^*)
  M[14] = (s12 - s34).imag();
  M[15] = (s12 - s34).real();
}

AngularAverages angular_averages(int64_t n, const cplx* f1, const cplx* f2,
                                 const double* theta, const double* phi, const double* omega,
                                 double kd, double aeff) {
  AngularAverages a{};
  const double pi = 3.14159265358979323846;
  double cs = 0.0, g[3] = {0, 0, 0}, c2 = 0.0, back = 0.0, tback = -1.0;
  for (int64_t i = 0; i < n; ++i) {
    const double dc = (std::norm(f1[i]) + std::norm(f2[i])) / (kd * kd);
    const double w = omega[i] * dc;
    const double ct = std::cos(theta[i]), st = std::sin(theta[i]);
    cs += w;
    g[0] += w * ct;
    g[1] += w * st * std::cos(phi[i]);
    g[2] += w * st * std::sin(phi[i]);
    c2 += w * ct * ct;
    if (theta[i] > tback) { tback = theta[i]; back = dc; }
  }
  const double geo = pi * aeff * aeff;
  a.Qsca = cs / geo;
  for (int c = 0; c < 3; ++c) a.g[c] = cs > 0 ? g[c] / cs : 0.0;
  a.cos2 = cs > 0 ? c2 / cs : 0.0;
  a.Qbk = back / geo;
  return a;
}

void orientation_grid(const double range[6], const int n[3], double* beta, double* theta,
                      double* phi, double* wb, double* wa) {
  const int nb = n[0], nt = n[1], np = n[2];
  for (int i = 0; i < nb; ++i) {
    beta[i] = range[0] + (range[1] - range[0]) * (i + 0.5) / nb;
    wb[i] = 1.0 / nb;
  }
  for (int i = 0; i < np; ++i) phi[i] = range[4] + (range[5] - range[4]) * (i + 0.5) / np;
  const double c0 = std::cos(range[2]), c1 = std::cos(range[3]);
  std::vector<double> wt(nt);
  for (int i = 0; i < nt; ++i) {
    double c;
    if (nt == 1) {
      theta[i] = range[2];
      wt[i] = 1.0;
      continue;
    }
    if (nt % 2) {
      c = c0 + (c1 - c0) * i / (nt - 1);
      wt[i] = (i == 0 || i == nt - 1 ? 1.0 : (i % 2 ? 4.0 : 2.0)) / (3.0 * (nt - 1));
    } else {
      c = c0 + (c1 - c0) * (i + 0.5) / nt;
      wt[i] = 1.0 / nt;
    }
    theta[i] = std::acos(std::fmax(-1.0, std::fmin(1.0, c)));
  }
  for (int i = 0; i < nt; ++i)
    for (int k = 0; k < np; ++k) wa[i * np + k] = wt[i] / np;
}

void lab_axes(double theta, double phi, double beta, double x[3], double y[3], double z[3]) {
  const double ct = std::cos(theta), st = std::sin(theta);
  const double cp = std::cos(phi), sp = std::sin(phi);
  const double cb = std::cos(beta), sb = std::sin(beta);
  // rows of the inverse of (a1, a2, a3 in Lab-Frame coordinates)
  x[0] = ct;      x[1] = -st * cb;                x[2] = st * sb;
  y[0] = st * cp; y[1] = ct * cb * cp - sb * sp;  y[2] = -ct * sb * cp - cb * sp;
  z[0] = st * sp; z[1] = ct * cb * sp + sb * cp;  z[2] = -ct * sb * sp + cb * cp;
}

}  // namespace dda

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int64_t dda_scattering_directions(double x, double eta, int64_t capacity, double* theta_phi,
                                  double* omega) {
  if (!(x > 0.0) || !(eta > 0.0) || !std::isfinite(x) || !std::isfinite(eta) || eta < 1e-3)
    return -1;
  std::vector<double> th, ph, om;
  dda::scattering_directions(x, eta, th, ph, om);
  const int64_t n = (int64_t)th.size();
  for (int64_t i = 0; i < n && i < capacity; ++i) {
    if (theta_phi) { theta_phi[2 * i] = th[i]; theta_phi[2 * i + 1] = ph[i]; }
    if (omega) omega[i] = om[i];
  }
  return n;
}

dda_status dda_mueller(int64_t n, const double* f, const double* e01_lab, const double* phi_s,
                       double* S, double* M) {
  if (n < 0 || (n > 0 && (!f || !e01_lab || !phi_s))) return DDA_ERR_INVALID_ARG;
  dda::cplx e[3];
  double en = 0.0;
  for (int c = 0; c < 3; ++c) {
    e[c] = dda::cplx(e01_lab[2 * c], e01_lab[2 * c + 1]);
    en += std::norm(e[c]);
  }
  if (!(en > 0.0) || std::abs(e[0]) > 1e-6 * std::sqrt(en)) return DDA_ERR_INVALID_ARG;
  for (int c = 0; c < 3; ++c) e[c] /= std::sqrt(en);
  for (int64_t i = 0; i < n; ++i) {
    dda::cplx ff[2][2];
    for (int m = 0; m < 2; ++m)
      for (int l = 0; l < 2; ++l)
        ff[m][l] = dda::cplx(f[8 * i + 4 * m + 2 * l], f[8 * i + 4 * m + 2 * l + 1]);
    dda::cplx s[4];
    dda::amplitude_matrix(ff, e, phi_s[i], s);
    if (S)
      for (int k = 0; k < 4; ++k) { S[8 * i + 2 * k] = s[k].real(); S[8 * i + 2 * k + 1] = s[k].imag(); }
    if (M) dda::mueller_matrix(s, M + 16 * i);
  }
  return DDA_OK;
}

dda_status dda_orientation_grid(const double* range, const int* n, double* beta, double* theta,
                                double* phi, double* wbeta, double* wthetaphi) {
  if (!range || !n || !beta || !theta || !phi || !wbeta || !wthetaphi) return DDA_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (n[a] < 1 || n[a] > 4096) return DDA_ERR_INVALID_ARG;
  for (int a = 0; a < 6; ++a)
    if (!std::isfinite(range[a])) return DDA_ERR_INVALID_ARG;
  dda::orientation_grid(range, n, beta, theta, phi, wbeta, wthetaphi);
  return DDA_OK;
}

}  // extern "C"
