// Host-side scattering post-processing shared by the C ABI (internal).
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

namespace dda {

// (theta, phi, Omega) of the direction set for averages over scattering angle.
void scattering_directions(double x, double eta, std::vector<double>& theta,
                           std::vector<double>& phi, std::vector<double>& omega);
// S_1..S_4 from f[m][l] at azimuth phi_s; e01: unit Lab-Frame polarization 1.
void amplitude_matrix(const std::complex<double> f[2][2], const std::complex<double> e01[3],
                      double phi_s, std::complex<double> S[4]);
// Row-major 4x4 Mueller matrix S_ij from S_1..S_4.
void mueller_matrix(const std::complex<double> S[4], double M[16]);

struct AngularAverages {
  double Qsca;   // quadrature of dC_sca/dOmega, / (pi a_eff^2)
  double g[3];   // <n_LF> weighted by dC_sca/dOmega: <cos>, <sin cos phi>, <sin sin phi>
  double cos2;   // <cos^2 theta>
  double Qbk;    // dC_sca/dOmega at the largest theta in the set, / (pi a_eff^2)
};
// f1, f2: f_1l and f_2l of one incident polarization l at the n directions.
AngularAverages angular_averages(int64_t n, const std::complex<double>* f1,
                                 const std::complex<double>* f2, const double* theta,
                                 const double* phi, const double* omega, double kd,
                                 double aeff);
// beta[nb], theta[nt], phi[np], wb[nb], wa[nt * np]; range = (bmin, bmax,
// tmin, tmax, pmin, pmax), n = (nb, nt, np).
void orientation_grid(const double range[6], const int n[3], double* beta, double* theta,
                      double* phi, double* wb, double* wa);
// x_LF, y_LF, z_LF in Target-Frame coordinates for the orientation.
void lab_axes(double theta, double phi, double beta, double x[3], double y[3], double z[3]);

}  // namespace dda
