// Host-side problem set-up (csrc/problem.cpp): theta of Sec. 7.1.1, the
// interval of the spectrum of D, the ground-energy lower bound behind the shift,
// alpha_0 / c of Cor. lrprecond and the lowest determinants of Sec. 7.1.4.
#pragma once

#include <cstdint>
#include <vector>

namespace bsm {

std::vector<double> precond_theta(int n_orb, const double* h, const double* eri, int spin, int n_particles,
                                  double gamma);
void precond_interval(int n_orb, int spin, const double* theta, const double* h, int n_up, int n_dn, double* t_min,
                      double* t_max);
double energy_lower_bound(int n_orb, const double* h, const double* eri, int spin, int n_up, int n_dn,
                          int cholesky);
void precond_alpha0(double c0, double t_min, double c_lower, double c_upper, double* alpha0, double* c);
void lowest_determinants(int K, const double* t_diag, int spin, int n_up, int n_dn, int D, int64_t max_configs,
                         unsigned char* occ_out);

}  // namespace bsm
