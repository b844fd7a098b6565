// Host-side numerical set-up (see setup.cpp).
#pragma once
#include <vector>

namespace pmg {
namespace host {

std::vector<double> gauss_points(int n, std::vector<double>* weights);
std::vector<double> gll_points(int k);
double lagrange(const std::vector<double>& nodes, int a, double x);
double lagrange_deriv(const std::vector<double>& nodes, int a, double x);
void reference_1d(int p, std::vector<double>& M, std::vector<double>& K);
void patch_1d(int p, std::vector<double>& MP, std::vector<double>& KP);
std::vector<double> p_transfer(int q, int p);
double default_omega_jacobi(int d, int p);
void fill_coefficients(int K, double* out);
void cell_tables(int p, std::vector<double>& S, std::vector<double>& Dq, std::vector<double>& W);

}  // namespace host
}  // namespace pmg
