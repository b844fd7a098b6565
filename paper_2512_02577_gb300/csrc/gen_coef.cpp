// Build-time generator of the per-degree coefficient blocks as C initialiser
// macros (coef_tables.h, written into the build directory): the numbers
// fill_coefficients computes at run time for degree K (1D reference and
// patch matrices, p-transfers, h-prolongation table, Gauss tables; layout
// coef_layout(K)), printed exactly (17 significant digits for double, 9 for
// float), so that kernels can read them from compile-time tables whose
// entries the compiler folds into the unrolled 1D contractions.
#include <cstdio>
#include <vector>

#include "pmg_common.cuh"
#include "setup.h"

int main() {
  std::printf("// Generated at build time by gen_coef from fill_coefficients; not edited by hand.\n");
  std::printf("#pragma once\n");
  for (int K = 1; K <= 8; ++K) {
    std::vector<double> c(pmg::kMaxCoef, 0.0);
    pmg::host::fill_coefficients(K, c.data());
    const int n = pmg::coef_layout(K).total;
    std::printf("#define PMG_COEF64_K%d {", K);
    for (int i = 0; i < n; ++i) std::printf("%s%.17e", i ? "," : "", c[i]);
    std::printf("}\n#define PMG_COEF32_K%d {", K);
    for (int i = 0; i < n; ++i) std::printf("%s%.9ef", i ? "," : "", (double)(float)c[i]);
    std::printf("}\n");
  }
  return 0;
}
