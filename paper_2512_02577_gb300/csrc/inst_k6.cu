// Kernels and launch wrappers for polynomial degree 6.
#define PMG_K 6
#define PMG_KNS k6
#define PMG_TABLE_FN kernel_table_k6
#include "inst_k.cuh"
