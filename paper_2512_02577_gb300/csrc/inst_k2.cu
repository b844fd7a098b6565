// Kernels and launch wrappers for polynomial degree 2.
#define PMG_K 2
#define PMG_KNS k2
#define PMG_TABLE_FN kernel_table_k2
#include "inst_k.cuh"
