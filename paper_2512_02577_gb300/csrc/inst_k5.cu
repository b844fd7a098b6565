// Kernels and launch wrappers for polynomial degree 5.
#define PMG_K 5
#define PMG_KNS k5
#define PMG_TABLE_FN kernel_table_k5
#include "inst_k.cuh"
