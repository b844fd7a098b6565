// Kernels and launch wrappers for polynomial degree 1.
#define PMG_K 1
#define PMG_KNS k1
#define PMG_TABLE_FN kernel_table_k1
#include "inst_k.cuh"
