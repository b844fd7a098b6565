// Kernels and launch wrappers for polynomial degree 7.
#define PMG_K 7
#define PMG_KNS k7
#define PMG_TABLE_FN kernel_table_k7
#include "inst_k.cuh"
