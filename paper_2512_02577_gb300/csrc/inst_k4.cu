// Kernels and launch wrappers for polynomial degree 4.
#define PMG_K 4
#define PMG_KNS k4
#define PMG_TABLE_FN kernel_table_k4
#include "inst_k.cuh"
