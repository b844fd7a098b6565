// Kernels and launch wrappers for polynomial degree 3.
#define PMG_K 3
#define PMG_KNS k3
#define PMG_TABLE_FN kernel_table_k3
#include "inst_k.cuh"
