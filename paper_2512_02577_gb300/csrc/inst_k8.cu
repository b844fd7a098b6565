// Kernels and launch wrappers for polynomial degree 8.
#define PMG_K 8
#define PMG_KNS k8
#define PMG_TABLE_FN kernel_table_k8
#include "inst_k.cuh"
