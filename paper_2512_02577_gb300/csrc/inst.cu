// One part of the kernel library: the kernels and launch wrappers of degree
// PMG_K (1..8), dimension PMG_DIM (2 or 3) and precision PMG_PREC (0 = double,
// 1 = float).  The build compiles this file once per part with -D flags, so
// the 32 parts compile in parallel; each exports kernel_table_k<K>_d<D>_p<P>.
#if !defined(PMG_K) || !defined(PMG_DIM) || !defined(PMG_PREC)
#error "compile with -DPMG_K=<1..8> -DPMG_DIM=<2|3> -DPMG_PREC=<0|1>"
#endif
#define PMG_CAT_(a, b) a##b
#define PMG_CAT(a, b) PMG_CAT_(a, b)
#define PMG_KNS PMG_CAT(PMG_CAT(PMG_CAT(k, PMG_K), PMG_CAT(_d, PMG_DIM)), PMG_CAT(_p, PMG_PREC))
#define PMG_TABLE_FN PMG_CAT(kernel_table_, PMG_KNS)
#include "inst_k.cuh"
