// The plain double-word path's instantiation of kernels_dw_rows.cu (element
// type cdwx: every FFT butterfly in dw.cuh arithmetic).
#define SAG_DW_C cdwx
#include "kernels_dw_rows.cu"
