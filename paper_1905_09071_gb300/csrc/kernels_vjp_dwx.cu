// The plain double-word path's instantiation of kernels_vjp_dw.cu (element
// type cdwx: every FFT butterfly in dw.cuh arithmetic).
#define SAG_DW_C cdwx
#include "kernels_vjp_dw.cu"
