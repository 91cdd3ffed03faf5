// Row kernels instantiated for padded width 8.
#define RTD_PB 8
#include "rtd_rows_inst.cuh"
