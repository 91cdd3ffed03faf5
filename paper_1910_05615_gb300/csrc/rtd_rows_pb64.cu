// Row kernels instantiated for padded width 64.
#define RTD_PB 64
#include "rtd_rows_inst.cuh"
