// Row kernels instantiated for padded width 16.
#define RTD_PB 16
#include "rtd_rows_inst.cuh"
