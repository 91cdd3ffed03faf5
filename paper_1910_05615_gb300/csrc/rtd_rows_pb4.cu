// Row kernels instantiated for padded width 4.
#define RTD_PB 4
#include "rtd_rows_inst.cuh"
