// Row kernels instantiated for padded width 12.
#define RTD_PB 12
#include "rtd_rows_inst.cuh"
