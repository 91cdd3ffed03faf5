// Row kernels instantiated for padded width 24.
#define RTD_PB 24
#include "rtd_rows_inst.cuh"
