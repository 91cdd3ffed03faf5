// Row kernels instantiated for padded width 40.
#define RTD_PB 40
#include "rtd_rows_inst.cuh"
