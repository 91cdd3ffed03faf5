// Row kernels instantiated for padded width 48.
#define RTD_PB 48
#include "rtd_rows_inst.cuh"
