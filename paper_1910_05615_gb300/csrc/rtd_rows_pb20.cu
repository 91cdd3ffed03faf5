// Row kernels instantiated for padded width 20.
#define RTD_PB 20
#include "rtd_rows_inst.cuh"
