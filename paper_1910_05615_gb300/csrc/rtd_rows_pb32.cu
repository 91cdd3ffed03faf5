// Row kernels instantiated for padded width 32.
#define RTD_PB 32
#include "rtd_rows_inst.cuh"
