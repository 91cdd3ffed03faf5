// rtd_rows_inst.cuh - instantiates the row kernels for one padded width
// RTD_PB (one translation unit per width, so that nvcc runs them in parallel).
#pragma once
#include "rtd_rows.cuh"

#ifndef RTD_PB
#error "define RTD_PB before including rtd_rows_inst.cuh"
#endif

#define RTD_CAT_(a, b) a##b
#define RTD_CAT(a, b) RTD_CAT_(a, b)
#define RTD_FN(name) RTD_CAT(name, RTD_PB)

namespace rtd {

void RTD_FN(start1_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) start1_t<RTD_PB, double, unsigned long long>(P, s);
    else start1_t<RTD_PB, float, uint32_t>(P, s);
}
void RTD_FN(start2_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) start2_t<RTD_PB, double, unsigned long long>(P, s);
    else start2_t<RTD_PB, float, uint32_t>(P, s);
}
void RTD_FN(transform_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) transform_t<RTD_PB, double, unsigned long long>(P, s);
    else transform_t<RTD_PB, float, uint32_t>(P, s);
}
void RTD_FN(dist_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) dist_t<RTD_PB, double>(P, s);
    else dist_t<RTD_PB, float>(P, s);
}
void RTD_FN(dist_win_pb)(const Plan& P, cudaStream_t s) { dist_win_t<RTD_PB>(P, s); }
void RTD_FN(dist_tc_pb)(const Plan& P, cudaStream_t s) { dist_tc_t<RTD_PB>(P, s); }
void RTD_FN(band64_pb)(const Plan& P, cudaStream_t s) { band64_t<RTD_PB>(P, s); }
void RTD_FN(grad_pb)(const float* X, long long n, int p, long long ld, const uint8_t* wset, int wbit,
                     const RowParams* rp, double* partial, size_t slot_d, double* tot, double c, double w_ld,
                     double w_rd, GradCot cot, float* grad, int nsm, cudaStream_t s) {
    grad_t<RTD_PB>(X, n, p, ld, wset, wbit, rp, partial, slot_d, tot, c, w_ld, w_rd, cot, grad, nsm, s);
}
void RTD_FN(memb_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) memb_t<RTD_PB, double>(P, s);
    else memb_t<RTD_PB, float>(P, s);
}
void RTD_FN(rew_pb)(const Plan& P, cudaStream_t s) {
    if (P.precision == RTD_FP64) rew_t<RTD_PB, double>(P, s);
    else rew_t<RTD_PB, float>(P, s);
}
void RTD_FN(member_gram_pb)(const Plan& P, cudaStream_t s) { member_gram_t<RTD_PB>(P, s); }
void RTD_FN(score_pb)(const float* X, long long n, int p, long long ld, const RowParams* rp, const double* cutp,
                      const Status* st, float* d2, uint8_t* fl, unsigned long long* cnt, int nsm, cudaStream_t s) {
    score_t<RTD_PB>(X, n, p, ld, rp, cutp, st, d2, fl, cnt, nsm, s);
}
void RTD_FN(final_pb)(const float* X, long long n, int p, long long ld, int precision, const RowParams* rp,
                      const double* cutp, int decide, float* d2, uint8_t* fl, unsigned long long* cnt,
                      int nsm, cudaStream_t s) {
    if (precision == RTD_FP64) final_t<RTD_PB, double>(X, n, p, ld, 0, rp, cutp, decide, d2, fl, cnt, nsm, s);
    else final_t<RTD_PB, float>(X, n, p, ld, 1, rp, cutp, decide, d2, fl, cnt, nsm, s);
}

}  // namespace rtd
