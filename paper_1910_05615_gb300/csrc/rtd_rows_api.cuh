// rtd_rows_api.cuh - per-width entry points of the row kernels.
#pragma once
#include "rtd_internal.cuh"

namespace rtd {

#define RTD_DECL_PB(N)                                                                              \
    void start1_pb##N(const Plan& P, cudaStream_t s);                                               \
    void start2_pb##N(const Plan& P, cudaStream_t s);                                               \
    void transform_pb##N(const Plan& P, cudaStream_t s);                                            \
    void dist_pb##N(const Plan& P, cudaStream_t s);                                                 \
    void dist_win_pb##N(const Plan& P, cudaStream_t s);                                             \
    void dist_tc_pb##N(const Plan& P, cudaStream_t s);                                              \
    void band64_pb##N(const Plan& P, cudaStream_t s);                                               \
    void grad_pb##N(const float* X, long long n, int p, long long ld, const uint8_t* wset, int wbit,   \
                    const RowParams* rp, double* partial, size_t slot_d, double* tot, double c,       \
                    double w_ld, double w_rd, GradCot cot, float* grad, int nsm, cudaStream_t s);      \
    void memb_pb##N(const Plan& P, cudaStream_t s);                                                 \
    void rew_pb##N(const Plan& P, cudaStream_t s);                                                  \
    void member_gram_pb##N(const Plan& P, cudaStream_t s);                                          \
    void score_pb##N(const float* X, long long n, int p, long long ld, const RowParams* rp,          \
                     const double* cutp, const Status* st, float* d2, uint8_t* fl,                  \
                     unsigned long long* cnt, int nsm, cudaStream_t s);                             \
    void final_pb##N(const float* X, long long n, int p, long long ld, int precision,               \
                     const RowParams* rp, const double* cutp, int decide, float* d2, uint8_t* fl,   \
                     unsigned long long* cnt, int nsm, cudaStream_t s);
RTD_DECL_PB(4)
RTD_DECL_PB(8)
RTD_DECL_PB(12)
RTD_DECL_PB(16)
RTD_DECL_PB(20)
RTD_DECL_PB(24)
RTD_DECL_PB(32)
RTD_DECL_PB(40)
RTD_DECL_PB(48)
RTD_DECL_PB(64)
#undef RTD_DECL_PB

#define RTD_PB_CALL(pb, fn, ...)                        \
    switch (pb) {                                       \
        case 4: fn##_pb4(__VA_ARGS__); break;           \
        case 8: fn##_pb8(__VA_ARGS__); break;           \
        case 12: fn##_pb12(__VA_ARGS__); break;         \
        case 16: fn##_pb16(__VA_ARGS__); break;         \
        case 20: fn##_pb20(__VA_ARGS__); break;         \
        case 24: fn##_pb24(__VA_ARGS__); break;         \
        case 32: fn##_pb32(__VA_ARGS__); break;         \
        case 40: fn##_pb40(__VA_ARGS__); break;         \
        case 48: fn##_pb48(__VA_ARGS__); break;         \
        default: fn##_pb64(__VA_ARGS__); break;         \
    }

}  // namespace rtd
