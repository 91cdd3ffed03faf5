// rtd_common.cuh - internal definitions shared by the RT-DetMCD CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/rtdetmcd.h"

namespace rtd {

constexpr int PMAX = RTD_MAX_P;
constexpr int HIST_BITS = 12;                 // top digit of a distance key
constexpr int HIST_BINS = 1 << HIST_BITS;
// Relative half-width of the band around every threshold inside which an
// FP32 distance is recomputed in FP64 before a decision is taken.  The FP32
// error of d2 = ||M (x - mu)||^2 is bounded by about 2 gamma_p kappa(L) with
// kappa(L) < sqrt(kappa_max) = 32 for chains the condition monitor admits,
// i.e. < 2.6e-4 at p = 64; 2^-9 leaves a margin of 7.
constexpr double BAND_EPS = 1.0 / 512.0;

// ---------------------------------------------------------------- statuses
enum ChainStatus { CH_OK = 0, CH_DROPPED = 1, CH_REFUSED = 2, CH_MAXITER = 3 };

struct Status {
    int code;          // first RTD_E* error seen on the device
    int warnings;      // RTD_WARN_* bits
    int active;        // chains still iterating (C-step loop control)
    int active_blocks; // blocks with an iterating chain (written by the last finalize CTA)
    int done;          // finalize CTAs finished in this step
    int pad;
    unsigned long long n_flagged;
    unsigned long long gram_rows;   // rows the last step's Gram update touched
};

// Per-fit constants, written by the setup kernels.
struct Consts {
    int n, p, pb, q, m, hb;
    long long h;
    int precision, max_steps, rew_mode, select_path;
    double alpha, c_alpha, c_rew, cutoff_d2, kappa_max;
    double uni_cut2;          // chi2_{1,cutoff_q}
    double c1_n, c1_m;        // univariate raw consistency factors at h~/n, h~/m
    double crew1;             // univariate reweight factor
    double mu_uni[PMAX], s_uni[PMAX];
    // reweighted / raw fits (Z units)
    double mu_raw[PMAX], Sigma_raw[PMAX * PMAX];
    double mu_rew[PMAX], Sigma_rew[PMAX * PMAX];
    double logdet_raw, logdet_rew;
    double f_rew;             // factor applied to the reweighted scatter
    long long n_rew;
    int chains_ok, csteps_max;
};

// Row-pass parameters of one fit: y = M (x - mu), d2 = ||y||^2, in X units.
// M = L^-1 D^-1 (lower triangular, row-major pb x pb, zero elsewhere).
struct RowParams {
    double M[PMAX * PMAX];
    double mu[PMAX];
    float  Mf[PMAX * PMAX];
    float  mu_hi[PMAX], mu_lo[PMAX];
    // reference centre of the Gram accumulation (X units)
    double ref[PMAX];
    float  ref_hi[PMAX], ref_lo[PMAX];
    // centre folded into the product for rows centred at the FP32 univariate
    // centre u: y = M (x - u) - bf with bf = M (mu - u) (FP64, rounded once)
    float  bf[PMAX];
};

// C-step chain (one per block and start).
struct Chain {
    double mu[PMAX];            // current centre, Z units
    double Sigma[PMAX * PMAX];  // current scatter Lambda/(h_b-1), Z units
    double S[PMAX];             // sum over H of (x - ref), X units
    double G[PMAX * PMAX];      // sum over H of (x - ref)(x - ref)^T, X units
    double Sinit[PMAX * PMAX];  // initial scatter S~_k
    double V[PMAX * PMAX];      // eigenvectors of S~_k, columns, decreasing eigenvalues
    double lam[PMAX];
    double D[PMAX];             // refined eigenvalues (univariate MCD of the scores)
    double mu0[PMAX], Sigma0[PMAX * PMAX];   // refined start
    double logdet, kappa1;
    int active, steps, status, swaps;
    int full;                   // next membership pass recomputes S, G from scratch
    int full_count, started, pad;
    RowParams rp;
};

// Selection rule of one chain for the current C-step.
struct SelRule {
    unsigned long long lo, hi;      // candidate range of the compaction (coarse keys)
    unsigned long long t_lo, t_hi;  // FP32 form: band [t_lo, t_hi] of full keys
    unsigned long long t_key;       // FP64 form: threshold key
    unsigned int t_pos;             //            and position
    int below;                      // rows with coarse key < lo (atomic)
    int cand;                       // candidates (atomic)
    int band;
    // FP32 form, from the second step on: rows are classified against a
    // window [w_lo, w_hi] of FP32 keys predicted from the last thresholds.
    // When the h_b-th key and its FP64 band fall inside the window the
    // selection needs only the window's rows (fast); otherwise the
    // histogram path runs for this chain.
    unsigned int w_lo, w_hi;
    int w_sh;                       // window bin of a key: (key - w_lo) >> w_sh, < WIN_BINS
    int win;                        // this step classifies against the window
    int fast;                       // the window held
    int need_hist;                  // the window missed: histogram from the keys
    int nlo;                        // rows below the band (window path)
    int have_t;                     // t_prev holds the last threshold
    float t_prev, t_prev2;          // FP32 thresholds of the last two steps
    int bandsel;                    // histogram path: band listed, FP64 ranking pending
    int band_off;                   // offset of the band list in the chain's band buffer
    int done;                       // CTAs of the one-launch window selection finished
    int nseg;                       // window candidates: segments (CTAs per block of the distance pass)
    // counters over the whole fit (profiling)
    int acc_win, acc_miss;
    long long acc_cand, acc_band;
};
constexpr int WIN_BINS = 1024;      // bins of the window histogram
// Window candidates are listed per CTA of the distance pass: CTA b of a
// block writes its candidates from its own first row's offset on (it cannot
// have more candidates than rows) and its count to segcnt[chain][b].
constexpr int SEG_MAX = 1024;       // CTAs per block of a distance pass, at most

struct Cand {
    unsigned long long key;
    unsigned int pos;
    unsigned int pad;
};

// --------------------------------------------------------- key transforms
__host__ __device__ inline uint32_t f2key(float f) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key2f(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ inline unsigned long long d2key(double d) {
    unsigned long long u;
#ifdef __CUDA_ARCH__
    u = (unsigned long long)__double_as_longlong(d);
#else
    memcpy(&u, &d, 8);
#endif
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ inline double key2d(unsigned long long k) {
    unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

template <typename K> struct KeyOps;
template <> struct KeyOps<uint32_t> {
    typedef float value_type;
    __device__ static uint32_t enc(float v) { return f2key(v); }
    __device__ static uint32_t enc(double v) { return f2key((float)v); }
    __device__ static double dec(uint32_t k) { return (double)key2f(k); }
};
template <> struct KeyOps<unsigned long long> {
    typedef double value_type;
    __device__ static unsigned long long enc(double v) { return d2key(v); }
    __device__ static unsigned long long enc(float v) { return d2key((double)v); }
    __device__ static double dec(unsigned long long k) { return key2d(k); }
};

// Coarse 32-bit key of a non-negative distance (monotone in d2).
__device__ inline uint32_t coarse_key(float d2) { return __float_as_uint(d2); }
__device__ inline uint32_t coarse_key(double d2) { return __float_as_uint((float)d2); }

// ---- compensated FP32 pairs ("float-float", value hi + lo, about 48
// significant bits): TwoSum (Knuth), FastTwoSum and TwoProduct through FMA
// (Dekker).  Sums of 32-bit keys use them instead of FP64, whose rate is a
// small fraction of the FP32 rate on this GPU; every pair converts exactly
// to a double.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    FF s = ff_two_sum(a.hi, b.hi);
    const FF t = ff_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ FF ff_sq(FF a) {          // a^2, dropping lo^2
    const float p = a.hi * a.hi;
    float e = fmaf(a.hi, a.hi, -p);
    e = fmaf(2.f * a.hi, a.lo, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ double ff_d(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
    return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ FF ff_shfl_up(FF a, int o) {
    return FF{__shfl_up_sync(0xffffffffu, a.hi, o), __shfl_up_sync(0xffffffffu, a.lo, o)};
}

// ------------------------------------------------------ status helpers
__device__ inline void set_error(Status* st, int code) { atomicCAS(&st->code, 0, code); }
__device__ inline void set_warning(Status* st, int w) { atomicOr(&st->warnings, w); }

// -------------------------------------------------- special functions
// Regularised lower incomplete gamma P(a, x): power series for x < a + 1,
// otherwise 1 - Q(a, x) with Q by Lentz's modified continued fraction
// (Abramowitz & Stegun 6.5.29 and 6.5.31; Lentz 1976).
__host__ __device__ inline double gammp(double a, double x) {
    if (x <= 0.0) return 0.0;
    const double eps = 1e-16, tiny = 1e-300;
    double lg = lgamma(a);
    if (x < a + 1.0) {
        double ap = a, sum = 1.0 / a, del = sum;
        for (int n = 0; n < 1000; ++n) {
            ap += 1.0;
            del *= x / ap;
            sum += del;
            if (fabs(del) < fabs(sum) * eps) break;
        }
        return sum * exp(-x + a * log(x) - lg);
    }
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, hh = d;
    for (int i = 1; i < 1000; ++i) {
        double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        double del = d * c;
        hh *= del;
        if (fabs(del - 1.0) < eps) break;
    }
    return 1.0 - exp(-x + a * log(x) - lg) * hh;
}

__host__ __device__ inline double chi2_cdf(double x, int k) { return gammp(0.5 * k, 0.5 * x); }

// chi2_{k,q}: bracket by doubling, then safeguarded Newton on the CDF with
// bisection fallback, to 1e-15 relative.
__host__ __device__ inline double chi2_quantile(int k, double q) {
    if (!(q > 0.0)) return 0.0;
    if (!(q < 1.0)) return INFINITY;
    double a = 0.5 * k;
    double lo = 0.0, hi = (double)k + 10.0;
    while (chi2_cdf(hi, k) < q) { lo = hi; hi *= 2.0; }
    double x = 0.5 * (lo + hi);
    double lg = lgamma(a);
    for (int it = 0; it < 200; ++it) {
        double f = chi2_cdf(x, k) - q;
        if (f > 0.0) hi = x; else lo = x;
        double logpdf = (a - 1.0) * log(x) - 0.5 * x - a * log(2.0) - lg;
        double pdf = exp(logpdf);
        double xn = (pdf > 0.0) ? x - f / pdf : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 * x) { x = xn; break; }
        x = xn;
        if (hi - lo <= 1e-15 * hi) break;
    }
    return x;
}

// c(alpha) of eq. mcdraw: alpha / F_{chi2_{p+2}}(chi2_{p,alpha}).
__host__ __device__ inline double consistency(double alpha, int p) {
    return alpha / chi2_cdf(chi2_quantile(p, alpha), p + 2);
}

// ------------------------------------------------- warp / block helpers
__device__ inline int warp_sum_int(int v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// pb (padded p) buckets the row kernels are compiled for.
__host__ __device__ inline int pad_p(int p) {
    if (p <= 4) return 4;
    if (p <= 8) return 8;
    if (p <= 12) return 12;
    if (p <= 16) return 16;
    if (p <= 20) return 20;
    if (p <= 24) return 24;
    if (p <= 32) return 32;
    if (p <= 40) return 40;
    if (p <= 48) return 48;
    return 64;
}

#define RTD_PB_SWITCH(pb, ...)                                  \
    switch (pb) {                                               \
        case 4:  { constexpr int PB = 4;  __VA_ARGS__; } break; \
        case 8:  { constexpr int PB = 8;  __VA_ARGS__; } break; \
        case 12: { constexpr int PB = 12; __VA_ARGS__; } break; \
        case 16: { constexpr int PB = 16; __VA_ARGS__; } break; \
        case 20: { constexpr int PB = 20; __VA_ARGS__; } break; \
        case 24: { constexpr int PB = 24; __VA_ARGS__; } break; \
        case 32: { constexpr int PB = 32; __VA_ARGS__; } break; \
        case 40: { constexpr int PB = 40; __VA_ARGS__; } break; \
        case 48: { constexpr int PB = 48; __VA_ARGS__; } break; \
        default: { constexpr int PB = 64; __VA_ARGS__; } break; \
    }

}  // namespace rtd
