// rtd_internal.cuh - launchers shared between the RT-DetMCD translation units.
#pragma once
#include "rtd_common.cuh"

namespace rtd {

// Random partition of Section 4: a 4-round Feistel network over k-bit
// integers with SplitMix64 round functions, restricted to [0, n) by cycle
// walking.  Position t of the permuted order holds row perm(t).
struct Feistel {
    unsigned long long key[4];
    unsigned long long mask;
    int half;
    int identity;          // q == 1: the serial algorithm keeps the input order
    long long n;
};

__host__ __device__ inline unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Work decomposition of one fit.
struct Plan {
    long long n, h, ld;
    int p, pb, q, m, hb, precision, cpb, nsm, max_steps;
    int cpb_dist;           // CTAs per block of the distance and compaction passes
    int tc;                 // Grams on the tensor cores (split-BF16 form)
    int win_rows;           // rows per CTA, at least, of the window distance pass (0: the kernel's own)
    int sel_ctas;           // CTAs per chain of the window selection (0: 8)
    int key_bytes;          // 4 (FP32 form) or 8 (FP64 form) for refinement sorts
    long long t0;           // first permuted position of block 0 (a block range of a larger partition)
    Feistel F;
    // device buffers
    Status* st;
    Consts* cs;
    Chain* ch;
    SelRule* rule;
    RowParams* fitrp;       // raw / reweighted fit row parameters
    const float* X;         // rows as given (device), stride ld
    float* Xp;              // permuted, padded rows (stride pb), q*m rows
    int* perm;
    void* arenaA;           // sort arena (ping)
    void* arenaB;           // sort arena (pong)
    unsigned* sort_hist;
    unsigned* sort_tot;     // [2][segments][256] digit totals of the sort passes
    double* uni;            // per-segment univariate MCD results (4 doubles)
    double* uscratch;       // univariate MCD chunk sums and window argmins
    double* gss;            // per-block GSSCM cutoffs (A, B)
    void* dkeys;            // C-step distance keys [2][q*m]
    uint8_t* memb;          // [2q][m] membership bytes
    Cand* cand;             // [2q][m]
    int* segcnt;            // [2q][SEG_MAX] window candidates per distance CTA
    Cand* band;             // [2q][m]
    unsigned* hist;         // [2q][HIST_BINS]
    int* swaps;             // [2q]
    int* blk_active;        // [q] iterating chains per block after a step
    double* partial;        // Gram partial slots
    double* gsum;           // reduced Gram of each chain [2q][slot]
    size_t slot_doubles;    // doubles per slot
    uint8_t* wset;          // [q*m] reweighting set
    int* chosen;            // [q] chosen start per block (-1 none)
    int* amb;               // [q] start choice within the FP32 error band
    int* kept;              // [q] block kept by the aggregation
    double* kl;             // [q] KL deviation of each block fit
    double* scratch;        // FP64 scratch of the aggregation (p + p^2 + ...)
};

// ---- rows (rtd_rows.cu)
void launch_gather(const Plan& P, cudaStream_t s);
void launch_col_keys(const Plan& P, uint32_t* keys, cudaStream_t s);
void launch_start1(const Plan& P, cudaStream_t s);
void launch_start2(const Plan& P, cudaStream_t s);
void launch_transform(const Plan& P, int which, cudaStream_t s);
void launch_dist(const Plan& P, cudaStream_t s);
void launch_dist_win(const Plan& P, cudaStream_t s);
void launch_dist_tc(const Plan& P, cudaStream_t s);
void launch_band64(const Plan& P, cudaStream_t s);
void launch_compact(const Plan& P, cudaStream_t s);
void launch_memb(const Plan& P, cudaStream_t s);
void launch_rew(const Plan& P, cudaStream_t s);
// ---- the fit in stages (rtd_small.cu)
void launch_block_fits_out(const Plan& P, double* out, cudaStream_t s);
void launch_block_fits_in(const Plan& P, const double* in, cudaStream_t s);
void launch_moments_out(const Plan& P, double* out, cudaStream_t s);
void launch_moments_finalize(const Plan& P, const double* in, cudaStream_t s);
void launch_final(const Plan& P, float* d2_out, uint8_t* flags_out, cudaStream_t s);
void launch_subset_out(const Plan& P, uint8_t* out, cudaStream_t s);
void launch_member_gram(const Plan& P, cudaStream_t s);
void launch_score(const float* X, long long n, int p, long long ld, const RowParams* rp,
                  int precision, float* d2_out, cudaStream_t s);
void launch_flag(const float* d2, long long n, double cut, uint8_t* flags,
                 unsigned long long* count, cudaStream_t s);

// ---- sort / select (rtd_sort.cu)
void sort_segments(const Plan& P, void* keys, void* tmp, int key_bytes, int nseg,
                   long long L, cudaStream_t s);
// returns the number of kernels it launched
int launch_unimcd(const Plan& P, const void* keys, int key_bytes, int nseg, long long L,
                  int which_c1, double* out, cudaStream_t s);
size_t unimcd_scratch_doubles(int nseg, long long L);
void launch_gsscm(const Plan& P, const void* rkeys, cudaStream_t s);
void launch_select_bucket(const Plan& P, cudaStream_t s);
void launch_select_finish(const Plan& P, cudaStream_t s);
void launch_select_band(const Plan& P, cudaStream_t s);
void launch_select_fast(const Plan& P, cudaStream_t s);

// ---- small FP64 kernels (rtd_small.cu)
void launch_setup(const Plan& P, const rtd_options& o, cudaStream_t s);
void launch_uni_finish(const Plan& P, cudaStream_t s);
void launch_start_reduce(const Plan& P, cudaStream_t s);
void launch_refine_eigen(const Plan& P, cudaStream_t s);
void launch_refine_mid(const Plan& P, cudaStream_t s);
void launch_refine_end(const Plan& P, cudaStream_t s);
void launch_warm_start(const Plan& P, const double* init, cudaStream_t s);
void launch_chol_prep(const Plan& P, cudaStream_t s);
// hloop: conditional handle of a captured C-step loop (0: none)
void launch_cstep_finalize(const Plan& P, cudaStream_t s, unsigned long long hloop = 0);
// sets a captured conditional node's condition to (no error so far)
void launch_cond_ok(unsigned long long h, const Status* st, cudaStream_t s);
void launch_block_choose(const Plan& P, cudaStream_t s);
void launch_rechoose(const Plan& P, cudaStream_t s);
void launch_aggregate(const Plan& P, cudaStream_t s);
void launch_fit_prep(const Plan& P, int which, cudaStream_t s);
void launch_rew_finalize(const Plan& P, cudaStream_t s);
void launch_result(const Plan& P, rtd_result* dev_out, double* diag, cudaStream_t s);
void launch_score_prep(const double* mu, const double* Sigma, int p, RowParams* rp,
                       Status* st, cudaStream_t s, double* logdet_out = nullptr);
// A fit (mu and the lower triangle of Sigma, row by row) passed by value in
// the launch parameters of the scoring preparation: no host-to-device copy
// precedes the scoring stream.
struct FitArg {
    double mu[PMAX];
    double tri[PMAX * (PMAX + 1) / 2];
};
// (also zeroes the status word and stores the cutoff at cut_out)
void launch_score_prep_arg(const FitArg& a, int p, double cut, RowParams* rp, Status* st, double* cut_out,
                           cudaStream_t s);
// Distances and flags of the scoring call in one pass (Section 6): d2_out
// and flags nullable; FP32 rows decide in FP64 near the cutoff.  cut_dev:
// the cutoff in device memory; st: the status word of the fit's
// preparation (the FP32 pass writes nothing when it holds an error).
void launch_score_flags(const float* X, long long n, int p, long long ld, const RowParams* rp, int precision,
                        const double* cut_dev, const Status* st, float* d2_out, uint8_t* flags,
                        unsigned long long* count, cudaStream_t s);
// adjoint of steps 8-10 (rtd_rows.cu): slot count of the reduction pass
constexpr int GRAD_SLOTS = 1024;
// Cotangents of the vector-Jacobian product of the reweighted fit (device
// pointers, each nullable = zero): grd on RD (n floats; NULL = the scalar
// objective's weight w_rd on every row), gmu on mu (p doubles), gsig on
// Sigma (p x p doubles, row-major; its symmetric part is used).
struct GradCot {
    const float* grd;
    const double* gmu;
    const double* gsig;
};
// keys per tile of the segmented radix sort (threads x keys per thread)
constexpr int SORT_TILE_KEYS = 4096;
void launch_grad(const float* X, long long n, int p, long long ld, const uint8_t* wset, int wbit,
                 const RowParams* rp, double* partial, size_t slot_d, double* tot, double c, double w_ld,
                 double w_rd, GradCot cot, float* grad, int nsm, cudaStream_t s);

// Gram partial layout: blocks (bi <= bj) of 4 x 4 over the extended vector
// e = (v_0 .. v_{p-1}, 1, 0 ...) of length pe = pb + 4.
__host__ __device__ inline int gram_nb(int pb) { return (pb + 4) / 4; }
__host__ __device__ inline int gram_nblk(int pb) { int nb = gram_nb(pb); return nb * (nb + 1) / 2; }
__host__ __device__ inline int gram_blk_index(int bi, int bj, int nb) {
    return bi * nb - bi * (bi - 1) / 2 + (bj - bi);
}
// entry (i, j) of the extended Gram from one slot
__host__ __device__ inline double gram_get(const double* slot, int i, int j, int nb) {
    if (i > j) { int t = i; i = j; j = t; }
    int bi = i >> 2, bj = j >> 2;
    return slot[gram_blk_index(bi, bj, nb) * 16 + (i & 3) * 4 + (j & 3)];
}

}  // namespace rtd
