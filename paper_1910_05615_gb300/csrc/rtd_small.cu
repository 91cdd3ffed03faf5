// rtd_small.cu - FP64 p x p stages of RT-DetMCD: one CTA per chain, block
// or fit.  All matrices are in standardised (Z) units unless noted; the row
// passes receive M = L^-1 D^-1 and mu_x = mu_uni + D mu so that
// standardisation never touches the rows.
#include "rtd_internal.cuh"
#include "rtd_linalg.cuh"

namespace rtd {

constexpr int CT = 256;     // threads of the per-chain kernels
constexpr int AGG_T = 1024;
constexpr size_t MAT = (size_t)PMAX * LD;   // doubles of one shared matrix

template <typename K>
inline void big_smem(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Deterministic reduction of the Gram partial slots written by the row
// kernels: out[c][e] = sum over the CTAs b of block l = c / 2 of slot
// ((l cpb + b) 2 + c % 2)[e] (mode 0, one output per chain), or the sum of
// slot ((l cpb + b) 2)[e] over every block and CTA (mode 1, one output).
// Lanes take consecutive values, warps interleaved slots, and the warps are
// combined in a fixed order.
__global__ void __launch_bounds__(256) k_reduce_slots(const double* __restrict__ partial, size_t slot_d,
                                                      int nvals, int q, int cpb, int mode,
                                                      double* __restrict__ out) {
    __shared__ double red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    const int c = blockIdx.y;
    double acc = 0.0;
    if (e < nvals) {
        if (mode == 0) {
            const int l = c / 2, k = c % 2;
            for (int b = w; b < cpb; b += 8) acc += partial[(((size_t)l * cpb + b) * 2 + k) * slot_d + e];
        } else {
            const int ns = q * cpb;
            for (int t = w; t < ns; t += 8) acc += partial[((size_t)t * 2) * slot_d + e];
        }
    }
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0 && e < nvals) {
        double s = 0.0;
        for (int ww = 0; ww < 8; ++ww) s += red[ww][lane];
        out[(size_t)c * slot_d + e] = s;
    }
}

void launch_reduce_slots(const Plan& P, int mode, cudaStream_t s) {
    const int nv = gram_nblk(P.pb) * 16;
    dim3 grid((nv + 31) / 32, mode == 0 ? 2 * P.q : 1);
    k_reduce_slots<<<grid, 256, 0, s>>>(P.partial, P.slot_doubles, nv, P.q, P.cpb, mode, P.gsum);
}

// =====================================================================
// Constants of Section 2.1 (c(alpha), chi-square cutoffs) and of the
// univariate MCD (Section 3.1).
// =====================================================================
// Scalars of one fit, written by the host: they depend only on (n, p, h, m)
// and are the same chi-square functions the device uses.
struct SetupScalars {
    double alpha, c_alpha, cutoff_d2, c_rew, kappa_max, uni_cut2, crew1, c1_n, c1_m;
};

__global__ void k_setup(Consts* cs, long long n, int p, int pb, int q, int m, int hb, long long h,
                        int precision, int max_steps, int rew_mode, int select_path, SetupScalars sc) {
    if (threadIdx.x != 0) return;
    cs->n = (int)n; cs->p = p; cs->pb = pb; cs->q = q; cs->m = m; cs->hb = hb; cs->h = h;
    cs->precision = precision; cs->max_steps = max_steps; cs->rew_mode = rew_mode;
    cs->select_path = select_path;
    cs->alpha = sc.alpha;
    cs->c_alpha = sc.c_alpha;
    cs->cutoff_d2 = sc.cutoff_d2;
    cs->c_rew = sc.c_rew;
    cs->kappa_max = sc.kappa_max;
    cs->uni_cut2 = sc.uni_cut2;
    cs->crew1 = sc.crew1;
    cs->c1_n = sc.c1_n;
    cs->c1_m = sc.c1_m;
    cs->chains_ok = 0;
    cs->csteps_max = 0;
}

void launch_setup(const Plan& P, const rtd_options& o, cudaStream_t s) {
    SetupScalars sc;
    // Section 2.1: c(alpha), alpha = h/n; cutoff chi2_{p,q}; reweighting factor
    sc.alpha = (double)P.h / (double)P.n;
    sc.c_alpha = consistency(sc.alpha, P.p);
    sc.cutoff_d2 = chi2_quantile(P.p, o.cutoff_q);
    sc.c_rew = o.cutoff_q / chi2_cdf(sc.cutoff_d2, P.p + 2);
    sc.kappa_max = o.kappa_max;
    // Section 3.1: univariate MCD with coverage [L/2] + 1 of L = n and L = m
    sc.uni_cut2 = chi2_quantile(1, o.cutoff_q);
    sc.crew1 = o.cutoff_q / chi2_cdf(sc.uni_cut2, 3);
    sc.c1_n = consistency((double)(P.n / 2 + 1) / (double)P.n, 1);
    sc.c1_m = consistency((double)(P.m / 2 + 1) / (double)P.m, 1);
    k_setup<<<1, 32, 0, s>>>(P.cs, P.n, P.p, P.pb, P.q, P.m, P.hb, P.h, P.precision, P.max_steps,
                             o.reweight_consistency, o.select_path, sc);
}

__global__ void k_uni_finish(Consts* cs, const double* __restrict__ uni, int p, Status* st) {
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double mu = uni[4 * j], s2 = uni[4 * j + 1];
        if (!(s2 > 0.0) || !isfinite(s2) || !isfinite(mu)) {
            set_error(st, RTD_EDEGENERATE);
            cs->mu_uni[j] = 0.0;
            cs->s_uni[j] = 1.0;
        } else {
            cs->mu_uni[j] = mu;
            cs->s_uni[j] = sqrt(s2);
        }
    }
}

void launch_uni_finish(const Plan& P, cudaStream_t s) {
    k_uni_finish<<<1, 64, 0, s>>>(P.cs, P.uni, P.p, P.st);
}

// =====================================================================
// Initial scatters (Section 3.2) from the Gram partials:
//   S~_1 = covariance (n-1 denominator) of the wrapped rows,
//   S~_2 = (1/m) sum xi^2 z z^T.
// =====================================================================
__global__ void __launch_bounds__(CT) k_start_reduce(Chain* ch, const Consts* __restrict__ cs,
                                                     const double* __restrict__ gsum, size_t slot_d) {
    const int c = blockIdx.x, k = c % 2;
    const int p = cs->p, nb = gram_nb(cs->pb);
    const double* ext = gsum + (size_t)c * slot_d;
    Chain& C = ch[c];
    const double cnt = gram_get(ext, p, p, nb);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double g = gram_get(ext, i, j, nb);
        double v;
        if (k == 0) {
            double si = gram_get(ext, i, p, nb), sj = gram_get(ext, j, p, nb);
            v = (g - si * sj / cnt) / (cnt - 1.0);
        } else {
            v = g / (double)cs->m;
        }
        C.Sinit[i * PMAX + j] = v;
    }
    if (threadIdx.x == 0) {
        C.status = CH_OK; C.active = 0; C.steps = 0; C.full = 1; C.full_count = 0;
        C.swaps = 0; C.started = 0; C.logdet = NAN; C.kappa1 = NAN;
    }
}

void launch_start_reduce(const Plan& P, cudaStream_t s) {
    launch_reduce_slots(P, 0, s);
    k_start_reduce<<<2 * P.q, CT, 0, s>>>(P.ch, P.cs, P.gsum, P.slot_doubles);
}

// =====================================================================
// Refinement (Section 3.3).
// eigen: S~_k = V D V^T, drop when lambda_1/lambda_p > kappa_max, and the
//        score transform W = V^T D_uni^-1 (T = Z V).
// mid:   Sigma_k = V diag(sigma_uni^2(T_j)) V^T and the sphering transform
//        W = Sigma_k^{-1/2} D_uni^-1.
// end:   mu_k = Sigma_k^{1/2} (mu_uni(Z~_j))_j; the chain starts here.
// Chain.G holds W while the refinement runs.
// =====================================================================
__global__ void __launch_bounds__(CT) k_refine_eigen(Chain* ch, const Consts* __restrict__ cs, Status* st) {
    extern __shared__ double sm[];
    double* A = sm;
    double* V = sm + MAT;
    double* Vs = sm + 2 * MAT;
    __shared__ double lam[PMAX];
    __shared__ int bad;
    Chain& C = ch[blockIdx.x];
    const int p = cs->p;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = C.Sinit[i * PMAX + j];
        if (!isfinite(v)) bad = 1;
        A[i * LD + j] = v;
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) { C.status = CH_DROPPED; set_warning(st, RTD_WARN_DROPPED_START); }
        return;
    }
    cta_jacobi_mixed(A, V, p, lam, Vs, sm + 3 * MAT);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        C.V[i * PMAX + j] = Vs[i * LD + j];
        // W[j][i] = V_ij / sigma_uni_i  (output j = score j)
        C.G[j * PMAX + i] = Vs[i * LD + j] / cs->s_uni[i];
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) C.lam[j] = lam[j];
    if (threadIdx.x == 0) {
        double l1 = lam[0], lp = lam[p - 1];
        if (!(lp > 0.0) || l1 / lp > cs->kappa_max || !isfinite(l1)) {
            C.status = CH_DROPPED;
            set_warning(st, RTD_WARN_DROPPED_START);
        }
    }
}

void launch_refine_eigen(const Plan& P, cudaStream_t s) {
    size_t sm = 4 * MAT * sizeof(double);
    auto k = k_refine_eigen;
    big_smem(k, sm);
    k<<<2 * P.q, CT, sm, s>>>(P.ch, P.cs, P.st);
}

__global__ void __launch_bounds__(CT) k_refine_mid(Chain* ch, const Consts* __restrict__ cs,
                                                   const double* __restrict__ uni, Status* st) {
    __shared__ double d[PMAX], dih[PMAX];
    __shared__ int bad;
    const int c = blockIdx.x;
    Chain& C = ch[c];
    if (C.status != CH_OK) return;
    const int p = cs->p;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double v = uni[4 * ((size_t)c * p + j) + 1];
        if (!(v > 0.0) || !isfinite(v)) bad = 1;
        d[j] = v;
        dih[j] = 1.0 / sqrt(v);
        C.D[j] = v;
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) { C.status = CH_DROPPED; set_warning(st, RTD_WARN_DROPPED_START); }
        return;
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double sg = 0.0, sh = 0.0;
        for (int t = 0; t < p; ++t) {
            double vi = C.V[i * PMAX + t], vj = C.V[j * PMAX + t];
            sg += vi * d[t] * vj;
            sh += vi * dih[t] * vj;
        }
        C.Sigma0[i * PMAX + j] = sg;
        // W[i][j] = (Sigma^{-1/2})_ij / sigma_uni_j
        C.G[i * PMAX + j] = sh / cs->s_uni[j];
    }
}

void launch_refine_mid(const Plan& P, cudaStream_t s) {
    k_refine_mid<<<2 * P.q, CT, 0, s>>>(P.ch, P.cs, P.uni, P.st);
}

__global__ void __launch_bounds__(CT) k_refine_end(Chain* ch, const Consts* __restrict__ cs,
                                                   const double* __restrict__ uni, Status* st) {
    __shared__ double mt[PMAX], u[PMAX];
    __shared__ int bad;
    const int c = blockIdx.x;
    Chain& C = ch[c];
    if (C.status != CH_OK) return;
    const int p = cs->p;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double v = uni[4 * ((size_t)c * p + j)];
        if (!isfinite(v)) bad = 1;
        mt[j] = v;
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) { C.status = CH_DROPPED; set_warning(st, RTD_WARN_DROPPED_START); }
        return;
    }
    // u = D^{1/2} V^T mu~ ;  mu = V u
    for (int t = threadIdx.x; t < p; t += blockDim.x) {
        double a = 0.0;
        for (int i = 0; i < p; ++i) a += C.V[i * PMAX + t] * mt[i];
        u[t] = a * sqrt(C.D[t]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double a = 0.0;
        for (int t = 0; t < p; ++t) a += C.V[i * PMAX + t] * u[t];
        C.mu0[i] = a;
        C.mu[i] = a;
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        C.Sigma[i * PMAX + j] = C.Sigma0[i * PMAX + j];
    }
    if (threadIdx.x == 0) { C.active = 1; C.full = 1; C.steps = 0; C.started = 1; }
}

void launch_refine_end(const Plan& P, cudaStream_t s) {
    k_refine_end<<<2 * P.q, CT, 0, s>>>(P.ch, P.cs, P.uni, P.st);
}

// =====================================================================
// Warm start (end of Section 4): the given fit (X units, init = mu then
// Sigma row-major) standardises Z by its centre and diagonal, and starts
// the one chain of every block (mu_z = 0, Sigma_z = D^-1 Sigma D^-1); the
// block's second chain has no start.
// =====================================================================
__global__ void __launch_bounds__(CT) k_warm_start(Chain* ch, Consts* cs, const double* __restrict__ init) {
    __shared__ double rs[PMAX];
    const int c = blockIdx.x;
    const int p = cs->p;
    const double* mu = init;
    const double* S = init + p;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const double d = sqrt(S[(size_t)j * p + j]);
        rs[j] = 1.0 / d;
        if (c == 0) { cs->mu_uni[j] = mu[j]; cs->s_uni[j] = d; }
    }
    __syncthreads();
    Chain& C = ch[c];
    if (c & 1) {
        if (threadIdx.x == 0) { C.active = 0; C.status = CH_DROPPED; }
        return;
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        const double v = S[(size_t)i * p + j] * rs[i] * rs[j];
        C.Sigma[i * PMAX + j] = v;
        C.Sigma0[i * PMAX + j] = v;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) { C.mu[j] = 0.0; C.mu0[j] = 0.0; }
    if (threadIdx.x == 0) { C.status = CH_OK; C.active = 1; C.full = 1; C.steps = 0; C.started = 1; }
}

void launch_warm_start(const Plan& P, const double* init, cudaStream_t s) {
    k_warm_start<<<2 * P.q, CT, 0, s>>>(P.ch, P.cs, init);
}

// =====================================================================
// Row parameters of a fit (mu, Sigma in Z units): Cholesky Sigma = L L^T
// (Section 3.4), M = L^-1 D^-1, mu_x = mu_uni + D mu, FP32 copies with the
// centre split into hi + lo.  Returns false if Sigma is not positive
// definite.  Leaves L in A and L^-1 in Li.
// =====================================================================
__device__ bool make_rowparams(const double* __restrict__ mu_z, const double* __restrict__ S_z,
                               const double* __restrict__ mu_uni, const double* __restrict__ s_uni,
                               int p, double* A, double* Li, RowParams& rp, double* logdet) {
    __shared__ double inv_s[PMAX], dm[PMAX], rdg[PMAX];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        A[i * LD + j] = S_z[i * PMAX + j];
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) inv_s[j] = 1.0 / s_uni[j];
    if (!cta_cholesky(A, p, rdg)) return false;
    // log det = 2 sum log L_jj, taken by the last warp while the others invert L
    double ld = 0.0;
    const int lw = (int)(blockDim.x >> 5) - 1;
    if (lw > 0) {
        if ((int)(threadIdx.x >> 5) == lw)
            for (int j = threadIdx.x & 31; j < p; j += 32) ld += log(A[j * LD + j]);
    } else {
        for (int j = threadIdx.x; j < p; j += blockDim.x) ld += log(A[j * LD + j]);
    }
    cta_tri_inverse(A, Li, p, rdg);
    ld = 2.0 * cta_sum(ld);
    *logdet = ld;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = (j <= i) ? Li[i * LD + j] * inv_s[j] : 0.0;
        rp.M[i * PMAX + j] = v;
        rp.Mf[i * PMAX + j] = (float)v;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double mx = mu_uni[j] + s_uni[j] * mu_z[j];
        rp.mu[j] = mx;
        float hi = (float)mx;
        rp.mu_hi[j] = hi;
        rp.mu_lo[j] = (float)(mx - (double)hi);
        // centre offset from the FP32 univariate centre u, in Z units
        dm[j] = (mx - (double)(float)mu_uni[j]) * inv_s[j];
    }
    __syncthreads();
    // bf = M (mu - u) = Li D^-1 (mu - u)
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a = fma(Li[i * LD + j], dm[j], a);
        rp.bf[i] = (float)a;
    }
    __syncthreads();
    return true;
}

// FP32 form: the window of keys the distance pass classifies against,
// predicted from the chain's last two thresholds (none before the first
// selection: the histogram path runs).
__device__ inline void set_window(SelRule& R, int fp32, int path) {
    R.below = 0; R.cand = 0; R.band = 0; R.nlo = 0; R.done = 0;
    R.fast = 0; R.need_hist = 0; R.bandsel = 0; R.band_off = 0;
    R.win = 0;
    if (!fp32 || path == 1 || !R.have_t || !(R.t_prev >= 0.f) || !isfinite(R.t_prev)) return;
    // centre: the last threshold.  Half-width: twice the last relative
    // change, within [4 eps, 1/2]; 1/2 for the first window (one threshold
    // known), whose step moves from the refined start to the first h-subset
    // scatter and shifts the threshold by tens of percent.
    const float t = R.t_prev;
    float d = 0.5f;
    if (R.t_prev2 > 0.f && t > 0.f) d = 2.f * fabsf(t - R.t_prev2) / t;
    d = fminf(fmaxf(d, 4.f * (float)BAND_EPS), 0.5f);
    if (path == 2) d = 4.f * (float)BAND_EPS;
    R.w_lo = __float_as_uint(t * (1.f - d));
    R.w_hi = __float_as_uint(t * (1.f + d));
    int sh = 0;
    while (((R.w_hi - R.w_lo) >> sh) >= (unsigned)WIN_BINS) ++sh;
    R.w_sh = sh;
    R.win = 1;
}

__device__ inline void clear_rule(SelRule& R) {
    R.win = 0; R.fast = 0; R.bandsel = 0; R.need_hist = 0; R.cand = 0; R.band = 0;
}

// Condition monitor (Section 3.4) and row parameters of a chain's current
// (mu, Sigma), and the selection window of its next step.  False when the
// chain is refused.  sm: 3 MAT doubles of shared memory.
__device__ bool chain_prep(Chain& C, SelRule& R, const Consts* __restrict__ cs, int* swap_slot, Status* st,
                           double* sm) {
    double* A = sm;
    double* Li = sm + MAT;
    double* S = sm + 2 * MAT;
    __shared__ double s_ld;
    const int p = cs->p;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        S[i * LD + j] = C.Sigma[i * PMAX + j];
    }
    if (threadIdx.x == 0) {
        *swap_slot = 0;
        set_window(R, cs->precision == RTD_FP32, cs->select_path);
    }
    __syncthreads();
    bool ok = make_rowparams(C.mu, C.Sigma, cs->mu_uni, cs->s_uni, p, A, Li, C.rp, &s_ld);
    double k1 = ok ? cta_kappa1(S, Li, A, p) : INFINITY;
    if (!ok || !(k1 < cs->kappa_max)) {
        if (threadIdx.x == 0) {
            C.active = 0;
            C.status = CH_REFUSED;
            C.kappa1 = k1;
            clear_rule(R);
            set_warning(st, RTD_WARN_CSTEP_REFUSED);
        }
        __syncthreads();
        return false;
    }
    if (C.full) {
        for (int j = threadIdx.x; j < p; j += blockDim.x) {
            C.rp.ref[j] = C.rp.mu[j];
            C.rp.ref_hi[j] = C.rp.mu_hi[j];
            C.rp.ref_lo[j] = C.rp.mu_lo[j];
        }
    }
    if (threadIdx.x == 0) { C.logdet = s_ld; C.kappa1 = k1; }
    __syncthreads();
    return true;
}

// Before the first C-step.
__global__ void __launch_bounds__(CT) k_chol_prep(Chain* ch, const Consts* __restrict__ cs, int* swaps,
                                                  SelRule* rule, Status* st) {
    extern __shared__ double sm[];
    const int c = blockIdx.x;
    Chain& C = ch[c];
    if (!C.active) {
        if (threadIdx.x == 0) clear_rule(rule[c]);   // a stopped chain selects nothing
        return;
    }
    (void)chain_prep(C, rule[c], cs, swaps + c, st, sm);
}

void launch_chol_prep(const Plan& P, cudaStream_t s) {
    size_t sm = 3 * MAT * sizeof(double);
    auto k = k_chol_prep;
    big_smem(k, sm);
    k<<<2 * P.q, CT, sm, s>>>(P.ch, P.cs, P.swaps, P.rule, P.st);
}

// =====================================================================
// End of a C-step: fold the Gram partials into (S, G) (Section 3.5 update,
// or a fresh sum), new mu and Sigma = Lambda/(h_b-1) (eqs. cstep4a/b),
// convergence when H_new = H_old (no swaps).
// =====================================================================
// Last of the 2q finalize CTAs: count the blocks that still iterate; under a
// captured graph, also set the C-step loop's condition (chains still
// iterating and no error).
__device__ inline void count_active_blocks(const Chain* ch, int q, int* blk, Status* st,
                                           cudaGraphConditionalHandle hloop) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&st->done, 1) == 2 * q - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int a = 0;
    for (int l = threadIdx.x; l < q; l += blockDim.x) {
        volatile const int* b = blk;
        a += b[l] > 0 ? 1 : 0;
    }
    a = (int)cta_sum((double)a);
    if (threadIdx.x == 0) {
        st->active_blocks = a;
        if (hloop) {
            volatile Status* vs = st;
            cudaGraphSetConditional(hloop, (vs->active > 0 && vs->code == 0) ? 1u : 0u);
        }
    }
}

// End of a C-step and start of the next one: fold the Gram partials into
// (S, G) (Section 3.5 update, or a fresh sum), new mu and
// Sigma = Lambda/(h_b-1) (eqs. cstep4a/b), convergence when H_new = H_old
// (no swaps); a chain that goes on gets its next row parameters and window.
__global__ void __launch_bounds__(CT) k_cstep_finalize(Chain* ch, const Consts* __restrict__ cs,
                                                       const double* __restrict__ gsum, size_t slot_d,
                                                       int* swaps, int* blk, SelRule* rule, Status* st,
                                                       cudaGraphConditionalHandle hloop) {
    extern __shared__ double sm[];
    __shared__ double dmu[PMAX], inv_s[PMAX], Ss[PMAX];
    __shared__ double s_m2;
    __shared__ int s_cont;
    const int c = blockIdx.x, l = c / 2;
    Chain& C = ch[c];
    if (!C.active) {
        if (threadIdx.x == 0) clear_rule(rule[c]);
        count_active_blocks(ch, cs->q, blk, st, hloop);
        return;
    }
    const int p = cs->p, nb = gram_nb(cs->pb);
    const double hb = (double)cs->hb, inv_hb = 1.0 / hb, inv_hb1 = 1.0 / (hb - 1.0);
    const double* ext = gsum + (size_t)c * slot_d;
    const int full = C.full;
    if (threadIdx.x == 0) {
        const double cnt = gram_get(ext, p, p, nb);
        double expect = full ? hb : 0.0;
        if (fabs(cnt - expect) > 0.5) set_error(st, RTD_EINTERNAL);
    }
    // new S and G, kept in shared memory for the centre and scatter below
    double* Gs = sm + MAT;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double v = gram_get(ext, j, p, nb);
        v = full ? v : C.S[j] + v;
        C.S[j] = v;
        Ss[j] = v;
        inv_s[j] = 1.0 / cs->s_uni[j];
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = gram_get(ext, i, j, nb);
        v = full ? v : C.G[i * PMAX + j] + v;
        C.G[i * PMAX + j] = v;
        Gs[i * LD + j] = v;
    }
    // the previous M, for the centre's move below
    double* Mo = sm;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        Mo[i * LD + j] = C.rp.M[i * PMAX + j];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double mx = C.rp.ref[j] + Ss[j] * inv_hb;
        C.mu[j] = (mx - cs->mu_uni[j]) * inv_s[j];
        dmu[j] = mx - C.rp.ref[j];
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double lam = Gs[i * LD + j] - Ss[i] * Ss[j] * inv_hb;
        C.Sigma[i * PMAX + j] = lam * inv_hb1 * inv_s[i] * inv_s[j];
    }
    __syncthreads();
    // squared distance of the centre's move from the reference, under the previous fit
    double a2 = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a = fma(Mo[i * LD + j], dmu[j], a);
        a2 = fma(a, a, a2);
    }
    a2 = cta_sum(a2);
    if (threadIdx.x == 0) {
        s_m2 = a2;
        int sw = swaps[c];
        C.swaps = sw;
        atomicAdd(&st->gram_rows, (unsigned long long)(full ? cs->hb : sw));
        C.steps += 1;
        C.full_count += full;
        s_cont = 0;
        if (C.steps >= 2 && sw == 0) {
            C.active = 0;
            C.status = CH_OK;
        } else if (C.steps >= cs->max_steps) {
            C.active = 0;
            C.status = CH_MAXITER;
            set_warning(st, RTD_WARN_MAXITER);
        } else {
            C.full = ((C.steps >= 2 && 4.0 * sw > hb) || s_m2 > 1.0) ? 1 : 0;
            s_cont = 1;
        }
        if (!s_cont) clear_rule(rule[c]);
    }
    __syncthreads();
    if (s_cont && chain_prep(C, rule[c], cs, swaps + c, st, sm)) {
        if (threadIdx.x == 0) {
            atomicAdd(&st->active, 1);
            atomicAdd(&blk[l], 1);
        }
    }
    count_active_blocks(ch, cs->q, blk, st, hloop);
}

void launch_cstep_finalize(const Plan& P, cudaStream_t s, unsigned long long hloop) {
    launch_reduce_slots(P, 0, s);
    size_t sm = 3 * MAT * sizeof(double);
    auto k = k_cstep_finalize;
    big_smem(k, sm);
    k<<<2 * P.q, CT, sm, s>>>(P.ch, P.cs, P.gsum, P.slot_doubles, P.swaps, P.blk_active, P.rule, P.st,
                              (cudaGraphConditionalHandle)hloop);
}

// Condition of a captured graph's conditional node: no error so far.
__global__ void k_cond_ok(cudaGraphConditionalHandle h, const Status* st) {
    if (threadIdx.x == 0) {
        volatile const Status* vs = st;
        cudaGraphSetConditional(h, vs->code == 0 ? 1u : 0u);
    }
}
void launch_cond_ok(unsigned long long h, const Status* st, cudaStream_t s) {
    k_cond_ok<<<1, 32, 0, s>>>((cudaGraphConditionalHandle)h, st);
}

// =====================================================================
// Section 4 step 4: the start with the lower determinant (start 1 on ties).
// =====================================================================
__global__ void __launch_bounds__(1024) k_block_choose(Chain* ch, Consts* cs, const uint8_t* __restrict__ memb,
                                                     int* chosen, int* amb, int fp32, Status* st) {
    extern __shared__ double sm[];
    double* A = sm;
    __shared__ int okk[2];
    __shared__ double ldk[2];
    __shared__ int ndiff;
    const int l = blockIdx.x, p = cs->p, m = cs->m;
    // Two starts that reach the same h-subset have equal determinants; the
    // comparison is then decided exactly (start 1 wins ties, as "<=").
    if (threadIdx.x == 0) ndiff = 0;
    __syncthreads();
    {
        const uint8_t* a = memb + (size_t)(2 * l) * m;
        const uint8_t* b = memb + (size_t)(2 * l + 1) * m;
        int d = 0;
        if ((m & 3) == 0) {   // 4 rows per word (rows of chain c start at c m)
            const unsigned* a4 = reinterpret_cast<const unsigned*>(a);
            const unsigned* b4 = reinterpret_cast<const unsigned*>(b);
            for (int t = threadIdx.x; t < m / 4; t += blockDim.x) d += __popc((a4[t] ^ b4[t]) & 0x01010101u);
        } else {
            for (int t = threadIdx.x; t < m; t += blockDim.x) d += ((a[t] ^ b[t]) & 1);
        }
        d = (int)cta_sum((double)d);
        if (threadIdx.x == 0) ndiff = d;
        __syncthreads();
    }
    for (int k = 0; k < 2; ++k) {
        Chain& C = ch[2 * l + k];
        bool has = C.started && C.steps > 0 && C.status != CH_DROPPED;
        __syncthreads();
        if (threadIdx.x == 0) { okk[k] = 0; ldk[k] = NAN; }
        __syncthreads();
        if (!has) continue;
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            A[i * LD + j] = C.Sigma[i * PMAX + j];
        }
        __syncthreads();
        bool ok = cta_cholesky(A, p);
        double ld = 0.0;
        for (int j = threadIdx.x; j < p; j += blockDim.x) ld += log(A[j * LD + j]);
        ld = 2.0 * cta_sum(ld);
        if (threadIdx.x == 0) {
            okk[k] = ok ? 1 : 0;
            ldk[k] = ld;
            C.logdet = ok ? ld : NAN;
            atomicMax(&cs->csteps_max, C.steps);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int ch_ = -1;
        if (okk[0] && okk[1]) ch_ = (ndiff == 0 || ldk[0] <= ldk[1]) ? 0 : 1;
        else if (okk[0]) ch_ = 0;
        else if (okk[1]) ch_ = 1;
        // FP32 form: different subsets whose log-determinants lie within the
        // FP32 Gram error are compared again from FP64 Grams (k_rechoose)
        amb[l] = (fp32 && okk[0] && okk[1] && ndiff > 0 &&
                  fabs(ldk[0] - ldk[1]) <= 1e-5 * fmax(1.0, fabs(ldk[0]))) ? 1 : 0;
        chosen[l] = ch_;
        if (ch_ < 0) set_warning(st, RTD_WARN_NO_BLOCK_FIT);
        else atomicAdd(&cs->chains_ok, okk[0] + okk[1]);
    }
}

void launch_block_choose(const Plan& P, cudaStream_t s) {
    size_t sm = MAT * sizeof(double);
    auto k = k_block_choose;
    big_smem(k, sm);
    k<<<P.q, 1024, sm, s>>>(P.ch, P.cs, P.memb, P.chosen, P.amb, P.precision == RTD_FP32, P.st);
}

// Ambiguous blocks: with Lambda_1 = G_1 - S_1 S_1^T / h_b of start 1 and the
// FP64 Gram (dS, dG) of the rows in exactly one subset, Lambda_2 = Lambda_1 +
// dL, dL = dG - (S_1 dS^T + dS S_1^T + dS dS^T) / h_b, and
// log det Lambda_2 - log det Lambda_1 = log det(I + L^-1 dL L^-T).  The
// common rounding of Lambda_1 cancels in the difference, which decides the
// choice of Section 4 step 4 (start 1 when det Sigma_1 <= det Sigma_2).
__global__ void __launch_bounds__(CT) k_rechoose(Chain* ch, const Consts* __restrict__ cs,
                                                 const double* __restrict__ gsum, size_t slot_d,
                                                 const int* __restrict__ amb, int* chosen, Status* st) {
    extern __shared__ double sm[];
    double* A = sm;             // Lambda_1, then L
    double* Li = sm + MAT;      // L^-1
    double* Dl = sm + 2 * MAT;  // dL, then I + L^-1 dL L^-T
    __shared__ double dS[PMAX];
    const int l = blockIdx.x;
    if (!amb[l]) return;
    const int p = cs->p, nb = gram_nb(cs->pb);
    const double hb = (double)cs->hb;
    const Chain& C = ch[2 * l];
    const double* ext = gsum + (size_t)(2 * l) * slot_d;
    if (threadIdx.x == 0 && fabs(gram_get(ext, p, p, nb)) > 0.5) set_error(st, RTD_EINTERNAL);
    for (int j = threadIdx.x; j < p; j += blockDim.x) dS[j] = gram_get(ext, j, p, nb);
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        A[i * LD + j] = C.G[i * PMAX + j] - C.S[i] * C.S[j] / hb;
        Dl[i * LD + j] = gram_get(ext, i, j, nb) - (C.S[i] * dS[j] + dS[i] * C.S[j] + dS[i] * dS[j]) / hb;
    }
    __syncthreads();
    if (!cta_cholesky(A, p)) return;
    cta_tri_inverse(A, Li, p);
    // T = L^-1 dL (into A), then Dl = I + T L^-T
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = 0.0;
        for (int k = 0; k <= i; ++k) v += Li[i * LD + k] * Dl[k * LD + j];
        A[i * LD + j] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = 0.0;
        for (int k = 0; k <= j; ++k) v += A[i * LD + k] * Li[j * LD + k];
        Dl[i * LD + j] = v + (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    // symmetrise against rounding
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        if (j < i) { double v = 0.5 * (Dl[i * LD + j] + Dl[j * LD + i]); Dl[i * LD + j] = v; Dl[j * LD + i] = v; }
    }
    __syncthreads();
    if (!cta_cholesky(Dl, p)) return;
    double ld = 0.0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) ld += log(Dl[j * LD + j]);
    ld = 2.0 * cta_sum(ld);
    if (threadIdx.x == 0) chosen[l] = (ld >= 0.0) ? 0 : 1;
}

void launch_rechoose(const Plan& P, cudaStream_t s) {
    launch_member_gram(P, s);
    launch_reduce_slots(P, 0, s);
    size_t sm = 3 * MAT * sizeof(double);
    auto k = k_rechoose;
    big_smem(k, sm);
    k<<<P.q, CT, sm, s>>>(P.ch, P.cs, P.gsum, P.slot_doubles, P.amb, P.chosen, P.st);
}

// =====================================================================
// Section 4 steps 5-7: entrywise median of the block fits, KL deviation of
// each fit from the median (eq. KL, log|det|), keep the ceil(q/2) closest,
// Bennett pooling of their h-subsets.
//   agg_median: one thread per entry of (mu, Sigma), insertion sort of the
//               fitted blocks' values;
//   agg_kl:     one CTA per block;
//   agg_pool:   one CTA: stable order by (KL, block), keep, pool.
// Scratch layout: [0, p) mu_med, [p, p + p^2) Sigma_med, then per-thread
// sort rows.
// =====================================================================
__global__ void k_agg_median(const Chain* __restrict__ ch, const Consts* __restrict__ cs,
                             const int* __restrict__ chosen, double* scratch) {
    const int p = cs->p, q = cs->q;
    const double ca = cs->c_alpha;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p + p * p) return;
    double* v = scratch + p + p * p + (size_t)e * q;
    int n = 0;
    for (int l = 0; l < q; ++l) {
        if (chosen[l] < 0) continue;
        const Chain& C = ch[2 * l + chosen[l]];
        double x = (e < p) ? C.mu[e] : ca * C.Sigma[((e - p) / p) * PMAX + (e - p) % p];
        int u = n - 1;
        while (u >= 0 && v[u] > x) { v[u + 1] = v[u]; --u; }
        v[u + 1] = x;
        ++n;
    }
    if (n == 0) return;
    scratch[e] = (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

__global__ void __launch_bounds__(CT) k_agg_kl(const Chain* __restrict__ ch, const Consts* __restrict__ cs,
                                               const int* __restrict__ chosen, const double* __restrict__ scratch,
                                               double* kl) {
    extern __shared__ double sm[];
    double* Smed = sm;
    double* A = sm + MAT;
    double* Li = sm + 2 * MAT;
    __shared__ double dv[PMAX];
    const int l = blockIdx.x, p = cs->p;
    if (chosen[l] < 0) { if (threadIdx.x == 0) kl[l] = NAN; return; }
    const double ca = cs->c_alpha;
    const Chain& C = ch[2 * l + chosen[l]];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = scratch[p + e];
        Smed[i * LD + j] = v;
        A[i * LD + j] = v;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) dv[j] = scratch[j] - C.mu[j];
    __syncthreads();
    const double lad = cta_logabsdet(A, p);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        A[i * LD + j] = ca * C.Sigma[i * PMAX + j];
    }
    __syncthreads();
    if (!cta_cholesky(A, p)) { if (threadIdx.x == 0) kl[l] = INFINITY; return; }
    cta_tri_inverse(A, Li, p);
    double ldb = 0.0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) ldb += log(A[j * LD + j]);
    ldb = 2.0 * cta_sum(ldb);
    // B^-1 = Li^T Li ; tr(Smed B^-1) and d^T B^-1 d
    double tr = 0.0, quad = 0.0;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        int k0 = i > j ? i : j;
        double bij = 0.0;
        for (int kk = k0; kk < p; ++kk) bij += Li[kk * LD + i] * Li[kk * LD + j];
        tr += Smed[j * LD + i] * bij;
        quad += dv[i] * bij * dv[j];
    }
    tr = cta_sum(tr);
    quad = cta_sum(quad);
    if (threadIdx.x == 0) {
        double v = tr - p - (lad - ldb) + quad;
        kl[l] = isfinite(v) ? v : INFINITY;
    }
}

__global__ void __launch_bounds__(AGG_T) k_agg_pool(const Chain* __restrict__ ch, Consts* cs,
                                                    const int* __restrict__ chosen, int* kept, double* kl,
                                                    Status* st) {
    extern __shared__ double sm[];
    double* Lam = sm;
    __shared__ int fl[1024];
    __shared__ int s_qf;
    __shared__ double mup[PMAX], dv[PMAX];
    __shared__ double s_np;
    const int p = cs->p, q = cs->q;
    const double ca = cs->c_alpha, hb = (double)cs->hb;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int l = 0; l < q && n < 1024; ++l) {
            kept[l] = 0;
            if (chosen[l] >= 0) fl[n++] = l;
        }
        s_qf = n;
        // stable order by (KL, block)
        for (int i = 1; i < n; ++i) {
            int v = fl[i];
            int u = i - 1;
            while (u >= 0 && kl[fl[u]] > kl[v]) { fl[u + 1] = fl[u]; --u; }
            fl[u + 1] = v;
        }
        for (int i = 0; i < (n + 1) / 2; ++i) kept[fl[i]] = 1;
    }
    __syncthreads();
    const int qf = s_qf;
    if (qf == 0) {
        if (threadIdx.x == 0) set_error(st, RTD_EILLCOND);
        return;
    }
    // Bennett pooling over the kept blocks in KL order, counts h_b
    const int nk = (qf + 1) / 2;
    {
        const Chain& C0 = ch[2 * fl[0] + chosen[fl[0]]];
        for (int j = threadIdx.x; j < p; j += blockDim.x) mup[j] = C0.mu[j];
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            Lam[i * LD + j] = (hb - 1.0) * C0.Sigma[i * PMAX + j];
        }
        if (threadIdx.x == 0) s_np = hb;
        __syncthreads();
    }
    for (int t = 1; t < nk; ++t) {
        const Chain& C = ch[2 * fl[t] + chosen[fl[t]]];
        const double np_ = s_np;
        for (int j = threadIdx.x; j < p; j += blockDim.x) dv[j] = C.mu[j] - mup[j];
        __syncthreads();
        const double wgt = np_ * hb / (np_ + hb);
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            Lam[i * LD + j] += (hb - 1.0) * C.Sigma[i * PMAX + j] + dv[i] * dv[j] * wgt;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < p; j += blockDim.x) mup[j] = (np_ * mup[j] + hb * C.mu[j]) / (np_ + hb);
        __syncthreads();
        if (threadIdx.x == 0) s_np = np_ + hb;
        __syncthreads();
    }
    const double npool = s_np;
    for (int j = threadIdx.x; j < p; j += blockDim.x) cs->mu_raw[j] = mup[j];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        cs->Sigma_raw[i * PMAX + j] = ca * Lam[i * LD + j] / (npool - 1.0);
    }
}

// q = 1: the serial algorithm's raw fit is the chosen start's C_k.
__global__ void k_agg_single(const Chain* __restrict__ ch, Consts* cs, const int* __restrict__ chosen,
                             int* kept, double* kl, Status* st) {
    const int p = cs->p;
    if (chosen[0] < 0) {
        if (threadIdx.x == 0) set_error(st, RTD_EILLCOND);
        return;
    }
    const Chain& C = ch[chosen[0]];
    for (int j = threadIdx.x; j < p; j += blockDim.x) cs->mu_raw[j] = C.mu[j];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        cs->Sigma_raw[i * PMAX + j] = cs->c_alpha * C.Sigma[i * PMAX + j];
    }
    if (threadIdx.x == 0) { kept[0] = 1; kl[0] = 0.0; }
}

void launch_aggregate(const Plan& P, cudaStream_t s) {
    if (P.q == 1) {
        k_agg_single<<<1, 256, 0, s>>>(P.ch, P.cs, P.chosen, P.kept, P.kl, P.st);
        return;
    }
    const int ne = P.p + P.p * P.p;
    k_agg_median<<<(ne + 127) / 128, 128, 0, s>>>(P.ch, P.cs, P.chosen, P.scratch);
    size_t sm = 3 * MAT * sizeof(double);
    auto k1 = k_agg_kl;
    big_smem(k1, sm);
    k1<<<P.q, CT, sm, s>>>(P.ch, P.cs, P.chosen, P.scratch, P.kl);
    size_t sm2 = MAT * sizeof(double);
    auto k2 = k_agg_pool;
    big_smem(k2, sm2);
    k2<<<1, AGG_T, sm2, s>>>(P.ch, P.cs, P.chosen, P.kept, P.kl, P.st);
}

// Row parameters of the raw (which = 0) or reweighted (which = 1) fit.
__global__ void __launch_bounds__(CT) k_fit_prep(Consts* cs, RowParams* fitrp, int which, Status* st) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Li = sm + MAT;
    __shared__ double s_ld;
    const int p = cs->p;
    const double* mu = which ? cs->mu_rew : cs->mu_raw;
    const double* S = which ? cs->Sigma_rew : cs->Sigma_raw;
    RowParams& rp = fitrp[which];
    bool ok = make_rowparams(mu, S, cs->mu_uni, cs->s_uni, p, A, Li, rp, &s_ld);
    if (!ok) {
        if (threadIdx.x == 0) set_error(st, RTD_EDEGENERATE);
        return;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        rp.ref[j] = rp.mu[j];
        rp.ref_hi[j] = rp.mu_hi[j];
        rp.ref_lo[j] = rp.mu_lo[j];
    }
    if (threadIdx.x == 0) {
        if (which) cs->logdet_rew = s_ld;
        else cs->logdet_raw = s_ld;
    }
}

void launch_fit_prep(const Plan& P, int which, cudaStream_t s) {
    size_t sm = 2 * MAT * sizeof(double);
    auto k = k_fit_prep;
    big_smem(k, sm);
    k<<<1, CT, sm, s>>>(P.cs, P.fitrp, which, P.st);
}

// Section 4 steps 8-9: mean and covariance of the reweighting set (the
// pooled per-block moments), times the reweighting consistency factor.
__global__ void __launch_bounds__(256) k_rew_finalize(Consts* cs, const RowParams* __restrict__ fitrp,
                                                      const double* __restrict__ ext, Status* st) {
    const int p = cs->p, nb = gram_nb(cs->pb);
    const double nw = gram_get(ext, p, p, nb);
    if (!(nw > (double)p + 1.0)) {
        if (threadIdx.x == 0) set_error(st, RTD_EDEGENERATE);
        return;
    }
    double f = 1.0;
    if (cs->rew_mode == 1) f = cs->c_rew;
    else if (cs->rew_mode == 2) f = consistency(nw / (double)cs->n, p);
    const RowParams& rp = fitrp[0];
    const double* su = cs->s_uni;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        double mx = rp.ref[j] + gram_get(ext, j, p, nb) / nw;
        cs->mu_rew[j] = (mx - cs->mu_uni[j]) / su[j];
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double si = gram_get(ext, i, p, nb), sj = gram_get(ext, j, p, nb);
        double lam = gram_get(ext, i, j, nb) - si * sj / nw;
        cs->Sigma_rew[i * PMAX + j] = f * lam / (nw - 1.0) / (su[i] * su[j]);
    }
    if (threadIdx.x == 0) { cs->n_rew = (long long)(nw + 0.5); cs->f_rew = f; }
}

void launch_rew_finalize(const Plan& P, cudaStream_t s) {
    launch_reduce_slots(P, 1, s);
    k_rew_finalize<<<1, 256, 0, s>>>(P.cs, P.fitrp, P.gsum, P.st);
}

// =====================================================================
// Result assembly (X units: mu_x = mu_uni + D mu, Sigma_x = D Sigma D) and
// the optional diagnostics record.
// =====================================================================
__global__ void k_result(const Consts* __restrict__ cs, const Status* __restrict__ st,
                         const Chain* __restrict__ ch, const int* __restrict__ chosen,
                         const int* __restrict__ kept, const double* __restrict__ kl,
                         rtd_result* out, double* diag) {
    const int p = cs->p;
    const double* su = cs->s_uni;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        out->mu[j] = cs->mu_uni[j] + su[j] * cs->mu_rew[j];
        out->mu_raw[j] = cs->mu_uni[j] + su[j] * cs->mu_raw[j];
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        out->sigma[e] = cs->Sigma_rew[i * PMAX + j] * su[i] * su[j];
        out->sigma_raw[e] = cs->Sigma_raw[i * PMAX + j] * su[i] * su[j];
    }
    if (threadIdx.x == 0) {
        double lds = 0.0;
        for (int j = 0; j < p; ++j) lds += 2.0 * log(su[j]);
        out->status = st->code;
        out->warnings = st->warnings;
        out->p = p; out->q = cs->q;
        out->n = cs->n; out->m = cs->m; out->h = cs->h; out->h_b = cs->hb;
        out->logdet = cs->logdet_rew + lds;
        out->logdet_raw = cs->logdet_raw + lds;
        out->cutoff_d2 = cs->cutoff_d2;
        out->n_flagged = (int64_t)st->n_flagged;
        out->n_reweight = cs->n_rew;
        out->csteps_max = cs->csteps_max;
        out->chains_ok = cs->chains_ok;
        out->c_rew = cs->f_rew;
    }
    if (!diag) return;
    for (int j = threadIdx.x; j < p; j += blockDim.x) { diag[j] = cs->mu_uni[j]; diag[p + j] = su[j]; }
    const size_t rec = 3 * (size_t)p * p + 2 * p + 6;
    const int q = cs->q;
    for (int c = 0; c < 2 * q; ++c) {
        const Chain& C = ch[c];
        double* r = diag + 2 * p + (size_t)c * rec;
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            r[e] = C.Sinit[i * PMAX + j];
            r[p * p + e] = C.Sigma0[i * PMAX + j];
            r[2 * p * p + p + e] = C.Sigma[i * PMAX + j];
        }
        for (int j = threadIdx.x; j < p; j += blockDim.x) {
            r[2 * p * p + j] = C.mu0[j];
            r[3 * p * p + p + j] = C.mu[j];
        }
        if (threadIdx.x == 0) {
            double* t = r + 3 * p * p + 2 * p;
            t[0] = C.logdet;
            t[1] = C.steps;
            int stt = C.status;
            if (stt == CH_REFUSED && C.steps > 0) stt = CH_OK;
            t[2] = stt;
            t[3] = C.full_count;
            t[4] = C.swaps;
            t[5] = C.kappa1;
        }
    }
    double* b = diag + 2 * p + (size_t)2 * q * rec;
    for (int l = threadIdx.x; l < q; l += blockDim.x) {
        b[3 * l] = chosen[l];
        b[3 * l + 1] = kl[l];
        b[3 * l + 2] = kept[l];
    }
}

void launch_result(const Plan& P, rtd_result* dev_out, double* diag, cudaStream_t s) {
    k_result<<<1, 256, 0, s>>>(P.cs, P.st, P.ch, P.chosen, P.kept, P.kl, dev_out, diag);
}

// Scoring: row parameters of a caller fit (X units, D = I).
__global__ void __launch_bounds__(CT) k_score_prep(const double* __restrict__ mu, const double* __restrict__ S,
                                                   int p, RowParams* rp, Status* st, double* logdet_out) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Li = sm + MAT;
    __shared__ double one[PMAX], zero[PMAX], Sp[PMAX * PMAX];
    __shared__ double s_ld;
    for (int j = threadIdx.x; j < p; j += blockDim.x) { one[j] = 1.0; zero[j] = 0.0; }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        Sp[i * PMAX + j] = S[e];
    }
    __syncthreads();
    // mu_x = 0 + 1 * mu
    bool ok = make_rowparams(mu, Sp, zero, one, p, A, Li, *rp, &s_ld);
    if (!ok && threadIdx.x == 0) set_error(st, RTD_EDEGENERATE);
    if (ok && logdet_out && threadIdx.x == 0) *logdet_out = s_ld;
}

// The same from a fit passed by value; also zeroes the status word first.
__global__ void __launch_bounds__(CT) k_score_prep_arg(const __grid_constant__ FitArg a, int p, double cut,
                                                       RowParams* rp, Status* st, double* cut_out) {
    extern __shared__ double sm[];
    double* A = sm;
    double* Li = sm + MAT;
    __shared__ double one[PMAX], zero[PMAX], mu[PMAX], Sp[PMAX * PMAX];
    __shared__ double s_ld;
    if (threadIdx.x == 0) {
        st->code = 0;
        st->n_flagged = 0ull;
        *cut_out = cut;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) { one[j] = 1.0; zero[j] = 0.0; mu[j] = a.mu[j]; }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        const int hi = i > j ? i : j, lo = i > j ? j : i;
        Sp[i * PMAX + j] = a.tri[hi * (hi + 1) / 2 + lo];
    }
    __syncthreads();
    const bool ok = make_rowparams(mu, Sp, zero, one, p, A, Li, *rp, &s_ld);
    if (!ok && threadIdx.x == 0) set_error(st, RTD_EDEGENERATE);
}

void launch_score_prep_arg(const FitArg& a, int p, double cut, RowParams* rp, Status* st, double* cut_out,
                           cudaStream_t s) {
    size_t sm = 2 * MAT * sizeof(double);
    auto k = k_score_prep_arg;
    big_smem(k, sm);
    k<<<1, CT, sm, s>>>(a, p, cut, rp, st, cut_out);
}

void launch_score_prep(const double* mu, const double* Sigma, int p, RowParams* rp, Status* st, cudaStream_t s,
                       double* logdet_out) {
    size_t sm = 2 * MAT * sizeof(double);
    auto k = k_score_prep;
    big_smem(k, sm);
    k<<<1, CT, sm, s>>>(mu, Sigma, p, rp, st, logdet_out);
}

// =====================================================================
// The fit in stages (a fit sharded over processes).  A block-fit record is
// [chosen start (-1 none, 0, 1), log det Sigma_l, mu_l[p], Sigma_l[p^2]] in
// Z units, Sigma_l = Lambda/(h_b - 1) without c(alpha): what steps 5-7 read
// of each block (Section 4 steps 4-7).
// =====================================================================
__global__ void k_block_fits_out(const Chain* __restrict__ ch, const Consts* __restrict__ cs,
                                 const int* __restrict__ chosen, double* out) {
    const int l = blockIdx.x, p = cs->p;
    const size_t rd = 2 + (size_t)p + (size_t)p * p;
    double* r = out + (size_t)l * rd;
    const int c = chosen[l];
    if (c < 0) {
        for (size_t e = threadIdx.x; e < rd; e += blockDim.x) r[e] = (e == 0) ? -1.0 : 0.0;
        return;
    }
    const Chain& C = ch[2 * l + c];
    if (threadIdx.x == 0) { r[0] = (double)c; r[1] = C.logdet; }
    for (int j = threadIdx.x; j < p; j += blockDim.x) r[2 + j] = C.mu[j];
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) r[2 + p + e] = C.Sigma[(e / p) * PMAX + e % p];
}

void launch_block_fits_out(const Plan& P, double* out, cudaStream_t s) {
    k_block_fits_out<<<P.q, 128, 0, s>>>(P.ch, P.cs, P.chosen, out);
}

// Records of all q blocks into the chains that steps 5-7 read; a record
// whose start is not -1, 0 or 1, or whose values are not finite, is refused.
__global__ void k_block_fits_in(Chain* ch, const Consts* __restrict__ cs, int* chosen, const double* __restrict__ in,
                                Status* st) {
    const int l = blockIdx.x, p = cs->p;
    const size_t rd = 2 + (size_t)p + (size_t)p * p;
    const double* r = in + (size_t)l * rd;
    const double cd = r[0];
    const int c = (cd == 0.0) ? 0 : (cd == 1.0) ? 1 : (cd == -1.0) ? -1 : -2;
    if (c == -2) {
        if (threadIdx.x == 0) { chosen[l] = -1; set_error(st, RTD_EINVAL); }
        return;
    }
    if (threadIdx.x == 0) {
        chosen[l] = c;
        if (c < 0) set_warning(st, RTD_WARN_NO_BLOCK_FIT);
    }
    if (c < 0) return;
    Chain& C = ch[2 * l + c];
    bool bad = false;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        C.mu[j] = r[2 + j];
        bad |= !isfinite(r[2 + j]);
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        C.Sigma[(e / p) * PMAX + e % p] = r[2 + p + e];
        bad |= !isfinite(r[2 + p + e]);
    }
    if (bad) set_error(st, RTD_EINVAL);
    if (threadIdx.x == 0) { C.logdet = r[1]; C.status = CH_OK; C.started = 1; }
}

void launch_block_fits_in(const Plan& P, const double* in, cudaStream_t s) {
    k_block_fits_in<<<P.q, 128, 0, s>>>(P.ch, P.cs, P.chosen, in, P.st);
}

// Reweighting moments [count, sum of (x - c), sum of (x - c)(x - c)^T] with
// c the raw centre in X units, from / to the extended Gram of the
// reweighting pass (entry (i, p) is the sum of coordinate i, (p, p) the
// count).
__global__ void k_moments_out(const Consts* __restrict__ cs, const double* __restrict__ gsum, double* out) {
    const int p = cs->p, nb = gram_nb(cs->pb);
    for (int e = threadIdx.x; e < 1 + p + p * p; e += blockDim.x) {
        double v;
        if (e == 0) v = gram_get(gsum, p, p, nb);
        else if (e <= p) v = gram_get(gsum, e - 1, p, nb);
        else v = gram_get(gsum, (e - 1 - p) / p, (e - 1 - p) % p, nb);
        out[e] = v;
    }
}

void launch_moments_out(const Plan& P, double* out, cudaStream_t s) {
    launch_reduce_slots(P, 1, s);
    k_moments_out<<<1, 256, 0, s>>>(P.cs, P.gsum, out);
}

__global__ void k_moments_in(const Consts* __restrict__ cs, const double* __restrict__ in, double* gsum,
                             size_t slot_d) {
    const int p = cs->p, nb = gram_nb(cs->pb);
    for (size_t e = threadIdx.x; e < slot_d; e += blockDim.x) gsum[e] = 0.0;
    __syncthreads();
    const int pe = p + 1;
    for (int e = threadIdx.x; e < pe * pe; e += blockDim.x) {
        const int i = e / pe, j = e % pe;
        if (i > j) continue;
        double v;
        if (j == p) v = (i == p) ? in[0] : in[1 + i];
        else v = in[1 + p + i * p + j];
        gsum[gram_blk_index(i >> 2, j >> 2, nb) * 16 + (i & 3) * 4 + (j & 3)] = v;
    }
}

void launch_moments_finalize(const Plan& P, const double* in, cudaStream_t s) {
    k_moments_in<<<1, 256, 0, s>>>(P.cs, in, P.gsum, P.slot_doubles);
    k_rew_finalize<<<1, 256, 0, s>>>(P.cs, P.fitrp, P.gsum, P.st);
}

}  // namespace rtd
