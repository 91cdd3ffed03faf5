// rtd_sort.cu - segmented radix sort, univariate MCD, GSSCM cutoffs and the
// block-wide radix select of the C-step.
#include "rtd_internal.cuh"

namespace rtd {

// =====================================================================
// Segmented LSD radix sort of equal-length segments (keys only, 8-bit
// digits, stable).  Per pass: tile histograms, per-segment exclusive scan
// in (digit, tile) order, stable scatter.  A tile is 4096 keys: 8 warps of
// 512 keys, ranked with warp match in 16 rounds of 32.
// =====================================================================
constexpr int ST = 256;                 // threads
constexpr int SW = ST / 32;             // warps
constexpr int SITEMS = 16;              // rounds per warp
constexpr int STILE = ST * SITEMS;      // keys per tile
constexpr int SKPW = STILE / SW;        // keys per warp

template <typename K>
__global__ void __launch_bounds__(ST) k_sort_hist(const K* __restrict__ keys, long long L, int tiles,
                                                  int shift, unsigned* __restrict__ hist) {
    __shared__ unsigned h[256];
    const int seg = blockIdx.y, tile = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    long long t0 = (long long)tile * STILE;
    int cnt = (int)((L - t0) < STILE ? (L - t0) : STILE);
    const K* in = keys + (long long)seg * L + t0;
    for (int i = threadIdx.x; i < cnt; i += ST) atomicAdd(&h[(unsigned)(in[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[((size_t)seg * 256 + threadIdx.x) * tiles + tile] = h[threadIdx.x];
}

// Exclusive scan of one segment's 256 * tiles counters (one CTA per segment).
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned* __restrict__ hist, int tiles) {
    __shared__ unsigned part[1024];
    const long long N = 256LL * tiles;
    unsigned* a = hist + (size_t)blockIdx.x * N;
    long long per = (N + blockDim.x - 1) / blockDim.x;
    long long b = threadIdx.x * per, e = b + per < N ? b + per : N;
    unsigned s = 0;
    for (long long i = b; i < e; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partials
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (long long i = b; i < e; ++i) {
        unsigned v = a[i];
        a[i] = run;
        run += v;
    }
}

template <typename K>
__global__ void __launch_bounds__(ST) k_sort_scatter(const K* __restrict__ in, K* __restrict__ out, long long L,
                                                     int tiles, int shift, const unsigned* __restrict__ offs) {
    __shared__ unsigned wcnt[SW][256];
    __shared__ unsigned goff[256];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < SW * 256; e += ST) (&wcnt[0][0])[e] = 0u;
    goff[threadIdx.x] = offs[((size_t)seg * 256 + threadIdx.x) * tiles + tile];
    __syncthreads();
    long long t0 = (long long)tile * STILE;
    int cnt = (int)((L - t0) < STILE ? (L - t0) : STILE);
    const K* src = in + (long long)seg * L + t0;
    K key[SITEMS];
    unsigned rank[SITEMS];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SITEMS; ++r) {
        int idx = w * SKPW + r * 32 + lane;
        bool valid = idx < cnt;
        key[r] = valid ? src[idx] : (K)0;
        unsigned d = (unsigned)(key[r] >> shift) & 255u;
        unsigned tag = valid ? d : 256u + lane;
        unsigned peers = __match_any_sync(0xffffffffu, tag);
        unsigned base = valid ? wcnt[w][d] : 0u;
        rank[r] = base + __popc(peers & lt);
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) wcnt[w][d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        unsigned run = 0;
        for (int ww = 0; ww < SW; ++ww) {
            unsigned c = wcnt[ww][threadIdx.x];
            wcnt[ww][threadIdx.x] = run;
            run += c;
        }
    }
    __syncthreads();
    K* dst = out + (long long)seg * L;
#pragma unroll
    for (int r = 0; r < SITEMS; ++r) {
        int idx = w * SKPW + r * 32 + lane;
        if (idx < cnt) {
            unsigned d = (unsigned)(key[r] >> shift) & 255u;
            unsigned pos = goff[d] + wcnt[w][d] + rank[r];
            if (pos < (unsigned)L) dst[pos] = key[r];
        }
    }
}

template <typename K>
static void sort_t(const Plan& P, K* keys, K* tmp, int nseg, long long L, cudaStream_t s) {
    int tiles = (int)((L + STILE - 1) / STILE);
    dim3 grid(tiles, nseg);
    const int passes = (int)sizeof(K);
    K* a = keys;
    K* b = tmp;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = 8 * ps;
        k_sort_hist<K><<<grid, ST, 0, s>>>(a, L, tiles, shift, P.sort_hist);
        k_sort_scan<<<nseg, 1024, 0, s>>>(P.sort_hist, tiles);
        k_sort_scatter<K><<<grid, ST, 0, s>>>(a, b, L, tiles, shift, P.sort_hist);
        K* t = a; a = b; b = t;
    }
    // an even number of passes leaves the result in `keys`
}

void sort_segments(const Plan& P, void* keys, void* tmp, int key_bytes, int nseg, long long L,
                   cudaStream_t s) {
    if (key_bytes == 8) sort_t<unsigned long long>(P, (unsigned long long*)keys, (unsigned long long*)tmp, nseg, L, s);
    else sort_t<uint32_t>(P, (uint32_t*)keys, (uint32_t*)tmp, nseg, L, s);
}

// =====================================================================
// Univariate reweighted MCD of a sorted segment (Section 3.1): coverage
// h~ = [L/2] + 1; the contiguous h~-window of minimum variance (first on
// ties) gives mu0 and c(h~/L) var; the reweighting keeps
// (x - mu0)^2 / s0^2 <= chi2_{1,q}, a contiguous range of the sorted values
// found by binary search.  Window sums come from FP64 running sums of the
// values shifted by the middle order statistic.
// out[seg] = (mu, s2, mu_raw, s2_raw); s2 <= 0 or NaN marks a degenerate
// segment.
// =====================================================================
constexpr int UT = 1024;

template <typename K>
__device__ inline double uval(const K* s, long long i) { return KeyOps<K>::dec(s[i]); }

template <typename K>
__global__ void __launch_bounds__(UT) k_unimcd(const K* __restrict__ sorted, long long L,
                                               const Consts* __restrict__ cs, int which_c1,
                                               double* __restrict__ out) {
    __shared__ double pre1[UT], pre2[UT];
    __shared__ double bv[UT / 32];
    __shared__ long long bj[UT / 32];
    __shared__ double s_res[2];
    __shared__ long long s_j;
    const K* s = sorted + (long long)blockIdx.x * L;
    const long long h = L / 2 + 1;
    const long long nwin = L - h + 1;
    const double c = uval(s, L / 2);
    const long long E = (L + UT - 1) / UT;
    const long long a0 = threadIdx.x * E;
    const long long a1 = (a0 + E < L) ? a0 + E : L;
    double s1 = 0.0, s2 = 0.0;
    for (long long i = a0; i < a1; ++i) {
        double d = uval(s, i) - c;
        s1 += d;
        s2 += d * d;
    }
    pre1[threadIdx.x] = s1;
    pre2[threadIdx.x] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {   // exclusive prefix of the chunk sums, fixed order
        double r1 = 0.0, r2 = 0.0;
        for (int t = 0; t < UT; ++t) {
            double v1 = pre1[t], v2 = pre2[t];
            pre1[t] = r1; pre2[t] = r2;
            r1 += v1; r2 += v2;
        }
    }
    __syncthreads();
    // running sums P(a) = sum_{i<a} (s_i - c), for any 0 <= a <= L
    auto prefix = [&](long long a, double& p1, double& p2) {
        long long t = a / E;
        if (t >= UT) t = UT - 1;
        p1 = pre1[t]; p2 = pre2[t];
        for (long long i = t * E; i < a; ++i) {
            double d = uval(s, i) - c;
            p1 += d;
            p2 += d * d;
        }
    };
    double best = INFINITY;
    long long bjj = -1;
    if (a0 < nwin) {
        long long w1 = (a1 < nwin) ? a1 : nwin;
        double P1a, P2a, P1b, P2b;
        prefix(a0, P1a, P2a);
        prefix(a0 + h, P1b, P2b);
        for (long long j = a0; j < w1; ++j) {
            double S1 = P1b - P1a, S2 = P2b - P2a;
            double var = (S2 - S1 * S1 / (double)h) / (double)(h - 1);
            if (var < best) { best = var; bjj = j; }
            double d0 = uval(s, j) - c;
            P1a += d0; P2a += d0 * d0;
            if (j + h < L) {
                double d1 = uval(s, j + h) - c;
                P1b += d1; P2b += d1 * d1;
            }
        }
    }
    // block argmin, ties to the lower window start
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, o);
        long long oj = __shfl_xor_sync(0xffffffffu, bjj, o);
        if (oj >= 0 && (bjj < 0 || ov < best || (ov == best && oj < bjj))) { best = ov; bjj = oj; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bj[threadIdx.x >> 5] = bjj; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = INFINITY;
        long long j = -1;
        for (int w = 0; w < UT / 32; ++w) {
            if (bj[w] >= 0 && (j < 0 || bv[w] < b || (bv[w] == b && bj[w] < j))) { b = bv[w]; j = bj[w]; }
        }
        s_j = j;
        s_res[0] = b;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double* o = out + 4 * (size_t)blockIdx.x;
    long long j = s_j;
    if (j < 0) { o[0] = o[1] = o[2] = o[3] = NAN; return; }
    double P1a, P2a, P1b, P2b;
    prefix(j, P1a, P2a);
    prefix(j + h, P1b, P2b);
    double S1 = P1b - P1a;
    const double c1 = which_c1 ? cs->c1_m : cs->c1_n;
    const double mu0 = c + S1 / (double)h;
    const double s20 = c1 * s_res[0];
    o[2] = mu0;
    o[3] = s20;
    if (!(s20 > 0.0) || !isfinite(s20)) { o[0] = NAN; o[1] = NAN; return; }
    const double cut2 = cs->uni_cut2;
    auto keep = [&](long long i) { double d = uval(s, i) - mu0; return d * d / s20 <= cut2; };
    // m0: first index with value >= mu0
    long long lo = 0, hi = L;
    while (lo < hi) { long long md = (lo + hi) / 2; if (uval(s, md) < mu0) lo = md + 1; else hi = md; }
    long long m0 = lo;
    // first kept index in [0, m0] (keep is false then true there)
    lo = 0; hi = m0;
    while (lo < hi) { long long md = (lo + hi) / 2; if (keep(md)) hi = md; else lo = md + 1; }
    long long wlo = lo;
    // first not-kept index in [m0, L] (keep is true then false there)
    lo = m0; hi = L;
    while (lo < hi) { long long md = (lo + hi) / 2; if (keep(md)) lo = md + 1; else hi = md; }
    long long whi = lo;
    long long nw = whi - wlo;
    if (nw < 2) { o[0] = NAN; o[1] = NAN; return; }
    prefix(wlo, P1a, P2a);
    prefix(whi, P1b, P2b);
    double T1 = P1b - P1a, T2 = P2b - P2a;
    double mu = c + T1 / (double)nw;
    double var = (T2 - T1 * T1 / (double)nw) / (double)(nw - 1);
    o[0] = mu;
    o[1] = cs->crew1 * var;
}

void launch_unimcd(const Plan& P, const void* keys, int key_bytes, int nseg, long long L, int which_c1,
                   double* out, cudaStream_t s) {
    if (key_bytes == 8)
        k_unimcd<unsigned long long><<<nseg, UT, 0, s>>>((const unsigned long long*)keys, L, P.cs, which_c1, out);
    else
        k_unimcd<uint32_t><<<nseg, UT, 0, s>>>((const uint32_t*)keys, L, P.cs, which_c1, out);
}

// =====================================================================
// GSSCM cutoffs (Section 3.2): A = median ||z||, B from the median m3 and
// the MAD of ||z||^(2/3); medians of even counts average the two middle
// values.  The MAD's order statistics come from the two sorted runs
// m3 - v (left of m3) and v - m3 (right of m3) by a k-th-of-two-arrays
// binary search.
// =====================================================================
template <typename K>
__device__ inline double r23(const K* s, long long i) { return pow(KeyOps<K>::dec(s[i]), 2.0 / 3.0); }

template <typename K>
__device__ double kth_absdev(const K* s, long long L, long long s0, double m3, long long k) {
    // left run: Lt = m3 - v[s0 - 1 - t], t < a; right run: Rt = v[s0 + t] - m3, t < b
    long long a = s0, b = L - s0;
    auto Lv = [&](long long t) { return m3 - r23(s, s0 - 1 - t); };
    auto Rv = [&](long long t) { return r23(s, s0 + t) - m3; };
    long long lo = k - b > 0 ? k - b : 0, hi = k < a ? k : a;
    while (lo < hi) {
        long long i = (lo + hi) / 2, j = k - i;
        if (i < a && j > 0 && Rv(j - 1) > Lv(i)) lo = i + 1;
        else hi = i;
    }
    long long i = lo, j = k - i;
    double x = (i > 0) ? Lv(i - 1) : -INFINITY;
    double y = (j > 0) ? Rv(j - 1) : -INFINITY;
    return x > y ? x : y;
}

template <typename K>
__global__ void k_gsscm(const K* __restrict__ rs, int q, long long m, double* __restrict__ AB) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= q) return;
    const K* s = rs + (size_t)l * m;
    double A, m3;
    if (m & 1) {
        A = KeyOps<K>::dec(s[m / 2]);
        m3 = r23(s, m / 2);
    } else {
        A = 0.5 * (KeyOps<K>::dec(s[m / 2 - 1]) + KeyOps<K>::dec(s[m / 2]));
        m3 = 0.5 * (r23(s, m / 2 - 1) + r23(s, m / 2));
    }
    long long lo = 0, hi = m;   // s0 = first index with v >= m3
    while (lo < hi) { long long md = (lo + hi) / 2; if (r23(s, md) < m3) lo = md + 1; else hi = md; }
    long long s0 = lo;
    double mad;
    if (m & 1) mad = kth_absdev(s, m, s0, m3, (m + 1) / 2);
    else mad = 0.5 * (kth_absdev(s, m, s0, m3, m / 2) + kth_absdev(s, m, s0, m3, m / 2 + 1));
    const double phi075 = 0.6744897501960817, madc = 1.4826;
    AB[2 * l] = A;
    AB[2 * l + 1] = pow(m3 + phi075 * madc * mad, 1.5);
}

void launch_gsscm(const Plan& P, const void* rkeys, cudaStream_t s) {
    int th = 64, bl = (P.q + th - 1) / th;
    if (P.key_bytes == 8) k_gsscm<unsigned long long><<<bl, th, 0, s>>>((const unsigned long long*)rkeys, P.q, P.m, P.gss);
    else k_gsscm<uint32_t><<<bl, th, 0, s>>>((const uint32_t*)rkeys, P.q, P.m, P.gss);
}

// =====================================================================
// Radix select, step 1 (per chain): the 12-bit bucket holding rank h_b
// from the histogram fused into the distance pass; the compaction range
// is that bucket, widened by the FP64 band in the FP32 form.
// =====================================================================
__global__ void __launch_bounds__(1024) k_select_bucket(unsigned* __restrict__ hist, const Chain* __restrict__ ch,
                                                        SelRule* __restrict__ rule, int hb, int fp32,
                                                        Status* st) {
    __shared__ unsigned cnt[1024];
    __shared__ int s_bin;
    const int c = blockIdx.x;
    if (!ch[c].active) return;
    unsigned* h = hist + (size_t)c * HIST_BINS;
    const int per = HIST_BINS / 1024;
    unsigned loc[HIST_BINS / 1024];
    unsigned sum = 0;
    for (int i = 0; i < per; ++i) { loc[i] = h[threadIdx.x * per + i]; sum += loc[i]; }
    cnt[threadIdx.x] = sum;
    if (threadIdx.x == 0) s_bin = -1;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned v = threadIdx.x >= o ? cnt[threadIdx.x - o] : 0u;
        __syncthreads();
        cnt[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = threadIdx.x ? cnt[threadIdx.x - 1] : 0u;
    for (int i = 0; i < per; ++i) {
        if (run < (unsigned)hb && (unsigned)hb <= run + loc[i]) s_bin = threadIdx.x * per + i;
        run += loc[i];
    }
    __syncthreads();
    for (int i = 0; i < per; ++i) h[threadIdx.x * per + i] = 0u;   // ready for the next step
    if (threadIdx.x != 0) return;
    int b = s_bin;
    SelRule& R = rule[c];
    R.below = 0;
    R.cand = 0;
    R.band = 0;
    if (b < 0) { set_error(st, RTD_EINTERNAL); R.lo = 1; R.hi = 0; return; }
    unsigned lo_bits = (unsigned)b << (32 - HIST_BITS);
    unsigned hi_bits = lo_bits | ((1u << (32 - HIST_BITS)) - 1u);
    if (fp32) {
        float flo = __uint_as_float(lo_bits) * (float)(1.0 - BAND_EPS);
        float fhi = __uint_as_float(hi_bits) * (float)(1.0 + BAND_EPS);
        R.lo = __float_as_uint(flo);
        R.hi = __float_as_uint(fhi);
    } else {
        R.lo = lo_bits;
        R.hi = hi_bits;
    }
}

void launch_select_bucket(const Plan& P, cudaStream_t s) {
    k_select_bucket<<<2 * P.q, 1024, 0, s>>>(P.hist, P.ch, P.rule, P.hb, P.precision == RTD_FP32, P.st);
}

// =====================================================================
// Radix select, step 2 (one CTA per chain): the r-th smallest (key, pos)
// of a candidate list, by 8-bit radix narrowing on the composite
// (key, position) until at most SEL_SMALL entries share the prefix, then
// direct ranking in shared memory.  Positions make every entry unique, so
// ties between equal distances go to the lower position.
// =====================================================================
constexpr int SEL_T = 1024;
constexpr int SEL_SMALL = 1024;
typedef unsigned __int128 u128;

__device__ inline u128 comp(const Cand& e) { return ((u128)e.key << 32) | (u128)e.pos; }

__device__ Cand cta_select_rank(const Cand* list, int C, int r, int key_bits, Cand* buf, Status* st) {
    __shared__ unsigned hcnt[256];
    __shared__ int s_digit, s_r, s_cnt, s_n;
    __shared__ Cand s_out;
    const int total = key_bits + 32;
    u128 prefix = 0;
    int pbits = 0, cnt = C, rr = r;
    if (threadIdx.x == 0) { s_out.key = ~0ull; s_out.pos = 0xffffffffu; s_out.pad = 1; }
    while (cnt > SEL_SMALL && pbits < total) {
        const int shift = total - pbits - 8;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hcnt[i] = 0u;
        __syncthreads();
        for (int i = threadIdx.x; i < C; i += blockDim.x) {
            u128 v = comp(list[i]);
            if (pbits == 0 || (v >> (total - pbits)) == prefix)
                atomicAdd(&hcnt[(unsigned)(v >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int cum = 0;
            s_digit = -1;
            for (int d = 0; d < 256; ++d) {
                int hd = (int)hcnt[d];
                if (cum + hd >= rr) { s_digit = d; s_r = rr - cum; s_cnt = hd; break; }
                cum += hd;
            }
        }
        __syncthreads();
        if (s_digit < 0) { if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL); __syncthreads(); return s_out; }
        prefix = (prefix << 8) | (u128)(unsigned)s_digit;
        pbits += 8;
        rr = s_r;
        cnt = s_cnt;
        __syncthreads();
    }
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        Cand e = list[i];
        u128 v = comp(e);
        if (pbits == 0 || (v >> (total - pbits)) == prefix) {
            int slot = atomicAdd(&s_n, 1);
            if (slot < SEL_SMALL) buf[slot] = e;
        }
    }
    __syncthreads();
    int n = s_n < SEL_SMALL ? s_n : SEL_SMALL;
    if (s_n > SEL_SMALL || rr < 1 || rr > n) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        __syncthreads();
        return s_out;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        u128 v = comp(buf[i]);
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += comp(buf[j]) < v ? 1 : 0;
        if (rank == rr - 1) s_out = buf[i];
    }
    __syncthreads();
    Cand res = s_out;
    __syncthreads();
    return res;
}

// FP64 distance of one row of Xp under a chain's current fit.
__device__ inline double row_d2_fp64(const float* __restrict__ x, const RowParams& rp, int p) {
    double cc[PMAX];
    for (int j = 0; j < p; ++j) cc[j] = (double)x[j] - rp.mu[j];
    double d2 = 0.0;
    for (int i = 0; i < p; ++i) {
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a += rp.M[i * PMAX + j] * cc[j];
        d2 += a * a;
    }
    return d2;
}

__global__ void __launch_bounds__(SEL_T) k_select_finish(const Chain* __restrict__ ch, SelRule* __restrict__ rule,
                                                          const Cand* __restrict__ cand_all, Cand* __restrict__ band_all,
                                                          uint8_t* __restrict__ memb_all, const float* __restrict__ Xp,
                                                          int m, int p, int pb, int hb, int fp32, Status* st) {
    __shared__ Cand buf[SEL_SMALL];
    __shared__ int s_nlo, s_nb;
    const int c = blockIdx.x;
    if (!ch[c].active) return;
    const int l = c / 2;
    SelRule& R = rule[c];
    const int C = R.cand < m ? R.cand : m;
    const int r = hb - R.below;
    if (r < 1 || r > C) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    const Cand* cand = cand_all + (size_t)c * m;
    Cand t = cta_select_rank(cand, C, r, fp32 ? 32 : 64, buf, st);
    if (t.pad) return;     // error already recorded
    if (!fp32) {
        if (threadIdx.x == 0) { R.t_key = t.key; R.t_pos = t.pos; }
        return;
    }
    // FP32 form: FP64 decision inside [t (1 - eps), t (1 + eps)]
    const float tf = __uint_as_float((unsigned)t.key);
    const unsigned long long t_lo = __float_as_uint(tf * (float)(1.0 - BAND_EPS));
    const unsigned long long t_hi = __float_as_uint(tf * (float)(1.0 + BAND_EPS));
    if (threadIdx.x == 0) { s_nlo = 0; s_nb = 0; }
    __syncthreads();
    Cand* band = band_all + (size_t)c * m;
    const RowParams& rp = ch[c].rp;
    int nlo = 0;
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        Cand e = cand[i];
        if (e.key < t_lo) { ++nlo; continue; }
        if (e.key > t_hi) continue;
        const float* x = Xp + ((size_t)l * m + e.pos) * pb;
        double d2 = row_d2_fp64(x, rp, p);
        int slot = atomicAdd(&s_nb, 1);
        Cand b;
        b.key = (unsigned long long)__double_as_longlong(d2);   // d2 >= 0: bits order as values
        b.pos = e.pos;
        b.pad = 0;
        band[slot] = b;
    }
    nlo = warp_sum_int(nlo);
    if ((threadIdx.x & 31) == 0 && nlo) atomicAdd(&s_nlo, nlo);
    __threadfence_block();
    __syncthreads();
    const int nb = s_nb;
    const int r2 = hb - R.below - s_nlo;
    if (r2 < 1 || r2 > nb) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    Cand tb = cta_select_rank(band, nb, r2, 64, buf, st);
    if (tb.pad) return;
    const u128 tv = comp(tb);
    uint8_t* mb = memb_all + (size_t)c * m;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        Cand e = band[i];
        bool in = comp(e) <= tv;
        mb[e.pos] = (uint8_t)((mb[e.pos] & 1) | (in ? 2 : 0));
    }
    if (threadIdx.x == 0) { R.t_lo = t_lo; R.t_hi = t_hi; R.band = nb; }
}

void launch_select_finish(const Plan& P, cudaStream_t s) {
    k_select_finish<<<2 * P.q, SEL_T, 0, s>>>(P.ch, P.rule, P.cand, P.band, P.memb, P.Xp, P.m, P.p, P.pb,
                                              P.hb, P.precision == RTD_FP32, P.st);
}

}  // namespace rtd
