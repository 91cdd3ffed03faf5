// rtd_rows.cuh - row-streaming kernels of the RT-DetMCD engine (templates).
//
// Every kernel here walks the n x p rows once.  Arithmetic is FP32 (FP32
// form) or FP64 (plain form) selected by the template type T; sums that
// leave a thread are FP64.  Rows of the permuted copy Xp are padded with
// zeros to pb floats (pb a multiple of 4) so that they load as float4.
#pragma once
#include "rtd_internal.cuh"
#include "rtd_async.cuh"
#include "rtd_tc.cuh"

namespace rtd {

constexpr int NT = 256;   // threads of every row kernel

// ----------------------------------------------------------- small helpers
__device__ inline long long feistel_pass(const Feistel& F, unsigned long long t) {
    unsigned long long L = t >> F.half, R = t & F.mask;
    for (int r = 0; r < 4; ++r) {
        unsigned long long nl = R;
        R = L ^ (splitmix64(F.key[r] ^ R) & F.mask);
        L = nl;
    }
    return (long long)((L << F.half) | R);
}
// perm(t) for t in [0, n); -1 if cycle walking did not return (impossible
// for a bijection, guarded anyway).
__device__ inline long long feistel_perm(const Feistel& F, long long t) {
    if (F.identity) return t;
    long long y = feistel_pass(F, (unsigned long long)t);
    for (int g = 0; y >= F.n; ++g) {
        if (g > (1 << 26)) return -1;
        y = feistel_pass(F, (unsigned long long)y);
    }
    return y;
}

// Load the first p floats of a row (zero beyond), from Xp rows (pb-aligned,
// padded) as float4.
template <int PB>
__device__ inline void load_row_padded(const float* __restrict__ row, float (&x)[PB]) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int j = 0; j < PB / 4; ++j) {
        float4 v = __ldg(r4 + j);
        x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
    }
}
// From caller rows of stride ld: exactly p floats, zero beyond.
template <int PB>
__device__ inline void load_row_user(const float* __restrict__ row, int p, bool vec4, float (&x)[PB]) {
    if (vec4) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int j = 0; j < PB / 4; ++j) {
            if (4 * j < p) {
                float4 v = __ldg(r4 + j);
                x[4 * j] = v.x; x[4 * j + 1] = v.y; x[4 * j + 2] = v.z; x[4 * j + 3] = v.w;
            } else {
                x[4 * j] = x[4 * j + 1] = x[4 * j + 2] = x[4 * j + 3] = 0.f;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < PB; ++j) x[j] = (j < p) ? __ldg(row + j) : 0.f;
    }
}

// Block-wide compaction: returns the slot of a thread whose predicate holds
// (-1 otherwise) and the total count.  All NT threads must call it.
__device__ inline int cta_compact(bool pred, int& total) {
    __shared__ int wc[NT / 32];
    unsigned mask = __ballot_sync(0xffffffffu, pred);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wc[w] = __popc(mask);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        int c = wc[i];
        if (i < w) off += c;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return pred ? off + __popc(mask & ((1u << lane) - 1u)) : -1;
}

__device__ inline int cta_sum_int(int v) {
    __shared__ int red[NT / 32];
    v = warp_sum_int(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
}

// ------------------------------------------------------ Gram accumulation
// Sum over rows of w * e e^T for the extended row vector e = (v, 1, 0...) of
// length PE = PB + 4, as 4 x 4 register blocks (bi <= bj).  Thread groups
// take interleaved rows; products in T, running sums flushed to FP64 every
// FLUSH rows (T = float) so that FP32 rounding stays local.
template <int PB, typename T>
struct GramShape {
    static constexpr int PE = PB + 4;
    static constexpr int NB = PE / 4;
    static constexpr int NBLK = NB * (NB + 1) / 2;
    static constexpr int G = (NT / NBLK) > 0 ? (NT / NBLK) : 1;
    // rows staged per tile: every thread loads one row where shared memory allows
    static constexpr int TR = (PE * (int)sizeof(T) <= 160) ? 256 : ((PE * (int)sizeof(T) <= 320) ? 128 : 64);
    static constexpr int FLUSH = 64;
};

// Running sums that leave the T chunks: FP64 for T = double; for T = float
// a compensated FP32 pair (TwoSum error terms collected in lo), which keeps
// the FP64 pipe free.
template <typename T> struct GramHi;
template <> struct GramHi<double> {
    double v[16];
    __device__ void zero() {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = 0.0;
    }
    __device__ void add(const double (&a)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] += a[e];
    }
};
template <> struct GramHi<float> {
    float hi[16], lo[16];
    __device__ void zero() {
#pragma unroll
        for (int e = 0; e < 16; ++e) { hi[e] = 0.f; lo[e] = 0.f; }
    }
    __device__ void add(const float (&a)[16]) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const FF t = ff_two_sum(hi[e], a[e]);
            hi[e] = t.hi;
            lo[e] += t.lo;
        }
    }
};

template <int PB, typename T>
struct GramAcc {
    typedef GramShape<PB, T> S;
    GramHi<T> big;
    T a32[16];
    int since, bi, bj, g, ng;
    bool on;
    // ng groups of NBLK threads take interleaved rows (ng <= G)
    __device__ void init(int groups = S::G, bool = false) {
        int t = threadIdx.x;
        ng = groups;
        g = t / S::NBLK;
        int blk = t % S::NBLK;
        on = g < ng;
        int b = blk;
        bi = 0;
        while (b >= S::NB - bi) { b -= S::NB - bi; ++bi; }
        bj = bi + b;
        big.zero();
#pragma unroll
        for (int e = 0; e < 16; ++e) a32[e] = (T)0;
        since = 0;
    }
    // before the put() calls of a batch (the tensor-core variant waits there)
    __device__ void begin() {}
    // row `slot` of the batch tile: values v (zero beyond p), then the
    // constant 1 at index p, weight w
    __device__ void put(T* tile, T* wt, int slot, const T (&v)[PB], int p, T w) {
        T* dst = tile + slot * S::PE;
#pragma unroll
        for (int j = 0; j < PB; ++j) dst[j] = v[j];
        dst[PB] = (T)0; dst[PB + 1] = (T)0; dst[PB + 2] = (T)0; dst[PB + 3] = (T)0;
        dst[p] = (T)1;
        wt[slot] = w;
    }
    __device__ void flush() {
        big.add(a32);
#pragma unroll
        for (int e = 0; e < 16; ++e) a32[e] = (T)0;
        since = 0;
    }
    // tile: k rows of PE values, weights wt
    __device__ void rows(const T* tile, const T* wt, int k) {
        if (!on) return;
        for (int r = g; r < k; r += ng) {
            const T* row = tile + r * S::PE;
            T w = wt[r];
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = row[4 * bi + i] * w; b[i] = row[4 * bj + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a32[i * 4 + j] += a[i] * b[j];
            if (++since >= S::FLUSH) flush();
        }
    }
    // Reduce over groups in fixed order and write one slot (NBLK*16 doubles).
    // red: shared scratch of G*NBLK*16 doubles.
    __device__ void store(double* red, double* slot) {
        flush();
        __syncthreads();
        if constexpr (sizeof(T) == 8) {
            if (on) {
                int blk = threadIdx.x % S::NBLK;
#pragma unroll
                for (int e = 0; e < 16; ++e) red[(g * S::NBLK + blk) * 16 + e] = big.v[e];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < S::NBLK * 16; e += NT) {
                double s = 0.0;
                for (int gg = 0; gg < ng; ++gg) s += red[gg * S::NBLK * 16 + e];
                slot[e] = s;
            }
        } else {
            FF* rf = reinterpret_cast<FF*>(red);
            if (on) {
                int blk = threadIdx.x % S::NBLK;
#pragma unroll
                for (int e = 0; e < 16; ++e) rf[(g * S::NBLK + blk) * 16 + e] = ff_two_sum(big.hi[e], big.lo[e]);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < S::NBLK * 16; e += NT) {
                FF s{0.f, 0.f};
                for (int gg = 0; gg < ng; ++gg) s = ff_add(s, rf[gg * S::NBLK * 16 + e]);
                slot[e] = ff_d(s);
            }
        }
        __syncthreads();
    }
};

// out[e] = sum over slots s (in order) of partial[s * slot_d + e], e < nv.
__global__ inline void k_sum_slots(const double* __restrict__ partial, int nslots, size_t slot_d, int nv,
                                   double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nv) return;
    double t = 0.0;
    for (int s = 0; s < nslots; ++s) t += partial[(size_t)s * slot_d + e];
    out[e] = t;
}

template <int PB, typename T>
constexpr size_t gram_smem_bytes() {
    typedef GramShape<PB, T> S;
    size_t tile = (size_t)S::TR * S::PE * sizeof(T) + (size_t)S::TR * sizeof(T);
    size_t red = (size_t)S::G * S::NBLK * 16 * sizeof(double);
    return tile > red ? tile : red;
}

// Opt in to more than the default 48 KB of dynamic shared memory.
template <typename K>
inline void set_smem(K kernel, size_t bytes) {
    if (bytes > 40 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
__host__ __device__ constexpr inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ constexpr inline size_t align128(size_t b) { return (b + 127) & ~(size_t)127; }

// Gram accumulator of a row kernel: CUDA-core GramAcc, or with TC the
// tensor-core GramTC (FP32 rows, split-BF16 products) and the extra dynamic
// shared memory it takes after the kernel's own.
template <int PB, typename T, bool TC>
struct GramPick {
    typedef GramAcc<PB, T> type;
    static constexpr size_t extra = 0;
};
template <int PB>
struct GramPick<PB, float, true> {
    typedef GramTC<PB, NT, GramShape<PB, float>::TR> type;
    static constexpr size_t extra = 128 + (size_t)type::SMEM;
};
template <typename A>
__device__ inline void gram_setup(A&, unsigned char*) {}
template <int PB, int NTH, int TR>
__device__ inline void gram_setup(GramTC<PB, NTH, TR>& a, unsigned char* region) {
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_err;
    a.setup(region, &s_taddr, &s_bar, &s_err);
}
// widths whose tensor-core Gram variants are built (25 <= p <= 48)
template <int PB> constexpr bool tc_width() { return PB == 32 || PB == 40 || PB == 48; }

// row range of CTA b of block l
__device__ inline void block_rows(int m, int cpb, int& r0, int& r1) {
    int l = blockIdx.y, b = blockIdx.x;
    long long chunk = ((long long)m + cpb - 1) / cpb;
    long long a = (long long)l * m + (long long)b * chunk;
    long long e = a + chunk;
    long long lim = (long long)(l + 1) * m;
    r0 = (int)(a < lim ? a : lim);
    r1 = (int)(e < lim ? e : lim);
}

__device__ inline unsigned long long full_key(float d) { return (unsigned long long)__float_as_uint(d); }
__device__ inline unsigned long long full_key(double d) { return (unsigned long long)__double_as_longlong(d); }

// Blocks whose start choice lies within the FP32 error band: FP64 Gram of
// the rows in exactly one of the two final h-subsets, +1 for start 2 and -1
// for start 1, relative to start 1's reference centre.  With it the
// log-determinant difference of the two subsets is exact (Section 4 step 4).
template <int PB>
__global__ void __launch_bounds__(NT) k_diff_gram(const float* __restrict__ Xp, int p, int m, int cpb,
                                                  const Chain* __restrict__ ch, const int* __restrict__ amb,
                                                  const uint8_t* __restrict__ memb, double* __restrict__ partial,
                                                  size_t slot_d) {
    typedef double T;
    typedef GramShape<PB, T> S;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    __shared__ double s_ref[PB];
    const int l = blockIdx.y;
    if (!amb[l]) return;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    for (int j = threadIdx.x; j < PB; j += NT) s_ref[j] = (j < p) ? ch[2 * l].rp.ref[j] : 0.0;
    __syncthreads();
    const uint8_t* m0 = memb + (size_t)(2 * l) * m;
    const uint8_t* m1 = memb + (size_t)(2 * l + 1) * m;
    GramAcc<PB, T> acc;
    acc.init();
    for (int base = r0; base < r1; base += S::TR) {
        int row = base + threadIdx.x;
        bool inc = false;
        T w = 0.0;
        if (threadIdx.x < S::TR && row < r1) {
            int a = m0[row - l * m] & 1, b = m1[row - l * m] & 1;
            inc = a != b;
            w = b ? 1.0 : -1.0;
        }
        int tot;
        int slot = cta_compact(inc, tot);
        if (slot >= 0) {
            float x[PB];
            load_row_padded<PB>(Xp + (size_t)row * PB, x);
            T* dst = tile + slot * S::PE;
#pragma unroll
            for (int j = 0; j < PB; ++j) dst[j] = (double)x[j] - s_ref[j];
            dst[PB] = 0.0; dst[PB + 1] = 0.0; dst[PB + 2] = 0.0; dst[PB + 3] = 0.0;
            dst[p] = 1.0;
            wt[slot] = w;
        }
        __syncthreads();
        if (tot) acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)l * cpb + blockIdx.x) * 2;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB>
void member_gram_t(const Plan& P, cudaStream_t s) {
    size_t sm = gram_smem_bytes<PB, double>();
    auto k = k_diff_gram<PB>;
    set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.ch, P.amb, P.memb, P.partial, P.slot_doubles);
}

// FP64 distance of one row (band recomputation).
// FP64 distance of one row (global memory, read through L1) under rp; used
// only for rows inside an FP64 band, so the centred row is not kept.
__device__ inline double d2_fp64(const float* __restrict__ x, const RowParams& rp, int p) {
    double d2 = 0.0;
    for (int i = 0; i < p; ++i) {
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a += rp.M[i * PMAX + j] * ((double)__ldg(x + j) - rp.mu[j]);
        d2 += a * a;
    }
    return d2;
}

// =====================================================================
// Initial estimators (Section 3.2), per block.
// Pass 1: S~_1 Gram of the wrapped rows, and the norms ||z|| as sort keys.
// Pass 2: S~_2 Gram of xi^2(||z||) z z^T.
// =====================================================================
template <typename T>
__device__ inline T wrap_g(T z) {
    const T b = (T)1.5, c = (T)4.0, q1 = (T)1.541, q2 = (T)0.862;
    T a = fabs(z);
    if (a <= b) return z;
    if (a <= c) return q1 * tanh(q2 * (c - a)) * (z < (T)0 ? (T)-1 : (T)1);
    return (T)0;
}

template <int PB, typename T, typename K, bool TC = false>
__global__ void __launch_bounds__(NT) k_start1(const float* __restrict__ Xp, int p, int m, int cpb,
                                               const Consts* __restrict__ cs, K* __restrict__ rkeys,
                                               double* __restrict__ partial, size_t slot_d) {
    typedef GramShape<PB, T> S;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    __shared__ T s_mu[PB], s_is[PB];
    for (int j = threadIdx.x; j < PB; j += NT) {
        s_mu[j] = (j < p) ? (T)cs->mu_uni[j] : (T)0;
        s_is[j] = (j < p) ? (T)(1.0 / cs->s_uni[j]) : (T)0;
    }
    __syncthreads();
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    typename GramPick<PB, T, TC>::type acc;
    gram_setup(acc, smem + (TC ? 0 : align128(gram_smem_bytes<PB, T>())));   // the tensor-core Gram stages its own rows
    acc.init();
    for (int base = r0; base < r1; base += S::TR) {
        int row = base + threadIdx.x;
        bool pred = threadIdx.x < S::TR && row < r1;
        T w[PB];
        if (pred) {
            float x[PB];
            load_row_padded<PB>(Xp + (size_t)row * PB, x);
            T r2 = 0;
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                T z = ((T)x[j] - s_mu[j]) * s_is[j];
                r2 += z * z;
                w[j] = wrap_g<T>(z);
            }
            rkeys[row] = KeyOps<K>::enc(sqrt(r2));
        }
        int tot;
        int slot = cta_compact(pred, tot);
        acc.begin();
        if (slot >= 0) acc.put(tile, wt, slot, w, p, (T)1);
        __syncthreads();
        acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 0;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB, typename T, typename K, bool TC = false>
__global__ void __launch_bounds__(NT) k_start2(const float* __restrict__ Xp, int p, int m, int cpb,
                                               const Consts* __restrict__ cs, const double* __restrict__ gss,
                                               double* __restrict__ partial, size_t slot_d) {
    typedef GramShape<PB, T> S;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    __shared__ T s_mu[PB], s_is[PB];
    for (int j = threadIdx.x; j < PB; j += NT) {
        s_mu[j] = (j < p) ? (T)cs->mu_uni[j] : (T)0;
        s_is[j] = (j < p) ? (T)(1.0 / cs->s_uni[j]) : (T)0;
    }
    __syncthreads();
    const double A = gss[2 * blockIdx.y], B = gss[2 * blockIdx.y + 1];
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    typename GramPick<PB, T, TC>::type acc;
    gram_setup(acc, smem + (TC ? 0 : align128(gram_smem_bytes<PB, T>())));   // the tensor-core Gram stages its own rows
    acc.init();
    for (int base = r0; base < r1; base += S::TR) {
        int row = base + threadIdx.x;
        bool pred = threadIdx.x < S::TR && row < r1;
        T z[PB];
        T xi2 = 0;
        if (pred) {
            float x[PB];
            load_row_padded<PB>(Xp + (size_t)row * PB, x);
            T r2 = 0;
#pragma unroll
            for (int j = 0; j < PB; ++j) {
                z[j] = ((T)x[j] - s_mu[j]) * s_is[j];
                r2 += z[j] * z[j];
            }
            // the same norm as pass 1 (same operations), then xi of Section 3.2
            double r = (double)(T)sqrt(r2);
            double xi = (r <= A) ? 1.0 : (r <= B ? (B - r) / (B - A) : 0.0);
            xi2 = (T)(xi * xi);
            pred = xi2 != (T)0;
        }
        int tot;
        int slot = cta_compact(pred, tot);
        acc.begin();
        if (slot >= 0) acc.put(tile, wt, slot, z, p, xi2);
        __syncthreads();
        acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 1;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB, typename T, typename K, bool TC = false>
void start1_t(const Plan& P, cudaStream_t s) {
    if constexpr (!TC && tc_width<PB>() && sizeof(T) == 4) {
        if (P.tc) { start1_t<PB, T, K, true>(P, s); return; }
    }
    size_t sm = TC ? GramPick<PB, T, TC>::extra : gram_smem_bytes<PB, T>();
    auto k = k_start1<PB, T, K, TC>;
    if (TC) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.cs, (K*)P.arenaA, P.partial, P.slot_doubles);
}
template <int PB, typename T, typename K, bool TC = false>
void start2_t(const Plan& P, cudaStream_t s) {
    if constexpr (!TC && tc_width<PB>() && sizeof(T) == 4) {
        if (P.tc) { start2_t<PB, T, K, true>(P, s); return; }
    }
    size_t sm = TC ? GramPick<PB, T, TC>::extra : gram_smem_bytes<PB, T>();
    auto k = k_start2<PB, T, K, TC>;
    if (TC) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.cs, P.gss, P.partial, P.slot_doubles);
}

// =====================================================================
// Refinement transforms (Section 3.3): per block and start k, the p values
// W_k (x - mu_uni) of each row written as sort keys, segment
// ((l * 2 + k) * p + j) of length m.  W = V^T D^-1 gives the scores
// T = Z V; W = Sigma_k^{-1/2} D^-1 gives the sphered rows Z~.
// =====================================================================
template <int PB, typename T, typename K>
__global__ void __launch_bounds__(NT) k_transform(const float* __restrict__ Xp, int p, int m, int cpb,
                                                  const Consts* __restrict__ cs, const Chain* __restrict__ ch,
                                                  K* __restrict__ keys) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sW = reinterpret_cast<T*>(smem);          // [2][PB][PB]
    __shared__ T s_mu[PB];
    __shared__ int act[2];
    const int l = blockIdx.y;
    if (threadIdx.x < 2) act[threadIdx.x] = ch[2 * l + threadIdx.x].status == CH_OK;
    for (int e = threadIdx.x; e < 2 * PB * PB; e += NT) {
        int k = e / (PB * PB), r = (e / PB) % PB, c = e % PB;
        // Chain.G holds W during the refinement (row j = output j)
        sW[e] = (r < p && c < p) ? (T)ch[2 * l + k].G[r * PMAX + c] : (T)0;
    }
    for (int j = threadIdx.x; j < PB; j += NT) s_mu[j] = (j < p) ? (T)cs->mu_uni[j] : (T)0;
    __syncthreads();
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    for (int row = r0 + threadIdx.x; row < r1; row += NT) {
        float x[PB];
        load_row_padded<PB>(Xp + (size_t)row * PB, x);
        T c[PB];
#pragma unroll
        for (int j = 0; j < PB; ++j) c[j] = (T)x[j] - s_mu[j];
        int t = row - l * m;
        for (int k = 0; k < 2; ++k) {
            if (!act[k]) continue;
            K* out = keys + ((size_t)(l * 2 + k) * p) * m + t;
            for (int j = 0; j < p; ++j) {
                T acc = 0;
#pragma unroll
                for (int i = 0; i < PB; ++i) acc += sW[(k * PB + j) * PB + i] * c[i];
                out[(size_t)j * m] = KeyOps<K>::enc(acc);
            }
        }
    }
}

template <int PB, typename T, typename K>
void transform_t(const Plan& P, cudaStream_t s) {
    dim3 grid(P.cpb, P.q);
    size_t sm = 2 * PB * PB * sizeof(T);
    auto k = k_transform<PB, T, K>;
    set_smem(k, sm);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.cs, P.ch, (K*)P.arenaA);
}
// =====================================================================
// C-step distances (Sections 2.1 and 3.4): d2 = ||M (x - mu)||^2 with
// M = L^-1 D^-1 for both starts of the row's block, fused with the
// top-digit histogram of the radix select.
// =====================================================================
template <typename T> struct Vec4;
template <> struct Vec4<float> {
    __device__ static void ld(const float* p, float (&v)[4]) {
        float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct Vec4<double> {
    __device__ static void ld(const double* p, double (&v)[4]) {
        double2 a = *reinterpret_cast<const double2*>(p);
        double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

// rows per thread of the plain distance passes
template <int PB, typename T> struct DistRows { static constexpr int R = (PB <= 24 && sizeof(T) == 4) ? 2 : 1; };

// y = M c row by row (lower triangular M, row stride PB, zero above the
// diagonal), d2 = sum y^2, for R rows at once.
template <int PB, typename T, int R>
__device__ inline void tri_d2(const T* __restrict__ sM, int p, const T (&c)[R][PB], T (&d2)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) d2[r] = 0;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
        if (i < p) {
            T acc[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = 0;
#pragma unroll
            for (int j4 = 0; j4 <= i / 4; ++j4) {
                T mv[4];
                Vec4<T>::ld(sM + i * PB + 4 * j4, mv);
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[r] += mv[u] * c[r][4 * j4 + u];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) d2[r] += acc[r] * acc[r];
        }
    }
}

template <typename T> __device__ inline void load_center(const RowParams& rp, int j, T& hi, T& lo);
template <> __device__ inline void load_center<float>(const RowParams& rp, int j, float& hi, float& lo) {
    hi = rp.mu_hi[j]; lo = rp.mu_lo[j];
}
template <> __device__ inline void load_center<double>(const RowParams& rp, int j, double& hi, double& lo) {
    hi = rp.mu[j]; lo = 0.0;
}
template <typename T> __device__ inline T load_m(const RowParams& rp, int i, int j);
template <> __device__ inline float load_m<float>(const RowParams& rp, int i, int j) { return rp.Mf[i * PMAX + j]; }
template <> __device__ inline double load_m<double>(const RowParams& rp, int i, int j) { return rp.M[i * PMAX + j]; }

// Warp-aggregated increment of a shared histogram bin (lanes with equal
// bins add once).
__device__ inline void hist_add(unsigned* h, unsigned bin, bool valid) {
    const int lane = threadIdx.x & 31;
    unsigned tag = valid ? bin : (0x80000000u | lane);
    unsigned peers = __match_any_sync(0xffffffffu, tag);
    if (valid && (__ffs(peers) - 1) == lane) atomicAdd(h + bin, (unsigned)__popc(peers));
}

// Per-step counters of the membership pass and the finalize start at zero;
// the first kernel of a C-step clears them (stream-ordered before both).
__device__ __forceinline__ void clear_step_counters(Status* st, int* blk) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        blk[blockIdx.y] = 0;
        if (blockIdx.y == 0) {
            st->active = 0;
            st->active_blocks = 0;
            st->done = 0;
            st->gram_rows = 0ull;
        }
    }
}

template <int PB, typename T>
__global__ void __launch_bounds__(NT, 2) k_dist(const float* __restrict__ Xp, int p, int m, int cpb,
                                                const Chain* __restrict__ ch, T* __restrict__ dkeys,
                                                long long qm, unsigned* __restrict__ hist, Status* st, int* blk) {
    constexpr int R = DistRows<PB, T>::R;
    clear_step_counters(st, blk);
    extern __shared__ __align__(16) unsigned char smem[];
    T* sMb = reinterpret_cast<T*>(smem);                                   // [2][PB*PB]
    unsigned* shb = reinterpret_cast<unsigned*>(smem + 2 * PB * PB * sizeof(T));  // [2][HIST_BINS]
    __shared__ T s_hi[2][PB], s_lo[2][PB];
    __shared__ int act[2];
    const int l = blockIdx.y;
    if (threadIdx.x < 2) act[threadIdx.x] = ch[2 * l + threadIdx.x].active;
    for (int e = threadIdx.x; e < 2 * PB * PB; e += NT) {
        int k = e / (PB * PB), i = (e / PB) % PB, j = e % PB;
        sMb[e] = (i < p && j <= i) ? load_m<T>(ch[2 * l + k].rp, i, j) : (T)0;
    }
    for (int e = threadIdx.x; e < 2 * PB; e += NT) {
        int k = e / PB, j = e % PB;
        T hi = 0, lo = 0;
        if (j < p) load_center<T>(ch[2 * l + k].rp, j, hi, lo);
        s_hi[k][j] = hi; s_lo[k][j] = lo;
    }
    for (int e = threadIdx.x; e < 2 * HIST_BINS; e += NT) shb[e] = 0u;
    __syncthreads();
    const int a0 = act[0], a1 = act[1];
    if (!a0 && !a1) return;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    for (int base = r0 + threadIdx.x * R; base - threadIdx.x * R < r1; base += NT * R) {
        float x[R][PB];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (base + r < r1) load_row_padded<PB>(Xp + (size_t)(base + r) * PB, x[r]);
            else {
#pragma unroll
                for (int j = 0; j < PB; ++j) x[r][j] = 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!(k ? a1 : a0)) continue;
            T c[R][PB];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int j = 0; j < PB; ++j) c[r][j] = ((T)x[r][j] - s_hi[k][j]) - s_lo[k][j];
            T d2[R];
            tri_d2<PB, T, R>(sMb + k * PB * PB, p, c, d2);
            T* out = dkeys + (size_t)k * qm;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bool v = base + r < r1;
                if (v) out[base + r] = d2[r];
                hist_add(shb + k * HIST_BINS, coarse_key(d2[r]) >> (32 - HIST_BITS), v);
            }
        }
    }
    __syncthreads();
    for (int k = 0; k < 2; ++k) {
        if (!act[k]) continue;
        unsigned* gh = hist + (size_t)(2 * l + k) * HIST_BINS;
        for (int b = threadIdx.x; b < HIST_BINS; b += NT) {
            unsigned v = shb[k * HIST_BINS + b];
            if (v) atomicAdd(gh + b, v);
        }
    }
}

template <int PB, typename T>
void dist_t(const Plan& P, cudaStream_t s) {
    dim3 grid(P.cpb_dist, P.q);
    size_t sm = 2 * PB * PB * sizeof(T) + 2 * HIST_BINS * sizeof(unsigned);
    auto k = k_dist<PB, T>;
    set_smem(k, sm);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb_dist, P.ch, (T*)P.dkeys, (long long)P.q * P.m, P.hist, P.st,
                           P.blk_active);
}
// =====================================================================
// C-step distances of the FP32 form from the second step on (Sections 2.1,
// 3.4).  The block's rows stream through shared memory in tiles brought by
// bulk asynchronous copies (two stages, one thread issues them).  Rows are
// centred once at the FP32 univariate centre u; each start's
// y = M (x - u) - bf, bf = M (mu - u), is formed with packed FP32 FMAs that
// carry the even and odd columns of a row in the two halves.  Each key is
// then classified against the chain's predicted window [w_lo, w_hi]: rows
// below it are counted, rows inside it are listed as candidates and counted
// in a histogram of WIN_BINS bins over the window.  The keys are written
// for the membership pass and for the histogram path a missed window falls
// back to.
// =====================================================================
template <int PB> struct DistWin {
    static constexpr int R = 2;                      // rows per lane
    static constexpr int NTW = PB <= 40 ? 256 : 128; // threads
    static constexpr int NW = NTW / 32;              // warps
    static constexpr int WT = 32 * R;                // rows per warp tile
    static constexpr int STAGES = 2;                 // tiles in flight per warp
    static constexpr int PH = PB / 2;                // column pairs per row
    static constexpr size_t WTILE = (size_t)WT * PB * sizeof(float);
    static constexpr size_t SMEM = NW * STAGES * WTILE + 2 * (size_t)PB * PB * sizeof(float) +
                                   2 * (size_t)WIN_BINS * sizeof(unsigned);
    // resident CTAs per SM by shared memory (1 KB reserved per CTA), at most 2
    static constexpr int BY_SMEM = (int)((227 * 1024) / (SMEM + 1024));
    static constexpr int CTAS_PER_SM = BY_SMEM > 2 ? 2 : (BY_SMEM < 1 ? 1 : BY_SMEM);
    static_assert(SMEM + 1024 <= 227 * 1024, "row stages exceed shared memory");
};

// d2 of R rows for lower-triangular M stored as column pairs (row stride
// PB / 2 pairs, zero above the diagonal and beyond p); b the folded centre.
// Two rows of M at a time (they share their column pairs), and column pairs
// alternating between two accumulators, give 8 independent chains.
template <int PB, int R>
__device__ __forceinline__ void tri_d2_pk(const float2* __restrict__ sM, int p, const float2 (&c)[R][PB / 2],
                                          const float* __restrict__ b, float (&d2)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) d2[r] = 0.f;
#pragma unroll
    for (int i = 0; i < PB; i += 2) {
        if (i < p) {
            const int npair = i / 2 + 1;                    // pairs holding columns 0..i+1
            const float2 bi = make_float2(-b[i], 0.f), bj = make_float2(-b[i + 1], 0.f);
            float2 a0[R], a1[R], c0[R], c1[R];             // rows i (a) and i + 1 (c)
#pragma unroll
            for (int g = 0; 2 * g < npair; ++g) {
                const float4 mi = *reinterpret_cast<const float4*>(sM + i * (PB / 2) + 2 * g);
                const float4 mj = *reinterpret_cast<const float4*>(sM + (i + 1) * (PB / 2) + 2 * g);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    a0[r] = __ffma2_rn(make_float2(mi.x, mi.y), c[r][2 * g], g == 0 ? bi : a0[r]);
                    c0[r] = __ffma2_rn(make_float2(mj.x, mj.y), c[r][2 * g], g == 0 ? bj : c0[r]);
                }
                if (2 * g + 1 < npair) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float2 mi1 = make_float2(mi.z, mi.w), mj1 = make_float2(mj.z, mj.w);
                        a1[r] = (g == 0) ? __fmul2_rn(mi1, c[r][1]) : __ffma2_rn(mi1, c[r][2 * g + 1], a1[r]);
                        c1[r] = (g == 0) ? __fmul2_rn(mj1, c[r][1]) : __ffma2_rn(mj1, c[r][2 * g + 1], c1[r]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float2 a = a0[r], cc = c0[r];
                if (npair > 1) { a = __fadd2_rn(a, a1[r]); cc = __fadd2_rn(cc, c1[r]); }
                const float ya = a.x + a.y, yc = cc.x + cc.y;
                d2[r] = fmaf(ya, ya, d2[r]);
                d2[r] = fmaf(yc, yc, d2[r]);
            }
        }
    }
}

template <int PB>
__global__ void __launch_bounds__(DistWin<PB>::NTW, DistWin<PB>::CTAS_PER_SM)
    k_dist_win(const float* __restrict__ Xp, int p, int m, int cpb, const Consts* __restrict__ cs,
               const Chain* __restrict__ ch, SelRule* __restrict__ rule, float* __restrict__ dkeys,
               long long qm, Cand* __restrict__ cand, int* __restrict__ segcnt, unsigned* __restrict__ hist,
               Status* st, int* blk) {
    typedef DistWin<PB> D;
    clear_step_counters(st, blk);
    constexpr int R = D::R, PH = D::PH, NTW = D::NTW, NW = D::NW, WT = D::WT;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* sM = reinterpret_cast<float2*>(smem + NW * D::STAGES * D::WTILE);   // [2][PB][PH]
    unsigned* sh = reinterpret_cast<unsigned*>(smem + NW * D::STAGES * D::WTILE + 2 * (size_t)PB * PB * sizeof(float));
    __shared__ __align__(8) uint64_t bar[NW][D::STAGES];
    __shared__ float2 s_nu[PH];
    __shared__ float s_b[2][PB];
    __shared__ unsigned s_wlo[2], s_whi[2];
    __shared__ int s_wsh[2], s_on[2], s_below[2], s_ncand[2], s_fail;
    const int l = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    const int ntiles = (r1 - r0 + WT - 1) / WT;      // warp tiles of the CTA
    const int seg0 = r0 - l * m;                     // this CTA's candidate segment
    if (threadIdx.x < 2) {
        const int c = 2 * l + threadIdx.x;
        s_on[threadIdx.x] = ch[c].active && rule[c].win;
        s_wlo[threadIdx.x] = rule[c].w_lo;
        s_whi[threadIdx.x] = rule[c].w_hi;
        s_wsh[threadIdx.x] = rule[c].w_sh;
        s_below[threadIdx.x] = 0;
        s_ncand[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) s_fail = 0;
    if (lane == 0) {
        for (int s = 0; s < D::STAGES; ++s) mbar_init(&bar[w][s], 1);
        mbar_init_fence();
    }
    for (int e = threadIdx.x; e < 2 * WIN_BINS; e += NTW) sh[e] = 0u;
    for (int e = threadIdx.x; e < 2 * PB * PH; e += NTW) {
        const int k = e / (PB * PH), i = (e / PH) % PB, h = e % PH;
        const float* Mf = ch[2 * l + k].rp.Mf;
        const int j0 = 2 * h, j1 = 2 * h + 1;
        sM[e] = make_float2((i < p && j0 <= i) ? Mf[i * PMAX + j0] : 0.f, (i < p && j1 <= i) ? Mf[i * PMAX + j1] : 0.f);
    }
    for (int e = threadIdx.x; e < 2 * PB; e += NTW) {
        const int k = e / PB, j = e % PB;
        s_b[k][j] = (j < p) ? ch[2 * l + k].rp.bf[j] : 0.f;
    }
    for (int h = threadIdx.x; h < PH; h += NTW) {
        const float a = (2 * h < p) ? -(float)cs->mu_uni[2 * h] : 0.f;
        const float b = (2 * h + 1 < p) ? -(float)cs->mu_uni[2 * h + 1] : 0.f;
        s_nu[h] = make_float2(a, b);
    }
    __syncthreads();
    if (!s_on[0] && !s_on[1]) return;   // uniform; nothing issued yet

    // warp w takes the CTA's warp tiles w, w + NW, ...; its k-th tile sits in stage k % STAGES
    float* wst = reinterpret_cast<float*>(smem) + (size_t)w * D::STAGES * WT * PB;
    auto issue = [&](int k) {   // lane 0 only
        const int t = w + k * NW;
        const int row0 = r0 + t * WT;
        const int rows = min(WT, r1 - row0);
        const unsigned bytes = (unsigned)rows * PB * (unsigned)sizeof(float);
        uint64_t* br = &bar[w][k % D::STAGES];
        mbar_expect_tx(br, bytes);
        bulk_load(wst + (size_t)(k % D::STAGES) * WT * PB, Xp + (size_t)row0 * PB, bytes, br);
    };
    const int nmine = (ntiles > w) ? (ntiles - w + NW - 1) / NW : 0;
    if (lane == 0)
        for (int k = 0; k < D::STAGES && k < nmine; ++k) issue(k);
    __syncwarp();

    int below0 = 0, below1 = 0;
    bool failed = false;
    int k = 0;
    for (; k < nmine; ++k) {
        const int t = w + k * NW;
        const int row0 = r0 + t * WT;
        const int rows = min(WT, r1 - row0);
        const bool ok = mbar_wait(&bar[w][k % D::STAGES], (unsigned)(k / D::STAGES) & 1u);
        if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
        const float* T = wst + (size_t)(k % D::STAGES) * WT * PB;
        float2 c[R][PH];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = r * 32 + lane;
            if (j < rows) {
                const float4* src = reinterpret_cast<const float4*>(T + (size_t)j * PB);
#pragma unroll
                for (int q4 = 0; q4 < PB / 4; ++q4) {
                    const float4 v = src[q4];
                    c[r][2 * q4] = __fadd2_rn(make_float2(v.x, v.y), s_nu[2 * q4]);
                    c[r][2 * q4 + 1] = __fadd2_rn(make_float2(v.z, v.w), s_nu[2 * q4 + 1]);
                }
            } else {
#pragma unroll
                for (int h = 0; h < PH; ++h) c[r][h] = make_float2(0.f, 0.f);
            }
        }
        __syncwarp();   // the stage is read: lane 0 may refill it
        if (lane == 0 && k + D::STAGES < nmine) {
            async_proxy_fence();
            issue(k + D::STAGES);
        }
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            if (!s_on[kc]) continue;
            float d2[R];
            tri_d2_pk<PB, R>(sM + kc * PB * PH, p, c, s_b[kc], d2);
            const int cidx = 2 * l + kc;
            const unsigned wlo = s_wlo[kc], whi = s_whi[kc];
            const int wsh = s_wsh[kc];
            float* out = dkeys + (size_t)kc * qm;
            int nb = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = r * 32 + lane;
                const int row = row0 + j;
                const unsigned key = __float_as_uint(d2[r]);
                bool cnd = false;
                if (j < rows) {
                    const bool in = key < wlo;
                    cnd = !in && key <= whi;
                    nb += in ? 1 : 0;
                    out[row] = d2[r];
                    if (cnd) atomicAdd(&sh[kc * WIN_BINS + ((key - wlo) >> wsh)], 1u);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, cnd);
                if (bal) {
                    const int lead = __ffs(bal) - 1;
                    int b0 = 0;
                    if (lane == lead) b0 = atomicAdd(&s_ncand[kc], __popc(bal));
                    b0 = __shfl_sync(0xffffffffu, b0, lead);
                    if (cnd) {
                        Cand e;
                        e.key = key;
                        e.pos = (unsigned)(row - l * m);
                        e.pad = 0;
                        cand[(size_t)cidx * m + seg0 + b0 + __popc(bal & ((1u << lane) - 1u))] = e;
                    }
                }
            }
            if (kc == 0) below0 += nb; else below1 += nb;
        }
    }
    if (failed) {
        // let this warp's copies still in flight land before the CTA's shared memory is released
        if (lane == 0)
            for (int u = k; u < nmine && u < k + D::STAGES; ++u)
                (void)mbar_wait(&bar[w][u % D::STAGES], (unsigned)(u / D::STAGES) & 1u);
        if (lane == 0) s_fail = 1;
    }
    below0 = warp_sum_int(below0);
    below1 = warp_sum_int(below1);
    if (lane == 0) {
        if (below0) atomicAdd(&s_below[0], below0);
        if (below1) atomicAdd(&s_below[1], below1);
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    if (threadIdx.x < 2 && s_on[threadIdx.x]) {
        const int c = 2 * l + threadIdx.x;
        if (s_below[threadIdx.x]) atomicAdd(&rule[c].below, s_below[threadIdx.x]);
        segcnt[(size_t)c * SEG_MAX + blockIdx.x] = s_ncand[threadIdx.x];
        if (s_ncand[threadIdx.x]) atomicAdd(&rule[c].cand, s_ncand[threadIdx.x]);
        if (blockIdx.x == 0) rule[c].nseg = gridDim.x;
    }
    for (int kc = 0; kc < 2; ++kc) {
        if (!s_on[kc]) continue;
        unsigned* gh = hist + (size_t)(2 * l + kc) * HIST_BINS;
        for (int b = threadIdx.x; b < WIN_BINS; b += NTW) {
            const unsigned v = sh[kc * WIN_BINS + b];
            if (v) atomicAdd(gh + b, v);
        }
    }
}

template <int PB>
void dist_win_t(const Plan& P, cudaStream_t s) {
    typedef DistWin<PB> D;
    // one resident wave, at least 256 rows per CTA
    long long cw = (long long)D::CTAS_PER_SM * P.nsm / P.q;
    const long long rpc = P.win_rows > 256 ? P.win_rows : 256;
    const long long lim = ((long long)P.m + rpc - 1) / rpc;
    if (cw > lim) cw = lim;
    if (cw > SEG_MAX) cw = SEG_MAX;
    const int cpb = (int)(cw > 0 ? cw : 1);
    dim3 grid(cpb, P.q);
    auto k = k_dist_win<PB>;
    set_smem(k, D::SMEM);
    k<<<grid, D::NTW, D::SMEM, s>>>(P.Xp, P.p, P.m, cpb, P.cs, P.ch, P.rule, (float*)P.dkeys,
                                    (long long)P.q * P.m, P.cand, P.segcnt, P.hist, P.st, P.blk_active);
}

// =====================================================================
// C-step distances of the FP32 form from the second step on, on the tensor
// cores (Sections 2.1, 3.4).  For a tile of 128 rows centred at the FP32
// univariate centre u, Y = C [M_1^T | M_2^T] (both starts of the block) is a
// 128 x p x 2p product taken by tcgen05.mma kind::tf32 with split operands:
// c = c_hi + c_lo, M = M_hi + M_lo (c_hi, M_hi the TF32 high parts, the low
// parts exact FP32 differences), Y = C_hi M_hi + C_lo M_hi + C_hi M_lo, which
// leaves about 2^-19 relative error per product against |M| |c|: far inside
// the FP64 band of 2^-9 in which every decision is recomputed in FP64.  The
// accumulator (FP32, tensor memory: lane = row, column = output) is read back
// by the row's own thread, which forms d2_k = |y_k - b_k|^2 (b = M (mu - u)
// in FP64, rounded once) and classifies the key against the chain's window
// exactly as the CUDA-core pass does.  Rows arrive by bulk copies, two tiles
// ahead; every wait is bounded and records an error.
//
// Shared-memory operands are K-major without swizzle: element (r, k) of a
// part at ((r / 8) KCH + k / 4) 128 + (r % 8) 16 + (k % 4) 4 bytes, so that
// core matrices along K are 128 bytes apart (LBO) and 8-row groups KCH * 128
// bytes apart (SBO).
// =====================================================================
template <int PB> struct DistTC {
    static constexpr int KP = (PB + 7) / 8 * 8;            // K padded to the TF32 step (8)
    static constexpr int KCH = KP / 4;                     // 16-byte K chunks per row
    static constexpr int NC = 2 * KP;                      // N: both starts' outputs
    static constexpr int TM = 128;                         // rows per tile (M)
    static constexpr int NTH = 128;                        // one thread per tile row
    static constexpr int RS = PB <= 24 ? 3 : 2;            // raw tile stages (bulk copies in flight)
    static constexpr int TCOLS = 2 * NC <= 32 ? 32 : (2 * NC <= 64 ? 64 : (2 * NC <= 128 ? 128 : 256));
    static constexpr size_t RAW = (size_t)TM * PB * 4;    // one raw tile
    static constexpr size_t AOP = (size_t)TM * KP * 4;    // one part of one A buffer
    static constexpr size_t BOP = (size_t)NC * KP * 4;    // one part of B
    static constexpr size_t OFF_A = (RS * RAW + 127) / 128 * 128;
    static constexpr size_t OFF_B = OFF_A + 4 * AOP;      // A: 2 buffers x (hi, lo)
    static constexpr size_t SMEM = OFF_B + 2 * BOP;
    static constexpr int BY_SMEM = (int)((227 * 1024) / (SMEM + 1024));
    static constexpr int BY_TMEM = 512 / TCOLS;
    static constexpr int CTAS_PER_SM = BY_SMEM < BY_TMEM ? (BY_SMEM < 4 ? (BY_SMEM < 1 ? 1 : BY_SMEM) : 4)
                                                         : (BY_TMEM < 4 ? BY_TMEM : 4);
    static_assert(NC % 16 == 0 && NC <= 256, "N of the MMA");
    static_assert(SMEM + 1024 <= 227 * 1024, "operands exceed shared memory");
};

__device__ __forceinline__ unsigned kop_off(int r, int k, int kch) {
    return (unsigned)(((r >> 3) * kch + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// 32 lanes x 16 columns of tensor memory into registers, without the wait
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int PB>
__global__ void __launch_bounds__(DistTC<PB>::NTH, DistTC<PB>::CTAS_PER_SM)
    k_dist_tc(const float* __restrict__ Xp, int p, int m, int cpb, const Consts* __restrict__ cs,
              const Chain* __restrict__ ch, SelRule* __restrict__ rule, float* __restrict__ dkeys, long long qm,
              Cand* __restrict__ cand, int* __restrict__ segcnt, unsigned* __restrict__ hist, Status* st,
              int* blk) {
    typedef DistTC<PB> D;
    constexpr int KP = D::KP, KCH = D::KCH, NC = D::NC, TM = D::TM, NTH = D::NTH, RS = D::RS;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* raw = reinterpret_cast<float*>(smem);
    unsigned char* Abase = smem + D::OFF_A;        // [buffer][hi, lo]
    unsigned char* Bh = smem + D::OFF_B;
    unsigned char* Bl = Bh + D::BOP;
    __shared__ __align__(8) uint64_t bar_raw[RS];
    __shared__ __align__(8) uint64_t bar_mma[2];
    __shared__ uint32_t s_taddr;
    __shared__ float s_nu[PB];
    __shared__ float s_b[2][KP];
    __shared__ unsigned s_wlo[2], s_whi[2];
    __shared__ int s_wsh[2], s_on[2], s_below[2], s_ncand[2], s_fail;
    const int l = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    clear_step_counters(st, blk);
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    const int ntiles = (r1 - r0 + TM - 1) / TM;
    const int seg0 = r0 - l * m;                     // this CTA's candidate segment
    if (tid < 2) {
        const int c = 2 * l + tid;
        s_on[tid] = ch[c].active && rule[c].win;
        s_wlo[tid] = rule[c].w_lo;
        s_whi[tid] = rule[c].w_hi;
        s_wsh[tid] = rule[c].w_sh;
        s_below[tid] = 0;
        s_ncand[tid] = 0;
        if (s_on[tid]) {
            if (ntiles == 0) segcnt[(size_t)c * SEG_MAX + blockIdx.x] = 0;
            if (blockIdx.x == 0) rule[c].nseg = gridDim.x;
        }
    }
    if (tid == 0) {
        for (int i = 0; i < RS; ++i) mbar_init(&bar_raw[i], 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_init_fence();
        s_fail = 0;
    }
    // B = [M_1^T | M_2^T]: row n = k KP + i of B is row i of M_k (zero beyond p)
    for (int e = tid; e < NC * KP; e += NTH) {
        const int n = e / KP, j = e % KP;
        const int k = n / KP, i = n % KP;
        const float v = (i < p && j <= i) ? ch[2 * l + k].rp.Mf[i * PMAX + j] : 0.f;
        const float hi = tf32_hi(v);
        *reinterpret_cast<float*>(Bh + kop_off(n, j, KCH)) = hi;
        *reinterpret_cast<float*>(Bl + kop_off(n, j, KCH)) = v - hi;
    }
    for (int e = tid; e < 2 * KP; e += NTH) {
        const int k = e / KP, j = e % KP;
        s_b[k][j] = (j < p) ? ch[2 * l + k].rp.bf[j] : 0.f;
    }
    for (int j = tid; j < PB; j += NTH) s_nu[j] = (j < p) ? -(float)cs->mu_uni[j] : 0.f;
    async_proxy_fence();    // B, written by threads, is read by the tensor cores
    __syncthreads();
    if ((!s_on[0] && !s_on[1]) || ntiles == 0) return;   // uniform; nothing issued, nothing allocated
    if (w == 0) {
        tmem_alloc(&s_taddr, D::TCOLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    auto issue = [&](int t) {   // thread 0
        const int row0 = r0 + t * TM;
        const int rows = min(TM, r1 - row0);
        const unsigned bytes = (unsigned)rows * PB * (unsigned)sizeof(float);
        mbar_expect_tx(&bar_raw[t % RS], bytes);
        bulk_load(raw + (size_t)(t % RS) * TM * PB, Xp + (size_t)row0 * PB, bytes, &bar_raw[t % RS]);
    };
    if (tid == 0)
        for (int t = 0; t < RS && t < ntiles; ++t) issue(t);
    const uint32_t idesc = idesc_tf32(TM, NC);
    const uint32_t abase = smem_addr(Abase), boff_h = smem_addr(Bh), boff_l = smem_addr(Bl);
    int below0 = 0, below1 = 0;

    // epilogue of tile u: d2 of this thread's row from accumulator u & 1,
    // classification against the windows
    auto epilogue = [&](int u) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&bar_mma[u & 1], (unsigned)(u >> 1) & 1u));
        if (!ok) {
            if (lane == 0) s_fail = 1;
            return;
        }
        tc_fence_after();
        const int row0 = r0 + u * TM;
        const int rows = min(TM, r1 - row0);
        float d2[2] = {0.f, 0.f};
        const uint32_t lrow = taddr + ((uint32_t)(w * 32) << 16) + (uint32_t)((u & 1) * NC);
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 32) {
            uint32_t va[16], vb[16];
            tmem_ld16_nowait(lrow + (uint32_t)c0, va);
            if (c0 + 16 < NC) tmem_ld16_nowait(lrow + (uint32_t)(c0 + 16), vb);
            tmem_wait_ld();
#pragma unroll
            for (int u2 = 0; u2 < 32; ++u2) {
                const int col = c0 + u2;
                if (col < NC) {
                    const int kc = col / KP, i = col % KP;
                    if (i < p) {
                        const float y = __uint_as_float(u2 < 16 ? va[u2] : vb[u2 - 16]) - s_b[kc][i];
                        d2[kc] = fmaf(y, y, d2[kc]);
                    }
                }
            }
        }
        tc_fence_before();
        const int row = row0 + tid;
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            if (!s_on[kc]) continue;
            const int cidx = 2 * l + kc;
            const unsigned wlo = s_wlo[kc], whi = s_whi[kc];
            const unsigned key = __float_as_uint(d2[kc]);
            bool cnd = false;
            if (tid < rows) {
                const bool in = key < wlo;
                cnd = !in && key <= whi;
                if (kc == 0) below0 += in ? 1 : 0; else below1 += in ? 1 : 0;
                dkeys[(size_t)kc * qm + row] = d2[kc];
                if (cnd) atomicAdd(hist + (size_t)cidx * HIST_BINS + ((key - wlo) >> s_wsh[kc]), 1u);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, cnd);
            if (bal) {
                const int lead = __ffs(bal) - 1;
                int b0 = 0;
                if (lane == lead) b0 = atomicAdd(&s_ncand[kc], __popc(bal));
                b0 = __shfl_sync(0xffffffffu, b0, lead);
                if (cnd) {
                    Cand e;
                    e.key = key;
                    e.pos = (unsigned)(row - l * m);
                    e.pad = 0;
                    cand[(size_t)cidx * m + seg0 + b0 + __popc(bal & ((1u << lane) - 1u))] = e;
                }
            }
        }
    };

    int t = 0;
    int issued = ntiles < RS ? ntiles : RS;   // raw tiles issued so far (thread 0's view)
    for (; t < ntiles; ++t) {
        const int row0 = r0 + t * TM;
        const int rows = min(TM, r1 - row0);
        const int ab = t & 1;
        unsigned char* Ah = Abase + (size_t)(2 * ab) * D::AOP;
        unsigned char* Al = Ah + D::AOP;
        const bool okr = __all_sync(0xffffffffu, mbar_wait(&bar_raw[t % RS], (unsigned)((t / RS) & 1)));
        if (!okr && lane == 0) s_fail = 1;
        // centre the row and split it into the two parts of A buffer t & 1
        // (that buffer's last reader, the MMA of tile t - 2, completed before
        // the epilogue of tile t - 2 ran)
        if (okr) {
            float c[KP];
            const float* src = raw + (size_t)(t % RS) * TM * PB + (size_t)tid * PB;
#pragma unroll
            for (int q4 = 0; q4 < PB / 4; ++q4) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (tid < rows) v = reinterpret_cast<const float4*>(src)[q4];
                c[4 * q4 + 0] = v.x + s_nu[4 * q4 + 0];
                c[4 * q4 + 1] = v.y + s_nu[4 * q4 + 1];
                c[4 * q4 + 2] = v.z + s_nu[4 * q4 + 2];
                c[4 * q4 + 3] = v.w + s_nu[4 * q4 + 3];
            }
#pragma unroll
            for (int j = PB; j < KP; ++j) c[j] = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < KCH; ++q4) {
                float4 h, lo;
                h.x = tf32_hi(c[4 * q4 + 0]); lo.x = c[4 * q4 + 0] - h.x;
                h.y = tf32_hi(c[4 * q4 + 1]); lo.y = c[4 * q4 + 1] - h.y;
                h.z = tf32_hi(c[4 * q4 + 2]); lo.z = c[4 * q4 + 2] - h.z;
                h.w = tf32_hi(c[4 * q4 + 3]); lo.w = c[4 * q4 + 3] - h.w;
                *reinterpret_cast<float4*>(Ah + kop_off(tid, 4 * q4, KCH)) = h;
                *reinterpret_cast<float4*>(Al + kop_off(tid, 4 * q4, KCH)) = lo;
            }
        }
        async_proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (s_fail) break;   // uniform
        if (tid == 0) {
            // the raw stage of tile t is read: refill it with tile t + RS
            if (t + RS < ntiles) { issue(t + RS); ++issued; }
            tc_fence_after();
            const uint32_t dcol = taddr + (uint32_t)(ab * NC);
            const uint32_t ah0 = abase + (uint32_t)(2 * ab) * (uint32_t)D::AOP;
            const uint32_t al0 = ah0 + (uint32_t)D::AOP;
#pragma unroll
            for (int ks = 0; ks < KP / 8; ++ks) {
                const uint32_t o = (uint32_t)ks * 256u;
                const uint64_t ah = smem_desc(ah0 + o, 128, KCH * 128), al = smem_desc(al0 + o, 128, KCH * 128);
                const uint64_t bh = smem_desc(boff_h + o, 128, KCH * 128), bl = smem_desc(boff_l + o, 128, KCH * 128);
                mma_tf32(dcol, ah, bh, idesc, ks > 0);
                mma_tf32(dcol, al, bh, idesc, true);
                mma_tf32(dcol, ah, bl, idesc, true);
            }
            mma_commit(&bar_mma[ab]);
        }
        // the MMA of tile t runs while tile t - 1 is read back
        if (t >= 1) epilogue(t - 1);
    }
    if (!s_fail && ntiles >= 1) epilogue(ntiles - 1);
    __syncthreads();
    const int failed = s_fail;
    if (failed && tid == 0) {
        // let copies and MMAs still in flight finish before shared memory and
        // tensor memory are released (each wait bounded)
        for (int u = t; u < issued; ++u) (void)mbar_wait(&bar_raw[u % RS], (unsigned)((u / RS) & 1));
        for (int u = (t >= 2 ? t - 2 : 0); u <= t && u < ntiles; ++u)
            (void)mbar_wait(&bar_mma[u & 1], (unsigned)(u >> 1) & 1u);
        set_error(st, RTD_EINTERNAL);
    }
    below0 = warp_sum_int(below0);
    below1 = warp_sum_int(below1);
    if (lane == 0) {
        if (below0) atomicAdd(&s_below[0], below0);
        if (below1) atomicAdd(&s_below[1], below1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_dealloc(taddr, D::TCOLS);
    if (failed) return;
    if (tid < 2 && s_on[tid]) {
        const int c = 2 * l + tid;
        if (s_below[tid]) atomicAdd(&rule[c].below, s_below[tid]);
        segcnt[(size_t)c * SEG_MAX + blockIdx.x] = s_ncand[tid];
        if (s_ncand[tid]) atomicAdd(&rule[c].cand, s_ncand[tid]);
    }
}

// widths whose double-buffered operands fit a CTA's shared memory
template <int PB> constexpr bool dist_tc_width() { return PB <= 40; }

template <int PB>
void dist_tc_t(const Plan& P, cudaStream_t s) {
    if constexpr (!dist_tc_width<PB>()) {   // 48, 64: the CUDA-core pass
        dist_win_t<PB>(P, s);
        return;
    } else {
    typedef DistTC<PB> D;
    // one resident wave, at least one tile per CTA
    long long cw = (long long)D::CTAS_PER_SM * P.nsm / P.q;
    const long long rpc = P.win_rows > D::TM ? P.win_rows : D::TM;
    const long long lim = ((long long)P.m + rpc - 1) / rpc;
    if (cw > lim) cw = lim;
    if (cw > SEG_MAX) cw = SEG_MAX;
    const int cpb = (int)(cw > 0 ? cw : 1);
    dim3 grid(cpb, P.q);
    auto k = k_dist_tc<PB>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D::SMEM);
    k<<<grid, D::NTH, D::SMEM, s>>>(P.Xp, P.p, P.m, cpb, P.cs, P.ch, P.rule, (float*)P.dkeys,
                                    (long long)P.q * P.m, P.cand, P.segcnt, P.hist, P.st, P.blk_active);
    }
}

// =====================================================================
// Membership update and update-based C-step (Section 3.5).  A row whose
// membership changed contributes delta * (x - ref)(x - ref)^T (delta = +1
// entering, -1 leaving) to the chain's Gram; with the reference centre ref
// fixed per chain this is the paper's sequential update summed over the
// swaps.  When Chain.full is set the Gram of the whole new subset is taken
// instead (first step, or after a re-centring).
// =====================================================================
// =====================================================================
// FP32 form: FP64 distances of the rows in a chain's band (Section 3.4
// distances; the band decision of the selection).  M and mu of the chain
// are staged in shared memory in FP64.
// =====================================================================
constexpr int BAND_CTAS = 16;    // CTAs per chain
// One warp per CTA and one band row per lane: an FP64 warp instruction costs
// the FP64 pipe the same whether 1 or 32 lanes are active, so full warps of
// rows use it best.
constexpr int BAND_T = 32;

template <int PB>
__global__ void __launch_bounds__(BAND_T) k_band64(const Chain* __restrict__ ch, const SelRule* __restrict__ rule,
                                                   Cand* __restrict__ band_all, const float* __restrict__ Xp,
                                                   int m, int p) {
    __shared__ double sM[PB * PB];
    __shared__ double smu[PB];
    const int c = blockIdx.x;
    if (!ch[c].active) return;
    const SelRule& R = rule[c];
    if (!(R.fast || R.bandsel)) return;
    const int nb = R.band, l = c / 2;
    if (nb <= (int)blockIdx.y * BAND_T) return;
    const RowParams& rp = ch[c].rp;
    for (int e = threadIdx.x; e < PB * PB; e += BAND_T) {
        const int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? rp.M[i * PMAX + j] : 0.0;
    }
    for (int j = threadIdx.x; j < PB; j += BAND_T) smu[j] = (j < p) ? rp.mu[j] : 0.0;
    __syncthreads();
    Cand* band = band_all + (size_t)c * m + R.band_off;
    for (int i = blockIdx.y * BAND_T + threadIdx.x; i < nb; i += gridDim.y * BAND_T) {
        Cand e = band[i];
        float x[PB];
        load_row_padded<PB>(Xp + ((size_t)l * m + e.pos) * PB, x);
        // y = M (x - mu) column by column: every FMA of a column step feeds a
        // different accumulator, so the FP64 latency is overlapped
        double y[PB];
#pragma unroll
        for (int ii = 0; ii < PB; ++ii) y[ii] = 0.0;
#pragma unroll
        for (int jj = 0; jj < PB; ++jj) {
            const double cj = (double)x[jj] - smu[jj];
#pragma unroll
            for (int ii = jj; ii < PB; ++ii) y[ii] = fma(sM[ii * PB + jj], cj, y[ii]);
        }
        // d2 = sum of y^2 as a pairwise tree
#pragma unroll
        for (int ii = 0; ii < PB; ++ii) y[ii] *= y[ii];
#pragma unroll
        for (int w2 = 1; w2 < PB; w2 <<= 1)
#pragma unroll
            for (int ii = 0; ii + w2 < PB; ii += 2 * w2) y[ii] += y[ii + w2];
        const double d2 = y[0];
        e.key = (unsigned long long)__double_as_longlong(d2);   // d2 >= 0: bits order as values
        band[i] = e;
    }
}

template <int PB>
void band64_t(const Plan& P, cudaStream_t s) {
    k_band64<PB><<<dim3(2 * P.q, BAND_CTAS), BAND_T, 0, s>>>(P.ch, P.rule, P.band, P.Xp, P.m, P.p);
}

// Exclusive prefix sum over the CTA (NT threads, all must call it).
__device__ inline int cta_excl_scan(int v, int& total) {
    __shared__ int ws[NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        int c = ws[i];
        if (i < w) off += c;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return off + x - v;
}

constexpr int MEMB_U = 8;                 // rows per thread per scan chunk
constexpr int MEMB_CHUNK = NT * MEMB_U;

template <int PB, typename T>
constexpr size_t memb_smem_bytes() { return align16(gram_smem_bytes<PB, T>()) + MEMB_CHUNK * sizeof(int); }

// New membership of every row, then the Gram over the rows that changed
// (or over all members when Chain.full is set).  A chunk of MEMB_CHUNK rows
// is scanned first (membership from the key and, inside the FP32 band, from
// the FP64 decision bit), the rows to add are listed in a fixed order, then
// staged in tiles for the Gram.
template <int PB, typename T, bool TC = false>
__global__ void __launch_bounds__(NT) k_memb(const float* __restrict__ Xp, const T* __restrict__ dkeys,
                                             int p, int m, int cpb, long long qm, int fp32,
                                             const Chain* __restrict__ ch, const SelRule* __restrict__ rule,
                                             uint8_t* __restrict__ memb, int* __restrict__ swaps,
                                             double* __restrict__ partial, size_t slot_d) {
    typedef GramShape<PB, T> S;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    // the tensor-core Gram stages its rows itself: the CUDA-core tile and
    // reduction scratch are not laid out then
    constexpr size_t lead = TC ? 0 : align16(gram_smem_bytes<PB, T>());
    int* lst = reinterpret_cast<int*>(smem + lead);
    __shared__ T s_hi[PB], s_lo[PB];
    const int l = blockIdx.y;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    {   // one start per CTA (blockIdx.z)
        const int k = blockIdx.z;
        const int c = 2 * l + k;
        if (!ch[c].active) return;       // uniform over the CTA
        const int full = ch[c].full;
        const SelRule R = rule[c];
        for (int j = threadIdx.x; j < PB; j += NT) {
            if (j < p) {
                if (fp32) { s_hi[j] = (T)ch[c].rp.ref_hi[j]; s_lo[j] = (T)ch[c].rp.ref_lo[j]; }
                else { s_hi[j] = (T)ch[c].rp.ref[j]; s_lo[j] = (T)0; }
            } else { s_hi[j] = (T)0; s_lo[j] = (T)0; }
        }
        __syncthreads();
        const T* keys = dkeys + (size_t)k * qm;
        uint8_t* mb = memb + (size_t)c * m;
        typename GramPick<PB, T, TC>::type acc;
        gram_setup(acc, smem + align128(lead + MEMB_CHUNK * sizeof(int)));
        acc.init(full ? S::G : 1, !full);   // few swapped rows: one group; swapped-out rows subtract
        int nswap = 0;
        for (int c0 = r0; c0 < r1; c0 += MEMB_CHUNK) {
            uint8_t bb[MEMB_U];
            unsigned long long kk[MEMB_U];
#pragma unroll
            for (int u = 0; u < MEMB_U; ++u) {
                const int row = c0 + u * NT + threadIdx.x;
                bb[u] = (row < r1) ? mb[row - l * m] : (uint8_t)0;
                kk[u] = (row < r1) ? full_key(keys[row]) : 0ull;
            }
            unsigned incm = 0, negm = 0;
#pragma unroll
            for (int u = 0; u < MEMB_U; ++u) {
                const int row = c0 + u * NT + threadIdx.x;
                if (row >= r1) continue;
                const int t = row - l * m;
                const uint8_t b = bb[u];
                bool in;
                if (fp32) in = kk[u] < R.t_lo || (kk[u] <= R.t_hi && (b & 2));
                else in = kk[u] < R.t_key || (kk[u] == R.t_key && (unsigned)t <= R.t_pos);
                const bool old = b & 1;
                nswap += (in != old);
                const bool inc = full ? in : (in != old);
                if (inc) {
                    incm |= 1u << u;
                    if (!full && !in) negm |= 1u << u;
                }
                const uint8_t nb = in ? 1 : 0;
                if (b != nb) mb[t] = nb;
            }
            int total;
            int off = cta_excl_scan(__popc(incm), total);
#pragma unroll
            for (int u = 0; u < MEMB_U; ++u)
                if (incm >> u & 1u) lst[off++] = (c0 + u * NT + threadIdx.x) | (int)((negm >> u & 1u) << 31);
            __syncthreads();
            for (int b0 = 0; b0 < total; b0 += S::TR) {
                const int nbat = min(S::TR, total - b0);
                acc.begin();
                if (threadIdx.x < nbat) {
                    const int e = lst[b0 + threadIdx.x];
                    const int row = e & 0x7fffffff;
                    float x[PB];
                    load_row_padded<PB>(Xp + (size_t)row * PB, x);
                    T v[PB];
#pragma unroll
                    for (int j = 0; j < PB; ++j) v[j] = ((T)x[j] - s_hi[j]) - s_lo[j];
                    acc.put(tile, wt, threadIdx.x, v, p, (e < 0) ? (T)-1 : (T)1);
                }
                __syncthreads();
                acc.rows(tile, wt, nbat);
                __syncthreads();
            }
        }
        nswap = cta_sum_int(nswap);
        if (threadIdx.x == 0 && nswap) atomicAdd(swaps + c, nswap);
        size_t sl = ((size_t)l * cpb + blockIdx.x) * 2 + k;
        acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
    }
}

template <int PB, typename T, bool TC = false>
void memb_t(const Plan& P, cudaStream_t s) {
    if constexpr (!TC && tc_width<PB>() && sizeof(T) == 4) {
        if (P.tc) { memb_t<PB, T, true>(P, s); return; }
    }
    size_t sm = TC ? align128(MEMB_CHUNK * sizeof(int)) + GramPick<PB, T, TC>::extra : memb_smem_bytes<PB, T>();
    auto k = k_memb<PB, T, TC>;
    if (TC) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else set_smem(k, sm);
    dim3 grid(P.cpb, P.q, 2);
    k<<<grid, NT, sm, s>>>(P.Xp, (const T*)P.dkeys, P.p, P.m, P.cpb, (long long)P.q * P.m,
                           P.precision == RTD_FP32, P.ch, P.rule, P.memb, P.swaps, P.partial,
                           P.slot_doubles);
}
// =====================================================================
// Reweighting (Section 4 steps 8-9): rows of all blocks with
// d2(raw) <= chi2_{p,q} enter the Gram of the reweighted estimate.
// =====================================================================
template <int PB, typename T, bool TC = false>
__global__ void __launch_bounds__(NT) k_rew(const float* __restrict__ Xp, int p, int m, int cpb, int fp32,
                                            const Consts* __restrict__ cs, const RowParams* __restrict__ rp,
                                            uint8_t* __restrict__ wset, double* __restrict__ partial,
                                            size_t slot_d) {
    typedef GramShape<PB, T> S;
    constexpr int R = 1;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    T* sM = reinterpret_cast<T*>(smem + align16(gram_smem_bytes<PB, T>()));
    __shared__ T s_hi[PB], s_lo[PB];
    for (int e = threadIdx.x; e < PB * PB; e += NT) {
        int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? load_m<T>(*rp, i, j) : (T)0;
    }
    for (int j = threadIdx.x; j < PB; j += NT) {
        T hi = 0, lo = 0;
        if (j < p) load_center<T>(*rp, j, hi, lo);
        s_hi[j] = hi; s_lo[j] = lo;
    }
    __syncthreads();
    const double cut = cs->cutoff_d2;
    const T cut_lo = (T)(cut * (1.0 - BAND_EPS)), cut_hi = (T)(cut * (1.0 + BAND_EPS));
    // rows inside the FP64 band: listed, then decided one row per thread
    // (see k_final) and added to the Gram after the pass
    __shared__ int s_band[2 * NT];
    __shared__ int s_nb;
    if (threadIdx.x == 0) s_nb = 0;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    typename GramPick<PB, T, TC>::type acc;
    gram_setup(acc, smem + align128(align16(gram_smem_bytes<PB, T>()) + PB * PB * sizeof(T)));
    acc.init();
    auto band_pass = [&]() {   // all threads; s_nb <= 2 NT
        const int nb = s_nb;
        for (int k0 = 0; k0 < nb; k0 += NT) {
            const int k = k0 + threadIdx.x;
            bool in = false;
            int row = 0;
            if (k < nb) {
                row = s_band[k];
                in = d2_fp64(Xp + (size_t)row * PB, *rp, p) <= cut;
                wset[row] = in ? 2 : 0;
            }
            int tot;
            const int slot = cta_compact(in, tot);
            acc.begin();
            if (slot >= 0) {
                float x[PB];
                load_row_padded<PB>(Xp + (size_t)row * PB, x);
                T v[PB];
#pragma unroll
                for (int j = 0; j < PB; ++j) v[j] = ((T)x[j] - s_hi[j]) - s_lo[j];
                acc.put(tile, wt, slot, v, p, (T)1);
            }
            __syncthreads();
            if (tot) acc.rows(tile, wt, tot);
            __syncthreads();
        }
        if (threadIdx.x == 0) s_nb = 0;
        __syncthreads();
    };
    for (int base = r0; base < r1; base += S::TR) {
        int row = base + threadIdx.x;
        bool valid = threadIdx.x < S::TR && row < r1;
        bool in = false, inband = false;
        T c[R][PB];
        if (valid) {
            float x[PB];
            load_row_padded<PB>(Xp + (size_t)row * PB, x);
#pragma unroll
            for (int j = 0; j < PB; ++j) c[0][j] = ((T)x[j] - s_hi[j]) - s_lo[j];
            T d2[R];
            tri_d2<PB, T, R>(sM, p, c, d2);
            if (!fp32) in = (double)d2[0] <= cut;
            else if (d2[0] < cut_lo) in = true;
            else if (d2[0] > cut_hi) in = false;
            else inband = true;                       // decided in band_pass
            if (!inband) wset[row] = in ? 2 : 0;
        }
        {   // band rows listed in thread order, so that the Gram's order is fixed
            int btot;
            const int bs = cta_compact(inband, btot);
            if (bs >= 0) s_band[s_nb + bs] = row;
            __syncthreads();
            if (threadIdx.x == 0) s_nb += btot;
        }
        int tot;
        int slot = cta_compact(in, tot);
        acc.begin();
        if (slot >= 0) acc.put(tile, wt, slot, c[0], p, (T)1);
        __syncthreads();
        if (tot) acc.rows(tile, wt, tot);
        __syncthreads();
        if (s_nb >= NT) band_pass();   // at most NT - 1 + TR entries before the next tile
    }
    if (s_nb) band_pass();
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 0;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

// The reweighting Gram (steps 8-9) stays on the CUDA-core accumulator in
// every form: the reweighted fit decides the final flags, so it carries the
// FP32 form's error also when the starts and C-steps use the tensor cores.
template <int PB, typename T, bool TC = false>
void rew_t(const Plan& P, cudaStream_t s) {
    size_t sm = align16(gram_smem_bytes<PB, T>()) + PB * PB * sizeof(T);
    if (TC) sm = align128(sm) + GramPick<PB, T, TC>::extra;
    auto k = k_rew<PB, T, TC>;
    if (TC) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.precision == RTD_FP32, P.cs, P.fitrp + 0,
                           P.wset, P.partial, P.slot_doubles);
}
// =====================================================================
// Adjoint of Section 4 steps 8-10 with the reweighting set W fixed:
// mu = mean of W, Sigma = c S_W, RD_j = |M (x_j - mu)| over all rows.  The
// vector-Jacobian product for cotangents (gmu, gSigma, gld, gRD) on
// (mu, Sigma, log det Sigma, RD) follows from the chain rule through
// r = x - mu, y = M r (M = L^-1, Sigma = L L^T), RD = |y|, u = M^T y =
// Sigma^-1 r, with omega_j = gRD_j / RD_j and N = |W|:
//   the cotangents reaching mu and Sigma are
//     gmu_t = gmu - sum_j omega_j u_j,
//     G_t   = sym(gSigma) + gld Sigma^-1 - 1/2 sum_j omega_j u_j u_j^T;
//   d mu / d x_i = [W] I / N and d Sigma = a/2 sum_W (dx r^T + r dx^T),
//   a = 2 c / (N - 1), so that
//     grad_i = omega_i u_i + [W] (gmu_t / N + a G_t r_i).
//   pass 1: sum over all rows of omega (u, 1)(u, 1)^T, sum RD and |W|;
//   pass 2: the rows' gradients.
// The scalar objective w_ld log det Sigma + w_rd sum RD is the case
// gRD = w_rd, gld = w_ld, gmu = gSigma = 0 (then pass 1 weights rows by
// 1 / RD and w_rd scales its sums).  Rows with RD = 0 take the zero
// subgradient of their own term.  FP32 row arithmetic, FP64 cross-CTA sums.
// =====================================================================
template <int PB>
__device__ __forceinline__ void grad_row(const float* __restrict__ sM, const float (&c)[PB], float (&u)[PB],
                                         float& rd) {
    // row i of M gives y_i = M_i. c and then its share M_ij y_i of u_j
    float d2 = 0.f;
#pragma unroll
    for (int j = 0; j < PB; ++j) u[j] = 0.f;
#pragma unroll
    for (int i = 0; i < PB; ++i) {
        float m[PB];
        float a = 0.f;
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            m[j] = sM[i * PB + j];
            a = fmaf(m[j], c[j], a);
        }
        d2 = fmaf(a, a, d2);
#pragma unroll
        for (int j = 0; j <= i; ++j) u[j] = fmaf(m[j], a, u[j]);
    }
    rd = sqrtf(d2);
}

template <int PB>
__device__ inline void grad_load_m(const RowParams& rp, int p, float* sM, float* s_hi, float* s_lo) {
    for (int e = threadIdx.x; e < PB * PB; e += NT) {
        const int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? rp.Mf[i * PMAX + j] : 0.f;
    }
    for (int j = threadIdx.x; j < PB; j += NT) {
        s_hi[j] = (j < p) ? rp.mu_hi[j] : 0.f;
        s_lo[j] = (j < p) ? rp.mu_lo[j] : 0.f;
    }
}

template <int PB>
__global__ void __launch_bounds__(NT, 2) k_grad_gram(const float* __restrict__ X, long long n, int p, long long ld,
                                                  int vec4, const uint8_t* __restrict__ wset, int wbit,
                                                  const RowParams* __restrict__ rp, const float* __restrict__ grd,
                                                  double* __restrict__ partial, size_t slot_d) {
    typedef GramShape<PB, float> S;
    extern __shared__ __align__(16) unsigned char smem[];
    float* tile = reinterpret_cast<float*>(smem);
    float* wt = tile + S::TR * S::PE;
    __shared__ float sM[PB * PB], s_hi[PB], s_lo[PB];
    grad_load_m<PB>(*rp, p, sM, s_hi, s_lo);
    __syncthreads();
    GramAcc<PB, float> acc;
    acc.init();
    double rdsum = 0.0;
    int nw = 0;
    for (long long tb = (long long)blockIdx.x * S::TR; tb < n; tb += (long long)gridDim.x * S::TR) {
        const long long row = tb + threadIdx.x;
        const int k = (int)((n - tb) < S::TR ? (n - tb) : S::TR);
        asm volatile("" ::: "memory");   // keep M in shared memory, not hoisted into registers
        if (threadIdx.x < k) {
            float x[PB], c[PB], u[PB], rd;
            load_row_user<PB>(X + row * ld, p, vec4 != 0, x);
#pragma unroll
            for (int j = 0; j < PB; ++j) c[j] = (x[j] - s_hi[j]) - s_lo[j];
            grad_row<PB>(sM, c, u, rd);
            rdsum += (double)rd;
            nw += (wset[row] >> wbit) & 1;
            float* dst = tile + threadIdx.x * S::PE;
#pragma unroll
            for (int j = 0; j < PB; ++j) dst[j] = u[j];
            dst[PB] = 0.f; dst[PB + 1] = 0.f; dst[PB + 2] = 0.f; dst[PB + 3] = 0.f;
            dst[p] = 1.f;
            wt[threadIdx.x] = rd > 0.f ? (grd ? grd[row] : 1.f) / rd : 0.f;
        }
        __syncthreads();
        acc.rows(tile, wt, k);
        __syncthreads();
    }
    double* slot = partial + (size_t)blockIdx.x * slot_d;
    acc.store(reinterpret_cast<double*>(smem), slot);
    // sum RD and |W|, fixed-order within the CTA
    __shared__ double srd[NT / 32];
    double v = warp_sum_d(rdsum);
    const int nws = cta_sum_int(nw);
    if ((threadIdx.x & 31) == 0) srd[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += srd[w];
        slot[S::NBLK * 16] = t;
        slot[S::NBLK * 16 + 1] = (double)nws;
    }
}

template <int PB>
__global__ void __launch_bounds__(NT) k_grad_rows(const float* __restrict__ X, long long n, int p, long long ld,
                                                  int vec4, const uint8_t* __restrict__ wset, int wbit,
                                                  const RowParams* __restrict__ rp, const double* __restrict__ tot,
                                                  double c, double w_ld, double w_rd, GradCot cot,
                                                  float* __restrict__ grad) {
    typedef GramShape<PB, float> S;
    __shared__ float sM[PB * PB], sG[PB * PB], sg[PB], s_hi[PB], s_lo[PB];
    grad_load_m<PB>(*rp, p, sM, s_hi, s_lo);
    const int nb = S::NB;
    // pass 1 summed omega (u,1)(u,1)^T with omega = gRD / RD, or 1 / RD for
    // the scalar objective, whose weight w_rd then scales the sums here
    const double ws = cot.grd ? 1.0 : w_rd;
    for (int e = threadIdx.x; e < PB * PB; e += NT) {
        const int i = e / PB, j = e % PB;
        double v = 0.0;
        if (i < p && j < p) {
            v = -0.5 * ws * gram_get(tot, i, j, nb);
            if (cot.gsig) v += 0.5 * (cot.gsig[i * p + j] + cot.gsig[j * p + i]);
        }
        sG[e] = (float)v;
    }
    const double N = tot[S::NBLK * 16 + 1];
    for (int j = threadIdx.x; j < PB; j += NT)
        sg[j] = (j < p) ? (float)(((cot.gmu ? cot.gmu[j] : 0.0) - ws * gram_get(tot, j, p, nb)) / N) : 0.f;
    __syncthreads();
    const float a = (float)(2.0 * c / (N - 1.0)), wl = (float)w_ld, wr = (float)w_rd;
    for (long long row = (long long)blockIdx.x * NT + threadIdx.x; row < n; row += (long long)gridDim.x * NT) {
        asm volatile("" ::: "memory");   // keep M and G in shared memory, not hoisted into registers
        float x[PB], cc[PB], u[PB], rd;
        load_row_user<PB>(X + row * ld, p, vec4 != 0, x);
#pragma unroll
        for (int j = 0; j < PB; ++j) cc[j] = (x[j] - s_hi[j]) - s_lo[j];
        grad_row<PB>(sM, cc, u, rd);
        const float om = rd > 0.f ? (cot.grd ? cot.grd[row] : wr) / rd : 0.f;
        const bool inW = (wset[row] >> wbit) & 1;
        float* out = grad + row * p;
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            if (k >= p) break;
            float gk = om * u[k];
            if (inW) {
                float gr = 0.f;
#pragma unroll
                for (int j = 0; j < PB; ++j) gr = fmaf(sG[k * PB + j], cc[j], gr);
                gk += sg[k] + a * gr + wl * a * u[k];
            }
            out[k] = gk;
        }
    }
}

template <int PB>
void grad_t(const float* X, long long n, int p, long long ld, const uint8_t* wset, int wbit, const RowParams* rp,
            double* partial, size_t slot_d, double* tot, double c, double w_ld, double w_rd, GradCot cot, float* grad,
            int nsm, cudaStream_t s) {
    typedef GramShape<PB, float> S;
    const int vec4 = (p % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    long long tiles = (n + S::TR - 1) / S::TR;
    int g1 = (int)(tiles < 4LL * nsm ? tiles : 4LL * nsm);   // two resident CTAs per SM, two waves
    if (g1 > GRAD_SLOTS) g1 = GRAD_SLOTS;
    if (g1 < 1) g1 = 1;
    const size_t sm = gram_smem_bytes<PB, float>();
    auto k1 = k_grad_gram<PB>;
    // static M (up to 16 KB) plus the dynamic tile can pass 48 KB: always opt in
    cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k1<<<g1, NT, sm, s>>>(X, n, p, ld, vec4, wset, wbit, rp, cot.grd, partial, slot_d);
    const int nv = S::NBLK * 16 + 2;
    k_sum_slots<<<(nv + 255) / 256, 256, 0, s>>>(partial, g1, slot_d, nv, tot);
    if (grad) {
        long long blocks = (n + NT - 1) / NT;
        int g2 = (int)(blocks < 8LL * nsm ? blocks : 8LL * nsm);
        k_grad_rows<PB><<<g2, NT, 0, s>>>(X, n, p, ld, vec4, wset, wbit, rp, tot, c, w_ld, w_rd, cot, grad);
    }
}

// =====================================================================
// Final distances and flags (Section 4 step 10) for every row, original
// order; also the scoring call (Section 6).
// =====================================================================
template <int PB, typename T>
__global__ void __launch_bounds__(NT) k_final(const float* __restrict__ X, long long n, int p, long long ld,
                                              int vec4, int fp32, const RowParams* __restrict__ rp,
                                              const double* __restrict__ cutp, int decide, float* __restrict__ d2_out,
                                              uint8_t* __restrict__ flags, unsigned long long* __restrict__ count) {
    constexpr int R = DistRows<PB, T>::R;
    extern __shared__ __align__(16) unsigned char smem[];
    T* sM = reinterpret_cast<T*>(smem);
    __shared__ T s_hi[PB], s_lo[PB];
    for (int e = threadIdx.x; e < PB * PB; e += NT) {
        int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? load_m<T>(*rp, i, j) : (T)0;
    }
    for (int j = threadIdx.x; j < PB; j += NT) {
        T hi = 0, lo = 0;
        if (j < p) load_center<T>(*rp, j, hi, lo);
        s_hi[j] = hi; s_lo[j] = lo;
    }
    __syncthreads();
    const double cut = cutp ? *cutp : INFINITY;
    const T cut_lo = (T)(cut * (1.0 - BAND_EPS)), cut_hi = (T)(cut * (1.0 + BAND_EPS));
    int nflag = 0;
    // Rows inside the FP64 band are listed and recomputed together, one row
    // per thread: an FP64 instruction costs the pipe as much for one active
    // lane as for 32, so a warp must not recompute a lone band row.
    __shared__ int s_band[NT * (R + 1)];
    __shared__ int s_nb;
    if (threadIdx.x == 0) s_nb = 0;
    __syncthreads();
    auto band_pass = [&]() {
        const int nb = s_nb;
        for (int k = threadIdx.x; k < nb; k += NT) {
            const long long i = s_band[k];
            const double d = d2_fp64(X + i * ld, *rp, p);
            const bool out = d > cut;
            if (d2_out) d2_out[i] = (float)d;
            if (flags) flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nb = 0;
        __syncthreads();
    };
    // a CTA takes tiles of NT * R rows; thread t holds rows t, t + NT, ...
    // (each load instruction of a warp reads consecutive rows)
    const long long stride = (long long)gridDim.x * NT * R;
    for (long long tb = (long long)blockIdx.x * NT * R; tb < n; tb += stride) {
        T c[R][PB];
        float xs[R][PB];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long i = tb + (long long)r * NT + threadIdx.x;
            if (i < n) load_row_user<PB>(X + i * ld, p, vec4 != 0, xs[r]);
            else {
#pragma unroll
                for (int j = 0; j < PB; ++j) xs[r][j] = 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < PB; ++j) c[r][j] = ((T)xs[r][j] - s_hi[j]) - s_lo[j];
        T d2[R];
        tri_d2<PB, T, R>(sM, p, c, d2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long i = tb + (long long)r * NT + threadIdx.x;
            if (i >= n) continue;
            if (fp32 && decide && d2[r] >= cut_lo && d2[r] <= cut_hi) {
                s_band[atomicAdd(&s_nb, 1)] = (int)i;   // decided in band_pass
                continue;
            }
            // outside the FP64 band of the FP32 form, d2 > cut exactly when
            // d2 lies above the band (one FP32 compare, no FP64 operation)
            const bool out = fp32 ? (d2[r] > cut_hi) : ((double)d2[r] > cut);
            if (d2_out) d2_out[i] = (float)d2[r];
            if (flags) flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
        __syncthreads();
        if (s_nb >= NT) band_pass();   // at most NT - 1 + NT * R entries before the next tile
    }
    __syncthreads();
    if (s_nb) band_pass();
    if (count) {
        nflag = cta_sum_int(nflag);
        if (threadIdx.x == 0 && nflag) atomicAdd(count, (unsigned long long)nflag);
    }
}

// =====================================================================
// Scoring of new rows in one pass (Section 6; step 10 of Section 4 against
// a given fit): d2 (optional), the flag d2 > cutoff (optional) and the
// count.  FP32 rows; a row whose FP32 d2 lies within the FP64 band of the
// cutoff is queued per warp and recomputed in FP64 once the warp holds 32
// of them (one row per lane), so no CTA-wide barrier sits in the loop.
// Each thread keeps SR rows in flight.
// =====================================================================
template <int PB> struct ScoreRows { static constexpr int R = PB <= 4 ? 8 : (PB <= 8 ? 4 : (PB <= 24 ? 2 : 1)); };

// The fit's row parameters and the cutoff come from device memory (cutp),
// and nothing is written when the status word holds an error (a fit that
// could not be factorised).
template <int PB>
__global__ void __launch_bounds__(NT) k_score(const float* __restrict__ X, long long n, int p, long long ld,
                                              int vec4, const RowParams* __restrict__ rp,
                                              const double* __restrict__ cutp, const Status* __restrict__ st,
                                              float* __restrict__ d2_out, uint8_t* __restrict__ flags,
                                              unsigned long long* __restrict__ count) {
    constexpr int R = ScoreRows<PB>::R;
    if (st->code) return;
    const double cut = *cutp;
    constexpr int QCAP = 32 * (R + 1);
    __shared__ float sM[PB * PB];
    __shared__ float s_hi[PB], s_lo[PB];
    __shared__ long long s_q[NT / 32][QCAP];
    for (int e = threadIdx.x; e < PB * PB; e += NT) {
        const int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? rp->Mf[i * PMAX + j] : 0.f;
    }
    for (int j = threadIdx.x; j < PB; j += NT) {
        s_hi[j] = (j < p) ? rp->mu_hi[j] : 0.f;
        s_lo[j] = (j < p) ? rp->mu_lo[j] : 0.f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float cut_lo = (float)(cut * (1.0 - BAND_EPS)), cut_hi = (float)(cut * (1.0 + BAND_EPS));
    const bool decide = flags != nullptr;
    long long* q = s_q[w];
    int qn = 0;       // warp-uniform
    int nflag = 0;
    auto drain = [&](int k) {   // FP64 for the first k queued rows, one per lane
        if (lane < k) {
            const long long i = q[lane];
            const double d = d2_fp64(X + i * ld, *rp, p);
            const bool out = d > cut;
            if (d2_out) d2_out[i] = (float)d;
            flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
        __syncwarp();
        for (int e = lane; e + k < qn; e += 32) q[e] = q[e + k];
        __syncwarp();
        qn -= k;
    };
    const long long stride = (long long)gridDim.x * NT * R;
    for (long long tb = (long long)blockIdx.x * NT * R; tb < n; tb += stride) {
        float xs[R][PB];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long i = tb + (long long)r * NT + threadIdx.x;
            if (i < n) load_row_user<PB>(X + i * ld, p, vec4 != 0, xs[r]);
            else {
#pragma unroll
                for (int j = 0; j < PB; ++j) xs[r][j] = 0.f;
            }
        }
        float c[R][PB];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < PB; ++j) c[r][j] = (xs[r][j] - s_hi[j]) - s_lo[j];
        float d2[R];
        tri_d2<PB, float, R>(sM, p, c, d2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long i = tb + (long long)r * NT + threadIdx.x;
            const bool valid = i < n;
            const bool band = valid && decide && d2[r] >= cut_lo && d2[r] <= cut_hi;
            if (valid && !band) {
                const bool out = d2[r] > cut_hi;   // outside the band: exact in FP32
                if (d2_out) d2_out[i] = d2[r];
                if (decide) {
                    flags[i] = out ? 1 : 0;
                    nflag += out ? 1 : 0;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, band);
            if (band) q[qn + __popc(bal & ((1u << lane) - 1u))] = i;
            qn += __popc(bal);
        }
        __syncwarp();
        if (qn >= 32) drain(32);
    }
    __syncwarp();
    if (qn > 0) drain(qn);
    if (count && decide) {
        nflag = warp_sum_int(nflag);
        if (lane == 0 && nflag) atomicAdd(count, (unsigned long long)nflag);
    }
}

// The same pass for p = 4 with float4 rows: each thread scores G = 4
// consecutive rows, so their distances leave in one float4 store and their
// flags in one 4-byte store.  The products follow tri_d2's order (the same
// FP32 distances as k_score and the fit's passes).  A band row's FP32
// distance and flag are written first and overwritten by the warp's FP64
// pass later in the same warp.
template <int G>
__global__ void __launch_bounds__(NT, 8) k_score4(const float* __restrict__ X, long long n, long long ld,
                                               const RowParams* __restrict__ rp, const double* __restrict__ cutp,
                                               const Status* __restrict__ st, float* __restrict__ d2_out,
                                               uint8_t* __restrict__ flags, unsigned long long* __restrict__ count) {
    static_assert(G == 4, "four rows per thread: one float4 of distances, one 4-byte word of flags");
    constexpr int QCAP = 32 * (G + 1);
    __shared__ long long s_q[NT / 32][QCAP];
    if (st->code) return;
    const double cut = *cutp;
    float M[4][4], hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) M[i][j] = (j <= i) ? rp->Mf[i * PMAX + j] : 0.f;
        hi[i] = rp->mu_hi[i];
        lo[i] = rp->mu_lo[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float cut_lo = (float)(cut * (1.0 - BAND_EPS)), cut_hi = (float)(cut * (1.0 + BAND_EPS));
    const bool decide = flags != nullptr;
    long long* q = s_q[w];
    int qn = 0;       // warp-uniform
    int nflag = 0;
    auto drain = [&](int k) {   // FP64 for the first k queued rows, one per lane
        if (lane < k) {
            const long long i = q[lane];
            const double d = d2_fp64(X + i * ld, *rp, 4);
            const bool out = d > cut;
            if (d2_out) d2_out[i] = (float)d;
            flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
        __syncwarp();
        for (int e = lane; e + k < qn; e += 32) q[e] = q[e + k];
        __syncwarp();
        qn -= k;
    };
    const long long ngroups = (n + G - 1) / G;
    const long long stride = (long long)gridDim.x * NT;
    for (long long g0 = (long long)blockIdx.x * NT; g0 < ngroups; g0 += stride) {   // CTA-uniform bounds
        const long long g = g0 + threadIdx.x;
        const long long r0 = g * G;
        float4 v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {   // all loads in flight first
            const long long i = r0 + k;
            v[k] = (g < ngroups && i < n) ? __ldg(reinterpret_cast<const float4*>(X + i * ld))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float dd[G];
        bool band[G], valid[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            valid[k] = g < ngroups && r0 + k < n;
            const float c[4] = {(v[k].x - hi[0]) - lo[0], (v[k].y - hi[1]) - lo[1], (v[k].z - hi[2]) - lo[2],
                                (v[k].w - hi[3]) - lo[3]};
            float d2 = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += M[i][u] * c[u];
                d2 += acc * acc;
            }
            dd[k] = d2;
            band[k] = valid[k] && decide && d2 >= cut_lo && d2 <= cut_hi;
        }
        if (g < ngroups) {
            uint8_t f[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const bool out = dd[k] > cut_hi;   // exact outside the band; band rows are rewritten
                f[k] = out ? 1 : 0;
                nflag += (valid[k] && decide && !band[k] && out) ? 1 : 0;
            }
            if (r0 + G <= n) {
                if (d2_out) *reinterpret_cast<float4*>(d2_out + r0) = make_float4(dd[0], dd[1], dd[2], dd[3]);
                if (decide)
                    *reinterpret_cast<uchar4*>(flags + r0) = make_uchar4(f[0], f[1], f[2], f[3]);
            } else {
#pragma unroll
                for (int k = 0; k < G; ++k) {
                    if (!valid[k]) continue;
                    if (d2_out) d2_out[r0 + k] = dd[k];
                    if (decide) flags[r0 + k] = f[k];
                }
            }
        }
        __syncwarp();   // the provisional band values are stored before the FP64 pass rewrites them
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const unsigned bal = __ballot_sync(0xffffffffu, band[k]);
            if (band[k]) q[qn + __popc(bal & ((1u << lane) - 1u))] = r0 + k;
            qn += __popc(bal);
        }
        __syncwarp();
        while (qn >= 32) drain(32);
    }
    __syncwarp();
    if (qn > 0) drain(qn);
    if (count && decide) {
        nflag = warp_sum_int(nflag);
        if (lane == 0 && nflag) atomicAdd(count, (unsigned long long)nflag);
    }
}

// The same pass for p = 4 with contiguous rows (ld = 4): a persistent grid
// whose CTAs take every gridDim-th tile of SS_T rows and keep SS_S tiles in
// flight by bulk asynchronous copies into shared memory (one mbarrier per
// stage), so the bytes in flight do not depend on the number of threads.
// Rows are then scored from shared memory as in k_score (tri_d2's order,
// band rows to a per-warp FP64 queue).  Every wait is bounded: a copy that
// has not landed after ASYNC_WAIT_NS sets *err, the CTA waits (bounded) for
// its other copies and returns.
constexpr int SS_T = 1024;   // rows per tile (16 KB)
constexpr int SS_S = 4;      // tiles in flight per CTA

template <int G>
__global__ void __launch_bounds__(NT, 2) k_score_stream(const float* __restrict__ X, long long n,
                                                        const RowParams* __restrict__ rp,
                                                        const double* __restrict__ cutp, const Status* st, int* err,
                                                        float* __restrict__ d2_out, uint8_t* __restrict__ flags,
                                                        unsigned long long* __restrict__ count) {
    static_assert(G == 4, "rows of four floats");
    extern __shared__ __align__(128) unsigned char smem[];
    float4* sx = reinterpret_cast<float4*>(smem);                       // [SS_S][SS_T]
    __shared__ uint64_t bar[SS_S];
    __shared__ long long s_q[NT / 32][64];
    __shared__ int s_fail;
    if (st->code) return;
    const double cut = *cutp;
    float M[4][4], hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) M[i][j] = (j <= i) ? rp->Mf[i * PMAX + j] : 0.f;
        hi[i] = rp->mu_hi[i];
        lo[i] = rp->mu_lo[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float cut_lo = (float)(cut * (1.0 - BAND_EPS)), cut_hi = (float)(cut * (1.0 + BAND_EPS));
    const bool decide = flags != nullptr;
    const long long ntiles = (n + SS_T - 1) / SS_T;
    auto tile_bytes = [&](long long t) -> unsigned {
        const long long r = n - t * SS_T;
        return (unsigned)((r < SS_T ? r : SS_T) * 16);
    };
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int k = 0; k < SS_S; ++k) mbar_init(&bar[k], 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < SS_S; ++k) {
            const long long t = blockIdx.x + (long long)k * gridDim.x;
            if (t < ntiles) {
                mbar_expect_tx(&bar[k], tile_bytes(t));
                bulk_load(sx + (size_t)k * SS_T, X + t * SS_T * 4, tile_bytes(t), &bar[k]);
            }
        }
    }
    long long* q = s_q[w];
    int qn = 0;       // warp-uniform
    int nflag = 0;
    auto drain = [&](int k) {   // FP64 for the first k queued rows, one per lane
        if (lane < k) {
            const long long i = q[lane];
            const double d = d2_fp64(X + i * 4, *rp, 4);
            const bool out = d > cut;
            if (d2_out) d2_out[i] = (float)d;
            flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
        __syncwarp();
        for (int e = lane; e + k < qn; e += 32) q[e] = q[e + k];
        __syncwarp();
        qn -= k;
    };
    long long it = 0;
    for (;; ++it) {
        const long long t = blockIdx.x + it * gridDim.x;
        if (t >= ntiles) break;
        const int sidx = (int)(it % SS_S);
        const unsigned parity = (unsigned)((it / SS_S) & 1);
        const bool ok = mbar_wait(&bar[sidx], parity);
        if (!ok) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const float4* tx = sx + (size_t)sidx * SS_T;
        const long long r0 = t * SS_T;
#pragma unroll
        for (int k = 0; k < SS_T / NT; ++k) {
            const int j = k * NT + threadIdx.x;
            const long long i = r0 + j;
            const bool valid = i < n;
            const float4 v = valid ? tx[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float c[4] = {(v.x - hi[0]) - lo[0], (v.y - hi[1]) - lo[1], (v.z - hi[2]) - lo[2],
                                (v.w - hi[3]) - lo[3]};
            float d2 = 0.f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float acc = 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += M[a][u] * c[u];
                d2 += acc * acc;
            }
            const bool band = valid && decide && d2 >= cut_lo && d2 <= cut_hi;
            if (valid && !band) {
                const bool out = d2 > cut_hi;   // outside the band: exact in FP32
                if (d2_out) d2_out[i] = d2;
                if (decide) {
                    flags[i] = out ? 1 : 0;
                    nflag += out ? 1 : 0;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, band);
            if (bal) {
                if (band) q[qn + __popc(bal & ((1u << lane) - 1u))] = i;
                qn += __popc(bal);
                __syncwarp();
                if (qn >= 32) drain(32);
            }
        }
        __syncthreads();   // the stage is consumed
        if (threadIdx.x == 0) {
            const long long t2 = t + (long long)SS_S * gridDim.x;
            if (t2 < ntiles) {
                async_proxy_fence();
                mbar_expect_tx(&bar[sidx], tile_bytes(t2));
                bulk_load(sx + (size_t)sidx * SS_T, X + t2 * SS_T * 4, tile_bytes(t2), &bar[sidx]);
            }
        }
    }
    if (s_fail) {   // let this CTA's copies land (bounded) before leaving
        if (threadIdx.x == 0) {
            atomicExch(err, RTD_ECUDA);
            for (long long k = it; k < it + SS_S; ++k) {
                const long long t = blockIdx.x + k * gridDim.x;
                if (t >= ntiles) break;
                mbar_wait(&bar[(int)(k % SS_S)], (unsigned)((k / SS_S) & 1));
            }
        }
        return;
    }
    __syncwarp();
    if (qn > 0) drain(qn);
    if (count && decide) {
        nflag = warp_sum_int(nflag);
        if (lane == 0 && nflag) atomicAdd(count, (unsigned long long)nflag);
    }
}

template <int PB>
void score_t(const float* X, long long n, int p, long long ld, const RowParams* rp, const double* cutp,
             const Status* st, float* d2, uint8_t* fl, unsigned long long* cnt, int nsm, cudaStream_t s) {
    const int vec4 = (p % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const long long cap = (long long)nsm * 8;   // a resident wave of 256-thread CTAs
    if constexpr (PB == 4) {
        if (vec4 && p == 4 && ld == 4) {   // contiguous rows: streamed by bulk copies
            const long long ntiles = (n + SS_T - 1) / SS_T;
            const long long cs = (long long)nsm * 2;
            const int grids = (int)(ntiles < cs ? ntiles : cs);
            const size_t sm = (size_t)SS_S * SS_T * sizeof(float4);
            auto k = k_score_stream<4>;
            static bool attr_set[64] = {};   // the attribute is per device; setting it twice is harmless
            int dev = 0;
            cudaGetDevice(&dev);
            if (dev < 0 || dev >= 64 || !attr_set[dev]) {
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (dev >= 0 && dev < 64) attr_set[dev] = true;
            }
            k<<<grids > 0 ? grids : 1, NT, sm, s>>>(X, n, rp, cutp, st, const_cast<int*>(&st->code), d2, fl, cnt);
            return;
        }
        if (vec4 && p == 4 && (reinterpret_cast<uintptr_t>(d2) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(fl) & 3) == 0) {
            const long long groups = (n + 3) / 4;
            const long long ctas = (groups + NT - 1) / NT;
            const int grid4 = (int)(ctas < cap ? ctas : cap);
            k_score4<4><<<grid4 > 0 ? grid4 : 1, NT, 0, s>>>(X, n, ld, rp, cutp, st, d2, fl, cnt);
            return;
        }
    }
    constexpr int R = ScoreRows<PB>::R;
    const long long tiles = (n + (long long)NT * R - 1) / ((long long)NT * R);
    int grid = (int)(tiles < cap ? tiles : cap);
    if (grid < 1) grid = 1;
    k_score<PB><<<grid, NT, 0, s>>>(X, n, p, ld, vec4, rp, cutp, st, d2, fl, cnt);
}

template <int PB, typename T>
void final_t(const float* X, long long n, int p, long long ld, int fp32, const RowParams* rp,
                    const double* cutp, int decide, float* d2, uint8_t* fl, unsigned long long* cnt,
                    int nsm, cudaStream_t s) {
    // float4 rows only when they hold whole float4s: no read past column p
    int vec4 = (p % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    constexpr int R = DistRows<PB, T>::R;
    long long blocks = (n + (long long)NT * R - 1) / ((long long)NT * R);
    int grid = (int)(blocks < (long long)nsm * 4 ? blocks : (long long)nsm * 4);
    if (grid < 1) grid = 1;
    size_t sm = PB * PB * sizeof(T);
    auto k = k_final<PB, T>;
    set_smem(k, sm);
    k<<<grid, NT, sm, s>>>(X, n, p, ld, vec4, fp32, rp, cutp, decide, d2, fl, cnt);
}


}  // namespace rtd
