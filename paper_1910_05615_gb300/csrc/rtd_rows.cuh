// rtd_rows.cuh - row-streaming kernels of the RT-DetMCD engine (templates).
//
// Every kernel here walks the n x p rows once.  Arithmetic is FP32 (FP32
// form) or FP64 (plain form) selected by the template type T; sums that
// leave a thread are FP64.  Rows of the permuted copy Xp are padded with
// zeros to pb floats (pb a multiple of 4) so that they load as float4.
#pragma once
#include "rtd_internal.cuh"

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

template <int PB, typename T>
struct GramAcc {
    typedef GramShape<PB, T> S;
    double a64[16];
    T a32[16];
    int since, bi, bj, g;
    bool on;
    __device__ void init() {
        int t = threadIdx.x;
        g = t / S::NBLK;
        int blk = t % S::NBLK;
        on = g < S::G;
        int b = blk;
        bi = 0;
        while (b >= S::NB - bi) { b -= S::NB - bi; ++bi; }
        bj = bi + b;
#pragma unroll
        for (int e = 0; e < 16; ++e) { a64[e] = 0.0; a32[e] = (T)0; }
        since = 0;
    }
    __device__ void flush() {
#pragma unroll
        for (int e = 0; e < 16; ++e) { a64[e] += (double)a32[e]; a32[e] = (T)0; }
        since = 0;
    }
    // tile: k rows of PE values, weights wt
    __device__ void rows(const T* tile, const T* wt, int k) {
        if (!on) return;
        for (int r = g; r < k; r += S::G) {
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
    __device__ void store(double* red, double* slot) {
        flush();
        __syncthreads();
        if (on) {
            int blk = threadIdx.x % S::NBLK;
#pragma unroll
            for (int e = 0; e < 16; ++e) red[(g * S::NBLK + blk) * 16 + e] = a64[e];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < S::NBLK * 16; e += NT) {
            double s = 0.0;
            for (int gg = 0; gg < S::G; ++gg) s += red[gg * S::NBLK * 16 + e];
            slot[e] = s;
        }
        __syncthreads();
    }
};

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
__device__ inline double d2_fp64(const float* __restrict__ x, const RowParams& rp, int p) {
    double c[PMAX];
    for (int j = 0; j < p; ++j) c[j] = (double)x[j] - rp.mu[j];
    double d2 = 0.0;
    for (int i = 0; i < p; ++i) {
        double a = 0.0;
        for (int j = 0; j <= i; ++j) a += rp.M[i * PMAX + j] * c[j];
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

template <int PB, typename T, typename K>
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
    GramAcc<PB, T> acc;
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
        if (slot >= 0) {
            T* dst = tile + slot * S::PE;
#pragma unroll
            for (int j = 0; j < PB; ++j) dst[j] = w[j];
            dst[PB] = (T)0; dst[PB + 1] = (T)0; dst[PB + 2] = (T)0; dst[PB + 3] = (T)0;
            dst[p] = (T)1;
            wt[slot] = (T)1;
        }
        __syncthreads();
        acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 0;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB, typename T, typename K>
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
    GramAcc<PB, T> acc;
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
        if (slot >= 0) {
            T* dst = tile + slot * S::PE;
#pragma unroll
            for (int j = 0; j < PB; ++j) dst[j] = z[j];
            dst[PB] = (T)0; dst[PB + 1] = (T)0; dst[PB + 2] = (T)0; dst[PB + 3] = (T)0;
            dst[p] = (T)1;
            wt[slot] = xi2;
        }
        __syncthreads();
        acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 1;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB, typename T, typename K>
void start1_t(const Plan& P, cudaStream_t s) {
    size_t sm = gram_smem_bytes<PB, T>();
    auto k = k_start1<PB, T, K>;
    set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.cs, (K*)P.arenaA, P.partial, P.slot_doubles);
}
template <int PB, typename T, typename K>
void start2_t(const Plan& P, cudaStream_t s) {
    size_t sm = gram_smem_bytes<PB, T>();
    auto k = k_start2<PB, T, K>;
    set_smem(k, sm);
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

template <int PB, typename T>
__global__ void __launch_bounds__(NT, 2) k_dist(const float* __restrict__ Xp, int p, int m, int cpb,
                                                const Chain* __restrict__ ch, T* __restrict__ dkeys,
                                                long long qm, unsigned* __restrict__ hist) {
    constexpr int R = DistRows<PB, T>::R;
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
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb_dist, P.ch, (T*)P.dkeys, (long long)P.q * P.m, P.hist);
}
// =====================================================================
// Membership update and update-based C-step (Section 3.5).  A row whose
// membership changed contributes delta * (x - ref)(x - ref)^T (delta = +1
// entering, -1 leaving) to the chain's Gram; with the reference centre ref
// fixed per chain this is the paper's sequential update summed over the
// swaps.  When Chain.full is set the Gram of the whole new subset is taken
// instead (first step, or after a re-centring).
// =====================================================================
template <int PB, typename T>
__global__ void __launch_bounds__(NT) k_memb(const float* __restrict__ Xp, const T* __restrict__ dkeys,
                                             int p, int m, int cpb, long long qm, int fp32,
                                             const Chain* __restrict__ ch, const SelRule* __restrict__ rule,
                                             uint8_t* __restrict__ memb, int* __restrict__ swaps,
                                             double* __restrict__ partial, size_t slot_d) {
    typedef GramShape<PB, T> S;
    extern __shared__ __align__(16) unsigned char smem[];
    T* tile = reinterpret_cast<T*>(smem);
    T* wt = tile + S::TR * S::PE;
    __shared__ T s_hi[PB], s_lo[PB];
    const int l = blockIdx.y;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    for (int k = 0; k < 2; ++k) {
        const int c = 2 * l + k;
        if (!ch[c].active) continue;     // uniform over the CTA
        const int full = ch[c].full;
        const SelRule R = rule[c];
        __syncthreads();
        for (int j = threadIdx.x; j < PB; j += NT) {
            if (j < p) {
                if (fp32) { s_hi[j] = (T)ch[c].rp.ref_hi[j]; s_lo[j] = (T)ch[c].rp.ref_lo[j]; }
                else { s_hi[j] = (T)ch[c].rp.ref[j]; s_lo[j] = (T)0; }
            } else { s_hi[j] = (T)0; s_lo[j] = (T)0; }
        }
        __syncthreads();
        const T* keys = dkeys + (size_t)k * qm;
        uint8_t* mb = memb + (size_t)c * m;
        GramAcc<PB, T> acc;
        acc.init();
        int nswap = 0;
        for (int base = r0; base < r1; base += S::TR) {
            int row = base + threadIdx.x;
            bool valid = threadIdx.x < S::TR && row < r1;
            bool inc = false;
            T w = 0;
            if (valid) {
                int t = row - l * m;
                unsigned long long key = full_key(keys[row]);
                uint8_t b = mb[t];
                bool in;
                if (fp32) in = key < R.t_lo || (key <= R.t_hi && (b & 2));
                else in = key < R.t_key || (key == R.t_key && (unsigned)t <= R.t_pos);
                bool old = b & 1;
                nswap += (in != old);
                if (full) { inc = in; w = (T)1; }
                else { inc = in != old; w = in ? (T)1 : (T)-1; }
                mb[t] = in ? 1 : 0;
            }
            int tot;
            int slot = cta_compact(inc, tot);
            if (slot >= 0) {
                float x[PB];
                load_row_padded<PB>(Xp + (size_t)row * PB, x);
                T* dst = tile + slot * S::PE;
#pragma unroll
                for (int j = 0; j < PB; ++j) dst[j] = ((T)x[j] - s_hi[j]) - s_lo[j];
                dst[PB] = (T)0; dst[PB + 1] = (T)0; dst[PB + 2] = (T)0; dst[PB + 3] = (T)0;
                dst[p] = (T)1;
                wt[slot] = w;
            }
            __syncthreads();
            if (tot) acc.rows(tile, wt, tot);
            __syncthreads();
        }
        nswap = cta_sum_int(nswap);
        if (threadIdx.x == 0 && nswap) atomicAdd(swaps + c, nswap);
        size_t sl = ((size_t)l * cpb + blockIdx.x) * 2 + k;
        acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
    }
}

template <int PB, typename T>
void memb_t(const Plan& P, cudaStream_t s) {
    size_t sm = gram_smem_bytes<PB, T>();
    auto k = k_memb<PB, T>;
    set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, (const T*)P.dkeys, P.p, P.m, P.cpb, (long long)P.q * P.m,
                           P.precision == RTD_FP32, P.ch, P.rule, P.memb, P.swaps, P.partial,
                           P.slot_doubles);
}
// =====================================================================
// Reweighting (Section 4 steps 8-9): rows of all blocks with
// d2(raw) <= chi2_{p,q} enter the Gram of the reweighted estimate.
// =====================================================================
template <int PB, typename T>
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
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    GramAcc<PB, T> acc;
    acc.init();
    for (int base = r0; base < r1; base += S::TR) {
        int row = base + threadIdx.x;
        bool valid = threadIdx.x < S::TR && row < r1;
        bool in = false;
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
            else in = d2_fp64(x, *rp, p) <= cut;
            wset[row] = in ? 2 : 0;
        }
        int tot;
        int slot = cta_compact(in, tot);
        if (slot >= 0) {
            T* dst = tile + slot * S::PE;
#pragma unroll
            for (int j = 0; j < PB; ++j) dst[j] = c[0][j];
            dst[PB] = (T)0; dst[PB + 1] = (T)0; dst[PB + 2] = (T)0; dst[PB + 3] = (T)0;
            dst[p] = (T)1;
            wt[slot] = (T)1;
        }
        __syncthreads();
        if (tot) acc.rows(tile, wt, tot);
        __syncthreads();
    }
    size_t sl = ((size_t)blockIdx.y * cpb + blockIdx.x) * 2 + 0;
    acc.store(reinterpret_cast<double*>(smem), partial + sl * slot_d);
}

template <int PB, typename T>
void rew_t(const Plan& P, cudaStream_t s) {
    size_t sm = align16(gram_smem_bytes<PB, T>()) + PB * PB * sizeof(T);
    auto k = k_rew<PB, T>;
    set_smem(k, sm);
    dim3 grid(P.cpb, P.q);
    k<<<grid, NT, sm, s>>>(P.Xp, P.p, P.m, P.cpb, P.precision == RTD_FP32, P.cs, P.fitrp + 0,
                           P.wset, P.partial, P.slot_doubles);
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
    const long long stride = (long long)gridDim.x * NT * R;
    for (long long base = ((long long)blockIdx.x * NT + threadIdx.x) * R; base < n; base += stride) {
        T c[R][PB];
        float xs[R][PB];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (base + r < n) load_row_user<PB>(X + (base + r) * ld, p, vec4 != 0, xs[r]);
            else {
#pragma unroll
                for (int j = 0; j < PB; ++j) xs[r][j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < PB; ++j) c[r][j] = ((T)xs[r][j] - s_hi[j]) - s_lo[j];
        }
        T d2[R];
        tri_d2<PB, T, R>(sM, p, c, d2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long i = base + r;
            if (i >= n) continue;
            double d = (double)d2[r];
            if (fp32 && decide && d2[r] >= cut_lo && d2[r] <= cut_hi) d = d2_fp64(xs[r], *rp, p);
            const bool out = d > cut;
            if (d2_out) d2_out[i] = (float)d;
            if (flags) flags[i] = out ? 1 : 0;
            nflag += out ? 1 : 0;
        }
    }
    if (count) {
        nflag = cta_sum_int(nflag);
        if (threadIdx.x == 0 && nflag) atomicAdd(count, (unsigned long long)nflag);
    }
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
