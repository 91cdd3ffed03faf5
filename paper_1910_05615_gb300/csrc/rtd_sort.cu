// rtd_sort.cu - segmented radix sort, univariate MCD, GSSCM cutoffs and the
// block-wide radix select of the C-step.
#include "rtd_internal.cuh"

namespace rtd {

// =====================================================================
// Segmented LSD radix sort of equal-length segments (keys only, 8-bit
// digits, stable).  Per pass: tile histograms, per-segment exclusive scan
// in (digit, tile) order, stable scatter.  A tile is SORT_TILE_KEYS keys:
// 8 warps, ranked in rounds of 32 by warp matches and warp ballots.
// =====================================================================
constexpr int ST = 256;                 // threads
constexpr int SW = ST / 32;             // warps
constexpr int SITEMS = SORT_TILE_KEYS / ST;   // rounds per warp
constexpr int STILE = ST * SITEMS;      // keys per tile
constexpr int SKPW = STILE / SW;        // keys per warp
#ifndef RTD_SORT_MIN_CTAS
#define RTD_SORT_MIN_CTAS 4                // resident scatter CTAs per SM (32-bit keys)
#endif
// Ranking pipes: even rounds find a lane's digit peers by one warp match
// (the MIO pipe), odd rounds by eight ballots (the ALU pipe), so that neither
// pipe limits the pass alone.
constexpr int SMATCH = 2;
static_assert(SKPW <= 65536, "scatter ranks are packed in 16 bits");

template <typename K>
__global__ void __launch_bounds__(ST) k_sort_hist(const K* __restrict__ keys, long long L, int tiles,
                                                  int shift, unsigned* __restrict__ hist, unsigned* __restrict__ tot) {
    __shared__ unsigned h[256];
    const int seg = blockIdx.y, tile = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    long long t0 = (long long)tile * STILE;
    int cnt = (int)((L - t0) < STILE ? (L - t0) : STILE);
    const K* in = keys + (long long)seg * L + t0;
    for (int i = threadIdx.x; i < cnt; i += ST) atomicAdd(&h[(unsigned)(in[i] >> shift) & 255u], 1u);
    __syncthreads();
    const unsigned c = h[threadIdx.x];
    hist[((size_t)seg * 256 + threadIdx.x) * tiles + tile] = c;
    if (c) atomicAdd(&tot[(size_t)seg * 256 + threadIdx.x], c);   // the segment's digit totals
}

// Exclusive scan of one segment's 256 * tiles counters in (digit, tile)
// order, by CTAs of dpc digits each: a CTA starts at the sum of the digit
// totals before its first digit (from k_sort_hist) and scans its dpc * tiles
// counters (per-thread runs, then warp-shuffle scans of the run totals).
// It also clears its digits' totals for the next pass (tot_next).
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned* __restrict__ hist, int tiles, int dpc,
                                                    const unsigned* __restrict__ tot, unsigned* __restrict__ tot_next) {
    __shared__ unsigned wsum[32];
    __shared__ unsigned s_base;
    const int seg = blockIdx.y, d0 = blockIdx.x * dpc;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    {
        unsigned v = threadIdx.x < d0 ? tot[(size_t)seg * 256 + threadIdx.x] : 0u;   // d0 < 256 <= threads
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) s_base = 0u;
        __syncthreads();
        if (lane == 0 && v) atomicAdd(&s_base, v);
        if (threadIdx.x < dpc) tot_next[(size_t)seg * 256 + d0 + threadIdx.x] = 0u;
    }
    const long long N = (long long)dpc * tiles;
    unsigned* a = hist + ((size_t)seg * 256 + d0) * tiles;
    long long per = (N + blockDim.x - 1) / blockDim.x;
    long long b = threadIdx.x * per, e = b + per < N ? b + per : N;
    unsigned s = 0;
    for (long long i = b; i < e; ++i) s += a[i];
    unsigned x = s;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {     // exclusive scan of the warp totals
        const int nw = blockDim.x >> 5;
        const unsigned t = lane < nw ? wsum[lane] : 0u;
        unsigned z = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) wsum[lane] = z - t;
    }
    __syncthreads();
    unsigned run = s_base + wsum[w] + x - s;
    for (long long i = b; i < e; ++i) {
        unsigned v = a[i];
        a[i] = run;
        run += v;
    }
}

template <typename K>
__global__ void __launch_bounds__(ST, sizeof(K) == 4 ? RTD_SORT_MIN_CTAS : 2) k_sort_scatter(const K* __restrict__ in, K* __restrict__ out, long long L,
                                                     int tiles, int shift, const unsigned* __restrict__ offs) {
    __shared__ unsigned wcnt[SW][256];
    __shared__ unsigned goff[256];
    __shared__ unsigned tstart[256];
    __shared__ K stage[STILE];
    const int seg = blockIdx.y, tile = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < SW * 256; e += ST) (&wcnt[0][0])[e] = 0u;
    goff[threadIdx.x] = offs[((size_t)seg * 256 + threadIdx.x) * tiles + tile];
    __syncthreads();
    long long t0 = (long long)tile * STILE;
    int cnt = (int)((L - t0) < STILE ? (L - t0) : STILE);
    const K* src = in + (long long)seg * L + t0;
    K key[SITEMS];
    unsigned rank[(SITEMS + 1) / 2];   // two 16-bit ranks per word (a rank is below SKPW)
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SITEMS; ++r) {     // all loads in flight before the ranking
        int idx = w * SKPW + r * 32 + lane;
        key[r] = idx < cnt ? __ldg(src + idx) : (K)0;
    }
#pragma unroll
    for (int r = 0; r < SITEMS; ++r) {
        int idx = w * SKPW + r * 32 + lane;
        bool valid = idx < cnt;
        unsigned d = (unsigned)(key[r] >> shift) & 255u;
        // lanes holding the same digit: a warp match (a lane past the end
        // matches no other), or the intersection over the digit's 8 bits of
        // the ballots that agree with this lane's bit
        unsigned peers;
        if (r % SMATCH == 0) {
            peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
        } else {
            peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = 1u << lane;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bb : ~bb;
            }
        }
        // the group's first lane reads and advances the warp's digit count
        const int leader = __ffs(peers) - 1;
        unsigned base = (valid && lane == leader) ? wcnt[w][d] : 0u;
        base = __shfl_sync(0xffffffffu, base, leader);
        const unsigned rk = base + __popc(peers & lt);
        rank[r >> 1] = (r & 1) ? (rank[r >> 1] | (rk << 16)) : rk;
        if (valid && lane == leader) wcnt[w][d] = base + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: exclusive prefix over warps, and the tile's digit total
        unsigned run = 0;
        for (int ww = 0; ww < SW; ++ww) {
            unsigned c = wcnt[ww][threadIdx.x];
            wcnt[ww][threadIdx.x] = run;
            run += c;
        }
        tstart[threadIdx.x] = run;
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the 256 digit totals
        unsigned v[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { v[k] = tstart[threadIdx.x * 8 + k]; sum += v[k]; }
        unsigned inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        unsigned ex = inc - sum;
#pragma unroll
        for (int k = 0; k < 8; ++k) { tstart[threadIdx.x * 8 + k] = ex; ex += v[k]; }
    }
    __syncthreads();
    {   // fold the digit starts into the per-warp bases and the global offsets,
        // so that staging and writing each read one digit-indexed word per key
        const unsigned ts = tstart[threadIdx.x];
#pragma unroll
        for (int ww = 0; ww < SW; ++ww) wcnt[ww][threadIdx.x] += ts;
        goff[threadIdx.x] -= ts;
    }
    __syncthreads();
    // tile-local sorted order in shared memory
#pragma unroll
    for (int r = 0; r < SITEMS; ++r) {
        int idx = w * SKPW + r * 32 + lane;
        if (idx < cnt) {
            unsigned d = (unsigned)(key[r] >> shift) & 255u;
            stage[wcnt[w][d] + ((rank[r >> 1] >> ((r & 1) * 16)) & 0xffffu)] = key[r];
        }
    }
    __syncthreads();
    // consecutive threads write consecutive keys of one digit run
    K* dst = out + (long long)seg * L;
    for (int i = threadIdx.x; i < cnt; i += ST) {
        K k = stage[i];
        unsigned d = (unsigned)(k >> shift) & 255u;
        unsigned pos = goff[d] + (unsigned)i;
        if (pos < (unsigned)L) dst[pos] = k;
    }
}

template <typename K>
static void sort_t(const Plan& P, K* keys, K* tmp, int nseg, long long L, cudaStream_t s) {
    int tiles = (int)((L + STILE - 1) / STILE);
    dim3 grid(tiles, nseg);
    const int passes = (int)sizeof(K);
    K* a = keys;
    K* b = tmp;
    // digit totals of the passes, in two alternating buffers (the scan of
    // one pass clears the other for the next)
    unsigned* tot[2] = {P.sort_tot, P.sort_tot + (size_t)nseg * 256};
    cudaMemsetAsync(P.sort_tot, 0, 2 * (size_t)nseg * 256 * sizeof(unsigned), s);
    int dpc = 1;   // digits per scan CTA: about 4096 counters each
    while (dpc < 256 && (long long)dpc * tiles < 4096) dpc <<= 1;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = 8 * ps;
        k_sort_hist<K><<<grid, ST, 0, s>>>(a, L, tiles, shift, P.sort_hist, tot[ps & 1]);
        k_sort_scan<<<dim3(256 / dpc, nseg), 1024, 0, s>>>(P.sort_hist, tiles, dpc, tot[ps & 1], tot[(ps + 1) & 1]);
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
// Univariate reweighted MCD of sorted segments (Section 3.1): coverage
// h~ = [L/2] + 1; the contiguous h~-window of minimum variance (first on
// ties) gives mu0 and c(h~/L) var; the reweighting keeps
// (x - mu0)^2 / s0^2 <= chi2_{1,q}, a contiguous range of the sorted values.
// All sums are FP64 over the values shifted by the middle order statistic c;
// q_j = h S2_j - S1_j^2 = h (h-1) var_j orders the windows.
//
// Windows are grouped in ranges of UW starts.  Every window of a range
// contains the core of sorted positions shared by all of them, and for any
// subset C of a window  sum_window (x - mean)^2 >= (|C| - 1) var(C), so
// q_j >= h q_C / |C| bounds the whole range from below (C taken on the chunk
// grid so that it comes from chunk prefix sums).  Ranges whose bound exceeds
// the exact q of some window are skipped; the others are evaluated window by
// window.  Kernels:
//   U1 chunk sums (UC positions)        U2 exclusive scan of chunk sums
//   U3 per range: bound and q at its first window
//   U4 per segment: least first-window q     U5 per range: exact windows
//   U6 per segment: argmin, reweighting bounds by a 256-ary search, sums.
// out[seg] = (mu, s2, mu_raw, s2_raw); NaN marks a degenerate segment.
// =====================================================================
constexpr int UT = 256;              // threads
constexpr int UC = 256;              // chunk of positions (prefix anchors)
constexpr int UW = 256;              // range of window starts

// float or double value of a sort key as a double; for 32-bit keys the
// conversion is done with integer operations (exact for every float).
__device__ inline double kval(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;    // float bits
    uint32_t e = (u >> 23) & 0xffu, mant = u & 0x7fffffu;
    unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (e == 0u) {
        if (mant == 0u) return __longlong_as_double((long long)sign);
        return (double)__uint_as_float(u);                       // subnormal: rare
    }
    if (e == 0xffu) return (double)__uint_as_float(u);            // inf / nan
    unsigned long long b = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)mant << 29);
    return __longlong_as_double((long long)b);
}
__device__ inline double kval(unsigned long long k) { return key2d(k); }

template <typename K>
__device__ inline double uval(const K* s, long long i) { return kval(s[i]); }

struct D2 { double a, b; };

// Shifted value d = s_i - c and d^2 of one sorted element: exact pair for
// 32-bit keys (float values), double otherwise.
struct FF2 { FF a, b; };
__device__ __forceinline__ FF2 ff_elem(uint32_t k, float c) {
    const float v = key2f(k);
    const FF d = ff_two_sum(v, -c);
    return FF2{d, ff_sq(d)};
}
__device__ __forceinline__ FF2 ff_zero2() { return FF2{FF{0.f, 0.f}, FF{0.f, 0.f}}; }
__device__ __forceinline__ FF2 ff_add2(FF2 x, FF2 y) { return FF2{ff_add(x.a, y.a), ff_add(x.b, y.b)}; }
__device__ __forceinline__ FF2 ff_warp_sum2(FF2 v) {
    for (int o = 16; o > 0; o >>= 1) v = ff_add2(v, FF2{ff_shfl_xor(v.a, o), ff_shfl_xor(v.b, o)});
    return v;
}

__device__ inline D2 warp_sum2(D2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.a += __shfl_xor_sync(0xffffffffu, v.a, o);
        v.b += __shfl_xor_sync(0xffffffffu, v.b, o);
    }
    return v;
}

__device__ inline D2 cta_sum2(D2 v) {
    __shared__ double wa[UT / 32], wb[UT / 32];
    v = warp_sum2(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { wa[w] = v.a; wb[w] = v.b; }
    __syncthreads();
    D2 t{0.0, 0.0};
    for (int k = 0; k < UT / 32; ++k) { t.a += wa[k]; t.b += wb[k]; }
    __syncthreads();
    return t;
}

// Middle order statistic c of a segment, in the arithmetic of the sums.
__device__ inline float ucenter(const uint32_t* s, long long L) { return key2f(s[L / 2]); }
__device__ inline double ucenter(const unsigned long long* s, long long L) { return key2d(s[L / 2]); }

// Sum of (s_i - c, (s_i - c)^2) over [a, b) by one warp / by the CTA
// (pairs for 32-bit keys, FP64 for 64-bit keys), returned as doubles.
// Each lane sums its elements' high parts by TwoSum and adds the low parts
// and the TwoSum errors in plain FP32 (a lane holds a few elements, so the
// error sum keeps the pair's precision); the lanes' pairs are then combined
// by the float-float warp reduction.
__device__ inline FF2 ff_range_sum(const uint32_t* s, float c, long long a, long long b) {
    float sa = 0.f, ea = 0.f, sb = 0.f, eb = 0.f;
    for (long long i = a + (threadIdx.x & 31); i < b; i += 32) {
        const FF2 x = ff_elem(s[i], c);
        const FF ta = ff_two_sum(sa, x.a.hi), tb = ff_two_sum(sb, x.b.hi);
        sa = ta.hi;
        ea += ta.lo + x.a.lo;
        sb = tb.hi;
        eb += tb.lo + x.b.lo;
    }
    return ff_warp_sum2(FF2{ff_two_sum(sa, ea), ff_two_sum(sb, eb)});
}
__device__ inline D2 warp_range_sum(const uint32_t* s, float c, long long a, long long b) {
    const FF2 acc = ff_range_sum(s, c, a, b);
    return D2{ff_d(acc.a), ff_d(acc.b)};
}
__device__ inline D2 warp_range_sum(const unsigned long long* s, double c, long long a, long long b) {
    D2 acc{0.0, 0.0};
    for (long long i = a + (threadIdx.x & 31); i < b; i += 32) {
        double d = key2d(s[i]) - c;
        acc.a += d;
        acc.b = fma(d, d, acc.b);
    }
    return warp_sum2(acc);
}
template <typename K, typename C>
__device__ inline D2 cta_range_sum(const K* s, C c, long long a, long long b) {
    __shared__ double wa[UT / 32], wb[UT / 32];
    // each warp sums a contiguous share, then the warp totals in fixed order
    const long long n = b - a, per = (n + (UT / 32) - 1) / (UT / 32);
    const int w = threadIdx.x >> 5;
    const long long wa0 = a + w * per, wb0 = (wa0 + per < b) ? wa0 + per : b;
    D2 t = (wa0 < wb0) ? warp_range_sum(s, c, wa0, wb0) : D2{0.0, 0.0};
    if ((threadIdx.x & 31) == 0) { wa[w] = t.a; wb[w] = t.b; }
    __syncthreads();
    D2 r{0.0, 0.0};
    for (int k = 0; k < UT / 32; ++k) { r.a += wa[k]; r.b += wb[k]; }
    __syncthreads();
    return r;
}

// U1: warp per chunk.
template <typename K>
__global__ void __launch_bounds__(UT) k_uni_chunks(const K* __restrict__ sorted, long long L, int nch,
                                                   double* __restrict__ csum) {
    const int seg = blockIdx.y;
    const int ch = blockIdx.x * (UT / 32) + (threadIdx.x >> 5);
    if (ch >= nch) return;
    const K* s = sorted + (long long)seg * L;
    const auto c = ucenter(s, L);
    long long a = (long long)ch * UC, b = a + UC < L ? a + UC : L;
    double* o = csum + ((size_t)seg * nch + ch) * 2;
    if constexpr (sizeof(K) == 4) {
        // the pair components as they are; k_uni_prefix converts them with one
        // thread per chunk (an FP64 instruction costs the pipe the same for
        // one lane as for 32, so a warp per chunk should not convert)
        const FF2 t = ff_range_sum(s, c, a, b);
        if ((threadIdx.x & 31) == 0)
            *reinterpret_cast<float4*>(o) = make_float4(t.a.hi, t.a.lo, t.b.hi, t.b.lo);
    } else {
        D2 t = warp_range_sum(s, c, a, b);
        if ((threadIdx.x & 31) == 0) {
            o[0] = t.a;
            o[1] = t.b;
        }
    }
}

// U2: cpre[seg][k] = sum of chunks < k, k = 0..nch (one CTA per segment):
// per-thread runs, then a shuffle scan of the run totals (fixed order).
__global__ void __launch_bounds__(1024) k_uni_prefix(double* __restrict__ csum, int nch, int pairs,
                                                     double* __restrict__ cpre, int* __restrict__ count) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0;   // candidate list of k_uni_ub
    __shared__ double wa[32], wb[32];
    const int seg = blockIdx.x;
    double* c = csum + (size_t)seg * nch * 2;
    double* o = cpre + (size_t)seg * (nch + 1) * 2;
    const int per = (nch + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = b0 + per < nch ? b0 + per : nch;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (pairs) {   // chunk sums stored as compensated pairs: to doubles, in place
        for (int k = b0; k < b1; ++k) {
            const float4 v = *reinterpret_cast<const float4*>(c + 2 * k);
            c[2 * k] = ff_d(FF{v.x, v.y});
            c[2 * k + 1] = ff_d(FF{v.z, v.w});
        }
    }
    double sa = 0.0, sb = 0.0;
    for (int k = b0; k < b1; ++k) { sa += c[2 * k]; sb += c[2 * k + 1]; }
    double xa = sa, xb = sb;
    for (int off = 1; off < 32; off <<= 1) {
        const double ya = __shfl_up_sync(0xffffffffu, xa, off), yb = __shfl_up_sync(0xffffffffu, xb, off);
        if (lane >= off) { xa += ya; xb += yb; }
    }
    if (lane == 31) { wa[w] = xa; wb[w] = xb; }
    __syncthreads();
    if (w == 0) {
        double ya = wa[lane], yb = wb[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const double za = __shfl_up_sync(0xffffffffu, ya, off), zb = __shfl_up_sync(0xffffffffu, yb, off);
            if (lane >= off) { ya += za; yb += zb; }
        }
        wa[lane] = ya;   // inclusive warp totals
        wb[lane] = yb;
    }
    __syncthreads();
    double ra = (w ? wa[w - 1] : 0.0) + xa - sa, rb = (w ? wb[w - 1] : 0.0) + xb - sb;
    for (int k = b0; k < b1; ++k) {
        o[2 * k] = ra;
        o[2 * k + 1] = rb;
        ra += c[2 * k];
        rb += c[2 * k + 1];
    }
    if (threadIdx.x == 1023) { o[2 * nch] = wa[31]; o[2 * nch + 1] = wb[31]; }
}

// Running sums up to position x: anchor plus a partial chunk.
template <typename K, typename C>
__device__ inline D2 warp_prefix(const K* s, C c, const double* cpre, long long x) {
    long long k = x / UC;
    D2 t = warp_range_sum(s, c, k * UC, x);
    return D2{cpre[2 * k] + t.a, cpre[2 * k + 1] + t.b};
}
template <typename K, typename C>
__device__ inline D2 cta_prefix(const K* s, C c, const double* cpre, long long x) {
    long long k = x / UC;
    D2 t = cta_range_sum(s, c, k * UC, x);
    return D2{cpre[2 * k] + t.a, cpre[2 * k + 1] + t.b};
}

// U3 body for range r (warp-uniform inputs, the partial sums pb at a + h).
__device__ inline void uni_bound_out(const double* cpre, long long L, int r, int nwr, D2 pb, double* o) {
    const long long h = L / 2 + 1, nwin = L - h + 1;
    const double hd = (double)h;
    const long long a = (long long)r * UW, b = a + UW < nwin ? a + UW : nwin;
    const long long lo = ((b - 1 + UC - 1) / UC) * UC, hi = ((a + h) / UC) * UC;
    double lb = -INFINITY;
    if (hi - lo >= 2) {
        double n = (double)(hi - lo);
        double s1 = cpre[2 * (hi / UC)] - cpre[2 * (lo / UC)];
        double s2 = cpre[2 * (hi / UC) + 1] - cpre[2 * (lo / UC) + 1];
        lb = hd * (n * s2 - s1 * s1) / n;
    }
    double S1 = pb.a - cpre[2 * (a / UC)], S2 = pb.b - cpre[2 * (a / UC) + 1];
    o[0] = lb;
    o[1] = hd * S2 - S1 * S1;
}

// U3, 32-bit keys: warp per range, the compensated sums of the partial chunk
// at a + h only (stored as pairs); k_uni_ub finishes the range with one
// thread per range, so that the FP64 arithmetic takes one instruction per 32
// ranges (an FP64 instruction costs the pipe the same for one lane as for 32).
__global__ void __launch_bounds__(UT) k_uni_part32(const uint32_t* __restrict__ sorted, long long L, int nwr,
                                                   float4* __restrict__ part) {
    const int seg = blockIdx.y;
    const int r = blockIdx.x * (UT / 32) + (threadIdx.x >> 5);
    if (r >= nwr) return;
    const uint32_t* s = sorted + (long long)seg * L;
    const long long x = (long long)r * UW + L / 2 + 1;
    const long long k = x / UC;
    const FF2 t = ff_range_sum(s, ucenter(s, L), k * UC, x);
    if ((threadIdx.x & 31) == 0) part[(size_t)seg * nwr + r] = make_float4(t.a.hi, t.a.lo, t.b.hi, t.b.lo);
}

// U3, warp per range: lower bound over the range and q at its first window.
template <typename K>
__global__ void __launch_bounds__(UT) k_uni_bound(const K* __restrict__ sorted, long long L, int nch, int nwr,
                                                  const double* __restrict__ cpre_all, double* __restrict__ wb) {
    const int seg = blockIdx.y;
    const int r = blockIdx.x * (UT / 32) + (threadIdx.x >> 5);
    if (r >= nwr) return;
    const K* s = sorted + (long long)seg * L;
    const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
    const long long h = L / 2 + 1, nwin = L - h + 1;
    const double hd = (double)h;
    const auto c = ucenter(s, L);
    const long long a = (long long)r * UW, b = a + UW < nwin ? a + UW : nwin;
    // aligned core [lo, hi) inside [b - 1, a + h)
    const long long lo = ((b - 1 + UC - 1) / UC) * UC, hi = ((a + h) / UC) * UC;
    double lb = -INFINITY;
    if (hi - lo >= 2) {
        double n = (double)(hi - lo);
        double s1 = cpre[2 * (hi / UC)] - cpre[2 * (lo / UC)];
        double s2 = cpre[2 * (hi / UC) + 1] - cpre[2 * (lo / UC) + 1];
        lb = hd * (n * s2 - s1 * s1) / n;
    }
    D2 pb = warp_prefix(s, c, cpre, a + h);
    double S1 = pb.a - cpre[2 * (a / UC)], S2 = pb.b - cpre[2 * (a / UC) + 1];
    double qa = hd * S2 - S1 * S1;
    if ((threadIdx.x & 31) == 0) {
        double* o = wb + ((size_t)seg * nwr + r) * 2;
        o[0] = lb;
        o[1] = qa;
    }
}

// U3 finish, 32-bit keys, for segments of many ranges: the range bounds from
// the partial-chunk pairs, one thread per range over several CTAs per
// segment (the FP64 arithmetic of one segment's ranges would otherwise run
// on one SM's FP64 pipe).
__global__ void __launch_bounds__(UT) k_uni_ubfin(double* __restrict__ wb, int nwr, const float4* __restrict__ part,
                                                  const double* __restrict__ cpre_all, long long L, int nch) {
    const int seg = blockIdx.y;
    const int r = blockIdx.x * UT + threadIdx.x;
    if (r >= nwr) return;
    const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
    const float4 v = part[(size_t)seg * nwr + r];
    const long long k = ((long long)r * UW + L / 2 + 1) / UC;
    const D2 pb{cpre[2 * k] + ff_d(FF{v.x, v.y}), cpre[2 * k + 1] + ff_d(FF{v.z, v.w})};
    uni_bound_out(cpre, L, r, nwr, pb, wb + ((size_t)seg * nwr + r) * 2);
}

// U4: least first-window q of each segment.
// Also lists the ranges the bound does not exclude (any order: each range's
// result has its own slot) and marks the excluded ones in wres, so that the
// exact pass runs over the list only.
// With part (32-bit keys) the range bounds are first finished here from the
// partial-chunk pairs, one thread per range.
__global__ void __launch_bounds__(UT) k_uni_ub(double* __restrict__ wb, int nwr, double* __restrict__ ub,
                                               double* __restrict__ wres, int2* __restrict__ list,
                                               int* __restrict__ count, const float4* __restrict__ part,
                                               const double* __restrict__ cpre_all, long long L, int nch) {
    __shared__ double red[UT / 32];
    __shared__ double s_ub;
    const int seg = blockIdx.x;
    if (part) {
        const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
        for (int r = threadIdx.x; r < nwr; r += UT) {
            const float4 v = part[(size_t)seg * nwr + r];
            const long long k = ((long long)r * UW + L / 2 + 1) / UC;
            const D2 pb{cpre[2 * k] + ff_d(FF{v.x, v.y}), cpre[2 * k + 1] + ff_d(FF{v.z, v.w})};
            uni_bound_out(cpre, L, r, nwr, pb, wb + ((size_t)seg * nwr + r) * 2);
        }
        __syncthreads();
    }
    double m = INFINITY;
    for (int r = threadIdx.x; r < nwr; r += UT) m = fmin(m, wb[((size_t)seg * nwr + r) * 2 + 1]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = INFINITY;
        for (int k = 0; k < UT / 32; ++k) v = fmin(v, red[k]);
        ub[seg] = v;
        s_ub = v;
    }
    __syncthreads();
    const double lim = s_ub * (1.0 + 1e-12);
    for (int r0 = 0; r0 < nwr; r0 += UT) {
        const int r = r0 + threadIdx.x;
        const bool live = r < nwr && !(wb[((size_t)seg * nwr + r) * 2] > lim);
        if (r < nwr && !live) {
            double* o = wres + ((size_t)seg * nwr + r) * 3;
            o[0] = INFINITY; o[1] = -1.0; o[2] = 0.0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, live);
        if (bal) {
            const int lane = threadIdx.x & 31;
            int base = 0;
            if (lane == 0) base = atomicAdd(count, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (live) list[base + __popc(bal & ((1u << lane) - 1u))] = make_int2(seg, r);
        }
    }
}

// U5: exact windows of the ranges the bound does not exclude.  For the
// window at j of a range starting at a,
//   S_k(j) = S_k(a) + sum_{a <= i < j} (d_{i+h}^k - d_i^k),  k = 1, 2,
// so one exclusive scan over the range gives every window.  32-bit keys:
// compensated FP32 pairs throughout.
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_from_d(double d) {
    const float hi = (float)d;
    return FF{hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ bool ff_less(FF a, FF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

__global__ void __launch_bounds__(UT) k_uni_eval_ff(const uint32_t* __restrict__ sorted, long long L, int nch,
                                                    int nwr, const double* __restrict__ cpre_all,
                                                    const int2* __restrict__ list, const int* __restrict__ count,
                                                    double* __restrict__ wres) {
    __shared__ FF sw[UT / 32][2];
    __shared__ FF sbase[2];
    __shared__ FF sq[UT / 32], ss[UT / 32];
    __shared__ long long sj[UT / 32];
    const int nlist = *count;
    for (int it = blockIdx.x; it < nlist; it += gridDim.x) {   // uniform over the CTA
        const int seg = list[it].x, r = list[it].y;
        double* o = wres + ((size_t)seg * nwr + r) * 3;
        const uint32_t* s = sorted + (long long)seg * L;
        const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
        const long long h = L / 2 + 1, nwin = L - h + 1;
        const float hf = (float)h;                       // exact: h < 2^24
        const float c = ucenter(s, L);
        const long long a = (long long)r * UW, b = a + UW < nwin ? a + UW : nwin;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (w == 0) {   // sums of the range's first window (a is on the chunk grid)
            D2 pb = warp_prefix(s, c, cpre, a + h);
            if (lane == 0) {
                sbase[0] = ff_from_d(pb.a - cpre[2 * (a / UC)]);
                sbase[1] = ff_from_d(pb.b - cpre[2 * (a / UC) + 1]);
            }
        }
        const long long j = a + threadIdx.x;
        FF e1{0.f, 0.f}, e2{0.f, 0.f};
        if (j < b && j + h < L) {
            const FF2 A = ff_elem(s[j], c), B = ff_elem(s[j + h], c);
            e1 = ff_add(B.a, ff_neg(A.a));
            e2 = ff_add(B.b, ff_neg(A.b));
        }
        // inclusive warp scan, then exclusive within the CTA
        FF x1 = e1, x2 = e2;
        for (int off = 1; off < 32; off <<= 1) {
            const FF y1 = ff_shfl_up(x1, off), y2 = ff_shfl_up(x2, off);
            if (lane >= off) { x1 = ff_add(x1, y1); x2 = ff_add(x2, y2); }
        }
        if (lane == 31) { sw[w][0] = x1; sw[w][1] = x2; }
        __syncthreads();
        if (threadIdx.x == 0) {   // exclusive prefix of the 8 warp totals, base folded in (fixed order)
            FF p1 = sbase[0], p2 = sbase[1];
            for (int k = 0; k < UT / 32; ++k) {
                const FF q1 = sw[k][0], q2 = sw[k][1];
                sw[k][0] = p1;
                sw[k][1] = p2;
                p1 = ff_add(p1, q1);
                p2 = ff_add(p2, q2);
            }
        }
        __syncthreads();
        // S_k(j) = warp prefix + exclusive lane prefix
        const FF S1 = ff_add(sw[w][0], ff_add(x1, ff_neg(e1)));
        const FF S2 = ff_add(sw[w][1], ff_add(x2, ff_neg(e2)));
        FF q{INFINITY, 0.f}, s1{0.f, 0.f};
        long long bj = -1;
        if (j < b) {
            q = ff_add(ff_mul_f(S2, hf), ff_neg(ff_sq(S1)));
            s1 = S1;
            bj = j;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const FF oq = ff_shfl_xor(q, off), os = ff_shfl_xor(s1, off);
            const long long oj = __shfl_xor_sync(0xffffffffu, bj, off);
            if (oj >= 0 && (bj < 0 || ff_less(oq, q) || (oq.hi == q.hi && oq.lo == q.lo && oj < bj))) {
                q = oq; bj = oj; s1 = os;
            }
        }
        if (lane == 0) { sq[w] = q; sj[w] = bj; ss[w] = s1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            FF bq{INFINITY, 0.f}, bs{0.f, 0.f};
            long long jj = -1;
            for (int k = 0; k < UT / 32; ++k)
                if (sj[k] >= 0 && (jj < 0 || ff_less(sq[k], bq) || (sq[k].hi == bq.hi && sq[k].lo == bq.lo && sj[k] < jj))) {
                    bq = sq[k]; jj = sj[k]; bs = ss[k];
                }
            o[0] = jj >= 0 ? ff_d(bq) : INFINITY;
            o[1] = (double)jj;
            o[2] = ff_d(bs);
        }
        __syncthreads();   // shared state is reused by the next listed range
    }
}

template <typename K>
__global__ void __launch_bounds__(UT) k_uni_eval(const K* __restrict__ sorted, long long L, int nch, int nwr,
                                                 const double* __restrict__ cpre_all, const double* __restrict__ wb,
                                                 const double* __restrict__ ub, double* __restrict__ wres) {
    __shared__ double sw[UT / 32][4];
    __shared__ double sq[UT / 32], ss[UT / 32];
    __shared__ long long sj[UT / 32];
    __shared__ double s_pb[2];
    const int seg = blockIdx.y, r = blockIdx.x;
    double* o = wres + ((size_t)seg * nwr + r) * 3;
    const double lb = wb[((size_t)seg * nwr + r) * 2];
    if (lb > ub[seg] * (1.0 + 1e-12)) {
        if (threadIdx.x == 0) { o[0] = INFINITY; o[1] = -1.0; o[2] = 0.0; }
        return;
    }
    const K* s = sorted + (long long)seg * L;
    const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
    const long long h = L / 2 + 1, nwin = L - h + 1;
    const double hd = (double)h;
    const auto c = ucenter(s, L);
    const long long a = (long long)r * UW, b = a + UW < nwin ? a + UW : nwin;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {
        D2 pb = warp_prefix(s, c, cpre, a + h);
        if (lane == 0) { s_pb[0] = pb.a; s_pb[1] = pb.b; }
    }
    const long long j = a + threadIdx.x;
    double da = 0.0, db = 0.0;
    if (j < b) {
        da = uval(s, j) - c;
        if (j + h < L) db = uval(s, j + h) - c;
    }
    // exclusive scans of (da, da^2, db, db^2) over the range
    double x0 = da, x1 = da * da, x2 = db, x3 = db * db;
    for (int off = 1; off < 32; off <<= 1) {
        double y0 = __shfl_up_sync(0xffffffffu, x0, off), y1 = __shfl_up_sync(0xffffffffu, x1, off);
        double y2 = __shfl_up_sync(0xffffffffu, x2, off), y3 = __shfl_up_sync(0xffffffffu, x3, off);
        if (lane >= off) { x0 += y0; x1 += y1; x2 += y2; x3 += y3; }
    }
    if (lane == 31) { sw[w][0] = x0; sw[w][1] = x1; sw[w][2] = x2; sw[w][3] = x3; }
    __syncthreads();
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
    for (int k = 0; k < w; ++k) { p0 += sw[k][0]; p1 += sw[k][1]; p2 += sw[k][2]; p3 += sw[k][3]; }
    const double A1 = cpre[2 * (a / UC)] + p0 + x0 - da, A2 = cpre[2 * (a / UC) + 1] + p1 + x1 - da * da;
    const double B1 = s_pb[0] + p2 + x2 - db, B2 = s_pb[1] + p3 + x3 - db * db;
    double q = INFINITY, s1 = 0.0;
    long long bj = -1;
    if (j < b) {
        s1 = B1 - A1;
        q = hd * (B2 - A2) - s1 * s1;
        bj = j;
    }
    for (int off = 16; off > 0; off >>= 1) {
        double oq = __shfl_xor_sync(0xffffffffu, q, off);
        double os = __shfl_xor_sync(0xffffffffu, s1, off);
        long long oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (oj >= 0 && (bj < 0 || oq < q || (oq == q && oj < bj))) { q = oq; bj = oj; s1 = os; }
    }
    if (lane == 0) { sq[w] = q; sj[w] = bj; ss[w] = s1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bq = INFINITY, bs = 0.0;
        long long jj = -1;
        for (int k = 0; k < UT / 32; ++k)
            if (sj[k] >= 0 && (jj < 0 || sq[k] < bq || (sq[k] == bq && sj[k] < jj))) { bq = sq[k]; jj = sj[k]; bs = ss[k]; }
        o[0] = bq;
        o[1] = (double)jj;
        o[2] = bs;
    }
}

// First index in [lo, hi) where the monotone (false ... true) predicate
// holds, hi if none; 256-ary search by the whole CTA.
template <typename Pred>
__device__ inline long long cta_first_true(long long lo, long long hi, Pred pred) {
    __shared__ int s_t;
    while (true) {
        if (hi - lo <= UT) {
            if (threadIdx.x == 0) s_t = UT;
            __syncthreads();
            long long x = lo + threadIdx.x;
            if (x < hi && pred(x)) atomicMin(&s_t, (int)threadIdx.x);
            __syncthreads();
            long long r = (s_t < UT) ? lo + s_t : hi;
            __syncthreads();
            return r;
        }
        long long step = (hi - lo + UT - 1) / UT;
        if (threadIdx.x == 0) s_t = UT;
        __syncthreads();
        long long x = lo + (threadIdx.x + 1) * step - 1;
        if (x > hi - 1) x = hi - 1;
        if (pred(x)) atomicMin(&s_t, (int)threadIdx.x);
        __syncthreads();
        int t = s_t;
        __syncthreads();
        if (t == UT) return hi;
        long long nlo = lo + (long long)t * step;
        long long nhi = lo + ((long long)t + 1) * step;
        if (nhi > hi) nhi = hi;
        lo = nlo;
        hi = nhi;     // pred(nhi - 1) holds: the answer lies in [lo, hi)
    }
}

// U6
template <typename K>
__global__ void __launch_bounds__(UT) k_uni_finish_seg(const K* __restrict__ sorted, long long L, int nch, int nwr,
                                                       const double* __restrict__ cpre_all,
                                                       const double* __restrict__ wres,
                                                       const Consts* __restrict__ cs, int which_c1,
                                                       double* __restrict__ out) {
    __shared__ double sv[UT], ss[UT];
    __shared__ long long sj[UT];
    __shared__ double s_q, s_s1;
    __shared__ long long s_j;
    const int seg = blockIdx.x;
    const K* s = sorted + (long long)seg * L;
    const double* cpre = cpre_all + (size_t)seg * (nch + 1) * 2;
    const long long h = L / 2 + 1;
    const double hd = (double)h;
    const auto cc = ucenter(s, L);
    const double c = (double)cc;
    double best = INFINITY, bs1 = 0.0;
    long long bj = -1;
    for (int r = threadIdx.x; r < nwr; r += UT) {
        const double* x = wres + ((size_t)seg * nwr + r) * 3;
        long long jj = (long long)x[1];
        if (jj >= 0 && (bj < 0 || x[0] < best || (x[0] == best && jj < bj))) { best = x[0]; bj = jj; bs1 = x[2]; }
    }
    // least (q, j) over the CTA: warp butterflies, then the warp results in
    // order (the same total order as one pass over all threads)
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off), os = __shfl_xor_sync(0xffffffffu, bs1, off);
        const long long oj = __shfl_xor_sync(0xffffffffu, bj, off);
        if (oj >= 0 && (bj < 0 || ob < best || (ob == best && oj < bj))) { best = ob; bj = oj; bs1 = os; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; ss[threadIdx.x >> 5] = bs1; sj[threadIdx.x >> 5] = bj; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = INFINITY, bsum = 0.0;
        long long jj = -1;
        for (int t = 0; t < UT / 32; ++t)
            if (sj[t] >= 0 && (jj < 0 || sv[t] < b || (sv[t] == b && sj[t] < jj))) { b = sv[t]; jj = sj[t]; bsum = ss[t]; }
        s_q = b; s_j = jj; s_s1 = bsum;
    }
    __syncthreads();
    double* o = out + 4 * (size_t)seg;
    if (s_j < 0) { if (threadIdx.x == 0) { o[0] = o[1] = o[2] = o[3] = NAN; } return; }
    const double c1 = which_c1 ? cs->c1_m : cs->c1_n;
    const double mu0 = c + s_s1 / hd;
    // a window of equal values has variance exactly 0 (degenerate column)
    const bool flat = uval(s, s_j) == uval(s, s_j + h - 1);
    const double s20 = flat ? 0.0 : c1 * (s_q / (hd * (hd - 1.0)));
    if (!(s20 > 0.0) || !isfinite(s20)) {
        if (threadIdx.x == 0) { o[0] = NAN; o[1] = NAN; o[2] = mu0; o[3] = s20; }
        return;
    }
    const double cut2 = cs->uni_cut2;
    auto keep = [&](long long i) { double d = uval(s, i) - mu0; return d * d / s20 <= cut2; };
    long long m0 = cta_first_true(0, L, [&](long long i) { return uval(s, i) >= mu0; });
    long long wlo = cta_first_true(0, m0, keep);
    long long whi = cta_first_true(m0, L, [&](long long i) { return !keep(i); });
    long long nw = whi - wlo;
    if (nw < 2) {
        if (threadIdx.x == 0) { o[0] = NAN; o[1] = NAN; o[2] = mu0; o[3] = s20; }
        return;
    }
    D2 Pa = cta_prefix(s, cc, cpre, wlo);
    D2 Pb = cta_prefix(s, cc, cpre, whi);
    if (threadIdx.x == 0) {
        double T1 = Pb.a - Pa.a, T2 = Pb.b - Pa.b;
        o[0] = c + T1 / (double)nw;
        o[1] = cs->crew1 * (T2 - T1 * T1 / (double)nw) / (double)(nw - 1);
        o[2] = mu0;
        o[3] = s20;
    }
}

struct UniDims { int nch, nwr; };
inline UniDims uni_dims(long long L) {
    const long long h = L / 2 + 1, nwin = L - h + 1;
    return UniDims{(int)((L + UC - 1) / UC), (int)((nwin + UW - 1) / UW)};
}

template <typename K>
static int unimcd_t(const Plan& P, const K* keys, int nseg, long long L, int which_c1, double* out,
                    cudaStream_t s) {
    const UniDims D = uni_dims(L);
    double* csum = P.uscratch;
    double* cpre = csum + (size_t)nseg * D.nch * 2;
    double* wb = cpre + (size_t)nseg * (D.nch + 1) * 2;
    double* ub = wb + (size_t)nseg * D.nwr * 2;
    double* wres = ub + nseg;
    int* count = reinterpret_cast<int*>(wres + (size_t)nseg * D.nwr * 3);
    int2* list = reinterpret_cast<int2*>(wres + (size_t)nseg * D.nwr * 3 + 1);
    const int wpb = UT / 32;
    k_uni_chunks<K><<<dim3((D.nch + wpb - 1) / wpb, nseg), UT, 0, s>>>(keys, L, D.nch, csum);
    k_uni_prefix<<<nseg, 1024, 0, s>>>(csum, D.nch, sizeof(K) == 4 ? 1 : 0, cpre, count);
    float4* part = nullptr;
    if (sizeof(K) == 4) {
        // 16-byte aligned after the list (one spare double in the scratch size)
        const uintptr_t pa = reinterpret_cast<uintptr_t>(list + (size_t)nseg * D.nwr);
        part = reinterpret_cast<float4*>((pa + 15) & ~(uintptr_t)15);
        k_uni_part32<<<dim3((D.nwr + wpb - 1) / wpb, nseg), UT, 0, s>>>((const uint32_t*)keys, L, D.nwr, part);
    } else {
        k_uni_bound<K><<<dim3((D.nwr + wpb - 1) / wpb, nseg), UT, 0, s>>>(keys, L, D.nch, D.nwr, cpre, wb);
    }
    int launches = 6;
    if (part && D.nwr > UT) {
        k_uni_ubfin<<<dim3((D.nwr + UT - 1) / UT, nseg), UT, 0, s>>>(wb, D.nwr, part, cpre, L, D.nch);
        part = nullptr;
        ++launches;
    }
    k_uni_ub<<<nseg, UT, 0, s>>>(wb, D.nwr, ub, wres, list, count, part, cpre, L, D.nch);
    if (sizeof(K) == 4) {
        long long g = (long long)nseg * D.nwr;
        if (g > 4LL * P.nsm) g = 4LL * P.nsm;
        k_uni_eval_ff<<<(int)g, UT, 0, s>>>((const uint32_t*)keys, L, D.nch, D.nwr, cpre, list, count, wres);
    } else
        k_uni_eval<K><<<dim3(D.nwr, nseg), UT, 0, s>>>(keys, L, D.nch, D.nwr, cpre, wb, ub, wres);
    k_uni_finish_seg<K><<<nseg, UT, 0, s>>>(keys, L, D.nch, D.nwr, cpre, wres, P.cs, which_c1, out);
    return launches;
}

int launch_unimcd(const Plan& P, const void* keys, int key_bytes, int nseg, long long L, int which_c1,
                  double* out, cudaStream_t s) {
    if (key_bytes == 8) return unimcd_t<unsigned long long>(P, (const unsigned long long*)keys, nseg, L, which_c1, out, s);
    return unimcd_t<uint32_t>(P, (const uint32_t*)keys, nseg, L, which_c1, out, s);
}

size_t unimcd_scratch_doubles(int nseg, long long L) {
    const UniDims D = uni_dims(L);
    return (size_t)nseg * (2 * (size_t)D.nch + 2 * ((size_t)D.nch + 1) + 2 * (size_t)D.nwr + 1 + 3 * (size_t)D.nwr +
                           (size_t)D.nwr + 2 * (size_t)D.nwr) + 2;   // + candidate list (int2), its count,
                                                                     // partial-chunk pairs (float4)
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

// First index in [lo, hi) where the monotone (false ... true) predicate
// holds, hi if none; 32-ary search by one warp.
template <typename Pred>
__device__ inline long long warp_first_true(long long lo, long long hi, Pred pred) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        long long step = (hi - lo + 31) / 32;
        long long x = lo + (lane + 1) * step - 1;
        if (x > hi - 1) x = hi - 1;
        unsigned b = __ballot_sync(0xffffffffu, pred(x));
        if (!b) return hi;
        int t = __ffs(b) - 1;
        long long nlo = lo + (long long)t * step, nhi = lo + ((long long)t + 1) * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    long long x = lo + lane;
    unsigned b = __ballot_sync(0xffffffffu, x < hi && pred(x));
    return b ? lo + (__ffs(b) - 1) : hi;
}

// k-th smallest (1-based) of |v_i - m3| over the sorted v = r^(2/3): the
// runs Lt = m3 - v[s0-1-t] and Rt = v[s0+t] - m3 are both ascending.
template <typename K>
__device__ double kth_absdev(const K* s, long long L, long long s0, double m3, long long k) {
    long long a = s0, b = L - s0;
    auto Lv = [&](long long t) { return m3 - r23(s, s0 - 1 - t); };
    auto Rv = [&](long long t) { return r23(s, s0 + t) - m3; };
    long long lo = k - b > 0 ? k - b : 0, hi = k < a ? k : a;
    // i = number taken from the left run: first i where R_{k-i-1} > L_i fails
    long long i = warp_first_true(lo, hi, [&](long long ii) {
        long long jj = k - ii;
        return !(ii < a && jj > 0 && Rv(jj - 1) > Lv(ii));
    });
    long long j = k - i;
    double x = (i > 0) ? Lv(i - 1) : -INFINITY;
    double y = (j > 0) ? Rv(j - 1) : -INFINITY;
    return x > y ? x : y;
}

// One warp per block.
template <typename K>
__global__ void __launch_bounds__(32) k_gsscm(const K* __restrict__ rs, int q, long long m, double* __restrict__ AB) {
    const int l = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
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
    long long s0 = warp_first_true(0, m, [&](long long i) { return r23(s, i) >= m3; });
    double mad;
    if (m & 1) mad = kth_absdev(s, m, s0, m3, (m + 1) / 2);
    else mad = 0.5 * (kth_absdev(s, m, s0, m3, m / 2) + kth_absdev(s, m, s0, m3, m / 2 + 1));
    const double phi075 = 0.6744897501960817, madc = 1.4826;
    if ((threadIdx.x & 31) == 0) {
        AB[2 * l] = A;
        AB[2 * l + 1] = pow(m3 + phi075 * madc * mad, 1.5);
    }
}

void launch_gsscm(const Plan& P, const void* rkeys, cudaStream_t s) {
    // one warp per CTA: the searches are chains of FP64 powers, and warps
    // sharing an SM would share its FP64 pipe
    int th = 32, bl = P.q;
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
    if (!ch[c].active || rule[c].fast) return;
    if (threadIdx.x == 0 && rule[c].win) rule[c].acc_miss += 1;
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
// of a candidate list.  Long lists are narrowed by 8-bit radix passes on
// the composite (key, position) until at most SEL_SMALL entries share the
// prefix; those are sorted in shared memory (bitonic network).  Positions
// make every entry unique, so ties between equal distances go to the lower
// position.
// =====================================================================
constexpr int SEL_T = 1024;
constexpr int SEL_SMALL = 2048;
typedef unsigned __int128 u128;

__device__ inline u128 comp(const Cand& e) { return ((u128)e.key << 32) | (u128)e.pos; }

// Ascending sort of a[0, n) (n <= SEL_SMALL) in shared memory; a must hold
// the next power of two of entries.
__device__ inline void cta_bitonic(Cand* a, int n) {
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = n + threadIdx.x; i < N; i += blockDim.x) {
        a[i].key = ~0ull; a[i].pos = 0xffffffffu; a[i].pad = 1;
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const Cand x = a[i], y = a[ixj];
                    const bool up = (i & k) == 0;
                    if ((comp(x) > comp(y)) == up) { a[i] = y; a[ixj] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// buf: SEL_SMALL entries of shared memory.
__device__ Cand cta_select_rank(const Cand* list, int C, int r, int key_bits, Cand* buf, Status* st) {
    __shared__ unsigned hcnt[256];
    __shared__ unsigned wtot[8];
    __shared__ unsigned long long s_and, s_or;
    __shared__ int s_digit, s_r, s_cnt, s_n;
    (void)key_bits;
    const int lane = threadIdx.x & 31;
    Cand bad;
    bad.key = ~0ull; bad.pos = 0xffffffffu; bad.pad = 1;
    if (r < 1 || r > C) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return bad;
    }
    if (threadIdx.x == 0) { s_and = ~0ull; s_or = 0ull; s_n = 0; }
    __syncthreads();
    const int total = 96;                 // composite value: key (64) : position (32)
    int pbits = 0;
    u128 prefix = 0;
    int cnt = C, rr = r;
    if (C > SEL_SMALL) {
        // key bits shared by every entry need no pass
        unsigned long long a = ~0ull, o = 0ull;
        for (int i = threadIdx.x; i < C; i += blockDim.x) { unsigned long long k = list[i].key; a &= k; o |= k; }
        for (int d = 16; d > 0; d >>= 1) {
            a &= __shfl_xor_sync(0xffffffffu, a, d);
            o |= __shfl_xor_sync(0xffffffffu, o, d);
        }
        if (lane == 0) { atomicAnd(&s_and, a); atomicOr(&s_or, o); }
        __syncthreads();
        const unsigned long long diff = s_and ^ s_or;
        const int top = diff ? 32 + 63 - __clzll((long long)diff) : 31;   // highest differing bit
        pbits = total - 1 - top;
        prefix = (((u128)s_and << 32) >> (top + 1));
        while (cnt > SEL_SMALL && pbits < total) {
            const int width = (total - pbits) < 8 ? (total - pbits) : 8;
            const int shift = total - pbits - width;
            for (int i = threadIdx.x; i < 256; i += blockDim.x) hcnt[i] = 0u;
            __syncthreads();
            for (int base = 0; base < C; base += blockDim.x) {
                const int i = base + threadIdx.x;
                unsigned tag = 0x1000u + lane;
                unsigned dg = 0;
                if (i < C) {
                    const u128 v = comp(list[i]);
                    if (pbits == 0 || (v >> (total - pbits)) == prefix) {
                        dg = (unsigned)(v >> shift) & ((1u << width) - 1u);
                        tag = dg;
                    }
                }
                const unsigned peers = __match_any_sync(0xffffffffu, tag);
                if (tag < 0x1000u && (__ffs(peers) - 1) == lane) atomicAdd(&hcnt[dg], (unsigned)__popc(peers));
            }
            if (threadIdx.x == 0) s_digit = -1;
            __syncthreads();
            // digit of rank rr: parallel inclusive scan of the 256 counts
            unsigned v = 0, x = 0;
            if (threadIdx.x < 256) {
                v = hcnt[threadIdx.x];
                x = v;
                for (int o2 = 1; o2 < 32; o2 <<= 1) {
                    unsigned y = __shfl_up_sync(0xffffffffu, x, o2);
                    if (lane >= o2) x += y;
                }
                if (lane == 31) wtot[threadIdx.x >> 5] = x;
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                unsigned off = 0;
                for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += wtot[w];
                const unsigned incl = off + x, excl = incl - v;
                if (v && excl < (unsigned)rr && (unsigned)rr <= incl) {
                    s_digit = threadIdx.x; s_r = rr - (int)excl; s_cnt = (int)v;
                }
            }
            __syncthreads();
            if (s_digit < 0) {
                if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
                __syncthreads();
                return bad;
            }
            prefix = (prefix << width) | (u128)(unsigned)s_digit;
            pbits += width;
            rr = s_r;
            cnt = s_cnt;
            __syncthreads();
        }
    }
    for (int base = 0; base < C; base += blockDim.x) {
        const int i = base + threadIdx.x;
        bool m = false;
        Cand e;
        if (i < C) {
            e = list[i];
            const u128 v = comp(e);
            m = (pbits == 0 || (v >> (total - pbits)) == prefix);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, m);
        int wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(&s_n, __popc(bal));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (m) {
            const int slot = wb + __popc(bal & ((1u << lane) - 1u));
            if (slot < SEL_SMALL) buf[slot] = e;
        }
    }
    __syncthreads();
    const int n = s_n;
    if (n > SEL_SMALL || rr < 1 || rr > n) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        __syncthreads();
        return bad;
    }
    cta_bitonic(buf, n);
    const Cand res = buf[rr - 1];
    __syncthreads();
    return res;
}

// FP32 form, histogram path: threshold t = the r-th smallest candidate; the
// band rows [t (1 - eps), t (1 + eps)] go to the chain's band list (their
// FP64 distances: k_band64; their ranking: k_select_band).  `below` rows
// lie under the candidate range.
__device__ void hist_path_band(SelRule& R, const Cand* cand, int C, int below, int hb, Cand* band_all_c,
                               Cand* buf, Status* st) {
    __shared__ int s_nlo, s_nb;
    const int r = hb - below;
    if (r < 1 || r > C) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    Cand t = cta_select_rank(cand, C, r, 32, buf, st);
    if (t.pad) return;     // error already recorded
    const float tf = __uint_as_float((unsigned)t.key);
    const unsigned long long t_lo = __float_as_uint(tf * (float)(1.0 - BAND_EPS));
    const unsigned long long t_hi = __float_as_uint(tf * (float)(1.0 + BAND_EPS));
    if (threadIdx.x == 0) { s_nlo = 0; s_nb = 0; }
    __syncthreads();
    int nlo = 0;
    const int lane = threadIdx.x & 31;
    for (int base = 0; base < C; base += blockDim.x) {
        int i = base + threadIdx.x;
        bool inb = false;
        Cand e;
        if (i < C) {
            e = cand[i];
            if (e.key < t_lo) ++nlo;
            else inb = e.key <= t_hi;
        }
        unsigned bal = __ballot_sync(0xffffffffu, inb);
        int wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(&s_nb, __popc(bal));
        wb = __shfl_sync(0xffffffffu, wb, 0);
        if (inb) band_all_c[wb + __popc(bal & ((1u << lane) - 1u))] = e;
    }
    nlo = warp_sum_int(nlo);
    if (lane == 0 && nlo) atomicAdd(&s_nlo, nlo);
    __syncthreads();
    if (threadIdx.x == 0) {
        R.t_lo = t_lo;
        R.t_hi = t_hi;
        R.band = s_nb;
        R.nlo = below + s_nlo;
        R.band_off = 0;
        R.bandsel = 1;
        R.t_prev2 = R.have_t ? R.t_prev : 0.f;
        R.t_prev = tf;
        R.have_t = 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(SEL_T) k_select_finish(const Chain* __restrict__ ch, SelRule* __restrict__ rule,
                                                          const Cand* __restrict__ cand_all, Cand* __restrict__ band_all,
                                                          int m, int hb, int fp32, Status* st) {
    __shared__ Cand buf[SEL_SMALL];
    const int c = blockIdx.x;
    if (!ch[c].active || rule[c].fast) return;
    SelRule& R = rule[c];
    const int C = R.cand < m ? R.cand : m;
    const Cand* cand = cand_all + (size_t)c * m;
    if (fp32) {
        hist_path_band(R, cand, C, R.below, hb, band_all + (size_t)c * m, buf, st);
        return;
    }
    const int r = hb - R.below;
    if (r < 1 || r > C) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    Cand t = cta_select_rank(cand, C, r, 64, buf, st);
    if (t.pad) return;     // error already recorded
    if (threadIdx.x == 0) { R.t_key = t.key; R.t_pos = t.pos; }
}

// The histogram path run by one CTA over one chain's FP32 keys (a window
// that missed): top-digit histogram, bucket of rank h_b, compaction of the
// bucket widened by the band, then the band as above.
__device__ void cta_hist_path(SelRule& R, const float* keys, int m, int hb, Cand* cand, Cand* band_all_c,
                              Cand* buf, unsigned* h, Status* st) {
    __shared__ int s_bin, s_below, s_cand;
    __shared__ unsigned wt[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = threadIdx.x; b < HIST_BINS; b += blockDim.x) h[b] = 0u;
    if (threadIdx.x == 0) { s_bin = -1; s_below = 0; s_cand = 0; }
    __syncthreads();
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool v = i < m;
        const float d = v ? keys[i] : 0.f;
        const unsigned bin = coarse_key(d) >> (32 - HIST_BITS);
        const unsigned tag = v ? bin : (0x80000000u | lane);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        if (v && (__ffs(peers) - 1) == lane) atomicAdd(h + bin, (unsigned)__popc(peers));
    }
    __syncthreads();
    // bin of rank hb: per-thread runs of HIST_BINS / blockDim bins, then a scan of the run totals
    const int per = HIST_BINS / blockDim.x;
    unsigned run = 0;
    for (int k = 0; k < per; ++k) run += h[threadIdx.x * per + k];
    unsigned x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    unsigned off = 0;
    for (int k = 0; k < w; ++k) off += wt[k];
    unsigned cum = off + x - run;
    for (int k = 0; k < per; ++k) {
        const unsigned v = h[threadIdx.x * per + k];
        if (cum < (unsigned)hb && (unsigned)hb <= cum + v) s_bin = threadIdx.x * per + k;
        cum += v;
    }
    (void)nw;
    __syncthreads();
    const int b = s_bin;
    if (b < 0) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    const unsigned lo_bits = (unsigned)b << (32 - HIST_BITS);
    const unsigned hi_bits = lo_bits | ((1u << (32 - HIST_BITS)) - 1u);
    const unsigned lo = __float_as_uint(__uint_as_float(lo_bits) * (float)(1.0 - BAND_EPS));
    const unsigned hi = __float_as_uint(__uint_as_float(hi_bits) * (float)(1.0 + BAND_EPS));
    int below = 0;
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const bool v = i < m;
        const float d = v ? keys[i] : 0.f;
        const unsigned ck = coarse_key(d);
        below += (v && ck < lo) ? 1 : 0;
        const bool take = v && ck >= lo && ck <= hi;
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        if (bal) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(&s_cand, __popc(bal));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (take) {
                Cand e;
                e.key = (unsigned long long)__float_as_uint(d);
                e.pos = (unsigned)i;
                e.pad = 0;
                cand[b0 + __popc(bal & ((1u << lane) - 1u))] = e;
            }
        }
    }
    below = warp_sum_int(below);
    if (lane == 0 && below) atomicAdd(&s_below, below);
    __syncthreads();
    const int C = s_cand < m ? s_cand : m;
    if (threadIdx.x == 0) { R.cand = C; R.below = s_below; R.lo = lo; R.hi = hi; R.acc_miss += 1; }
    hist_path_band(R, cand, C, s_below, hb, band_all_c, buf, st);
}

void launch_select_finish(const Plan& P, cudaStream_t s) {
    k_select_finish<<<2 * P.q, SEL_T, 0, s>>>(P.ch, P.rule, P.cand, P.band, P.m, P.hb,
                                              P.precision == RTD_FP32, P.st);
}

// Band ranking of the FP32 form (both paths): the band rows whose FP64
// (d2, position) is at most that of rank h_b - (rows below the band) get the
// decision bit (bit 1) the membership pass reads.
constexpr int BANDSEL_T = 256;   // band lists are short: fewer threads, cheaper barriers

__global__ void __launch_bounds__(BANDSEL_T) k_select_band(const Chain* __restrict__ ch, const SelRule* __restrict__ rule,
                                                        const Cand* __restrict__ band_all,
                                                        uint8_t* __restrict__ memb_all, int m, int hb, Status* st) {
    __shared__ Cand buf[SEL_SMALL];
    const int c = blockIdx.x;
    if (!ch[c].active) return;
    const SelRule& R = rule[c];
    if (!(R.fast || R.bandsel)) return;
    const int nb = R.band, r2 = hb - R.nlo;
    if (threadIdx.x == 0) const_cast<SelRule&>(R).acc_band += nb;
    if (r2 < 1 || r2 > nb) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return;
    }
    const Cand* band = band_all + (size_t)c * m + R.band_off;
    uint8_t* mb = memb_all + (size_t)c * m;
    if (nb <= 2 * BANDSEL_T) {
        // short band: each row counts the rows ordered before it and takes
        // its own decision (rank < r2), no sort
        for (int i = threadIdx.x; i < nb; i += blockDim.x) buf[i] = band[i];
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const u128 v = comp(buf[i]);
            int rank = 0;
            for (int j = 0; j < nb; ++j) rank += comp(buf[j]) < v ? 1 : 0;
            const unsigned pos = buf[i].pos;
            mb[pos] = (uint8_t)((mb[pos] & 1) | (rank < r2 ? 2 : 0));
        }
        return;
    }
    Cand tb = cta_select_rank(band, nb, r2, 64, buf, st);
    if (tb.pad) return;
    const u128 tv = comp(tb);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const Cand e = band[i];
        mb[e.pos] = (uint8_t)((mb[e.pos] & 1) | (comp(e) <= tv ? 2 : 0));
    }
}

// =====================================================================
// Window path of the FP32 form in one launch (from the second C-step on),
// gridDim.y CTAs per chain.  Every CTA finds the window bin b that holds rank
// r = h_b - (rows below the window).  The FP64 range is that bin widened
// by the band, [lo_b (1 - eps), hi_b (1 + eps)]: a row whose FP32 key lies
// below it is in, above it out (the FP32 error is under eps), and a row
// inside it is decided by its FP64 distance.  The rule needs no FP32
// threshold: every CTA counts its share of the candidates below the range
// and appends (FP64 d2, position) of those inside it to the chain's list;
// the chain's last CTA ranks the list (ties to the lower position) and sets
// the decision bits the membership pass reads.  A window that misses (the
// rank or the range outside it) is resolved by the last CTA with the
// histogram path over the block's keys and the same FP64 ranking.
// =====================================================================
constexpr int SF_T = 256;       // threads per CTA
constexpr int SF_CTAS = 8;      // CTAs per chain unless tuned

// FP64 d2 = |M (x - mu)|^2 of one padded row; M (lower triangular, row
// stride PB) and mu in shared memory.  Output rows are taken 16 at a time,
// column by column within a block, so that every FMA of a column step feeds
// a different accumulator and the accumulators stay in registers.
template <int PB>
__device__ __forceinline__ double row_d2_fp64(const float* __restrict__ xrow, const double* sM, const double* smu) {
    constexpr int IB = 16;
    asm volatile("" ::: "memory");   // keep M in shared memory, not hoisted into registers across rows
    float x[PB];
#pragma unroll
    for (int q4 = 0; q4 < PB / 4; ++q4) {
        const float4 v = reinterpret_cast<const float4*>(xrow)[q4];
        x[4 * q4] = v.x; x[4 * q4 + 1] = v.y; x[4 * q4 + 2] = v.z; x[4 * q4 + 3] = v.w;
    }
    double d2 = 0.0;
#pragma unroll
    for (int i0 = 0; i0 < PB; i0 += IB) {
        double y[IB];
#pragma unroll
        for (int ii = 0; ii < IB; ++ii) y[ii] = 0.0;
#pragma unroll
        for (int jj = 0; jj < PB && jj < i0 + IB; ++jj) {
            const double cj = (double)x[jj] - smu[jj];
#pragma unroll
            for (int ii = 0; ii < IB; ++ii)
                if (i0 + ii < PB && i0 + ii >= jj) y[ii] = fma(sM[(i0 + ii) * PB + jj], cj, y[ii]);
        }
#pragma unroll
        for (int ii = 0; ii < IB; ++ii) y[ii] *= y[ii];
#pragma unroll
        for (int w2 = 1; w2 < IB; w2 <<= 1)
#pragma unroll
            for (int ii = 0; ii + w2 < IB; ii += 2 * w2) y[ii] += y[ii + w2];
        d2 += y[0];
    }
    return d2;
}

template <int PB>
__device__ void stage_m64(const RowParams& rp, int p, double* sM, double* smu) {
    for (int e = threadIdx.x; e < PB * PB; e += blockDim.x) {
        const int i = e / PB, j = e % PB;
        sM[e] = (i < p && j <= i) ? rp.M[i * PMAX + j] : 0.0;
    }
    for (int j = threadIdx.x; j < PB; j += blockDim.x) smu[j] = (j < p) ? rp.mu[j] : 0.0;
}

// Rank the list (key = FP64 d2 bits, pos) and set decision bit 1 of the
// first r1 entries in (d2, pos) order, clearing it on the others; returns
// the d2 of entry r1 (rank r1 - 1) to every thread.  buf: SEL_SMALL entries.
__device__ double rank_and_mark(const Cand* list, int n, int r1, uint8_t* mb, Cand* buf, Status* st) {
    __shared__ double s_t;
    if (r1 < 1 || r1 > n) {
        if (threadIdx.x == 0) set_error(st, RTD_EINTERNAL);
        return 0.0;
    }
    if (n <= SEL_SMALL) {
        // other CTAs wrote the list in this launch: read it from L2
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(list) + i);
            buf[i].key = v.x;
            buf[i].pos = (unsigned)(v.y & 0xffffffffull);
            buf[i].pad = (unsigned)(v.y >> 32);
        }
        __syncthreads();
        if (n <= 512) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const u128 v = comp(buf[i]);
                int rank = 0;
                for (int j = 0; j < n; ++j) rank += comp(buf[j]) < v ? 1 : 0;
                const unsigned pos = buf[i].pos;
                mb[pos] = (uint8_t)((mb[pos] & 1) | (rank < r1 ? 2 : 0));
                if (rank == r1 - 1) s_t = __longlong_as_double((long long)buf[i].key);
            }
        } else {
            cta_bitonic(buf, n);
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const unsigned pos = buf[i].pos;
                mb[pos] = (uint8_t)((mb[pos] & 1) | (i < r1 ? 2 : 0));
            }
            if (threadIdx.x == 0) s_t = __longlong_as_double((long long)buf[r1 - 1].key);
        }
        __syncthreads();
        return s_t;
    }
    const Cand tb = cta_select_rank(list, n, r1, 64, buf, st);
    if (tb.pad) return 0.0;
    const u128 tv = comp(tb);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const Cand e = list[i];
        mb[e.pos] = (uint8_t)((mb[e.pos] & 1) | (comp(e) <= tv ? 2 : 0));
    }
    return __longlong_as_double((long long)tb.key);
}

template <int PB>
__global__ void __launch_bounds__(SF_T) k_select_fast(const Chain* __restrict__ ch, SelRule* __restrict__ rule,
                                                      const float* __restrict__ Xp, const float* __restrict__ dkeys,
                                                      long long qm, Cand* __restrict__ cand_all,
                                                      Cand* __restrict__ band_all, unsigned* __restrict__ hist,
                                                      uint8_t* __restrict__ memb_all, const int* __restrict__ segcnt,
                                                      int m, int p, int hb, Status* st) {
    static_assert(WIN_BINS % SF_T == 0, "window bins per thread");
    static_assert(SEL_SMALL * sizeof(Cand) >= HIST_BINS * sizeof(unsigned), "histogram aliases buf");
    __shared__ Cand buf[SEL_SMALL];
    extern __shared__ double sm64[];
    double* sM = sm64;              // PB x PB
    double* smu = sm64 + PB * PB;   // PB
    __shared__ unsigned wt[SF_T / 32];
    __shared__ int s_n, s_bin, s_last, s_base, s_nlo;
    const int c = blockIdx.x;
    if (!ch[c].active) return;
    SelRule& R = rule[c];
    if (!R.win) return;
    const int l = c / 2, k = c % 2;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int C = R.cand < m ? R.cand : m;
    const int r = hb - R.below;
    unsigned* h = hist + (size_t)c * HIST_BINS;
    uint8_t* mb = memb_all + (size_t)c * m;
    // 1. the window bin of rank r (each thread owns PER consecutive bins)
    constexpr int PER = WIN_BINS / SF_T;
    unsigned loc[PER];
    unsigned run = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) { loc[i] = h[tid * PER + i]; run += loc[i]; }
    unsigned x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    if (tid == 0) { s_bin = -1; s_nlo = 0; }
    __syncthreads();
    unsigned cum = x - run;
    for (int k2 = 0; k2 < w; ++k2) cum += wt[k2];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        if (r >= 1 && cum < (unsigned)r && (unsigned)r <= cum + loc[i]) s_bin = tid * PER + i;
        cum += loc[i];
    }
    __syncthreads();
    const int b = s_bin;
    bool miss = (r < 1 || r > C || b < 0);
    unsigned long long kb_lo = 0ull, kb_hi = 0ull;
    if (!miss) {
        const unsigned lo_key = R.w_lo + ((unsigned)b << R.w_sh);
        unsigned hi_key = lo_key + ((1u << R.w_sh) - 1u);
        if (hi_key > R.w_hi || hi_key < lo_key) hi_key = R.w_hi;
        kb_lo = __float_as_uint(__uint_as_float(lo_key) * (float)(1.0 - BAND_EPS));
        kb_hi = __float_as_uint(__uint_as_float(hi_key) * (float)(1.0 + BAND_EPS));
        // rows of the FP64 range outside the window were not listed
        if (kb_lo < (unsigned long long)R.w_lo || kb_hi > (unsigned long long)R.w_hi) miss = true;
    }
    // 2. this CTA's share of the candidates: the in-range rows are listed
    //    first (positions in buf), then their FP64 distances are taken in one
    //    pass, one row per thread, so the FP64 latency is paid once
    if (!miss) {
        stage_m64<PB>(ch[c].rp, p, sM, smu);
        constexpr int LCAP = (int)(SEL_SMALL * sizeof(Cand) / sizeof(int));
        int* lst = reinterpret_cast<int*>(buf);
        const Cand* cand = cand_all + (size_t)c * m;
        Cand* list = band_all + (size_t)c * m;
        const float* Xb = Xp + (size_t)l * m * PB;
        // the candidates sit in segments, one per CTA of the distance pass
        // (segment b from the first row of that CTA's range on)
        const int nseg = R.nseg;
        const int segw = nseg > 0 ? (m + nseg - 1) / nseg : m;
        int nlo = 0;
        // FP64 distances of the listed rows, one per thread, appended to the chain's list
        auto flush = [&]() {
            const int nl = s_n;
            if (tid == 0 && nl) s_base = atomicAdd(&R.band, nl);
            __syncthreads();
            for (int j = tid; j < nl; j += SF_T) {
                const unsigned ps = (unsigned)lst[j];
                Cand e;
                e.key = (unsigned long long)__double_as_longlong(row_d2_fp64<PB>(Xb + (size_t)ps * PB, sM, smu));
                e.pos = ps;
                e.pad = 0;
                list[s_base + j] = e;
            }
            __syncthreads();
            if (tid == 0) s_n = 0;
            __syncthreads();
        };
        if (tid == 0) s_n = 0;
        __syncthreads();
        for (int b = (int)blockIdx.y; b < nseg; b += (int)gridDim.y) {
            const int base = b * segw;
            const int cnt = segcnt[(size_t)c * SEG_MAX + b];
            for (int off = 0; off < cnt; off += SF_T) {
                const int i = off + tid;
                bool take = false;
                unsigned pos = 0;
                if (i < cnt) {
                    const Cand e = cand[base + i];
                    if (e.key < kb_lo) ++nlo;
                    else if (e.key <= kb_hi) { take = true; pos = e.pos; }
                }
                const unsigned bal = __ballot_sync(0xffffffffu, take);
                int wb = 0;
                if (lane == 0 && bal) wb = atomicAdd(&s_n, __popc(bal));
                wb = __shfl_sync(0xffffffffu, wb, 0);
                if (take) lst[wb + __popc(bal & ((1u << lane) - 1u))] = (int)pos;
                __syncthreads();
                if (s_n > LCAP - SF_T) flush();   // room for the next round
            }
        }
        flush();
        nlo = warp_sum_int(nlo);
        if (lane == 0 && nlo) atomicAdd(&s_nlo, nlo);
        __syncthreads();
        if (tid == 0 && s_nlo) atomicAdd(&R.nlo, s_nlo);
    }
    // 3. the chain's last CTA
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&R.done, 1) == (int)gridDim.y - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = tid; i < WIN_BINS; i += SF_T) h[i] = 0u;   // every CTA has read the bins
    if (!miss) {
        const int n64 = atomicAdd(&R.band, 0);
        const int nlo_all = atomicAdd(&R.nlo, 0);
        const double t = rank_and_mark(band_all + (size_t)c * m, n64, r - nlo_all, mb, buf, st);
        if (tid == 0) {
            R.t_lo = kb_lo;
            R.t_hi = kb_hi;
            R.nlo = R.below + nlo_all;
            R.band_off = 0;
            R.t_prev2 = R.t_prev;
            R.t_prev = (float)t;
            R.fast = 1;
            R.acc_win += 1;
            R.acc_cand += C;
            R.acc_band += n64;
        }
        return;
    }
    // the window missed: histogram path over the block's keys, then the
    // band's FP64 distances and ranking in this CTA
    if (tid == 0) { R.need_hist = 1; R.acc_win += 1; R.acc_cand += C; R.acc_miss += 1; }
    unsigned* cnt = reinterpret_cast<unsigned*>(buf);
    cta_hist_path(R, dkeys + (size_t)k * qm + (size_t)l * m, m, hb, cand_all + (size_t)c * m,
                  band_all + (size_t)c * m, buf, cnt, st);
    __syncthreads();
    if (!R.bandsel) return;   // an error was recorded
    stage_m64<PB>(ch[c].rp, p, sM, smu);
    __syncthreads();
    const int nb = R.band;
    Cand* band = band_all + (size_t)c * m + R.band_off;
    const float* Xb = Xp + (size_t)l * m * PB;
    for (int i = tid; i < nb; i += SF_T)
        band[i].key = (unsigned long long)__double_as_longlong(row_d2_fp64<PB>(Xb + (size_t)band[i].pos * PB, sM, smu));
    __syncthreads();
    (void)rank_and_mark(band, nb, hb - R.nlo, mb, buf, st);
    if (tid == 0) { R.acc_band += nb; R.bandsel = 0; R.fast = 1; }
}

void launch_select_fast(const Plan& P, cudaStream_t s) {
    RTD_PB_SWITCH(P.pb, {
        const size_t sm = (size_t)(PB * PB + PB) * sizeof(double);
        // static buffers plus M pass 48 KB at the larger widths: opt in
        cudaFuncSetAttribute(k_select_fast<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_select_fast<PB><<<dim3(2 * P.q, P.sel_ctas > 0 ? P.sel_ctas : SF_CTAS), SF_T, sm, s>>>(P.ch, P.rule, P.Xp, (const float*)P.dkeys,
                                                                   (long long)P.q * P.m, P.cand, P.band, P.hist,
                                                                   P.memb, P.segcnt, P.m, P.p, P.hb, P.st);
    });
}

void launch_select_band(const Plan& P, cudaStream_t s) {
    k_select_band<<<2 * P.q, BANDSEL_T, 0, s>>>(P.ch, P.rule, P.band, P.memb, P.m, P.hb, P.st);
}

}  // namespace rtd
