// rtd_tc.cuh - fifth-generation tensor-core (tcgen05) Gram accumulation for
// the split-BF16 form (the mean and scatter of a subset, Section 3.4, with
// the rows' products taken on the tensor cores).
//
// Every weighted row a = sqrt(w) e (centred in FP32) is split three ways,
// a = a_hi + a_mid + a_lo with a_hi = bf16(a), a_mid = bf16(a - a_hi),
// a_lo = bf16(a - a_hi - a_mid): 24 significant bits, the FP32 row itself.
// One 16-row step issues D += [a_hi | a_mid]^T [a_hi | a_mid | a_lo]
// (M = 128 lanes, features on the lanes; N = 3H columns, K = 16 rows), whose
// blocks are the products hi*hi, hi*mid, hi*lo, mid*hi, mid*mid and mid*lo,
// with FP32 accumulation in tensor memory; lo*hi and lo*mid are the
// transposes of hi*lo and mid*lo and are recovered when the sums are
// symmetrised.  Every FLUSH_ROWS rows the accumulators are read back and
// summed into compensated FP32 pairs in shared memory, which bounds the
// depth of the FP32 accumulation in tensor memory (whose additions need not
// round to nearest).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rtd_async.cuh"

namespace rtd {

// ------------------------------------------------------------- PTX wrappers
// Tensor-memory allocation: one warp, `ncols` a power of two >= 32; the
// column address is written to shared memory at `slot`.
__device__ inline void tmem_alloc(uint32_t* slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ inline void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// ordering of tensor-core operations around thread synchronisation
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor without swizzle; core matrices are 8 rows
// of 16 bytes.  K-major operands: `lbo` = byte distance between core
// matrices along K, `sbo` = between successive 8-row groups along M/N.
// MN-major operands: `lbo` = byte distance between successive 8-row groups
// along K, `sbo` = between core matrices along M/N.
__device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;                 // base offset 0, relative offsets, no swizzle
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                      // D format: F32
           | (1u << 7) | (1u << 10)       // A, B format: BF16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

// the same with both operands MN-major (transpose bits of A and B)
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// Instruction descriptor of kind::tf32: TF32 A and B (32-bit containers),
// FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                      // D format: F32
           | (2u << 7) | (2u << 10)       // A, B format: TF32
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ inline void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}

// TF32 high part of an FP32 value (sign, exponent and the top 10 mantissa
// bits); x - tf32_hi(x) is exact in FP32 and holds the rest.
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ inline void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
// arrive on `bar` once every tensor-core operation issued so far by this
// thread has completed
__device__ inline void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives
// lane (base lane + t), columns col .. col + 15
__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// split of two FP32 values into packed BF16 high, middle and low parts (the
// differences are exact in FP32; the three parts carry 24 significant bits)
__device__ inline void split_bf16x3(float x0, float x1, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float r0 = x0 - __low2float(h), r1 = x1 - __high2float(h);
    __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    __nv_bfloat162 l = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
    hi = *reinterpret_cast<uint32_t*>(&h);
    mid = *reinterpret_cast<uint32_t*>(&m);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// ---------------------------------------------------------------- GramTC
// Drop-in for GramAcc<PB, float> (same put()/rows()/store() contract, same
// slot layout) for 25 <= p <= 48.  Rows are put by the threads that hold
// them: a = sqrt(|w|) (v, 1, 0 ...) is split into BF16 high, middle and low
// parts and written as the MN-major operand [a_hi | a_mid | a_lo] (3H
// features) of one 16-row step.  The buffer serves as B (N = 3H) and its
// first 128 features as A (M = 128 lanes: a_hi on lanes 0 .. H-1, a_mid on
// lanes H .. 2H-1, the rest unused), so one MMA per step accumulates the six
// partial products.  In signed mode (rows of weight -1, the swapped-out rows
// of the update C-step) A is a buffer of its own holding s [a_hi | a_mid]
// with s the weight's sign (BF16 negation is exact), so one accumulator
// takes rows of both signs.  Needs SMEM bytes of dynamic shared memory
// (16-byte aligned) handed over by setup(), and 256 tensor-memory columns:
// two CTAs of an SM can hold their accumulators at once.
template <int PB, int NTH, int TROWS>
struct GramTC {
    static constexpr int PE = PB + 4;
    static constexpr int H = ((PB + 1) + 15) / 16 * 16;     // features incl. the constant (>= p + 1)
    static constexpr int N = 3 * H;                         // [a_hi | a_mid | a_lo]
    static constexpr int TR = TROWS;                        // rows per rows() call, at most
    static constexpr int CH = N / 8;                        // 16-byte feature chunks per row
    static constexpr int GROUP = CH * 128;                  // bytes per 8 rows: CH chunks of 8 rows x 16 B
    static constexpr int OPS1 = TR / 8 * GROUP;             // the B operand buffer
    static constexpr int CHA = 16;                          // A: 128 features, 16 chunks
    static constexpr int GROUP_A = CHA * 128;
    static constexpr int OPS_A = TR / 8 * GROUP_A;          // the signed A operand buffer
    static constexpr int PAD = 2048;
    static constexpr int ACC_LD = H + 1;                    // pair-sum row stride (bank spread)
    static constexpr int SMEM = OPS1 + OPS_A + PAD + H * ACC_LD * 8;
    // rows accumulated in FP32 in tensor memory between two flushes (one
    // batch: the accumulation there need not round to nearest, so its depth
    // is kept short)
    static constexpr int FLUSH_ROWS = 128;
    static_assert(2 * H <= 128 && CH >= 16, "A: hi and mid on at most 128 lanes, read within one row group");
    static_assert(N % 16 == 0 && N <= 256, "N a multiple of 16, at most 256");
    static_assert(TR % 16 == 0, "tile rows must be a multiple of 16");

    unsigned char* ops;
    FF* acc;            // H x ACC_LD compensated FP32 sums
    uint32_t* s_taddr;
    uint64_t* bar;
    int* err;           // shared failure flag
    unsigned phase;
    unsigned tcols;
    int pending;        // a commit not yet waited for
    int since;          // rows in the tensor-memory accumulators
    int fresh;          // next MMA starts the accumulators
    int sgn;            // signed mode: negative weights allowed

    __device__ void setup(unsigned char* region, uint32_t* taddr_slot, uint64_t* mbar, int* err_flag) {
        ops = region;
        acc = reinterpret_cast<FF*>(region + OPS1 + OPS_A + PAD);
        s_taddr = taddr_slot;
        bar = mbar;
        err = err_flag;
    }

    // all threads; signed_rows: some rows may carry negative weights
    __device__ void init(int = 0, bool signed_rows = false) {
        sgn = signed_rows ? 1 : 0;
        tcols = 256u;
        for (int e = threadIdx.x; e < H * ACC_LD; e += NTH) acc[e] = FF{0.f, 0.f};
        if (sgn) {   // A's lanes 2H .. 127 (never read back) hold zeros
            constexpr int c0 = 2 * H / 8, nz = CHA - c0;
            for (int e = threadIdx.x; e < TR * nz; e += NTH) {
                const int slot = e / nz, c = c0 + e % nz;
                *reinterpret_cast<uint4*>(ops + OPS1 + (slot >> 3) * GROUP_A + (slot & 7) * 16 + c * 128) =
                    make_uint4(0, 0, 0, 0);
            }
        }
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
            *err = 0;
        }
        if (threadIdx.x < 32) {
            tmem_alloc(s_taddr, tcols);
            tmem_relinquish();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        phase = 0;
        pending = 0;
        since = 0;
        fresh = 1;
    }

    __device__ void wait_mma() {
        if (!pending) return;
        if (!mbar_wait(bar, phase)) {
            if (threadIdx.x == 0) *err = 1;
        }
        phase ^= 1u;
        pending = 0;
        tc_fence_after();
    }

    // tensor memory -> compensated FP32 accumulators.  Lane L < H holds
    // feature L of the a_hi rows, lane H <= L < 2H feature L - H of the a_mid
    // rows; column c holds feature c % H of part c / H.  A lane first folds
    // its three column parts in FP32 (the lo part twice: the symmetric part
    // taken in store() restores the lo*hi and lo*mid blocks from hi*lo and
    // mid*lo), then adds the folded row into row L % H of the pair sums; the
    // hi and mid lanes of a feature add in two phases, one writer per row at
    // a time.
    __device__ void flush() {
        wait_mma();
        if (!fresh) {
            const int w = threadIdx.x >> 5;
            const int L = threadIdx.x;
            float t[H];
#pragma unroll
            for (int j = 0; j < H; ++j) t[j] = 0.f;
            if (w < 4) {
                const uint32_t base = *s_taddr + ((uint32_t)(w * 32) << 16);
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                    float v[16];
                    tmem_ld16(base + (uint32_t)c0, v);
                    const float f = (c0 >= 2 * H) ? 2.f : 1.f;   // a 16-column group lies in one part
#pragma unroll
                    for (int u = 0; u < 16; ++u) t[(c0 % H) + u] = fmaf(f, v[u], t[(c0 % H) + u]);
                }
            }
            for (int ph = 0; ph < 2; ++ph) {
                const bool mine = (ph == 0) ? (L < H) : (L >= H && L < 2 * H);
                if (mine) {
                    FF* arow = acc + (L % H) * ACC_LD;
#pragma unroll
                    for (int j = 0; j < H; ++j) {
                        const FF e = ff_two_sum(arow[j].hi, t[j]);
                        arow[j] = FF{e.hi, arow[j].lo + e.lo};
                    }
                }
                __syncthreads();
            }
            tc_fence_before();
        }
        __syncthreads();
        tc_fence_after();
        since = 0;
        fresh = 1;
    }

    // all threads, before the put() calls of a batch: operand buffers free
    __device__ void begin() {
        if (since + TR > FLUSH_ROWS) flush();
        else wait_mma();
    }

    // one thread: row `slot` (< TR) of the batch, centred values v (zero
    // beyond p), weight w
    __device__ void put(float*, float*, int slot, const float (&v)[PB], int p, float w) {
        const float sw = sqrtf(fabsf(w));
        unsigned char* dst = ops + (slot >> 3) * GROUP + (slot & 7) * 16;
        unsigned char* da = ops + OPS1 + (slot >> 3) * GROUP_A + (slot & 7) * 16;
        const uint32_t neg = (sgn && w < 0.f) ? 0x80008000u : 0u;   // sign bits of both BF16 halves
#pragma unroll
        for (int g = 0; g < H / 8; ++g) {
            uint32_t hi[4], mi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j0 = 8 * g + 2 * q, j1 = j0 + 1;
                const float a0 = (j0 < PB ? v[j0 < PB ? j0 : 0] : 0.f) * sw + (j0 == p ? sw : 0.f);
                const float a1 = (j1 < PB ? v[j1 < PB ? j1 : 0] : 0.f) * sw + (j1 == p ? sw : 0.f);
                split_bf16x3(a0, a1, hi[q], mi[q], lo[q]);
            }
            *reinterpret_cast<uint4*>(dst + g * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(dst + (H / 8 + g) * 128) = make_uint4(mi[0], mi[1], mi[2], mi[3]);
            *reinterpret_cast<uint4*>(dst + (2 * H / 8 + g) * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            if (sgn) {
                *reinterpret_cast<uint4*>(da + g * 128) =
                    make_uint4(hi[0] ^ neg, hi[1] ^ neg, hi[2] ^ neg, hi[3] ^ neg);
                *reinterpret_cast<uint4*>(da + (H / 8 + g) * 128) =
                    make_uint4(mi[0] ^ neg, mi[1] ^ neg, mi[2] ^ neg, mi[3] ^ neg);
            }
        }
    }

    // all threads, after the put() calls: k rows were put (slots 0 .. k-1)
    __device__ void rows(const float*, const float*, int k) {
        if (k <= 0) return;
        const int nks = (k + 15) >> 4;
        const int kpad = nks * 16;
        // zero rows k .. kpad-1 of the last step (B, and A's hi and mid in
        // signed mode)
        for (int e = threadIdx.x; e < (kpad - k) * CH; e += NTH) {
            const int slot = k + e / CH, g = e % CH;
            *reinterpret_cast<uint4*>(ops + (slot >> 3) * GROUP + (slot & 7) * 16 + g * 128) = make_uint4(0, 0, 0, 0);
        }
        if (sgn) {
            constexpr int ca = 2 * H / 8;
            for (int e = threadIdx.x; e < (kpad - k) * ca; e += NTH) {
                const int slot = k + e / ca, g = e % ca;
                *reinterpret_cast<uint4*>(ops + OPS1 + (slot >> 3) * GROUP_A + (slot & 7) * 16 + g * 128) =
                    make_uint4(0, 0, 0, 0);
            }
        }
        async_proxy_fence();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t t = *s_taddr;
            const uint32_t id = idesc_bf16_mn(128, N);
            const uint32_t base = smem_addr(ops);
            for (int s = 0; s < nks; ++s) {
                const bool accum = !(fresh && s == 0);
                const uint32_t b = base + (uint32_t)(s * 2 * GROUP);
                const uint64_t db = smem_desc(b, GROUP, 128);
                const uint64_t da = sgn ? smem_desc(base + (uint32_t)(OPS1 + s * 2 * GROUP_A), GROUP_A, 128) : db;
                mma_bf16(t, da, db, id, accum);
            }
            mma_commit(bar);
        }
        pending = 1;
        fresh = 0;
        since += k;
    }

    // Final FP64 sums -> one slot in the GramAcc block layout (blocks
    // (bi <= bj) of 4 x 4 over the PE-long extended vector); frees the
    // tensor memory.
    __device__ void store(double* /*red*/, double* slot) {
        flush();
        constexpr int NB = PE / 4, NBLK = NB * (NB + 1) / 2;
        // a wait that ran out leaves NaN in the slot: the fit's finalize
        // then reports the chain as failed instead of using partial sums
        const double bad = *err ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
        for (int e = threadIdx.x; e < NBLK * 16; e += NTH) {
            int b = e >> 4, bi = 0;
            while (b >= NB - bi) { b -= NB - bi; ++bi; }
            const int bj = bi + b;
            const int i = 4 * bi + ((e & 15) >> 2), j = 4 * bj + (e & 3);
            slot[e] = ((i < H && j < H) ? 0.5 * (ff_d(acc[i * ACC_LD + j]) + ff_d(acc[j * ACC_LD + i])) : 0.0) + bad;
        }
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(*s_taddr, tcols);
    }
};

}  // namespace rtd
