// rtd_tc.cuh - fifth-generation tensor-core (tcgen05) Gram accumulation for
// the split-BF16 form (Section 3.4's mean and scatter of a subset, with the
// rows' products taken on the tensor cores).
//
// Every row e (centred in FP32) is split as e = e_hi + e_lo with
// e_hi = bf16(e) and e_lo = bf16(e - e_hi) (16 significant bits together);
// the weighted row a = w e is split the same way.  One 16-row step issues
//   D1 += [a_hi]^T [e_hi | e_lo]      D2 += [a_lo]^T [e_hi | e_lo]
// (M = 128 lanes, features on the lanes; N = 2H columns, K = 16 rows), so
// that D1 + D2 holds all four products hi*hi, hi*lo, lo*hi, lo*lo with FP32
// accumulation in tensor memory.  Every FLUSH_ROWS rows the accumulators are
// read back and added to an FP64 copy in shared memory, which bounds the FP32
// accumulation error to that many rows.
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

// Shared-memory matrix descriptor, K-major, no swizzle: 8-row x 16-byte core
// matrices; `lbo` = byte distance between the two core matrices of a row
// group along K, `sbo` = byte distance between successive 8-row groups.
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

// split of two FP32 values into packed BF16 high and low parts
__device__ inline void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float h0 = __low2float(h), h1 = __high2float(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(x0 - h0, x1 - h1);
    hi = *reinterpret_cast<uint32_t*>(&h);
    lo = *reinterpret_cast<uint32_t*>(&l);
}

// ---------------------------------------------------------------- GramTC
// Drop-in for GramAcc<PB, float> (same rows()/store() contract, same slot
// layout) for 25 <= p <= 48.  Needs SMEM bytes of dynamic shared memory
// (16-byte aligned) handed over by setup(), and 256 tensor-memory columns.
template <int PB, int NTH, int TROWS>
struct GramTC {
    static constexpr int PE = PB + 4;
    static constexpr int H = ((PB + 1) + 15) / 16 * 16;     // features on lanes (>= p + 1)
    static constexpr int N = 2 * H;                         // [e_hi | e_lo]
    static constexpr int TR = TROWS;                        // rows per rows() call, at most
    static constexpr int KS = TR / 16;                      // 16-row MMA steps per call
    static constexpr int KSTEP = 128 * H;                   // bytes per step: A_hi, A_lo (H rows), B (2H rows)
    static constexpr int OPS = KS * KSTEP;
    static constexpr int ACC_LD = H + 1;                    // FP64 row stride (bank spread)
    static constexpr int SMEM = OPS + H * ACC_LD * 8;
    static constexpr unsigned TCOLS = 256;
    static constexpr int FLUSH_ROWS = 4096;
    static_assert(H >= 48 && H <= 64, "tensor-core Gram covers 25 <= p <= 63");
    static_assert(TR % 16 == 0, "tile rows must be a multiple of 16");
    static_assert(4 * H <= (int)TCOLS, "tensor memory columns");

    unsigned char* ops;
    double* acc;
    uint32_t* s_taddr;
    uint64_t* bar;
    unsigned phase;
    int pending;       // a commit not yet waited for
    int since;         // rows in the tensor-memory accumulators
    int fresh;         // next MMA starts the accumulators
    int* err;          // shared failure flag

    __device__ void setup(unsigned char* region, uint32_t* taddr_slot, uint64_t* mbar, int* err_flag) {
        ops = region;
        acc = reinterpret_cast<double*>(region + OPS);
        s_taddr = taddr_slot;
        bar = mbar;
        err = err_flag;
    }

    __device__ void init(int = 0) {
        for (int e = threadIdx.x; e < H * ACC_LD; e += NTH) acc[e] = 0.0;
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
            *err = 0;
        }
        if (threadIdx.x < 32) {
            tmem_alloc(s_taddr, TCOLS);
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

    // tensor memory -> FP64 accumulators (rows owned by lanes 0 .. H-1)
    __device__ void flush() {
        wait_mma();
        if (!fresh) {
            const int w = threadIdx.x >> 5;
            if (w < 2) {
                const uint32_t base = *s_taddr + ((uint32_t)(w * 32) << 16);
                const int i = threadIdx.x;       // lane = feature row
                double* arow = acc + i * ACC_LD;
#pragma unroll 1
                for (int c0 = 0; c0 < 4 * H; c0 += 16) {
                    float v[16];
                    tmem_ld16(base + (uint32_t)c0, v);
                    if (i < H) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int j = (c0 + u) % H;
                            arow[j] += (double)v[u];
                        }
                    }
                }
            }
            tc_fence_before();
        }
        __syncthreads();
        tc_fence_after();
        since = 0;
        fresh = 1;
    }

    // k rows of PE floats at tile (k <= TR), weights wt
    __device__ void rows(const float* tile, const float* wt, int k) {
        if (k <= 0) return;
        if (since + k > FLUSH_ROWS) flush();
        else wait_mma();                 // operand buffers free again
        const int nks = (k + 15) >> 4;
        const int items = H * nks * 2;   // (feature, 8-row chunk)
        for (int it = threadIdx.x; it < items; it += NTH) {
            const int j = it % H, c = it / H;
            uint32_t ah[4], al[4], bh[4], bl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r0 = 8 * c + 2 * q, r1 = r0 + 1;
                float e0 = 0.f, e1 = 0.f, w0 = 0.f, w1 = 0.f;
                if (j < PE) {
                    if (r0 < k) { e0 = tile[r0 * PE + j]; w0 = wt[r0]; }
                    if (r1 < k) { e1 = tile[r1 * PE + j]; w1 = wt[r1]; }
                }
                split_bf16x2(w0 * e0, w1 * e1, ah[q], al[q]);
                split_bf16x2(e0, e1, bh[q], bl[q]);
            }
            unsigned char* step = ops + (c >> 1) * KSTEP;
            const int off = (j >> 3) * 256 + (c & 1) * 128 + (j & 7) * 16;
            *reinterpret_cast<uint4*>(step + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
            *reinterpret_cast<uint4*>(step + 32 * H + off) = make_uint4(al[0], al[1], al[2], al[3]);
            *reinterpret_cast<uint4*>(step + 64 * H + off) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
            *reinterpret_cast<uint4*>(step + 96 * H + off) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
        }
        async_proxy_fence();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t t = *s_taddr;
            const uint32_t id = idesc_bf16(128, N);
            const uint32_t base = smem_addr(ops);
            for (int s = 0; s < nks; ++s) {
                const uint32_t a = base + (uint32_t)(s * KSTEP);
                const uint64_t bd = smem_desc(a + 64 * H, 128, 256);
                const bool accum = !(fresh && s == 0);
                mma_bf16(t, smem_desc(a, 128, 256), bd, id, accum);
                mma_bf16(t + (uint32_t)N, smem_desc(a + 32 * H, 128, 256), bd, id, accum);
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
            slot[e] = ((i < H && j < H) ? acc[i * ACC_LD + j] : 0.0) + bad;
        }
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(*s_taddr, TCOLS);
    }
};

}  // namespace rtd
