// rtd_rows.cu - row kernels that do not depend on the padded width, and the
// dispatch of the width-templated ones (instantiated in rtd_rows_pb*.cu).
#include <atomic>

#include "rtd_rows.cuh"
#include "rtd_rows_api.cuh"

namespace rtd {

// =====================================================================
// Partition (Section 4): permuted, padded copy of the rows.
// =====================================================================
__global__ void k_gather(const float* __restrict__ X, long long ld, int p, int pb, long long nq, long long t0,
                         Feistel F, float* __restrict__ Xp, int* __restrict__ perm, Status* st) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool vec = (p % 4 == 0) && (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nq; t += stride) {
        long long src = feistel_perm(F, t0 + t);
        float4* dst = reinterpret_cast<float4*>(Xp + t * pb);
        if (src < 0) {
            set_error(st, RTD_EINTERNAL);
            for (int j = 0; j < pb / 4; ++j) dst[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        perm[t] = (int)src;
        const float* row = X + src * ld;
        if (vec) {
            const float4* r4 = reinterpret_cast<const float4*>(row);
            for (int j = 0; j < pb / 4; ++j) dst[j] = (4 * j < p) ? __ldg(r4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            for (int j = 0; j < pb / 4; ++j) {
                float4 v;
                v.x = (4 * j + 0 < p) ? __ldg(row + 4 * j + 0) : 0.f;
                v.y = (4 * j + 1 < p) ? __ldg(row + 4 * j + 1) : 0.f;
                v.z = (4 * j + 2 < p) ? __ldg(row + 4 * j + 2) : 0.f;
                v.w = (4 * j + 3 < p) ? __ldg(row + 4 * j + 3) : 0.f;
                dst[j] = v;
            }
        }
    }
}

void launch_gather(const Plan& P, cudaStream_t s) {
    long long nq = (long long)P.q * P.m;
    int grid = P.nsm * 8;
    k_gather<<<grid, NT, 0, s>>>(P.X, P.ld, P.p, P.pb, nq, P.t0, P.F, P.Xp, P.perm, P.st);
}

// =====================================================================
// Whole-X column keys for the univariate MCD (Sections 3.1, 4) and the
// non-finite check.
// =====================================================================
__global__ void k_col_keys(const float* __restrict__ X, long long ld, int p, long long n,
                           uint32_t* __restrict__ keys, Status* st) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float* row = X + i * ld;
        bool bad = false;
        for (int j = 0; j < p; ++j) {
            float v = row[j];
            bad |= !isfinite(v);
            keys[(long long)j * n + i] = f2key(v);
        }
        if (bad) set_error(st, RTD_ENONFINITE);
    }
}

void launch_col_keys(const Plan& P, uint32_t* keys, cudaStream_t s) {
    k_col_keys<<<P.nsm * 8, NT, 0, s>>>(P.X, P.ld, P.p, P.n, keys, P.st);
}

// =====================================================================
// Candidate compaction of the radix select: rows whose coarse key lies in
// the bucket of rank h_b (widened by the FP64 band in the FP32 form) are
// appended to the chain's candidate list; rows below are counted.
// =====================================================================

template <typename T>
__global__ void __launch_bounds__(NT) k_compact(const T* __restrict__ dkeys, int m, int cpb, long long qm,
                                                const Chain* __restrict__ ch, SelRule* __restrict__ rule,
                                                Cand* __restrict__ cand) {
    const int l = blockIdx.y;
    int r0, r1;
    block_rows(m, cpb, r0, r1);
    for (int k = 0; k < 2; ++k) {
        const int c = 2 * l + k;
        if (!ch[c].active || rule[c].fast) continue;
        const unsigned long long lo = rule[c].lo, hi = rule[c].hi;
        const T* in = dkeys + (size_t)k * qm;
        Cand* out = cand + (size_t)c * m;
        int below = 0;
        // whole warps iterate together so that the ballot below is full
        for (int base = r0; base < r1; base += NT) {
            int row = base + threadIdx.x;
            bool valid = row < r1;
            T d = valid ? in[row] : (T)0;
            unsigned long long ck = coarse_key(d);
            below += (valid && ck < lo) ? 1 : 0;
            bool take = valid && ck >= lo && ck <= hi;
            unsigned mask = __ballot_sync(0xffffffffu, take);
            if (mask) {
                int lane = threadIdx.x & 31;
                int leader = __ffs(mask) - 1;
                int basei = 0;
                if (lane == leader) basei = atomicAdd(&rule[c].cand, __popc(mask));
                basei = __shfl_sync(0xffffffffu, basei, leader);
                if (take) {
                    int idx = basei + __popc(mask & ((1u << lane) - 1u));
                    if (idx < m) {
                        Cand e;
                        e.key = full_key(d);
                        e.pos = (unsigned)(row - l * m);
                        e.pad = 0;
                        out[idx] = e;
                    }
                }
            }
        }
        below = cta_sum_int(below);
        if (threadIdx.x == 0 && below) atomicAdd(&rule[c].below, below);
    }
}

void launch_compact(const Plan& P, cudaStream_t s) {
    dim3 grid(P.cpb_dist, P.q);
    long long qm = (long long)P.q * P.m;
    if (P.precision == RTD_FP64)
        k_compact<double><<<grid, NT, 0, s>>>((const double*)P.dkeys, P.m, P.cpb_dist, qm, P.ch, P.rule, P.cand);
    else
        k_compact<float><<<grid, NT, 0, s>>>((const float*)P.dkeys, P.m, P.cpb_dist, qm, P.ch, P.rule, P.cand);
}








// ---------------------------------------------------------------- flags
// Four distances per thread and step (one 16-byte load, one 4-byte store)
// when d2 and flags are 16- and 4-byte aligned; one otherwise.  cut_f is
// the largest float not above the cutoff, so x > cut_f exactly when the
// float x exceeds the FP64 cutoff (one FP32 compare per distance).
__global__ void k_flag(const float* __restrict__ d2, long long n, float cut, uint8_t* __restrict__ flags,
                       unsigned long long* __restrict__ count) {
    int nf = 0;
    const bool vec = ((reinterpret_cast<uintptr_t>(d2) & 15) == 0) &&
                     (!flags || (reinterpret_cast<uintptr_t>(flags) & 3) == 0);
    const long long nv = vec ? n / 4 : 0;
    const long long stride = (long long)gridDim.x * NT;
    for (long long v = (long long)blockIdx.x * NT + threadIdx.x; v < nv; v += stride) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(d2) + v);
        const unsigned o0 = q.x > cut, o1 = q.y > cut, o2 = q.z > cut, o3 = q.w > cut;
        if (flags) reinterpret_cast<unsigned*>(flags)[v] = o0 | (o1 << 8) | (o2 << 16) | (o3 << 24);
        nf += (int)(o0 + o1 + o2 + o3);
    }
    for (long long i = 4 * nv + (long long)blockIdx.x * NT + threadIdx.x; i < n; i += stride) {
        const bool o = d2[i] > cut;
        if (flags) flags[i] = o ? 1 : 0;
        nf += o ? 1 : 0;
    }
    nf = cta_sum_int(nf);
    if (threadIdx.x == 0 && nf && count) atomicAdd(count, (unsigned long long)nf);
}

void launch_flag(const float* d2, long long n, double cut, uint8_t* flags, unsigned long long* count,
                 cudaStream_t s) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n + NT - 1) / NT;
    int grid = (int)(blocks < (long long)nsm * 16 ? blocks : (long long)nsm * 16);
    if (grid < 1) grid = 1;
    float cut_f = (float)cut;   // the largest float not above cut
    if ((double)cut_f > cut) cut_f = std::nextafter(cut_f, -INFINITY);
    k_flag<<<grid, NT, 0, s>>>(d2, n, cut_f, flags, count);
}

// ------------------------------------------------------- subset output
__global__ void k_subset_out(const int* __restrict__ perm, const uint8_t* __restrict__ memb,
                             const uint8_t* __restrict__ wset, const Chain* __restrict__ ch,
                             const int* __restrict__ chosen, int m, long long qm, uint8_t* __restrict__ out) {
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < qm; t += stride) {
        int l = (int)(t / m);
        int k = chosen[l];
        uint8_t v = 0;
        if (k >= 0) v |= memb[(size_t)(2 * l + k) * m + (t - (long long)l * m)] & 1;
        v |= wset[t] & 2;
        out[perm[t]] = v;
    }
}

void launch_subset_out(const Plan& P, uint8_t* out, cudaStream_t s) {
    long long qm = (long long)P.q * P.m;
    k_subset_out<<<P.nsm * 8, NT, 0, s>>>(P.perm, P.memb, P.wset, P.ch, P.chosen, P.m, qm, out);
}


void launch_start1(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, start1, P, s); }
void launch_start2(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, start2, P, s); }
void launch_transform(const Plan& P, int which, cudaStream_t s) { (void)which; RTD_PB_CALL(P.pb, transform, P, s); }
void launch_dist(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, dist, P, s); }
void launch_dist_win(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, dist_win, P, s); }
void launch_dist_tc(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, dist_tc, P, s); }
void launch_band64(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, band64, P, s); }
void launch_grad(const float* X, long long n, int p, long long ld, const uint8_t* wset, int wbit,
                 const RowParams* rp, double* partial, size_t slot_d, double* tot, double c, double w_ld,
                 double w_rd, GradCot cot, float* grad, int nsm, cudaStream_t s) {
    RTD_PB_CALL(pad_p(p), grad, X, n, p, ld, wset, wbit, rp, partial, slot_d, tot, c, w_ld, w_rd, cot, grad, nsm,
                s);
}
void launch_memb(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, memb, P, s); }
void launch_rew(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, rew, P, s); }
void launch_member_gram(const Plan& P, cudaStream_t s) { RTD_PB_CALL(P.pb, member_gram, P, s); }

void launch_final(const Plan& P, float* d2_out, uint8_t* flags_out, cudaStream_t s) {
    RTD_PB_CALL(P.pb, final, P.X, P.n, P.p, P.ld, P.precision, P.fitrp + 1, &P.cs->cutoff_d2, 1,
                d2_out, flags_out, &P.st->n_flagged, P.nsm, s);
}

// SM count of the current device, looked up once per device (the scoring
// calls are launched per batch of rows, where every host microsecond shows)
static int sm_count_here() {
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        v = 148;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

void launch_score_flags(const float* X, long long n, int p, long long ld, const RowParams* rp, int precision,
                        const double* cut_dev, const Status* st, float* d2_out, uint8_t* flags,
                        unsigned long long* count, cudaStream_t s) {
    const int nsm = sm_count_here();
    if (precision == RTD_FP64) {   // FP64 rows decide exactly: the final pass of the fit
        RTD_PB_CALL(pad_p(p), final, X, n, p, ld, precision, rp, cut_dev, flags ? 1 : 0, d2_out, flags, count,
                    nsm, s);
        return;
    }
    RTD_PB_CALL(pad_p(p), score, X, n, p, ld, rp, cut_dev, st, d2_out, flags, count, nsm, s);
}

void launch_score(const float* X, long long n, int p, long long ld, const RowParams* rp,
                  int precision, float* d2_out, cudaStream_t s) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    RTD_PB_CALL(pad_p(p), final, X, n, p, ld, precision, rp, nullptr, 0, d2_out, nullptr, nullptr, nsm, s);
}

}  // namespace rtd
