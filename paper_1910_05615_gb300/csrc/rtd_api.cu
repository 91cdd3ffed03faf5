#include <vector>
#include <cmath>
#include <atomic>
#include <mutex>
#include <thread>
#include <algorithm>
// rtd_api.cu - C ABI entry points and host orchestration of RT-DetMCD.
//
// The host validates arguments, lays out the caller's workspace, and issues
// the device stages on the caller's stream.  The only values that come back
// to the host before the end of a fit are the status word (to stop early on
// bad data) and the number of chains still iterating (C-step loop control).
#include <stdio.h>
#include <string.h>

#include "rtd_internal.cuh"

using namespace rtd;

namespace {

constexpr int TARGET_CTAS = 304;      // row-kernel CTAs per pass (all blocks): 2 per SM
constexpr int MIN_ROWS_PER_CTA = 256;
constexpr int MAX_BLOCKS = RTD_MAX_BLOCKS;
constexpr int SF_CTAS_DEFAULT = 8;    // CTAs per chain of the window selection unless tuned

struct Region {
    size_t off, bytes;
};

struct Layout {
    size_t total = 0;
    Region add(size_t bytes) {
        total = (total + 255) & ~(size_t)255;
        Region r{total, bytes};
        total += bytes;
        return r;
    }
};

struct Shape {
    long long n, h, ld;
    int p, pb, q, m, hb, precision, cpb, key_bytes, max_steps, tc;
    size_t slot_doubles;
};

struct Regions {
    Region st, cs, ch, rule, fitrp, res, xstage, d2stage, flagstage, substage, diagstage,
        Xp, perm, arenaA, arenaB, sort_hist, uni, uscratch, gss, dkeys, memb, cand, segcnt, band, hist, swaps,
        blk, partial, gsum, wset, chosen, amb, kept, kl, scratch, fits, moments, sort_tot;
};

rtd_options defaults() {
    rtd_options o;
    memset(&o, 0, sizeof(o));
    o.precision = RTD_FP32;
    o.omega = 4096;
    o.q_override = 0;
    o.max_csteps = 100;
    o.cutoff_q = 0.975;
    o.kappa_max = 1000.0;
    o.seed = 0;
    o.reweight_consistency = 1;
    o.subset_out = nullptr;
    o.diag_out = nullptr;
    o.profile = nullptr;
    o.autotune = 1;
    return o;
}

int make_shape(long long n, int p, long long ld, long long h, const rtd_options& o, Shape& S) {
    if (p < 1 || p > RTD_MAX_P) return RTD_EINVAL;
    if (n <= 2LL * p || n >= (1LL << 31)) return RTD_EINVAL;
    if (ld < p) return RTD_EINVAL;
    if (o.precision != RTD_FP32 && o.precision != RTD_FP64 && o.precision != RTD_BF16) return RTD_EINVAL;
    if (o.precision == RTD_BF16 && (p < 25 || p > 48)) return RTD_EINVAL;
    if (o.omega < 1 || o.max_csteps < 1 || o.q_override < 0 || o.q_override > MAX_BLOCKS) return RTD_EINVAL;
    if (!(o.cutoff_q > 0.0 && o.cutoff_q < 1.0) || !(o.kappa_max > 1.0)) return RTD_EINVAL;
    if (o.reweight_consistency < 0 || o.reweight_consistency > 2) return RTD_EINVAL;
    if (o.select_path < 0 || o.select_path > 2) return RTD_EINVAL;
    if (o.dist_path < 0 || o.dist_path > 1) return RTD_EINVAL;
    if (o.graph < 0 || o.graph > 1 || o.autotune < 0 || o.autotune > 1) return RTD_EINVAL;
    if ((o.init_mu == nullptr) != (o.init_sigma == nullptr)) return RTD_EINVAL;
    if (o.init_mu) {   // warm start: finite, positive diagonal (host memory)
        for (int j = 0; j < p; ++j) {
            if (!std::isfinite(o.init_mu[j]) || !(o.init_sigma[(size_t)j * p + j] > 0.0)) return RTD_EINVAL;
            for (int i = 0; i < p; ++i)
                if (!std::isfinite(o.init_sigma[(size_t)i * p + j])) return RTD_EINVAL;
        }
    }
    S.n = n; S.h = h; S.ld = ld; S.p = p; S.pb = pad_p(p);
    // the split-BF16 form is the FP32 form with its Grams on the tensor cores
    S.precision = (o.precision == RTD_BF16) ? RTD_FP32 : o.precision;
    S.tc = o.precision == RTD_BF16;
    S.max_steps = o.max_csteps;
    // eq. partitionsize, at most MAX_BLOCKS blocks (the paper caps q by the
    // number of CPU cores instead); an explicit q above it is refused above
    long long q = o.q_override ? o.q_override : n / ((long long)p * o.omega);
    if (q < 1) q = 1;
    if (q > MAX_BLOCKS) q = MAX_BLOCKS;
    S.q = (int)q;
    S.m = (int)(n / q);
    S.hb = (q == 1) ? (int)h : (int)((h * (long long)S.m) / n);
    S.key_bytes = (o.precision == RTD_FP64) ? 8 : 4;
    long long cpb = (TARGET_CTAS + S.q - 1) / S.q;
    long long lim = (S.m + MIN_ROWS_PER_CTA - 1) / MIN_ROWS_PER_CTA;
    if (cpb > lim) cpb = lim;
    if (cpb < 1) cpb = 1;
    S.cpb = (int)cpb;
    S.slot_doubles = (size_t)gram_nblk(S.pb) * 16;
    return RTD_OK;
}

int check_h(const Shape& S) {
    // Section 2.1: [(n+p+1)/2] <= h < n; each block needs h_b > p and m > 2p.
    if (S.h < (S.n + S.p + 1) / 2 || S.h >= S.n) return RTD_EINVAL;
    if (S.hb <= S.p || S.m <= 2 * S.p || S.hb >= S.m) return RTD_EINVAL;
    return RTD_OK;
}

size_t tiles_of(long long L) { return (size_t)((L + SORT_TILE_KEYS - 1) / SORT_TILE_KEYS); }

size_t layout(const Shape& S, Regions& R) {
    Layout L;
    const size_t n = (size_t)S.n, p = (size_t)S.p, q = (size_t)S.q, m = (size_t)S.m;
    const size_t qm = q * m, K = (size_t)S.key_bytes;
    R.st = L.add(sizeof(Status));
    R.cs = L.add(sizeof(Consts));
    R.ch = L.add(2 * q * sizeof(Chain));
    R.rule = L.add(2 * q * sizeof(SelRule));
    R.fitrp = L.add(2 * sizeof(RowParams));
    R.res = L.add(sizeof(rtd_result));
    R.xstage = L.add(n * p * sizeof(float));
    R.d2stage = L.add(n * sizeof(float));
    R.flagstage = L.add(n);
    R.substage = L.add(n);
    R.diagstage = L.add(rtdetmcd_diag_size((int)p, (int)q));
    R.Xp = L.add(qm * (size_t)S.pb * sizeof(float));
    R.perm = L.add(qm * sizeof(int));
    size_t arena = p * n * 4;
    if (2 * p * qm * K > arena) arena = 2 * p * qm * K;
    if (qm * K > arena) arena = qm * K;
    R.arenaA = L.add(arena);
    R.arenaB = L.add(arena);
    size_t hs = p * 256 * tiles_of(S.n);
    size_t h2 = 2 * p * q * 256 * tiles_of(S.m);
    if (h2 > hs) hs = h2;
    R.sort_hist = L.add(hs * sizeof(unsigned));
    R.sort_tot = L.add(2 * (2 * p * q > p ? 2 * p * q : p) * 256 * sizeof(unsigned));
    R.uni = L.add(4 * ((2 * p * q > p) ? 2 * p * q : p) * sizeof(double));
    {
        size_t a = unimcd_scratch_doubles((int)p, S.n), b = unimcd_scratch_doubles(2 * (int)(p * q), S.m);
        size_t c = (size_t)p + (size_t)p * p;   // a warm start's (mu, Sigma)
        size_t u = a > b ? a : b;
        R.uscratch = L.add((u > c ? u : c) * sizeof(double));
    }
    R.gss = L.add(2 * q * sizeof(double));
    R.dkeys = L.add(2 * qm * K);
    R.memb = L.add(2 * qm);
    R.cand = L.add(2 * qm * sizeof(Cand));
    R.segcnt = L.add(2 * q * SEG_MAX * sizeof(int));
    R.band = L.add(2 * qm * sizeof(Cand));
    R.hist = L.add(2 * q * HIST_BINS * sizeof(unsigned));
    R.swaps = L.add(2 * q * sizeof(int));
    R.blk = L.add(q * sizeof(int));
    R.partial = L.add(q * (size_t)S.cpb * 2 * S.slot_doubles * sizeof(double));
    R.gsum = L.add(2 * q * S.slot_doubles * sizeof(double));
    R.wset = L.add(qm);
    R.chosen = L.add(q * sizeof(int));
    R.amb = L.add(q * sizeof(int));
    R.kept = L.add(q * sizeof(int));
    R.kl = L.add(q * sizeof(double));
    R.scratch = L.add(((p + p * p) * (q + 1) + 64) * sizeof(double));
    R.fits = L.add(q * (2 + p + p * p) * sizeof(double));
    R.moments = L.add((1 + p + p * p) * sizeof(double));
    return (L.total + 255) & ~(size_t)255;
}

template <typename T>
T* at(void* base, const Region& r) {
    return reinterpret_cast<T*>(reinterpret_cast<char*>(base) + r.off);
}

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of a device other than the current one (where the kernels
// run): such pointers are refused rather than read as peer memory.
bool on_other_device(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.device != dev;
}

#define RTD_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) { return RTD_ECUDA; }    \
    } while (0)

int fetch_status(Status* dev, cudaStream_t s, Status& h) {
    RTD_CUDA(cudaMemcpyAsync(&h, dev, sizeof(Status), cudaMemcpyDeviceToHost, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    RTD_CUDA(cudaGetLastError());
    return RTD_OK;
}

void feistel_setup(Feistel& F, long long n, unsigned long long seed, bool identity) {
    int k = 2;
    while ((1LL << k) < n) k += 2;
    F.half = k / 2;
    F.mask = (1ull << F.half) - 1ull;
    for (int r = 0; r < 4; ++r) F.key[r] = splitmix64(seed + (unsigned long long)r);
    F.identity = identity ? 1 : 0;
    F.n = n;
}

// Stage profile: CUDA events recorded on the fit's stream around each stage,
// read back at the host synchronisation points the fit already has.
struct Prof {
    rtd_profile* out = nullptr;
    cudaStream_t s = nullptr;
    struct Rec { int stage; cudaEvent_t a, b; };
    Rec recs[64];
    int nrec = 0;
    int cur = -1;
    cudaEvent_t ea = nullptr;
    void init(rtd_profile* o, cudaStream_t st) {
        out = o;
        s = st;
        if (out) memset(out, 0, sizeof(*out));
    }
    void begin(int stage) {
        if (!out) return;
        cudaEventCreate(&ea);
        cudaEventRecord(ea, s);
        cur = stage;
    }
    void end(int launches, double bytes) {
        if (!out) return;
        cudaEvent_t eb;
        cudaEventCreate(&eb);
        cudaEventRecord(eb, s);
        if (nrec == 64) collect();
        recs[nrec++] = Rec{cur, ea, eb};
        out->launches[cur] += launches;
        out->bytes[cur] += bytes;
    }
    // after a stream synchronisation
    void collect() {
        if (!out) return;
        for (int i = 0; i < nrec; ++i) {
            float ms = 0.f;
            cudaEventSynchronize(recs[i].b);
            if (cudaEventElapsedTime(&ms, recs[i].a, recs[i].b) == cudaSuccess) out->ms[recs[i].stage] += ms;
            cudaEventDestroy(recs[i].a);
            cudaEventDestroy(recs[i].b);
        }
        nrec = 0;
    }
    ~Prof() { collect(); }
};

// ---------------------------------------------------------------- autotuner
// Launch shapes picked by timing: rows per CTA of the window distance pass
// and CTAs per chain of the window selection.  Neither changes any value a
// fit computes (distances are per row, counts are exact sums, and the
// selection ranks its list in FP64 whatever order it was filled in), so a
// tuned fit equals an untuned one bit for bit.  Choices are kept per
// process, keyed by what the best shape depends on.
struct TuneKey {
    int pb, q, mbucket, precision, tc, dist_path, select_path, dev;
};
struct TuneVal {
    int win_rows, sel_ctas;
};
std::mutex g_tune_lock;
std::vector<std::pair<TuneKey, TuneVal>> g_tune;
thread_local const TuneVal* t_force = nullptr;   // a candidate under test on this thread

int m_bucket(long long m) {   // pairs of octaves of the block length
    int b = 0;
    while ((1LL << (2 * (b + 1))) <= m) ++b;
    return b;
}

TuneKey tune_key(const Shape& S, const rtd_options& o, int dev) {
    TuneKey k;
    memset(&k, 0, sizeof(k));
    k.pb = S.pb; k.q = S.q; k.mbucket = m_bucket(S.m); k.precision = S.precision; k.tc = S.tc;
    k.dist_path = o.dist_path; k.select_path = o.select_path; k.dev = dev;
    return k;
}

bool tune_get(const TuneKey& k, TuneVal& v) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    for (auto& e : g_tune)
        if (memcmp(&e.first, &k, sizeof(TuneKey)) == 0) { v = e.second; return true; }
    return false;
}

void tune_put(const TuneKey& k, const TuneVal& v) {
    std::lock_guard<std::mutex> g(g_tune_lock);
    for (auto& e : g_tune)
        if (memcmp(&e.first, &k, sizeof(TuneKey)) == 0) { e.second = v; return; }
    g_tune.push_back({k, v});
}

TuneVal resolve_tuning(const Shape& S, const rtd_options& o, int dev) {
    TuneVal v{0, 0};
    if (t_force) v = *t_force;
    else tune_get(tune_key(S, o, dev), v);
    return v;
}

// The work decomposition of one fit over the caller's workspace.  With
// q_full > 0, S.q blocks starting at permuted position t0 of a partition
// into q_full blocks (the launch shapes are those of the whole partition).
int make_plan(const float* X, const Shape& S, const rtd_options& o, void* ws, const Regions& R, Plan& P,
              int q_full = 0, long long t0 = 0) {
    memset(&P, 0, sizeof(P));
    Shape SF = S;
    if (q_full) SF.q = q_full;
    P.t0 = t0;
    P.n = S.n; P.h = S.h; P.ld = S.ld; P.p = S.p; P.pb = S.pb; P.q = S.q; P.m = S.m; P.hb = S.hb;
    P.precision = S.precision; P.tc = S.tc; P.cpb = S.cpb; P.max_steps = S.max_steps; P.key_bytes = S.key_bytes;
    int dev = 0;
    RTD_CUDA(cudaGetDevice(&dev));
    RTD_CUDA(cudaDeviceGetAttribute(&P.nsm, cudaDevAttrMultiProcessorCount, dev));
    {
        const TuneVal tv = resolve_tuning(SF, o, dev);
        P.win_rows = tv.win_rows;
        P.sel_ctas = tv.sel_ctas;
    }
    {   // distance pass: one resident wave (two CTAs per SM), at least 512 rows each
        long long cd = (2LL * P.nsm + SF.q - 1) / SF.q;
        long long lim = (S.m + 511) / 512;
        P.cpb_dist = (int)(cd < lim ? (cd > 0 ? cd : 1) : lim);
    }
    feistel_setup(P.F, S.n, o.seed, SF.q == 1);
    P.X = X;
    P.st = at<Status>(ws, R.st);
    P.cs = at<Consts>(ws, R.cs);
    P.ch = at<Chain>(ws, R.ch);
    P.rule = at<SelRule>(ws, R.rule);
    P.fitrp = at<RowParams>(ws, R.fitrp);
    P.Xp = at<float>(ws, R.Xp);
    P.perm = at<int>(ws, R.perm);
    P.arenaA = at<void>(ws, R.arenaA);
    P.arenaB = at<void>(ws, R.arenaB);
    P.sort_hist = at<unsigned>(ws, R.sort_hist);
    P.sort_tot = at<unsigned>(ws, R.sort_tot);
    P.uni = at<double>(ws, R.uni);
    P.uscratch = at<double>(ws, R.uscratch);
    P.gss = at<double>(ws, R.gss);
    P.dkeys = at<void>(ws, R.dkeys);
    P.memb = at<uint8_t>(ws, R.memb);
    P.cand = at<Cand>(ws, R.cand);
    P.segcnt = at<int>(ws, R.segcnt);
    P.band = at<Cand>(ws, R.band);
    P.hist = at<unsigned>(ws, R.hist);
    P.swaps = at<int>(ws, R.swaps);
    P.blk_active = at<int>(ws, R.blk);
    P.partial = at<double>(ws, R.partial);
    P.slot_doubles = S.slot_doubles;
    P.gsum = at<double>(ws, R.gsum);
    P.wset = at<uint8_t>(ws, R.wset);
    P.chosen = at<int>(ws, R.chosen);
    P.amb = at<int>(ws, R.amb);
    P.kept = at<int>(ws, R.kept);
    P.kl = at<double>(ws, R.kl);
    P.scratch = at<double>(ws, R.scratch);
    return RTD_OK;
}

int run_fit(const float* X, const Shape& S, const rtd_options& o, void* ws, cudaStream_t s,
            rtd_result* out, float* d2_out, uint8_t* flags_out) {
    Regions R;
    layout(S, R);
    Plan P;
    { int e = make_plan(X, S, o, ws, R, P); if (e) return e; }

    // rows: stage host data through the workspace
    if (is_device_ptr(X)) {
        P.X = X;
    } else {
        float* xs = at<float>(ws, R.xstage);
        if (S.ld == S.p)   // contiguous rows: one copy
            RTD_CUDA(cudaMemcpyAsync(xs, X, (size_t)S.n * S.p * sizeof(float), cudaMemcpyHostToDevice, s));
        else
            RTD_CUDA(cudaMemcpy2DAsync(xs, (size_t)S.p * sizeof(float), X, (size_t)S.ld * sizeof(float),
                                       (size_t)S.p * sizeof(float), (size_t)S.n, cudaMemcpyHostToDevice, s));
        P.X = xs;
        P.ld = S.p;
    }
    const size_t q2 = 2 * (size_t)S.q, qm = (size_t)S.q * S.m;
    RTD_CUDA(cudaMemsetAsync(P.st, 0, sizeof(Status), s));
    RTD_CUDA(cudaMemsetAsync(P.cs, 0, sizeof(Consts), s));
    RTD_CUDA(cudaMemsetAsync(P.ch, 0, q2 * sizeof(Chain), s));
    RTD_CUDA(cudaMemsetAsync(P.rule, 0, q2 * sizeof(SelRule), s));
    RTD_CUDA(cudaMemsetAsync(P.hist, 0, q2 * HIST_BINS * sizeof(unsigned), s));
    RTD_CUDA(cudaMemsetAsync(P.memb, 0, 2 * qm, s));
    RTD_CUDA(cudaMemsetAsync(P.wset, 0, qm, s));
    RTD_CUDA(cudaMemsetAsync(P.swaps, 0, q2 * sizeof(int), s));

    Status hs;
    Prof pf;
    pf.init(o.profile, s);
    const bool warm = o.init_mu != nullptr;
    const double n_ = (double)S.n, p_ = (double)S.p, qm_ = (double)qm, K_ = (double)S.key_bytes;
    // Section 4: random partition copy
    pf.begin(RTD_STAGE_PARTITION);
    launch_gather(P, s);
    pf.end(1, qm_ * p_ * 4 + qm_ * S.pb * 4);
    // segmented sort timed as its own stage; `stage` resumes afterwards
    auto sorted_ = [&](void* keys, int kb, int nseg, long long L, int stage) {
        pf.end(0, 0.0);
        pf.begin(RTD_STAGE_SORT);
        sort_segments(P, keys, P.arenaB, kb, nseg, L, s);
        // algorithmic bytes: every key read and written once per 8-bit pass
        // (the histogram pass's extra read of the keys is overhead)
        pf.end(3 * kb, (double)nseg * L * kb * 2.0 * kb);
        pf.begin(stage);
    };
    // Sections 3.1 and 4: setup, univariate MCD of every column
    pf.begin(RTD_STAGE_UNIVARIATE);
    launch_setup(P, o, s);
    launch_col_keys(P, (uint32_t*)P.arenaA, s);   // also the non-finite check
    if (warm) {
        // warm start (end of Section 4): standardisation and one chain per
        // block from the given fit; steps 1-2 are skipped
        RTD_CUDA(cudaMemcpyAsync(P.uscratch, o.init_mu, (size_t)S.p * sizeof(double), cudaMemcpyHostToDevice, s));
        RTD_CUDA(cudaMemcpyAsync(P.uscratch + S.p, o.init_sigma, (size_t)S.p * S.p * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
        launch_warm_start(P, P.uscratch, s);
        pf.end(3, n_ * p_ * (4 + 4));
    } else {
        sorted_(P.arenaA, 4, S.p, S.n, RTD_STAGE_UNIVARIATE);
        const int nl = launch_unimcd(P, P.arenaA, 4, S.p, S.n, 0, P.uni, s);
        launch_uni_finish(P, s);
        // rows read, keys written, window search (chunk sums read the keys once)
        pf.end(3 + nl, n_ * p_ * (4 + 4 + 4 + 4));
    }
    { int e = fetch_status(P.st, s, hs); if (e) return e; }
    pf.collect();
    if (hs.code) goto finish;
    if (warm) goto csteps;
    // Section 3.2: initial estimators per block
    pf.begin(RTD_STAGE_STARTS);
    launch_start1(P, s);
    sorted_(P.arenaA, S.key_bytes, S.q, S.m, RTD_STAGE_STARTS);
    launch_gsscm(P, P.arenaA, s);
    launch_start2(P, s);
    launch_start_reduce(P, s);
    pf.end(5, 2 * qm_ * p_ * 4 + qm_ * K_);
    // Section 3.3: refinement
    pf.begin(RTD_STAGE_REFINE);
    launch_refine_eigen(P, s);
    launch_transform(P, 0, s);
    sorted_(P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, RTD_STAGE_REFINE);
    {
        int nl = launch_unimcd(P, P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, 1, P.uni, s);
        launch_refine_mid(P, s);
        launch_transform(P, 1, s);
        sorted_(P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, RTD_STAGE_REFINE);
        nl += launch_unimcd(P, P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, 1, P.uni, s);
        launch_refine_end(P, s);
        pf.end(5 + nl, 2 * (qm_ * p_ * 4 + 2 * p_ * qm_ * K_ * 2));
    }
    // Sections 2.1, 3.4, 3.5: C-steps of every chain until all have stopped
csteps:
    {
        int act_chains = 2 * S.q, act_blocks = S.q;
        pf.begin(RTD_STAGE_CPREP);
        launch_chol_prep(P, s);   // later steps are prepared by the previous step's finalize
        pf.end(1, 0.0);
        for (int it = 0; it <= S.max_steps; ++it) {
            const double mch = (double)S.m * act_chains;
            // FP32 form from the second step on: classification against the
            // predicted window, selection from the window's rows; chains whose
            // window missed take the histogram path below
            const bool win = S.precision == RTD_FP32 && it > 0 && o.select_path != 1;
            // (the first kernel of a step also clears the counters that the
            // membership pass and the finalize accumulate)
            pf.begin(RTD_STAGE_CDIST);
            if (win) {
                if (o.dist_path == 1) launch_dist_tc(P, s);
                else launch_dist_win(P, s);
            } else {
                launch_dist(P, s);
            }
            // rows read, keys written
            pf.end(1, (double)S.m * act_blocks * p_ * 4 + mch * K_);
            if (o.profile) o.profile->flops[RTD_STAGE_CDIST] += mch * p_ * (p_ + 3.0);
            pf.begin(RTD_STAGE_CSELECT);
            if (win) {
                // one launch: bin of the rank, FP64 range, ranking (a chain
                // whose window missed takes the histogram path there)
                launch_select_fast(P, s);
            } else {
                launch_select_bucket(P, s);
                launch_compact(P, s);
                launch_select_finish(P, s);
                if (S.precision == RTD_FP32) {
                    launch_band64(P, s);
                    launch_select_band(P, s);
                }
            }
            pf.end(win ? 1 : 3 + (S.precision == RTD_FP32 ? 2 : 0), win ? 0.0 : mch * K_);
            pf.begin(RTD_STAGE_CUPDATE);
            launch_memb(P, s);
            launch_cstep_finalize(P, s);
            pf.end(3, mch * (K_ + 2));
            int e = fetch_status(P.st, s, hs);
            if (e) return e;
            if (o.profile) {
                o.profile->bytes[RTD_STAGE_CUPDATE] += (double)hs.gram_rows * p_ * 4;
                o.profile->csteps = it + 1;
            }
            pf.collect();
            act_chains = hs.active;
            act_blocks = hs.active_blocks;
            if (hs.code || hs.active == 0) break;
        }
    }
    if (o.profile) {   // selection counters of the C-steps (profiling only: one more copy)
        std::vector<SelRule> hr((size_t)2 * S.q);
        RTD_CUDA(cudaMemcpyAsync(hr.data(), P.rule, hr.size() * sizeof(SelRule), cudaMemcpyDeviceToHost, s));
        RTD_CUDA(cudaStreamSynchronize(s));
        for (const SelRule& r : hr) {
            o.profile->win_steps += r.acc_win;
            o.profile->win_miss += r.acc_miss;
            o.profile->sel_cand += r.acc_cand;
            o.profile->sel_band += r.acc_band;
        }
    }
    if (hs.code) goto finish;
    // Section 4 steps 4-7
    pf.begin(RTD_STAGE_AGGREGATE);
    launch_block_choose(P, s);
    if (S.precision == RTD_FP32) launch_rechoose(P, s);
    launch_aggregate(P, s);
    launch_fit_prep(P, 0, s);
    pf.end((S.q == 1 ? 3 : 5) + (S.precision == RTD_FP32 ? 3 : 0), 2 * qm_);
    // steps 8-9
    pf.begin(RTD_STAGE_REWEIGHT);
    launch_rew(P, s);
    launch_rew_finalize(P, s);
    launch_fit_prep(P, 1, s);
    pf.end(4, qm_ * p_ * 4 + qm_);
    {
        int e = fetch_status(P.st, s, hs);
        if (e) return e;
        pf.collect();
        if (hs.code) goto finish;
    }
    // step 10
    {
        bool d2dev = is_device_ptr(d2_out), fldev = is_device_ptr(flags_out);
        float* d2 = d2_out ? (d2dev ? d2_out : at<float>(ws, R.d2stage)) : nullptr;
        uint8_t* fl = flags_out ? (fldev ? flags_out : at<uint8_t>(ws, R.flagstage)) : nullptr;
        pf.begin(RTD_STAGE_FINAL);
        launch_final(P, d2, fl, s);
        pf.end(1, n_ * p_ * 4 + (d2 ? n_ * 4 : 0) + (fl ? n_ : 0));
        if (d2_out && !d2dev)
            RTD_CUDA(cudaMemcpyAsync(d2_out, d2, (size_t)S.n * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (flags_out && !fldev)
            RTD_CUDA(cudaMemcpyAsync(flags_out, fl, (size_t)S.n, cudaMemcpyDeviceToHost, s));
        if (o.subset_out) {
            bool sdev = is_device_ptr(o.subset_out);
            uint8_t* so = sdev ? o.subset_out : at<uint8_t>(ws, R.substage);
            RTD_CUDA(cudaMemsetAsync(so, 0, (size_t)S.n, s));
            launch_subset_out(P, so, s);
            if (!sdev) RTD_CUDA(cudaMemcpyAsync(o.subset_out, so, (size_t)S.n, cudaMemcpyDeviceToHost, s));
        }
    }
finish:
    {
        rtd_result* dres = at<rtd_result>(ws, R.res);
        RTD_CUDA(cudaMemsetAsync(dres, 0, sizeof(rtd_result), s));
        double* diag = nullptr;
        bool ddev = false;
        if (o.diag_out) {
            ddev = is_device_ptr(o.diag_out);
            diag = ddev ? o.diag_out : at<double>(ws, R.diagstage);
        }
        launch_result(P, dres, diag, s);
        RTD_CUDA(cudaGetLastError());
        RTD_CUDA(cudaMemcpyAsync(out, dres, sizeof(rtd_result), cudaMemcpyDeviceToHost, s));
        if (o.diag_out && !ddev)
            RTD_CUDA(cudaMemcpyAsync(o.diag_out, diag, rtdetmcd_diag_size(S.p, S.q), cudaMemcpyDeviceToHost, s));
        RTD_CUDA(cudaStreamSynchronize(s));
        RTD_CUDA(cudaGetLastError());
        pf.collect();
    }
    return out->status;
}

// =====================================================================
// The fit as one captured CUDA graph.  The kernel sequence of run_fit is
// issued into a graph whose control flow stays on the device:
//   - an IF node after the univariate stage (a data error ends the fit),
//   - a WHILE node for the C-step loop, whose condition the finalize
//     kernel's last CTA sets (chains still iterating, no error),
//   - IF nodes before the aggregation and before the final pass.
// No value comes back to the host until the result record.  Executable
// graphs are kept per host thread, keyed by every argument they bake in, so
// a repeated call is one graph launch and one read of the result.
// =====================================================================
struct GraphKey {
    const float* X;
    long long n, ld, h;
    int p, dev;
    void* ws;
    float* d2;
    uint8_t* fl;
    uint8_t* sub;
    double* diag;
    int precision, omega, q_override, max_csteps, rew, select_path, dist_path;
    int win_rows, sel_ctas;
    double cutoff_q, kappa_max;
    unsigned long long seed;
};

bool key_equal(const GraphKey& a, const GraphKey& b) { return memcmp(&a, &b, sizeof(GraphKey)) == 0; }

// What fixes a graph's topology (its nodes and conditionals): graphs of the
// same topology differ only in their nodes' parameters, so one executable
// graph can be updated in place from the capture of another call.
struct TopoKey {
    int pb, single_block, precision, tc, select_path, dist_path, subset, dev;
};

TopoKey topo_of(const GraphKey& k, const Shape& S) {
    TopoKey t;
    memset(&t, 0, sizeof(t));
    t.pb = S.pb;
    t.single_block = S.q == 1;
    t.precision = S.precision;
    t.tc = S.tc;
    t.select_path = k.select_path;
    t.dist_path = k.dist_path;
    t.subset = k.sub != nullptr;
    t.dev = k.dev;
    return t;
}

struct GraphEntry {
    GraphKey key;
    TopoKey topo;
    cudaGraphExec_t exec = nullptr;
    unsigned long long used = 0;
};

constexpr int GRAPH_CACHE = 8;

struct GraphThreadState {
    GraphEntry entries[GRAPH_CACHE];
    unsigned long long clock = 0;
    cudaStream_t cap = nullptr;        // capture stream
    cudaStream_t body[3] = {nullptr, nullptr, nullptr};   // conditional bodies, by nesting depth
    ~GraphThreadState() {
        for (GraphEntry& e : entries)
            if (e.exec) cudaGraphExecDestroy(e.exec);
        if (cap) cudaStreamDestroy(cap);
        for (cudaStream_t b : body)
            if (b) cudaStreamDestroy(b);
    }
};

GraphThreadState& graph_state() {
    static thread_local GraphThreadState g;
    return g;
}

// A conditional handle of the graph being captured on `s`.
int cond_handle(cudaStream_t s, unsigned def, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    RTD_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, nullptr, nullptr, nullptr));
    if (cst != cudaStreamCaptureStatusActive) return RTD_ECUDA;
    RTD_CUDA(cudaGraphConditionalHandleCreate(h, g, def, cudaGraphCondAssignDefault));
    return RTD_OK;
}

// Append a conditional node to the capture on `s` and start capturing its
// body on `body`.
int cond_open(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaStream_t body) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    RTD_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd));
    if (cst != cudaStreamCaptureStatusActive) return RTD_ECUDA;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    RTD_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    RTD_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    RTD_CUDA(cudaStreamBeginCaptureToGraph(body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal));
    return RTD_OK;
}

int cond_close(cudaStream_t body) {
    cudaGraph_t g = nullptr;
    RTD_CUDA(cudaStreamEndCapture(body, &g));
    return RTD_OK;
}

// One C-step of run_fit (window or histogram selection), then the finalize
// that sets the loop condition hloop.
void issue_cstep(const Plan& P, const Shape& S, const rtd_options& o, bool win, unsigned long long hloop,
                 cudaStream_t s) {
    if (win) {
        if (o.dist_path == 1) launch_dist_tc(P, s);
        else launch_dist_win(P, s);
        launch_select_fast(P, s);
    } else {
        launch_dist(P, s);
        launch_select_bucket(P, s);
        launch_compact(P, s);
        launch_select_finish(P, s);
        if (S.precision == RTD_FP32) {
            launch_band64(P, s);
            launch_select_band(P, s);
        }
    }
    launch_memb(P, s);
    launch_cstep_finalize(P, s, hloop);
}

// Capture the whole fit into a graph (device rows and outputs, no profile,
// no warm start); dres and diag receive the result record.
int capture_fit(Plan& P, const Shape& S, const rtd_options& o, const Regions& R, void* ws, float* d2,
                uint8_t* fl, rtd_result* dres, double* diag, cudaGraph_t* graph_out) {
    GraphThreadState& G = graph_state();
    for (int i = 0; i < 3; ++i)
        if (!G.body[i]) RTD_CUDA(cudaStreamCreateWithFlags(&G.body[i], cudaStreamNonBlocking));
    cudaStream_t s = G.cap;
    RTD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int e = RTD_OK;
    auto body = [&]() -> int {
        const size_t q2 = 2 * (size_t)S.q, qm = (size_t)S.q * S.m;
        RTD_CUDA(cudaMemsetAsync(P.st, 0, sizeof(Status), s));
        RTD_CUDA(cudaMemsetAsync(P.cs, 0, sizeof(Consts), s));
        RTD_CUDA(cudaMemsetAsync(P.ch, 0, q2 * sizeof(Chain), s));
        RTD_CUDA(cudaMemsetAsync(P.rule, 0, q2 * sizeof(SelRule), s));
        RTD_CUDA(cudaMemsetAsync(P.hist, 0, q2 * HIST_BINS * sizeof(unsigned), s));
        RTD_CUDA(cudaMemsetAsync(P.memb, 0, 2 * qm, s));
        RTD_CUDA(cudaMemsetAsync(P.wset, 0, qm, s));
        RTD_CUDA(cudaMemsetAsync(P.swaps, 0, q2 * sizeof(int), s));
        launch_gather(P, s);
        launch_setup(P, o, s);
        launch_col_keys(P, (uint32_t*)P.arenaA, s);
        sort_segments(P, P.arenaA, P.arenaB, 4, S.p, S.n, s);
        launch_unimcd(P, P.arenaA, 4, S.p, S.n, 0, P.uni, s);
        launch_uni_finish(P, s);
        // the rest of the fit runs only if the rows passed the checks so far
        cudaGraphConditionalHandle hA, hW, hB, hC;
        int r = cond_handle(s, 0, &hA);
        if (r) return r;
        launch_cond_ok(hA, P.st, s);
        if ((r = cond_open(s, hA, cudaGraphCondTypeIf, G.body[0]))) return r;
        {
            cudaStream_t b1 = G.body[0];
            launch_start1(P, b1);
            sort_segments(P, P.arenaA, P.arenaB, S.key_bytes, S.q, S.m, b1);
            launch_gsscm(P, P.arenaA, b1);
            launch_start2(P, b1);
            launch_start_reduce(P, b1);
            launch_refine_eigen(P, b1);
            launch_transform(P, 0, b1);
            sort_segments(P, P.arenaA, P.arenaB, S.key_bytes, 2 * S.p * S.q, S.m, b1);
            launch_unimcd(P, P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, 1, P.uni, b1);
            launch_refine_mid(P, b1);
            launch_transform(P, 1, b1);
            sort_segments(P, P.arenaA, P.arenaB, S.key_bytes, 2 * S.p * S.q, S.m, b1);
            launch_unimcd(P, P.arenaA, S.key_bytes, 2 * S.p * S.q, S.m, 1, P.uni, b1);
            launch_refine_end(P, b1);
            launch_chol_prep(P, b1);
            // the C-step loop: the first step, then steps while a chain
            // iterates (condition set by each finalize)
            if ((r = cond_handle(b1, 0, &hW))) return r;
            issue_cstep(P, S, o, false, hW, b1);
            if ((r = cond_open(b1, hW, cudaGraphCondTypeWhile, G.body[1]))) return r;
            issue_cstep(P, S, o, S.precision == RTD_FP32 && o.select_path != 1, hW, G.body[1]);
            if ((r = cond_close(G.body[1]))) return r;
            // Section 4 steps 4-9, then step 10
            if ((r = cond_handle(b1, 0, &hB))) return r;
            launch_cond_ok(hB, P.st, b1);
            if ((r = cond_open(b1, hB, cudaGraphCondTypeIf, G.body[1]))) return r;
            {
                cudaStream_t b2 = G.body[1];
                launch_block_choose(P, b2);
                if (S.precision == RTD_FP32) launch_rechoose(P, b2);
                launch_aggregate(P, b2);
                launch_fit_prep(P, 0, b2);
                launch_rew(P, b2);
                launch_rew_finalize(P, b2);
                launch_fit_prep(P, 1, b2);
                if ((r = cond_handle(b2, 0, &hC))) return r;
                launch_cond_ok(hC, P.st, b2);
                if ((r = cond_open(b2, hC, cudaGraphCondTypeIf, G.body[2]))) return r;
                launch_final(P, d2, fl, G.body[2]);
                if (o.subset_out) {
                    RTD_CUDA(cudaMemsetAsync(o.subset_out, 0, (size_t)S.n, G.body[2]));
                    launch_subset_out(P, o.subset_out, G.body[2]);
                }
                if ((r = cond_close(G.body[2]))) return r;
            }
            if ((r = cond_close(G.body[1]))) return r;
        }
        if ((r = cond_close(G.body[0]))) return r;
        RTD_CUDA(cudaMemsetAsync(dres, 0, sizeof(rtd_result), s));
        launch_result(P, dres, diag, s);
        return RTD_OK;
    };
    e = body();
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (e || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return e ? e : RTD_ECUDA;
    }
    *graph_out = g;
    return RTD_OK;
}

// run_fit through a cached executable graph.  Returns -1 when the call does
// not qualify (host rows or outputs, a profile, a warm start), so that the
// caller takes the stream path.
int run_fit_graph(const float* X, const Shape& S, const rtd_options& o, void* ws, cudaStream_t s,
                  rtd_result* out, float* d2_out, uint8_t* flags_out) {
    if (o.profile || o.init_mu || !is_device_ptr(X) || (d2_out && !is_device_ptr(d2_out)) ||
        (flags_out && !is_device_ptr(flags_out)) || (o.subset_out && !is_device_ptr(o.subset_out)) ||
        (o.diag_out && !is_device_ptr(o.diag_out)))
        return -1;
    GraphThreadState& G = graph_state();
    if (!G.cap) RTD_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    GraphKey k;
    memset(&k, 0, sizeof(k));
    k.X = X; k.n = S.n; k.ld = S.ld; k.h = S.h; k.p = S.p;
    RTD_CUDA(cudaGetDevice(&k.dev));
    k.ws = ws; k.d2 = d2_out; k.fl = flags_out; k.sub = o.subset_out; k.diag = o.diag_out;
    k.precision = o.precision; k.omega = o.omega; k.q_override = o.q_override; k.max_csteps = o.max_csteps;
    k.rew = o.reweight_consistency; k.select_path = o.select_path; k.dist_path = o.dist_path;
    k.cutoff_q = o.cutoff_q; k.kappa_max = o.kappa_max; k.seed = o.seed;
    {
        const TuneVal tv = resolve_tuning(S, o, k.dev);
        k.win_rows = tv.win_rows;
        k.sel_ctas = tv.sel_ctas;
    }
    Regions R;
    layout(S, R);
    rtd_result* dres = at<rtd_result>(ws, R.res);
    GraphEntry* hit = nullptr;
    for (GraphEntry& e : G.entries)
        if (e.exec && key_equal(e.key, k)) hit = &e;
    if (!hit) {
        Plan P;
        int e = make_plan(X, S, o, ws, R, P);
        if (e) return e;
        cudaGraph_t g = nullptr;
        e = capture_fit(P, S, o, R, ws, d2_out, flags_out, dres, o.diag_out, &g);
        if (e) return -1;   // not capturable here: the stream path
        const TopoKey tk = topo_of(k, S);
        // an executable graph of the same topology is updated in place
        for (GraphEntry& en : G.entries) {
            if (!en.exec || memcmp(&en.topo, &tk, sizeof(TopoKey)) != 0) continue;
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(en.exec, g, &info) == cudaSuccess) {
                en.key = k;
                hit = &en;
                break;
            }
            cudaGetLastError();
        }
        if (!hit) {
            GraphEntry* slot = &G.entries[0];
            for (GraphEntry& en : G.entries) {
                if (!en.exec) { slot = &en; break; }
                if (en.used < slot->used) slot = &en;
            }
            if (slot->exec) { cudaGraphExecDestroy(slot->exec); slot->exec = nullptr; }
            cudaError_t ie = cudaGraphInstantiate(&slot->exec, g, 0);
            if (ie != cudaSuccess) {
                cudaGraphDestroy(g);
                cudaGetLastError();
                slot->exec = nullptr;
                return -1;
            }
            slot->key = k;
            slot->topo = tk;
            hit = slot;
        }
        cudaGraphDestroy(g);
    }
    hit->used = ++G.clock;
    RTD_CUDA(cudaGraphLaunch(hit->exec, s));
    RTD_CUDA(cudaMemcpyAsync(out, dres, sizeof(rtd_result), cudaMemcpyDeviceToHost, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    RTD_CUDA(cudaGetLastError());
    return out->status;
}

// One fit through the graph path (or the stream path when it does not
// qualify).
int fit_once(const float* X, const Shape& S, const rtd_options& o, void* ws, cudaStream_t s, rtd_result* out,
             float* d2, uint8_t* fl) {
    int r = -1;
    if (o.graph == 1) r = run_fit_graph(X, S, o, ws, s, out, d2, fl);
    if (r == -1) r = run_fit(X, S, o, ws, s, out, d2, fl);
    return r;
}

// Time every candidate launch shape on this problem (one warm-up and three
// timed fits each, CUDA events on the stream) and keep the fastest.
int autotune_shape(const float* X, const Shape& S, const rtd_options& o, void* ws, cudaStream_t s,
                   rtd_tuning* res) {
    static const int WROWS[3] = {0, 1024, 4096};
    static const int SCTAS[3] = {2, 4, 8};
    int dev = 0;
    RTD_CUDA(cudaGetDevice(&dev));
    cudaEvent_t e0, e1;
    RTD_CUDA(cudaEventCreate(&e0));
    RTD_CUDA(cudaEventCreate(&e1));
    rtd_result tmp;
    TuneVal best{0, 0};
    float best_ms = 1e30f, dflt_ms = -1.f;
    int ncand = 0, err = RTD_OK;
    for (int a = 0; a < 3 && !err; ++a) {
        for (int b = 0; b < 3 && !err; ++b) {
            const TuneVal cand{WROWS[a], SCTAS[b]};
            t_force = &cand;
            err = fit_once(X, S, o, ws, s, &tmp, nullptr, nullptr);   // warm-up (captures the graph)
            float ms[3];
            for (int r = 0; r < 3 && !err; ++r) {
                cudaEventRecord(e0, s);
                err = fit_once(X, S, o, ws, s, &tmp, nullptr, nullptr);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms[r], e0, e1);
            }
            t_force = nullptr;
            if (err) break;
            // median of three
            float lo = fminf(ms[0], fminf(ms[1], ms[2])), hi = fmaxf(ms[0], fmaxf(ms[1], ms[2]));
            const float med = ms[0] + ms[1] + ms[2] - lo - hi;
            ++ncand;
            if (cand.win_rows == 0 && cand.sel_ctas == SF_CTAS_DEFAULT) dflt_ms = med;
            if (med < best_ms) { best_ms = med; best = cand; }
        }
    }
    t_force = nullptr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err) return err;
    tune_put(tune_key(S, o, dev), best);
    if (res) {
        memset(res, 0, sizeof(*res));
        res->win_rows = best.win_rows;
        res->sel_ctas = best.sel_ctas;
        res->candidates = ncand;
        res->ms_best = best_ms;
        res->ms_default = dflt_ms;
    }
    return RTD_OK;
}

// =====================================================================
// The fit in stages, for a fit sharded over processes (one per GPU).
// Section 4's steps grouped by what they need from the other processes:
//   STAGE_UNI      the univariate MCD of a range of columns (step
//                  "standardization"; each column alone),
//   STAGE_BLOCKS   steps 2-4 of a range of blocks (each block alone),
//   STAGE_MOMENTS  steps 5-7 from all q block fits, then the step-8
//                  distances and the reweighting moments of the rows of a
//                  range of blocks,
//   STAGE_FINISH   step 9 from the moments summed over all blocks, then
//                  step 10 for a range of the original rows.
// =====================================================================
enum { STAGE_UNI = 1, STAGE_BLOCKS = 2, STAGE_MOMENTS = 3, STAGE_FINISH = 4 };

struct StageArgs {
    int kind;
    long long lo, hi;        // columns (UNI), blocks (BLOCKS, MOMENTS) or rows (FINISH)
    const double* uni;       // 2p: mu_uni then s_uni
    const double* fits;      // q block-fit records
    const double* moments;   // reweighting moments summed over all blocks
    double* out;             // uni (UNI), records (BLOCKS) or moments (MOMENTS)
    rtd_result* res;         // FINISH
    float* d2;               // FINISH, nullable: hi - lo floats
    uint8_t* fl;             // FINISH, nullable: hi - lo bytes
};

size_t fit_record_doubles(int p) { return 2 + (size_t)p + (size_t)p * p; }
size_t moment_doubles(int p) { return 1 + (size_t)p + (size_t)p * p; }

// Rows on the device: as given, or staged through the workspace.
int device_rows(const float* X, const Shape& S, void* ws, const Regions& R, Plan& P, cudaStream_t s) {
    if (is_device_ptr(X)) {
        P.X = X;
        return RTD_OK;
    }
    float* xs = at<float>(ws, R.xstage);
    if (S.ld == S.p)
        RTD_CUDA(cudaMemcpyAsync(xs, X, (size_t)S.n * S.p * sizeof(float), cudaMemcpyHostToDevice, s));
    else
        RTD_CUDA(cudaMemcpy2DAsync(xs, (size_t)S.p * sizeof(float), X, (size_t)S.ld * sizeof(float),
                                   (size_t)S.p * sizeof(float), (size_t)S.n, cudaMemcpyHostToDevice, s));
    P.X = xs;
    P.ld = S.p;
    return RTD_OK;
}

int clear_plan(const Plan& P, cudaStream_t s) {
    const size_t q2 = 2 * (size_t)P.q, qm = (size_t)P.q * P.m;
    RTD_CUDA(cudaMemsetAsync(P.st, 0, sizeof(Status), s));
    RTD_CUDA(cudaMemsetAsync(P.cs, 0, sizeof(Consts), s));
    RTD_CUDA(cudaMemsetAsync(P.ch, 0, q2 * sizeof(Chain), s));
    RTD_CUDA(cudaMemsetAsync(P.rule, 0, q2 * sizeof(SelRule), s));
    RTD_CUDA(cudaMemsetAsync(P.hist, 0, q2 * HIST_BINS * sizeof(unsigned), s));
    RTD_CUDA(cudaMemsetAsync(P.memb, 0, 2 * qm, s));
    RTD_CUDA(cudaMemsetAsync(P.wset, 0, qm, s));
    RTD_CUDA(cudaMemsetAsync(P.swaps, 0, q2 * sizeof(int), s));
    return RTD_OK;
}

// The given standardisation (2p doubles, host or device memory) into the
// constants of the plan; scales must be positive and finite.
int set_uni(const Plan& P, const double* uni, cudaStream_t s) {
    const int p = P.p;
    std::vector<double> h(2 * (size_t)p);
    RTD_CUDA(cudaMemcpyAsync(h.data(), uni, h.size() * sizeof(double), cudaMemcpyDefault, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < p; ++j)
        if (!std::isfinite(h[j]) || !std::isfinite(h[p + j]) || !(h[p + j] > 0.0)) return RTD_EINVAL;
    char* cs = reinterpret_cast<char*>(P.cs);
    RTD_CUDA(cudaMemcpyAsync(cs + offsetof(Consts, mu_uni), h.data(), p * sizeof(double), cudaMemcpyHostToDevice, s));
    RTD_CUDA(cudaMemcpyAsync(cs + offsetof(Consts, s_uni), h.data() + p, p * sizeof(double), cudaMemcpyHostToDevice, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    return RTD_OK;
}

// Host copy of `count` doubles (host or device memory), all finite.
int host_finite(const double* src, size_t count, cudaStream_t s, std::vector<double>& h) {
    h.resize(count);
    RTD_CUDA(cudaMemcpyAsync(h.data(), src, count * sizeof(double), cudaMemcpyDefault, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    for (double v : h)
        if (!std::isfinite(v)) return RTD_EINVAL;
    return RTD_OK;
}

// Steps 5-7 from the q records a.fits (whole-partition plan P); leaves the
// raw fit's row parameters in P.fitrp[0].  Records are checked on the host
// first: start -1, 0 or 1 and finite values.
int pool_blocks(const Plan& P, const Regions& R, void* ws, const StageArgs& a, cudaStream_t s) {
    const size_t rd = fit_record_doubles(P.p);
    std::vector<double> h;
    { int e = host_finite(a.fits, (size_t)P.q * rd, s, h); if (e) return e; }
    for (int l = 0; l < P.q; ++l) {
        const double c = h[(size_t)l * rd];
        if (c != -1.0 && c != 0.0 && c != 1.0) return RTD_EINVAL;
    }
    double* rec = at<double>(ws, R.fits);
    RTD_CUDA(cudaMemcpyAsync(rec, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    launch_block_fits_in(P, rec, s);
    launch_aggregate(P, s);
    launch_fit_prep(P, 0, s);
    return RTD_OK;
}

int run_stage(const float* X, const Shape& S, const rtd_options& o, void* ws, cudaStream_t s, const StageArgs& a) {
    Regions R;
    layout(S, R);
    Plan P;
    { int e = make_plan(X, S, o, ws, R, P); if (e) return e; }
    { int e = device_rows(X, S, ws, R, P, s); if (e) return e; }
    const bool ranged = a.kind == STAGE_BLOCKS || a.kind == STAGE_MOMENTS;
    Plan PL = P;   // the block range: blocks [lo, hi) of the q-block partition
    if (ranged && a.hi > a.lo) {
        Shape SL = S;
        SL.q = (int)(a.hi - a.lo);
        int e = make_plan(X, SL, o, ws, R, PL, S.q, a.lo * (long long)S.m);
        if (e) return e;
        PL.X = P.X;
        PL.ld = P.ld;
    }
    const int p = S.p;
    Status hs;
    if (a.kind == STAGE_UNI) {
        { int e = clear_plan(P, s); if (e) return e; }
        launch_setup(P, o, s);
        Plan PC = P;   // columns [lo, hi) as a matrix of their own
        PC.X = P.X + a.lo;
        PC.p = (int)(a.hi - a.lo);
        launch_col_keys(PC, (uint32_t*)P.arenaA, s);   // also the non-finite check
        sort_segments(PC, P.arenaA, P.arenaB, 4, PC.p, S.n, s);
        launch_unimcd(PC, P.arenaA, 4, PC.p, S.n, 0, P.uni, s);
        launch_uni_finish(PC, s);
        char* cs = reinterpret_cast<char*>(P.cs);
        RTD_CUDA(cudaMemcpyAsync(a.out, cs + offsetof(Consts, mu_uni), PC.p * sizeof(double), cudaMemcpyDefault, s));
        RTD_CUDA(cudaMemcpyAsync(a.out + PC.p, cs + offsetof(Consts, s_uni), PC.p * sizeof(double),
                                 cudaMemcpyDefault, s));
        int e = fetch_status(P.st, s, hs);
        return e ? e : hs.code;
    }
    if (a.kind == STAGE_BLOCKS) {
        if (a.hi == a.lo) return RTD_OK;
        { int e = clear_plan(PL, s); if (e) return e; }
        launch_setup(PL, o, s);
        { int e = set_uni(PL, a.uni, s); if (e) return e; }
        launch_col_keys(P, (uint32_t*)P.arenaA, s);   // the non-finite check: no further work on bad rows
        { int e = fetch_status(PL.st, s, hs); if (e) return e; }
        if (hs.code) return hs.code;
        launch_gather(PL, s);
        // Section 3.2: initial estimators; Section 3.3: refinement
        launch_start1(PL, s);
        sort_segments(PL, PL.arenaA, PL.arenaB, S.key_bytes, PL.q, S.m, s);
        launch_gsscm(PL, PL.arenaA, s);
        launch_start2(PL, s);
        launch_start_reduce(PL, s);
        launch_refine_eigen(PL, s);
        for (int pass = 0; pass < 2; ++pass) {
            launch_transform(PL, pass, s);
            sort_segments(PL, PL.arenaA, PL.arenaB, S.key_bytes, 2 * p * PL.q, S.m, s);
            launch_unimcd(PL, PL.arenaA, S.key_bytes, 2 * p * PL.q, S.m, 1, PL.uni, s);
            if (pass == 0) launch_refine_mid(PL, s);
        }
        launch_refine_end(PL, s);
        launch_chol_prep(PL, s);
        { int e = fetch_status(PL.st, s, hs); if (e) return e; }
        if (hs.code) return hs.code;
        // Sections 2.1, 3.4, 3.5: C-steps until every chain has stopped
        for (int it = 0; it <= S.max_steps; ++it) {
            const bool win = S.precision == RTD_FP32 && it > 0 && o.select_path != 1;
            issue_cstep(PL, S, o, win, 0, s);
            int e = fetch_status(PL.st, s, hs);
            if (e) return e;
            if (hs.code || hs.active == 0) break;
        }
        if (hs.code) return hs.code;
        // step 4
        launch_block_choose(PL, s);
        if (S.precision == RTD_FP32) launch_rechoose(PL, s);
        double* rec = at<double>(ws, R.fits);
        launch_block_fits_out(PL, rec, s);
        RTD_CUDA(cudaMemcpyAsync(a.out, rec, (size_t)PL.q * fit_record_doubles(p) * sizeof(double),
                                 cudaMemcpyDefault, s));
        int e = fetch_status(PL.st, s, hs);
        return e ? e : hs.code;
    }
    // steps 5-7 on the whole partition
    { int e = clear_plan(P, s); if (e) return e; }
    launch_setup(P, o, s);
    { int e = set_uni(P, a.uni, s); if (e) return e; }
    { int e = pool_blocks(P, R, ws, a, s); if (e) return e; }
    { int e = fetch_status(P.st, s, hs); if (e) return e; }
    if (hs.code) return hs.code;
    double* mo = at<double>(ws, R.moments);
    if (a.kind == STAGE_MOMENTS) {
        if (a.hi > a.lo) {
            launch_gather(PL, s);
            launch_rew(PL, s);
            launch_moments_out(PL, mo, s);
        } else {
            RTD_CUDA(cudaMemsetAsync(mo, 0, moment_doubles(p) * sizeof(double), s));
        }
        RTD_CUDA(cudaMemcpyAsync(a.out, mo, moment_doubles(p) * sizeof(double), cudaMemcpyDefault, s));
        int e = fetch_status(P.st, s, hs);
        return e ? e : hs.code;
    }
    // STAGE_FINISH: step 9, then step 10 for rows [lo, hi)
    {
        std::vector<double> h;
        int e = host_finite(a.moments, moment_doubles(p), s, h);
        if (e) return e;
        RTD_CUDA(cudaMemcpyAsync(mo, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        RTD_CUDA(cudaStreamSynchronize(s));
    }
    launch_moments_finalize(P, mo, s);
    launch_fit_prep(P, 1, s);
    { int e = fetch_status(P.st, s, hs); if (e) return e; }
    if (!hs.code && a.hi > a.lo) {
        const long long nr = a.hi - a.lo;
        Plan PR = P;
        PR.X = P.X + a.lo * P.ld;
        PR.n = nr;
        const bool d2dev = is_device_ptr(a.d2), fldev = is_device_ptr(a.fl);
        float* d2 = a.d2 ? (d2dev ? a.d2 : at<float>(ws, R.d2stage)) : nullptr;
        uint8_t* fl = a.fl ? (fldev ? a.fl : at<uint8_t>(ws, R.flagstage)) : nullptr;
        launch_final(PR, d2, fl, s);
        if (a.d2 && !d2dev) RTD_CUDA(cudaMemcpyAsync(a.d2, d2, nr * sizeof(float), cudaMemcpyDeviceToHost, s));
        if (a.fl && !fldev) RTD_CUDA(cudaMemcpyAsync(a.fl, fl, nr, cudaMemcpyDeviceToHost, s));
    }
    rtd_result* dres = at<rtd_result>(ws, R.res);
    RTD_CUDA(cudaMemsetAsync(dres, 0, sizeof(rtd_result), s));
    launch_result(P, dres, nullptr, s);
    RTD_CUDA(cudaGetLastError());
    RTD_CUDA(cudaMemcpyAsync(a.res, dres, sizeof(rtd_result), cudaMemcpyDeviceToHost, s));
    RTD_CUDA(cudaStreamSynchronize(s));
    RTD_CUDA(cudaGetLastError());
    return a.res->status;
}

// Validation shared by the stage entry points.
int stage_call(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
               void* workspace, size_t ws_bytes, void* stream, const StageArgs& a) {
    rtd_options o = opt ? *opt : defaults();
    o.graph = 0;
    Shape S;
    int e = make_shape(n, p, ld, h, o, S);
    if (!e) e = check_h(S);
    if (e) return e;
    if (!X || o.init_mu) return RTD_EINVAL;
    long long top = a.kind == STAGE_UNI ? p : a.kind == STAGE_FINISH ? n : S.q;
    if (a.lo < 0 || a.hi < a.lo || a.hi > top) return RTD_EINVAL;
    if (a.kind == STAGE_UNI && a.hi == a.lo) return RTD_EINVAL;
    if (a.kind != STAGE_UNI && !a.uni) return RTD_EINVAL;
    if ((a.kind == STAGE_MOMENTS || a.kind == STAGE_FINISH) && !a.fits) return RTD_EINVAL;
    if (a.kind == STAGE_FINISH && (!a.moments || !a.res)) return RTD_EINVAL;
    if (a.kind != STAGE_FINISH && !a.out && !(a.kind == STAGE_BLOCKS && a.hi == a.lo)) return RTD_EINVAL;
    Regions R;
    size_t need = layout(S, R);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    if (on_other_device(X) || on_other_device(workspace) || on_other_device(a.uni) || on_other_device(a.fits) ||
        on_other_device(a.moments) || on_other_device(a.out) || on_other_device(a.d2) || on_other_device(a.fl))
        return RTD_EINVAL;
    return run_stage(X, S, o, workspace, reinterpret_cast<cudaStream_t>(stream), a);
}

}  // namespace

extern "C" {

void rtdetmcd_default_options(rtd_options* opt) {
    if (opt) *opt = defaults();
}

size_t rtdetmcd_diag_size(int32_t p, int32_t q) {
    if (p < 1 || q < 1) return 0;
    size_t rec = 3 * (size_t)p * p + 2 * (size_t)p + 6;
    return (2 * (size_t)p + 2 * (size_t)q * rec + 3 * (size_t)q) * sizeof(double);
}

size_t rtdetmcd_workspace_size(int64_t n, int32_t p, const rtd_options* opt) {
    rtd_options o = opt ? *opt : defaults();
    Shape S;
    if (make_shape(n, p, p, (n + p + 1) / 2, o, S) != RTD_OK) return 0;
    Regions R;
    return layout(S, R);
}

int rtdetmcd_fit(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                 void* workspace, size_t ws_bytes, void* stream, rtd_result* out, float* d2_out,
                 uint8_t* flags_out) {
    if (!out) return RTD_EINVAL;
    memset(out, 0, sizeof(*out));
    rtd_options o = opt ? *opt : defaults();
    Shape S;
    int e = make_shape(n, p, ld, h, o, S);
    if (!e) e = check_h(S);
    if (!X) e = RTD_EINVAL;
    if (e) { out->status = e; return e; }
    Regions R;
    size_t need = layout(S, R);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
        out->status = RTD_EWORKSPACE;
        return RTD_EWORKSPACE;
    }
    if (on_other_device(X) || on_other_device(d2_out) || on_other_device(flags_out) ||
        on_other_device(workspace) || on_other_device(o.subset_out) || on_other_device(o.diag_out)) {
        out->status = RTD_EINVAL;
        return RTD_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int r = -1;
    if (o.graph == 1) r = run_fit_graph(X, S, o, workspace, s, out, d2_out, flags_out);
    if (r == -1) r = run_fit(X, S, o, workspace, s, out, d2_out, flags_out);
    out->status = r;
    return r;
}

int rtdetmcd_partition(int64_t n, int32_t p, int64_t h, const rtd_options* opt, int32_t* q, int64_t* m) {
    rtd_options o = opt ? *opt : defaults();
    Shape S;
    int e = make_shape(n, p, p, h, o, S);
    if (!e) e = check_h(S);
    if (e) return e;
    if (q) *q = S.q;
    if (m) *m = S.m;
    return RTD_OK;
}

int rtdetmcd_standardize(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                         int32_t col_lo, int32_t col_hi, void* workspace, size_t ws_bytes, void* stream,
                         double* uni_out) {
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = STAGE_UNI; a.lo = col_lo; a.hi = col_hi; a.out = uni_out;
    return stage_call(X, n, p, ld, h, opt, workspace, ws_bytes, stream, a);
}

int rtdetmcd_fit_blocks(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                        const double* uni, int32_t blk_lo, int32_t blk_hi, void* workspace, size_t ws_bytes,
                        void* stream, double* fits_out) {
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = STAGE_BLOCKS; a.lo = blk_lo; a.hi = blk_hi; a.uni = uni; a.out = fits_out;
    return stage_call(X, n, p, ld, h, opt, workspace, ws_bytes, stream, a);
}

int rtdetmcd_reweight_moments(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                              const double* uni, const double* fits, int32_t blk_lo, int32_t blk_hi,
                              void* workspace, size_t ws_bytes, void* stream, double* moments_out) {
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = STAGE_MOMENTS; a.lo = blk_lo; a.hi = blk_hi; a.uni = uni; a.fits = fits; a.out = moments_out;
    return stage_call(X, n, p, ld, h, opt, workspace, ws_bytes, stream, a);
}

int rtdetmcd_reweight_finish(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                             const double* uni, const double* fits, const double* moments, int64_t row_lo,
                             int64_t row_hi, void* workspace, size_t ws_bytes, void* stream, rtd_result* out,
                             float* d2_out, uint8_t* flags_out) {
    if (!out) return RTD_EINVAL;
    memset(out, 0, sizeof(*out));
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = STAGE_FINISH; a.lo = row_lo; a.hi = row_hi; a.uni = uni; a.fits = fits; a.moments = moments;
    a.res = out; a.d2 = d2_out; a.fl = flags_out;
    int r = stage_call(X, n, p, ld, h, opt, workspace, ws_bytes, stream, a);
    out->status = r;
    return r;
}

size_t rtdetmcd_fit_batch_workspace_size(int32_t nframes, const int64_t* n, const int32_t* p,
                                         const rtd_options* opt, int32_t nstreams) {
    if (nframes < 1 || !n || !p || nstreams < 1 || nstreams > RTD_BATCH_MAX_STREAMS) return 0;
    rtd_options o = opt ? *opt : defaults();
    size_t slice = 0;
    for (int f = 0; f < nframes; ++f) {
        Shape S;
        if (make_shape(n[f], p[f], p[f], (n[f] + p[f] + 1) / 2, o, S) != RTD_OK) return 0;
        Regions R;
        size_t b = layout(S, R);
        if (b > slice) slice = b;
    }
    slice = (slice + 255) & ~(size_t)255;
    return slice * (size_t)(nstreams < nframes ? nstreams : nframes);
}

int rtdetmcd_fit_batch(int32_t nframes, const float* const* X, const int64_t* n, const int32_t* p,
                       const int64_t* ld, const int64_t* h, const rtd_options* opt, void* workspace,
                       size_t ws_bytes, void* stream, int32_t nstreams, rtd_result* out, float* const* d2_out,
                       uint8_t* const* flags_out) {
    if (nframes < 1 || !X || !n || !p || !ld || !h || !out || nstreams < 1 || nstreams > RTD_BATCH_MAX_STREAMS)
        return RTD_EINVAL;
    rtd_options o = opt ? *opt : defaults();
    o.subset_out = nullptr;    // per-frame outputs of the single-fit options do not apply
    o.diag_out = nullptr;
    o.profile = nullptr;
    // every frame is checked before any device work
    std::vector<Shape> shapes((size_t)nframes);
    int bad = RTD_OK;
    for (int f = 0; f < nframes; ++f) {
        memset(&out[f], 0, sizeof(rtd_result));
        int e = make_shape(n[f], p[f], ld[f], h[f], o, shapes[f]);
        if (!e) e = check_h(shapes[f]);
        if (!X[f]) e = RTD_EINVAL;
        out[f].status = e;
        if (e && !bad) bad = e;
    }
    if (bad) return bad;
    const int nw = nstreams < nframes ? nstreams : nframes;
    const size_t need = rtdetmcd_fit_batch_workspace_size(nframes, n, p, &o, nstreams);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    const size_t slice = need / (size_t)nw;
    int dev = 0;
    RTD_CUDA(cudaGetDevice(&dev));
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    if (o.graph == 1 && o.autotune == 1) {
        // tune each class of frames (same tuning key) that has no choice yet,
        // on the frame of median size in the class, before the pool starts
        std::vector<int> todo;
        for (int f = 0; f < nframes; ++f) {
            TuneVal v;
            if (!tune_get(tune_key(shapes[f], o, dev), v)) todo.push_back(f);
        }
        while (!todo.empty()) {
            const TuneKey k0 = tune_key(shapes[todo[0]], o, dev);
            std::vector<int> cls, rest;
            for (int f : todo) {
                const TuneKey kf = tune_key(shapes[f], o, dev);
                (memcmp(&kf, &k0, sizeof(TuneKey)) == 0 ? cls : rest).push_back(f);
            }
            std::sort(cls.begin(), cls.end(), [&](int a, int b) { return n[a] < n[b]; });
            const int f = cls[cls.size() / 2];
            if (is_device_ptr(X[f])) {
                const int e = autotune_shape(X[f], shapes[f], o, workspace, caller, nullptr);
                if (e) return e;
            }
            todo.swap(rest);
        }
    }
    // the workers' streams start after the caller's earlier work
    cudaEvent_t ready;
    RTD_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    RTD_CUDA(cudaEventRecord(ready, caller));
    std::vector<cudaStream_t> ss((size_t)nw, nullptr);
    int serr = RTD_OK;
    for (int w = 0; w < nw; ++w) {
        if (cudaStreamCreateWithFlags(&ss[w], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(ss[w], ready, 0) != cudaSuccess) {
            serr = RTD_ECUDA;
            break;
        }
    }
    if (!serr) {
        // frames are taken in order from a shared counter, so that workers
        // stay busy whatever the mix of frame sizes
        std::atomic<int> next(0);
        auto worker = [&](int w) {
            cudaSetDevice(dev);
            void* wsw = static_cast<unsigned char*>(workspace) + slice * (size_t)w;
            for (int f = next.fetch_add(1); f < nframes; f = next.fetch_add(1)) {
                float* d2f = d2_out ? d2_out[f] : nullptr;
                uint8_t* flf = flags_out ? flags_out[f] : nullptr;
                int r = -1;
                if (o.graph == 1) r = run_fit_graph(X[f], shapes[f], o, wsw, ss[w], &out[f], d2f, flf);
                if (r == -1) r = run_fit(X[f], shapes[f], o, wsw, ss[w], &out[f], d2f, flf);
                out[f].status = r;
            }
        };
        std::vector<std::thread> th;
        for (int w = 1; w < nw; ++w) th.emplace_back(worker, w);
        worker(0);
        for (auto& t : th) t.join();
    }
    for (int w = 0; w < nw; ++w)
        if (ss[w]) cudaStreamDestroy(ss[w]);
    cudaEventDestroy(ready);
    if (serr) return serr;
    for (int f = 0; f < nframes; ++f)
        if (out[f].status) return out[f].status;
    return RTD_OK;
}

size_t rtdetmcd_distances_workspace_size(int64_t n, int32_t p) {
    if (n < 1 || p < 1 || p > RTD_MAX_P) return 0;
    Layout L;
    L.add(sizeof(Status));
    L.add(sizeof(RowParams));
    L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));
    L.add((size_t)n * p * sizeof(float));
    L.add((size_t)n * sizeof(float));
    return (L.total + 255) & ~(size_t)255;
}

int rtdetmcd_distances(const float* X, int64_t n, int32_t p, int64_t ld, const double* mu_host,
                       const double* sigma_host, int32_t precision, float* d2_out, void* workspace,
                       size_t ws_bytes, void* stream) {
    if (!X || !mu_host || !sigma_host || !d2_out || n < 1 || p < 1 || p > RTD_MAX_P || ld < p ||
        (precision != RTD_FP32 && precision != RTD_FP64) || n >= (1LL << 31))
        return RTD_EINVAL;
    size_t need = rtdetmcd_distances_workspace_size(n, p);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    if (on_other_device(X) || on_other_device(d2_out) || on_other_device(workspace)) return RTD_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rrp = L.add(sizeof(RowParams));
    Region rms = L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));
    Region rxs = L.add((size_t)n * p * sizeof(float));
    Region rds = L.add((size_t)n * sizeof(float));
    Status* st = at<Status>(workspace, rst);
    RowParams* rp = at<RowParams>(workspace, rrp);
    double* ms = at<double>(workspace, rms);
    RTD_CUDA(cudaMemsetAsync(st, 0, sizeof(Status), s));
    RTD_CUDA(cudaMemcpyAsync(ms, mu_host, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, s));
    RTD_CUDA(cudaMemcpyAsync(ms + RTD_MAX_P, sigma_host, (size_t)p * p * sizeof(double), cudaMemcpyHostToDevice, s));
    const float* Xd = X;
    long long ldd = ld;
    if (!is_device_ptr(X)) {
        float* xs = at<float>(workspace, rxs);
        if (ld == p)
            RTD_CUDA(cudaMemcpyAsync(xs, X, (size_t)n * p * sizeof(float), cudaMemcpyHostToDevice, s));
        else
            RTD_CUDA(cudaMemcpy2DAsync(xs, (size_t)p * sizeof(float), X, (size_t)ld * sizeof(float),
                                       (size_t)p * sizeof(float), (size_t)n, cudaMemcpyHostToDevice, s));
        Xd = xs;
        ldd = p;
    }
    bool ddev = is_device_ptr(d2_out);
    float* d2 = ddev ? d2_out : at<float>(workspace, rds);
    launch_score_prep(ms, ms + RTD_MAX_P, p, rp, st, s);
    launch_score(Xd, n, p, ldd, rp, precision, d2, s);
    if (!ddev) RTD_CUDA(cudaMemcpyAsync(d2_out, d2, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    Status hs;
    int e = fetch_status(st, s, hs);
    if (e) return e;
    return hs.code;
}

size_t rtdetmcd_score_workspace_size(int64_t n, int32_t p) {
    if (n < 1 || p < 1 || p > RTD_MAX_P) return 0;
    Layout L;
    L.add(sizeof(Status));
    L.add(sizeof(RowParams));
    L.add(sizeof(double));
    L.add((size_t)n * p * sizeof(float));
    L.add((size_t)n * sizeof(float));
    L.add((size_t)n);
    return (L.total + 255) & ~(size_t)255;
}

int rtdetmcd_score(const float* X, int64_t n, int32_t p, int64_t ld, const double* mu_host,
                   const double* sigma_host, double cutoff_d2, int32_t precision, float* d2_out,
                   uint8_t* flags_out, int64_t* n_flagged, void* workspace, size_t ws_bytes, void* stream) {
    if (!X || !mu_host || !sigma_host || n < 1 || p < 1 || p > RTD_MAX_P || ld < p ||
        (precision != RTD_FP32 && precision != RTD_FP64) || n >= (1LL << 31) || !(cutoff_d2 == cutoff_d2))
        return RTD_EINVAL;
    size_t need = rtdetmcd_score_workspace_size(n, p);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    if (on_other_device(X) || on_other_device(d2_out) || on_other_device(flags_out) || on_other_device(workspace))
        return RTD_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rrp = L.add(sizeof(RowParams));
    Region rcut = L.add(sizeof(double));
    Region rxs = L.add((size_t)n * p * sizeof(float));
    Region rds = L.add((size_t)n * sizeof(float));
    Region rfs = L.add((size_t)n);
    Status* st = at<Status>(workspace, rst);
    RowParams* rp = at<RowParams>(workspace, rrp);
    // the fit travels in the launch parameters: no copy precedes the stream
    FitArg a;
    for (int j = 0; j < p; ++j) a.mu[j] = mu_host[j];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j <= i; ++j) a.tri[i * (i + 1) / 2 + j] = sigma_host[(size_t)i * p + j];
    const float* Xd = X;
    long long ldd = ld;
    if (!is_device_ptr(X)) {
        float* xs = at<float>(workspace, rxs);
        if (ld == p)
            RTD_CUDA(cudaMemcpyAsync(xs, X, (size_t)n * p * sizeof(float), cudaMemcpyHostToDevice, s));
        else
            RTD_CUDA(cudaMemcpy2DAsync(xs, (size_t)p * sizeof(float), X, (size_t)ld * sizeof(float),
                                       (size_t)p * sizeof(float), (size_t)n, cudaMemcpyHostToDevice, s));
        Xd = xs;
        ldd = p;
    }
    const bool ddev = !d2_out || is_device_ptr(d2_out), fdev = !flags_out || is_device_ptr(flags_out);
    float* d2 = d2_out ? (ddev ? d2_out : at<float>(workspace, rds)) : nullptr;
    uint8_t* fl = flags_out ? (fdev ? flags_out : at<uint8_t>(workspace, rfs)) : nullptr;
    launch_score_prep_arg(a, p, cutoff_d2, rp, st, at<double>(workspace, rcut), s);
    launch_score_flags(Xd, n, p, ldd, rp, precision, at<double>(workspace, rcut), st, d2, fl,
                       &st->n_flagged, s);
    if (d2_out && !ddev) RTD_CUDA(cudaMemcpyAsync(d2_out, d2, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (flags_out && !fdev) RTD_CUDA(cudaMemcpyAsync(flags_out, fl, (size_t)n, cudaMemcpyDeviceToHost, s));
    Status hs;
    int e = fetch_status(st, s, hs);
    if (e) return e;
    if (n_flagged) *n_flagged = flags_out ? (int64_t)hs.n_flagged : -1;
    return hs.code;
}

// A prepared fit: the status word, the row parameters and the cutoff, laid
// out as the first three regions of the scoring workspace.
size_t rtdetmcd_prepared_size(void) {
    Layout L;
    L.add(sizeof(Status));
    L.add(sizeof(RowParams));
    L.add(sizeof(double));
    return (L.total + 255) & ~(size_t)255;
}

int rtdetmcd_score_prepare(const double* mu_host, const double* sigma_host, int32_t p, double cutoff_d2,
                           void* prepared, void* stream) {
    if (!mu_host || !sigma_host || p < 1 || p > RTD_MAX_P || !std::isfinite(cutoff_d2)) return RTD_EINVAL;
    if (!prepared || (reinterpret_cast<uintptr_t>(prepared) & 255) || !is_device_ptr(prepared) ||
        on_other_device(prepared))
        return RTD_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rrp = L.add(sizeof(RowParams));
    Region rcut = L.add(sizeof(double));
    FitArg a;
    for (int j = 0; j < p; ++j) a.mu[j] = mu_host[j];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j <= i; ++j) a.tri[i * (i + 1) / 2 + j] = sigma_host[(size_t)i * p + j];
    Status* st = at<Status>(prepared, rst);
    launch_score_prep_arg(a, p, cutoff_d2, at<RowParams>(prepared, rrp), st, at<double>(prepared, rcut), s);
    Status hs;
    int e = fetch_status(st, s, hs);
    return e ? e : hs.code;
}

int rtdetmcd_score_prepared(const float* X, int64_t n, int32_t p, int64_t ld, const void* prepared,
                            int32_t precision, float* d2_out, uint8_t* flags_out, unsigned long long* count,
                            void* stream) {
    if (!X || !prepared || n < 1 || n >= (1LL << 31) || p < 1 || p > RTD_MAX_P || ld < p ||
        (precision != RTD_FP32 && precision != RTD_FP64) || (reinterpret_cast<uintptr_t>(prepared) & 255))
        return RTD_EINVAL;
    if (count && !flags_out) return RTD_EINVAL;
    int dev = 0;
    RTD_CUDA(cudaGetDevice(&dev));
    const void* dev_ptrs[5] = {X, prepared, d2_out, flags_out, count};
    for (const void* q : dev_ptrs) {   // device memory of the current device, one query each
        if (!q) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, q) != cudaSuccess) { cudaGetLastError(); return RTD_EINVAL; }
        if (a.type != cudaMemoryTypeDevice || a.device != dev) return RTD_EINVAL;
    }
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rrp = L.add(sizeof(RowParams));
    Region rcut = L.add(sizeof(double));
    void* pp = const_cast<void*>(prepared);
    launch_score_flags(X, n, p, ld, at<RowParams>(pp, rrp), precision, at<double>(pp, rcut), at<Status>(pp, rst),
                       d2_out, flags_out, count, reinterpret_cast<cudaStream_t>(stream));
    RTD_CUDA(cudaGetLastError());
    return RTD_OK;
}

size_t rtdetmcd_grad_workspace_size(int64_t n, int32_t p) {
    if (n < 1 || p < 1 || p > RTD_MAX_P) return 0;
    const size_t slot_d = (size_t)gram_nblk(pad_p(p)) * 16 + 2;
    Layout L;
    L.add(sizeof(Status));
    L.add(sizeof(RowParams));
    L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));
    L.add((size_t)GRAD_SLOTS * slot_d * sizeof(double));
    L.add(slot_d * sizeof(double));
    L.add(sizeof(double));
    L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));   // cotangents on mu and Sigma
    return (L.total + 255) & ~(size_t)255;
}

namespace {

// The adjoint passes of rtdetmcd_grad and rtdetmcd_vjp: device cotangents
// `grd` (nullable), host cotangents gmu (p) / gsig (p x p) (nullable).
int grad_impl(const float* X, int64_t n, int32_t p, int64_t ld, const uint8_t* wset, int32_t wbit,
              const double* mu_host, const double* sigma_host, double c, double w_logdet, double w_rd,
              const float* grd, const double* gmu_host, const double* gsig_host, double* value_out,
              float* grad_out, void* workspace, size_t ws_bytes, void* stream) {
    size_t need = rtdetmcd_grad_workspace_size(n, p);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    if (on_other_device(X) || on_other_device(wset) || on_other_device(grad_out) || on_other_device(workspace) ||
        on_other_device(grd))
        return RTD_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t slot_d = (size_t)gram_nblk(pad_p(p)) * 16 + 2;
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rrp = L.add(sizeof(RowParams));
    Region rms = L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));
    Region rpa = L.add((size_t)GRAD_SLOTS * slot_d * sizeof(double));
    Region rto = L.add(slot_d * sizeof(double));
    Region rld = L.add(sizeof(double));
    Region rcot = L.add((size_t)RTD_MAX_P * (RTD_MAX_P + 1) * sizeof(double));
    Status* st = at<Status>(workspace, rst);
    RowParams* rp = at<RowParams>(workspace, rrp);
    double* ms = at<double>(workspace, rms);
    double* tot = at<double>(workspace, rto);
    double* ldv = at<double>(workspace, rld);
    double* cot = at<double>(workspace, rcot);
    int dev = 0, nsm = 0;
    RTD_CUDA(cudaGetDevice(&dev));
    RTD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    RTD_CUDA(cudaMemsetAsync(st, 0, sizeof(Status), s));
    RTD_CUDA(cudaMemcpyAsync(ms, mu_host, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, s));
    RTD_CUDA(cudaMemcpyAsync(ms + RTD_MAX_P, sigma_host, (size_t)p * p * sizeof(double), cudaMemcpyHostToDevice, s));
    GradCot gc{grd, nullptr, nullptr};
    if (gmu_host) {
        RTD_CUDA(cudaMemcpyAsync(cot, gmu_host, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, s));
        gc.gmu = cot;
    }
    if (gsig_host) {
        RTD_CUDA(cudaMemcpyAsync(cot + RTD_MAX_P, gsig_host, (size_t)p * p * sizeof(double), cudaMemcpyHostToDevice,
                                 s));
        gc.gsig = cot + RTD_MAX_P;
    }
    launch_score_prep(ms, ms + RTD_MAX_P, p, rp, st, s, ldv);
    launch_grad(X, n, p, ld, wset, (int)wbit, rp, at<double>(workspace, rpa), slot_d, tot, c, w_logdet, w_rd, gc,
                grad_out, nsm, s);
    RTD_CUDA(cudaGetLastError());
    double h[3];
    RTD_CUDA(cudaMemcpyAsync(h, tot + slot_d - 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    RTD_CUDA(cudaMemcpyAsync(h + 2, ldv, sizeof(double), cudaMemcpyDeviceToHost, s));
    Status hs;
    int e = fetch_status(st, s, hs);
    if (e) return e;
    if (hs.code) return hs.code;
    // |W| must allow a non-singular covariance
    if (h[1] < (double)p + 1.0) return RTD_EDEGENERATE;
    if (value_out) *value_out = w_logdet * h[2] + w_rd * h[0];
    return RTD_OK;
}

bool finite_all(const double* a, size_t k) {
    for (size_t i = 0; i < k; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace

int rtdetmcd_grad(const float* X, int64_t n, int32_t p, int64_t ld, const uint8_t* wset, int32_t wbit,
                  const double* mu_host, const double* sigma_host, double c, double w_logdet, double w_rd,
                  double* value_out, float* grad_out, void* workspace, size_t ws_bytes, void* stream) {
    if (!X || !wset || !mu_host || !sigma_host || n < 2 || p < 1 || p > RTD_MAX_P || ld < p || wbit < 0 ||
        wbit > 7 || !(c > 0.0) || !std::isfinite(c) || !std::isfinite(w_logdet) || !std::isfinite(w_rd) ||
        !is_device_ptr(X) || !is_device_ptr(wset) || (grad_out && !is_device_ptr(grad_out)))
        return RTD_EINVAL;
    return grad_impl(X, n, p, ld, wset, wbit, mu_host, sigma_host, c, w_logdet, w_rd, nullptr, nullptr, nullptr,
                     value_out, grad_out, workspace, ws_bytes, stream);
}

int rtdetmcd_vjp(const float* X, int64_t n, int32_t p, int64_t ld, const uint8_t* wset, int32_t wbit,
                 const double* mu_host, const double* sigma_host, double c, const double* gmu_host,
                 const double* gsigma_host, double g_logdet, const float* grd, float* grad_out, void* workspace,
                 size_t ws_bytes, void* stream) {
    if (!X || !wset || !mu_host || !sigma_host || !grad_out || n < 2 || p < 1 || p > RTD_MAX_P || ld < p ||
        wbit < 0 || wbit > 7 || !(c > 0.0) || !std::isfinite(c) || !std::isfinite(g_logdet) || !is_device_ptr(X) ||
        !is_device_ptr(wset) || !is_device_ptr(grad_out) || (grd && !is_device_ptr(grd)))
        return RTD_EINVAL;
    if ((gmu_host && !finite_all(gmu_host, (size_t)p)) || (gsigma_host && !finite_all(gsigma_host, (size_t)p * p)))
        return RTD_EINVAL;
    // without a cotangent on RD its rows carry weight zero
    return grad_impl(X, n, p, ld, wset, wbit, mu_host, sigma_host, c, g_logdet, 0.0, grd, gmu_host, gsigma_host,
                     nullptr, grad_out, workspace, ws_bytes, stream);
}

int rtdetmcd_flag(const float* d2, int64_t n, double cutoff_d2, uint8_t* flags_out, int64_t* n_flagged,
                  void* workspace, size_t ws_bytes, void* stream) {
    if (!d2 || n < 1 || !(cutoff_d2 == cutoff_d2)) return RTD_EINVAL;
    Layout L;
    Region rst = L.add(sizeof(Status));
    Region rd = L.add((size_t)n * sizeof(float));
    Region rf = L.add((size_t)n);
    bool d2dev = is_device_ptr(d2), fdev = is_device_ptr(flags_out);
    size_t need = 256;
    if (!d2dev || (flags_out && !fdev)) need = (L.total + 255) & ~(size_t)255;
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Status* st = at<Status>(workspace, rst);
    RTD_CUDA(cudaMemsetAsync(st, 0, sizeof(Status), s));
    const float* dd = d2;
    if (!d2dev) {
        float* ds = at<float>(workspace, rd);
        RTD_CUDA(cudaMemcpyAsync(ds, d2, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s));
        dd = ds;
    }
    uint8_t* fl = flags_out ? (fdev ? flags_out : at<uint8_t>(workspace, rf)) : nullptr;
    launch_flag(dd, n, cutoff_d2, fl, &st->n_flagged, s);
    if (flags_out && !fdev) RTD_CUDA(cudaMemcpyAsync(flags_out, fl, (size_t)n, cudaMemcpyDeviceToHost, s));
    Status hs;
    int e = fetch_status(st, s, hs);
    if (e) return e;
    if (n_flagged) *n_flagged = (int64_t)hs.n_flagged;
    return hs.code;
}

int rtdetmcd_autotune(const float* X, int64_t n, int32_t p, int64_t ld, int64_t h, const rtd_options* opt,
                      void* workspace, size_t ws_bytes, void* stream, rtd_tuning* out) {
    rtd_options o = opt ? *opt : defaults();
    o.subset_out = nullptr;
    o.diag_out = nullptr;
    o.profile = nullptr;
    Shape S;
    int e = make_shape(n, p, ld, h, o, S);
    if (!e) e = check_h(S);
    if (!X || !is_device_ptr(X)) e = RTD_EINVAL;
    if (e) return e;
    Regions R;
    size_t need = layout(S, R);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return RTD_EWORKSPACE;
    if (on_other_device(X) || on_other_device(workspace)) return RTD_EINVAL;
    return autotune_shape(X, S, o, workspace, reinterpret_cast<cudaStream_t>(stream), out);
}

int rtdetmcd_tuned(int64_t n, int32_t p, const rtd_options* opt, rtd_tuning* out) {
    rtd_options o = opt ? *opt : defaults();
    Shape S;
    if (make_shape(n, p, p, (n + p + 1) / 2, o, S) != RTD_OK) return 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
    TuneVal v;
    if (!tune_get(tune_key(S, o, dev), v)) return 0;
    if (out) {
        memset(out, 0, sizeof(*out));
        out->win_rows = v.win_rows;
        out->sel_ctas = v.sel_ctas;
    }
    return 1;
}

double rtdetmcd_chi2_quantile(int32_t p, double q) {
    if (p < 1) return NAN;
    return chi2_quantile(p, q);
}

const char* rtdetmcd_status_string(int status) {
    switch (status) {
        case RTD_OK: return "ok";
        case RTD_EINVAL: return "invalid argument";
        case RTD_ENONFINITE: return "non-finite value in the rows";
        case RTD_EILLCOND: return "every start of every block was ill-conditioned";
        case RTD_EDEGENERATE: return "degenerate data (zero scale or singular scatter)";
        case RTD_EWORKSPACE: return "workspace too small or misaligned";
        case RTD_ECUDA: return "CUDA runtime error";
        case RTD_EINTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

}  // extern "C"
