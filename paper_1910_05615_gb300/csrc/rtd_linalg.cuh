// rtd_linalg.cuh - CTA-cooperative FP64 dense algebra for p x p matrices
// (p <= 64) held in shared memory with leading dimension LD.
#pragma once
#include "rtd_common.cuh"

namespace rtd {

constexpr int LD = PMAX + 1;   // padded leading dimension of shared matrices

// In-place Cholesky A = L L^T (lower triangle overwritten by L; the strict
// upper triangle is zeroed); rdiag (optional) receives 1 / L_kk.  Returns
// false (uniformly) if A is not numerically positive definite.
// Computed as A = U D U^T (U unit lower) and scaled to L = U D^{1/2} at the
// end, so the column-to-column chain holds one FP64 reciprocal per pivot and
// no square root (FP64 square roots are long dependent sequences on this
// GPU; the p square roots of the final scaling run in parallel).
// Right-looking, one barrier per column: step k updates the trailing block
// from the unscaled column k and scales column k - 1 (no thread reads it any
// more); the next pivot's reciprocal is taken once, by the thread that
// updates that diagonal entry, and passed on in shared memory.
__device__ inline bool cta_cholesky(double* A, int p, double* rdiag = nullptr) {
    __shared__ double piv[2];       // 1 / D_k by column parity
    __shared__ double sd[PMAX];
    __shared__ int bad;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double a = A[0];
        bad = !(a > 0.0) || !isfinite(a);
        if (!bad) piv[0] = 1.0 / a;
    }
    __syncthreads();
    if (bad) return false;
    double rprev = 0.0;   // 1 / D_{k-1}, kept in registers
    for (int k = 0; k < p; ++k) {
        // piv[k & 1] was written before the last barrier; piv[(k + 1) & 1] is written below
        const double rk = piv[k & 1];
        if (k > 0)
            for (int i = k + threadIdx.x; i < p; i += blockDim.x) A[i * LD + (k - 1)] *= rprev;
        const int rem = p - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            if (j <= i) {
                const double v = A[i * LD + j] - A[i * LD + k] * A[j * LD + k] * rk;
                A[i * LD + j] = v;
                if (e == 0) {   // (k+1, k+1): the next pivot D_{k+1}
                    if (!(v > 0.0) || !isfinite(v)) bad = 1;
                    else piv[(k + 1) & 1] = 1.0 / v;
                }
            }
        }
        rprev = rk;
        __syncthreads();
        if (bad) return false;
    }
    // L = U D^{1/2}
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const double d = sqrt(A[j * LD + j]);
        sd[j] = d;
        if (rdiag) rdiag[j] = 1.0 / d;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int i = e / p, j = e % p;
        if (j < i) A[i * LD + j] *= sd[j];
        else if (j == i) A[i * LD + j] = sd[j];
        else A[i * LD + j] = 0.0;
    }
    __syncthreads();
    return true;
}

// Li = L^-1 for lower-triangular L (column-parallel forward substitution
// with the reciprocal diagonal).
__device__ inline void cta_tri_inverse(const double* L, double* Li, int p, const double* rdiag = nullptr) {
    __shared__ double rdl[PMAX];
    const double* rd = rdiag;
    if (!rd) {
        for (int j = threadIdx.x; j < p; j += blockDim.x) rdl[j] = 1.0 / L[j * LD + j];
        __syncthreads();
        rd = rdl;
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        for (int i = 0; i < j; ++i) Li[i * LD + j] = 0.0;
        Li[j * LD + j] = rd[j];
        for (int i = j + 1; i < p; ++i) {
            double s0 = 0.0, s1 = 0.0;
            int k = j;
            for (; k + 1 < i; k += 2) {
                s0 = fma(L[i * LD + k], Li[k * LD + j], s0);
                s1 = fma(L[i * LD + k + 1], Li[(k + 1) * LD + j], s1);
            }
            if (k < i) s0 = fma(L[i * LD + k], Li[k * LD + j], s0);
            Li[i * LD + j] = -(s0 + s1) * rd[i];
        }
    }
    __syncthreads();
}

// Block-wide reductions (blockDim.x a multiple of 32, <= 1024).
__device__ inline double cta_sum(double v) {
    __shared__ double red[32];
    v = warp_sum_d(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < nw) ? red[l] : 0.0;
        r = warp_sum_d(r);
        if (l == 0) red[0] = r;
    }
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}
__device__ inline double cta_max(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    double r = -INFINITY;
    if (threadIdx.x < 32) {
        r = (l < nw) ? red[l] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (l == 0) red[0] = r;
    }
    __syncthreads();
    r = red[0];
    __syncthreads();
    return r;
}

// kappa_1 = ||S||_1 ||S^-1||_1 with S^-1 = Li^T Li (Section 3.4), from the
// FP64 factors but summed in FP32: the monitor only compares kappa_1 with
// kappa_max, and FP32 keeps the dependent sums off the (slow) FP64 pipe.
// W is a p x p shared scratch matrix (as floats).
__device__ inline float cta_max_f(float v) {
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    float r = 0.f;
    for (int k = 0; k < nw; ++k) r = fmaxf(r, red[k]);
    __syncthreads();
    return r;
}
__device__ inline double cta_kappa1(const double* S, const double* Li, double* Wd, int p) {
    float* W = reinterpret_cast<float*>(Wd);        // p x LD floats
    float* Lf = W + PMAX * LD;                      // FP32 copy of Li (same shared block)
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        Lf[i * LD + j] = (float)Li[i * LD + j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        int k0 = i > j ? i : j;
        float v = 0.f;
        for (int k = k0; k < p; ++k) v = fmaf(Lf[k * LD + i], Lf[k * LD + j], v);
        W[i * LD + j] = v;
    }
    __syncthreads();
    float n1 = 0.f, n1i = 0.f;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        float cs = 0.f, csi = 0.f;
        for (int i = 0; i < p; ++i) { cs += fabsf((float)S[i * LD + j]); csi += fabsf(W[i * LD + j]); }
        n1 = fmaxf(n1, cs);
        n1i = fmaxf(n1i, csi);
    }
    n1 = cta_max_f(n1);
    n1i = cta_max_f(n1i);
    return (double)n1 * (double)n1i;
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations in the
// round-robin (tournament) order, so that the p/2 rotations of one round act
// on disjoint index pairs and are applied in parallel.  On return A's
// diagonal holds the eigenvalues, V (columns) the eigenvectors; lam/Vs hold
// them sorted by decreasing eigenvalue.
// The same round-robin sweeps entirely in FP32 (A and V of p x LD floats),
// until the off-diagonal norm is below 1e-6 of the diagonal's or `sweeps`
// run out: the cheap first stage of cta_jacobi.
__device__ inline void jacobi_sweeps_f32(float* A, float* V, int p, int sweeps) {
    __shared__ float fc[PMAX / 2 + 1], fs[PMAX / 2 + 1];
    __shared__ int fi[PMAX / 2 + 1], fj[PMAX / 2 + 1];
    const int P = p + (p & 1);
    const int half = P / 2;
    for (int sweep = 0; sweep < sweeps && p > 1; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            double a = (double)A[i * LD + j];
            if (i != j) off += a * a; else dg += a * a;
        }
        off = cta_sum(off);
        dg = cta_sum(dg);
        if (off <= 1e-12 * dg || off == 0.0) break;
        for (int round = 0; round < P - 1; ++round) {
            if (threadIdx.x < half) {
                int k = threadIdx.x;
                int a = (k == 0) ? 0 : 1 + (k - 1 + round) % (P - 1);
                int b = 1 + (P - 2 - k + round) % (P - 1);
                int i = a < b ? a : b, j = a < b ? b : a;
                float c = 1.f, sn = 0.f;
                if (j < p) {
                    const float aij = A[i * LD + j];
                    if (aij != 0.f) {
                        const float d = A[j * LD + j] - A[i * LD + i];
                        const float q = sqrtf(fmaf(d, d, 4.f * aij * aij));
                        float t = 2.f * aij / (fabsf(d) + q);
                        if (d < 0.f) t = -t;
                        if (isfinite(t) && q > 0.f) {
                            c = rsqrtf(fmaf(t, t, 1.f));
                            sn = t * c;
                        }
                    }
                }
                fc[k] = c; fs[k] = sn; fi[k] = i; fj[k] = (j < p) ? j : -1;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
                int k = e / p, r = e % p;
                int i = fi[k], j = fj[k];
                if (j < 0 || fs[k] == 0.f) continue;
                float c = fc[k], sn = fs[k];
                float a = A[r * LD + i], b = A[r * LD + j];
                A[r * LD + i] = c * a - sn * b;
                A[r * LD + j] = sn * a + c * b;
                a = V[r * LD + i]; b = V[r * LD + j];
                V[r * LD + i] = c * a - sn * b;
                V[r * LD + j] = sn * a + c * b;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
                int k = e / p, r = e % p;
                int i = fi[k], j = fj[k];
                if (j < 0 || fs[k] == 0.f) continue;
                float c = fc[k], sn = fs[k];
                float a = A[i * LD + r], b = A[j * LD + r];
                A[i * LD + r] = c * a - sn * b;
                A[j * LD + r] = sn * a + c * b;
            }
            __syncthreads();
            if (threadIdx.x < half) {
                int k = threadIdx.x;
                if (fj[k] >= 0 && fs[k] != 0.f) A[fj[k] * LD + fi[k]] = A[fi[k] * LD + fj[k]];
            }
            __syncthreads();
        }
    }
}

// C = op(X) Y for p x p shared matrices (leading dimension LD), op = X^T when tx
__device__ inline void cta_matmul(const double* X, const double* Y, double* C, int p, bool tx) {
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        double v = 0.0;
        for (int k = 0; k < p; ++k) v = fma(tx ? X[k * LD + i] : X[i * LD + k], Y[k * LD + j], v);
        C[i * LD + j] = v;
    }
    __syncthreads();
}

// Symmetric eigen-decomposition in two stages.  FP32 sweeps bring A close to
// diagonal; their rotations V32 are made orthogonal to FP64 precision by two
// Newton-Schulz steps V <- V (3 I - V^T V) / 2, A is replaced by V^T A V in
// FP64, and the FP64 sweeps of cta_jacobi finish (one or two sweeps, as the
// convergence is quadratic).  T is a fourth p x LD double scratch matrix.
__device__ inline void cta_jacobi(double* A, double* V, int p, double* lam, double* Vs, double* T);

__device__ inline void cta_jacobi_mixed(double* A, double* V, int p, double* lam, double* Vs, double* T) {
    float* A32 = reinterpret_cast<float*>(T);
    float* V32 = A32 + PMAX * LD;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        A32[i * LD + j] = (float)A[i * LD + j];
        V32[i * LD + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    jacobi_sweeps_f32(A32, V32, p, 30);
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        V[i * LD + j] = (double)V32[i * LD + j];
    }
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        cta_matmul(V, V, Vs, p, true);                       // G = V^T V
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            Vs[i * LD + j] = ((i == j) ? 1.5 : 0.0) - 0.5 * Vs[i * LD + j];
        }
        __syncthreads();
        cta_matmul(V, Vs, T, p, false);                      // V (3 I - G) / 2
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            V[i * LD + j] = T[i * LD + j];
        }
        __syncthreads();
    }
    cta_matmul(A, V, T, p, false);                           // A V
    cta_matmul(V, T, A, p, true);                            // V^T A V
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {  // exact symmetry
        int i = e / p, j = e % p;
        if (i < j) A[j * LD + i] = A[i * LD + j];
    }
    __syncthreads();
    cta_jacobi(A, V, p, lam, Vs, nullptr);
}

// T == nullptr: V already holds the rotations so far (cta_jacobi_mixed);
// otherwise V starts as the identity.
__device__ inline void cta_jacobi(double* A, double* V, int p, double* lam, double* Vs, double* T) {
    __shared__ double rc[PMAX / 2 + 1], rs[PMAX / 2 + 1];
    __shared__ int ri[PMAX / 2 + 1], rj[PMAX / 2 + 1];
    __shared__ int order[PMAX];
    if (T) {
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            V[i * LD + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    __syncthreads();
    const int P = p + (p & 1);
    const int half = P / 2;
    for (int sweep = 0; sweep < 40 && p > 1; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
            int i = e / p, j = e % p;
            double a = A[i * LD + j];
            if (i != j) off += a * a; else dg += a * a;
        }
        off = cta_sum(off);
        dg = cta_sum(dg);
        // converged: off-diagonal norm below 1e-14 of the diagonal norm
        if (off <= 1e-28 * dg || off == 0.0) break;
        for (int round = 0; round < P - 1; ++round) {
            if (threadIdx.x < half) {
                int k = threadIdx.x;
                // positions: 0 fixed, others rotate
                int a = (k == 0) ? 0 : 1 + (k - 1 + round) % (P - 1);
                int b = 1 + (P - 2 - k + round) % (P - 1);
                int i = a < b ? a : b, j = a < b ? b : a;
                double c = 1.0, s = 0.0;
                if (j < p) {
                    double aij = A[i * LD + j];
                    if (aij != 0.0) {
                        // t = tan(theta) solves t^2 + 2 tau t - 1 = 0, tau = (a_jj - a_ii) / (2 a_ij),
                        // smaller root: t = sgn(d) 2 a_ij / (|d| + sqrt(d^2 + 4 a_ij^2)), d = a_jj - a_ii.
                        // The angle is taken in FP32 (FP64 square roots and divisions are
                        // long on this GPU); (c, s) is then normalised in FP64 by two
                        // first-order steps, so the rotation is orthogonal to FP64 precision
                        // and whatever the FP32 angle leaves of a_ij goes in the next sweep.
                        const double d = A[j * LD + j] - A[i * LD + i];
                        const float df = (float)d, cf = (float)aij;
                        const float q = sqrtf(fmaf(df, df, 4.f * cf * cf));
                        float tf = 2.f * cf / (fabsf(df) + q);
                        if (df < 0.f) tf = -tf;
                        if (isfinite(tf) && q > 0.f) {
                            const float cr = rsqrtf(fmaf(tf, tf, 1.f));
                            c = (double)cr;
                            s = (double)(tf * cr);
                            for (int it = 0; it < 2; ++it) {   // c^2 + s^2 - 1: 1e-7 -> 1e-14 -> rounding
                                const double f = fma(-0.5, fma(c, c, s * s), 1.5);
                                c *= f;
                                s *= f;
                            }
                        } else {   // out of FP32 range: FP64 formula
                            double th = d / (2.0 * aij);
                            double t;
                            if (fabs(th) > 1e150) t = 0.5 / th;
                            else t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                            c = 1.0 / sqrt(t * t + 1.0);
                            s = t * c;
                        }
                    }
                }
                rc[k] = c; rs[k] = s; ri[k] = i; rj[k] = (j < p) ? j : -1;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
                int k = e / p, r = e % p;
                int i = ri[k], j = rj[k];
                if (j < 0 || rs[k] == 0.0) continue;
                double c = rc[k], s = rs[k];
                double a = A[r * LD + i], b = A[r * LD + j];
                A[r * LD + i] = c * a - s * b;
                A[r * LD + j] = s * a + c * b;
                a = V[r * LD + i]; b = V[r * LD + j];
                V[r * LD + i] = c * a - s * b;
                V[r * LD + j] = s * a + c * b;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = threadIdx.x; e < half * p; e += blockDim.x) {
                int k = e / p, r = e % p;
                int i = ri[k], j = rj[k];
                if (j < 0 || rs[k] == 0.0) continue;
                double c = rc[k], s = rs[k];
                double a = A[i * LD + r], b = A[j * LD + r];
                A[i * LD + r] = c * a - s * b;
                A[j * LD + r] = s * a + c * b;
            }
            __syncthreads();
            // the rotated pair keeps what the FP32 angle left of it (removed by
            // the next sweep); its two copies are made equal
            if (threadIdx.x < half) {
                int k = threadIdx.x;
                if (rj[k] >= 0 && rs[k] != 0.0) A[rj[k] * LD + ri[k]] = A[ri[k] * LD + rj[k]];
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < p; ++i) order[i] = i;
        for (int i = 1; i < p; ++i) {       // stable insertion sort, decreasing
            int v = order[i];
            double dv = A[v * LD + v];
            int j = i - 1;
            while (j >= 0 && A[order[j] * LD + order[j]] < dv) { order[j + 1] = order[j]; --j; }
            order[j + 1] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        int i = e / p, j = e % p;
        Vs[i * LD + j] = V[i * LD + order[j]];
    }
    for (int j = threadIdx.x; j < p; j += blockDim.x) lam[j] = A[order[j] * LD + order[j]];
    __syncthreads();
}

// log|det A| by LU with partial pivoting (A overwritten).  -inf if singular.
__device__ inline double cta_logabsdet(double* A, int p) {
    __shared__ int piv;
    __shared__ int zero;
    __shared__ double pv[PMAX];
    if (threadIdx.x == 0) zero = 0;
    __syncthreads();
    for (int k = 0; k < p; ++k) {
        if (threadIdx.x == 0) {
            int best = k;
            double bv = fabs(A[k * LD + k]);
            for (int i = k + 1; i < p; ++i) {
                double v = fabs(A[i * LD + k]);
                if (v > bv) { bv = v; best = i; }
            }
            piv = best;
            pv[k] = bv;
            if (bv == 0.0) zero = 1;
        }
        __syncthreads();
        if (zero) break;
        int pr = piv;
        if (pr != k) {
            for (int j = threadIdx.x; j < p; j += blockDim.x) {
                double t = A[k * LD + j];
                A[k * LD + j] = A[pr * LD + j];
                A[pr * LD + j] = t;
            }
        }
        __syncthreads();
        // multipliers once per row (one division each), then the update
        const double d = A[k * LD + k];
        for (int i = k + 1 + threadIdx.x; i < p; i += blockDim.x) A[i * LD + k] = A[i * LD + k] / d;
        __syncthreads();
        int rem = p - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            int i = k + 1 + e / rem, j = k + 1 + e % rem;
            A[i * LD + j] -= A[i * LD + k] * A[k * LD + j];
        }
        __syncthreads();
    }
    // log|det| = sum of the pivots' logs, taken in parallel (a log is long
    // on this GPU, so not one after another on the pivot thread)
    double r = 0.0;
    if (!zero)
        for (int k = threadIdx.x; k < p; k += blockDim.x) r += log(pv[k]);
    r = cta_sum(r);
    const double out = zero ? -INFINITY : r;
    __syncthreads();
    return out;
}

}  // namespace rtd
