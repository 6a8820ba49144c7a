// cr_lipschitz.cu -- the step constant of Step 2 (Eq. (lischitz) and Lemma "O1-constant").
//
// With K = N, C = [A1 A2] and A2 = blkdiag(X_l), X_l = -T_l Xbar (Definition 1), so
// sigma_max(A2)^2 = max_l lambda_max(S_l), S_l = X_l^T X_l = sum_j (x_j - x_l)(x_j - x_l)^T
// (this is the paper's "Preprocess", sigma_max(A4) for K = N).  Writing xhat for the mean
// point, d_l = x_l - xhat and Sc = sum_j (x_j - xhat)(x_j - xhat)^T, the cross terms
// cancel and S_l = Sc + N d_l d_l^T: a rank-one update of one n x n matrix.  With
// Sc = V diag(D) V^T and e = V^T d_l, lambda_max(S_l) is the largest root mu > max D of
// the secular equation  1 - N sum_k e_k^2 / (mu - D_k) = 0,  which lies in
// (max D, max D + N ||e||^2] and is found by bisection (the upper end is kept, so the
// result never underestimates).  Cost: O(N n^2) for Sc, one n x n Jacobi
// eigendecomposition, O(N n) bisection steps per point.
#include <math.h>
#include <string.h>

#include <algorithm>

#include <mutex>

#include "cr_host.h"

namespace cr {
namespace {

constexpr int kT = 256;

__device__ double block_sum(double v) {
    __shared__ double sh[kT];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// one block per component k: mean[k]
__global__ void mean_kernel(const double *X, int N, int n, double *mean) {
    const int k = blockIdx.x;
    double s = 0.0;
    for (int l = threadIdx.x; l < N; l += kT) s += X[(long long)l * n + k];
    s = block_sum(s);
    if (threadIdx.x == 0) mean[k] = s / N;
}

// one block per (k, m), k <= m: Sc[k][m] = Sc[m][k]
__global__ void scatter_kernel(const double *X, int N, int n, const double *mean, double *Sc) {
    int k = 0, m = blockIdx.x, w = n;
    while (m >= w) {  // unrank the upper-triangular index
        m -= w;
        ++k;
        --w;
    }
    m += k;
    double s = 0.0;
    for (int l = threadIdx.x; l < N; l += kT)
        s += (X[(long long)l * n + k] - mean[k]) * (X[(long long)l * n + m] - mean[m]);
    s = block_sum(s);
    if (threadIdx.x == 0) {
        Sc[k * n + m] = s;
        Sc[m * n + k] = s;
    }
}

// Jacobi eigendecomposition of the n x n symmetric Sc by one block of kJT threads, parallel
// ordering: each sweep has m-1 rounds (m = n rounded up to even) of m/2 disjoint pairs (circle
// schedule).  Thread i computes the rotation of pair i; then the n * m/2 (row, pair) updates
// of A <- A J and V <- V J, and after them the (pair, column) updates of A <- J^T A, are spread
// over the block.  The pairs of a round are disjoint, so every element receives exactly the
// rotations of its own pair, in the same order, whichever thread applies them.  A lives in
// dynamic shared memory (n^2 doubles) and so do the accumulated rotations when both fit
// (n <= kJacobiVShared); above that they accumulate directly in V (n x n, columns =
// eigenvectors).  D (n) and V are written at the end.
constexpr int kJT = 512;
static_assert(kJT % 32 == 0 && kJT >= CR_MAX_N, "whole warps, one thread per pair at least");
constexpr int kJacobiVShared = 112;  // 2 n^2 doubles <= 200 KB of shared memory

size_t jacobi_smem(int n) { return sizeof(double) * (size_t)n * n * (n <= kJacobiVShared ? 2 : 1); }

__global__ void __launch_bounds__(kJT) jacobi_kernel(const double *Sc, int n, double *D, double *V) {
    extern __shared__ double A[];  // n x n, then (n <= kJacobiVShared) the rotations
    __shared__ double rc[CR_MAX_N / 2], rs[CR_MAX_N / 2];
    __shared__ int rp[CR_MAX_N / 2], rq[CR_MAX_N / 2];
    __shared__ double red[2][kJT / 32];
    __shared__ int done;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int m = (n + 1) & ~1, h = m / 2;
    double *Q = n <= kJacobiVShared ? A + (size_t)n * n : V;
    for (int i = t; i < n * n; i += kJT) {
        A[i] = Sc[i];
        Q[i] = (i / n == i % n) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = t; i < n * n; i += kJT) {
            const int p = i / n, q = i % n;
            if (p == q)
                dia += A[i] * A[i];
            else if (p < q)
                off += A[i] * A[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (lane == 0) {
            red[0][warp] = off;
            red[1][warp] = dia;
        }
        __syncthreads();
        if (t == 0) {
            double so = 0.0, sd = 0.0;
            for (int w = 0; w < kJT / 32; ++w) {
                so += red[0][w];
                sd += red[1][w];
            }
            done = (so <= 1e-32 * sd || so == 0.0) ? 1 : 0;
        }
        __syncthreads();
        if (done) break;
        for (int round = 0; round < m - 1; ++round) {
            if (t < h) {
                // circle method: position 0 fixed, the others rotate by `round`
                const int a0 = t == 0 ? 0 : ((t - 1 + round) % (m - 1)) + 1;
                const int b0 = ((m - 1 - t - 1 + round) % (m - 1)) + 1;
                const int p = min(a0, b0), q = max(a0, b0);
                double c = 1.0, sn = 0.0;
                if (q < n) {
                    const double apq = A[p * n + q];
                    if (apq != 0.0) {
                        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                rp[t] = p;
                rq[t] = q;
                rc[t] = c;
                rs[t] = sn;
            }
            __syncthreads();
            for (int w = t; w < n * h; w += kJT) {  // A <- A J and V <- V J: (row r, pair i)
                const int r = w / h, i = w - r * h;
                const int p = rp[i], q = rq[i];
                if (q >= n || rs[i] == 0.0) continue;
                const double c = rc[i], sn = rs[i];
                const double arp = A[r * n + p], arq = A[r * n + q];
                A[r * n + p] = c * arp - sn * arq;
                A[r * n + q] = sn * arp + c * arq;
                const double qrp = Q[r * n + p], qrq = Q[r * n + q];
                Q[r * n + p] = c * qrp - sn * qrq;
                Q[r * n + q] = sn * qrp + c * qrq;
            }
            __syncthreads();
            for (int w = t; w < n * h; w += kJT) {  // A <- J^T A: (pair i, column col)
                const int i = w / n, col = w - i * n;
                const int p = rp[i], q = rq[i];
                if (q >= n || rs[i] == 0.0) continue;
                const double c = rc[i], sn = rs[i];
                const double apr = A[p * n + col], aqr = A[q * n + col];
                A[p * n + col] = c * apr - sn * aqr;
                A[q * n + col] = sn * apr + c * aqr;
            }
            __syncthreads();
        }
    }
    for (int i = t; i < n; i += kJT) D[i] = A[i * n + i];
    if (Q != V)
        for (int i = t; i < n * n; i += kJT) V[i] = Q[i];
}

// one thread per point; small blocks so that a few thousand points still spread over the SMs
constexpr int kST = 64;

__global__ void __launch_bounds__(kST) secular_kernel(const double *X, int N, int n, const double *mean,
                                                      const double *D, const double *V,
                                                      unsigned long long *best_bits) {
    extern __shared__ double sV[];  // n x n eigenvectors
    __shared__ double sD[CR_MAX_N];
    __shared__ double smean[CR_MAX_N];
    for (int i = threadIdx.x; i < n * n; i += kST) sV[i] = V[i];
    for (int i = threadIdx.x; i < n; i += kST) {
        sD[i] = D[i];
        smean[i] = mean[i];
    }
    __syncthreads();
    const int l = blockIdx.x * kST + threadIdx.x;
    double mu = 0.0;
    if (l < N) {
        double e[CR_MAX_N];
        double ee = 0.0, Dm = sD[0];
        for (int k = 1; k < n; ++k) Dm = fmax(Dm, sD[k]);
        for (int k = 0; k < n; ++k) {
            double v = 0.0;
            for (int m = 0; m < n; ++m) v += sV[m * n + k] * (X[(long long)l * n + m] - smean[m]);
            e[k] = v;
            ee += v * v;
        }
        double lo = Dm, hi = Dm + (double)N * ee;
        if (ee > 0.0) {
            // f(mu) = 1 - N sum e_k^2 / (mu - D_k) is increasing and concave on (max D, inf);
            // 16 bisection steps, then Newton from the left end (monotone towards the root)
            for (int it = 0; it < 16; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double f = 1.0;
                for (int k = 0; k < n; ++k) f -= (double)N * e[k] * e[k] / (mid - sD[k]);
                if (f < 0.0)
                    lo = mid;
                else
                    hi = mid;
            }
            double mu_n = lo;
            for (int it = 0; it < 40 && mu_n > Dm; ++it) {
                double f = 1.0, fp = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double w = 1.0 / (mu_n - sD[k]);
                    const double t = (double)N * e[k] * e[k] * w;
                    f -= t;
                    fp += t * w;
                }
                if (f >= 0.0) {  // at or right of the root: an upper bound
                    hi = fmin(hi, mu_n);
                    break;
                }
                lo = mu_n;
                const double next = mu_n - f / fp;
                if (!(next > mu_n) || next >= hi) break;
                if (next - mu_n <= 1e-16 * next) {
                    mu_n = next;
                    continue;
                }
                mu_n = next;
            }
            // Newton approached the root from below: try a right end just above it
            {
                const double cand = lo + fmax(8e-16 * fabs(lo), 1e-300);
                if (cand < hi) {
                    double f = 1.0;
                    for (int k = 0; k < n; ++k) f -= (double)N * e[k] * e[k] / (cand - sD[k]);
                    if (f >= 0.0) hi = cand;
                }
            }
            // finish with bisection on the (now tiny) bracket; hi is kept, never underestimating
            for (int it = 0; it < 200; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double f = 1.0;
                for (int k = 0; k < n; ++k) f -= (double)N * e[k] * e[k] / (mid - sD[k]);
                if (f < 0.0)
                    lo = mid;
                else
                    hi = mid;
            }
        }
        mu = hi;
    }
    __shared__ double sm[kST];
    sm[threadIdx.x] = mu;
    __syncthreads();
    for (int w = kST / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(best_bits, (unsigned long long)__double_as_longlong(sm[0]));
}

constexpr int kAttrDevices = 128;

// The two kernels with n^2 doubles of dynamic shared memory (up to 128 KB at n = 128).
cudaError_t launch_eig_and_secular(const double *X, int N, int n, const double *mean, const double *Sc, double *D,
                                   double *V, unsigned long long *best, cudaStream_t s) {
    // the large dynamic shared-memory attribute applies to the current device only: set it
    // once per device, under a lock (callers on several threads or devices share this)
    static std::mutex mu;
    static bool attr_set[kAttrDevices] = {};
    const int big = (int)(sizeof(double) * CR_MAX_N * CR_MAX_N);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr_set[dev]) {
            const int jbig = (int)std::max(jacobi_smem(kJacobiVShared), jacobi_smem(CR_MAX_N));
            e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, jbig);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(secular_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
            if (e != cudaSuccess) return e;
            attr_set[dev] = true;
        }
    }
    const size_t sm = sizeof(double) * (size_t)n * n;
    jacobi_kernel<<<1, kJT, jacobi_smem(n), s>>>(Sc, n, D, V);
    secular_kernel<<<(unsigned)((N + kST - 1) / kST), kST, sm, s>>>(X, N, n, mean, D, V, best);
    return cudaGetLastError();
}

}  // namespace

cudaError_t a2_sigma_sq(const double *X, int N, int n, double *out_host, cudaStream_t s) {
    double *buf = nullptr;
    const size_t cnt = (size_t)n + 2 * (size_t)n * n + (size_t)n + 1;
    cudaError_t e = cudaMallocAsync((void **)&buf, cnt * sizeof(double), s);
    if (e != cudaSuccess) return e;
    double *mean = buf, *Sc = mean + n, *V = Sc + (size_t)n * n, *D = V + (size_t)n * n;
    unsigned long long *best = reinterpret_cast<unsigned long long *>(D + n);
    cudaMemsetAsync(best, 0, sizeof(unsigned long long), s);
    mean_kernel<<<n, kT, 0, s>>>(X, N, n, mean);
    scatter_kernel<<<n * (n + 1) / 2, kT, 0, s>>>(X, N, n, mean, Sc);
    e = launch_eig_and_secular(X, N, n, mean, Sc, D, V, best, s);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, best, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return e;
    double v;
    memcpy(&v, &bits, sizeof(v));
    *out_host = v;
    return cudaGetLastError();
}

}  // namespace cr

// ------------------------------------------------------------------------------------
// Allocation-free variant of the step-constant computation above.
//
// Some callers cannot allocate device memory when they need L: a serving front end that
// budgets HBM exactly and decides admission before reserving anything, code that runs
// under a framework whose caching allocator owns all of HBM, or latency-critical loops in
// which cudaMalloc/cudaFree would synchronise the device.  For them the scratch of the
// four kernels (mean, centred scatter, eigenvectors, eigenvalues, the max word) lives in
// one fixed array in device memory that every GPU loading this library holds until the
// process exits.
// ------------------------------------------------------------------------------------
namespace {

// mean (n) + scatter (n^2) + eigenvectors (n^2) + eigenvalues (n), then (in the last two
// words) the non-finite flag of X and the 64-bit max word, for n <= CR_MAX_N:
// 2 * 128 * 128 + 2 * 128 + 8 doubles = 264 KB.
constexpr int kLipScratchDoubles = 2 * CR_MAX_N * CR_MAX_N + 2 * CR_MAX_N + 8;
static __device__ __align__(256) double g_lip_scratch[kLipScratchDoubles];

constexpr int kMaxDevices = 128;
std::mutex g_lip_mu;
double *g_lip_addr[kMaxDevices] = {};

}  // namespace

extern "C" CR_API cr_status cr_lipschitz_noalloc(const double *X, long long N, int n, double gamma, int rule,
                                                void *stream, double *L) {
    using crh::set_err;
    if (!X || !L) {
        set_err("X or L is NULL");
        return CR_EINVAL;
    }
    if (N < 2 || N > (1LL << 30)) {
        set_err("N = %lld out of range [2, 2^30]", N);
        return CR_EINVAL;
    }
    if (n < 1 || n > CR_MAX_N) {
        set_err("n = %d exceeds the fixed scratch of cr_lipschitz_noalloc (1 <= n <= %d)", n, CR_MAX_N);
        return CR_EINVAL;
    }
    if (!(gamma > 0.0) || !isfinite(gamma) || (rule != CR_L_HESSIAN && rule != CR_L_PAPER)) {
        set_err("gamma must be finite and > 0, rule CR_L_HESSIAN or CR_L_PAPER");
        return CR_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_err("cudaGetDevice failed or device %d out of range: %s", dev, cudaGetErrorString(e));
        return CR_ECUDA;
    }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, X) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        set_err("X must be device memory (the allocation-free path cannot stage host data)");
        return CR_EINVAL;
    }
    if (at.type == cudaMemoryTypeDevice && at.device != dev) {
        set_err("X lives on device %d but device %d is current: make X's device current first", at.device, dev);
        return CR_EINVAL;
    }
    double *scr = nullptr;
    {
        // first call on this device (with it current): the device address of the array
        std::lock_guard<std::mutex> lock(g_lip_mu);
        if (!g_lip_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_lip_scratch);
            if (e != cudaSuccess || !p) {
                set_err("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
                return CR_ECUDA;
            }
            g_lip_addr[dev] = static_cast<double *>(p);
        }
        scr = g_lip_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *mean = scr, *Sc = mean + n, *V = Sc + (size_t)n * n, *D = V + (size_t)n * n;
    // the last two words: the non-finite flag of X and the max word; they are the only
    // scratch read before it is written, so both are cleared on every call
    unsigned long long *words = reinterpret_cast<unsigned long long *>(scr + kLipScratchDoubles - 2);
    int *finite_flag = reinterpret_cast<int *>(words);
    unsigned long long *best = words + 1;
    e = cudaMemsetAsync(words, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cr::launch_check_finite(X, N * (long long)n, finite_flag, s);
    if (e == cudaSuccess) {
        mean_kernel<<<n, kT, 0, s>>>(X, (int)N, n, mean);
        scatter_kernel<<<n * (n + 1) / 2, kT, 0, s>>>(X, (int)N, n, mean, Sc);
        e = cr::launch_eig_and_secular(X, (int)N, n, mean, Sc, D, V, best, s);
    }
    unsigned long long hw[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hw, words, sizeof(hw), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_err("cr_lipschitz_noalloc failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    int nonfinite = 0;
    memcpy(&nonfinite, &hw[0], sizeof(nonfinite));
    if (nonfinite) {
        set_err("X contains a non-finite value");
        return CR_EINVAL;
    }
    double s2;
    memcpy(&s2, &hw[1], sizeof(s2));
    const double Lv = (rule == CR_L_PAPER) ? (2.0 * (double)N + s2) / gamma : 2.0 * (double)N + s2 / gamma;
    if (!(Lv > 0.0) || !isfinite(Lv)) {
        set_err("non-finite or non-positive step constant L = %g", Lv);
        return CR_ENUMERIC;
    }
    *L = Lv;
    return CR_OK;
}
