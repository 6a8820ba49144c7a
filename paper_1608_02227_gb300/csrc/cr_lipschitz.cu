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

#include "cr_internal.cuh"

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

// cyclic Jacobi on the n x n symmetric Sc, one warp: every lane recomputes the rotation
// and updates one row/column index r of A and of the accumulated vectors V (columns =
// eigenvectors).  D (n) and V (n x n) are written at the end.
__global__ void jacobi_kernel(const double *Sc, int n, double *D, double *V) {
    __shared__ double A[CR_MAX_N * CR_MAX_N];
    __shared__ double Q[CR_MAX_N * CR_MAX_N];
    const int lane = threadIdx.x;
    for (int i = lane; i < n * n; i += 32) {
        A[i] = Sc[i];
        Q[i] = (i / n == i % n) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = lane; i < n * n; i += 32) {
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
        if (off <= 1e-32 * dia || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                __syncwarp();
                if (lane < n) {  // A <- A J (columns p, q)
                    const double arp = A[lane * n + p], arq = A[lane * n + q];
                    A[lane * n + p] = c * arp - s * arq;
                    A[lane * n + q] = s * arp + c * arq;
                    const double qrp = Q[lane * n + p], qrq = Q[lane * n + q];
                    Q[lane * n + p] = c * qrp - s * qrq;
                    Q[lane * n + q] = s * qrp + c * qrq;
                }
                __syncwarp();
                if (lane < n) {  // A <- J^T A (rows p, q)
                    const double apr = A[p * n + lane], aqr = A[q * n + lane];
                    A[p * n + lane] = c * apr - s * aqr;
                    A[q * n + lane] = s * apr + c * aqr;
                }
                __syncwarp();
            }
    }
    for (int i = lane; i < n; i += 32) D[i] = A[i * n + i];
    for (int i = lane; i < n * n; i += 32) V[i] = Q[i];
}

__global__ void secular_kernel(const double *X, int N, int n, const double *mean, const double *D,
                               const double *V, unsigned long long *best_bits) {
    __shared__ double sV[CR_MAX_N * CR_MAX_N];
    __shared__ double sD[CR_MAX_N];
    __shared__ double smean[CR_MAX_N];
    for (int i = threadIdx.x; i < n * n; i += kT) sV[i] = V[i];
    for (int i = threadIdx.x; i < n; i += kT) {
        sD[i] = D[i];
        smean[i] = mean[i];
    }
    __syncthreads();
    const int l = blockIdx.x * kT + threadIdx.x;
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
            for (int it = 0; it < 400; ++it) {
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
    __shared__ double sm[kT];
    sm[threadIdx.x] = mu;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(best_bits, (unsigned long long)__double_as_longlong(sm[0]));
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
    jacobi_kernel<<<1, 32, 0, s>>>(Sc, n, D, V);  // one warp
    secular_kernel<<<(N + kT - 1) / kT, kT, 0, s>>>(X, N, n, mean, D, V, best);
    unsigned long long bits = 0;
    e = cudaMemcpyAsync(&bits, best, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return e;
    double v;
    memcpy(&v, &bits, sizeof(v));
    *out_host = v;
    return cudaGetLastError();
}

}  // namespace cr
