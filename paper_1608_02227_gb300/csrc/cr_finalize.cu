// cr_finalize.cu -- the O(N n) kernels around the sweep:
//   * finalize + recovery (Steps 1 and 3 of Figure "papg", K = N): reduce the sweep's
//     partials into C^T lambda^k = (a, b) in FP64, the scalars g_gamma(lambda^k),
//     r_gamma(eta(lambda^k)), <lambda^k, C eta(lambda^k)>, the t/beta update, and the
//     closed-form Step 1 minimiser eta(lambda~^{k+1}) for the next sweep;
//   * eta(lambda^k) for the caller, point transposes, Lambda export, finiteness check.
#include <math.h>

#include "cr_internal.cuh"

namespace cr {
namespace {

constexpr int kFinThreads = 256;

__device__ __forceinline__ void split_hi_lo(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// Deterministic block sum of three doubles (fixed tree order).
__device__ void block_sum3(double v0, double v1, double v2, double *out3) {
    __shared__ double sh[3][kFinThreads];
    const int t = threadIdx.x;
    sh[0][t] = v0;
    sh[1][t] = v1;
    sh[2][t] = v2;
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
            sh[0][t] += sh[0][t + w];
            sh[1][t] += sh[1][t + w];
            sh[2][t] += sh[2][t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        out3[0] = sh[0][0];
        out3[1] = sh[1][0];
        out3[2] = sh[2][0];
    }
}

template <typename PT>
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const FinArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    DevState *st = a.st;
    const double gamma = st->gamma;
    const double tk = st->t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));           // Step 3
    const double beta = (st->accelerate && !a.init) ? (tk - 1.0) / tn : 0.0;  // Step 4 coefficient
    const PT *rowp = reinterpret_cast<const PT *>(a.rowpart);
    const PT *colp = reinterpret_cast<const PT *>(a.colpart);
    const int W = a.NP + 1;

    double saa = 0.0, say = 0.0, sbb = 0.0;
    if (l < a.N) {
        // C^T lambda^k: a_l = c_l - r_l, b_l = r_l x_l - sum_j lambda_lj x_j
        double r = 0.0, c = 0.0;
        if (!a.init) {
            for (int s = 0; s < a.col_splits; ++s) r += (double)rowp[((long long)s * a.N + l) * W + a.NP];
            for (int b = 0; b < a.row_blocks; ++b) c += (double)colp[(long long)b * a.ld + l];
        }
        const double al = c - r;
        a.a_new[l] = al;
        saa = al * al;
        say = al * a.ybar[l];
        // Step 1 for the next iteration: eta(lambda~^{k+1}) with
        // C^T lambda~^{k+1} = (1 + beta) C^T lambda^k - beta C^T lambda^{k-1}
        const double at = (1.0 + beta) * al - beta * a.a_old[l];
        const double y = a.ybar[l] + at;
        double u = y;
        for (int k = 0; k < a.n; ++k) {
            double Bk = 0.0;
            if (!a.init)
                for (int s = 0; s < a.col_splits; ++s) Bk += (double)rowp[((long long)s * a.N + l) * W + k];
            const double xk = a.X[(long long)l * a.n + k];
            const double bl = r * xk - Bk;
            a.b_new[(long long)l * a.n + k] = bl;
            sbb += bl * bl;
            const double bt = (1.0 + beta) * bl - beta * a.b_old[(long long)l * a.n + k];
            const double xi = bt / gamma;
            if (a.precision == CR_FP64) {
                a.xiT64[(long long)k * a.ldv + l] = xi;
                u -= xi * xk;
            } else {
                // the sweep sees the rounded xi and x; u is formed from exactly those
                const float xf = (float)xi;
                a.xiT[(long long)k * a.ldv + l] = xf;
                u -= (double)xf * (double)a.xT32[(long long)k * a.ldv + l];
            }
        }
        if (a.precision == CR_FP64) {
            a.y64[l] = y;
            a.u64[l] = u;
        } else {
            split_hi_lo(y, a.yh + l, a.yl + l);
            split_hi_lo(u, a.uh + l, a.ul + l);
        }
    }
    if (a.init) return;

    __shared__ double part[3];
    block_sum3(saa, say, sbb, part);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.blockpart[blockIdx.x * 3 + 0] = part[0];
        a.blockpart[blockIdx.x * 3 + 1] = part[1];
        a.blockpart[blockIdx.x * 3 + 2] = part[2];
        __threadfence();
        const unsigned ticket = atomicAdd(&st->fin_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double aa = 0.0, ay = 0.0, bb = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            aa += ((volatile double *)a.blockpart)[b * 3 + 0];
            ay += ((volatile double *)a.blockpart)[b * 3 + 1];
            bb += ((volatile double *)a.blockpart)[b * 3 + 2];
        }
        // g_gamma(lambda) = -1/2||a||^2 - a.ybar - ||b||^2/(2 gamma)   (Eq. g_gamma at eta(lambda))
        const double g = -0.5 * aa - ay - bb / (2.0 * gamma);
        const double rr = 0.5 * aa + bb / (2.0 * gamma);
        const double lg = aa + ay + bb / gamma;
        st->last_g = g;
        st->last_r = rr;
        st->last_lg = lg;
        const long long k = st->k + 1;
        double *lp = a.log + (size_t)((k - 1) % kLogCap) * 3;
        lp[0] = g;
        lp[1] = rr;
        lp[2] = lg;
        st->k = k;
        st->t = tn;
        st->beta = st->accelerate ? (tk - 1.0) / tn : 0.0;
        st->fin_counter = 0u;
        __threadfence();
    }
}

__global__ void primal_kernel(int N, int n, const double *ybar, const double *av, const double *bv,
                              const DevState *st, double *y, double *xi) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const double gamma = st->gamma;
    if (q < N) y[q] = ybar[q] + av[q];
    if (q < (long long)N * n) xi[q] = bv[q] / gamma;
}

__global__ void transpose_points_kernel(const double *X, int N, int n, int NP, long long ldv,
                                        float *xT32, double *xT64) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)NP * ldv) return;
    const int k = (int)(q / ldv);
    const long long l = q - (long long)k * ldv;
    const double v = (k < n && l < N) ? X[l * n + k] : 0.0;
    if (xT32) xT32[q] = (float)v;
    if (xT64) xT64[q] = v;
}

__global__ void lambda_to_f64_kernel(const void *lam, int is_f32, int N, long long ld, long long row0,
                                     long long rows, double *out, long long ldo) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= rows * N) return;
    const long long r = q / N, j = q - r * N, i = row0 + r;
    out[r * ldo + j] = is_f32 ? (double)((const float *)lam)[i * ld + j] : ((const double *)lam)[i * ld + j];
}

__global__ void check_finite_kernel(const double *v, long long count, int *flag) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[q])) atomicExch(flag, 1);
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_finalize(const FinArgs &a, cudaStream_t s) {
    const unsigned g = blocks_for(a.N, kFinThreads);
    if (a.precision == CR_FP64)
        finalize_kernel<double><<<g, kFinThreads, 0, s>>>(a);
    else
        finalize_kernel<float><<<g, kFinThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_primal(int N, int n, const double *ybar, const double *a, const double *b,
                          const DevState *st, double *y, double *xi, cudaStream_t s) {
    const long long cnt = (long long)N * (n > 1 ? n : 1);
    primal_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(N, n, ybar, a, b, st, y, xi);
    return cudaGetLastError();
}

cudaError_t launch_transpose_points(const double *X, int N, int n, int NP, long long ldv, float *xT32,
                                    double *xT64, cudaStream_t s) {
    transpose_points_kernel<<<blocks_for((long long)NP * ldv, 256), 256, 0, s>>>(X, N, n, NP, ldv, xT32,
                                                                                  xT64);
    return cudaGetLastError();
}

cudaError_t launch_lambda_to_f64(const void *lam, int is_f32, int N, long long ld, long long row0,
                                 long long rows, double *out, long long ldo, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    lambda_to_f64_kernel<<<blocks_for(rows * N, 256), 256, 0, s>>>(lam, is_f32, N, ld, row0, rows, out,
                                                                   ldo);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double *v, long long count, int *flag, cudaStream_t s) {
    unsigned g = blocks_for(count, 256);
    if (g > 1024) g = 1024;
    if (g == 0) g = 1;
    check_finite_kernel<<<g, 256, 0, s>>>(v, count, flag);
    return cudaGetLastError();
}

}  // namespace cr
