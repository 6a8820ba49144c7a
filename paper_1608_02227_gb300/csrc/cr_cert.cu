// cr_cert.cu -- convergence record of eta(lambda^k): exact infeasibility over all pairs and
// a certified upper bound on p*_gamma.
//
// For eta = (y, xi) = eta(lambda^k) and u_i = y_i - xi_i . x_i, piece i of the max-affine
// function f(x) = max_i (y_i + xi_i . (x - x_i)) has value v_ij = u_i + xi_i . x_j at x_j,
// and (C eta)_ij = y_j - v_ij (Eq. (original)).  One pass over all pairs (no Lambda
// traffic, 2 N^2 n flops) gives, per column j,
//     M_j = max_{i != j} v_ij (smallest maximising i)   and   sum_i min(0, (C eta)_ij)^2.
// y_rep_j = max(y_j, M_j) = f(x_j) and xi_rep_j = the slope of a maximising piece (own
// piece when it attains the max) are values and subgradients of the convex f, hence
// satisfy every constraint of Eq. (regularize): r_gamma(y_rep, xi_rep) >= p*_gamma.
// The pass is split into R row ranges so the grid fills the GPU; the per-range results
// are combined in increasing row order (deterministic).
#include <math.h>

#include <type_traits>

#include "cr_internal.cuh"

namespace cr {
namespace {

constexpr int kCT = 256;   // columns per CTA (one per thread)
constexpr int kRT = 64;    // rows per shared-memory tile

__device__ __forceinline__ void split_hi_lo(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// eta(lambda^k) vectors in the layout of the sweep (transposed xi, split y and u)
__global__ void cert_prep_kernel(const CertArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.N) return;
    const double gamma = a.st->gamma;
    const double y = a.ybar[l] + a.a[l];
    double u = y;
    for (int k = 0; k < a.n; ++k) {
        const double xi = a.b[(long long)l * a.n + k] / gamma;
        if (a.precision == CR_FP64) {
            a.xiT64[(long long)k * a.ldv + l] = xi;
            u -= xi * a.X[(long long)l * a.n + k];
        } else {
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

template <int NP>
__global__ void __launch_bounds__(kCT) cert_pass_f32(const CertArgs a) {
    __shared__ float su_h[kRT], su_l[kRT];
    __shared__ float sxi[NP][kRT];
    const int j = blockIdx.x * kCT + threadIdx.x;
    const int rs = blockIdx.y;
    const int rows_per = (a.N + a.row_splits - 1) / a.row_splits;
    const int r0 = rs * rows_per, r1 = min(a.N, r0 + rows_per);
    float xj[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) xj[k] = (j < a.N) ? a.xT32[(long long)k * a.ldv + j] : 0.f;
    const float yhj = (j < a.N) ? a.yh[j] : 0.f, ylj = (j < a.N) ? a.yl[j] : 0.f;
    float best = -INFINITY;
    int arg = -1;
    double inf = 0.0;
    for (int t0 = r0; t0 < r1; t0 += kRT) {
        __syncthreads();
        for (int q = threadIdx.x; q < kRT * (NP + 2); q += kCT) {
            const int c = q / kRT, r = q - c * kRT, i = t0 + r;
            const bool ok = i < r1;
            if (c < NP)
                sxi[c][r] = ok ? a.xiT[(long long)c * a.ldv + i] : 0.f;
            else if (c == NP)
                su_h[r] = ok ? a.uh[i] : 0.f;
            else
                su_l[r] = ok ? a.ul[i] : 0.f;
        }
        __syncthreads();
        const int cnt = min(kRT, r1 - t0);
        float infs = 0.f;
        for (int r = 0; r < cnt; ++r) {
            float d = 0.f;
#pragma unroll
            for (int k = 0; k < NP; ++k) d = fmaf(sxi[k][r], xj[k], d);
            // v_ij - y_j, with the hi and lo parts of u_i - y_j subtracted separately
            const float v = ((su_h[r] - yhj) + (su_l[r] - ylj)) + d;
            const int i = t0 + r;
            if (i != j) {
                if (v > best) {
                    best = v;
                    arg = i;
                }
                if (v > 0.f) infs = fmaf(v, v, infs);
            }
        }
        inf += (double)infs;
    }
    if (j < a.N) {
        const long long o = (long long)rs * a.N + j;
        a.pmax[o] = (double)best;
        a.parg[o] = arg;
        a.pinf[o] = inf;
    }
}

template <int NP>
__global__ void __launch_bounds__(kCT) cert_pass_f64(const CertArgs a) {
    __shared__ double su[kRT];
    __shared__ double sxi[NP][kRT];
    const int j = blockIdx.x * kCT + threadIdx.x;
    const int rs = blockIdx.y;
    const int rows_per = (a.N + a.row_splits - 1) / a.row_splits;
    const int r0 = rs * rows_per, r1 = min(a.N, r0 + rows_per);
    double xj[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) xj[k] = (j < a.N) ? a.xT64[(long long)k * a.ldv + j] : 0.0;
    const double yj = (j < a.N) ? a.y64[j] : 0.0;
    double best = -INFINITY;
    int arg = -1;
    double inf = 0.0;
    for (int t0 = r0; t0 < r1; t0 += kRT) {
        __syncthreads();
        for (int q = threadIdx.x; q < kRT * (NP + 1); q += kCT) {
            const int c = q / kRT, r = q - c * kRT, i = t0 + r;
            const bool ok = i < r1;
            if (c < NP)
                sxi[c][r] = ok ? a.xiT64[(long long)c * a.ldv + i] : 0.0;
            else
                su[r] = ok ? a.u64[i] : 0.0;
        }
        __syncthreads();
        const int cnt = min(kRT, r1 - t0);
        for (int r = 0; r < cnt; ++r) {
            double d = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) d = fma(sxi[k][r], xj[k], d);
            const double v = (su[r] - yj) + d;
            const int i = t0 + r;
            if (i != j) {
                if (v > best) {
                    best = v;
                    arg = i;
                }
                if (v > 0.0) inf = fma(v, v, inf);
            }
        }
    }
    if (j < a.N) {
        const long long o = (long long)rs * a.N + j;
        a.pmax[o] = best;
        a.parg[o] = arg;
        a.pinf[o] = inf;
    }
}

// Wide points (NP > 32): x_j no longer fits in registers next to the row loop, so the
// dot products of a 32-row tile are accumulated over components in chunks of 16 (x_j of the
// chunk in registers, xi of the tile read as 16-byte broadcasts); the order of the sum over
// k is the same as above.
constexpr int kRW = 32;  // rows per tile (wide)
constexpr int kKC = 16;  // components per register chunk (NP is a multiple of 16)

template <typename T>
__global__ void __launch_bounds__(kCT) cert_pass_wide(const CertArgs a) {
    constexpr bool F32 = std::is_same<T, float>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sxi = reinterpret_cast<T *>(smem_raw);  // [NP][kRW]
    T *su0 = sxi + (size_t)a.NP * kRW;          // [kRW] u (FP32: hi)
    T *su1 = su0 + kRW;                         // [kRW] FP32: u lo
    const T *xT = F32 ? (const T *)a.xT32 : (const T *)a.xT64;
    const T *xiT = F32 ? (const T *)a.xiT : (const T *)a.xiT64;
    const T *u0 = F32 ? (const T *)a.uh : (const T *)a.u64;
    const T *u1 = F32 ? (const T *)a.ul : (const T *)a.u64;
    const T *y0 = F32 ? (const T *)a.yh : (const T *)a.y64;
    const T *y1 = F32 ? (const T *)a.yl : (const T *)a.y64;
    const int j = blockIdx.x * kCT + threadIdx.x;
    const bool jv = j < a.N;
    const int rs = blockIdx.y;
    const int rows_per = (a.N + a.row_splits - 1) / a.row_splits;
    const int r0 = rs * rows_per, r1 = min(a.N, r0 + rows_per);
    const T yj0 = jv ? y0[j] : (T)0, yj1 = (F32 && jv) ? y1[j] : (T)0;
    T best = (T)-INFINITY;
    int arg = -1;
    double inf = 0.0;
    for (int t0 = r0; t0 < r1; t0 += kRW) {
        __syncthreads();
        for (int q = threadIdx.x; q < kRW * (a.NP + 2); q += kCT) {
            const int c = q / kRW, r = q - c * kRW, i = t0 + r;
            const bool ok = i < r1;
            if (c < a.NP)
                sxi[c * kRW + r] = ok ? xiT[(long long)c * a.ldv + i] : (T)0;
            else if (c == a.NP)
                su0[r] = ok ? u0[i] : (T)0;
            else
                su1[r] = (F32 && ok) ? u1[i] : (T)0;
        }
        __syncthreads();
        T d[kRW];
#pragma unroll
        for (int r = 0; r < kRW; ++r) d[r] = (T)0;
        for (int kc = 0; kc < a.NP; kc += kKC) {
            T xj[kKC];
#pragma unroll
            for (int k = 0; k < kKC; ++k) xj[k] = jv ? xT[(long long)(kc + k) * a.ldv + j] : (T)0;
#pragma unroll
            for (int k = 0; k < kKC; ++k) {
                const T *row = sxi + (kc + k) * kRW;
#pragma unroll
                for (int r = 0; r < kRW; r += 16 / sizeof(T)) {
                    if constexpr (F32) {
                        const float4 v = *reinterpret_cast<const float4 *>(row + r);
                        d[r + 0] = fmaf(v.x, (float)xj[k], (float)d[r + 0]);
                        d[r + 1] = fmaf(v.y, (float)xj[k], (float)d[r + 1]);
                        d[r + 2] = fmaf(v.z, (float)xj[k], (float)d[r + 2]);
                        d[r + 3] = fmaf(v.w, (float)xj[k], (float)d[r + 3]);
                    } else {
                        const double2 v = *reinterpret_cast<const double2 *>(row + r);
                        d[r + 0] = fma(v.x, (double)xj[k], (double)d[r + 0]);
                        d[r + 1] = fma(v.y, (double)xj[k], (double)d[r + 1]);
                    }
                }
            }
        }
        const int cnt = min(kRW, r1 - t0);
        float infs = 0.f;  // FP32: per tile, then added in FP64 (as the narrow pass)
#pragma unroll
        for (int r = 0; r < kRW; ++r) {
            if (r >= cnt) break;
            // v_ij - y_j (FP32: hi and lo parts of u_i - y_j subtracted separately)
            T v;
            if constexpr (F32)
                v = ((su0[r] - yj0) + (su1[r] - yj1)) + d[r];
            else
                v = (su0[r] - yj0) + d[r];
            const int i = t0 + r;
            if (i != j) {
                if (v > best) {
                    best = v;
                    arg = i;
                }
                if (v > (T)0) {
                    if constexpr (F32)
                        infs = fmaf(v, v, infs);
                    else
                        inf = fma(v, v, inf);
                }
            }
        }
        if constexpr (F32) inf += (double)infs;
    }
    if (jv) {
        const long long o = (long long)rs * a.N + j;
        a.pmax[o] = (double)best;
        a.parg[o] = arg;
        a.pinf[o] = inf;
    }
}

size_t cert_wide_smem(int NP, bool f64) { return (f64 ? 8 : 4) * ((size_t)NP * kRW + 2 * kRW); }

template <typename T>
cudaError_t run_cert_wide(const CertArgs &a, dim3 grid, cudaStream_t s) {
    const size_t sm = cert_wide_smem(CR_MAX_N, sizeof(T) == 8);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(cert_pass_wide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    cert_pass_wide<T><<<grid, kCT, cert_wide_smem(a.NP, sizeof(T) == 8), s>>>(a);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kCT) cert_combine_kernel(const CertArgs a) {
    const int j = blockIdx.x * kCT + threadIdx.x;
    DevState *st = a.st;
    const double gamma = st->gamma;
    double pobj = 0.0, inf = 0.0;
    if (j < a.N) {
        double best = -INFINITY;
        int arg = j;
        for (int rs = 0; rs < a.row_splits; ++rs) {
            const long long o = (long long)rs * a.N + j;
            if (a.parg[o] >= 0 && a.pmax[o] > best) {
                best = a.pmax[o];
                arg = a.parg[o];
            }
            inf += a.pinf[o];
        }
        const double y = a.ybar[j] + a.a[j];
        double yrep = y;
        int m = j;
        if (best > 0.0) {  // another piece lies strictly above the own piece at x_j
            yrep = y + best;
            m = arg;
        }
        double xx = 0.0;
        for (int k = 0; k < a.n; ++k) {
            const double xi = a.b[(long long)m * a.n + k] / gamma;
            xx += xi * xi;
        }
        pobj = 0.5 * (yrep - a.ybar[j]) * (yrep - a.ybar[j]) + 0.5 * gamma * xx;
    }
    __shared__ double sh[2][kCT];
    sh[0][threadIdx.x] = pobj;
    sh[1][threadIdx.x] = inf;
    __syncthreads();
    for (int w = kCT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        a.blockpart[blockIdx.x * 2 + 0] = sh[0][0];
        a.blockpart[blockIdx.x * 2 + 1] = sh[1][0];
        __threadfence();
        const unsigned ticket = atomicAdd(&st->cert_counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // last CTA: fixed-order parallel reduction of the per-CTA partials
    __threadfence();
    {
        double P = 0.0, I = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += kCT) {
            P += __ldcg(a.blockpart + b * 2 + 0);
            I += __ldcg(a.blockpart + b * 2 + 1);
        }
        sh[0][threadIdx.x] = P;
        sh[1][threadIdx.x] = I;
    }
    __syncthreads();
    for (int w = kCT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double P = sh[0][0], I = sh[1][0];
        st->cert_P = P;
        st->cert_infeas_sq = I;
        st->cert_counter = 0u;
        __threadfence();
    }
}

#define CR_NP_LIST(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(28) X(32)

}  // namespace

cudaError_t launch_cert(const CertArgs &a, cudaStream_t s) {
    const unsigned gN = (unsigned)((a.N + kCT - 1) / kCT);
    cert_prep_kernel<<<gN, kCT, 0, s>>>(a);
    dim3 grid(gN, (unsigned)a.row_splits);
    if (a.NP > 32) {
        if (a.NP > CR_MAX_N || a.NP % kKC != 0) return cudaErrorInvalidValue;
        const cudaError_t e = a.precision == CR_FP64 ? run_cert_wide<double>(a, grid, s) : run_cert_wide<float>(a, grid, s);
        if (e != cudaSuccess) return e;
    } else if (a.precision == CR_FP64) {
        switch (a.NP) {
#define CASE(V) \
    case V: cert_pass_f64<V><<<grid, kCT, 0, s>>>(a); break;
            CR_NP_LIST(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (a.NP) {
#define CASE(V) \
    case V: cert_pass_f32<V><<<grid, kCT, 0, s>>>(a); break;
            CR_NP_LIST(CASE)
#undef CASE
            default: return cudaErrorInvalidValue;
        }
    }
    cert_combine_kernel<<<gN, kCT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cr
