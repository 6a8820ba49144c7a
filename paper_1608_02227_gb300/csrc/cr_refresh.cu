// cr_refresh.cu -- the periodic exact re-evaluation of C^T lambda^k (Definition 1) for the
// reduced-precision modes.
//
// In CR_FP32 and CR_MIXED_TF32 the sweep reduces the CHANGE of the multipliers,
// Delta^k = lambda^k - lambda^{k-1}, and the finalize accumulates
//     (a, b)^k = (a, b)^{k-1} + C^T Delta^k          (FP64, linearity of C^T)
// instead of forming C^T lambda^k from scratch.  b_l = sum_j lambda_lj (x_l - x_j) cancels
// from O(sum_j lambda_lj |x_l - x_j|) down to O(gamma |xi_l|); formed from FP32 partials its
// error sits at the FP32 level of the large terms, and that error moves the fixed point of
// the iteration (the duality gap stalls near 1e-4 on N = 20000 instances).  Reduced from the
// increments, the error scales with |Delta^k|, which vanishes as the iteration converges.
// The increments' rounding errors accumulate in the history, so every `period` iterations
// these kernels recompute C^T lambda^k from the stored FP32 multipliers in FP64 (each
// product and sum in FP64, over the nonzero multipliers, in a fixed order), shift C^T
// lambda^{k-1} by the same correction, recompute g_gamma, r_gamma and <lambda, C eta> of
// lambda^k, and rebuild eta(lambda~^{k+1}) for the next sweep.
//
// The kernels are enqueued after every iteration and decide on the device whether the
// refresh is due (k a multiple of the period from twice the period on, not yet refreshed), so CUDA-graph
// replays and the adaptive step (whose accepted count lives on the device) need no host
// round trip.
#include <math.h>

#include <algorithm>

#include "cr_internal.cuh"

namespace cr {
namespace {

constexpr int kRowWarps = 8;    // rows per CTA of the row pass (one warp per row)
constexpr int kColThreads = 256;
constexpr int kFinThreads = 256;

__host__ __device__ __forceinline__ int refresh_finish_blocks_dev(int N) { return (N + kFinThreads - 1) / kFinThreads; }

// Due at k = 2 period, 3 period, ...: the first period's increments are the largest, but the
// multipliers are still dense then (a fifth of the pairs nonzero at k = 64 on the N = 20000
// workload), which makes the FP64 row pass cost a few sweeps; one period later they are sparse.
__device__ __forceinline__ bool refresh_due(const DevState *st, int period) {
    const long long k = st->k;
    return period > 0 && k >= 2 * period && k % period == 0 && st->refreshed_k != k;
}

// lambda^k lives in lam[k & 1] with the constant step, in lam[ring] with the adaptive one
__device__ __forceinline__ const float *lam_k(const RefreshArgs &a) {
    const DevState *st = a.st;
    const int b = st->adaptive ? st->ring : (int)(st->k & 1);
    return b == 0 ? a.lam[0] : (b == 1 ? a.lam[1] : a.lam[2]);
}

// Row pass: r_l = sum_j lambda_lj and B_l = sum_j lambda_lj (x_l - x_j), FP64, one warp per
// row (grid-stride).  The warp reads its row 128 columns at a time and queues the nonzero
// multipliers in shared memory (ballot + prefix count, so the queue order depends only on the
// data); every full round of 32 queued terms is taken one per lane, so the FP64 work is spread
// over all lanes however sparse the row.  Each lane sums its terms in queue order and a fixed
// butterfly combines the lanes: the result does not depend on scheduling.
constexpr int kQueue = 160;  // < 32 left over + 128 new terms
template <int NP>
__device__ __forceinline__ void rows_body(const RefreshArgs &a, int cta, int ncta) {
    if (!refresh_due(a.st, a.period)) return;
    __shared__ float s_w[kRowWarps][kQueue];
    __shared__ int s_j[kRowWarps][kQueue];
    const float *lam = lam_k(a);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *qw = s_w[warp];
    int *qj = s_j[warp];
    const unsigned below = (1u << lane) - 1u;
    for (int l = cta * kRowWarps + warp; l < a.N; l += ncta * kRowWarps) {
        double xl[NP], B[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            xl[k] = k < a.n ? a.X[(long long)l * a.n + k] : 0.0;
            B[k] = 0.0;
        }
        double r = 0.0;
        auto take = [&](int idx) {
            const double w = (double)qw[idx];
            const double *xj = a.X + (long long)qj[idx] * a.n;
            r += w;
#pragma unroll
            for (int k = 0; k < NP; ++k)
                if (k < a.n) B[k] = fma(w, xl[k] - xj[k], B[k]);
        };
        const float *row = lam + (long long)l * a.ld;
        int qn = 0;  // warp-uniform queue length
        for (long long j0 = 0; j0 < a.N; j0 += 128) {
            const long long jj = j0 + 4 * lane;  // < ld: ld is a multiple of 32, the padding holds 0
            float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jj < a.ld) v4 = *reinterpret_cast<const float4 *>(row + jj);
            const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const bool nz = v[c] != 0.f;  // the diagonal and the columns >= N hold 0
                const unsigned m = __ballot_sync(0xffffffffu, nz);
                if (nz) {
                    const int pos = qn + __popc(m & below);
                    qw[pos] = v[c];
                    qj[pos] = (int)(jj + c);
                }
                qn += __popc(m);
            }
            __syncwarp();
            while (qn >= 32) {
                take(qn - 32 + lane);
                qn -= 32;
            }
            __syncwarp();
        }
        if (lane < qn) take(lane);
        __syncwarp();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            r += __shfl_xor_sync(0xffffffffu, r, o);
#pragma unroll
            for (int k = 0; k < NP; ++k) B[k] += __shfl_xor_sync(0xffffffffu, B[k], o);
        }
        if (lane == 0) {
            a.r_out[l] = r;
#pragma unroll
            for (int k = 0; k < NP; ++k)
                if (k < a.n) a.B_out[(long long)l * a.n + k] = B[k];
        }
    }
}

// Column pass: partial column sums over row segments, FP64 ([segs][N]); thread = column.
__device__ __forceinline__ void cols_body(const RefreshArgs &a, int colblk, int seg) {
    if (!refresh_due(a.st, a.period)) return;
    const float *lam = lam_k(a);
    const long long j = (long long)colblk * kColThreads + threadIdx.x;
    if (j >= a.N) return;
    const long long per = (a.N + a.segs - 1) / a.segs;
    const long long i0 = (long long)seg * per, i1 = min((long long)a.N, i0 + per);
    double c = 0.0;
    long long i = i0;
    for (; i + 4 <= i1; i += 4) {  // four loads in flight, added in row order
        const float v0 = lam[i * a.ld + j], v1 = lam[(i + 1) * a.ld + j];
        const float v2 = lam[(i + 2) * a.ld + j], v3 = lam[(i + 3) * a.ld + j];
        c += (double)v0;
        c += (double)v1;
        c += (double)v2;
        c += (double)v3;
    }
    for (; i < i1; ++i) c += (double)lam[i * a.ld + j];
    a.cpart[(long long)seg * a.N + j] = c;
}

__device__ __forceinline__ void split_hi_lo(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// Finish: a = c - r, b = B into the history of lambda^k; the same correction shifts the
// history of lambda^{k-1}; eta(lambda~^{k+1}) for the next sweep; block partials of
// ||a||^2, a.ybar, ||b||^2 and, in the last block, the scalars of lambda^k.
__device__ __forceinline__ void finish_body(const RefreshArgs &a, int blk, int nblk) {
    DevState *st = a.st;
    if (!refresh_due(st, a.period)) return;
    __syncthreads();  // the shared arrays below may still be read from this CTA's previous block
    const int l = blk * kFinThreads + threadIdx.x;
    const long long k = st->k;
    double *a0 = a.hist_a[k & 1], *b0 = a.hist_b[k & 1];
    double *a1 = a.hist_a[(k - 1) & 1], *b1 = a.hist_b[(k - 1) & 1];
    const double beta = st->beta, opb = 1.0 + beta, inv_gamma = st->inv_gamma;
    double saa = 0.0, say = 0.0, sbb = 0.0;
    if (l < a.N) {
        double c = 0.0;
        for (int s = 0; s < a.segs; ++s) c += a.cpart[(long long)s * a.N + l];
        const double al = c - a.r_out[l];
        a1[l] += al - a0[l];
        a0[l] = al;
        const double y = a.ybar[l] + (opb * al - beta * a1[l]);
        double u = y;
        for (int kk = 0; kk < a.n; ++kk) {
            const long long o = (long long)l * a.n + kk;
            const double bl = a.B_out[o];
            b1[o] += bl - b0[o];
            b0[o] = bl;
            sbb += bl * bl;
            const float xf = (float)((opb * bl - beta * b1[o]) * inv_gamma);
            a.xiT[(long long)kk * a.ldv + l] = xf;
            if (a.xi_rm) {
                a.xi_rm[(long long)l * 32 + kk] = xf;
                a.xi_rm[a.ldv * 32 + (long long)l * 32 + kk] = xf - __uint_as_float(__float_as_uint(xf) & 0xFFFFE000u);
            }
            u -= (double)xf * (double)a.xT32[(long long)kk * a.ldv + l];
        }
        split_hi_lo(y, a.yh + l, a.yl + l);
        split_hi_lo(u, a.uh + l, a.ul + l);
        saa = al * al;
        say = al * a.ybar[l];
    }
    __shared__ double s_red[3][kFinThreads];
    s_red[0][threadIdx.x] = saa;
    s_red[1][threadIdx.x] = say;
    s_red[2][threadIdx.x] = sbb;
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 3; ++q) s_red[q][threadIdx.x] += s_red[q][threadIdx.x + w];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) a.blockpart[blk * 3 + q] = s_red[q][0];
        __threadfence();
        last = atomicAdd(&st->fin_counter, 1u) == (unsigned)nblk - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += kFinThreads)
#pragma unroll
        for (int q = 0; q < 3; ++q) v[q] += __ldcg(a.blockpart + b * 3 + q);
#pragma unroll
    for (int q = 0; q < 3; ++q) s_red[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 3; ++q) s_red[q][threadIdx.x] += s_red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double aa = s_red[0][0], ay = s_red[1][0], bb = s_red[2][0], gamma = st->gamma;
        const double g = -0.5 * aa - ay - bb / (2.0 * gamma);
        st->last_g = g;
        st->last_r = 0.5 * aa + bb / (2.0 * gamma);
        st->last_lg = aa + ay + bb / gamma;
        double *lp = a.log + (size_t)((k - 1) % kLogCap) * 3;
        lp[0] = g;
        lp[1] = st->last_r;
        lp[2] = st->last_lg;
        st->prev_g = g;  // the restart test compares with the refreshed value
        st->refreshed_k = k;
        st->refreshes += 1;
        st->fin_counter = 0u;
        __threadfence();
    }
}

__device__ __forceinline__ RefreshArgs args_of(const InstDesc &D) {
    RefreshArgs r{};
    r.N = D.N;
    r.n = D.n;
    r.period = D.rf_period;
    r.segs = D.rf_segs;
    r.ld = D.ld;
    r.ldv = D.ldv;
    for (int i = 0; i < 3; ++i) r.lam[i] = D.lam[i];
    r.X = D.X;
    r.ybar = D.ybar;
    for (int i = 0; i < 2; ++i) {
        r.hist_a[i] = D.ha[i];
        r.hist_b[i] = D.hb[i];
    }
    r.r_out = D.rf_r;
    r.B_out = D.rf_B;
    r.cpart = D.rf_c;
    r.blockpart = D.finblk;
    r.log = D.log;
    r.yh = D.yh;
    r.yl = D.yl;
    r.uh = D.uh;
    r.ul = D.ul;
    r.xiT = D.xiT;
    r.xi_rm = D.xi_rm;
    r.xT32 = D.xT32;
    r.st = D.st;
    return r;
}

// Batched passes: every CTA walks the instances on the due list in list order and takes its
// strided share of each instance's rows, column blocks or point blocks.
__global__ void __launch_bounds__(kRowWarps * 32) refresh_rows_batch_kernel(const InstDesc *d, const int *due) {
    const int nd = due[0];
    for (int q = 0; q < nd; ++q) rows_body<32>(args_of(d[due[1 + q]]), blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kColThreads) refresh_cols_batch_kernel(const InstDesc *d, const int *due) {
    const int nd = due[0];
    for (int q = 0; q < nd; ++q) {
        const RefreshArgs a = args_of(d[due[1 + q]]);
        const int ncb = (a.N + kColThreads - 1) / kColThreads;
        for (int v = blockIdx.x; v < ncb * a.segs; v += gridDim.x) cols_body(a, v % ncb, v / ncb);
    }
}
__global__ void __launch_bounds__(kFinThreads) refresh_finish_batch_kernel(const InstDesc *d, const int *due) {
    const int nd = due[0];
    for (int q = 0; q < nd; ++q) {
        const RefreshArgs a = args_of(d[due[1 + q]]);
        const int nblk = refresh_finish_blocks_dev(a.N);
        for (int v = blockIdx.x; v < nblk; v += gridDim.x) finish_body(a, v, nblk);
    }
}

template <int NP>
__global__ void __launch_bounds__(kRowWarps * 32) refresh_rows_kernel(const RefreshArgs a) {
    rows_body<NP>(a, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kColThreads) refresh_cols_kernel(const RefreshArgs a) {
    cols_body(a, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(kFinThreads) refresh_finish_kernel(const RefreshArgs a) {
    finish_body(a, blockIdx.x, gridDim.x);
}

}  // namespace

int refresh_segments(int N, int sms) {
    const int colblocks = (N + kColThreads - 1) / kColThreads;
    int segs = std::max(1, (4 * sms + colblocks - 1) / colblocks);
    return std::min(segs, std::max(1, N / 64));
}

int refresh_finish_blocks(int N) { return refresh_finish_blocks_dev(N); }

cudaError_t launch_refresh_batch(const InstDesc *d, const int *due, int max_due, int sms, cudaStream_t s) {
    if (max_due <= 0) return cudaSuccess;
    refresh_rows_batch_kernel<<<4 * sms, kRowWarps * 32, 0, s>>>(d, due);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    refresh_cols_batch_kernel<<<4 * sms, kColThreads, 0, s>>>(d, due);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    refresh_finish_batch_kernel<<<2 * sms, kFinThreads, 0, s>>>(d, due);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const RefreshArgs &a, int sms, cudaStream_t s) {
    const int rgrid = std::max(1, std::min((a.N + kRowWarps - 1) / kRowWarps, 8 * sms));
    switch (bucket_np(a.n)) {
#define CASE(V) \
    case V: refresh_rows_kernel<V><<<rgrid, kRowWarps * 32, 0, s>>>(a); break;
        CASE(2) CASE(4) CASE(6) CASE(8) CASE(10) CASE(12) CASE(14) CASE(16) CASE(20) CASE(24) CASE(28) CASE(32)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    refresh_cols_kernel<<<dim3((a.N + kColThreads - 1) / kColThreads, a.segs), kColThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    refresh_finish_kernel<<<refresh_finish_blocks(a.N), kFinThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cr
