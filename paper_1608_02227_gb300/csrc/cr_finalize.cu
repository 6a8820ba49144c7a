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

__device__ __forceinline__ void split_hi_lo(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

// Sum over the column splits of entry e of point l's row partials.  FP32 partials are
// added in FP32 in groups of 8 (pairwise; error ~3 ulp of the group, the level of the FP32
// multipliers themselves) and the groups in FP64: GB300's FP64 pipe bounds this kernel
// otherwise.  FP64 partials are summed in FP64.
template <typename PT>
__device__ __forceinline__ double split_sum(const PT *rowp, int S, long long N, long long l, int W, int e) {
    if constexpr (sizeof(PT) == 8) {
        double s = 0.0;
        for (int sp = 0; sp < S; ++sp) s += rowp[((long long)sp * N + l) * W + e];
        return s;
    } else {
        double s = 0.0;
        int sp = 0;
        for (; sp + 8 <= S; sp += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = rowp[((long long)(sp + u) * N + l) * W + e];
            s += (double)(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
        }
        if (sp == S) return s;
        float t = 0.f;
        for (; sp < S; ++sp) t += rowp[((long long)sp * N + l) * W + e];
        return s + (double)t;
    }
}

constexpr int kFX = 32;   // points per CTA
constexpr int kFY = 8;    // slices per point (row blocks, components)

// One CTA finalizes 32 points; the 8 warps split each point's reductions (row blocks of
// the column sums, components of b) and combine them through shared memory in a fixed
// order, so the result does not depend on scheduling.
template <typename PT>
__device__ __forceinline__ void finalize_body(const FinArgs &a, const int blk, const int nblk) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int l = blk * kFX + tx;
    const bool valid = l < a.N;
    DevState *st = a.st;
    const double gamma = st->gamma, inv_gamma = st->inv_gamma;
    // Steps 3 and 4: t_{k+1} and the extrapolation coefficient, once per CTA (an FP64 square
    // root and divide per thread would dominate this kernel on GB300's narrow FP64 pipe)
    __shared__ double s_tb[2];
    if (threadIdx.x == 0) {
        const double tk = st->t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
        s_tb[0] = tn;
        s_tb[1] = (st->accelerate && !a.init) ? (tk - 1.0) / tn : 0.0;
    }
    const PT *rowp = reinterpret_cast<const PT *>(a.rowpart);
    const PT *colp = reinterpret_cast<const PT *>(a.colpart);
    const int W = a.NP + 1;
    __shared__ double s_c[kFY][kFX], s_u[kFY][kFX], s_b[kFY][kFX];
    __shared__ double s_r[kFX];

    // C^T lambda^k: a_l = c_l - r_l (Definition 1), c_l from the per-row-block partials
    double c = 0.0;
    if (valid && !a.init) {
        // eight independent loads in flight per thread, added in row-block order
        int b = ty;
        for (; b + 7 * kFY < a.row_blocks; b += 8 * kFY) {
            PT v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = colp[(long long)(b + u * kFY) * a.ld + l];
            // FP32 partials: pairwise sums of 8 in FP32 (error ~3 ulp of the group, the level
            // of the FP32 multipliers themselves), groups accumulated in FP64; GB300's FP64
            // pipe is the limit of this kernel otherwise.  FP64 partials stay FP64 throughout.
            c += (double)(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
        }
        for (; b < a.row_blocks; b += kFY) c += (double)colp[(long long)b * a.ld + l];
    }
    s_c[ty][tx] = c;
    if (ty == 0) {
        double r = 0.0;
        if (valid && !a.init) r = split_sum<PT>(rowp, a.col_splits, a.N, l, W, a.NP);
        s_r[tx] = r;
    }
    __syncthreads();
    const double r = s_r[tx];
    const double tn = s_tb[0], beta = s_tb[1], opb = 1.0 + beta;
    // b_l = r_l x_l - sum_j lambda_lj x_j, and Step 1 of the next iteration:
    // C^T lambda~^{k+1} = (1 + beta) C^T lambda^k - beta C^T lambda^{k-1}; xi = b~ / gamma
    double upart = 0.0, bpart = 0.0;
    if (valid) {
        for (int k = ty; k < a.n; k += kFY) {
            const double Bk = a.init ? 0.0 : split_sum<PT>(rowp, a.col_splits, a.N, l, W, k);
            const double xk = a.X[(long long)l * a.n + k];
            // delta form: the partials are of lambda^k - lambda^{k-1} and add to C^T lambda^{k-1}
            const double bl = (a.delta ? a.b_old[(long long)l * a.n + k] : 0.0) + (r * xk - Bk);
            a.b_new[(long long)l * a.n + k] = bl;
            bpart += bl * bl;
            const double bt = opb * bl - beta * a.b_old[(long long)l * a.n + k];
            const double xi = bt * inv_gamma;
            if (a.precision == CR_FP64) {
                a.xiT64[(long long)k * a.ldv + l] = xi;
                upart -= xi * xk;
            } else {
                // the sweep sees the rounded xi and x; u is formed from exactly those
                const float xf = (float)xi;
                a.xiT[(long long)k * a.ldv + l] = xf;
                if (a.xi_rm) {  // tensor-core operand: hi = xf (read as trunc(xf)), lo = xf - trunc(xf)
                    a.xi_rm[(long long)l * 32 + k] = xf;
                    a.xi_rm[a.ldv * 32 + (long long)l * 32 + k] = xf - __uint_as_float(__float_as_uint(xf) & 0xFFFFE000u);
                }
                upart -= (double)xf * (double)a.xT32[(long long)k * a.ldv + l];
            }
        }
    }
    s_u[ty][tx] = upart;
    s_b[ty][tx] = bpart;
    __syncthreads();
    double saa = 0.0, say = 0.0, sbb = 0.0;
    if (ty == 0 && valid) {
        double cc = 0.0;
#pragma unroll
        for (int y = 0; y < kFY; ++y) cc += s_c[y][tx];
        const double al = (a.delta ? a.a_old[l] : 0.0) + (cc - r);
        a.a_new[l] = al;
        const double at = opb * al - beta * a.a_old[l];
        const double y = a.ybar[l] + at;
        double u = y;
#pragma unroll
        for (int q = 0; q < kFY; ++q) {
            u += s_u[q][tx];
            sbb += s_b[q][tx];
        }
        if (a.precision == CR_FP64) {
            a.y64[l] = y;
            a.u64[l] = u;
        } else {
            split_hi_lo(y, a.yh + l, a.yl + l);
            split_hi_lo(u, a.uh + l, a.ul + l);
        }
        saa = al * al;
        say = al * a.ybar[l];
    }
    if (a.init) return;

    __shared__ bool last;
    if (ty == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            saa += __shfl_xor_sync(0xffffffffu, saa, o);
            say += __shfl_xor_sync(0xffffffffu, say, o);
            sbb += __shfl_xor_sync(0xffffffffu, sbb, o);
        }
        if (tx == 0) {
            a.blockpart[blk * 3 + 0] = saa;
            a.blockpart[blk * 3 + 1] = say;
            a.blockpart[blk * 3 + 2] = sbb;
            __threadfence();
            const unsigned ticket = atomicAdd(&st->fin_counter, 1u);
            last = (ticket == (unsigned)nblk - 1u);
        }
    }
    __syncthreads();
    if (!last) return;
    // last CTA: reduce the per-CTA partials in a fixed order (thread t takes CTAs t, t+256, ...)
    __threadfence();
    {
        double aa = 0.0, ay = 0.0, bb = 0.0;
        for (int b = threadIdx.x; b < nblk; b += kFX * kFY) {
            aa += __ldcg(a.blockpart + b * 3 + 0);
            ay += __ldcg(a.blockpart + b * 3 + 1);
            bb += __ldcg(a.blockpart + b * 3 + 2);
        }
        s_c[ty][tx] = aa;
        s_u[ty][tx] = ay;
        s_b[ty][tx] = bb;
    }
    __syncthreads();
    for (int w = kFX * kFY / 2; w > 0; w >>= 1) {
        const int t = threadIdx.x;
        if (t < w) {
            (&s_c[0][0])[t] += (&s_c[0][0])[t + w];
            (&s_u[0][0])[t] += (&s_u[0][0])[t + w];
            (&s_b[0][0])[t] += (&s_b[0][0])[t + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double aa = s_c[0][0], ay = s_u[0][0], bb = s_b[0][0];
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
        st->beta = beta;
        st->fin_counter = 0u;
        if (a.due && a.refresh_period > 0 && k >= 2 * a.refresh_period && k % a.refresh_period == 0)
            a.due[1 + atomicAdd(a.due, 1)] = a.inst;
        __threadfence();
    }
}

template <typename PT>
__global__ void __launch_bounds__(kFX * kFY) finalize_kernel(const FinArgs a) {
    finalize_body<PT>(a, blockIdx.x, gridDim.x);
}

// Adaptive step size (Section 4), pass 1 of an iteration: C^T of the candidate lambda^k,
// the terms of Eq. (adaptive-check), g_gamma(lambda^k), and the accept/reject decision.
// g_gamma is quadratic, so g(l) - g(l~) - <grad g(l~), l - l~> = -1/2 (||da||^2 + ||db||^2/gamma)
// with (da, db) = C^T (l - l~) = (a,b)^k - (a~,b~) (linearity), and the check reads
//     ||da||^2 + ||db||^2 / gamma  <=  s_k ||lambda^k - lambda~^k||^2,
// the last norm summed over all pairs by the sweep.  Accepted: k, t, beta, the log advance,
// the buffer roles rotate and the next candidate tries s_{k+1} = s_k / upsilon; rejected:
// the same sweep runs again with min(s_k * upsilon, L).  Fixed-order reductions throughout.
template <typename PT>
__device__ __forceinline__ void finalize_adapt_body(const FinArgs &a, const int blk, const int nblk) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int l = blk * kFX + tx;
    const bool valid = l < a.N;
    DevState *st = a.st;
    __shared__ long long s_k;
    __shared__ double s_bo;
    if (threadIdx.x == 0) {
        s_k = st->k + 1;  // index of the iteration being tried
        s_bo = st->beta;  // beta of lambda~^k
    }
    const PT *rowp = reinterpret_cast<const PT *>(a.rowpart);
    const PT *colp = reinterpret_cast<const PT *>(a.colpart);
    const int W = a.NP + 1;
    __shared__ double s_c[kFY][kFX], s_u[kFY][kFX], s_b[kFY][kFX];
    __shared__ double s_r[kFX];
    double c = 0.0;
    if (valid) {
        int b = ty;
        for (; b + 7 * kFY < a.row_blocks; b += 8 * kFY) {
            PT v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = colp[(long long)(b + u * kFY) * a.ld + l];
            c += (double)(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])));
        }
        for (; b < a.row_blocks; b += kFY) c += (double)colp[(long long)b * a.ld + l];
    }
    s_c[ty][tx] = c;
    if (ty == 0) s_r[tx] = valid ? split_sum<PT>(rowp, a.col_splits, a.N, l, W, a.NP) : 0.0;
    __syncthreads();
    const double r = s_r[tx];
    const long long k = s_k;
    const double bo = s_bo, opbo = 1.0 + bo;
    const double *a1 = a.hist_a[(k - 1) & 1], *a2 = a.hist_a[k & 1];
    const double *b1 = a.hist_b[(k - 1) & 1], *b2 = a.hist_b[k & 1];
    double bpart = 0.0, dbpart = 0.0;
    if (valid) {
        for (int kk = ty; kk < a.n; kk += kFY) {
            const long long o = (long long)l * a.n + kk;
            const double bl = (a.delta ? b1[o] : 0.0) + (r * a.X[o] - split_sum<PT>(rowp, a.col_splits, a.N, l, W, kk));
            a.b_new[o] = bl;
            bpart += bl * bl;
            const double db = bl - (opbo * b1[o] - bo * b2[o]);  // b^k - b~ of lambda~^k
            dbpart += db * db;
        }
    }
    s_u[ty][tx] = dbpart;
    s_b[ty][tx] = bpart;
    __syncthreads();
    double v6[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // ||a||^2, a.ybar, ||b||^2, ||da||^2, ||db||^2, ||dl||^2
    if (ty == 0 && valid) {
        double cc = 0.0, bb = 0.0, dbb = 0.0;
#pragma unroll
        for (int y = 0; y < kFY; ++y) {
            cc += s_c[y][tx];
            bb += s_b[y][tx];
            dbb += s_u[y][tx];
        }
        const double al = (a.delta ? a1[l] : 0.0) + (cc - r);
        a.a_new[l] = al;
        const double da = al - (opbo * a1[l] - bo * a2[l]);
        const PT *dp = reinterpret_cast<const PT *>(a.dpart);
        double dl = 0.0;
        for (int g = 0; g < a.dgroups; ++g) dl += (double)dp[(long long)g * a.N + l];
        v6[0] = al * al;
        v6[1] = al * a.ybar[l];
        v6[2] = bb;
        v6[3] = da * da;
        v6[4] = dbb;
        v6[5] = dl;
    }
    __shared__ bool last;
    if (ty == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 6; ++q) v6[q] += __shfl_xor_sync(0xffffffffu, v6[q], o);
        if (tx == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q) a.blockpart[blk * 6 + q] = v6[q];
            __threadfence();
            const unsigned ticket = atomicAdd(&st->fin_counter, 1u);
            last = (ticket == (unsigned)nblk - 1u);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double s_red[6][kFX * kFY];
    {
        double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < nblk; b += kFX * kFY)
#pragma unroll
            for (int q = 0; q < 6; ++q) acc[q] += __ldcg(a.blockpart + b * 6 + q);
#pragma unroll
        for (int q = 0; q < 6; ++q) s_red[q][threadIdx.x] = acc[q];
    }
    __syncthreads();
    for (int w = kFX * kFY / 2; w > 0; w >>= 1) {
        const int t = threadIdx.x;
        if (t < w)
#pragma unroll
            for (int q = 0; q < 6; ++q) s_red[q][t] += s_red[q][t + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double gamma = st->gamma, inv_gamma = st->inv_gamma;
        const double aa = s_red[0][0], ay = s_red[1][0], bb = s_red[2][0];
        const double lhs = (s_red[3][0] + s_red[4][0] * inv_gamma) * st->s;  // st->s = 1 / s_k
        const double rhs = s_red[5][0];
        st->check_lhs = lhs;
        st->check_rhs = rhs;
        st->sweeps += 1;
        // s_k = L satisfies the check in exact arithmetic (L bounds the curvature of g_gamma,
        // and Section 4 allows any s_k <= L), so a candidate at 1/L is kept: rounding in the
        // check cannot push the step below the constant one
        if (lhs <= rhs || st->s <= st->inv_L) {
            const double g = -0.5 * aa - ay - bb / (2.0 * gamma);
            const double rr = 0.5 * aa + bb / (2.0 * gamma);
            const double lg = aa + ay + bb / gamma;
            st->last_g = g;
            st->last_r = rr;
            st->last_lg = lg;
            double *lp = a.log + (size_t)((k - 1) % kLogCap) * 3;
            lp[0] = g;
            lp[1] = rr;
            lp[2] = lg;
            const double tk = st->t;
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
            const bool reset = st->restart && k > 1 && g < st->prev_g;  // the ascent went backwards
            st->prev_g = g;
            st->k = k;
            st->t = reset ? 1.0 : tn;
            st->beta = (st->accelerate && !reset) ? (tk - 1.0) / tn : 0.0;
            st->restarts += reset ? 1 : 0;
            st->ring = st->ring == 0 ? 2 : st->ring - 1;  // the candidate becomes lambda^k
            st->s = st->s * st->upsilon;
            st->accepted = 1;
            if (a.due && a.refresh_period > 0 && k >= 2 * a.refresh_period && k % a.refresh_period == 0)
                a.due[1 + atomicAdd(a.due, 1)] = a.inst;
        } else {
            st->s = fmax(st->s / st->upsilon, st->inv_L);
            st->accepted = 0;
        }
        st->fin_counter = 0u;
        __threadfence();
    }
}

template <typename PT>
__global__ void __launch_bounds__(kFX * kFY) finalize_adapt_kernel(const FinArgs a) {
    finalize_adapt_body<PT>(a, blockIdx.x, gridDim.x);
}

// Adaptive step, pass 2 (one thread per point): after an accepted candidate, (a,b)^k takes the
// history slot of (a,b)^{k-2} and Step 1 of the next iteration builds eta(lambda~^{k+1}) with
// C^T lambda~^{k+1} = (1 + beta) C^T lambda^k - beta C^T lambda^{k-1}; after a rejected one
// nothing changes and the next sweep retries from the same lambda~^k.
__device__ __forceinline__ void commit_point(const FinArgs &a, const int l) {
    const DevState *st = a.st;
    if (l >= a.N || !st->accepted) return;
    const long long k = st->k;
    const double beta = st->beta, opb = 1.0 + beta, inv_gamma = st->inv_gamma;
    double *a0 = a.hist_a[k & 1], *b0 = a.hist_b[k & 1];
    const double *a1 = a.hist_a[(k - 1) & 1], *b1 = a.hist_b[(k - 1) & 1];
    const double al = a.a_new[l];
    a0[l] = al;
    const double y = a.ybar[l] + (opb * al - beta * a1[l]);
    double u = y;
    for (int kk = 0; kk < a.n; ++kk) {
        const long long o = (long long)l * a.n + kk;
        const double bl = a.b_new[o];
        b0[o] = bl;
        const double xi = (opb * bl - beta * b1[o]) * inv_gamma;
        if (a.precision == CR_FP64) {
            a.xiT64[(long long)kk * a.ldv + l] = xi;
            u -= xi * a.X[o];
        } else {
            const float xf = (float)xi;
            a.xiT[(long long)kk * a.ldv + l] = xf;
            if (a.xi_rm) {
                a.xi_rm[(long long)l * 32 + kk] = xf;
                a.xi_rm[a.ldv * 32 + (long long)l * 32 + kk] = xf - __uint_as_float(__float_as_uint(xf) & 0xFFFFE000u);
            }
            u -= (double)xf * (double)a.xT32[(long long)kk * a.ldv + l];
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

__global__ void commit_kernel(const FinArgs a) { commit_point(a, blockIdx.x * blockDim.x + threadIdx.x); }

// Batched finalize: one CTA per (instance, 32-point block) of the work-list.
__global__ void __launch_bounds__(kFX * kFY) finalize_batch_kernel(const InstDesc *d, const FinItem *items,
                                                                   int *due) {
    const FinItem it = items[blockIdx.x];
    const InstDesc &D = d[it.inst];
    const long long k = D.st->k + 1;  // index of the iteration being finalized
    FinArgs a{};
    a.N = D.N;
    a.n = D.n;
    a.NP = D.NP;
    a.precision = CR_FP32;
    a.col_splits = D.col_splits;
    a.row_blocks = D.row_blocks;
    a.ld = D.ld;
    a.ldv = D.ldv;
    a.rowpart = D.rowpart;
    a.colpart = D.colpart;
    a.X = D.X;
    a.ybar = D.ybar;
    a.a_new = D.ha[k & 1];
    a.b_new = D.hb[k & 1];
    a.a_old = D.ha[(k - 1) & 1];
    a.b_old = D.hb[(k - 1) & 1];
    a.yh = D.yh;
    a.yl = D.yl;
    a.uh = D.uh;
    a.ul = D.ul;
    a.xiT = D.xiT;
    a.xT32 = D.xT32;
    a.xi_rm = D.xi_rm;
    a.delta = D.delta;
    if (D.delta) {
        a.due = due;
        a.inst = it.inst;
        a.refresh_period = D.rf_period;
    }
    a.blockpart = D.finblk;
    a.log = D.log;
    a.st = D.st;
    a.init = 0;
    if (D.adaptive) {
        a.adaptive = 1;
        a.a_new = D.ha_c;
        a.b_new = D.hb_c;
        for (int i = 0; i < 2; ++i) {
            a.hist_a[i] = D.ha[i];
            a.hist_b[i] = D.hb[i];
        }
        a.dpart = D.dpart;
        a.dgroups = D.dgroups;
        finalize_adapt_body<float>(a, it.block, D.fin_blocks);
    } else {
        finalize_body<float>(a, it.block, D.fin_blocks);
    }
}

// Batched commit (adaptive step): one warp per (instance, 32-point block) of the work-list.
__global__ void commit_batch_kernel(const InstDesc *d, const FinItem *items) {
    const FinItem it = items[blockIdx.x];
    const InstDesc &D = d[it.inst];
    FinArgs a{};
    a.N = D.N;
    a.n = D.n;
    a.precision = CR_FP32;
    a.ldv = D.ldv;
    a.X = D.X;
    a.ybar = D.ybar;
    a.a_new = D.ha_c;
    a.b_new = D.hb_c;
    for (int i = 0; i < 2; ++i) {
        a.hist_a[i] = D.ha[i];
        a.hist_b[i] = D.hb[i];
    }
    a.yh = D.yh;
    a.yl = D.yl;
    a.uh = D.uh;
    a.ul = D.ul;
    a.xiT = D.xiT;
    a.xT32 = D.xT32;
    a.xi_rm = D.xi_rm;
    a.st = D.st;
    commit_point(a, it.block * kFX + (int)threadIdx.x);
}

__global__ void primal_kernel(int N, int n, const double *ybar, const double *av, const double *bv,
                              const DevState *st, double *y, double *xi) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const double gamma = st->gamma;
    if (q < N) y[q] = ybar[q] + av[q];
    if (q < (long long)N * n) xi[q] = bv[q] / gamma;
}

__global__ void transpose_points_kernel(const double *X, int N, int n, int NP, long long ldv,
                                        float *xT32, double *xT64, float *xT2) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)NP * ldv) return;
    const int k = (int)(q / ldv);
    const long long l = q - (long long)k * ldv;
    const double v = (k < n && l < N) ? X[l * n + k] : 0.0;
    if (xT32) xT32[q] = (float)v;
    if (xT64) xT64[q] = v;
    if (xT2) {  // [NP][2 ldv]: every x_lk twice, (x_lk, x_lk) pairs for packed FMAs
        xT2[(long long)k * 2 * ldv + 2 * l] = (float)v;
        xT2[(long long)k * 2 * ldv + 2 * l + 1] = (float)v;
    }
}

__global__ void tc_points_kernel(const double *X, int N, int n, long long ldv, float *xr, float *xt) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= ldv * 32) return;
    const long long j = q / 32;
    const int k = (int)(q - j * 32);
    float hi = 0.f, lo = 0.f, one = 0.f;
    if (j < N && k < n) {
        hi = (float)X[j * n + k];
        lo = hi - __uint_as_float(__float_as_uint(hi) & 0xFFFFE000u);
    }
    if (j < N && k == n) one = 1.f;
    xr[j * 32 + k] = hi;
    xr[ldv * 32 + j * 32 + k] = lo;
    xt[(long long)k * ldv + j] = (k == n) ? one : hi;
    xt[32 * ldv + (long long)k * ldv + j] = lo;
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

int finalize_blocks(int N) { return (int)blocks_for(N, kFX); }

cudaError_t launch_finalize_batch(const InstDesc *d, const FinItem *items, int nitems, int *due, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    finalize_batch_kernel<<<nitems, kFX * kFY, 0, s>>>(d, items, due);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinArgs &a, cudaStream_t s) {
    const unsigned g = blocks_for(a.N, kFX);
    if (a.adaptive) {
        if (a.precision == CR_FP64)
            finalize_adapt_kernel<double><<<g, kFX * kFY, 0, s>>>(a);
        else
            finalize_adapt_kernel<float><<<g, kFX * kFY, 0, s>>>(a);
    } else if (a.precision == CR_FP64) {
        finalize_kernel<double><<<g, kFX * kFY, 0, s>>>(a);
    } else {
        finalize_kernel<float><<<g, kFX * kFY, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_commit_batch(const InstDesc *d, const FinItem *items, int nitems, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    commit_batch_kernel<<<nitems, kFX, 0, s>>>(d, items);
    return cudaGetLastError();
}

cudaError_t launch_commit(const FinArgs &a, cudaStream_t s) {
    commit_kernel<<<blocks_for(a.N, 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_primal(int N, int n, const double *ybar, const double *a, const double *b,
                          const DevState *st, double *y, double *xi, cudaStream_t s) {
    const long long cnt = (long long)N * (n > 1 ? n : 1);
    primal_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(N, n, ybar, a, b, st, y, xi);
    return cudaGetLastError();
}

cudaError_t launch_transpose_points(const double *X, int N, int n, int NP, long long ldv, float *xT32,
                                    double *xT64, float *xT2, cudaStream_t s) {
    transpose_points_kernel<<<blocks_for((long long)NP * ldv, 256), 256, 0, s>>>(X, N, n, NP, ldv, xT32,
                                                                                  xT64, xT2);
    return cudaGetLastError();
}

cudaError_t launch_lambda_to_f64(const void *lam, int is_f32, int N, long long ld, long long row0,
                                 long long rows, double *out, long long ldo, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    lambda_to_f64_kernel<<<blocks_for(rows * N, 256), 256, 0, s>>>(lam, is_f32, N, ld, row0, rows, out,
                                                                   ldo);
    return cudaGetLastError();
}

cudaError_t launch_tc_points(const double *X, int N, int n, long long ldv, float *xr, float *xt, cudaStream_t s) {
    tc_points_kernel<<<blocks_for(ldv * 32, 256), 256, 0, s>>>(X, N, n, ldv, xr, xt);
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
