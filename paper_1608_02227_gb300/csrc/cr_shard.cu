// cr_shard.cu -- row sharding of the multipliers over several GPUs (one shard per context).
//
// A shard holds rows [row0, row_end) of Lambda (every column).  One P-APG iteration (Figure
// "papg", K = N) is then
//   1. the sweep over the shard's rows (the kernels of the whole-instance path, offset to the
//      rows held) and the local reductions (cr_shard_sweep): for every point l the partial
//          v_l = sum over the held rows i of lambda_il  -  [l held] sum_j lambda_lj,
//      i.e. the shard's share of a_l = c_l - r_l (Definition 1), and, appended, ||b_l||^2 summed
//      over the held rows, where b_l = r_l x_l - sum_j lambda_lj x_j needs only row l;
//   2. one all-reduce (sum) of those N + 1 FP64 values over the shards, by the caller;
//   3. the rest of the iteration on every shard alike (cr_shard_finish): a = the summed vector,
//      g_gamma, r_gamma and <lambda, C eta> from ||a||^2, a.ybar and the summed ||b||^2, the t/beta
//      update, and Step 1 of the next iteration: y for every point (the column side of the next
//      sweep), xi and u for the held rows (the row side).
// Every shard keeps X, ybar and a in full and b only for its rows.  The exchange is 8 (N + 1)
// bytes per iteration against 12 (row_end - row0) N bytes of multiplier traffic.
#include <math.h>

#include "cr_host.h"

using namespace crh;

namespace cr {
namespace {

constexpr int kT = 256;

template <typename PT>
__device__ __forceinline__ double sum_splits(const PT *rowp, int S, long long N, long long l, int W, int e) {
    double s = 0.0;
    for (int sp = 0; sp < S; ++sp) s += (double)rowp[((long long)sp * N + l) * W + e];
    return s;
}

struct ShardArgs {
    int N, n, NP, S, RB, row0, row_end, precision;
    long long ld, ldv;
    const void *rowpart, *colpart;
    const double *X, *ybar;
    double *a_new, *b_new;
    const double *a_old, *b_old;
    double *xch;             // N + 1: the exchange vector
    double *blockpart;       // per-block partial sums
    float *yh, *yl, *uh, *ul, *xiT, *xi_rm;
    double *y64, *u64, *xiT64;
    const float *xT32;
    double *log;
    DevState *st;
};

template <typename PT>
__global__ void __launch_bounds__(kT) shard_partial_kernel(const ShardArgs a) {
    const int l = blockIdx.x * kT + threadIdx.x;
    const PT *rowp = reinterpret_cast<const PT *>(a.rowpart);
    const PT *colp = reinterpret_cast<const PT *>(a.colpart);
    const int W = a.NP + 1;
    double bb = 0.0;
    if (l < a.N) {
        double c = 0.0;
        for (int rb = 0; rb < a.RB; ++rb) c += (double)colp[(long long)rb * a.ld + l];
        double v = c;
        if (l >= a.row0 && l < a.row_end) {
            const double r = sum_splits<PT>(rowp, a.S, a.N, l, W, a.NP);
            v -= r;
            for (int k = 0; k < a.n; ++k) {
                const long long o = (long long)l * a.n + k;
                const double bl = r * a.X[o] - sum_splits<PT>(rowp, a.S, a.N, l, W, k);
                a.b_new[o] = bl;
                bb += bl * bl;
            }
        }
        a.xch[l] = v;
    }
    // ||b||^2 of the held rows: block sums, then the last block adds them in block order
    __shared__ double sh[kT];
    __shared__ bool last;
    sh[threadIdx.x] = bb;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.blockpart[blockIdx.x] = sh[0];
        __threadfence();
        last = atomicAdd(&a.st->fin_counter, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kT) t += __ldcg(a.blockpart + b);
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.xch[a.N] = sh[0];
        a.st->fin_counter = 0u;
        __threadfence();
    }
}

__device__ __forceinline__ void split_hi_lo(double v, float *hi, float *lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}

__global__ void __launch_bounds__(kT) shard_finish_kernel(const ShardArgs a) {
    DevState *st = a.st;
    __shared__ double s_tb[2];
    if (threadIdx.x == 0) {  // Steps 3 and 4 (read before the last block updates t)
        const double tk = st->t;
        const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
        s_tb[0] = tn;
        s_tb[1] = st->accelerate ? (tk - 1.0) / tn : 0.0;
    }
    __syncthreads();
    const double tn = s_tb[0], beta = s_tb[1], opb = 1.0 + beta, inv_gamma = st->inv_gamma;
    const int l = blockIdx.x * kT + threadIdx.x;
    double saa = 0.0, say = 0.0;
    if (l < a.N) {
        const double al = a.xch[l];
        a.a_new[l] = al;
        const double y = a.ybar[l] + (opb * al - beta * a.a_old[l]);
        double u = y;
        if (l >= a.row0 && l < a.row_end) {
            for (int k = 0; k < a.n; ++k) {
                const long long o = (long long)l * a.n + k;
                const double xi = (opb * a.b_new[o] - beta * a.b_old[o]) * inv_gamma;
                if (a.precision == CR_FP64) {
                    a.xiT64[(long long)k * a.ldv + l] = xi;
                    u -= xi * a.X[o];
                } else {
                    const float xf = (float)xi;
                    a.xiT[(long long)k * a.ldv + l] = xf;
                    if (a.xi_rm) {
                        a.xi_rm[(long long)l * 32 + k] = xf;
                        a.xi_rm[a.ldv * 32 + (long long)l * 32 + k] = xf - __uint_as_float(__float_as_uint(xf) & 0xFFFFE000u);
                    }
                    u -= (double)xf * (double)a.xT32[(long long)k * a.ldv + l];
                }
            }
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
    __shared__ double sh[2][kT];
    __shared__ bool last;
    sh[0][threadIdx.x] = saa;
    sh[1][threadIdx.x] = say;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.blockpart[2 * blockIdx.x] = sh[0][0];
        a.blockpart[2 * blockIdx.x + 1] = sh[1][0];
        __threadfence();
        last = atomicAdd(&st->fin_counter, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t0 = 0.0, t1 = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kT) {
        t0 += __ldcg(a.blockpart + 2 * b);
        t1 += __ldcg(a.blockpart + 2 * b + 1);
    }
    sh[0][threadIdx.x] = t0;
    sh[1][threadIdx.x] = t1;
    __syncthreads();
    for (int w = kT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double aa = sh[0][0], ay = sh[1][0], bb = a.xch[a.N], gamma = st->gamma;
        const double g = -0.5 * aa - ay - bb / (2.0 * gamma);
        st->last_g = g;
        st->last_r = 0.5 * aa + bb / (2.0 * gamma);
        st->last_lg = aa + ay + bb / gamma;
        const long long k = st->k + 1;
        double *lp = a.log + (size_t)((k - 1) % kLogCap) * 3;
        lp[0] = g;
        lp[1] = st->last_r;
        lp[2] = st->last_lg;
        st->k = k;
        st->t = tn;
        st->beta = beta;
        st->fin_counter = 0u;
        __threadfence();
    }
}

}  // namespace
}  // namespace cr

namespace {

ShardArgs shard_args(const cr_ctx *c, long long k, const double *xch) {
    ShardArgs a{};
    a.N = c->N;
    a.n = c->n;
    a.NP = c->NP;
    a.S = c->S;
    a.RB = c->RB;
    a.row0 = c->row0;
    a.row_end = c->row_end;
    a.precision = c->opt.precision;
    a.ld = c->ld;
    a.ldv = c->ldv;
    a.rowpart = c->rowpart;
    a.colpart = c->colpart;
    a.X = c->X;
    a.ybar = c->ybar;
    a.a_new = c->ha[k & 1];
    a.b_new = c->hb[k & 1];
    a.a_old = c->ha[(k - 1) & 1];
    a.b_old = c->hb[(k - 1) & 1];
    a.xch = const_cast<double *>(xch);
    a.blockpart = c->finblk;
    a.yh = c->yh;
    a.yl = c->yl;
    a.uh = c->uh;
    a.ul = c->ul;
    a.xiT = c->xiT;
    a.xi_rm = c->xi_rm;
    a.y64 = c->y64;
    a.u64 = c->u64;
    a.xiT64 = c->xiT64;
    a.xT32 = c->xT32;
    a.log = c->log;
    a.st = c->st;
    return a;
}

bool shard_ctx(const cr_ctx *c, const char *what) {
    if (!c || !c->shard) {
        set_err("%s needs a context made by cr_shard_create", what);
        return false;
    }
    return true;
}

bool device_ptr(const void *p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

CR_API cr_status cr_shard_create(const double *X, const double *ybar, long long N, int n, long long row0,
                                 long long rows, const cr_options *opt, void *stream, cr_ctx **out) {
    if (!out) {
        set_err("out is NULL");
        return CR_EINVAL;
    }
    *out = nullptr;
    cr_options o;
    if (opt)
        o = *opt;
    else
        cr_default_options(&o);
    if (N < 2 || row0 < 0 || rows < 1 || row0 + rows > N || row0 % 128 != 0) {
        set_err("shard rows [%lld, %lld) of N = %lld: row0 must be a multiple of 128 and the rows inside [0, N)",
                row0, row0 + rows, N);
        return CR_EINVAL;
    }
    if (n > CR_MAX_N_BATCH) {
        set_err("shards hold points with n <= %d", CR_MAX_N_BATCH);
        return CR_EINVAL;
    }
    if (o.step_rule != CR_STEP_CONSTANT) {
        set_err("shards run the constant step of Figure \"papg\" (the adaptive check needs two exchanges)");
        return CR_EUNSUPPORTED;
    }
    o.refresh_every = 0;  // C^T formed from the partials every iteration (no exact refresh across shards)
    o.graph_iters = 0;    // the exchange sits between the launches of an iteration
    cr_ctx *c = nullptr;
    cr_status st = create_window(X, ybar, N, n, (int)row0, (int)(row0 + rows), true, &o, stream, &c);
    if (st != CR_OK) return st;
    *out = c;
    return CR_OK;
}

CR_API cr_status cr_shard_sweep(cr_ctx *c, double *exchange) {
    if (!shard_ctx(c, "cr_shard_sweep")) return CR_EINVAL;
    if (!exchange || !device_ptr(exchange, c->device)) {
        set_err("exchange must be device memory of the context's device (N + 1 doubles)");
        return CR_EINVAL;
    }
    const long long k = c->k + 1;
    CR_TRY(enqueue_sweep(c, k, nullptr));
    const ShardArgs a = shard_args(c, k, exchange);
    const unsigned g = (unsigned)((c->N + kT - 1) / kT);
    if (is_f64(c))
        shard_partial_kernel<double><<<g, kT, 0, c->stream>>>(a);
    else
        shard_partial_kernel<float><<<g, kT, 0, c->stream>>>(a);
    CR_CUDA(cudaGetLastError());
    return CR_OK;
}

CR_API cr_status cr_shard_finish(cr_ctx *c, const double *exchange) {
    if (!shard_ctx(c, "cr_shard_finish")) return CR_EINVAL;
    if (!exchange || !device_ptr(exchange, c->device)) {
        set_err("exchange must be device memory of the context's device (N + 1 doubles)");
        return CR_EINVAL;
    }
    const long long k = c->k + 1;
    const ShardArgs a = shard_args(c, k, exchange);
    shard_finish_kernel<<<(unsigned)((c->N + kT - 1) / kT), kT, 0, c->stream>>>(a);
    CR_CUDA(cudaGetLastError());
    c->k = k;
    return CR_OK;
}

CR_API cr_status cr_shard_state(cr_ctx *c, double *y, double *xi, cr_gap_info *out) {
    if (!shard_ctx(c, "cr_shard_state")) return CR_EINVAL;
    const long long kk = c->k;
    CR_CUDA(launch_primal(c->N, c->n, c->ybar, c->ha[kk & 1], c->hb[kk & 1], c->st, c->tmp_y, c->tmp_xi,
                          c->stream));
    const long long rows = c->row_end - c->row0;
    if (y) CR_CUDA(cudaMemcpyAsync(y, c->tmp_y, sizeof(double) * c->N, cudaMemcpyDefault, c->stream));
    if (xi)
        CR_CUDA(cudaMemcpyAsync(xi, c->tmp_xi + (size_t)c->row0 * c->n, sizeof(double) * rows * c->n,
                                cudaMemcpyDefault, c->stream));
    DevState h{};
    CR_CUDA(cudaMemcpyAsync(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    if (out) {
        cr_gap_info g{};
        g.k = h.k;
        g.dual_g = h.k ? h.last_g : 0.0;
        g.primal_r = h.k ? h.last_r : 0.0;
        g.lagr_gap = h.k ? h.last_lg : 0.0;
        g.step = h.s;
        g.sweeps = h.k;
        g.rel_gap = fabs(g.lagr_gap) / (fabs(g.primal_r) > 1e-300 ? fabs(g.primal_r) : 1e-300);
        *out = g;
    }
    return CR_OK;
}

}  // extern "C"
