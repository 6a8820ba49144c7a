// cr_api.cu -- host side of the C ABI declared in include/cr.h: context set-up, the
// per-iteration launch sequence (sweep -> finalize/recovery), CUDA-graph replay of
// iteration blocks, the solve loop and the result copies.
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "cr_host.h"

using namespace cr;

namespace crh {

thread_local char g_err[512] = "";

void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

bool is_f64(const cr_ctx *c) { return c->opt.precision == CR_FP64; }

// Column splits: enough work items for every SM to get several, with the tail wave as
// full as possible; a split is a whole number of 128-column chunks.
void choose_split(cr_ctx *c) {
    const long long chunks = (c->ld + kChunk - 1) / kChunk;
    const int G = std::max(1, c->sms * std::max(1, c->occ));
    if (c->opt.tile_cols > 0) {
        c->cps = (int)round_up(c->opt.tile_cols, kChunk);
        c->S = (int)((c->ld + c->cps - 1) / c->cps);
    } else {
        int bestS = 1;
        double bestCost = 1e300;
        const int Smax = (int)std::min<long long>(chunks, 64);
        for (int S = 1; S <= Smax; ++S) {
            const long long cps_chunks = (chunks + S - 1) / S;
            const int Sreal = (int)((chunks + cps_chunks - 1) / cps_chunks);
            const long long items = (long long)c->RB * Sreal;
            const long long waves = (items + G - 1) / G;
            // time ~ waves x item length (+ a per-item start cost of ~2 chunks)
            const double cost = (double)waves * (double)(cps_chunks + 2);
            if (cost < bestCost * 0.999) {
                bestCost = cost;
                bestS = S;
            }
        }
        const long long cps_chunks = (chunks + bestS - 1) / bestS;
        c->cps = (int)(cps_chunks * kChunk);
        c->S = (int)((chunks + cps_chunks - 1) / cps_chunks);
    }
    const long long items = (long long)c->RB * c->S;
    c->grid = (int)std::min<long long>(items, (long long)G);
    if (c->tc && c->opt.tile_cols <= 0) {
        // equal ranges of 32-column chunks: the largest CTA share is at most one chunk above the
        // average, where whole items leave a tail wave (N = 20000: 9 items of 80 chunks on some
        // CTAs against 8.26 on average)
        c->seg = true;
        c->seg_nchr = (int)((c->ld + 31) / 32);
        c->seg_total = (long long)c->RB * c->seg_nchr;
        c->grid = (int)std::min<long long>(c->seg_total, (long long)G);
        const long long tmin = c->seg_total / c->grid;
        c->S = (int)((c->seg_nchr + tmin - 1) / tmin + 1);
        c->cps = (int)std::min<long long>(tmin * 32, c->ld);
    }
}

RefreshArgs refresh_args(const cr_ctx *c) {
    RefreshArgs r{};
    r.N = c->N;
    r.n = c->n;
    r.period = c->opt.refresh_every;
    r.segs = c->rf_segs;
    r.ld = c->ld;
    r.ldv = c->ldv;
    for (int i = 0; i < 3; ++i) r.lam[i] = (float *)c->lam[i];
    r.X = c->X;
    r.ybar = c->ybar;
    for (int i = 0; i < 2; ++i) {
        r.hist_a[i] = c->ha[i];
        r.hist_b[i] = c->hb[i];
    }
    r.r_out = c->rf_r;
    r.B_out = c->rf_B;
    r.cpart = c->rf_c;
    r.blockpart = c->finblk;
    r.log = c->log;
    r.yh = c->yh;
    r.yl = c->yl;
    r.uh = c->uh;
    r.ul = c->ul;
    r.xiT = c->xiT;
    r.xi_rm = c->xi_rm;
    r.xT32 = c->xT32;
    r.st = c->st;
    return r;
}

// The sweep of iteration k (1-based): Steps 2 and 4 and the partials of C^T, over the rows the
// context holds.
cr_status enqueue_sweep(cr_ctx *c, long long k, cudaEvent_t e0) {
    const int P = (int)((k - 1) & 1), Q = (int)(k & 1);
    if (e0) CR_CUDA(cudaEventRecord(e0, c->stream));
    if (is_f64(c)) {
        SweepArgsD a{};
        a.P = (const double *)c->lam[P];
        a.Q = (double *)c->lam[Q];
        a.ld = c->ld;
        a.N = c->N;
        a.row_blocks = c->RB;
        a.col_splits = c->S;
        a.cols_per_split = c->cps;
        a.ldv = c->ldv;
        a.xT = c->xT64;
        a.y = c->y64;
        a.u = c->u64;
        a.xiT = c->xiT64;
        a.st = c->st;
        a.rowpart = (double *)c->rowpart;
        a.colpart = (double *)c->colpart;
        a.adaptive = c->adaptive ? 1 : 0;
        for (int i = 0; i < 3; ++i) a.B[i] = (double *)c->lam[i];
        a.dpart = (double *)c->dpart;
        a.row0 = c->row0;
        a.row_end = c->row_end;
        CR_CUDA(launch_sweep_d(c->NP, a, c->grid, c->stream));
    } else if (c->tc) {
        TcSweepArgs a{};
        a.ld = c->ld;
        a.N = c->N;
        a.n = c->n;
        a.NP = c->NP;
        a.row_blocks = c->RB;
        a.col_splits = c->S;
        a.cols_per_split = c->cps;
        a.st = c->st;
        a.ldv = c->ldv;
        a.xi_rm = c->xi_rm;
        a.u = c->uh;
        a.rowpart = (float *)c->rowpart;
        a.colpart = (float *)c->colpart;
        a.err = reinterpret_cast<int *>(reinterpret_cast<char *>(c->st) + offsetof(DevState, err));
        a.lmaps = c->tc_ld;
        a.p_host = P;
        a.adaptive = c->adaptive ? 1 : 0;
        a.dpart = (float *)c->dpart;
        a.delta = c->delta ? 1 : 0;
        a.row0 = c->row0;
        a.row_end = c->row_end;
        a.seg = c->seg ? 1 : 0;
        a.seg_nchr = c->seg_nchr;
        a.seg_total = c->seg_total;
        CR_CUDA(launch_sweep_tc(c->tcm, a, c->grid, c->stream));
    } else if (c->tma) {
        TmaSweepArgs a{};
        a.Q = (float *)c->lam[Q];
        a.ld = c->ld;
        a.N = c->N;
        a.row_blocks = c->RB;
        a.col_splits = c->S;
        a.cols_per_split = c->cps;
        a.st = c->st;
        a.rowpart = (float *)c->rowpart;
        a.colpart = (float *)c->colpart;
        a.err = reinterpret_cast<int *>(reinterpret_cast<char *>(c->st) + offsetof(DevState, err));
        a.adaptive = c->adaptive ? 1 : 0;
        a.lmaps = c->tm_ld;
        for (int i = 0; i < 3; ++i) a.B[i] = (float *)c->lam[i];
        a.dpart = (float *)c->dpart;
        a.consumer_wait_ns = c->consumer_wait_ns;
        a.delta = c->delta ? 1 : 0;
        a.row0 = c->row0;
        a.row_end = c->row_end;
        TmaMaps m = c->tm;
        m.P = &c->tm_lam[P];
        m.Q = &c->tm_lam[Q];
        CR_CUDA(launch_sweep_tma(c->NP, m, a, c->grid, c->stream));
    } else {
        SweepArgsF a{};
        a.P = (const float *)c->lam[P];
        a.Q = (float *)c->lam[Q];
        a.ld = c->ld;
        a.N = c->N;
        a.row_blocks = c->RB;
        a.col_splits = c->S;
        a.cols_per_split = c->cps;
        a.ldv = c->ldv;
        a.xT = c->xT32;
        a.yh = c->yh;
        a.yl = c->yl;
        a.uh = c->uh;
        a.ul = c->ul;
        a.xiT = c->xiT;
        a.st = c->st;
        a.rowpart = (float *)c->rowpart;
        a.colpart = (float *)c->colpart;
        a.adaptive = c->adaptive ? 1 : 0;
        for (int i = 0; i < 3; ++i) a.B[i] = (float *)c->lam[i];
        a.dpart = (float *)c->dpart;
        CR_CUDA(launch_sweep_f(c->NP, a, c->grid, c->stream));
    }
    return CR_OK;
}

cr_status enqueue_iteration(cr_ctx *c, long long k /* 1-based iteration index */, cudaEvent_t e0,
                            cudaEvent_t e1) {
    CR_TRY(enqueue_sweep(c, k, e0));
    if (e1) CR_CUDA(cudaEventRecord(e1, c->stream));
    FinArgs f{};
    f.N = c->N;
    f.n = c->n;
    f.NP = c->NP;
    f.precision = c->opt.precision;
    f.col_splits = c->S;
    f.row_blocks = c->RB;
    f.ld = c->ld;
    f.ldv = c->ldv;
    f.rowpart = c->rowpart;
    f.colpart = c->colpart;
    f.X = c->X;
    f.ybar = c->ybar;
    f.a_new = c->ha[k & 1];
    f.b_new = c->hb[k & 1];
    f.a_old = c->ha[(k - 1) & 1];
    f.b_old = c->hb[(k - 1) & 1];
    f.yh = c->yh;
    f.yl = c->yl;
    f.uh = c->uh;
    f.ul = c->ul;
    f.xiT = c->xiT;
    f.y64 = c->y64;
    f.u64 = c->u64;
    f.xiT64 = c->xiT64;
    f.xT32 = c->xT32;
    f.xi_rm = c->xi_rm;
    f.blockpart = c->finblk;
    f.log = c->log;
    f.st = c->st;
    f.init = 0;
    f.delta = c->delta ? 1 : 0;
    if (c->adaptive) {  // pass 1 decides on the device; the roles of the buffers follow from it
        f.adaptive = 1;
        f.a_new = c->ha_c;
        f.b_new = c->hb_c;
        for (int i = 0; i < 2; ++i) {
            f.hist_a[i] = c->ha[i];
            f.hist_b[i] = c->hb[i];
        }
        f.dpart = c->dpart;
        f.dgroups = c->dgroups;
    }
    CR_CUDA(launch_finalize(f, c->stream));
    if (c->adaptive) CR_CUDA(launch_commit(f, c->stream));
    if (c->delta) CR_CUDA(launch_refresh(refresh_args(c), c->sms, c->stream));
    return CR_OK;
}

cr_status build_graph(cr_ctx *c) {
    if (c->gexec) return CR_OK;
    const int len = c->opt.graph_iters;
    cudaGraph_t g = nullptr;
    CR_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cr_status s = CR_OK;
    // replays start when an even number of iterations is done, so the first captured
    // iteration has the odd index k + 1 (reads lam[0], writes lam[1])
    for (int i = 0; i < len && s == CR_OK; ++i) s = enqueue_iteration(c, 1 + i, nullptr, nullptr);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != CR_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        set_err("graph capture failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        set_err("graph instantiation failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    c->glen = len;
    return CR_OK;
}

cr_status fetch_state(const cr_ctx *c, DevState *h) {
    CR_CUDA(cudaMemcpyAsync(h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

cr_status check_finite_host(cr_ctx *c, const double *dev, long long count, const char *what) {
    CR_CUDA(cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    CR_CUDA(launch_check_finite(dev, count, c->flag, c->stream));
    int h = 0;
    CR_CUDA(cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        set_err("%s contains a non-finite value", what);
        return CR_EINVAL;
    }
    return CR_OK;
}

cr_status create_impl(cr_ctx *c, const double *X, const double *ybar) {
    const int N = c->N, n = c->n;
    CR_CUDA(cudaGetDevice(&c->device));
    CR_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device));
    c->NP = bucket_np(n);
    c->ld = round_up(N, 32);
    c->ldv = round_up(N, kChunk);
    const bool f64 = is_f64(c);
    const size_t tsz = f64 ? sizeof(double) : sizeof(float);

    SweepConfig cfg{};
    if (!(f64 ? sweep_config_d(c->NP, &cfg) : sweep_config_f(c->NP, &cfg))) {
        set_err("no sweep kernel for n = %d", n);
        return CR_EINVAL;
    }
    // FP32 runs the TMA-pipelined sweep; CR_SWEEP=simple selects the plain FP32 kernel
    // (same arithmetic, loads through registers) for A/B measurements.
    const char *variant = getenv("CR_SWEEP");
    c->tc = c->opt.precision == CR_MIXED_TF32;
    c->tma = !f64 && !c->tc && c->NP <= 32 && !(variant && strcmp(variant, "simple") == 0);
    c->rows = c->tc ? sweep_tc_rows() : (c->tma ? sweep_tma_rows(c->NP) : cfg.rows);
    const int LR = c->row_end - c->row0;  // rows of Lambda held (all N, or a shard's)
    c->RB = (LR + c->rows - 1) / c->rows;
    if (c->tc)
        CR_CUDA(sweep_tc_occupancy(&c->occ));
    else if (c->tma)
        CR_CUDA(sweep_tma_occupancy(c->NP, &c->occ));
    else
        CR_CUDA(f64 ? sweep_occupancy_d(c->NP, &c->occ) : sweep_occupancy_f(c->NP, &c->occ));
    if (c->occ < 1) {
        int d[4] = {0, 0, 0, 0};
        if (c->tma) sweep_tma_diag(d);
        set_err("the sweep kernel for n = %d does not fit on this device (occupancy 0; regs %d, max threads %d, "
                "smem %d, threads %d)", n, d[0], d[1], d[2], d[3]);
        return CR_EUNSUPPORTED;
    }
    choose_split(c);
    if (c->shard && !f64 && !c->tc && !c->tma) {
        set_err("shards run the FP64, TMA or tensor-core sweep");
        return CR_EUNSUPPORTED;
    }
    if (c->adaptive && !f64 && !c->tc && !c->tma && c->NP <= 32) {
        set_err("the adaptive step needs the TMA, tensor-core or FP64 sweep (CR_SWEEP=simple has none)");
        return CR_EUNSUPPORTED;
    }

    CR_TRY(dev_alloc(c, &c->X, (size_t)N * n));
    CR_TRY(dev_alloc(c, &c->ybar, (size_t)N));
    CR_TRY(dev_alloc(c, &c->flag, 1));
    CR_CUDA(cudaMemcpyAsync(c->X, X, sizeof(double) * N * n, cudaMemcpyDefault, c->stream));
    CR_CUDA(cudaMemcpyAsync(c->ybar, ybar, sizeof(double) * N, cudaMemcpyDefault, c->stream));
    CR_TRY(check_finite_host(c, c->X, (long long)N * n, "X"));
    CR_TRY(check_finite_host(c, c->ybar, N, "ybar"));
    {
        std::vector<double> hy(N);
        CR_CUDA(cudaMemcpy(hy.data(), c->ybar, sizeof(double) * N, cudaMemcpyDeviceToHost));
        double s = 0.0;
        for (double v : hy) s += v * v;
        c->ybar_rms = sqrt(s / N);
        if (!(c->ybar_rms > 0.0)) c->ybar_rms = 1.0;
    }

    const size_t vec = (size_t)c->ldv;
    const size_t tvec = (size_t)c->NP * c->ldv;
    if (f64) {
        CR_TRY(dev_alloc(c, &c->xT64, tvec));
        CR_TRY(dev_alloc(c, &c->y64, vec));
        CR_TRY(dev_alloc(c, &c->u64, vec));
        CR_TRY(dev_alloc(c, &c->xiT64, tvec));
        CR_TRY(dev_alloc(c, &c->c_y64, vec));
        CR_TRY(dev_alloc(c, &c->c_u64, vec));
        CR_TRY(dev_alloc(c, &c->c_xiT64, tvec));
        CR_CUDA(cudaMemsetAsync(c->xiT64, 0, tvec * sizeof(double), c->stream));
        CR_CUDA(cudaMemsetAsync(c->c_xiT64, 0, tvec * sizeof(double), c->stream));
        CR_CUDA(cudaMemsetAsync(c->y64, 0, vec * sizeof(double), c->stream));
        CR_CUDA(cudaMemsetAsync(c->u64, 0, vec * sizeof(double), c->stream));
    } else {
        CR_TRY(dev_alloc(c, &c->xT32, tvec));
        // hi and lo halves adjacent ([2][ldv]) so one 2-D TMA box fetches both
        float **f[] = {&c->yh, &c->uh, &c->c_yh, &c->c_uh};
        for (float **p : f) {
            CR_TRY(dev_alloc(c, p, 2 * vec));
            CR_CUDA(cudaMemsetAsync(*p, 0, 2 * vec * sizeof(float), c->stream));
        }
        c->yl = c->yh + vec;
        c->ul = c->uh + vec;
        c->c_yl = c->c_yh + vec;
        c->c_ul = c->c_uh + vec;
        CR_TRY(dev_alloc(c, &c->xiT, tvec));
        CR_TRY(dev_alloc(c, &c->c_xiT, tvec));
        CR_CUDA(cudaMemsetAsync(c->xiT, 0, tvec * sizeof(float), c->stream));
        CR_CUDA(cudaMemsetAsync(c->c_xiT, 0, tvec * sizeof(float), c->stream));
    }
    CR_CUDA(launch_transpose_points(c->X, N, n, c->NP, c->ldv, c->xT32, c->xT64, nullptr, c->stream));

    // step constant (Section 3 "Preprocess" + Eq. (lischitz))
    if (c->opt.lipschitz > 0.0) {
        c->L = c->opt.lipschitz;
    } else {
        CR_CUDA(a2_sigma_sq(c->X, N, n, &c->a2s2, c->stream));
        c->L = (c->opt.lipschitz_rule == CR_L_PAPER) ? (2.0 * N + c->a2s2) / c->opt.gamma
                                                     : 2.0 * N + c->a2s2 / c->opt.gamma;
    }
    if (!(c->L > 0.0) || !isfinite(c->L)) {
        set_err("invalid Lipschitz constant %g", c->L);
        return CR_ENUMERIC;
    }

    // multipliers: lambda^0 = lambda^{-1} = 0 (and a zeroed third buffer for the adaptive step)
    const size_t lam_count = (size_t)LR * c->ld;
    const int nbuf = c->adaptive ? 3 : 2;
    for (int i = 0; i < nbuf; ++i) {
        if (f64) {
            double *p;
            CR_TRY(dev_alloc(c, &p, lam_count));
            c->lam[i] = p;
        } else {
            float *p;
            CR_TRY(dev_alloc(c, &p, lam_count));
            c->lam[i] = p;
        }
        CR_CUDA(cudaMemsetAsync(c->lam[i], 0, lam_count * tsz, c->stream));
    }
    for (int i = 0; i < 2; ++i) {
        CR_TRY(dev_alloc(c, &c->ha[i], (size_t)N));
        CR_TRY(dev_alloc(c, &c->hb[i], (size_t)N * n));
        CR_CUDA(cudaMemsetAsync(c->ha[i], 0, sizeof(double) * N, c->stream));
        CR_CUDA(cudaMemsetAsync(c->hb[i], 0, sizeof(double) * N * n, c->stream));
    }
    if (c->adaptive) {
        CR_TRY(dev_alloc(c, &c->ha_c, (size_t)N));
        CR_TRY(dev_alloc(c, &c->hb_c, (size_t)N * n));
        c->dgroups = c->S * (c->tc ? 2 : 1);
        if (f64) {
            double *p;
            CR_TRY(dev_alloc(c, &p, (size_t)c->dgroups * N));
            c->dpart = p;
        } else {
            float *p;
            CR_TRY(dev_alloc(c, &p, (size_t)c->dgroups * N));
            c->dpart = p;
        }
        // slots no sweep item writes (fewer pieces in a row block than S) stay zero
        CR_CUDA(cudaMemsetAsync(c->dpart, 0, (size_t)c->dgroups * N * tsz, c->stream));
    }
    if (c->tc) {
        const size_t rm = (size_t)c->ldv * 32;
        CR_TRY(dev_alloc(c, &c->xr, 2 * rm));
        CR_TRY(dev_alloc(c, &c->xt, 2 * rm));
        CR_TRY(dev_alloc(c, &c->xi_rm, 2 * rm));
        CR_CUDA(cudaMemsetAsync(c->xi_rm, 0, 2 * rm * sizeof(float), c->stream));
        CR_CUDA(launch_tc_points(c->X, N, n, c->ldv, c->xr, c->xt, c->stream));
        // one map per buffer, box 32 x 128: the loads of lambda^{k-1}, lambda^{k-2} and the store
        // of lambda^k (rows past the buffer's last are filled with zeros / not written)
        CUtensorMap hl[3];
        memset(hl, 0, sizeof(hl));
        for (int i = 0; i < nbuf; ++i)
            CR_CUDA(make_tmap_2d(&hl[i], (const float *)c->lam[i], c->ld, LR, c->ld, 32, 128, true));
        CR_TRY(dev_alloc(c, &c->tc_ld, 3));
        memcpy(c->tc_lam_ld, hl, sizeof(hl));
        CR_CUDA(cudaMemcpyAsync(c->tc_ld, c->tc_lam_ld, sizeof(hl), cudaMemcpyHostToDevice, c->stream));
        CR_CUDA(make_tmap_2d(&c->tcm.XRh, c->xr, 32, c->ldv, 32, 32, 128, true));
        CR_CUDA(make_tmap_2d(&c->tcm.XRl, c->xr + rm, 32, c->ldv, 32, 32, 128, true));
        CR_CUDA(make_tmap_2d(&c->tcm.XT, c->xt, c->ldv, 64, c->ldv, 32, 64, true));
        CR_CUDA(make_tmap_2d(&c->tcm.Y, c->yh, c->ldv, 2, c->ldv, 32, 2));
    }
    if (c->tma) {
        memset(c->tm_lam, 0, sizeof(c->tm_lam));
        for (int i = 0; i < nbuf; ++i)
            CR_CUDA(make_tmap_2d(&c->tm_lam[i], (const float *)c->lam[i], c->ld, LR, c->ld, kChunk, c->rows));
        if (c->adaptive) {
            CR_TRY(dev_alloc(c, &c->tm_ld, 3));
            CR_CUDA(cudaMemcpyAsync(c->tm_ld, c->tm_lam, sizeof(c->tm_lam), cudaMemcpyHostToDevice, c->stream));
        }
        CR_CUDA(make_tmap_2d(&c->tm.X, c->xT32, c->ldv, c->NP, c->ldv, kChunk, c->NP));
        CR_CUDA(make_tmap_2d(&c->tm.Y, c->yh, c->ldv, 2, c->ldv, kChunk, 2));
        CR_CUDA(make_tmap_2d(&c->tm.Xi, c->xiT, c->ldv, c->NP, c->ldv, c->rows, c->NP));
        CR_CUDA(make_tmap_2d(&c->tm.U, c->uh, c->ldv, 2, c->ldv, c->rows, 2));
    }
    const size_t rp = (size_t)c->S * N * (c->NP + 1), cp = (size_t)c->RB * c->ld;
    if (f64) {
        double *a, *b;
        CR_TRY(dev_alloc(c, &a, rp));
        CR_TRY(dev_alloc(c, &b, cp));
        c->rowpart = a;
        c->colpart = b;
    } else {
        float *a, *b;
        CR_TRY(dev_alloc(c, &a, rp));
        CR_TRY(dev_alloc(c, &b, cp));
        c->rowpart = a;
        c->colpart = b;
    }
    CR_CUDA(cudaMemsetAsync(c->rowpart, 0, rp * tsz, c->stream));  // slots no item writes stay zero
    // delta form of the C^T reductions (FP32 TMA sweep), with its exact refresh scratch
    c->delta = c->opt.refresh_every > 0 && (c->tma || c->tc);
    if (c->delta) {
        c->rf_segs = refresh_segments(N, c->sms);
        CR_TRY(dev_alloc(c, &c->rf_r, (size_t)N));
        CR_TRY(dev_alloc(c, &c->rf_B, (size_t)N * n));
        CR_TRY(dev_alloc(c, &c->rf_c, (size_t)c->rf_segs * N));
    }
    const int gN = (N + 255) / 256;
    CR_TRY(dev_alloc(c, &c->finblk, (size_t)std::max(finalize_blocks(N) * 6, refresh_finish_blocks(N) * 3)));
    CR_TRY(dev_alloc(c, &c->certblk, (size_t)gN * 2));
    CR_TRY(dev_alloc(c, &c->log, (size_t)kLogCap * 3));
    CR_TRY(dev_alloc(c, &c->st, 1));
    CR_TRY(dev_alloc(c, &c->tmp_y, (size_t)N));
    CR_TRY(dev_alloc(c, &c->tmp_xi, (size_t)N * n));
    // certificate row splits: fill about two waves of the GPU
    c->cert_R = std::max(1, std::min(64, (2 * c->sms + gN - 1) / gN));
    while (c->cert_R > 1 && (N + c->cert_R - 1) / c->cert_R < 64) --c->cert_R;
    CR_TRY(dev_alloc(c, &c->pmax, (size_t)c->cert_R * N));
    CR_TRY(dev_alloc(c, &c->pinf, (size_t)c->cert_R * N));
    CR_TRY(dev_alloc(c, &c->parg, (size_t)c->cert_R * N));

    DevState h{};
    h.t = 1.0;
    h.beta = 0.0;
    h.s = 1.0 / c->L;
    h.gamma = c->opt.gamma;
    h.inv_gamma = 1.0 / c->opt.gamma;
    h.k = 0;
    h.accelerate = c->opt.accelerate ? 1 : 0;
    if (c->adaptive) {  // the first candidate tries s_1 = s_0 / upsilon with s_0 = L
        h.adaptive = 1;
        h.ring = 0;
        h.upsilon = c->opt.upsilon;
        h.inv_L = 1.0 / c->L;
        h.restart = c->opt.restart ? 1 : 0;
        h.s = c->opt.upsilon / c->L;
    }
    CR_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));

    // eta(lambda~^1) = eta(lambda^0) = (ybar, 0)
    FinArgs f{};
    f.N = N;
    f.n = n;
    f.NP = c->NP;
    f.precision = c->opt.precision;
    f.col_splits = c->S;
    f.row_blocks = c->RB;
    f.ld = c->ld;
    f.ldv = c->ldv;
    f.X = c->X;
    f.ybar = c->ybar;
    f.a_new = c->ha[0];
    f.b_new = c->hb[0];
    f.a_old = c->ha[1];
    f.b_old = c->hb[1];
    f.yh = c->yh;
    f.yl = c->yl;
    f.uh = c->uh;
    f.ul = c->ul;
    f.xiT = c->xiT;
    f.y64 = c->y64;
    f.u64 = c->u64;
    f.xiT64 = c->xiT64;
    f.xT32 = c->xT32;
    f.xi_rm = c->xi_rm;
    f.blockpart = c->finblk;
    f.log = c->log;
    f.st = c->st;
    f.init = 1;
    CR_CUDA(launch_finalize(f, c->stream));
    CR_CUDA(cudaEventCreate(&c->ev[0]));
    CR_CUDA(cudaEventCreate(&c->ev[1]));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

// The accepted iteration count and the buffer holding lambda^k: host-side with the constant
// step, from the device state with the adaptive one (its accept/reject runs on the device).
cr_status current_k(const cr_ctx *c, long long *k, int *lam_buf) {
    if (!c->adaptive) {
        *k = c->k;
        *lam_buf = (int)(c->k & 1);
        return CR_OK;
    }
    DevState h{};
    CR_TRY(fetch_state(c, &h));
    *k = h.k;
    *lam_buf = h.ring;
    return CR_OK;
}

// Enqueues the pass over all pairs for eta(lambda^k) (certificate + infeasibility).
cr_status gap_launch(cr_ctx *c) {
    long long kk = 0;
    int lb = 0;
    CR_TRY(current_k(c, &kk, &lb));
    return gap_launch_k(c, kk);
}

// The same for a known accepted iteration count k (no device round trip).
cr_status gap_launch_k(cr_ctx *c, long long kk) {
    CertArgs a{};
    a.N = c->N;
    a.n = c->n;
    a.NP = c->NP;
    a.precision = c->opt.precision;
    a.row_splits = c->cert_R;
    a.ldv = c->ldv;
    a.X = c->X;
    a.ybar = c->ybar;
    a.a = c->ha[kk & 1];
    a.b = c->hb[kk & 1];
    a.yh = c->c_yh;
    a.yl = c->c_yl;
    a.uh = c->c_uh;
    a.ul = c->c_ul;
    a.xiT = c->c_xiT;
    a.y64 = c->c_y64;
    a.u64 = c->c_u64;
    a.xiT64 = c->c_xiT64;
    a.xT32 = c->xT32;
    a.xT64 = c->xT64;
    a.pmax = c->pmax;
    a.parg = c->parg;
    a.pinf = c->pinf;
    a.blockpart = c->certblk;
    a.st = c->st;
    CR_CUDA(launch_cert(a, c->stream));
    return CR_OK;
}

// Convergence record from the device scalars (after gap_launch and a copy of the state).
cr_status gap_finish(const cr_ctx *c, DevState h, cr_gap_info *out) {
    if (h.err) {
        set_err("a device-side wait ran out (status %d) before iteration %lld", h.err, h.k + 1);
        return CR_ETIMEOUT;
    }
    cr_gap_info g{};
    g.k = h.k;
    if (h.k == 0) {  // lambda^0 = 0: eta = (ybar, 0), g = r = 0
        h.last_g = 0.0;
        h.last_r = 0.0;
        h.last_lg = 0.0;
    }
    g.dual_g = h.last_g;
    g.primal_r = h.last_r;
    g.lagr_gap = h.last_lg;
    const double pairs = (double)c->N * (double)(c->N - 1);
    g.infeas_norm = sqrt(h.cert_infeas_sq / pairs);
    const double rden = fabs(g.primal_r) > 1e-300 ? fabs(g.primal_r) : 1e-300;
    g.rel_gap = std::max(fabs(g.lagr_gap) / rden, g.infeas_norm / c->ybar_rms);
    g.cert_primal = h.cert_P;
    g.cert_gap_rel = (h.cert_P - h.last_g) / (fabs(h.cert_P) > 1e-300 ? fabs(h.cert_P) : 1e-300);
    g.step = h.s;
    g.sweeps = c->adaptive ? h.sweeps : h.k;
    if (out) *out = g;
    if (!isfinite(g.dual_g) || !isfinite(g.primal_r) || !isfinite(g.cert_primal)) {
        set_err("non-finite objective at k = %lld", h.k);
        return CR_ENUMERIC;
    }
    return CR_OK;
}

}  // namespace crh

using namespace crh;

extern "C" {

CR_API void cr_default_options(cr_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->gamma = 1e-4;
    o->lipschitz = 0.0;
    o->lipschitz_rule = CR_L_HESSIAN;
    o->precision = CR_FP32;
    o->accelerate = 1;
    o->check_every = 100;
    o->graph_iters = 32;
    o->tile_cols = 0;
    o->deterministic = 1;
    o->step_rule = CR_STEP_CONSTANT;
    o->upsilon = 2.0;
    o->refresh_every = 64;
}

CR_API cr_status cr_create(const double *X, const double *ybar, long long N, int n, const cr_options *opt,
                           void *stream, cr_ctx **out) {
    return create_window(X, ybar, N, n, 0, (int)std::min<long long>(N, 1LL << 30), false, opt, stream, out);
}
}  // extern "C"

namespace crh {

// A context over rows [row0, row_end) of Lambda (all N for cr_create, a shard for
// cr_shard_create).
cr_status create_window(const double *X, const double *ybar, long long N, int n, int row0, int row_end, bool shard,
                        const cr_options *opt, void *stream, cr_ctx **out) {
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
    if (!X || !ybar) {
        set_err("X or ybar is NULL");
        return CR_EINVAL;
    }
    if (N < 2 || N > (1LL << 30)) {
        set_err("N = %lld out of range [2, 2^30]", N);
        return CR_EINVAL;
    }
    if (n < 1 || n > CR_MAX_N) {
        set_err("n = %d out of range [1, %d]", n, CR_MAX_N);
        return CR_EINVAL;
    }
    if (!(o.gamma > 0.0) || !isfinite(o.gamma)) {
        set_err("gamma must be finite and > 0");
        return CR_EINVAL;
    }
    if (o.precision != CR_FP64 && o.precision != CR_FP32 && o.precision != CR_MIXED_TF32) {
        set_err("unknown precision %d", o.precision);
        return CR_EINVAL;
    }
    if (o.precision == CR_MIXED_TF32 && n > CR_MAX_N_TF32) {
        set_err("CR_MIXED_TF32 handles n <= 31 (a row of ones joins the 32-wide operand)");
        return CR_EUNSUPPORTED;
    }
    if (!(o.lipschitz >= 0.0) || !isfinite(o.lipschitz)) {
        set_err("lipschitz must be finite and >= 0");
        return CR_EINVAL;
    }
    if (o.step_rule != CR_STEP_CONSTANT && o.step_rule != CR_STEP_ADAPTIVE) {
        set_err("unknown step rule %d", o.step_rule);
        return CR_EINVAL;
    }
    if (o.step_rule == CR_STEP_ADAPTIVE) {
        if (!(o.upsilon > 1.0) || !isfinite(o.upsilon)) {
            set_err("upsilon must be finite and > 1");
            return CR_EINVAL;
        }

    }
    if (o.check_every < 1) o.check_every = 1;
    if (o.graph_iters < 0 || (o.graph_iters & 1)) {
        set_err("graph_iters must be even and >= 0");
        return CR_EINVAL;
    }
    if (o.tile_cols < 0) {
        set_err("tile_cols must be >= 0");
        return CR_EINVAL;
    }
    if (o.refresh_every < 0) {
        set_err("refresh_every must be >= 0");
        return CR_EINVAL;
    }
    cr_ctx *c = new (std::nothrow) cr_ctx();
    if (!c) {
        set_err("host allocation failed");
        return CR_ENOMEM;
    }
    c->N = (int)N;
    c->row0 = row0;
    c->row_end = row_end;
    c->shard = shard;
    c->n = n;
    c->opt = o;
    c->adaptive = o.step_rule == CR_STEP_ADAPTIVE;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            set_err("cudaStreamCreate failed: %s", cudaGetErrorString(e));
            delete c;
            return CR_ECUDA;
        }
        c->own_stream = true;
    }
    cr_status s = create_impl(c, X, ybar);
    if (s != CR_OK) {
        cr_destroy(c);
        return s;
    }
    *out = c;
    return CR_OK;
}

}  // namespace crh

extern "C" {

CR_API cr_status cr_dual_step(cr_ctx *c, int iters) {
    if (c && c->shard) {
        set_err("cr_dual_step works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || iters < 0) {
        set_err("bad argument to cr_dual_step");
        return CR_EINVAL;
    }
    int left = iters;
    const int G = c->opt.graph_iters;
    if (G > 0 && left >= G + (int)(c->k & 1)) {
        if (c->k & 1) {  // graphs start at an even iteration count
            CR_TRY(enqueue_iteration(c, c->k + 1, nullptr, nullptr));
            ++c->k;
            --left;
        }
        CR_TRY(build_graph(c));
        while (left >= G) {
            CR_CUDA(cudaGraphLaunch(c->gexec, c->stream));
            c->k += G;
            left -= G;
        }
    }
    while (left > 0) {
        CR_TRY(enqueue_iteration(c, c->k + 1, nullptr, nullptr));
        ++c->k;
        --left;
    }
    return CR_OK;
}

CR_API cr_status cr_dual_step_timed(cr_ctx *c, int iters, float *sweep_ms, float *total_ms) {
    if (c && c->shard) {
        set_err("cr_dual_step_timed works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || iters < 0) {
        set_err("bad argument to cr_dual_step_timed");
        return CR_EINVAL;
    }
    std::vector<cudaEvent_t> evs(2 * (size_t)iters + 1);
    for (auto &e : evs) CR_CUDA(cudaEventCreate(&e));
    cr_status s = CR_OK;
    cudaEvent_t start = evs[2 * (size_t)iters];
    CR_CUDA(cudaEventRecord(start, c->stream));
    for (int i = 0; i < iters && s == CR_OK; ++i) {
        s = enqueue_iteration(c, c->k + 1, evs[2 * i], evs[2 * i + 1]);
        if (s == CR_OK) ++c->k;
    }
    float sw = 0.f, tot = 0.f;
    if (s == CR_OK) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            set_err("stream failed: %s", cudaGetErrorString(e));
            s = CR_ECUDA;
        }
    }
    if (s == CR_OK) {
        for (int i = 0; i < iters; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]);
            sw += ms;
        }
        if (iters > 0) {
            // total: from the stream start marker to the end of the last finalize
            cudaEvent_t endev;
            cudaEventCreate(&endev);
            cudaEventRecord(endev, c->stream);
            cudaEventSynchronize(endev);
            cudaEventElapsedTime(&tot, start, endev);
            cudaEventDestroy(endev);
        }
    }
    for (auto &e : evs) cudaEventDestroy(e);
    if (sweep_ms) *sweep_ms = sw;
    if (total_ms) *total_ms = tot;
    return s;
}

CR_API cr_status cr_set_wait_limit(cr_ctx *c, long long consumer_wait_ns) {
    if (!c || consumer_wait_ns < 0) {
        set_err("bad argument to cr_set_wait_limit");
        return CR_EINVAL;
    }
    if (!c->tma) {
        set_err("cr_set_wait_limit applies to the FP32 TMA sweep only");
        return CR_EUNSUPPORTED;
    }
    if (c->gexec) {  // captured graphs hold the old bound
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    c->consumer_wait_ns = (unsigned long long)consumer_wait_ns;
    return CR_OK;
}

CR_API cr_status cr_gap(cr_ctx *c, cr_gap_info *out) {
    if (c && c->shard) {
        set_err("cr_gap works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c) {
        set_err("ctx is NULL");
        return CR_EINVAL;
    }
    CR_TRY(gap_launch(c));
    DevState h{};
    CR_TRY(fetch_state(c, &h));
    return gap_finish(c, h, out);
}

CR_API cr_status cr_solve(cr_ctx *c, double tol, long long max_iter, cr_gap_info *out) {
    if (c && c->shard) {
        set_err("cr_solve works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || !(tol >= 0.0) || max_iter < 0) {
        set_err("bad argument to cr_solve");
        return CR_EINVAL;
    }
    cr_gap_info g{};
    for (;;) {
        CR_TRY(cr_gap(c, &g));
        if (out) *out = g;
        if (c->k > 0 && g.rel_gap <= tol) return CR_OK;
        if (c->k >= max_iter) {
            set_err("rel_gap %.3e > %.3e after %lld iterations", g.rel_gap, tol, c->k);
            return CR_ENOTCONV;
        }
        const long long step = std::min<long long>(c->opt.check_every, max_iter - c->k);
        CR_TRY(cr_dual_step(c, (int)step));
    }
}

CR_API cr_status cr_primal(const cr_ctx *c, double *y, double *xi) {
    if (c && c->shard) {
        set_err("cr_primal works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c) {
        set_err("ctx is NULL");
        return CR_EINVAL;
    }
    long long kk = 0;
    int lb = 0;
    CR_TRY(current_k(c, &kk, &lb));
    CR_CUDA(launch_primal(c->N, c->n, c->ybar, c->ha[kk & 1], c->hb[kk & 1], c->st, c->tmp_y, c->tmp_xi,
                          c->stream));
    if (y) CR_CUDA(cudaMemcpyAsync(y, c->tmp_y, sizeof(double) * c->N, cudaMemcpyDefault, c->stream));
    if (xi)
        CR_CUDA(cudaMemcpyAsync(xi, c->tmp_xi, sizeof(double) * c->N * c->n, cudaMemcpyDefault, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

CR_API cr_status cr_lambda(const cr_ctx *c, long long row0, long long rows, double *out, long long ld) {
    if (c && c->shard) {
        set_err("cr_lambda works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || !out || row0 < 0 || rows < 0 || row0 + rows > c->N || ld < c->N) {
        set_err("bad argument to cr_lambda");
        return CR_EINVAL;
    }
    if (rows == 0) return CR_OK;
    long long kk = 0;
    int lb = 0;
    CR_TRY(current_k(c, &kk, &lb));
    const void *lam = c->lam[lb];  // constant step: lambda^k lives in lam[k & 1] (lam[0] = lambda^0 at k = 0)
    cudaPointerAttributes at{};
    bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
        CR_CUDA(launch_lambda_to_f64(lam, !is_f64(c), c->N, c->ld, row0, rows, out, ld, c->stream));
        CR_CUDA(cudaStreamSynchronize(c->stream));
        return CR_OK;
    }
    // host destination: convert through a bounded device staging buffer
    const long long per = std::max<long long>(1, (64LL << 20) / (8LL * c->N));
    double *stage = nullptr;
    CR_CUDA(cudaMalloc(&stage, sizeof(double) * std::min(per, rows) * c->N));
    cr_status s = CR_OK;
    for (long long r = 0; r < rows && s == CR_OK; r += per) {
        const long long cnt = std::min(per, rows - r);
        cudaError_t e = launch_lambda_to_f64(lam, !is_f64(c), c->N, c->ld, row0 + r, cnt, stage, c->N, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(out + r * ld, sizeof(double) * ld, stage, sizeof(double) * c->N,
                                  sizeof(double) * c->N, cnt, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            set_err("lambda copy failed: %s", cudaGetErrorString(e));
            s = CR_ECUDA;
        }
    }
    cudaFree(stage);
    return s;
}

CR_API cr_status cr_lipschitz(const cr_ctx *c, double *L) {
    if (!c || !L) {
        set_err("bad argument to cr_lipschitz");
        return CR_EINVAL;
    }
    *L = c->L;
    return CR_OK;
}

CR_API long long cr_iterations(const cr_ctx *c) { return c ? c->k : -1; }

namespace crh {

// Rebuilds eta(lambda~^{k+1}) from the C^T history and the device beta (the commit kernel with
// the accepted flag forced and (a,b)^k in place), after gamma or the whole state changed.
cr_status rebuild_recovery(cr_ctx *c, const DevState &h) {
    FinArgs f{};
    f.N = c->N;
    f.n = c->n;
    f.NP = c->NP;
    f.precision = c->opt.precision;
    f.ldv = c->ldv;
    f.X = c->X;
    f.ybar = c->ybar;
    f.a_new = c->ha[h.k & 1];
    f.b_new = c->hb[h.k & 1];
    for (int i = 0; i < 2; ++i) {
        f.hist_a[i] = c->ha[i];
        f.hist_b[i] = c->hb[i];
    }
    f.yh = c->yh;
    f.yl = c->yl;
    f.uh = c->uh;
    f.ul = c->ul;
    f.xiT = c->xiT;
    f.y64 = c->y64;
    f.u64 = c->u64;
    f.xiT64 = c->xiT64;
    f.xT32 = c->xT32;
    f.xi_rm = c->xi_rm;
    f.st = c->st;
    CR_CUDA(launch_commit(f, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

// The vectors of eta(lambda~^{k+1}) the next sweep reads (saved as they are, so that a resume
// is bitwise: rebuilding them would add in another order).
struct VecRef {
    void *p;
    size_t bytes;
};
int derived_vectors(const cr_ctx *c, VecRef *v) {
    const size_t vec = (size_t)c->ldv, tvec = (size_t)c->NP * c->ldv;
    int m = 0;
    if (is_f64(c)) {
        v[m++] = {c->y64, 8 * vec};
        v[m++] = {c->u64, 8 * vec};
        v[m++] = {c->xiT64, 8 * tvec};
    } else {
        v[m++] = {c->yh, 4 * 2 * vec};
        v[m++] = {c->uh, 4 * 2 * vec};
        v[m++] = {c->xiT, 4 * tvec};
        if (c->xi_rm) v[m++] = {c->xi_rm, 4 * 2 * 32 * vec};
    }
    return m;
}

struct CkptHeader {
    char magic[8];
    long long N, ld, k, nbuf, tsz;
    int n, precision, step_rule, pad;
    unsigned long long data_fp;  // FNV-1a of the instance's X and ybar bytes
};
constexpr char kCkptMagic[9] = "CRCKPT02";

// FNV-1a (64-bit) over the bytes of X and ybar as the context holds them: a checkpoint is
// restored only into a context created for the same data.
cr_status data_fingerprint(cr_ctx *c, unsigned long long *fp) {
    const size_t nx = (size_t)c->N * c->n;
    std::vector<double> hx(nx), hy((size_t)c->N);
    CR_CUDA(cudaMemcpyAsync(hx.data(), c->X, sizeof(double) * nx, cudaMemcpyDeviceToHost, c->stream));
    CR_CUDA(cudaMemcpyAsync(hy.data(), c->ybar, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    unsigned long long h = 1469598103934665603ull;
    auto eat = [&h](const std::vector<double> &v) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(v.data());
        for (size_t i = 0, e = v.size() * sizeof(double); i < e; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    };
    eat(hx);
    eat(hy);
    *fp = h;
    return CR_OK;
}

}  // namespace crh

CR_API cr_status cr_set_gamma(cr_ctx *c, double gamma) {
    if (c && c->shard) {
        set_err("cr_set_gamma works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || !(gamma > 0.0) || !isfinite(gamma)) {
        set_err("bad argument to cr_set_gamma");
        return CR_EINVAL;
    }
    if (c->opt.lipschitz > 0.0) {
        set_err("the context was created with a given L, which cannot follow gamma");
        return CR_EINVAL;
    }
    DevState h{};
    CR_TRY(fetch_state(c, &h));
    const int N = c->N;
    c->opt.gamma = gamma;
    c->L = (c->opt.lipschitz_rule == CR_L_PAPER) ? (2.0 * N + c->a2s2) / gamma : 2.0 * N + c->a2s2 / gamma;
    h.gamma = gamma;
    h.inv_gamma = 1.0 / gamma;
    h.t = 1.0;
    h.beta = 0.0;
    h.inv_L = 1.0 / c->L;
    h.s = c->adaptive ? c->opt.upsilon / c->L : 1.0 / c->L;
    h.prev_g = -DBL_MAX;
    h.accepted = 1;
    // g, r and lambda^T C eta of lambda^k at the new gamma (the record held the old gamma's):
    // the finalize's sums of (a, b)^k, in FP64 on the host
    {
        const size_t nb = (size_t)N * c->n;
        std::vector<double> av((size_t)N), bv(nb), yv((size_t)N);
        CR_CUDA(cudaMemcpyAsync(av.data(), c->ha[h.k & 1], sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
        CR_CUDA(cudaMemcpyAsync(bv.data(), c->hb[h.k & 1], sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream));
        CR_CUDA(cudaMemcpyAsync(yv.data(), c->ybar, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
        CR_CUDA(cudaStreamSynchronize(c->stream));
        double aa = 0.0, ay = 0.0, bb = 0.0;
        for (int l = 0; l < N; ++l) {
            aa += av[l] * av[l];
            ay += av[l] * yv[l];
        }
        for (size_t q = 0; q < nb; ++q) bb += bv[q] * bv[q];
        h.last_g = -0.5 * aa - ay - bb / (2.0 * gamma);
        h.last_r = 0.5 * aa + bb / (2.0 * gamma);
        h.last_lg = aa + ay + bb / gamma;
    }
    CR_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    return rebuild_recovery(c, h);
}

CR_API cr_status cr_solve_path(cr_ctx *c, const double *gammas, const double *tols, int stages,
                               long long max_sweeps, cr_gap_info *out) {
    if (!c || !gammas || !tols || stages < 1 || max_sweeps < 0) {
        set_err("bad argument to cr_solve_path");
        return CR_EINVAL;
    }
    for (int t = 0; t < stages; ++t) {
        if (gammas[t] != c->opt.gamma) CR_TRY(cr_set_gamma(c, gammas[t]));
        cr_gap_info g{};
        const cr_status s = cr_solve(c, tols[t], c->k + max_sweeps, &g);
        if (out) *out = g;
        if (s != CR_OK) return s;
    }
    return CR_OK;
}

CR_API cr_status cr_solve_continuation(cr_ctx *c, double eps0, double beta, double kappa_gamma,
                                       double kappa_delta, double infeas_tol, int stages,
                                       long long max_sweeps, cr_gap_info *out) {
    if (!c || !(eps0 > 0.0) || !(beta > 1.0) || !(kappa_gamma > 0.0) || !(kappa_delta > 0.0) || stages < 1 ||
        max_sweeps < 0 || !isfinite(eps0 * kappa_gamma * kappa_delta * beta) || isnan(infeas_tol)) {
        set_err("bad argument to cr_solve_continuation");
        return CR_EINVAL;
    }
    double eps = eps0;
    for (int t = 1; t <= stages; ++t) {
        eps /= beta;  // eps_t = eps0 / beta^t
        const double gamma_t = kappa_gamma * eps, delta_t = kappa_delta * eps;
        if (!(gamma_t > 0.0)) {
            set_err("gamma underflows at stage %d", t);
            return CR_EINVAL;
        }
        CR_TRY(cr_set_gamma(c, gamma_t));
        const long long cap = c->k + max_sweeps;
        cr_gap_info g{};
        for (;;) {
            CR_TRY(cr_gap(c, &g));
            if (out) *out = g;
            // cert_primal >= p*_gamma = max g_gamma, so this gap bounds the dual suboptimality
            const bool certified = g.cert_primal - g.dual_g <= delta_t;
            // Section 5's test: |lambda^T C eta| and the normalised infeasibility
            const bool practical = fabs(g.lagr_gap) <= delta_t && g.infeas_norm <= infeas_tol;
            if (c->k > 0 && (certified || practical)) break;
            if (c->k >= cap) {
                set_err("stage %d: gap %.3e / certified %.3e > delta_t %.3e after %lld sweeps", t,
                        fabs(g.lagr_gap), g.cert_primal - g.dual_g, delta_t, max_sweeps);
                return CR_ENOTCONV;
            }
            CR_TRY(cr_dual_step(c, (int)std::min<long long>(c->opt.check_every, cap - c->k)));
        }
    }
    return CR_OK;
}

CR_API long long cr_checkpoint_bytes(const cr_ctx *c) {
    if (!c) return -1;
    const long long tsz = is_f64(c) ? 8 : 4, nbuf = c->adaptive ? 3 : 2;
    VecRef v[4];
    long long vb = 0;
    for (int i = 0, m = derived_vectors(c, v); i < m; ++i) vb += (long long)v[i].bytes;
    return (long long)sizeof(CkptHeader) + (long long)sizeof(DevState) + nbuf * c->N * c->ld * tsz +
           2 * 8LL * c->N * (c->n + 1) + vb;
}

CR_API cr_status cr_checkpoint(cr_ctx *c, void *buf, long long bytes) {
    if (c && c->shard) {
        set_err("cr_checkpoint works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || !buf || bytes < cr_checkpoint_bytes(c)) {
        set_err("bad argument to cr_checkpoint");
        return CR_EINVAL;
    }
    CkptHeader hd{};
    memcpy(hd.magic, kCkptMagic, 8);
    CR_TRY(data_fingerprint(c, &hd.data_fp));
    hd.N = c->N;
    hd.ld = c->ld;
    hd.k = c->k;
    hd.nbuf = c->adaptive ? 3 : 2;
    hd.tsz = is_f64(c) ? 8 : 4;
    hd.n = c->n;
    hd.precision = c->opt.precision;
    hd.step_rule = c->opt.step_rule;
    char *p = (char *)buf;
    CR_CUDA(cudaStreamSynchronize(c->stream));
    CR_CUDA(cudaMemcpy(p, &hd, sizeof(hd), cudaMemcpyDefault));
    p += sizeof(hd);
    CR_CUDA(cudaMemcpyAsync(p, c->st, sizeof(DevState), cudaMemcpyDefault, c->stream));
    p += sizeof(DevState);
    const size_t lb = (size_t)c->N * c->ld * hd.tsz;
    for (int i = 0; i < hd.nbuf; ++i, p += lb) CR_CUDA(cudaMemcpyAsync(p, c->lam[i], lb, cudaMemcpyDefault, c->stream));
    for (int i = 0; i < 2; ++i) {
        CR_CUDA(cudaMemcpyAsync(p, c->ha[i], 8 * (size_t)c->N, cudaMemcpyDefault, c->stream));
        p += 8 * (size_t)c->N;
        CR_CUDA(cudaMemcpyAsync(p, c->hb[i], 8 * (size_t)c->N * c->n, cudaMemcpyDefault, c->stream));
        p += 8 * (size_t)c->N * c->n;
    }
    VecRef v[4];
    for (int i = 0, m = derived_vectors(c, v); i < m; p += v[i].bytes, ++i)
        CR_CUDA(cudaMemcpyAsync(p, v[i].p, v[i].bytes, cudaMemcpyDefault, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

CR_API cr_status cr_restore(cr_ctx *c, const void *buf, long long bytes) {
    if (c && c->shard) {
        set_err("cr_restore works on whole instances; a shard iterates with cr_shard_sweep / cr_shard_finish");
        return CR_EINVAL;
    }
    if (!c || !buf || bytes < cr_checkpoint_bytes(c)) {
        set_err("bad argument to cr_restore");
        return CR_EINVAL;
    }
    CkptHeader hd{};
    const char *p = (const char *)buf;
    CR_CUDA(cudaMemcpy(&hd, p, sizeof(hd), cudaMemcpyDefault));
    p += sizeof(hd);
    if (memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.N != c->N || hd.n != c->n || hd.ld != c->ld ||
        hd.precision != c->opt.precision || hd.step_rule != c->opt.step_rule ||
        hd.nbuf != (c->adaptive ? 3 : 2) || hd.tsz != (is_f64(c) ? 8 : 4)) {
        set_err("the checkpoint belongs to another instance shape, precision or step rule");
        return CR_EINVAL;
    }
    unsigned long long fp = 0;
    CR_TRY(data_fingerprint(c, &fp));
    if (fp != hd.data_fp) {
        set_err("the checkpoint was taken on other data (X or ybar differ)");
        return CR_EINVAL;
    }
    DevState h{};
    CR_CUDA(cudaMemcpy(&h, p, sizeof(DevState), cudaMemcpyDefault));
    p += sizeof(DevState);
    const size_t lb = (size_t)c->N * c->ld * hd.tsz;
    CR_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < hd.nbuf; ++i, p += lb) CR_CUDA(cudaMemcpyAsync(c->lam[i], p, lb, cudaMemcpyDefault, c->stream));
    for (int i = 0; i < 2; ++i) {
        CR_CUDA(cudaMemcpyAsync(c->ha[i], p, 8 * (size_t)c->N, cudaMemcpyDefault, c->stream));
        p += 8 * (size_t)c->N;
        CR_CUDA(cudaMemcpyAsync(c->hb[i], p, 8 * (size_t)c->N * c->n, cudaMemcpyDefault, c->stream));
        p += 8 * (size_t)c->N * c->n;
    }
    VecRef v[4];
    for (int i = 0, m = derived_vectors(c, v); i < m; p += v[i].bytes, ++i)
        CR_CUDA(cudaMemcpyAsync(v[i].p, p, v[i].bytes, cudaMemcpyDefault, c->stream));
    // the saved context's gamma and L (a restore also carries a continuation stage)
    c->opt.gamma = h.gamma;
    c->L = 1.0 / (c->adaptive ? h.inv_L : h.s);
    c->k = hd.k;
    h.fin_counter = 0u;
    h.cert_counter = 0u;
    CR_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    CR_CUDA(cudaStreamSynchronize(c->stream));
    return CR_OK;
}

CR_API cr_status cr_describe(const cr_ctx *c, char *buf, int len) {
    if (!c || !buf || len <= 0) {
        set_err("bad argument to cr_describe");
        return CR_EINVAL;
    }
    const double tsz = is_f64(c) ? 8.0 : 4.0;
    const double pairs = (double)c->N * (double)(c->N - 1);
    snprintf(buf, (size_t)len,
             "{\"N\": %d, \"n\": %d, \"NP\": %d, \"precision\": %d, \"ld\": %lld, \"rows_per_item\": %d, "
             "\"row_blocks\": %d, \"col_splits\": %d, \"cols_per_split\": %d, \"grid\": %d, "
             "\"ctas_per_sm\": %d, \"sms\": %d, \"pairs\": %.0f, \"lambda_bytes_per_iter\": %.0f, "
             "\"L\": %.17g, \"sigma_a2_sq\": %.17g, \"cert_row_splits\": %d, \"graph_iters\": %d, "
             "\"step_rule\": %d, \"upsilon\": %.17g, \"delta\": %d, \"refresh_every\": %d, \"equal_chunk_ranges\": %d, "
             "\"sweep\": \"%s\"}",
             c->N, c->n, c->NP, c->opt.precision, c->ld, c->rows, c->RB, c->S, c->cps, c->grid, c->occ, c->sms,
             pairs, 3.0 * tsz * pairs, c->L, c->a2s2, c->cert_R, c->opt.graph_iters, c->opt.step_rule,
             c->opt.upsilon, c->delta ? 1 : 0, c->delta ? c->opt.refresh_every : 0, c->seg ? 1 : 0,
             c->tc ? "tcgen05"
                   : (c->tma ? "tma" : (c->NP > 32 ? (is_f64(c) ? "wide-fp64" : "wide-fp32") : (is_f64(c) ? "fp64" : "simple"))));
    return CR_OK;
}

CR_API void cr_destroy(cr_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

CR_API const char *cr_strerror(cr_status s) {
    switch (s) {
        case CR_OK: return "ok";
        case CR_EINVAL: return "invalid argument";
        case CR_ENOMEM: return "out of memory";
        case CR_ECUDA: return "CUDA error";
        case CR_ENOTCONV: return "not converged";
        case CR_ETIMEOUT: return "device wait timed out";
        case CR_ENUMERIC: return "non-finite result";
        case CR_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

CR_API const char *cr_last_error(void) { return g_err; }

CR_API int cr_version(void) { return 100; }

}  // extern "C"
