// cr_batch.cu -- batched solving of many independent instances (the K = N method of
// Figure "papg" applied to each instance), with one persistent sweep launch per
// point-dimension bucket per iteration and one finalize launch for all instances.
//
// Each instance is an ordinary context (cr_ctx: its own multipliers, vectors, step
// constant and device scalars t_k, beta_k, k).  The batch keeps, in device memory, one
// InstDesc per active instance (its tensor maps and pointers) and three work-lists:
// sweep items (instance, 32-row block, column split) grouped by bucket, and finalize items
// (instance, 32-point block).  Iterations are captured as a CUDA graph of graph_iters
// iterations: the bucket launches fork onto parallel streams and join before the finalize.
// Instances are checked (one pass over all their pairs each) between graph blocks and
// retired at their own tolerance; the work-lists are then rebuilt.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "cr_host.h"

using namespace crh;

namespace {

constexpr int kMaxBuckets = 13;  // twelve FP32 widths and the tensor-core sweep
constexpr int kMinSplit = 512;  // smallest column-split width (sizes the row partials)
constexpr int kDefaultSplit = 4096;

struct BatchInst {
    cr_ctx *c = nullptr;
    double tol = 0.0;
    long long max_iter = 0;
    bool done = false;
    bool removed = false;
    int status = CR_OK;
    cr_gap_info info{};
};

// np > 0: the FP32 TMA sweep of that padded width; np == kTcBucket: the tensor-core sweep
struct Bucket {
    int np, off, count, grid;
};
constexpr int kTcBucket = 0;

}  // namespace

struct cr_batch {
    cr_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    std::vector<BatchInst> inst;
    // device schedule
    InstDesc *d_desc = nullptr;
    int desc_cap = 0;
    WorkItem *d_items = nullptr;
    int items_cap = 0;
    FinItem *d_fin = nullptr;
    int fin_cap = 0;
    int *d_err = nullptr;
    int *d_due = nullptr;     // instances whose exact C^T refresh is due ([0] = count)
    int due_cap = 0;
    std::vector<int> active;  // instance ids in descriptor order
    std::vector<Bucket> buckets;
    int nfin = 0;
    bool any_delta = false;   // some active instance reduces in delta form
    bool dirty = true;
    int cps = kMinSplit;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t aux[kMaxBuckets] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxBuckets] = {};
};

namespace {

template <typename T>
cr_status grow(T **p, int *cap, int need) {
    if (need <= *cap) return CR_OK;
    int nc = std::max(need, 2 * *cap);
    if (nc < 16) nc = 16;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)nc);
    if (e != cudaSuccess) {
        set_err("batch schedule allocation failed: %s", cudaGetErrorString(e));
        return CR_ENOMEM;
    }
    *cap = nc;
    return CR_OK;
}

void drop_graph(cr_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

void fill_desc(const cr_batch *b, const cr_ctx *c, InstDesc *d, int id) {
    memset(d, 0, sizeof(*d));
    for (int i = 0; i < 3; ++i) d->tm_lam[i] = c->tm_lam[i];
    d->lam[2] = (float *)c->lam[2];
    d->adaptive = c->adaptive ? 1 : 0;
    d->dpart = (float *)c->dpart;
    d->ha_c = c->ha_c;
    d->hb_c = c->hb_c;
    d->tm_x = c->tm.X;
    d->tm_y = c->tm.Y;
    d->tm_xi = c->tm.Xi;
    d->tm_u = c->tm.U;
    d->lam[0] = (float *)c->lam[0];
    d->lam[1] = (float *)c->lam[1];
    d->ld = c->ld;
    d->ldv = c->ldv;
    d->N = c->N;
    d->n = c->n;
    d->NP = c->NP;
    d->cols_per_split = c->cps;
    d->row_blocks = c->RB;
    d->col_splits = c->S;
    d->fin_blocks = finalize_blocks(c->N);
    d->inst_id = id;
    d->st = c->st;
    d->rowpart = (float *)c->rowpart;
    d->colpart = (float *)c->colpart;
    d->X = c->X;
    d->ybar = c->ybar;
    d->ha[0] = c->ha[0];
    d->ha[1] = c->ha[1];
    d->hb[0] = c->hb[0];
    d->hb[1] = c->hb[1];
    d->yh = c->yh;
    d->yl = c->yl;
    d->uh = c->uh;
    d->ul = c->ul;
    d->xiT = c->xiT;
    d->xT32 = c->xT32;
    d->finblk = c->finblk;
    d->log = c->log;
    d->tc = c->tc ? 1 : 0;
    d->delta = c->delta ? 1 : 0;
    d->rf_period = c->delta ? c->opt.refresh_every : 0;
    d->rf_segs = c->rf_segs;
    d->rf_r = c->rf_r;
    d->rf_B = c->rf_B;
    d->rf_c = c->rf_c;
    d->dgroups = c->S * (c->tc ? 2 : 1);  // the tensor-core sweep keeps two groups per split
    if (c->tc) {
        for (int i = 0; i < 3; ++i) d->tc_lam_ld[i] = c->tc_lam_ld[i];
        d->tc_xrh = c->tcm.XRh;
        d->tc_xrl = c->tcm.XRl;
        d->tc_xt = c->tcm.XT;
        d->tc_y = c->tcm.Y;
        d->xi_rm = c->xi_rm;
    }
    (void)b;
}

// Rebuilds descriptors and work-lists for the active instances (host -> device, synchronous).
cr_status rebuild(cr_batch *b) {
    drop_graph(b);
    b->active.clear();
    b->any_delta = false;
    for (int id = 0; id < (int)b->inst.size(); ++id)
        if (!b->inst[id].done && !b->inst[id].removed) {
            b->active.push_back(id);
            b->any_delta = b->any_delta || b->inst[id].c->delta;
        }
    const int na = (int)b->active.size();
    std::vector<InstDesc> desc(na);
    std::vector<std::vector<WorkItem>> per(kMaxBuckets);
    std::vector<double> work(kMaxBuckets, 0.0);
    std::vector<FinItem> fin;
    static const int npv[kMaxBuckets] = {kTcBucket, 2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
    for (int di = 0; di < na; ++di) {
        cr_ctx *c = b->inst[b->active[di]].c;
        c->cps = std::max(kMinSplit, (int)std::min<long long>(b->cps, round_up(c->ld, kChunk)));
        c->S = (int)((c->ld + c->cps - 1) / c->cps);
        fill_desc(b, c, &desc[di], b->active[di]);
        int bi = 0;
        if (!c->tc)
            while (npv[bi] != c->NP) ++bi;
        for (int rb = 0; rb < c->RB; ++rb)
            for (int sp = 0; sp < c->S; ++sp) per[bi].push_back(WorkItem{di, rb, sp});
        // sweep cost of a pair grows with the padded width in the FP32 TMA kernel (GB300: about
        // (6 + NP) x 0.16 ps per pair from n = 8 to 32), and is about 2.2 ps (~14 of those units)
        // for any n in the tensor-core kernel, so the concurrent buckets share the SMs by
        // pairs x cost, not by pairs alone
        work[bi] += (double)c->N * (double)c->ld * (c->tc ? 14.0 : 6.0 + (double)c->NP);
        for (int blk = 0; blk < desc[di].fin_blocks; ++blk) fin.push_back(FinItem{di, blk});
    }
    // largest items first, so that the strided assignment of items to CTAs stays balanced
    std::vector<WorkItem> items;
    b->buckets.clear();
    double total = 0.0;
    for (double w : work) total += w;
    for (int bi = 0; bi < kMaxBuckets; ++bi) {
        if (per[bi].empty()) continue;
        auto &v = per[bi];
        std::stable_sort(v.begin(), v.end(), [&](const WorkItem &x, const WorkItem &y) {
            const InstDesc &dx = desc[x.inst], &dy = desc[y.inst];
            const long long wx = std::min<long long>(dx.cols_per_split, dx.ld - (long long)x.sp * dx.cols_per_split);
            const long long wy = std::min<long long>(dy.cols_per_split, dy.ld - (long long)y.sp * dy.cols_per_split);
            return wx > wy;
        });
        Bucket bk;
        bk.np = npv[bi];
        bk.off = (int)items.size();
        bk.count = (int)v.size();
        int occ = 1;
        if (bk.np == kTcBucket)
            sweep_tc_occupancy(&occ);
        else
            sweep_tma_occupancy(bk.np, &occ);
        const double share = total > 0 ? work[bi] / total : 1.0;
        bk.grid = (int)std::max(1.0, std::round(share * b->sms * std::max(1, occ)));
        bk.grid = std::min(bk.grid, bk.count);
        b->buckets.push_back(bk);
        items.insert(items.end(), v.begin(), v.end());
    }
    b->nfin = (int)fin.size();
    CR_TRY(grow(&b->d_desc, &b->desc_cap, std::max(1, na)));
    CR_TRY(grow(&b->d_due, &b->due_cap, na + 1));
    CR_TRY(grow(&b->d_items, &b->items_cap, std::max(1, (int)items.size())));
    CR_TRY(grow(&b->d_fin, &b->fin_cap, std::max(1, b->nfin)));
    if (na) CR_CUDA(cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(InstDesc) * na, cudaMemcpyHostToDevice, b->stream));
    if (!items.empty())
        CR_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice,
                                b->stream));
    if (b->nfin)
        CR_CUDA(cudaMemcpyAsync(b->d_fin, fin.data(), sizeof(FinItem) * fin.size(), cudaMemcpyHostToDevice, b->stream));
    CR_CUDA(cudaStreamSynchronize(b->stream));
    b->dirty = false;
    return CR_OK;
}

cr_status enqueue_batch_iteration(cr_batch *b) {
    if (b->active.empty()) return CR_OK;
    CR_CUDA(cudaMemsetAsync(b->d_due, 0, sizeof(int), b->stream));
    CR_CUDA(cudaEventRecord(b->ev_fork, b->stream));
    for (size_t i = 0; i < b->buckets.size(); ++i) {
        const Bucket &bk = b->buckets[i];
        CR_CUDA(cudaStreamWaitEvent(b->aux[i], b->ev_fork, 0));
        if (bk.np == kTcBucket)
            CR_CUDA(launch_sweep_tc_batch(b->d_desc, b->d_items + bk.off, bk.count, b->d_err, bk.grid, b->aux[i]));
        else
            CR_CUDA(launch_sweep_tma_batch(bk.np, b->d_desc, b->d_items + bk.off, bk.count, b->d_err, bk.grid,
                                           b->opt.step_rule == CR_STEP_ADAPTIVE, b->aux[i]));
        CR_CUDA(cudaEventRecord(b->ev_join[i], b->aux[i]));
        CR_CUDA(cudaStreamWaitEvent(b->stream, b->ev_join[i], 0));
    }
    CR_CUDA(launch_finalize_batch(b->d_desc, b->d_fin, b->nfin, b->d_due, b->stream));
    if (b->opt.step_rule == CR_STEP_ADAPTIVE) CR_CUDA(launch_commit_batch(b->d_desc, b->d_fin, b->nfin, b->stream));
    if (b->any_delta) CR_CUDA(launch_refresh_batch(b->d_desc, b->d_due, (int)b->active.size(), b->sms, b->stream));
    return CR_OK;
}

cr_status build_batch_graph(cr_batch *b) {
    if (b->gexec) return CR_OK;
    cudaGraph_t g = nullptr;
    CR_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cr_status s = CR_OK;
    for (int i = 0; i < b->opt.graph_iters && s == CR_OK; ++i) s = enqueue_batch_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (s != CR_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        set_err("batch graph capture failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        set_err("batch graph instantiation failed: %s", cudaGetErrorString(e));
        return CR_ECUDA;
    }
    return CR_OK;
}

cr_status run_iterations(cr_batch *b, int iters) {
    if (b->dirty) CR_TRY(rebuild(b));
    if (b->active.empty() || iters <= 0) return CR_OK;
    int left = iters;
    const int G = b->opt.graph_iters;
    if (G > 0 && left >= G) {
        CR_TRY(build_batch_graph(b));
        while (left >= G) {
            CR_CUDA(cudaGraphLaunch(b->gexec, b->stream));
            left -= G;
        }
    }
    for (; left > 0; --left) CR_TRY(enqueue_batch_iteration(b));
    for (int id : b->active) b->inst[id].c->k += iters;
    return CR_OK;
}

// One pass over all pairs for every active instance, then retirement decisions.
cr_status check(cr_batch *b) {
    const int na = (int)b->active.size();
    if (!na) return CR_OK;
    std::vector<DevState> hs(na);
    if (b->opt.step_rule == CR_STEP_ADAPTIVE) {  // accepted counts live on the device: one round trip
        for (int di = 0; di < na; ++di)
            CR_CUDA(cudaMemcpyAsync(&hs[di], b->inst[b->active[di]].c->st, sizeof(DevState), cudaMemcpyDeviceToHost,
                                    b->stream));
        CR_CUDA(cudaStreamSynchronize(b->stream));
    }
    for (int di = 0; di < na; ++di) {
        cr_ctx *c = b->inst[b->active[di]].c;
        CR_TRY(gap_launch_k(c, b->opt.step_rule == CR_STEP_ADAPTIVE ? hs[di].k : c->k));
        CR_CUDA(cudaMemcpyAsync(&hs[di], c->st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    }
    int err = 0;
    CR_CUDA(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CR_CUDA(cudaStreamSynchronize(b->stream));
    if (err) {
        set_err("a device-side wait of the batched sweep ran out");
        return CR_ETIMEOUT;
    }
    for (int di = 0; di < na; ++di) {
        BatchInst &bi = b->inst[b->active[di]];
        const cr_status st = gap_finish(bi.c, hs[di], &bi.info);
        if (st != CR_OK) {
            bi.done = true;
            bi.status = st;
            b->dirty = true;
            continue;
        }
        if (bi.info.k > 0 && bi.info.rel_gap <= bi.tol) {
            bi.done = true;
            bi.status = CR_OK;
            b->dirty = true;
        } else if (bi.c->k >= bi.max_iter) {
            bi.done = true;
            bi.status = CR_ENOTCONV;
            b->dirty = true;
        }
    }
    return CR_OK;
}

cr_batch *checked(cr_batch *b) {
    if (!b) set_err("batch is NULL");
    return b;
}

bool valid_id(cr_batch *b, int id) {
    if (id < 0 || id >= (int)b->inst.size() || b->inst[id].removed) {
        set_err("invalid instance id %d", id);
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

CR_API cr_status cr_batch_create(const cr_options *opt, void *stream, cr_batch **out) {
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
    if (o.precision != CR_FP32 && o.precision != CR_MIXED_TF32) {
        set_err("batches run the FP32 or the mixed-precision sweep (precision CR_FP32 or CR_MIXED_TF32)");
        return CR_EINVAL;
    }
    if (o.graph_iters < 0 || (o.graph_iters & 1)) {
        set_err("graph_iters must be even and >= 0");
        return CR_EINVAL;
    }
    if (o.check_every < 1) o.check_every = 1;
    cr_batch *b = new (std::nothrow) cr_batch();
    if (!b) {
        set_err("host allocation failed");
        return CR_ENOMEM;
    }
    b->opt = o;
    // column-split width: the caller's tile_cols, else 4096 (what the autotuner picks for the
    // 256-instance workload; 512-wide splits cost ~8x the items on large instances)
    b->cps = o.tile_cols > 0 ? (int)round_up(std::max(o.tile_cols, kMinSplit), kChunk) : kDefaultSplit;
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = true;
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < kMaxBuckets && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        set_err("batch set-up failed: %s", cudaGetErrorString(e));
        cr_batch_destroy(b);
        return CR_ECUDA;
    }
    *out = b;
    return CR_OK;
}

CR_API cr_status cr_batch_add(cr_batch *b, const double *X, const double *ybar, long long N, int n,
                              double rel_gap_tol, long long max_iter, int *id) {
    if (!checked(b)) return CR_EINVAL;
    if (!id || !(rel_gap_tol >= 0.0) || max_iter < 0) {
        set_err("bad argument to cr_batch_add");
        return CR_EINVAL;
    }
    if (n > CR_MAX_N_BATCH) {
        set_err("batched instances have n <= %d (n = %d)", CR_MAX_N_BATCH, n);
        return CR_EINVAL;
    }
    cr_options o = b->opt;
    o.tile_cols = kMinSplit;  // row partials sized for the narrowest split the batch may use
    o.graph_iters = 0;
    // the tensor-core sweep carries a row of ones in its 32-wide operand (n <= 31): a
    // mixed-precision batch runs an n = 32 instance on the FP32 sweep
    if (o.precision == CR_MIXED_TF32 && n > CR_MAX_N_TF32) o.precision = CR_FP32;
    cr_ctx *c = nullptr;
    CR_TRY(cr_create(X, ybar, N, n, &o, b->stream, &c));
    if (!c->tma && !c->tc) {
        cr_destroy(c);
        set_err("batches need the TMA or the tensor-core sweep");
        return CR_EUNSUPPORTED;
    }
    BatchInst bi;
    bi.c = c;
    bi.tol = rel_gap_tol;
    bi.max_iter = max_iter;
    b->inst.push_back(bi);
    *id = (int)b->inst.size() - 1;
    b->dirty = true;
    return CR_OK;
}

CR_API cr_status cr_batch_step(cr_batch *b, int iters, int *active) {
    if (!checked(b) || iters < 0) {
        set_err("bad argument to cr_batch_step");
        return CR_EINVAL;
    }
    CR_TRY(run_iterations(b, iters));
    CR_TRY(check(b));
    if (active) {
        int a = 0;
        for (const auto &bi : b->inst)
            if (!bi.done && !bi.removed) ++a;
        *active = a;
    }
    return CR_OK;
}

CR_API cr_status cr_batch_run(cr_batch *b) {
    if (!checked(b)) return CR_EINVAL;
    for (;;) {
        int a = 0;
        CR_TRY(cr_batch_step(b, b->opt.check_every, &a));
        if (a == 0) return CR_OK;
    }
}

CR_API cr_status cr_batch_poll(cr_batch *b, int id, int *done, int *status, cr_gap_info *info) {
    if (!checked(b) || !valid_id(b, id)) return CR_EINVAL;
    const BatchInst &bi = b->inst[id];
    if (done) *done = bi.done ? 1 : 0;
    if (status) *status = bi.status;
    if (info) *info = bi.info;
    return CR_OK;
}

CR_API cr_status cr_batch_primal(cr_batch *b, int id, double *y, double *xi) {
    if (!checked(b) || !valid_id(b, id)) return CR_EINVAL;
    return cr_primal(b->inst[id].c, y, xi);
}

CR_API cr_status cr_batch_remove(cr_batch *b, int id) {
    if (!checked(b) || !valid_id(b, id)) return CR_EINVAL;
    CR_CUDA(cudaStreamSynchronize(b->stream));
    cr_destroy(b->inst[id].c);
    b->inst[id].c = nullptr;
    b->inst[id].removed = true;
    b->dirty = true;
    return CR_OK;
}

CR_API long long cr_batch_instance_bytes(long long N, int n) {
    if (N < 2 || n < 1 || n > CR_MAX_N_BATCH) return -1;
    const long long ld = round_up(N, 32), ldv = round_up(N, kChunk);
    const long long NP = bucket_np(n);
    const long long RB = (N + 31) / 32, S = (ld + kMinSplit - 1) / kMinSplit;
    const long long gN = (N + 255) / 256, R = 64;
    long long b = 2 * N * ld * 4;                 // two multiplier buffers
    b += RB * ld * 4 + S * N * (NP + 1) * 4;      // column and row partials
    b += 3 * NP * ldv * 4 + 8 * ldv * 4;          // points, xi (sweep, certificate), y/u splits
    b += 8 * N * n + 8 * N + 4 * 8 * N * (n + 1); // X, ybar, C^T history
    b += 8 * (N + N * n) + 16 * R * N + 8 * gN * 5 + 8 * 3 * 4096 + 4096;
    if (n <= CR_MAX_N_TF32) b += 3 * 2 * ldv * 32 * 4 + 6 * 128 + 4096;  // tensor-core operands and maps
    // exact C^T refresh scratch: r, B and at most 4 x 152 x 256 / N + 1 column segments (up to 152 SMs)
    b += 8 * N + 8 * N * n + 8 * (4LL * 152 * 256 + N);
    return b;
}

CR_API cr_status cr_batch_autotune(cr_batch *b, int iters, int *tile_cols) {
    if (!checked(b) || iters < 1) {
        set_err("bad argument to cr_batch_autotune");
        return CR_EINVAL;
    }
    static const int cand[] = {512, 1024, 2048, 4096, 1 << 30};
    int best = b->cps;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    CR_CUDA(cudaEventCreate(&e0));
    CR_CUDA(cudaEventCreate(&e1));
    cr_status s = CR_OK;
    for (int w : cand) {
        b->cps = w;
        b->dirty = true;
        s = rebuild(b);
        if (s != CR_OK || b->active.empty()) break;
        cudaEventRecord(e0, b->stream);
        for (int i = 0; i < iters && s == CR_OK; ++i) s = enqueue_batch_iteration(b);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            set_err("autotune timing failed");
            s = CR_ECUDA;
        }
        if (s != CR_OK) break;
        for (int id : b->active) b->inst[id].c->k += iters;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cps = best;
    b->dirty = true;
    if (tile_cols) *tile_cols = best;
    return s;
}

CR_API void cr_batch_destroy(cr_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto &bi : b->inst)
        if (bi.c) cr_destroy(bi.c);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_fin) cudaFree(b->d_fin);
    if (b->d_err) cudaFree(b->d_err);
    if (b->d_due) cudaFree(b->d_due);
    for (int i = 0; i < kMaxBuckets; ++i) {
        if (b->aux[i]) cudaStreamDestroy(b->aux[i]);
        if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
