// cr_host.h -- host-side context shared by the single-instance (cr_api.cu) and batched
// (cr_batch.cu) front ends.  Not part of the ABI.
#pragma once

#include <vector>

#include "cr_internal.cuh"

using namespace cr;

struct cr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int N = 0, n = 0, NP = 0;
    // rows of Lambda this context holds: [row0, row_end) (a shard of cr_shard_create; 0 and N
    // otherwise); the buffers hold them from their row 0
    int row0 = 0, row_end = 0;
    bool shard = false;
    double *xch_b = nullptr;     // shard: ||b||^2 block partials of the local rows
    long long ld = 0, ldv = 0;
    cr_options opt{};
    double L = 0.0, a2s2 = 0.0, ybar_rms = 1.0;
    long long k = 0;  // iterations enqueued
    int sms = 0;

    std::vector<void *> allocs;
    double *X = nullptr, *ybar = nullptr;
    float *xT32 = nullptr;
    double *xT64 = nullptr;
    void *lam[3] = {nullptr, nullptr, nullptr};  // the third only with the adaptive step
    bool adaptive = false;       // CR_STEP_ADAPTIVE
    double *ha_c = nullptr, *hb_c = nullptr;    // adaptive: C^T of the candidate
    void *dpart = nullptr;       // adaptive: row sums of (lambda^k - lambda~^k)^2 per split (and group)
    int dgroups = 0;
    double *ha[2] = {nullptr, nullptr}, *hb[2] = {nullptr, nullptr};
    float *yh = nullptr, *yl = nullptr, *uh = nullptr, *ul = nullptr, *xiT = nullptr;
    double *y64 = nullptr, *u64 = nullptr, *xiT64 = nullptr;
    void *rowpart = nullptr, *colpart = nullptr;
    double *finblk = nullptr, *certblk = nullptr, *log = nullptr;
    DevState *st = nullptr;
    // certificate buffers
    float *c_yh = nullptr, *c_yl = nullptr, *c_uh = nullptr, *c_ul = nullptr, *c_xiT = nullptr;
    double *c_y64 = nullptr, *c_u64 = nullptr, *c_xiT64 = nullptr;
    double *pmax = nullptr, *pinf = nullptr;
    int *parg = nullptr;
    int cert_R = 1;
    // primal scratch
    double *tmp_y = nullptr, *tmp_xi = nullptr;
    int *flag = nullptr;
    // sweep shape
    int rows = 0, RB = 0, S = 0, cps = 0, grid = 0, occ = 0;
    // tensor-core sweep with the automatic split: CTAs take equal ranges of the RB x seg_nchr
    // 32-column chunks (S is then the most pieces a row block can be cut into)
    bool seg = false;
    int seg_nchr = 0;
    long long seg_total = 0;
    bool tma = false;            // FP32: TMA-pipelined sweep (cr_sweep_tma.cu)
    unsigned long long consumer_wait_ns = 0;  // cr_set_wait_limit (0: the default bound)
    // C^T in delta form with a periodic exact refresh (cr_refresh.cu)
    bool delta = false;
    double *rf_r = nullptr, *rf_B = nullptr, *rf_c = nullptr;
    int rf_segs = 0;
    CUtensorMap tm_lam[3];
    CUtensorMap *tm_ld = nullptr;  // adaptive step: device copy of tm_lam (roles chosen on the device)
    TmaMaps tm{};
    bool tc = false;             // CR_MIXED_TF32: tensor-core sweep (cr_sweep_tc.cu)
    CUtensorMap *tc_ld = nullptr;                    // device array: maps of the buffers (box 32 x 128)
    CUtensorMap tc_lam_ld[3];                        // host copies of the same maps (batch descriptors)
    TcMaps tcm{};
    float *xr = nullptr, *xt = nullptr, *xi_rm = nullptr;
    // graph of graph_iters iterations starting at an even k
    cudaGraphExec_t gexec = nullptr;
    int glen = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace crh {

void set_err(const char *fmt, ...);

#define CR_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? CR_ENOMEM : CR_ECUDA;                 \
        }                                                                                  \
    } while (0)

#define CR_TRY(x)                       \
    do {                                \
        cr_status s_ = (x);             \
        if (s_ != CR_OK) return s_;     \
    } while (0)

template <typename T>
cr_status dev_alloc(cr_ctx *c, T **p, size_t count) {
    void *q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        set_err("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? CR_ENOMEM : CR_ECUDA;
    }
    c->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return CR_OK;
}

bool is_f64(const cr_ctx *c);
void choose_split(cr_ctx *c);
cr_status create_impl(cr_ctx *c, const double *X, const double *ybar);
cr_status fetch_state(const cr_ctx *c, DevState *h);
cr_status enqueue_iteration(cr_ctx *c, long long k, cudaEvent_t e0, cudaEvent_t e1);
cr_status enqueue_sweep(cr_ctx *c, long long k, cudaEvent_t e0);
cr_status create_window(const double *X, const double *ybar, long long N, int n, int row0, int row_end, bool shard,
                        const cr_options *opt, void *stream, cr_ctx **out);
cr_status gap_launch(cr_ctx *c);
cr_status gap_launch_k(cr_ctx *c, long long k);
cr_status gap_finish(const cr_ctx *c, DevState h, cr_gap_info *out);

}  // namespace crh
