// cr_internal.cuh -- shared declarations of the CUDA library (not part of the ABI).
//
// Data layout in HBM for one instance (N points in R^n, NP = n rounded up to a
// kernel bucket, ld = N rounded up to 32, ldv = N rounded up to 128):
//   lam[0], lam[1]   N x ld   multipliers (T = float or double), ping-pong:
//                              iteration k reads lam[(k-1)&1] = lambda^{k-1} and
//                              lam[k&1] = lambda^{k-2}, and writes lambda^k over
//                              lam[k&1].  Columns >= N and the diagonal stay 0.
//   xT               NP x ldv  points, transposed (component-major), zero padded
//   row side         uh, ul (ldv), xiT (NP x ldv): u_i = y_i - xi_i . x_i and xi_i
//                              of eta(lambda~^k); FP32 mode splits u = uh + ul
//   column side      yh, yl (ldv): y_j of eta(lambda~^k), split hi + lo
//   hist_a[2], hist_b[2]       C^T lambda^{k-1}, C^T lambda^{k-2} (FP64, N and N x n)
//   rowpart          S x N x (NP+1)   per column split: sum_j lambda_ij x_j, sum_j lambda_ij
//   colpart          RB x ld          per row block: sum_i lambda_ij
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cr.h"

namespace cr {

constexpr int kChunk = 128;  // columns of Lambda per chunk (32 lanes x 4 columns)
constexpr int kLogCap = 4096;

// Device-resident scalars of one context.
struct DevState {
    double t;           // t_k for the iteration about to run (t_1 = 1)
    double beta;        // beta_k of the sweep about to run
    double s;           // step 1/L
    double gamma;
    long long k;        // completed iterations
    unsigned int fin_counter;   // last-block counter of the finalize kernel
    unsigned int cert_counter;  // last-block counter of the certificate kernel
    double last_g, last_r, last_lg;      // scalars of lambda^k
    double cert_P, cert_infeas_sq;       // last certificate
    int accelerate;
    int err;            // CR_ETIMEOUT when a bounded device-side wait ran out
    double inv_gamma;   // 1 / gamma (the finalize multiplies; GB300's FP64 divide is costly)
    // adaptive step size (Section 4, Eq. (adaptive-check)); s above is 1/s_k of the next candidate
    int adaptive;       // 1: three multiplier buffers, accept/reject decided on the device
    int ring;           // lambda^{k-1} is buffer ring, lambda^{k-2} ring+1, the candidate ring+2 (mod 3)
    int accepted;       // the last candidate passed the check
    double upsilon;     // step factor
    double inv_L;       // 1/L: the step never drops below it, and a candidate at 1/L is always kept
    int restart;        // momentum reset when the dual objective decreases
    long long restarts; // resets so far
    double prev_g;      // g_gamma of the last accepted iterate
    long long sweeps;   // candidate steps taken
    double check_lhs, check_rhs;  // last check: (||da||^2 + ||db||^2/gamma)/s_k <= ||lambda^k - lambda~^k||^2
    long long refreshed_k;  // iteration of the last exact re-evaluation of C^T lambda (cr_refresh.cu)
    long long refreshes;    // exact re-evaluations so far
};

// Roles of the multiplier buffers in the sweep about to run: inputs lambda^{k-1} (p),
// lambda^{k-2} (q), output (r).  Constant step: two buffers, the caller's parity p_host and
// r = q.  Adaptive step: three buffers rotated on the device (accept: ring += 2 mod 3).
__device__ __forceinline__ void lam_roles(const DevState *st, int adaptive, int p_host, int *p, int *q, int *r) {
    if (adaptive) {
        const int rr = st->ring;
        *p = rr;
        *q = rr == 2 ? 0 : rr + 1;
        *r = rr == 0 ? 2 : rr - 1;
    } else {
        *p = p_host;
        *q = p_host ^ 1;
        *r = *q;
    }
}

inline int bucket_np(int n) {
    static const int b[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
    for (int v : b)
        if (n <= v) return v;
    if (n <= CR_MAX_N) return (n + 15) / 16 * 16;  // wide points: the sweep of cr_sweep_wide.cu
    return -1;
}

inline long long round_up(long long a, long long m) { return (a + m - 1) / m * m; }

// ---------------------------------------------------------------- sweep (S2)
struct SweepArgsF {
    const float *P;          // lambda^{k-1}
    float *Q;                // lambda^{k-2} in, lambda^k out
    float *B[3];             // adaptive step (wide points only): the three multiplier buffers
    int adaptive;
    float *dpart;            // adaptive step: S x N row sums of (lambda^k - lambda~^k)^2
    long long ld;            // leading dimension of P, Q
    int N;
    int row_blocks;          // RB = ceil(N / ROWS)
    int col_splits;          // S
    int cols_per_split;      // multiple of kChunk
    long long ldv;           // leading dimension of the transposed vectors
    const float *xT;         // NP x ldv
    const float *yh, *yl;    // column side
    const float *uh, *ul;    // row side
    const float *xiT;        // NP x ldv
    const DevState *st;
    float *rowpart;          // S x N x (NP+1)
    float *colpart;          // RB x ld
};

struct SweepArgsD {
    const double *P;
    double *Q;
    int row0, row_end;       // rows [row0, row_end) of Lambda (a shard: the buffers hold these rows
                             // from their row 0); row0 = 0, row_end = N for a whole instance
                             // (read by the FP64 kernel of cr_sweep.cu)
    double *B[3];            // adaptive step: the three multiplier buffers (roles from DevState)
    int adaptive;
    double *dpart;           // adaptive step: S x N row sums of (lambda^k - lambda~^k)^2
    long long ld;
    int N;
    int row_blocks;
    int col_splits;
    int cols_per_split;
    long long ldv;
    const double *xT;
    const double *y;
    const double *u;
    const double *xiT;
    const DevState *st;
    double *rowpart;
    double *colpart;
};

struct SweepConfig {
    int rows;      // rows of Lambda per work item (CTA tile height)
    int threads;   // threads per CTA
    size_t smem;   // dynamic shared memory bytes
};

// Returns false if NP has no instantiation.
bool sweep_config_f(int np, SweepConfig *cfg);
bool sweep_config_d(int np, SweepConfig *cfg);
cudaError_t launch_sweep_f(int np, const SweepArgsF &a, int grid, cudaStream_t s);
cudaError_t launch_sweep_d(int np, const SweepArgsD &a, int grid, cudaStream_t s);
cudaError_t sweep_occupancy_f(int np, int *blocks_per_sm);
cudaError_t sweep_occupancy_d(int np, int *blocks_per_sm);

// Wide points, 32 < NP <= CR_MAX_N, NP a multiple of 16 (cr_sweep_wide.cu); the plain
// FP32/FP64 entry points above route such NP here.  Both support the adaptive step.
bool sweep_wide_config(int np, bool f64, SweepConfig *cfg);
cudaError_t launch_sweep_wide_f(int np, const SweepArgsF &a, int grid, cudaStream_t s);
cudaError_t launch_sweep_wide_d(int np, const SweepArgsD &a, int grid, cudaStream_t s);
cudaError_t sweep_wide_occupancy(int np, bool f64, bool adaptive, int *blocks_per_sm);

// FP32 sweep with the TMA / mbarrier pipeline (cr_sweep_tma.cu)
struct TmaSweepArgs {
    float *Q;                // lambda^k is written here (the buffer that held lambda^{k-2})
    int adaptive;            // adaptive step: roles of the three buffers from the device state
    const CUtensorMap *lmaps;  // adaptive step: device array of the buffers' load maps
    float *B[3];             // adaptive step: the three buffers
    float *dpart;            // adaptive step: [S][N] row sums of (lambda^k - lambda~^k)^2
    long long ld;
    int N;
    int row_blocks, col_splits, cols_per_split;
    const DevState *st;
    float *rowpart;          // S x N x (NP+1)
    float *colpart;          // RB x ld
    int *err;
    unsigned long long consumer_wait_ns;  // bound of the consumers' data waits (0: the default 2 s)
    int delta;               // 1: the reductions are of lambda^k - lambda^{k-1} (C^T increments)
    int row0, row_end;       // rows [row0, row_end) of Lambda (a shard; 0 and N for a whole instance)
};
struct TmaMaps {
    const CUtensorMap *P, *Q;            // lambda^{k-1}, lambda^{k-2}: [N][ld], box 128 x R
    CUtensorMap X, Y, Xi, U;             // xT [NP][ldv] box 128 x NP; y hi/lo [2][ldv] box 128 x 2;
                                         // xiT [NP][ldv] box R x NP; u hi/lo [2][ldv] box R x 2
                                         // (R = sweep_tma_rows(NP))
};
cudaError_t launch_sweep_tma(int np, const TmaMaps &m, const TmaSweepArgs &a, int grid, cudaStream_t s);
cudaError_t sweep_tma_occupancy(int np, int *blocks_per_sm);
int sweep_tma_rows(int np);
void sweep_tma_diag(int *v4);  // regs, max threads, smem, threads of a kernel that did not fit   // rows per work item of the TMA sweep for bucket np
cudaError_t make_tmap_2d(CUtensorMap *tm, const float *base, long long cols, long long rows, long long ld,
                         int box_cols, int box_rows, bool swizzle128 = false);

// Tensor-core sweep (cr_sweep_tc.cu, CR_MIXED_TF32): 128-row items, 32-column chunks
struct TcSweepArgs {
    long long ld, ldv;
    int N, n, NP;
    int row_blocks, col_splits, cols_per_split;
    const DevState *st;
    const float *xi_rm;      // xi rows [2][ldv][32] (hi, TF32 low part)
    const float *u;          // u [2][ldv] (hi, lo)
    float *rowpart;          // S x N x (NP+1)
    float *colpart;          // RB x ld (128-row blocks)
    int *err;
    const CUtensorMap *lmaps;  // device array: maps of the multiplier buffers (box 32 x 128; loads and stores)
    int p_host;              // constant step: buffer holding lambda^{k-1}
    int adaptive;
    int delta;               // 1: the reductions are of lambda^k - lambda^{k-1}
    float *dpart;            // adaptive step: [S][2][N] row sums of (lambda^k - lambda~^k)^2 per epilogue group
    int row0, row_end;       // rows [row0, row_end) of Lambda (a shard; 0 and N for a whole instance)
    int seg;                 // 1: each CTA takes an equal range of 32-column chunks in row-block order
    int seg_nchr;            // 32-column chunks of a row block (seg = 1)
    long long seg_total;     // row_blocks x seg_nchr (seg = 1)
};
struct TcMaps {
    CUtensorMap XRh, XRl;                // points row-major [ldv][32] hi / lo, box 32 x 128, swizzle
    CUtensorMap XT;                      // points transposed, hi rows (with the ones row) then lo rows [64][ldv], box 32 x 64, swizzle
    CUtensorMap Y;                       // y hi / lo [2][ldv], box 32 x 2
};
cudaError_t launch_sweep_tc(const TcMaps &m, const TcSweepArgs &a, int grid, cudaStream_t s);
cudaError_t sweep_tc_occupancy(int *blocks_per_sm);
int sweep_tc_rows();
// points for the tensor-core sweep: xr [2][ldv][32] (hi = x as FP32, lo = x - trunc(x)),
// xt [2][32][ldv] (transposed, with a row of ones at index n in the hi half)
cudaError_t launch_tc_points(const double *X, int N, int n, long long ldv, float *xr, float *xt, cudaStream_t s);

// Batched sweep: one descriptor per instance (device memory, tensor maps included) and a
// work-list of items; the P/Q parity of an instance is its device counter k modulo 2.
struct WorkItem {
    int inst, rb, sp;
};
struct InstDesc {
    CUtensorMap tm_lam[3];               // lam[0..2]: [N][ld], box 128 x R (the third with the adaptive step)
    CUtensorMap tm_x, tm_y, tm_xi, tm_u; // as in TmaMaps
    // tensor-core instances (tc = 1): maps of the multiplier buffers (box 32 x 128, loads and the
    // store) and the point / y maps of TcMaps
    CUtensorMap tc_lam_ld[3];
    CUtensorMap tc_xrh, tc_xrl, tc_xt, tc_y;
    int tc;
    int delta;                           // reductions of lambda^k - lambda^{k-1} (see cr_refresh.cu)
    int rf_period, rf_segs;              // delta form: exact refresh every rf_period iterations
    double *rf_r, *rf_B, *rf_c;          // its scratch (N, N x n, rf_segs x N)
    int dgroups;                         // adaptive step: groups of the row sums in dpart
    float *xi_rm;                        // tensor-core instances: xi rows [2][ldv][32]
    float *lam[3];
    int adaptive;
    float *dpart;                        // adaptive step: [S][N] row sums of (lambda^k - lambda~^k)^2
    double *ha_c, *hb_c;                 // adaptive step: C^T of the candidate
    long long ld, ldv;
    int N, n, NP, cols_per_split;
    int row_blocks, col_splits, fin_blocks, inst_id;
    DevState *st;
    float *rowpart, *colpart;
    const double *X, *ybar;
    double *ha[2], *hb[2];
    float *yh, *yl, *uh, *ul, *xiT;
    const float *xT32;
    double *finblk, *log;
};
cudaError_t launch_sweep_tma_batch(int np, const InstDesc *d, const WorkItem *w, int nitems, int *err, int grid,
                                   bool adaptive, cudaStream_t s);
// the tensor-core sweep over a work-list of (instance, 128-row block, column split) items of
// tensor-core instances (any n <= CR_MAX_N_TF32 in one launch)
cudaError_t launch_sweep_tc_batch(const InstDesc *d, const WorkItem *w, int nitems, int *err, int grid,
                                  cudaStream_t s);
struct FinItem {
    int inst, block;
};
cudaError_t launch_finalize_batch(const InstDesc *d, const FinItem *items, int nitems, int *due, cudaStream_t s);
// adaptive step: the commit of every instance whose candidate was accepted
cudaError_t launch_commit_batch(const InstDesc *d, const FinItem *items, int nitems, cudaStream_t s);

// ---------------------------------------------------------------- finalize + recovery (S1, S3)
struct FinArgs {
    int N, n, NP;
    int precision;           // 0: FP64 vectors, else FP32 vectors
    int col_splits, row_blocks;
    long long ld, ldv;
    const void *rowpart;     // float or double, S x N x (NP+1)
    const void *colpart;     // float or double, RB x ld
    const double *X;         // N x n FP64
    const double *ybar;
    double *a_new, *b_new;   // C^T lambda^k (written)
    const double *a_old, *b_old;  // C^T lambda^{k-1}
    // recovery outputs for the next sweep
    float *yh, *yl, *uh, *ul, *xiT;      // FP32 mode
    double *y64, *u64, *xiT64;           // FP64 mode
    const float *xT32;                   // FP32 points (u uses the rounded xi and x)
    float *xi_rm;                        // tensor-core sweep: xi row-major [2][ldv][32] (hi, lo), or NULL
    double *blockpart;       // gridDim x 3
    double *log;             // kLogCap x 3
    DevState *st;
    int init;                // 1: no partials, a = b = 0 (builds eta(lambda^0))
    // adaptive step: this launch is pass 1 of an iteration.  (a,b)^k goes to a_new/b_new (the
    // candidate buffers), C^T lambda^{k-1} and C^T lambda^{k-2} are taken from hist_a/hist_b
    // by the parity of the device-side k, the recovery waits for launch_commit.
    int adaptive;
    double *hist_a[2], *hist_b[2];
    const void *dpart;       // float or double, dgroups x N: row sums of (lambda^k - lambda~^k)^2
    int dgroups;
    // 1: the partials reduce lambda^k - lambda^{k-1}, so (a,b)^k = (a,b)^{k-1} + their C^T
    int delta;
    // batches: when an exact refresh of this instance becomes due (k a multiple of
    // refresh_period) the last CTA appends inst to the device list due ([0] = count)
    int *due, inst, refresh_period;
};
cudaError_t launch_finalize(const FinArgs &a, cudaStream_t s);
// adaptive step, pass 2: when the candidate was accepted, store (a,b)^k in the history and
// build eta(lambda~^{k+1}) for the next sweep; otherwise nothing changes
cudaError_t launch_commit(const FinArgs &a, cudaStream_t s);
int finalize_blocks(int N);   // CTAs of the finalize kernel (size of its block-partial buffer / 3)

// ---------------------------------------------------------------- exact C^T refresh (cr_refresh.cu)
struct RefreshArgs {
    int N, n, period, segs;
    long long ld, ldv;
    float *lam[3];           // the multiplier buffers (lambda^k chosen on the device)
    const double *X, *ybar;
    double *hist_a[2], *hist_b[2];
    double *r_out, *B_out;   // N, N x n scratch
    double *cpart;           // segs x N scratch
    double *blockpart;       // refresh_finish_blocks(N) x 3
    double *log;
    float *yh, *yl, *uh, *ul, *xiT, *xi_rm;
    const float *xT32;
    DevState *st;
};
int refresh_segments(int N, int sms);
int refresh_finish_blocks(int N);
cudaError_t launch_refresh(const RefreshArgs &a, int sms, cudaStream_t s);
// batches: the refresh of every instance on the device list due (filled by the batched finalize)
cudaError_t launch_refresh_batch(const InstDesc *d, const int *due, int max_due, int sms, cudaStream_t s);

// eta(lambda^k) from the history: y = ybar + a, xi = b / gamma (FP64, row-major)
cudaError_t launch_primal(int N, int n, const double *ybar, const double *a, const double *b,
                          const DevState *st, double *y, double *xi, cudaStream_t s);

// ---------------------------------------------------------------- certificate (S4)
struct CertArgs {
    int N, n, NP;
    int precision;
    int row_splits;          // R
    long long ldv;
    const double *X, *ybar;
    const double *a, *b;     // C^T lambda^k
    // vectors of eta(lambda^k) built by the prep kernel
    float *yh, *yl, *uh, *ul, *xiT;  // FP32
    double *y64, *u64, *xiT64;       // FP64
    const float *xT32;
    const double *xT64;
    // partial results per (row split, column)
    double *pmax; int *parg; double *pinf;   // R x N
    double *blockpart;
    DevState *st;
};
cudaError_t launch_cert(const CertArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- Lipschitz (S0)
// Returns max_l lambda_max(sum_j (x_l - x_j)(x_l - x_j)^T) = sigma_max(A2)^2.
cudaError_t a2_sigma_sq(const double *X, int N, int n, double *out_host, cudaStream_t s);

// ---------------------------------------------------------------- helpers
cudaError_t launch_transpose_points(const double *X, int N, int n, int NP, long long ldv,
                                    float *xT32, double *xT64, float *xT2, cudaStream_t s);
cudaError_t launch_lambda_to_f64(const void *lam, int is_f32, int N, long long ld, long long row0,
                                 long long rows, double *out, long long ldo, cudaStream_t s);
cudaError_t launch_check_finite(const double *v, long long count, int *flag, cudaStream_t s);

}  // namespace cr
