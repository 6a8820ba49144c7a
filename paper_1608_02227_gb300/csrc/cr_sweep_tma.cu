// cr_sweep_tma.cu -- FP32 Lambda sweep with a TMA / mbarrier pipeline (the production
// kernel of CR_FP32).  Same arithmetic as the FP32 kernel of cr_sweep.cu (Steps 2 and 4
// of Figure "papg" with K = N, plus the C^T reductions), organised for sm_103a:
//
//   * one producer warp issues 2-D TMA copies (cp.async.bulk.tensor) of each 32 x 128
//     tile of lambda^{k-1} and lambda^{k-2}, the 128 x_j and y_j of the chunk, and once
//     per work item the xi_i and u_i of its 32 rows, into a ring of shared-memory stages
//     guarded by mbarriers (full: transaction bytes; empty: released by the consumers);
//   * eight consumer warps own 4 rows each (2 above 20 components); lane l owns columns
//     4l..4l+3 of the chunk.  Residuals xi_i.x_j and the Lambda.X accumulation use packed
//     f32x2 FMAs; lambda^k is written with 128-bit streaming stores straight from registers;
//   * per-chunk column sums: every warp parks its partial in its own (already consumed)
//     rows of the P tile; the last warp to finish the chunk (shared-memory ticket) adds the
//     partials in warp order -- deterministic -- writes one partial per (row block, column)
//     and releases the stage;
//   * every mbarrier wait is bounded (2 s); on expiry the CTA sets an abort flag, stops
//     waiting, records CR_ETIMEOUT in device memory and drains its outstanding copies.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "cr_internal.cuh"

namespace cr {
namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the CTA is aborting or the wait ran out (then abort is set).
// A bound shorter than the default (the failure-path hook) polls with the non-blocking test,
// so that a blocking try_wait cannot outlast it.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *gerr, unsigned long long limit_ns = kWaitNs) {
    if (limit_ns < kWaitNs) {
        const uint64_t t0 = globaltimer();
        for (;;) {
            if (mbar_test_wait(bar, parity)) return true;
            if (*abort_flag) return false;
            if (globaltimer() - t0 >= limit_ns) {
                *abort_flag = 1;
                atomicExch(gerr, CR_ETIMEOUT);
                return false;
            }
        }
    }
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicExch(gerr, CR_ETIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *tm) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}
template <int NP>
struct TmaShape {
    // 8 consumer warps; 4 rows each up to 20 components, 2 rows each above (registers)
    static constexpr int MR = NP <= 20 ? 4 : 2;            // rows per consumer warp
    static constexpr int CW = 8;                           // consumer warps
    static constexpr int kRowsT = MR * CW;                 // rows per work item
    static constexpr int THREADS = (CW + 1) * 32;
    static constexpr int TILE = kRowsT * kChunk;           // floats in one Lambda tile
    static constexpr int STAGE_FLOATS = 2 * TILE + NP * kChunk + 2 * kChunk;
    static constexpr int STAGE_BYTES = ((STAGE_FLOATS * 4 + 1023) / 1024) * 1024;
    static constexpr int ROWBUF_FLOATS = NP * kRowsT + 2 * kRowsT;
    static constexpr int STAGES = (4 * STAGE_BYTES + 5 * ROWBUF_FLOATS * 4 + 2048 <= 227 * 1024) ? 4 : 3;
    static constexpr int XB = STAGES + 1;                  // per-item row buffers
    static constexpr int TX_CHUNK = STAGE_FLOATS * 4;
    static constexpr int TX_ROWS = ROWBUF_FLOATS * 4;
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + (size_t)XB * ROWBUF_FLOATS * 4 + 256;
};

// Per-item view of the data a work item needs (tensor maps, pointers, tile bounds).
struct ItemView {
    const CUtensorMap *P, *Q, *X, *Y, *Xi, *U;
    int delta;               // reduce lambda^k - lambda^{k-1} instead of lambda^k
    int row0, row_end;       // the Lambda buffers hold rows [row0, row_end) from their row 0
    float *Qp;               // lambda^k is written here
    float *dpart;            // adaptive step: row sums of (lambda^k - lambda~^k)^2, [S][N]
    long long ld, c0, c1;
    int N, i0, rb, sp;
    float *rowpart, *colpart;
    const DevState *st;
};

// One instance: the tensor maps are kernel parameters, items tile [0, N) x [0, ld).
struct SrcSingle {
    const CUtensorMap *P, *Q, *X, *Y, *Xi, *U;
    TmaSweepArgs a;
    __device__ __forceinline__ int count() const { return a.row_blocks * a.col_splits; }
    __device__ __forceinline__ unsigned long long consumer_wait_ns() const {
        return a.consumer_wait_ns ? a.consumer_wait_ns : kWaitNs;
    }
    __device__ __forceinline__ void prefetch() const {
        prefetch_tmap(P);
        prefetch_tmap(Q);
        prefetch_tmap(X);
        prefetch_tmap(Y);
        prefetch_tmap(Xi);
        prefetch_tmap(U);
    }
    __device__ __forceinline__ ItemView view(int item, int rows) const {
        ItemView v;
        v.P = P; v.Q = Q; v.X = X; v.Y = Y; v.Xi = Xi; v.U = U;
        v.delta = a.delta;
        v.Qp = a.Q;
        v.dpart = a.dpart;
        if (a.adaptive) {  // buffer roles rotate on the device (three buffers)
            int bp, bq, br;
            lam_roles(a.st, 1, 0, &bp, &bq, &br);
            v.P = a.lmaps + bp;
            v.Q = a.lmaps + bq;
            v.Qp = br == 0 ? a.B[0] : (br == 1 ? a.B[1] : a.B[2]);  // no dynamic index into the parameters
        }
        v.ld = a.ld;
        v.N = a.N;
        v.row0 = a.row0;
        v.row_end = a.row_end;
        v.rb = item / a.col_splits;
        v.sp = item - v.rb * a.col_splits;
        v.i0 = a.row0 + v.rb * rows;
        v.c0 = (long long)v.sp * a.cols_per_split;
        v.c1 = min(v.c0 + (long long)a.cols_per_split, a.ld);
        v.rowpart = a.rowpart;
        v.colpart = a.colpart;
        v.st = a.st;
        return v;
    }
};

// Many instances: per-instance descriptors (with their tensor maps) in global memory and a
// work-list of (instance, row block, column split).  The ping-pong parity of each instance
// comes from its own device iteration counter, so a captured graph replays correctly for
// instances that joined at any iteration.
struct SrcBatch {
    const InstDesc *d;
    const WorkItem *w;
    int n;
    __device__ __forceinline__ int count() const { return n; }
    __device__ __forceinline__ unsigned long long consumer_wait_ns() const { return kWaitNs; }
    __device__ __forceinline__ void prefetch() const {}
    __device__ __forceinline__ ItemView view(int item, int rows) const {
        const WorkItem wi = w[item];
        const InstDesc &D = d[wi.inst];
        int bp, bq, br;
        lam_roles(D.st, D.adaptive, (int)(D.st->k & 1), &bp, &bq, &br);
        ItemView v;
        v.P = &D.tm_lam[bp];
        v.Q = &D.tm_lam[bq];
        v.X = &D.tm_x; v.Y = &D.tm_y; v.Xi = &D.tm_xi; v.U = &D.tm_u;
        v.delta = D.delta;
        v.Qp = D.lam[br];
        v.dpart = D.dpart;
        v.ld = D.ld;
        v.N = D.N;
        v.row0 = 0;
        v.row_end = D.N;
        v.rb = wi.rb;
        v.sp = wi.sp;
        v.i0 = wi.rb * rows;
        v.c0 = (long long)wi.sp * D.cols_per_split;
        v.c1 = min(v.c0 + (long long)D.cols_per_split, D.ld);
        v.rowpart = D.rowpart;
        v.colpart = D.colpart;
        v.st = D.st;
        return v;
    }
};

template <int NP, bool ADAPT, class Src>
__device__ __forceinline__ void sweep_body(const Src &src, int *err) {
    using S = TmaShape<NP>;
    constexpr int MR = S::MR, CW = S::CW, STAGES = S::STAGES, XB = S::XB, kRowsT = S::kRowsT;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float *stages = reinterpret_cast<float *>(base);
    float *rowbuf = reinterpret_cast<float *>(base + (size_t)STAGES * S::STAGE_BYTES);
    uint64_t *full = reinterpret_cast<uint64_t *>(rowbuf + XB * S::ROWBUF_FLOATS);
    uint64_t *empty = full + STAGES;
    int *ticket = reinterpret_cast<int *>(empty + STAGES);
    volatile int *abort_flag = ticket + STAGES;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int items = src.count();

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            ticket[s] = 0;
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == CW) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            src.prefetch();
            uint32_t fill = 0, item_no = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++item_no) {
                const ItemView v = src.view(item, kRowsT);
                const int i0 = v.i0;
                const long long c0 = v.c0, c1 = v.c1;
                bool first = true;
                for (long long j0 = c0; j0 < c1; j0 += kChunk, ++fill) {
                    const int s = fill % STAGES;
                    const uint32_t ph = (fill / STAGES) & 1u;
                    // after an abort no new copy is issued: a consumer that gave up on a stage
                    // releases it with that stage's copy possibly still in flight
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, err) || *abort_flag) {
                        ok = false;
                        break;
                    }
                    float *st = stages + (size_t)s * (S::STAGE_BYTES / 4);
                    mbar_arrive_expect_tx(&full[s], S::TX_CHUNK + (first ? S::TX_ROWS : 0));
                    if (first) {
                        float *rbuf = rowbuf + (item_no % XB) * S::ROWBUF_FLOATS;
                        tma_load_2d(rbuf, v.Xi, &full[s], i0, 0);
                        tma_load_2d(rbuf + NP * kRowsT, v.U, &full[s], i0, 0);
                        first = false;
                    }
                    tma_load_2d(st, v.P, &full[s], (int)j0, i0 - v.row0);
                    tma_load_2d(st + S::TILE, v.Q, &full[s], (int)j0, i0 - v.row0);
                    tma_load_2d(st + 2 * S::TILE, v.X, &full[s], (int)j0, 0);
                    tma_load_2d(st + 2 * S::TILE + NP * kChunk, v.Y, &full[s], (int)j0, 0);
                }
            }
            // drain: every issued copy must land before the CTA exits
            const uint32_t issued = fill;
            for (uint32_t f = issued > (uint32_t)STAGES ? issued - STAGES : 0; f < issued; ++f) {
                const int s = f % STAGES;
                const uint32_t ph = (f / STAGES) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&full[s], ph) && globaltimer() - t0 < 200000000ull) {
                }
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        const float2 m1 = make_float2(-1.f, -1.f);
        const unsigned long long cwait = src.consumer_wait_ns();
        uint32_t fill = 0, item_no = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++item_no) {
            const ItemView v = src.view(item, kRowsT);
            const int i0 = v.i0, rb = v.rb, sp = v.sp, NN = v.N, RE = v.row_end;  // RE: end of the rows held
            const long long c0 = v.c0, c1 = v.c1, ld = v.ld;
            const float beta = (float)v.st->beta;
            const float sstep = (float)v.st->s;
            const float2 beta2 = make_float2(beta, beta), s2 = make_float2(sstep, sstep);
            // the reductions see lambda^k - dsub * lambda^{k-1}: the C^T increments in delta form
            const float dsub = v.delta ? 1.f : 0.f;
            const float2 dsub2 = make_float2(-dsub, -dsub);
            const float *rbuf = rowbuf + (item_no % XB) * S::ROWBUF_FLOATS;
            const float *xis = rbuf;                  // [NP][kRowsT]
            const float *ush = rbuf + NP * kRowsT;    // [2][kRowsT]: u hi, u lo
            const int rloc = warp * MR;
            float uh[MR], ul[MR];
            float2 Bp[MR / 2][NP];
            float2 rs2[MR / 2];
            float dd[MR];  // adaptive step: this lane's part of ||lambda^k - lambda~^k||^2 per row
#pragma unroll
            for (int r = 0; r < MR; ++r) dd[r] = 0.f;
#pragma unroll
            for (int p = 0; p < MR / 2; ++p) {
                rs2[p] = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < NP; ++k) Bp[p][k] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < MR; ++r) uh[r] = ul[r] = 0.f;
            bool have_rows = false;
            for (long long j0 = c0; j0 < c1; j0 += kChunk, ++fill) {
                const int s = fill % STAGES;
                const uint32_t ph = (fill / STAGES) & 1u;
                const bool ok = mbar_wait(&full[s], ph, abort_flag, err, cwait);
                float *st = stages + (size_t)s * (S::STAGE_BYTES / 4);
                if (ok) {
                    float lam[MR][4];
                    if (!have_rows) {
#pragma unroll
                        for (int r = 0; r < MR; ++r) {
                            uh[r] = ush[rloc + r];
                            ul[r] = ush[kRowsT + rloc + r];
                        }
                        have_rows = true;
                    }
                    const float *Pt = st, *Qt = st + S::TILE, *Xt = st + 2 * S::TILE;
                    const float *Yt = Xt + NP * kChunk;
                    const float4 yh4 = *reinterpret_cast<const float4 *>(Yt + 4 * lane);
                    const float4 yl4 = *reinterpret_cast<const float4 *>(Yt + kChunk + 4 * lane);
                    // d = (u_i - y_j) (hi and lo parts separately) + xi_i . x_j
                    float2 d[MR][2];
#pragma unroll
                    for (int r = 0; r < MR; ++r) {
                        d[r][0] = make_float2((uh[r] - yh4.x) + (ul[r] - yl4.x), (uh[r] - yh4.y) + (ul[r] - yl4.y));
                        d[r][1] = make_float2((uh[r] - yh4.z) + (ul[r] - yl4.z), (uh[r] - yh4.w) + (ul[r] - yl4.w));
                    }
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const float4 xv = *reinterpret_cast<const float4 *>(Xt + k * kChunk + 4 * lane);
                        const float2 xa = make_float2(xv.x, xv.y), xb = make_float2(xv.z, xv.w);
                        float xr[MR];
                        if constexpr (MR == 4) {
                            const float4 q = *reinterpret_cast<const float4 *>(xis + k * kRowsT + rloc);
                            xr[0] = q.x; xr[1] = q.y; xr[2] = q.z; xr[3] = q.w;
                        } else {
                            const float2 q = *reinterpret_cast<const float2 *>(xis + k * kRowsT + rloc);
                            xr[0] = q.x; xr[1] = q.y;
                        }
#pragma unroll
                        for (int r = 0; r < MR; ++r) {
                            const float2 x2 = make_float2(xr[r], xr[r]);
                            d[r][0] = __ffma2_rn(x2, xa, d[r][0]);
                            d[r][1] = __ffma2_rn(x2, xb, d[r][1]);
                        }
                    }
                    // Steps 4 + 2: lambda~ = P + beta (P - Q); lambda = max(0, lambda~ + s rho)
                    const bool edge = (j0 < (long long)i0 + kRowsT && j0 + kChunk > i0) ||
                                      (j0 + kChunk > NN) || (i0 + kRowsT > RE);
                    float2 cs01 = make_float2(0.f, 0.f), cs23 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int r = 0; r < MR; ++r) {
                        const float4 p4 = *reinterpret_cast<const float4 *>(Pt + (rloc + r) * kChunk + 4 * lane);
                        const float4 q4 = *reinterpret_cast<const float4 *>(Qt + (rloc + r) * kChunk + 4 * lane);
                        const float2 pa = make_float2(p4.x, p4.y), pb = make_float2(p4.z, p4.w);
                        const float2 qa = make_float2(q4.x, q4.y), qb = make_float2(q4.z, q4.w);
                        const float2 lta = __ffma2_rn(beta2, __ffma2_rn(qa, m1, pa), pa);
                        const float2 ltb = __ffma2_rn(beta2, __ffma2_rn(qb, m1, pb), pb);
                        const float2 va = __ffma2_rn(s2, d[r][0], lta);
                        const float2 vb = __ffma2_rn(s2, d[r][1], ltb);
                        lam[r][0] = fmaxf(va.x, 0.f);
                        lam[r][1] = fmaxf(va.y, 0.f);
                        lam[r][2] = fmaxf(vb.x, 0.f);
                        lam[r][3] = fmaxf(vb.y, 0.f);
                        if (edge) {
                            const int i = i0 + rloc + r;
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const long long j = j0 + 4 * lane + c;
                                if (i >= RE || j >= NN || j == i) lam[r][c] = 0.f;
                            }
                        }
                        if constexpr (ADAPT) {  // s rho where the step is not clipped: no cancellation
                            const float2 sra = __fmul2_rn(s2, d[r][0]), srb = __fmul2_rn(s2, d[r][1]);
                            const float e0 = lam[r][0] > 0.f ? sra.x : -lta.x;
                            const float e1 = lam[r][1] > 0.f ? sra.y : -lta.y;
                            const float e2 = lam[r][2] > 0.f ? srb.x : -ltb.x;
                            const float e3 = lam[r][3] > 0.f ? srb.y : -ltb.y;
                            dd[r] = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, dd[r]))));
                        }
                        if (4 * lane + j0 < c1 && i0 + rloc + r < RE)
                            __stcs(reinterpret_cast<float4 *>(v.Qp + (long long)(i0 + rloc + r - v.row0) * ld + j0 + 4 * lane),
                                   make_float4(lam[r][0], lam[r][1], lam[r][2], lam[r][3]));
                        // from here on lam holds what the reductions sum: lambda^k, or its change
                        // (lambda^{k-1} is 0 on the diagonal and the padding, as lambda^k is)
                        {
                            const float2 da = __ffma2_rn(dsub2, pa, make_float2(lam[r][0], lam[r][1]));
                            const float2 db = __ffma2_rn(dsub2, pb, make_float2(lam[r][2], lam[r][3]));
                            lam[r][0] = da.x, lam[r][1] = da.y, lam[r][2] = db.x, lam[r][3] = db.y;
                        }
                        cs01 = __fadd2_rn(cs01, make_float2(lam[r][0], lam[r][1]));
                        cs23 = __fadd2_rn(cs23, make_float2(lam[r][2], lam[r][3]));
                    }
#pragma unroll
                    for (int p = 0; p < MR / 2; ++p) {
                        const float2 a01 = make_float2(lam[2 * p][0], lam[2 * p + 1][0]);
                        const float2 a11 = make_float2(lam[2 * p][1], lam[2 * p + 1][1]);
                        const float2 a21 = make_float2(lam[2 * p][2], lam[2 * p + 1][2]);
                        const float2 a31 = make_float2(lam[2 * p][3], lam[2 * p + 1][3]);
                        rs2[p] = __fadd2_rn(rs2[p], __fadd2_rn(__fadd2_rn(a01, a11), __fadd2_rn(a21, a31)));
                    }
                    // park the column partial in this lane's own (consumed) slot of P
                    *reinterpret_cast<float4 *>(st + rloc * kChunk + 4 * lane) =
                        make_float4(cs01.x, cs01.y, cs23.x, cs23.y);
                    // B_i += sum_j lambda_ij x_j  (rows paired into f32x2)
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const float4 xv = *reinterpret_cast<const float4 *>(Xt + k * kChunk + 4 * lane);
#pragma unroll
                        for (int p = 0; p < MR / 2; ++p) {
                            float2 acc = Bp[p][k];
                            acc = __ffma2_rn(make_float2(lam[2 * p][0], lam[2 * p + 1][0]), make_float2(xv.x, xv.x), acc);
                            acc = __ffma2_rn(make_float2(lam[2 * p][1], lam[2 * p + 1][1]), make_float2(xv.y, xv.y), acc);
                            acc = __ffma2_rn(make_float2(lam[2 * p][2], lam[2 * p + 1][2]), make_float2(xv.z, xv.z), acc);
                            acc = __ffma2_rn(make_float2(lam[2 * p][3], lam[2 * p + 1][3]), make_float2(xv.w, xv.w), acc);
                            Bp[p][k] = acc;
                        }
                    }
                }
                // stage hand-off: the last warp through reduces the column partials (in warp
                // order) and releases the stage to the producer
                __syncwarp();
                int last = 0;
                if (lane == 0) {
                    __threadfence_block();
                    last = (atomicAdd(&ticket[s], 1) == CW - 1);
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence_block();
                    if (ok && !*abort_flag) {
                        const long long jl = j0 + 4 * lane;
                        float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int w = 0; w < CW; ++w) {
                            const float4 t = *reinterpret_cast<const float4 *>(st + w * MR * kChunk + 4 * lane);
                            cv.x += t.x;
                            cv.y += t.y;
                            cv.z += t.z;
                            cv.w += t.w;
                        }
                        if (jl < c1) *reinterpret_cast<float4 *>(v.colpart + (long long)rb * ld + jl) = cv;
                    }
                    __syncwarp();
                    if (lane == 0) {
                        ticket[s] = 0;
                        mbar_arrive(&empty[s]);
                    }
                }
            }
            // row partials of this item: reduce across the 32 lanes
#pragma unroll
            for (int p = 0; p < MR / 2; ++p) {
                const int ia = i0 + rloc + 2 * p, ib = ia + 1;
                float *da = v.rowpart + ((long long)sp * NN + ia) * (NP + 1);
                float *db = v.rowpart + ((long long)sp * NN + ib) * (NP + 1);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    float vx = Bp[p][k].x, vy = Bp[p][k].y;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        vx += __shfl_xor_sync(0xffffffffu, vx, o);
                        vy += __shfl_xor_sync(0xffffffffu, vy, o);
                    }
                    if (lane == 0) {
                        if (ia < RE) da[k] = vx;
                        if (ib < RE) db[k] = vy;
                    }
                }
                float vx = rs2[p].x, vy = rs2[p].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vx += __shfl_xor_sync(0xffffffffu, vx, o);
                    vy += __shfl_xor_sync(0xffffffffu, vy, o);
                }
                if (lane == 0) {
                    if (ia < RE) da[NP] = vx;
                    if (ib < RE) db[NP] = vy;
                }
            }
            if constexpr (ADAPT) {
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    float v2 = dd[r];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v2 += __shfl_xor_sync(0xffffffffu, v2, o);
                    const int i = i0 + rloc + r;
                    if (lane == 0 && i < RE) v.dpart[(long long)sp * NN + i] = v2;
                }
            }
        }
    }
}


template <int NP, bool ADAPT>
__global__ void __launch_bounds__(TmaShape<NP>::THREADS, 1)
    sweep_tma_kernel(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmQ,
                     const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY,
                     const __grid_constant__ CUtensorMap tmXi, const __grid_constant__ CUtensorMap tmU,
                     const TmaSweepArgs a) {
    SrcSingle src{&tmP, &tmQ, &tmX, &tmY, &tmXi, &tmU, a};
    sweep_body<NP, ADAPT>(src, a.err);
}

template <int NP, bool ADAPT>
__global__ void __launch_bounds__(TmaShape<NP>::THREADS, 1)
    sweep_tma_batch_kernel(const InstDesc *d, const WorkItem *w, int nitems, int *err) {
    SrcBatch src{d, w, nitems};
    sweep_body<NP, ADAPT>(src, err);
}

#define CR_NP_LIST(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(28) X(32)

int tma_diag_regs = 0, tma_diag_maxthreads = 0, tma_diag_smem = 0, tma_diag_threads = 0;

template <int NP>
cudaError_t run_tma(const TmaMaps &m, const TmaSweepArgs &a, int grid, cudaStream_t st, int *occ) {
    using S = TmaShape<NP>;
    auto k = a.adaptive ? sweep_tma_kernel<NP, true> : sweep_tma_kernel<NP, false>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tma_kernel<NP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)S::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sweep_tma_kernel<NP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)S::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (occ) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, S::THREADS, S::SMEM);
        if (e == cudaSuccess && *occ == 0) {
            cudaFuncAttributes fa{};
            cudaFuncGetAttributes(&fa, k);
            tma_diag_regs = fa.numRegs;
            tma_diag_maxthreads = fa.maxThreadsPerBlock;
            tma_diag_smem = (int)S::SMEM;
            tma_diag_threads = S::THREADS;
        }
        return e;
    }
    k<<<grid, S::THREADS, S::SMEM, st>>>(*m.P, *m.Q, m.X, m.Y, m.Xi, m.U, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_tma(int np, const TmaMaps &m, const TmaSweepArgs &a, int grid, cudaStream_t s) {
    switch (np) {
#define CASE(V) \
    case V: return run_tma<V>(m, a, grid, s, nullptr);
        CR_NP_LIST(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <int NP>
cudaError_t run_tma_batch(const InstDesc *d, const WorkItem *w, int nitems, int *err, int grid, bool adaptive,
                          cudaStream_t st) {
    using S = TmaShape<NP>;
    auto k = adaptive ? sweep_tma_batch_kernel<NP, true> : sweep_tma_batch_kernel<NP, false>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tma_batch_kernel<NP, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sweep_tma_batch_kernel<NP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)S::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k<<<grid, S::THREADS, S::SMEM, st>>>(d, w, nitems, err);
    return cudaGetLastError();
}

cudaError_t launch_sweep_tma_batch(int np, const InstDesc *d, const WorkItem *w, int nitems, int *err, int grid,
                                   bool adaptive, cudaStream_t s) {
    switch (np) {
#define CASE(V) \
    case V: return run_tma_batch<V>(d, w, nitems, err, grid, adaptive, s);
        CR_NP_LIST(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_tma_occupancy(int np, int *blocks_per_sm) {
    TmaMaps m{};
    TmaSweepArgs a{};
    switch (np) {
#define CASE(V) \
    case V: return run_tma<V>(m, a, 0, 0, blocks_per_sm);
        CR_NP_LIST(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

void sweep_tma_diag(int *v4) {
    v4[0] = tma_diag_regs;
    v4[1] = tma_diag_maxthreads;
    v4[2] = tma_diag_smem;
    v4[3] = tma_diag_threads;
}

int sweep_tma_rows(int np) {
    switch (np) {
#define CASE(V) \
    case V: return TmaShape<V>::kRowsT;
        CR_NP_LIST(CASE)
#undef CASE
        default: return 0;
    }
}

// 2-D FP32 tensor map over a row-major [rows][cols] array with leading dimension ld (elements)
cudaError_t make_tmap_2d(CUtensorMap *tm, const float *base, long long cols, long long rows, long long ld,
                         int box_cols, int box_rows, bool swizzle128) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * sizeof(float))};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace cr
