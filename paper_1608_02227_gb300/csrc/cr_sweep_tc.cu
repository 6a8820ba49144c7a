// cr_sweep_tc.cu -- the Lambda sweep with both contractions on the tensor cores
// (CR_MIXED_TF32): Steps 2 and 4 of Figure "papg" (K = N) and the C^T reductions, with
//     S   = Xi_blk . X_block^T         (rho_ij = u_i - y_j + S_ij)             [GEMM1]
//     ACC += Lambda_blk . [X | 1]_chunk    (row sums of Lambda.X and of Lambda)   [GEMM2]
// as tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory.  TF32 keeps the top
// 19 bits of each FP32 operand (the hardware truncates), so every operand v is split into
// hi = v (read as trunc(v)) and lo = v - trunc(v):
//   GEMM1 forms hi.hi + hi.lo + lo.hi with xi (the A operand) held in tensor memory;
//   GEMM2 stacks the hi and lo parts of [X | 1] along N (N = 64) and runs the hi and the
//   lo part of Lambda (or of its change, in delta form) against it, so the accumulator holds
//   Lambda.[X|1]_hi in columns 0..31 and Lambda.X_lo in columns 32..63.
// A tcgen05.mma kind::tf32 with M = 128 takes the same time at N = 64 and at N = 128 (timed on
// this kernel: the tensor pipe is paid per instruction, one K step of 8), so GEMM1 covers a
// block of four 32-column chunks with each instruction (N = 128) and GEMM2 the two halves of
// the operand split.  GEMM2 (8 instructions a chunk) goes to the tensor pipe before the next
// block's GEMM1 (12 instructions a block), so a stage is released soon after its epilogue.
//
// CTA = 12 warps, one CTA per SM, work items of 128 rows x a range of columns, walked in
// chunks of 32 columns (blocks of four chunks for GEMM1):
//   warp 0  producer: 2-D TMA loads (128-byte swizzle) of the lambda^{k-1}, lambda^{k-2}
//           tiles (128 x 32), the chunk's transposed points with a row of ones (hi rows
//           then lo rows; 64 x 32) and y (hi, lo), into a ring of stages;
//   warp 10 second producer: the point rows of each block (hi, lo; 128 x 32 each) for
//           GEMM1, freed as soon as GEMM1 is done;
//   warp 1  tensor-memory allocation and the single MMA-issuing thread: GEMM1 runs one
//           block ahead of the epilogue (two S tiles in tensor memory);
//   warps 2-9  epilogue in two groups of four (one warp per tensor-memory lane quarter)
//           that take the even and the odd chunks of an item, thread = row: reads S from
//           tensor memory, forms lambda^k (packed FP32x2 arithmetic), writes it over the
//           consumed lambda^{k-1} tile (the source of the TMA store) and the A operand of
//           GEMM2 over the lambda^{k-2} tile (in delta form the change, its TF32 low part
//           going to the group's slot in tensor memory); the first group also copies the xi
//           rows of the next item into tensor memory; at the end of an item both groups read
//           the GEMM2 accumulator (row partials);
//   warp 11 the TMA store of each new lambda^k tile (128 rows) and its column sums (the
//           column partials), off the epilogue's path; it releases the stage once it has read
//           the tile and the store has read it too.
// Every wait is bounded (2 s); on expiry the CTA aborts cleanly and reports CR_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "cr_internal.cuh"

namespace cr {
namespace {

constexpr int kM = 128;       // rows per item (MMA M, tensor-memory lanes)
constexpr int kC = 32;        // columns per chunk (GEMM2 K)
constexpr int kK = 32;        // point dimension padded (GEMM1 K)
constexpr int kStages = 4;    // ring of lambda / transposed-point stages
constexpr int kQ = 4;         // chunks per GEMM1 block (N = 128: a tcgen05.mma costs the same at N = 64)
constexpr int kXr = 1;        // ring of point-row block tiles (GEMM1 B operand)
constexpr int kSBufs = 2;     // block S tiles in tensor memory
constexpr int kTiles = kM * kC * 4;             // bytes of one 128 x 32 FP32 tile (16 KB)
constexpr int kXtBytes = 2 * kK * kC * 4;       // transposed points, hi and lo rows (64 x 32, 8 KB)
// stage layout (bytes): P | Q | XT; y (hi 32, lo 32) and the column partials of each
// stage sit in small arrays after the point-row ring
constexpr int kOffP = 0, kOffQ = kTiles, kOffXT = 2 * kTiles;
constexpr int kStageBytes = 2 * kTiles + kXtBytes;
constexpr int kYBytes = 2 * kC * 4;
constexpr int kTxStage = kStageBytes + kYBytes;
constexpr int kXrHalf = kQ * kC * kK * 4;       // one 128 x 32 point-row tile (16 KB)
constexpr int kXrBytes = 2 * kXrHalf;           // hi | lo
constexpr int kEpiWarps = 8;                    // two groups of four (one warp per lane quarter)
constexpr int kHalf = kC / 2;                   // accumulator columns read by each group
constexpr int kXrWarp = 2 + kEpiWarps;          // second producer
constexpr int kColWarp = 3 + kEpiWarps;         // column sums of the new tiles
constexpr int kThreads = (4 + kEpiWarps) * 32;  // 384 x 168 registers: the whole register file
constexpr size_t kSmemData =
    (size_t)kStages * kStageBytes + (size_t)kXr * kXrBytes + (size_t)kStages * kYBytes;
constexpr size_t kSmem = 1024 + kSmemData + 512;
static_assert(kStageBytes % 1024 == 0 && kXrBytes % 1024 == 0, "swizzled tiles keep 1024-byte alignment");
static_assert(kSmem <= 232448, "shared memory budget");
// tensor memory: S[b] (128 columns each: a block of four chunks) at 128 b, ACC (64) at 256,
// XI[0..1] (hi 32 + lo 32 each) at 320, DLO[0..1] (32 each; delta form: the TF32 low part of
// the change of lambda, the second A operand of GEMM2, one slot per epilogue group) at 448.
// One accumulator is enough: both groups read it at the end of an item before they start on
// the next one.
constexpr uint32_t kTmemCols = 512;
constexpr int kAccBufs = 1, kDloBufs = 1;
constexpr uint32_t kColS = (uint32_t)(kQ * kC);
constexpr uint32_t kColAcc = kColS * kSBufs, kColXi = kColAcc + 64u * kAccBufs, kColDlo = kColXi + 128u;
static_assert(kColDlo + 64u * kDloBufs <= kTmemCols, "tensor-memory budget");
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr uint32_t kSuspendNs = 1000000u;     // a polling thread sleeps in try_wait up to 1 ms
constexpr int kTcDevices = 128;

__device__ __forceinline__ uint32_t su32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t *b, uint32_t ph) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(ph), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
// non-blocking test of the same condition
__device__ __forceinline__ bool bar_test(uint64_t *b, uint32_t ph) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(ph)
        : "memory");
    return ok != 0;
}
// bounded wait on the phase `use` of a barrier (completes when the barrier has finished
// phase number `use`); false when the CTA aborts
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t use, volatile int *abort_flag, int *err) {
    const uint32_t ph = use & 1u;
    if (bar_try(b, ph)) return true;
    const uint64_t t0 = gtimer();
    for (;;) {
        if (bar_try(b, ph)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicExch(err, CR_ETIMEOUT);
            return false;
        }
    }
}
// wait for the release of the previous use of a slot (first use passes at once)
__device__ __forceinline__ bool slot_wait(uint64_t *b, uint32_t use, volatile int *abort_flag, int *err) {
    return use == 0 ? true : bar_wait(b, use - 1, abort_flag, err);
}
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap *tm, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(su32(src)), "r"(x), "r"(y)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand in a 128-byte-swizzled tile: rows of 128 B, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}
// kind::tf32, D = F32, A and B TF32 K-major, M = 128, N = 64 (GEMM2) or N = kQ * 32 (GEMM1)
constexpr uint32_t idesc_tf32(uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}
constexpr uint32_t kIdesc = idesc_tf32(64), kIdesc1 = idesc_tf32(kColS);

__device__ __forceinline__ void mma_ss(uint32_t tmem_d, uint64_t ad, uint64_t bd, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"((uint32_t)acc)
        : "memory");
}
__device__ __forceinline__ void mma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, bool acc,
                                       uint32_t idesc = kIdesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bd), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// GEMM1: S = xi_hi.x_hi + xi_hi.x_lo + xi_lo.x_hi, xi in tensor memory (hi at column a,
// lo at a + 32), the block's 128 point rows in shared memory (hi tile at bh, lo at bl)
__device__ __forceinline__ void gemm1(uint32_t tmem_d, uint32_t a, uint32_t bh, uint32_t bl) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const uint32_t A = p < 2 ? a : a + 32u, B = p == 1 ? bl : bh;
#pragma unroll
        for (int k = 0; k < kK / 8; ++k) mma_ts(tmem_d, A + 8u * k, sdesc(B + 32 * k), p > 0 || k > 0, kIdesc1);
    }
}
// GEMM2: ACC (+)= lambda_hi.[X|1 ; X_lo] + lambda_lo.[X|1 ; X_lo] over the chunk's 32 columns
__device__ __forceinline__ void gemm2(uint32_t tmem_d, uint32_t ah, uint32_t al, uint32_t b, bool acc_first) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const uint32_t A = p == 0 ? ah : al;
#pragma unroll
        for (int k = 0; k < kC / 8; ++k) mma_ss(tmem_d, sdesc(A + 32 * k), sdesc(b + 32 * k), acc_first || p > 0 || k > 0);
    }
}
// GEMM2 in delta form: the change of lambda (FP32, read as TF32) from shared memory and its
// TF32 low part from tensor memory (columns dlo .. dlo + 31)
__device__ __forceinline__ void gemm2_delta(uint32_t tmem_d, uint32_t ah, uint32_t dlo, uint32_t b, bool acc_first) {
#pragma unroll
    for (int k = 0; k < kC / 8; ++k) mma_ss(tmem_d, sdesc(ah + 32 * k), sdesc(b + 32 * k), acc_first || k > 0);
#pragma unroll
    for (int k = 0; k < kC / 8; ++k) mma_ts(tmem_d, dlo + 8u * k, sdesc(b + 32 * k), true);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15])),
        "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])),
        "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])), "r"(__float_as_uint(v[27])),
        "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}
__device__ __forceinline__ float tf32_lo(float v) { return v - __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// Everything one work item of 128 rows x one column split needs: the tensor maps of its
// instance, its vectors and partial buffers, the roles of its multiplier buffers and its bounds.
struct TcView {
    const CUtensorMap *P, *Q, *R;            // lambda^{k-1}, lambda^{k-2} (loads), lambda^k (store)
    const CUtensorMap *XRh, *XRl, *XT, *Y;   // point rows (hi, lo), transposed points, y (hi, lo)
    const float *xi_rm, *u;
    float *rowpart, *colpart, *dpart;
    const DevState *st;
    long long ld, ldv, c0, c1;
    int N, n, NP, rb, sp, i0, nch, adaptive, delta;
    int row0, row_end;                       // the Lambda buffers hold rows [row0, row_end) from their row 0
};

__device__ __forceinline__ void tc_bounds(TcView &v, int cols_per_split) {
    v.i0 = v.row0 + v.rb * kM;
    v.c0 = (long long)v.sp * cols_per_split;
    v.c1 = min(v.c0 + (long long)cols_per_split, v.ld);
    v.nch = (int)((v.c1 - v.c0 + kC - 1) / kC);
}

// One instance: the point maps are kernel parameters.  Items tile [0, N) x [0, ld) in one of
// two ways: 128 rows x one column split, dealt to the CTAs in turn (a->seg = 0); or (a->seg = 1)
// CTA b takes the 32-column chunks [T b / G, T (b + 1) / G) of the T = row_blocks x nchr chunks
// in row-block order (G CTAs, nchr chunks to a row block), so that no CTA has more than one
// chunk above the average, and its items are the pieces of that range in each row block.
// Piece sp of a row block (sp = the CTAs before b that reach into it) writes row-partial slot sp.
struct TcSrcSingle {
    const CUtensorMap *XRh, *XRl, *XT, *Y;
    const TcSweepArgs *a;
    __device__ __forceinline__ long long seg_lo(long long b) const { return b * a->seg_total / gridDim.x; }
    __device__ __forceinline__ int begin() const { return a->seg ? 0 : (int)blockIdx.x; }
    __device__ __forceinline__ int step() const { return a->seg ? 1 : (int)gridDim.x; }
    __device__ __forceinline__ int end() const {
        if (!a->seg) return a->row_blocks * a->col_splits;
        const long long g0 = seg_lo(blockIdx.x), g1 = seg_lo(blockIdx.x + 1);
        return g1 > g0 ? (int)((g1 - 1) / a->seg_nchr - g0 / a->seg_nchr + 1) : 0;
    }
    __device__ __forceinline__ TcView view(int item) const {
        TcView v;
        int bp, bq, br;
        lam_roles(a->st, a->adaptive, a->p_host, &bp, &bq, &br);
        v.P = a->lmaps + bp;
        v.Q = a->lmaps + bq;
        v.R = a->lmaps + br;
        v.delta = a->delta;
        v.XRh = XRh, v.XRl = XRl, v.XT = XT, v.Y = Y;
        v.xi_rm = a->xi_rm;
        v.u = a->u;
        v.rowpart = a->rowpart;
        v.colpart = a->colpart;
        v.dpart = a->dpart;
        v.st = a->st;
        v.ld = a->ld;
        v.ldv = a->ldv;
        v.N = a->N;
        v.n = a->n;
        v.NP = a->NP;
        v.adaptive = a->adaptive;
        v.row0 = a->row0;
        v.row_end = a->row_end;
        if (a->seg) {
            const long long g0 = seg_lo(blockIdx.x), g1 = seg_lo(blockIdx.x + 1), T = a->seg_total;
            const long long rb = g0 / a->seg_nchr + item, rs = rb * a->seg_nchr;
            const long long cs = max(g0, rs) - rs, ce = min(g1, rs + a->seg_nchr) - rs;
            // the first CTA whose range holds chunk rs: the largest b' with T b' / G <= rs
            const long long bfirst = ((rs + 1) * gridDim.x + T - 1) / T - 1;
            v.rb = (int)rb;
            v.sp = (int)(blockIdx.x - bfirst);
            v.i0 = v.row0 + v.rb * kM;
            v.c0 = cs * kC;
            v.c1 = min(ce * kC, v.ld);
            v.nch = (int)(ce - cs);
        } else {
            v.rb = item / a->col_splits;
            v.sp = item - v.rb * a->col_splits;
            tc_bounds(v, a->cols_per_split);
        }
        return v;
    }
};

// Many instances: per-instance descriptors (tensor maps included) in global memory and a
// work-list of (instance, 128-row block, column split).  The roles of each instance's
// multiplier buffers follow from its own device state (iteration parity, or the ring of
// the adaptive step), so a captured graph replays correctly for instances that joined late.
struct TcSrcBatch {
    const InstDesc *d;
    const WorkItem *w;
    int n;
    __device__ __forceinline__ int begin() const { return (int)blockIdx.x; }
    __device__ __forceinline__ int step() const { return (int)gridDim.x; }
    __device__ __forceinline__ int end() const { return n; }
    __device__ __forceinline__ TcView view(int item) const {
        const WorkItem wi = w[item];
        const InstDesc &D = d[wi.inst];
        TcView v;
        int bp, bq, br;
        lam_roles(D.st, D.adaptive, (int)(D.st->k & 1), &bp, &bq, &br);
        v.P = &D.tc_lam_ld[bp];
        v.Q = &D.tc_lam_ld[bq];
        v.R = &D.tc_lam_ld[br];
        v.delta = D.delta;
        v.XRh = &D.tc_xrh, v.XRl = &D.tc_xrl, v.XT = &D.tc_xt, v.Y = &D.tc_y;
        v.xi_rm = D.xi_rm;
        v.u = D.uh;
        v.rowpart = D.rowpart;
        v.colpart = D.colpart;
        v.dpart = D.dpart;
        v.st = D.st;
        v.ld = D.ld;
        v.ldv = D.ldv;
        v.N = D.N;
        v.n = D.n;
        v.NP = D.NP;
        v.adaptive = D.adaptive;
        v.row0 = 0;
        v.row_end = D.N;
        v.rb = wi.rb;
        v.sp = wi.sp;
        tc_bounds(v, D.cols_per_split);
        return v;
    }
};

// Steps 4 and 2 for one thread's 32 entries of a chunk row: lambda~ = P + beta (P - Q),
// lambda = max(0, lambda~ + s rho), rho = (u_h - y_h) + (u_l - y_l) + S; the new lambda
// overwrites P and its TF32 low part overwrites Q (both 128-byte swizzled).  EDGE adds the
// zeroing of the diagonal and of padding rows and columns.
// DELTA: P receives lambda^k (the source of the TMA store), Qs the full FP32 change
// lambda^k - lambda^{k-1} (the operand of the C^T reductions in delta form) and dlo its TF32 low
// part, which the caller moves to tensor memory.
// One half of the chunk row (16-byte groups 4 HALF .. 4 HALF + 3); dlo receives the half's low parts.
template <bool EDGE, bool ADAPT, bool DELTA, int HALF>
__device__ __forceinline__ void epi_half(float *P, float *Qs, const float *Y, const float (&v)[kC], int r,
                                         float2 uh2, float2 ul2, float2 beta2, float2 s2, bool rv, int i,
                                         long long j0, int N, float &dsum, float (&dlo)[kC / 2]) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const int rx = r & 7;
#pragma unroll
    for (int g = 4 * HALF; g < 4 * HALF + 4; ++g) {  // 16-byte chunk g of the row sits at position g ^ (r % 8)
        const int off = r * 32 + ((g ^ rx) << 2);
        const float4 p4 = *reinterpret_cast<const float4 *>(P + off);
        const float4 q4 = *reinterpret_cast<const float4 *>(Qs + off);
        const float4 yh = *reinterpret_cast<const float4 *>(Y + 4 * g);
        const float4 yl = *reinterpret_cast<const float4 *>(Y + kC + 4 * g);
        const float2 pv[2] = {make_float2(p4.x, p4.y), make_float2(p4.z, p4.w)};
        const float2 qv[2] = {make_float2(q4.x, q4.y), make_float2(q4.z, q4.w)};
        const float2 yhv[2] = {make_float2(yh.x, yh.y), make_float2(yh.z, yh.w)};
        const float2 ylv[2] = {make_float2(yl.x, yl.y), make_float2(yl.z, yl.w)};
        float l[4], lo[4], sr[4], ltv[4];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float2 sv = make_float2(v[4 * g + 2 * e], v[4 * g + 2 * e + 1]);
            const float2 rho = __fadd2_rn(__fadd2_rn(__ffma2_rn(yhv[e], m1, uh2), __ffma2_rn(ylv[e], m1, ul2)), sv);
            const float2 lt = __ffma2_rn(beta2, __ffma2_rn(qv[e], m1, pv[e]), pv[e]);
            const float2 w = __ffma2_rn(s2, rho, lt);
            l[2 * e] = fmaxf(0.f, w.x);
            l[2 * e + 1] = fmaxf(0.f, w.y);
            if (ADAPT) {
                const float2 srv = __fmul2_rn(s2, rho);
                sr[2 * e] = srv.x, sr[2 * e + 1] = srv.y;
                ltv[2 * e] = lt.x, ltv[2 * e + 1] = lt.y;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (EDGE) {
                const long long j = j0 + 4 * g + e;
                if (!rv || j >= N || j == i) l[e] = 0.f;
            }
            if (!DELTA) lo[e] = tf32_lo(l[e]);
            if (ADAPT) {  // lambda^k - lambda~^k without cancellation: s rho where the step is not clipped
                const float d = l[e] > 0.f ? sr[e] : -ltv[e];
                dsum = fmaf(d, d, dsum);
            }
        }
        *reinterpret_cast<float4 *>(P + off) = make_float4(l[0], l[1], l[2], l[3]);
        if (DELTA) {  // lambda^{k-1} is 0 on the diagonal and the padding, as lambda^k is
            const float d[4] = {l[0] - p4.x, l[1] - p4.y, l[2] - p4.z, l[3] - p4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) dlo[4 * (g - 4 * HALF) + e] = tf32_lo(d[e]);
            *reinterpret_cast<float4 *>(Qs + off) = make_float4(d[0], d[1], d[2], d[3]);
        } else {
            *reinterpret_cast<float4 *>(Qs + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

template <class Src>
__device__ __forceinline__ void sweep_tc_body(const Src &src, int *err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *stage0 = base;
    unsigned char *xr0 = base + (size_t)kStages * kStageBytes;
    unsigned char *y0 = xr0 + (size_t)kXr * kXrBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(y0 + (size_t)kStages * kYBytes);
    uint64_t *full = bars;                  // [kStages] TMA data of a stage landed
    uint64_t *empty = full + kStages;       // [kStages] GEMM2 done; lambda^k stored and read for the column sums (2 arrivals)
    uint64_t *lamr = empty + kStages;       // [kStages] lambda tiles written by the epilogue (4 arrivals)
    uint64_t *sfull = lamr + kStages;       // [kSBufs] GEMM1 result of a block in S[b]
    uint64_t *sempty = sfull + kSBufs;      // [kSBufs] S[b] read by the epilogue (4 arrivals per chunk)
    uint64_t *xfull = sempty + kSBufs;      // [2] xi rows of an item in tensor memory (4 arrivals)
    uint64_t *xempty = xfull + 2;           // [2] all GEMM1 of the item that used them done
    uint64_t *rfull = xempty + 2;           // [kXr] point-row block tiles landed
    uint64_t *rempty = rfull + kXr;         // [kXr] GEMM1 that read them done
    uint64_t *afull = rempty + kXr;         // [kAccBufs] accumulator of an item complete
    uint64_t *aempty = afull + kAccBufs;    // [kAccBufs] accumulator read (one per warp)
    uint64_t *dloe = aempty + kAccBufs;     // [2 kDloBufs] delta form: the GEMM2 that read a DLO slot done
    uint64_t *fin = dloe + 2 * kDloBufs;    // all MMAs done (teardown)
    volatile int *abort_flag = reinterpret_cast<int *>(fin + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1) + 1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ibeg = src.begin(), iend = src.end(), istep = src.step();  // this CTA's items

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 2);
            bar_init(&lamr[s], 4);
        }
        for (int b = 0; b < kSBufs; ++b) {
            bar_init(&sfull[b], 1);
            bar_init(&sempty[b], 4 * kQ);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init(&xfull[b], 4);
            bar_init(&xempty[b], 1);
        }
        for (int b = 0; b < kAccBufs; ++b) {
            bar_init(&afull[b], 1);
            bar_init(&aempty[b], kEpiWarps);
        }
        for (int b = 0; b < 2 * kDloBufs; ++b) bar_init(&dloe[b], 1);
        for (int b = 0; b < kXr; ++b) {
            bar_init(&rfull[b], 1);
            bar_init(&rempty[b], 1);
        }
        bar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto tS = [tmem](int b) { return tmem + kColS * (uint32_t)b; };
    auto tA = [tmem](int b) { return tmem + kColAcc + 64u * (uint32_t)b; };
    auto tX = [tmem](int b) { return tmem + kColXi + 64u * (uint32_t)b; };
    auto tD = [tmem](int slot) { return tmem + kColDlo + 32u * (uint32_t)slot; };  // slot kDloBufs h + use % kDloBufs

    if (warp == 0) {
        // ---------------------------------------------------------------- stage producer
        if (lane == 0) {
            uint32_t fill = 0;
            bool ok = true;
            for (int item = ibeg; item < iend && ok; item += istep) {
                const TcView it = src.view(item);
                for (int c = 0; c < it.nch; ++c, ++fill) {
                    const int s = fill % kStages;
                    const int j0 = (int)(it.c0 + (long long)c * kC);
                    if (!slot_wait(&empty[s], fill / kStages, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    unsigned char *st = stage0 + (size_t)s * kStageBytes;
                    bar_expect(&full[s], kTxStage);
                    tma_load(st + kOffP, it.P, &full[s], j0, it.i0 - it.row0);
                    tma_load(st + kOffQ, it.Q, &full[s], j0, it.i0 - it.row0);
                    tma_load(st + kOffXT, it.XT, &full[s], j0, 0);
                    tma_load(y0 + (size_t)s * kYBytes, it.Y, &full[s], j0, 0);
                }
            }
            // drain the copies still in flight before the CTA can exit
            for (uint32_t f = fill > (uint32_t)kStages ? fill - kStages : 0; f < fill; ++f) {
                const uint64_t t0 = gtimer();
                while (!bar_try(&full[f % kStages], (f / kStages) & 1u) && gtimer() - t0 < 200000000ull) {
                }
            }
        }
    } else if (warp == kXrWarp) {
        // ---------------------------------------------------------------- point-row producer
        if (lane == 0) {
            uint32_t pf = 0;
            bool ok = true;
            for (int item = ibeg; item < iend && ok; item += istep) {
                const TcView it = src.view(item);
                for (int bc = 0; kQ * bc < it.nch; ++bc, ++pf) {
                    const int x = pf % kXr;
                    const int j0 = (int)(it.c0 + (long long)bc * kQ * kC);
                    if (!slot_wait(&rempty[x], pf / kXr, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    unsigned char *xr = xr0 + (size_t)x * kXrBytes;
                    bar_expect(&rfull[x], kXrBytes);
                    tma_load(xr, it.XRh, &rfull[x], 0, j0);
                    tma_load(xr + kXrHalf, it.XRl, &rfull[x], 0, j0);
                }
            }
            for (uint32_t f = pf > (uint32_t)kXr ? pf - kXr : 0; f < pf; ++f) {
                const uint64_t t0 = gtimer();
                while (!bar_try(&rfull[f % kXr], (f / kXr) & 1u) && gtimer() - t0 < 200000000ull) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t fill = 0, itn = 0, cur_blk = 0;
            uint32_t dlo_n[2] = {0u, 0u};  // chunks of each epilogue group so far (DLO slot turns)
            bool ok = true;
            // GEMM1 state: the next block to issue (flattened index g1_blk), its item and chunk count
            int g1_item = ibeg, g1_bc = 0, g1_nch = ibeg < iend ? src.view(ibeg).nch : 0;
            uint32_t g1_blk = 0, g1_itn = 0;
            auto g1_norm = [&](void) -> bool {  // advance to a valid (item, block); false at the end
                while (g1_item < iend) {
                    if (kQ * g1_bc < g1_nch) return true;
                    g1_item += istep;
                    g1_bc = 0;
                    ++g1_itn;
                    if (g1_item < iend) g1_nch = src.view(g1_item).nch;
                }
                return false;
            };
            auto g1_ready = [&](void) -> bool {  // inputs of the next GEMM1 present (no waiting)
                const int x = g1_blk % kXr, b = g1_blk % kSBufs;
                if (!bar_test(&rfull[x], (g1_blk / kXr) & 1u)) return false;
                if (g1_bc == 0 && !bar_test(&xfull[g1_itn & 1], (g1_itn >> 1) & 1u)) return false;
                return g1_blk < (uint32_t)kSBufs || bar_test(&sempty[b], (g1_blk / kSBufs - 1) & 1u);
            };
            auto issue_gemm1 = [&](void) -> bool {
                const int x = g1_blk % kXr, b = g1_blk % kSBufs, xb = g1_itn & 1;
                if (!bar_wait(&rfull[x], g1_blk / kXr, abort_flag, err)) return false;
                if (g1_bc == 0 && !bar_wait(&xfull[xb], g1_itn >> 1, abort_flag, err)) return false;
                if (!slot_wait(&sempty[b], g1_blk / kSBufs, abort_flag, err)) return false;
                tc_fence_after();
                const uint32_t xr = su32(xr0 + (size_t)x * kXrBytes);
                gemm1(tS(b), tX(xb), xr, xr + kXrHalf);
                mma_commit(&sfull[b]);
                mma_commit(&rempty[x]);
                if (kQ * (g1_bc + 1) >= g1_nch) mma_commit(&xempty[xb]);
                ++g1_bc;
                ++g1_blk;
                return true;
            };
            for (int item = ibeg; item < iend && ok; item += istep, ++itn) {
                const TcView it = src.view(item);
                const int ab = itn % kAccBufs;
                for (int c = 0; c < it.nch && ok; ++c, ++fill) {
                    if (c > 0 && c % kQ == 0) ++cur_blk;
                    // the S block of this chunk has to be in before its epilogue can finish
                    while (ok && g1_blk <= cur_blk && g1_norm()) ok = issue_gemm1();
                    if (!ok) break;
                    const int s = fill % kStages;
                    if (!bar_wait(&full[s], fill / kStages, abort_flag, err) ||
                        !bar_wait(&lamr[s], fill / kStages, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    if (c == 0 && !slot_wait(&aempty[ab], itn / kAccBufs, abort_flag, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = su32(stage0 + (size_t)s * kStageBytes);
                    // A operand (hi, lo): lambda^k in P and its TF32 low part in Q, or in delta form
                    // the change of lambda in Q and its low part in the chunk's group's DLO slot
                    if (it.delta) {
                        const int slot = kDloBufs * (c & 1) + (int)(dlo_n[c & 1]++ % kDloBufs);
                        gemm2_delta(tA(ab), st + kOffQ, tD(slot), st + kOffXT, c > 0);
                        mma_commit(&dloe[slot]);
                    } else {
                        gemm2(tA(ab), st + kOffP, st + kOffQ, st + kOffXT, c > 0);
                    }
                    mma_commit(&empty[s]);
                    if (c == it.nch - 1) mma_commit(&afull[ab]);
                    // then the next block's GEMM1 as soon as its inputs are there: it runs ahead
                    // of the epilogue, queued behind this GEMM2 rather than in front of it
                    if (g1_blk == cur_blk + 1 && g1_norm() && g1_ready()) ok = issue_gemm1();
                }
                ++cur_blk;  // the next item starts a new block
            }
            mma_commit(fin);
            const uint64_t t0 = gtimer();
            while (!bar_try(fin, 0) && gtimer() - t0 < 500000000ull) {
            }
        }
    } else if (warp == kColWarp) {
        // ---------------------------------------------------------------- column sums
        // once the epilogue has written a chunk's tiles: the sums over the block's rows of each
        // column of the new tile (lambda^k, or its change in delta form; rows past the last
        // count as zero), in a fixed order: per lane quarter q, lane = (row group rg of 8 rows,
        // column group g of 4 columns) sums its 8 rows, a butterfly adds the four row groups,
        // and the quarters are added in order
        uint32_t fill = 0;
        bool ok = true;
        const int g = lane & 7, rg = lane >> 3;
        for (int item = ibeg; item < iend && ok; item += istep) {
            const TcView it = src.view(item);
            const int vrows = min(kM, it.row_end - it.i0);  // rows of the block that exist
            for (int c = 0; c < it.nch; ++c, ++fill) {
                const int s = fill % kStages;
                ok = __all_sync(0xffffffffu, bar_wait(&lamr[s], fill / kStages, abort_flag, err));
                if (!ok) break;
                const unsigned char *st = stage0 + (size_t)s * kStageBytes;
                // lambda^k of the 128 rows goes out at once (rows past the buffer's last are clipped)
                if (lane == 0) tma_store(it.R, st + kOffP, (int)(it.c0 + (long long)c * kC), it.i0 - it.row0);
                const float *Red = reinterpret_cast<const float *>(st + (it.delta ? kOffQ : kOffP));
                // the four quarters side by side (independent chains), each in row order
                float2 ca[4], cb[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) ca[q] = cb[q] = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int rr = 32 * q + 8 * rg + t;
                        const float4 x = rr < vrows ? *reinterpret_cast<const float4 *>(Red + rr * 32 + ((g ^ (rr & 7)) << 2))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                        ca[q] = __fadd2_rn(ca[q], make_float2(x.x, x.y));
                        cb[q] = __fadd2_rn(cb[q], make_float2(x.z, x.w));
                    }
                }
                // the tile has been read (the arrive orders this warp's loads before it) and so,
                // once waited for, has the store: the stage may be refilled while the sums are
                // finished
                __syncwarp();
                if (lane == 0) {
                    tma_store_wait_read();
                    bar_arrive(&empty[s]);
                }
#pragma unroll
                for (int o = 8; o <= 16; o <<= 1) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 oa = make_float2(__shfl_xor_sync(0xffffffffu, ca[q].x, o), __shfl_xor_sync(0xffffffffu, ca[q].y, o));
                        const float2 ob = make_float2(__shfl_xor_sync(0xffffffffu, cb[q].x, o), __shfl_xor_sync(0xffffffffu, cb[q].y, o));
                        ca[q] = __fadd2_rn(ca[q], oa);
                        cb[q] = __fadd2_rn(cb[q], ob);
                    }
                }
                const float2 ta = __fadd2_rn(__fadd2_rn(__fadd2_rn(ca[0], ca[1]), ca[2]), ca[3]);
                const float2 tb = __fadd2_rn(__fadd2_rn(__fadd2_rn(cb[0], cb[1]), cb[2]), cb[3]);
                if (rg == 0 && !*abort_flag) {
                    const long long j = it.c0 + (long long)c * kC + 4 * g;
                    float *dst = it.colpart + (long long)it.rb * it.ld + j;
                    const float cv[4] = {ta.x, ta.y, tb.x, tb.y};
                    if (j + 4 <= it.c1) {
                        *reinterpret_cast<float4 *>(dst) = make_float4(cv[0], cv[1], cv[2], cv[3]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j + e < it.c1) dst[e] = cv[e];
                    }
                }
            }
        }
        if (lane == 0) tma_store_wait_all();
    } else {
        // ---------------------------------------------------------------- epilogue
        const int q = warp & 3;                 // tensor-memory lane quarter of this warp
        const int h = (warp - 2) >> 2;          // group: takes the chunks of parity h in an item
        const int r = 32 * q + lane;            // row within the item
        const uint32_t lq = (uint32_t)(32 * q) << 16;
        // the first group copies the xi rows (hi, lo) of an item into tensor-memory buffer
        // xitn & 1, once the GEMM1s of the item that used that buffer before are done
        auto put_xi = [&](int item, uint32_t xitn) -> bool {
            const int xb = xitn & 1;
            const bool ok = __all_sync(0xffffffffu, slot_wait(&xempty[xb], xitn >> 1, abort_flag, err));
            if (ok) {
                const TcView xv = src.view(item);
                const long long row = (long long)xv.i0 + r;  // < ldv
                const float4 *hi = reinterpret_cast<const float4 *>(xv.xi_rm + row * 32);
                const float4 *lo = reinterpret_cast<const float4 *>(xv.xi_rm + xv.ldv * 32 + row * 32);
                float v[32];
                tc_fence_after();
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float4 w = __ldg(hi + t);
                    v[4 * t] = w.x, v[4 * t + 1] = w.y, v[4 * t + 2] = w.z, v[4 * t + 3] = w.w;
                }
                tmem_st32(tX(xb) + lq, v);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float4 w = __ldg(lo + t);
                    v[4 * t] = w.x, v[4 * t + 1] = w.y, v[4 * t + 2] = w.z, v[4 * t + 3] = w.w;
                }
                tmem_st32(tX(xb) + 32u + lq, v);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&xfull[xb]);
            return ok;
        };
        uint32_t fill = 0, itn = 0, blk = 0, dlo_use = 0;
        bool ok = true;
        if (h == 0 && ibeg < iend) ok = put_xi(ibeg, 0);
        for (int item = ibeg; item < iend; item += istep, ++itn) {
            const TcView it = src.view(item);
            const int ab = itn % kAccBufs;
            const int i = it.i0 + r;
            const bool rv = i < it.row_end;
            const float2 beta2 = make_float2((float)it.st->beta, (float)it.st->beta);
            const float2 s2 = make_float2((float)it.st->s, (float)it.st->s);
            // xi rows of the next item go into the other tensor-memory buffer now, so that
            // GEMM1 can run ahead across the item boundary
            if (h == 0 && item + istep < iend) ok = put_xi(item + istep, itn + 1) && ok;
            const float uh = it.u[i], ul = it.u[it.ldv + i];  // i < ldv
            const float2 uh2 = make_float2(uh, uh), ul2 = make_float2(ul, ul);
            float dsum = 0.f;  // this thread's part of the row's ||lambda^k - lambda~^k||^2
            for (int c = 0; c < it.nch; ++c, ++fill) {
                if (c > 0 && c % kQ == 0) ++blk;
                if ((c & 1) != h) continue;  // the other group's chunk
                const int s = fill % kStages, b = blk % kSBufs;
                const long long j0 = it.c0 + (long long)c * kC;
                unsigned char *st = stage0 + (size_t)s * kStageBytes;
                ok = ok && bar_wait(&full[s], fill / kStages, abort_flag, err);
                ok = ok && bar_wait(&sfull[b], blk / kSBufs, abort_flag, err);
                ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
                float v[kC];
                tc_fence_after();
                if (ok) tmem_ld32(tS(b) + 32u * (uint32_t)(c % kQ) + lq, v);  // S, row r, this chunk's columns
                tc_fence_before();
                __syncwarp();
                // the last chunk of an item also stands in for the missing chunks of its block
                if (lane == 0) bar_arrive_n(&sempty[b], c + 1 < it.nch ? 1u : (uint32_t)(kQ - c % kQ));
                float *P = reinterpret_cast<float *>(st + kOffP);
                float *Qs = reinterpret_cast<float *>(st + kOffQ);
                int dslot = 0;
                if (it.delta) {
                    // the group's next DLO slot is free once the GEMM2 of the chunk that used it last is done
                    dslot = kDloBufs * h + (int)(dlo_use % kDloBufs);
                    ok = __all_sync(0xffffffffu, ok && slot_wait(&dloe[dslot], dlo_use / kDloBufs, abort_flag, err));
                    ++dlo_use;
                }
                if (ok) {
                    const float *Y = reinterpret_cast<const float *>(y0 + (size_t)s * kYBytes);
                    // the checks of the diagonal and of padding columns; rows past the last
                    // (a partial last block) need none: their values are neither stored (the
                    // maps clip them), nor summed by columns (warp 11 masks them), nor kept in
                    // the row partials
                    const bool edge = (j0 < (long long)it.i0 + kM && j0 + kC > it.i0) || (j0 + kC > it.N);
                    // each half of the row at a time; in delta form the half's low parts go to
                    // this warp's lane quarter of the group's DLO slot right away
#define CR_EPI(E, A, D)                                                                                \
    do {                                                                                               \
        float dlo[kC / 2];                                                                             \
        epi_half<E, A, D, 0>(P, Qs, Y, v, r, uh2, ul2, beta2, s2, rv, i, j0, it.N, dsum, dlo);         \
        if (D) {                                                                                       \
            tc_fence_after();                                                                          \
            tmem_st16(tD(dslot) + lq, dlo);                                                            \
        }                                                                                              \
        epi_half<E, A, D, 1>(P, Qs, Y, v, r, uh2, ul2, beta2, s2, rv, i, j0, it.N, dsum, dlo);         \
        if (D) {                                                                                       \
            tmem_st16(tD(dslot) + lq + 16u, dlo);                                                      \
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");                               \
        }                                                                                              \
    } while (0)
                    if (it.delta) {
                        if (it.adaptive) {
                            if (edge) CR_EPI(true, true, true); else CR_EPI(false, true, true);
                        } else {
                            if (edge) CR_EPI(true, false, true); else CR_EPI(false, false, true);
                        }
                    } else if (it.adaptive) {
                        if (edge) CR_EPI(true, true, false); else CR_EPI(false, true, false);
                    } else {
                        if (edge) CR_EPI(true, false, false); else CR_EPI(false, false, false);
                    }
#undef CR_EPI
                    fence_async_smem();  // make the tiles visible to the tensor cores and the TMA store
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&lamr[s]);  // the store and the column sums are warp 11's
            }
            ++blk;  // the next item starts a new block
            // end of item: row partials from the GEMM2 accumulator: columns k < n of the two
            // halves give sum_j lambda_ij x_jk, column n of the first gives sum_j lambda_ij;
            // this group reads columns [16 h, 16 h + 16) of both halves
            const bool ok2 = __all_sync(0xffffffffu, ok && bar_wait(&afull[ab], itn / kAccBufs, abort_flag, err));
            float acc[kHalf], acl[kHalf];
            tc_fence_after();
            if (ok2) {
                tmem_ld16(tA(ab) + lq + (uint32_t)(kHalf * h), acc);
                tmem_ld16(tA(ab) + lq + 32u + (uint32_t)(kHalf * h), acl);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&aempty[ab]);
            if (it.adaptive && ok && rv) it.dpart[((long long)it.sp * 2 + h) * it.N + i] = dsum;
            if (ok2 && rv) {
                float *dst = it.rowpart + ((long long)it.sp * it.N + i) * (it.NP + 1);
#pragma unroll
                for (int e = 0; e < kHalf; ++e) {
                    const int k = kHalf * h + e;
                    if (k < it.n) dst[k] = acc[e] + acl[e];
                    if (k == it.n) dst[it.NP] = acc[e];
                }
            }
            ok = ok && ok2;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    sweep_tc_kernel(const __grid_constant__ CUtensorMap tmXRh, const __grid_constant__ CUtensorMap tmXRl,
                    const __grid_constant__ CUtensorMap tmXT, const __grid_constant__ CUtensorMap tmY,
                    const TcSweepArgs a) {
    const TcSrcSingle src{&tmXRh, &tmXRl, &tmXT, &tmY, &a};
    sweep_tc_body(src, a.err);
}

__global__ void __launch_bounds__(kThreads, 1)
    sweep_tc_batch_kernel(const InstDesc *d, const WorkItem *w, int nitems, int *err) {
    const TcSrcBatch src{d, w, nitems};
    sweep_tc_body(src, err);
}

}  // namespace

size_t sweep_tc_smem() { return kSmem; }
int sweep_tc_rows() { return kM; }

cudaError_t sweep_tc_occupancy(int *blocks_per_sm) {
    // the large shared-memory attribute is per device: set it once on each, under a lock
    static std::mutex mu;
    static bool attr[kTcDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kTcDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(sweep_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_tc_kernel, kThreads, kSmem);
}

cudaError_t launch_sweep_tc(const TcMaps &m, const TcSweepArgs &a, int grid, cudaStream_t s) {
    int occ = 0;
    cudaError_t e = sweep_tc_occupancy(&occ);
    if (e != cudaSuccess) return e;
    sweep_tc_kernel<<<grid, kThreads, kSmem, s>>>(m.XRh, m.XRl, m.XT, m.Y, a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_tc_batch(const InstDesc *d, const WorkItem *w, int nitems, int *err, int grid,
                                  cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static bool attr[kTcDevices] = {};
    if (dev < 0 || dev >= kTcDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!attr[dev]) {
            e = cudaFuncSetAttribute(sweep_tc_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    sweep_tc_batch_kernel<<<grid, kThreads, kSmem, s>>>(d, w, nitems, err);
    return cudaGetLastError();
}

}  // namespace cr
