// cr_sweep.cu -- the fused Lambda sweep (Steps 2 and 4 of Figure "papg" with K = N,
// plus the reductions of C^T lambda^k that Step 1 of the next iteration needs).
//
// One pass reads lambda^{k-1} (P) and lambda^{k-2} (Q) once and writes lambda^k over Q
// once (12 B per pair in FP32, 24 B in FP64).  For every pair (i, j), i != j:
//     lambda~   = P_ij + beta_k (P_ij - Q_ij)                       (Step 4 of k-1)
//     rho_ij    = u_i - y_j + xi_i . x_j,  u_i = y_i - xi_i . x_i    (-(C eta(lambda~))_ij)
//     lambda^k  = max(0, lambda~ + rho_ij / L)                       (Step 2)
// and the same pass accumulates, for C^T lambda^k (Definition 1):
//     row sums   r_i = sum_j lambda_ij,  B_i = sum_j lambda_ij x_j   (per column split)
//     column sums c_j = sum_i lambda_ij                               (per row block)
//
// Work decomposition: a work item is ROWS rows of Lambda times one column split; the
// CTA walks its split in chunks of 128 columns.  Warp w owns MR consecutive rows, lane l
// owns 4 consecutive columns of each chunk, so every warp load/store of Lambda is a
// fully coalesced 512 B (FP32) row segment issued as 128-bit accesses.  xi_i of the
// ROWS rows sits in shared memory for the whole item and B_i, r_i in registers; x_j
// and y_j of a chunk are staged in shared memory once and reused by all rows.  Column
// sums are reduced across warps through shared memory once per chunk and written as
// one partial per (row block, column); row sums are reduced across lanes once per item.
// Every reduction has a fixed order, so results are bitwise reproducible.
#include "cr_internal.cuh"

namespace cr {
namespace {

__device__ __forceinline__ float4 ld_stream4(const float *p) { return __ldcs((const float4 *)p); }
__device__ __forceinline__ void st_stream4(float *p, float4 v) { __stcs((float4 *)p, v); }
__device__ __forceinline__ double2 ld_stream2(const double *p) { return __ldcs((const double2 *)p); }
__device__ __forceinline__ void st_stream2(double *p, double2 v) { __stcs((double2 *)p, v); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------ FP32 sweep
template <int NP, int MR, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) sweep_f32_kernel(const SweepArgsF a) {
    constexpr int ROWS = MR * WARPS;
    constexpr int NT = WARPS * 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *xs = reinterpret_cast<float *>(smem_raw);  // NP x kChunk
    float *ysh = xs + NP * kChunk;                     // kChunk
    float *ysl = ysh + kChunk;                         // kChunk
    float *cred = ysl + kChunk;                        // 2 x WARPS x kChunk
    float *xis = cred + 2 * WARPS * kChunk;            // NP x ROWS

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float beta = (float)a.st->beta;
    const float s = (float)a.st->s;
    const int items = a.row_blocks * a.col_splits;

    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int rb = item / a.col_splits, sp = item % a.col_splits;
        const int i0 = rb * ROWS;
        const long long c0 = (long long)sp * a.cols_per_split;
        const long long c1 = min(c0 + (long long)a.cols_per_split, a.ld);

        __syncthreads();  // the previous item is done with shared memory
        for (int q = tid; q < NP * ROWS; q += NT) {
            const int k = q / ROWS, r = q - k * ROWS, i = i0 + r;
            xis[q] = (i < a.N) ? a.xiT[(long long)k * a.ldv + i] : 0.f;
        }
        int ir[MR];
        bool rv[MR];
        float uhr[MR], ulr[MR], rs[MR];
        float B[MR][NP];
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            ir[r] = i0 + warp * MR + r;
            rv[r] = ir[r] < a.N;
            uhr[r] = rv[r] ? a.uh[ir[r]] : 0.f;
            ulr[r] = rv[r] ? a.ul[ir[r]] : 0.f;
            rs[r] = 0.f;
#pragma unroll
            for (int k = 0; k < NP; ++k) B[r][k] = 0.f;
        }

        int chunk = 0;
        for (long long j0 = c0; j0 < c1; j0 += kChunk, ++chunk) {
            __syncthreads();  // (A) column partials of chunk-1 are in cred; xs is free
            if (chunk > 0 && tid < kChunk) {
                const long long j = j0 - kChunk + tid;
                if (j < c1) {
                    const float *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                    float v = 0.f;
#pragma unroll
                    for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                    a.colpart[(long long)rb * a.ld + j] = v;
                }
            }
            for (int q = tid; q < NP * kChunk; q += NT) {
                const int k = q / kChunk, c = q - k * kChunk;
                const long long j = j0 + c;
                xs[q] = (j < a.ldv) ? a.xT[(long long)k * a.ldv + j] : 0.f;
            }
            if (tid < kChunk) {
                const long long j = j0 + tid;
                ysh[tid] = (j < a.ldv) ? a.yh[j] : 0.f;
                ysl[tid] = (j < a.ldv) ? a.yl[j] : 0.f;
            }
            __syncthreads();  // (B)

            const long long jl = j0 + 4 * lane;
            const bool cv = jl < c1;
            float4 pv[MR], qv[MR];
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                if (rv[r] && cv) {
                    const long long off = (long long)ir[r] * a.ld + jl;
                    pv[r] = ld_stream4(a.P + off);
                    qv[r] = ld_stream4(a.Q + off);
                } else {
                    pv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                    qv[r] = pv[r];
                }
            }
            float d[MR][4];
#pragma unroll
            for (int r = 0; r < MR; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) d[r][c] = 0.f;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float4 xv = *reinterpret_cast<const float4 *>(xs + k * kChunk + 4 * lane);
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    const float xi = xis[k * ROWS + warp * MR + r];
                    d[r][0] = fmaf(xi, xv.x, d[r][0]);
                    d[r][1] = fmaf(xi, xv.y, d[r][1]);
                    d[r][2] = fmaf(xi, xv.z, d[r][2]);
                    d[r][3] = fmaf(xi, xv.w, d[r][3]);
                }
            }
            const float4 yhv = *reinterpret_cast<const float4 *>(ysh + 4 * lane);
            const float4 ylv = *reinterpret_cast<const float4 *>(ysl + 4 * lane);
            const float yh4[4] = {yhv.x, yhv.y, yhv.z, yhv.w};
            const float yl4[4] = {ylv.x, ylv.y, ylv.z, ylv.w};
            float lam[MR][4];
            float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                const float p4[4] = {pv[r].x, pv[r].y, pv[r].z, pv[r].w};
                const float q4[4] = {qv[r].x, qv[r].y, qv[r].z, qv[r].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float rho = ((uhr[r] - yh4[c]) + (ulr[r] - yl4[c])) + d[r][c];
                    const float lt = fmaf(beta, p4[c] - q4[c], p4[c]);
                    float l = fmaxf(0.f, fmaf(s, rho, lt));
                    const long long j = jl + c;
                    if (!rv[r] || !cv || j == ir[r] || j >= a.N) l = 0.f;
                    lam[r][c] = l;
                    rs[r] += l;
                    cs[c] += l;
                }
                if (rv[r] && cv)
                    st_stream4(a.Q + (long long)ir[r] * a.ld + jl,
                               make_float4(lam[r][0], lam[r][1], lam[r][2], lam[r][3]));
            }
            *reinterpret_cast<float4 *>(cred + ((chunk & 1) * WARPS + warp) * kChunk + 4 * lane) =
                make_float4(cs[0], cs[1], cs[2], cs[3]);
            // re-read x_j from shared memory below instead of keeping 4 x NP values live
            asm volatile("" ::: "memory");
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float4 xv = *reinterpret_cast<const float4 *>(xs + k * kChunk + 4 * lane);
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    float v = B[r][k];
                    v = fmaf(lam[r][0], xv.x, v);
                    v = fmaf(lam[r][1], xv.y, v);
                    v = fmaf(lam[r][2], xv.z, v);
                    v = fmaf(lam[r][3], xv.w, v);
                    B[r][k] = v;
                }
            }
        }
        __syncthreads();
        if (chunk > 0 && tid < kChunk) {
            const long long j = c0 + (long long)(chunk - 1) * kChunk + tid;
            if (j < c1) {
                const float *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                float v = 0.f;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                a.colpart[(long long)rb * a.ld + j] = v;
            }
        }
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            float *dst = a.rowpart + ((long long)sp * a.N + ir[r]) * (NP + 1);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float v = warp_sum(B[r][k]);
                if (lane == 0 && rv[r]) dst[k] = v;
            }
            const float v = warp_sum(rs[r]);
            if (lane == 0 && rv[r]) dst[NP] = v;
        }
    }
}

// ------------------------------------------------------------------ FP64 sweep
template <int NP, int MR, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) sweep_f64_kernel(const SweepArgsD a) {
    constexpr int ROWS = MR * WARPS;
    constexpr int NT = WARPS * 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *xs = reinterpret_cast<double *>(smem_raw);  // NP x kChunk
    double *ys = xs + NP * kChunk;                       // kChunk
    double *cred = ys + kChunk;                          // 2 x WARPS x kChunk
    double *xis = cred + 2 * WARPS * kChunk;             // NP x ROWS

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double beta = a.st->beta;
    const double s = a.st->s;
    const int items = a.row_blocks * a.col_splits;
    // buffer roles: lambda^{k-1} (Pp), lambda^{k-2} (Qp), output (Rp)
    const double *Pp = a.P, *Qp = a.Q;
    double *Rp = a.Q;
    if (a.adaptive) {
        int ip, iq, ir;
        lam_roles(a.st, 1, 0, &ip, &iq, &ir);
        Pp = a.B[ip];
        Qp = a.B[iq];
        Rp = a.B[ir];
    }

    // a shard holds rows [row0, row_end) of Lambda from its row 0 on (row_end = N, row0 = 0 for a
    // whole instance); rows are global everywhere else
    const long long rbase = (long long)a.row0 * a.ld;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int rb = item / a.col_splits, sp = item % a.col_splits;
        const int i0 = a.row0 + rb * ROWS;
        const long long c0 = (long long)sp * a.cols_per_split;
        const long long c1 = min(c0 + (long long)a.cols_per_split, a.ld);

        __syncthreads();
        for (int q = tid; q < NP * ROWS; q += NT) {
            const int k = q / ROWS, r = q - k * ROWS, i = i0 + r;
            xis[q] = (i < a.row_end) ? a.xiT[(long long)k * a.ldv + i] : 0.0;
        }
        int ir[MR];
        bool rv[MR];
        double ur[MR], rs[MR], dd[MR];
        double B[MR][NP];
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            ir[r] = i0 + warp * MR + r;
            rv[r] = ir[r] < a.row_end;
            ur[r] = rv[r] ? a.u[ir[r]] : 0.0;
            rs[r] = 0.0;
            dd[r] = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) B[r][k] = 0.0;
        }

        int chunk = 0;
        for (long long j0 = c0; j0 < c1; j0 += kChunk, ++chunk) {
            __syncthreads();
            if (chunk > 0 && tid < kChunk) {
                const long long j = j0 - kChunk + tid;
                if (j < c1) {
                    const double *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                    double v = 0.0;
#pragma unroll
                    for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                    a.colpart[(long long)rb * a.ld + j] = v;
                }
            }
            for (int q = tid; q < NP * kChunk; q += NT) {
                const int k = q / kChunk, c = q - k * kChunk;
                const long long j = j0 + c;
                xs[q] = (j < a.ldv) ? a.xT[(long long)k * a.ldv + j] : 0.0;
            }
            if (tid < kChunk) {
                const long long j = j0 + tid;
                ys[tid] = (j < a.ldv) ? a.y[j] : 0.0;
            }
            __syncthreads();

            const long long jl = j0 + 4 * lane;
            const bool cv = jl < c1;
            double p4[MR][4], q4[MR][4];
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                if (rv[r] && cv) {
                    const long long off = (long long)ir[r] * a.ld + jl - rbase;
                    const double2 p01 = ld_stream2(Pp + off), p23 = ld_stream2(Pp + off + 2);
                    const double2 q01 = ld_stream2(Qp + off), q23 = ld_stream2(Qp + off + 2);
                    p4[r][0] = p01.x; p4[r][1] = p01.y; p4[r][2] = p23.x; p4[r][3] = p23.y;
                    q4[r][0] = q01.x; q4[r][1] = q01.y; q4[r][2] = q23.x; q4[r][3] = q23.y;
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) p4[r][c] = q4[r][c] = 0.0;
                }
            }
            double d[MR][4];
#pragma unroll
            for (int r = 0; r < MR; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) d[r][c] = 0.0;
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const double2 x01 = *reinterpret_cast<const double2 *>(xs + k * kChunk + 4 * lane);
                const double2 x23 = *reinterpret_cast<const double2 *>(xs + k * kChunk + 4 * lane + 2);
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    const double xi = xis[k * ROWS + warp * MR + r];
                    d[r][0] = fma(xi, x01.x, d[r][0]);
                    d[r][1] = fma(xi, x01.y, d[r][1]);
                    d[r][2] = fma(xi, x23.x, d[r][2]);
                    d[r][3] = fma(xi, x23.y, d[r][3]);
                }
            }
            const double2 y01 = *reinterpret_cast<const double2 *>(ys + 4 * lane);
            const double2 y23 = *reinterpret_cast<const double2 *>(ys + 4 * lane + 2);
            const double y4[4] = {y01.x, y01.y, y23.x, y23.y};
            double lam[MR][4];
            double cs[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int r = 0; r < MR; ++r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double rho = (ur[r] - y4[c]) + d[r][c];
                    const double lt = fma(beta, p4[r][c] - q4[r][c], p4[r][c]);
                    double l = fmax(0.0, fma(s, rho, lt));
                    const long long j = jl + c;
                    if (!rv[r] || !cv || j == ir[r] || j >= a.N) l = 0.0;
                    lam[r][c] = l;
                    rs[r] += l;
                    cs[c] += l;
                    dd[r] = fma(l - lt, l - lt, dd[r]);  // ||lambda^k - lambda~^k||^2 (adaptive step)
                }
                if (rv[r] && cv) {
                    const long long off = (long long)ir[r] * a.ld + jl - rbase;
                    st_stream2(Rp + off, make_double2(lam[r][0], lam[r][1]));
                    st_stream2(Rp + off + 2, make_double2(lam[r][2], lam[r][3]));
                }
            }
            double *cw = cred + ((chunk & 1) * WARPS + warp) * kChunk + 4 * lane;
            *reinterpret_cast<double2 *>(cw) = make_double2(cs[0], cs[1]);
            *reinterpret_cast<double2 *>(cw + 2) = make_double2(cs[2], cs[3]);
            asm volatile("" ::: "memory");
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const double2 x01 = *reinterpret_cast<const double2 *>(xs + k * kChunk + 4 * lane);
                const double2 x23 = *reinterpret_cast<const double2 *>(xs + k * kChunk + 4 * lane + 2);
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    double v = B[r][k];
                    v = fma(lam[r][0], x01.x, v);
                    v = fma(lam[r][1], x01.y, v);
                    v = fma(lam[r][2], x23.x, v);
                    v = fma(lam[r][3], x23.y, v);
                    B[r][k] = v;
                }
            }
        }
        __syncthreads();
        if (chunk > 0 && tid < kChunk) {
            const long long j = c0 + (long long)(chunk - 1) * kChunk + tid;
            if (j < c1) {
                const double *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                a.colpart[(long long)rb * a.ld + j] = v;
            }
        }
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            double *dst = a.rowpart + ((long long)sp * a.N + ir[r]) * (NP + 1);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const double v = warp_sum(B[r][k]);
                if (lane == 0 && rv[r]) dst[k] = v;
            }
            const double v = warp_sum(rs[r]);
            if (lane == 0 && rv[r]) dst[NP] = v;
            if (a.adaptive) {
                const double dv = warp_sum(dd[r]);
                if (lane == 0 && rv[r]) a.dpart[(long long)sp * a.N + ir[r]] = dv;
            }
        }
    }
}

// ------------------------------------------------------------------ dispatch tables
template <int NP>
struct ShapeF {
    // 32 rows per CTA: 4 rows per warp below 14 components, 2 rows per warp above
    static constexpr int MR = NP <= 12 ? 4 : 2;
    static constexpr int WARPS = 32 / MR;
};
template <int NP>
struct ShapeD {
    // 16 rows per CTA (FP64 accumulators take twice the registers)
    static constexpr int MR = NP <= 16 ? 2 : 1;
    static constexpr int WARPS = 16 / MR;
};

template <int NP>
size_t smem_f() {
    using S = ShapeF<NP>;
    return sizeof(float) * (NP * kChunk + 2 * kChunk + 2 * S::WARPS * kChunk + NP * S::MR * S::WARPS);
}
template <int NP>
size_t smem_d() {
    using S = ShapeD<NP>;
    return sizeof(double) * (NP * kChunk + kChunk + 2 * S::WARPS * kChunk + NP * S::MR * S::WARPS);
}

template <int NP>
cudaError_t run_f(const SweepArgsF &a, int grid, cudaStream_t st, int *occ) {
    using S = ShapeF<NP>;
    auto k = sweep_f32_kernel<NP, S::MR, S::WARPS>;
    const size_t sm = smem_f<NP>();
    static bool attr_set = false;  // per process; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, S::WARPS * 32, sm);
    k<<<grid, S::WARPS * 32, sm, st>>>(a);
    return cudaGetLastError();
}

template <int NP>
cudaError_t run_d(const SweepArgsD &a, int grid, cudaStream_t st, int *occ) {
    using S = ShapeD<NP>;
    auto k = sweep_f64_kernel<NP, S::MR, S::WARPS>;
    const size_t sm = smem_d<NP>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, S::WARPS * 32, sm);
    k<<<grid, S::WARPS * 32, sm, st>>>(a);
    return cudaGetLastError();
}

#define CR_NP_LIST(X) X(2) X(4) X(6) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(28) X(32)

cudaError_t dispatch_f(int np, const SweepArgsF *a, int grid, cudaStream_t st, int *occ) {
    SweepArgsF dummy{};
    const SweepArgsF &args = a ? *a : dummy;
    switch (np) {
#define CASE(V) \
    case V: return run_f<V>(args, grid, st, occ);
        CR_NP_LIST(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_d(int np, const SweepArgsD *a, int grid, cudaStream_t st, int *occ) {
    SweepArgsD dummy{};
    const SweepArgsD &args = a ? *a : dummy;
    switch (np) {
#define CASE(V) \
    case V: return run_d<V>(args, grid, st, occ);
        CR_NP_LIST(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool sweep_config_f(int np, SweepConfig *cfg) {
    if (np > 32) return sweep_wide_config(np, false, cfg);
    switch (np) {
#define CASE(V)                                                            \
    case V:                                                                \
        cfg->rows = ShapeF<V>::MR * ShapeF<V>::WARPS;                      \
        cfg->threads = ShapeF<V>::WARPS * 32;                              \
        cfg->smem = smem_f<V>();                                           \
        return true;
        CR_NP_LIST(CASE)
#undef CASE
        default: return false;
    }
}

bool sweep_config_d(int np, SweepConfig *cfg) {
    if (np > 32) return sweep_wide_config(np, true, cfg);
    switch (np) {
#define CASE(V)                                                            \
    case V:                                                                \
        cfg->rows = ShapeD<V>::MR * ShapeD<V>::WARPS;                      \
        cfg->threads = ShapeD<V>::WARPS * 32;                              \
        cfg->smem = smem_d<V>();                                           \
        return true;
        CR_NP_LIST(CASE)
#undef CASE
        default: return false;
    }
}

cudaError_t launch_sweep_f(int np, const SweepArgsF &a, int grid, cudaStream_t s) {
    if (np > 32) return launch_sweep_wide_f(np, a, grid, s);
    return dispatch_f(np, &a, grid, s, nullptr);
}
cudaError_t launch_sweep_d(int np, const SweepArgsD &a, int grid, cudaStream_t s) {
    if (np > 32) return launch_sweep_wide_d(np, a, grid, s);
    return dispatch_d(np, &a, grid, s, nullptr);
}
cudaError_t sweep_occupancy_f(int np, int *blocks_per_sm) {
    if (np > 32) return sweep_wide_occupancy(np, false, false, blocks_per_sm);
    return dispatch_f(np, nullptr, 0, 0, blocks_per_sm);
}
cudaError_t sweep_occupancy_d(int np, int *blocks_per_sm) {
    if (np > 32) return sweep_wide_occupancy(np, true, false, blocks_per_sm);
    return dispatch_d(np, nullptr, 0, 0, blocks_per_sm);
}

}  // namespace cr
