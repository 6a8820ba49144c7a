// cr_sweep_wide.cu -- the fused Lambda sweep (Steps 2 and 4 of Figure "papg", K = N) for
// wide points, 32 < n <= CR_MAX_N, in FP32 or FP64, constant or adaptive step.
//
// Same per-pair arithmetic and the same partial sums as cr_sweep.cu:
//     lambda~ = P + beta (P - Q),  rho = u_i - y_j + xi_i . x_j,  lambda = max(0, lambda~ + s rho)
//     rowpart[sp][i] = (sum_j lambda_ij x_j, sum_j lambda_ij),  colpart[rb][j] = sum_i lambda_ij
// (the paper's Section 5 workloads have n = 80).  What changes is where the n-long vectors
// live: the narrow kernels keep B_i = sum_j lambda_ij x_j as n per-lane partials in registers,
// which does not fit for n up to 128 in FP64.  Here a lane owns the strided columns
// c = lane + 32 q of a 128-column chunk while it forms rho and lambda, writes its lambda to
// shared memory, and then owns the components k = lane + 32 m while it accumulates
// B_i[k] += sum_c lambda_ic x_ck over the chunk; B_i needs ceil(n/32) registers per row and
// no cross-lane reduction.  x of the chunk sits in shared memory k-major with an odd row
// stride (kChunk + 1), so both access patterns (consecutive c, consecutive k across the
// warp) are free of bank conflicts; xi of the CTA's rows and lambda of the chunk are read
// as 16-byte broadcasts of the warp's MR rows.  Every sum has a fixed order.
#include <type_traits>

#include "cr_internal.cuh"

namespace cr {
namespace {

template <typename T>
struct WideArgs {
    const T *P;
    T *Q;
    T *B[3];
    int adaptive;
    T *dpart;
    long long ld;
    int N, NP;
    int row_blocks, col_splits, cols_per_split;
    long long ldv;
    const T *xT, *xiT;
    const T *y0, *y1;  // FP32: y hi, y lo; FP64: y, unused
    const T *u0, *u1;  // FP32: u hi, u lo; FP64: u, unused
    const DevState *st;
    T *rowpart, *colpart;
};

template <typename T>
struct WideShape;
template <>
struct WideShape<float> {
    static constexpr int MR = 4, WARPS = 8;
};
template <>
struct WideShape<double> {
    static constexpr int MR = 2, WARPS = 8;
};

constexpr int kStride = kChunk + 1;  // odd: conflict-free by column and by component

template <typename T>
size_t wide_smem(int NP) {
    using S = WideShape<T>;
    const int rows = S::MR * S::WARPS;
    return sizeof(T) * ((size_t)NP * kStride + (size_t)kChunk * rows + 2 * (size_t)S::WARPS * kChunk +
                        (size_t)NP * rows + 2 * kChunk);
}

// MR consecutive values of type T as one 16-byte vector (MR * sizeof(T) == 16)
template <typename T, int MR>
struct Vec16;
template <>
struct Vec16<float, 4> {
    using V = float4;
    static __device__ __forceinline__ void get(const float *p, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void put(float *p, const float (&o)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <>
struct Vec16<double, 2> {
    static __device__ __forceinline__ void get(const double *p, double (&o)[2]) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void put(double *p, const double (&o)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]);
    }
};

__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int M, bool ADAPT>
__global__ void __launch_bounds__(WideShape<T>::WARPS * 32) sweep_wide_kernel(const WideArgs<T> a) {
    using S = WideShape<T>;
    constexpr int MR = S::MR, WARPS = S::WARPS, ROWS = MR * WARPS, NT = WARPS * 32;
    constexpr bool F32 = std::is_same<T, float>::value;
    static_assert(MR * sizeof(T) == 16, "one 16-byte vector per warp row group");
    const int NP = a.NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);   // [NP][kStride]   x_j of the chunk, k-major
    T *lsh = xs + (size_t)NP * kStride;          // [kChunk][ROWS]  lambda^k of the chunk
    T *cred = lsh + (size_t)kChunk * ROWS;       // [2][WARPS][kChunk] column partials
    T *xis = cred + 2 * WARPS * kChunk;          // [NP][ROWS]      xi_i of the item's rows
    T *ysh = xis + (size_t)NP * ROWS;            // [2][kChunk]     y_j (FP32: hi, lo)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T beta = (T)a.st->beta;
    const T s = (T)a.st->s;
    const int items = a.row_blocks * a.col_splits;
    // buffer roles: lambda^{k-1} (Pp), lambda^{k-2} (Qp), output (Rp)
    const T *Pp = a.P, *Qp = a.Q;
    T *Rp = a.Q;
    if (ADAPT) {
        int ip, iq, ir;
        lam_roles(a.st, 1, 0, &ip, &iq, &ir);
        Pp = ip == 0 ? a.B[0] : (ip == 1 ? a.B[1] : a.B[2]);  // no dynamic index into the parameters
        Qp = iq == 0 ? a.B[0] : (iq == 1 ? a.B[1] : a.B[2]);
        Rp = ir == 0 ? a.B[0] : (ir == 1 ? a.B[1] : a.B[2]);
    }

    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int rb = item / a.col_splits, sp = item % a.col_splits;
        const int i0 = rb * ROWS;
        const long long c0 = (long long)sp * a.cols_per_split;
        const long long c1 = min(c0 + (long long)a.cols_per_split, a.ld);

        __syncthreads();  // the previous item is done with shared memory
        for (int q = tid; q < NP * ROWS; q += NT) {
            const int k = q / ROWS, r = q - k * ROWS, i = i0 + r;
            xis[q] = (i < a.N) ? a.xiT[(long long)k * a.ldv + i] : (T)0;
        }
        int ir[MR];
        bool rv[MR];
        T u0r[MR], u1r[MR], rs[MR], dd[MR];
        T B[MR][M];
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            ir[r] = i0 + warp * MR + r;
            rv[r] = ir[r] < a.N;
            u0r[r] = rv[r] ? a.u0[ir[r]] : (T)0;
            u1r[r] = (F32 && rv[r]) ? a.u1[ir[r]] : (T)0;
            rs[r] = (T)0;
            dd[r] = (T)0;
#pragma unroll
            for (int m = 0; m < M; ++m) B[r][m] = (T)0;
        }

        int chunk = 0;
        for (long long j0 = c0; j0 < c1; j0 += kChunk, ++chunk) {
            __syncthreads();  // (A) column partials of chunk-1 are in cred; xs and lsh are free
            if (chunk > 0 && tid < kChunk) {
                const long long j = j0 - kChunk + tid;
                if (j < c1) {
                    const T *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                    T v = (T)0;
#pragma unroll
                    for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                    a.colpart[(long long)rb * a.ld + j] = v;
                }
            }
            for (int q = tid; q < NP * kChunk; q += NT) {
                const int k = q / kChunk, c = q - k * kChunk;
                const long long j = j0 + c;
                xs[k * kStride + c] = (j < a.ldv) ? a.xT[(long long)k * a.ldv + j] : (T)0;
            }
            if (tid < kChunk) {
                const long long j = j0 + tid;
                ysh[tid] = (j < a.ldv) ? a.y0[j] : (T)0;
                ysh[kChunk + tid] = (F32 && j < a.ldv) ? a.y1[j] : (T)0;
            }
            __syncthreads();  // (B)

            // Lambda of the warp's rows at columns j0 + lane + 32 q (coalesced per q)
            T pv[MR][4], qv[MR][4];
#pragma unroll
            for (int r = 0; r < MR; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long j = j0 + lane + 32 * q;
                    if (rv[r] && j < c1) {
                        const long long off = (long long)ir[r] * a.ld + j;
                        pv[r][q] = __ldcs(Pp + off);
                        qv[r][q] = __ldcs(Qp + off);
                    } else {
                        pv[r][q] = (T)0;
                        qv[r][q] = (T)0;
                    }
                }
            // xi_i . x_j, components in increasing order
            T d[MR][4];
#pragma unroll
            for (int r = 0; r < MR; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) d[r][q] = (T)0;
#pragma unroll 4
            for (int k = 0; k < NP; ++k) {
                T xv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xv[q] = xs[k * kStride + lane + 32 * q];
                T xi[MR];
                Vec16<T, MR>::get(xis + k * ROWS + warp * MR, xi);
#pragma unroll
                for (int r = 0; r < MR; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) d[r][q] = fma_t(xi[r], xv[q], d[r][q]);
            }
            T cs[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = lane + 32 * q;
                const long long j = j0 + c;
                const T yj0 = ysh[c], yj1 = ysh[kChunk + c];
                T lv[MR];
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    const T rho = F32 ? ((u0r[r] - yj0) + (u1r[r] - yj1)) + d[r][q] : (u0r[r] - yj0) + d[r][q];
                    const T lt = fma_t(beta, pv[r][q] - qv[r][q], pv[r][q]);
                    T l = fma_t(s, rho, lt);
                    l = l > (T)0 ? l : (T)0;
                    if (!rv[r] || j >= c1 || j == ir[r] || j >= a.N) l = (T)0;
                    if (ADAPT) {
                        // FP32: s rho where the step is not clipped (no cancellation); FP64: l - lt
                        T e;
                        if (F32)
                            e = l > (T)0 ? s * rho : -lt;
                        else
                            e = l - lt;
                        if (!rv[r] || j >= c1 || j == ir[r] || j >= a.N) e = (T)0;
                        dd[r] = fma_t(e, e, dd[r]);
                    }
                    lv[r] = l;
                    rs[r] += l;
                    cs[q] += l;
                    if (rv[r] && j < c1) __stcs(Rp + (long long)ir[r] * a.ld + j, l);
                }
                Vec16<T, MR>::put(lsh + c * ROWS + warp * MR, lv);
                cred[((chunk & 1) * WARPS + warp) * kChunk + c] = cs[q];
            }
            __syncwarp();
            // B_i[k] += sum_c lambda_ic x_ck, k = lane + 32 m, columns in increasing order
#pragma unroll 2
            for (int c = 0; c < kChunk; ++c) {
                T lr[MR];
                Vec16<T, MR>::get(lsh + c * ROWS + warp * MR, lr);
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int k = lane + 32 * m;
                    const T xk = (k < NP) ? xs[k * kStride + c] : (T)0;
#pragma unroll
                    for (int r = 0; r < MR; ++r) B[r][m] = fma_t(lr[r], xk, B[r][m]);
                }
            }
        }
        __syncthreads();
        if (chunk > 0 && tid < kChunk) {
            const long long j = c0 + (long long)(chunk - 1) * kChunk + tid;
            if (j < c1) {
                const T *cb = cred + ((chunk - 1) & 1) * WARPS * kChunk + tid;
                T v = (T)0;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) v += cb[w * kChunk];
                a.colpart[(long long)rb * a.ld + j] = v;
            }
        }
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            T *dst = a.rowpart + ((long long)sp * a.N + ir[r]) * (NP + 1);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int k = lane + 32 * m;
                if (rv[r] && k < NP) dst[k] = B[r][m];
            }
            const T v = warp_sum_t(rs[r]);
            if (lane == 0 && rv[r]) dst[NP] = v;
            if (ADAPT) {
                const T dv = warp_sum_t(dd[r]);
                if (lane == 0 && rv[r]) a.dpart[(long long)sp * a.N + ir[r]] = dv;
            }
        }
    }
}

template <typename T, int M, bool ADAPT>
cudaError_t run_wide(const WideArgs<T> &a, int NP, int grid, cudaStream_t st, int *occ) {
    auto k = sweep_wide_kernel<T, M, ADAPT>;
    const size_t sm = wide_smem<T>(32 * M);  // attribute for the largest NP of this M
    static bool attr_set = false;            // per process; the attribute is per device function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    constexpr int threads = WideShape<T>::WARPS * 32;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, wide_smem<T>(NP));
    k<<<grid, threads, wide_smem<T>(NP), st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_wide(const WideArgs<T> &a, int NP, int grid, cudaStream_t st, int *occ) {
    if (NP <= 32 || NP > CR_MAX_N || NP % 16 != 0) return cudaErrorInvalidValue;
    const int M = (NP + 31) / 32;
    const bool ad = a.adaptive != 0;
    switch (M) {
        case 2: return ad ? run_wide<T, 2, true>(a, NP, grid, st, occ) : run_wide<T, 2, false>(a, NP, grid, st, occ);
        case 3: return ad ? run_wide<T, 3, true>(a, NP, grid, st, occ) : run_wide<T, 3, false>(a, NP, grid, st, occ);
        case 4: return ad ? run_wide<T, 4, true>(a, NP, grid, st, occ) : run_wide<T, 4, false>(a, NP, grid, st, occ);
        default: return cudaErrorInvalidValue;
    }
}

WideArgs<float> wide_args(const SweepArgsF &s, int NP) {
    WideArgs<float> a{};
    a.P = s.P;
    a.Q = s.Q;
    for (int i = 0; i < 3; ++i) a.B[i] = s.B[i];
    a.adaptive = s.adaptive;
    a.dpart = s.dpart;
    a.ld = s.ld;
    a.N = s.N;
    a.NP = NP;
    a.row_blocks = s.row_blocks;
    a.col_splits = s.col_splits;
    a.cols_per_split = s.cols_per_split;
    a.ldv = s.ldv;
    a.xT = s.xT;
    a.xiT = s.xiT;
    a.y0 = s.yh;
    a.y1 = s.yl;
    a.u0 = s.uh;
    a.u1 = s.ul;
    a.st = s.st;
    a.rowpart = s.rowpart;
    a.colpart = s.colpart;
    return a;
}

WideArgs<double> wide_args(const SweepArgsD &s, int NP) {
    WideArgs<double> a{};
    a.P = s.P;
    a.Q = s.Q;
    for (int i = 0; i < 3; ++i) a.B[i] = s.B[i];
    a.adaptive = s.adaptive;
    a.dpart = s.dpart;
    a.ld = s.ld;
    a.N = s.N;
    a.NP = NP;
    a.row_blocks = s.row_blocks;
    a.col_splits = s.col_splits;
    a.cols_per_split = s.cols_per_split;
    a.ldv = s.ldv;
    a.xT = s.xT;
    a.xiT = s.xiT;
    a.y0 = s.y;
    a.y1 = s.y;
    a.u0 = s.u;
    a.u1 = s.u;
    a.st = s.st;
    a.rowpart = s.rowpart;
    a.colpart = s.colpart;
    return a;
}

}  // namespace

bool sweep_wide_config(int np, bool f64, SweepConfig *cfg) {
    if (np <= 32 || np > CR_MAX_N || np % 16 != 0) return false;
    if (f64) {
        cfg->rows = WideShape<double>::MR * WideShape<double>::WARPS;
        cfg->threads = WideShape<double>::WARPS * 32;
        cfg->smem = wide_smem<double>(np);
    } else {
        cfg->rows = WideShape<float>::MR * WideShape<float>::WARPS;
        cfg->threads = WideShape<float>::WARPS * 32;
        cfg->smem = wide_smem<float>(np);
    }
    return true;
}

cudaError_t launch_sweep_wide_f(int np, const SweepArgsF &a, int grid, cudaStream_t s) {
    return dispatch_wide(wide_args(a, np), np, grid, s, nullptr);
}
cudaError_t launch_sweep_wide_d(int np, const SweepArgsD &a, int grid, cudaStream_t s) {
    return dispatch_wide(wide_args(a, np), np, grid, s, nullptr);
}
cudaError_t sweep_wide_occupancy(int np, bool f64, bool adaptive, int *blocks_per_sm) {
    if (f64) {
        WideArgs<double> a{};
        a.adaptive = adaptive ? 1 : 0;
        return dispatch_wide(a, np, 0, 0, blocks_per_sm);
    }
    WideArgs<float> a{};
    a.adaptive = adaptive ? 1 : 0;
    return dispatch_wide(a, np, 0, 0, blocks_per_sm);
}

}  // namespace cr
