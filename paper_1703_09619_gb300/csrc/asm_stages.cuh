// Device pieces of the global assembly shared by the staged kernel (assembly.cu) and the fused
// operator-contraction + assembly kernel (contract_opn.cu): the mesh's 1-D tables, the change to
// the hierarchic basis l_0 = (P_0 - P_1)/2, l_1 = (P_0 + P_1)/2, l_k = (P_k - P_{k-2}) / sqrt(2 (2k-1))
// applied axis by axis to an element matrix staged in shared memory, and the scatter into CSR.
#pragma once

#include "arith.cuh"
#include "dw.cuh"
#include "p2s_internal.h"

namespace p2s {

// Device view of one axis.
struct AxisDev {
    int n_el, N, ng;
    const int32_t* cnt;
    const int32_t* rank;
};

// The mesh's CSR tables on the device (plain pointers into the assembly's buffers).
struct AsmMeshDev {
    const int64_t* row_ptr;  // [rows + 1]
    double* values;          // CSR values
    AxisDev ax[3];
    int nx, ny, nz;
};
// The bubble normalisation 1 / sqrt(2 (2k - 1)), in FP64 and as (hi, lo) FP32 pairs.
struct AsmCoef {
    double ck[kMaxOrder];
    float ckf[2 * kMaxOrder];
};

namespace {

__device__ __forceinline__ int axis_g(const AxisDev& A, int i, int m) {
    return m == 0 ? i : (m == 1 ? i + 1 : A.n_el + 1 + i * (A.N - 2) + (m - 2));
}

// Shared-memory tables of one element for the scatter (n = N^3 local dofs):
//   base[r]  CSR start of the global row of local row r,
//   cvw[r]   neighbour counts (cnt_v(gv), cnt_w(gw)) of that row,
//   dec[r]   the digits (m, n, p) of r packed in bytes,
//   rank[a][x][y]  rank of the element's axis-a dof y among the neighbours of its dof x,
// so the position of entry (r, c) is base[r] + (ru cnt_v + rv) cnt_w + rw.
__host__ __device__ constexpr size_t asm_table_bytes_staged(int N) {
    return sizeof(int64_t) * (N * N * N) + sizeof(int2) * (N * N * N) + sizeof(int) * 3 * N * N;
}
// T applied in place to x[0], x[S], ..., x[(N-1) S] (compile-time indices, so x stays in
// registers); k descends so that x[(k-2) S] is still the input when x[k S] is formed.
template <int N, int S>
__device__ __forceinline__ void hier_T(double* x, const AsmCoef& C) {
    const double y0 = 0.5 * (x[0] - x[S]), y1 = 0.5 * (x[0] + x[S]);
#pragma unroll
    for (int k = N - 1; k >= 2; --k) x[k * S] = C.ck[k] * (x[k * S] - x[(k - 2) * S]);
    x[0] = y0;
    x[S] = y1;
}
// The same in float-float (SloppyDWPlusDW sums, normalised products): absolute error
// O(u^2 (|x_a| + |x_b|)) per output, u = 2^-24, and every result normalised (|lo| <= ulp(hi)/2),
// as the conversion to FP64 requires.  Halving is exact.
template <int N, int S>
__device__ __forceinline__ void hier_T(dw* x, const AsmCoef& C) {
    const dw d = dw_sub_fast(x[0], x[S]), a = dw_add_fast(x[0], x[S]);
#pragma unroll
    for (int k = N - 1; k >= 2; --k)
        x[k * S] = dw_mul(dw_sub_fast(x[k * S], x[(k - 2) * S]), dw{C.ckf[2 * k], C.ckf[2 * k + 1]});
    x[0] = dw{0.5f * d.hi, 0.5f * d.lo};
    x[S] = dw{0.5f * a.hi, 0.5f * a.lo};
}

// Values of the staged kernel: FP64, or float-float pairs (the mixed fill's output kept as
// (hi, lo) FP32 words in each 8-byte slot).  R in registers, M in memory.
template <bool kFF>
struct AsmVal {
    using R = double;
    using M = double;
    __device__ static R ld(const M* p) { return *p; }
    __device__ static void st(M* p, R v) { *p = v; }
    __device__ static R ldg(const double* p) { return __ldg(p); }
    __device__ static double out(const M* p) { return *p; }
};
template <>
struct AsmVal<true> {
    using R = dw;
    using M = float2;
    __device__ static R ld(const M* p) {
        const float2 f = *p;
        return dw{f.x, f.y};
    }
    __device__ static void st(M* p, R v) { *p = make_float2(v.hi, v.lo); }
    __device__ static R ldg(const double* p) {
        const float2 f = __ldg(reinterpret_cast<const float2*>(p));
        return dw{f.x, f.y};
    }
    __device__ static double out(const M* p) { return ArithFF::to_double_fast(*p); }
};

// Staged layout of an element matrix (order N, n = N^3 dofs): entry (r, c), c = m2 N^2 + j, at
// (r N + m2) P + j with P = N^2 rounded up to odd, so rows of N^2 trial entries start on distinct
// banks.

// The scatter tables of element (i, j, k).
template <int N>
__device__ __forceinline__ void asm_element_tables(const AsmMeshDev& m, int i, int j, int k, int64_t* s_base,
                                                   int2* s_cvw, int* s_rank, int tid, int nth) {
    constexpr int NN = N * N, n = NN * N;
    for (int t = tid; t < 3 * NN; t += nth) {
        const int a = t / NN, xy = t - a * NN;
        s_rank[t] = m.ax[a].rank[(a == 0 ? i : (a == 1 ? j : k)) * NN + xy];
    }
    for (int r = tid; r < n; r += nth) {
        const int gu = axis_g(m.ax[0], i, r / NN), gv = axis_g(m.ax[1], j, (r / N) % N), gw = axis_g(m.ax[2], k, r % N);
        s_base[r] = m.row_ptr[((int64_t)gu * m.ax[1].ng + gv) * m.ax[2].ng + gw];
        s_cvw[r] = make_int2(m.ax[1].cnt[gv], m.ax[2].cnt[gw]);
    }
}

// Pass A (test u) from an element matrix in HBM (row-major n x n): lines lo = rr n + c (rr: test
// v, w digits), the N values at m n N^2 + lo; coalesced along c.
template <int N, bool kFF>
__device__ __forceinline__ void asm_pass_a_global(const double* __restrict__ src, typename AsmVal<kFF>::M* s_x,
                                                  const AsmCoef& C, int tid, int nth) {
    using AV = AsmVal<kFF>;
    constexpr int NN = N * N, n = NN * N, P = NN | 1;
#pragma unroll 4
    for (int lo = tid; lo < n * NN; lo += nth) {
        typename AV::R x[N];
#pragma unroll
        for (int m = 0; m < N; ++m) x[m] = AV::ldg(src + m * (n * NN) + lo);
        hier_T<N, 1>(x, C);
        const int rr = lo / n, c = lo - rr * n, m2 = c / NN, jj = c - m2 * NN;
#pragma unroll
        for (int m = 0; m < N; ++m) AV::st(s_x + ((m * NN + rr) * N + m2) * P + jj, x[m]);
    }
}

// Pass A (test u) on a matrix already staged.
template <int N, bool kFF>
__device__ __forceinline__ void asm_pass_a_shared(typename AsmVal<kFF>::M* s_x, const AsmCoef& C, int tid, int nth) {
    using AV = AsmVal<kFF>;
    constexpr int NN = N * N, n = NN * N, P = NN | 1;
    for (int lo = tid; lo < n * NN; lo += nth) {
        const int rr = lo / n, c = lo - rr * n, m2 = c / NN, jj = c - m2 * NN;
        typename AsmVal<kFF>::M* base = s_x + (rr * N + m2) * P + jj;  // row (0, rr)
        typename AV::R x[N];
#pragma unroll
        for (int m = 0; m < N; ++m) x[m] = AV::ld(base + m * NN * N * P);
        hier_T<N, 1>(x, C);
#pragma unroll
        for (int m = 0; m < N; ++m) AV::st(base + m * NN * N * P, x[m]);
    }
}

// Passes B (test v and w of one (m, c)), C (trial u of one (r, j)) and D (trial v and w of one
// padded row (r, m2)), each holding its values in registers; a barrier after each.
template <int N, bool kFF>
__device__ __forceinline__ void asm_passes_bcd(typename AsmVal<kFF>::M* s_x, const AsmCoef& C, int tid, int nth) {
    using AV = AsmVal<kFF>;
    using R = typename AV::R;
    using M = typename AV::M;
    constexpr int NN = N * N, n = NN * N, P = NN | 1, G = n * N;
    for (int g = tid; g < N * n; g += nth) {
        const int m = g / n, c = g - m * n, m2 = c / NN, jj = c - m2 * NN;
        M* base = s_x + ((m * NN) * N + m2) * P + jj;  // row (m, 0, 0)
        R x[NN];
#pragma unroll
        for (int v = 0; v < NN; ++v) x[v] = AV::ld(base + v * N * P);  // row (m, v / N, v % N)
#pragma unroll
        for (int a = 0; a < N; ++a) hier_T<N, 1>(x + a * N, C);  // w
#pragma unroll
        for (int b = 0; b < N; ++b) hier_T<N, N>(x + b, C);      // v
#pragma unroll
        for (int v = 0; v < NN; ++v) AV::st(base + v * N * P, x[v]);
    }
    __syncthreads();
    for (int l = tid; l < n * NN; l += nth) {
        const int r = l / NN, jj = l - r * NN;
        M* base = s_x + r * N * P + jj;
        R x[N];
#pragma unroll
        for (int m2 = 0; m2 < N; ++m2) x[m2] = AV::ld(base + m2 * P);
        hier_T<N, 1>(x, C);
#pragma unroll
        for (int m2 = 0; m2 < N; ++m2) AV::st(base + m2 * P, x[m2]);
    }
    __syncthreads();
    for (int g = tid; g < G; g += nth) {
        M* base = s_x + g * P;
        R x[NN];
#pragma unroll
        for (int v = 0; v < NN; ++v) x[v] = AV::ld(base + v);
#pragma unroll
        for (int a = 0; a < N; ++a) hier_T<N, 1>(x + a * N, C);  // w
#pragma unroll
        for (int b = 0; b < N; ++b) hier_T<N, N>(x + b, C);      // v
#pragma unroll
        for (int v = 0; v < NN; ++v) AV::st(base + v, x[v]);
    }
    __syncthreads();
}

// Every entry of the staged (hierarchic-basis) matrix added to its CSR position by an L2
// reduction (red.global.add.f64); within one colour every position receives at most one.
template <int N, bool kFF>
__device__ __forceinline__ void asm_scatter(const typename AsmVal<kFF>::M* s_x, const int64_t* s_base,
                                            const int2* s_cvw, const int* s_rank, double* values, int tid, int nth) {
    using AV = AsmVal<kFF>;
    constexpr int NN = N * N, n = NN * N, nn = n * n, P = NN | 1;
    for (int t = tid; t < nn; t += nth) {
        const int r = t / n, c = t - r * n, m2 = c / NN, jj = c - m2 * NN;
        const int ru = s_rank[(r / NN) * N + m2];
        const int rv = s_rank[NN + ((r / N) % N) * N + jj / N];
        const int rw = s_rank[2 * NN + (r % N) * N + jj % N];
        const int2 cvw = s_cvw[r];
        atomicAdd(values + s_base[r] + ((ru * cvw.x + rv) * cvw.y + rw), AV::out(s_x + (r * N + m2) * P + jj));
    }
}

__host__ __device__ constexpr size_t staged_smem_bytes(int N) {
    return sizeof(double) * (size_t)(N * N * N * N) * (size_t)((N * N) | 1) + asm_table_bytes_staged(N);
}

}  // namespace
}  // namespace p2s
