// Shared pieces of the specialised contractions (contract_ff.cu: the four uniform product types;
// contract_ffb.cu: orders up to 8; contract_opn.cu: operator term lists): the compile-time coefficient runs of
// Eq. (3) for Legendre products, the coefficient table in constant memory (one copy per
// translation unit, all filled by contract_ff_upload), stages 1 and 2 of the contraction of
// Eq. (4), an asynchronous 8-byte copy into shared memory and a 256-bit streaming store.
#pragma once

#include "arith.cuh"
#include "p2s_internal.h"

namespace p2s {

__host__ __device__ constexpr int run_kmin(int t, int a, int b) {
    return t == 2 ? run_kmin(1, b, a)
         : t == 0 ? (a > b ? a - b : b - a)
         : t == 1 ? (a == 0 ? 0 : (b >= a - 1 ? b - a + 1 : ((a - 1 - b) & 1)))
                  : ((a == 0 || b == 0) ? 0 : ((a > b ? a - b : b - a) & 1));
}

__host__ __device__ constexpr int run_cnt(int t, int a, int b) {
    return t == 2 ? run_cnt(1, b, a)
         : t == 0 ? (a < b ? a : b) + 1
         : t == 1 ? (a == 0 ? 0 : (a + b - 1 - run_kmin(1, a, b)) / 2 + 1)
                  : ((a == 0 || b == 0) ? 0 : (a + b - 2 - run_kmin(3, a, b)) / 2 + 1);
}

// Longest run of type t over the first index a < 8 for a fixed second index b: the bound of
// a stage-2 coefficient loop whose n1 is a run-time value but whose n2 is unrolled.
__host__ __device__ constexpr int max_run_over_a(int t, int b) {
    int m = 0;
    for (int a = 0; a < 8; ++a) m = run_cnt(t, a, b) > m ? run_cnt(t, a, b) : m;
    return m;
}

namespace {

constexpr int kSpec = 8;     // coefficient table extent
constexpr int kSpecMax = 8;    // largest specialised order of the four-type kernel
constexpr int kSpecOpMax = 6;  // largest order of the operator kernel (N^2 float-float registers)
__constant__ float2 c_runs[4][kSpec][kSpec][kSpec];  // [t][a][b][r]: coefficient of P_{kmin + 2r}

// Stages 1 and 2 for one (m1, m2, q) per thread (product type TT on u, TV on v):
//   A[l]                      = sum_k C[m1,m2,k] I[k][l][q]
//   Bt[m1][n1][m2][n2][q]     = sum_l C[n1,n2,l] A[l]      (all n1, n2)
template <int N, int TT, int TV = TT>
__device__ __forceinline__ void stages12(const float2* __restrict__ sI, float2* __restrict__ sB, int m1a, int m1n,
                                         int tid, int nth) {
    constexpr int K = 2 * N - 1;
    const int items = m1n * N * K;
    for (int it = tid; it < items; it += nth) {
        const int q = it % K, mm = it / K;
        const int m2 = mm % N, im1 = mm / N;
        const int m1 = m1a + im1;
        const int k0 = run_kmin(TT, m1, m2), cnt = run_cnt(TT, m1, m2);
        float2 A[K];
        if (cnt > 0) {
            const float2 c = c_runs[TT][m1][m2][0];
            const float2* Ik = sI + k0 * K * K + q;
#pragma unroll
            for (int l = 0; l < K; ++l) A[l] = ArithFF::mul(c, Ik[l * K]);
        } else {
#pragma unroll
            for (int l = 0; l < K; ++l) A[l] = ArithFF::zero();
        }
        for (int r = 1; r < cnt; ++r) {
            const float2 c = c_runs[TT][m1][m2][r];
            const float2* Ik = sI + (k0 + 2 * r) * K * K + q;
#pragma unroll
            for (int l = 0; l < K; ++l) ArithFF::fma_acc(A[l], c, Ik[l * K]);
        }
#pragma unroll
        for (int l = 0; l < K; ++l) A[l] = ArithFF::finish(A[l]);
        float2* dst = sB + ((size_t)(im1 * N) * N + m2) * N * K + q;
#pragma unroll
        for (int n1 = 0; n1 < N; ++n1)
#pragma unroll
            for (int n2 = 0; n2 < N; ++n2) {
                const int l0 = run_kmin(TV, n1, n2), lc = run_cnt(TV, n1, n2);
                float2 acc = lc > 0 ? ArithFF::mul(c_runs[TV][n1][n2][0], A[l0]) : ArithFF::zero();
#pragma unroll
                for (int r = 1; r < N; ++r)
                    if (r < lc) ArithFF::fma_acc(acc, c_runs[TV][n1][n2][r], A[l0 + 2 * r]);
                dst[((size_t)n1 * N * N + n2) * K] = ArithFF::finish(acc);
            }
    }
}

// 8-byte asynchronous global -> shared copy (complete after cp_async_wait_all).
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned sh = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sh), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Streaming 256-bit store of four doubles (a whole 32-byte sector; p 32-byte aligned).  Two
// 16-byte stores per sector would send each sector to L2 in two halves.
__device__ __forceinline__ void st_cs_v4(double* p, double a, double b, double c, double d) {
    asm volatile("st.global.cs.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}

}  // namespace
}  // namespace p2s
