// Operator fills (term lists) of one field component of uniform order N (2..6) in mixed precision:
// step a4 (Eq. (3)-(4) of arXiv:1703.09619) with each term's own per-axis product types.
#include "asm_stages.cuh"
#include "contract_ff_stages.cuh"

namespace p2s {
namespace {

// Operator fills (term lists) of one field component of uniform order N: the same stages with
// each term's per-axis product types (tu on u, tv on v in stages 1-2, tw on w in stage 3).  A
// unit is an m1 slab of the element's single block; every thread owns one (m1, n1, m2, n2)
// combination and keeps its N x N (p1, p2) results in float-float registers across the terms, so
// the terms add without a shared-memory tile and the rows are written once.  Each term's
// moments (its coupling pair) are staged with the term's scale folded in.

// acc[p1][p2] += sum_q C_tw[p1,p2,q] b[q] for one combination
template <int N, int TW>
__device__ __forceinline__ void stage3_acc(const float2* __restrict__ b, float2 (&acc)[N][N]) {
#pragma unroll
    for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
        for (int p2 = 0; p2 < N; ++p2) {
            const int q0 = run_kmin(TW, p1, p2), qc = run_cnt(TW, p1, p2);
#pragma unroll
            for (int r = 0; r < N; ++r)
                if (r < qc) ArithFF::fma_acc(acc[p1][p2], c_runs[TW][p1][p2][r], b[q0 + 2 * r]);
        }
}

template <int N>
__device__ __forceinline__ void stages12_op(int tu, int tv, const float2* sI, float2* sB, int m1a, int m1n, int tid,
                                            int nth) {
    switch (tu * 4 + tv) {
#define P2S_S12(a, b) case a * 4 + b: stages12<N, a, b>(sI, sB, m1a, m1n, tid, nth); break;
        P2S_S12(0, 0) P2S_S12(0, 1) P2S_S12(0, 2) P2S_S12(0, 3)
        P2S_S12(1, 0) P2S_S12(1, 1) P2S_S12(1, 2) P2S_S12(1, 3)
        P2S_S12(2, 0) P2S_S12(2, 1) P2S_S12(2, 2) P2S_S12(2, 3)
        P2S_S12(3, 0) P2S_S12(3, 1) P2S_S12(3, 2) P2S_S12(3, 3)
#undef P2S_S12
    default: break;
    }
}

template <int N>
__global__ void __launch_bounds__(256, 2) k_contract_opn(ContractLaunch L) {
    constexpr int K = 2 * N - 1, K3 = K * K * K, MJ = N * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2* sI = reinterpret_cast<float2*>(smraw);
    float2* sB = sI + L.a_cap;
    __shared__ ContractUnit s_cu;
    __shared__ int s_term[64];
    __shared__ float s_scale[64][2];
    const int tid = threadIdx.x, nth = blockDim.x;
    const unsigned long long nu = (unsigned long long)L.n_units;
    const bool out_aligned32 = (reinterpret_cast<uintptr_t>(L.out) & 31) == 0;
    const int term0 = L.op_block[0], n_terms = L.op_block[1];
    for (;;) {
        if (tid == 0) {
            const unsigned long long a = atomicAdd(L.counter, 1ull);
            ContractUnit u{};
            u.e = -1;
            s_cu = a < nu ? L.units[a] : u;
        }
        __syncthreads();
        const ContractUnit cu = s_cu;
        if (cu.e < 0) break;
        const ElemDesc* d = L.desc + cu.e;
        const int m1a = cu.m1a, m1n = cu.m1n;
        const int64_t n = d->n;
        const int ncombo = m1n * N * MJ;
        float2 acc[N][N];
#pragma unroll
        for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2) acc[p1][p2] = ArithFF::zero();
        for (int kt0 = 0; kt0 < n_terms; kt0 += 64) {
            const int nk = min(64, n_terms - kt0);
            if (tid < nk) {  // the terms of this batch: packed types and the scale as (hi, lo)
                s_term[tid] = __ldg(L.op_terms + term0 + kt0 + tid);
                const double sc = __ldg(L.op_scales + term0 + kt0 + tid);
                const float hi = (float)sc;
                s_scale[tid][0] = hi;
                s_scale[tid][1] = (float)(sc - (double)hi);
            }
            __syncthreads();
            for (int kt = 0; kt < nk; ++kt) {
                const int32_t pk = s_term[kt];
                const int sp = pair_index(pk & 15, (pk >> 4) & 15, L.op_nalpha);
                const int tu = (pk >> 8) & 15, tv = (pk >> 12) & 15, tw = (pk >> 16) & 15;
                const float sh = s_scale[kt][0], sl = s_scale[kt][1];
                const float2* gI = reinterpret_cast<const float2*>(L.mom) + d->mom_off + d->pair_off[sp];
                for (int i = tid; i < K3; i += nth) sI[i] = ArithFF::scaled(__ldg(gI + i), 0.0, sh, sl);
                __syncthreads();
                stages12_op<N>(tu, tv, sI, sB, m1a, m1n, tid, nth);
                __syncthreads();
                if (tid < ncombo) {
                    float2 b[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) b[q] = sB[(size_t)tid * K + q];
                    switch (tw) {
                    case 0: stage3_acc<N, 0>(b, acc); break;
                    case 1: stage3_acc<N, 1>(b, acc); break;
                    case 2: stage3_acc<N, 2>(b, acc); break;
                    default: stage3_acc<N, 3>(b, acc); break;
                    }
                }
                __syncthreads();  // sI and sB are reused by the next term
            }
        }
        if (tid < ncombo) {
            const int mn = tid / MJ, mj = tid - mn * MJ;  // mn = im1 * N + n1, mj = m2 * N + n2
            double* r1 = L.out + d->out_off + (int64_t)(m1a * MJ + mn * N) * n + mj * N;
            if (L.out_ff) {  // float-float pairs in the 8-byte slots, for a float-float consumer
#pragma unroll
                for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                    for (int p2 = 0; p2 < N; ++p2)
                        __stcs(reinterpret_cast<float2*>(r1 + p1 * n + p2), ArithFF::finish(acc[p1][p2]));
            } else {
                double v[N][N];
#pragma unroll
                for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                    for (int p2 = 0; p2 < N; ++p2) v[p1][p2] = ArithFF::to_double_fast(ArithFF::finish(acc[p1][p2]));
                bool done = false;
                if constexpr (N == 4) {  // one whole 32-byte sector per store
                    if (out_aligned32 && (n % 4 == 0) && (d->out_off % 4 == 0)) {
#pragma unroll
                        for (int p1 = 0; p1 < N; ++p1) st_cs_v4(r1 + p1 * n, v[p1][0], v[p1][1], v[p1][2], v[p1][3]);
                        done = true;
                    }
                }
                if (!done) {
#pragma unroll
                    for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                        for (int p2 = 0; p2 < N; ++p2) __stcs(r1 + p1 * n + p2, v[p1][p2]);
                }
            }
        }
        __syncthreads();  // s_cu is replaced by thread 0
    }
}

// Fused operator fill and global assembly for one field component of uniform order N <= 4 (a unit
// is a whole element, N^4 <= 256 stage-3 combinations): the term loop of k_contract_opn leaves the
// element matrix in float-float registers, which go straight into the staged layout of the
// assembly; the change to the hierarchic basis and the scatter into CSR follow (asm_stages.cuh).
// No element matrix reaches HBM.  Launched once per colour of the mesh (the units of one colour),
// so that within a launch every CSR position receives at most one reduction.
template <int N>
__global__ void __launch_bounds__(256, 2) k_opn_assemble(ContractLaunch L, AsmMeshDev ms, AsmCoef coef) {
    constexpr int K = 2 * N - 1, K3 = K * K * K, MJ = N * N, NN = N * N, n = NN * N, P = NN | 1, G = n * N;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2* sI = reinterpret_cast<float2*>(smraw);
    float2* sB = sI + L.a_cap;
    float2* s_x = sB + L.b_cap;  // the element matrix, staged layout [G][P]
    int64_t* s_base = reinterpret_cast<int64_t*>(s_x + G * P);
    int2* s_cvw = reinterpret_cast<int2*>(s_base + n);
    int* s_rank = reinterpret_cast<int*>(s_cvw + n);
    __shared__ ContractUnit s_cu;
    __shared__ int s_term[64];
    __shared__ float s_scale[64][2];
    const int tid = threadIdx.x, nth = blockDim.x;
    const unsigned long long nu = (unsigned long long)L.n_units;
    const int term0 = L.op_block[0], n_terms = L.op_block[1];
    for (;;) {
        if (tid == 0) {
            const unsigned long long a = atomicAdd(L.counter, 1ull);
            ContractUnit u{};
            u.e = -1;
            s_cu = a < nu ? L.units[a] : u;
        }
        __syncthreads();
        const ContractUnit cu = s_cu;
        if (cu.e < 0) break;
        const ElemDesc* d = L.desc + cu.e;
        const int ncombo = N * N * MJ;
        float2 acc[N][N];
#pragma unroll
        for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2) acc[p1][p2] = ArithFF::zero();
        for (int kt0 = 0; kt0 < n_terms; kt0 += 64) {
            const int nk = min(64, n_terms - kt0);
            if (tid < nk) {
                s_term[tid] = __ldg(L.op_terms + term0 + kt0 + tid);
                const double sc = __ldg(L.op_scales + term0 + kt0 + tid);
                const float hi = (float)sc;
                s_scale[tid][0] = hi;
                s_scale[tid][1] = (float)(sc - (double)hi);
            }
            __syncthreads();
            for (int kt = 0; kt < nk; ++kt) {
                const int32_t pk = s_term[kt];
                const int sp = pair_index(pk & 15, (pk >> 4) & 15, L.op_nalpha);
                const int tu = (pk >> 8) & 15, tv = (pk >> 12) & 15, tw = (pk >> 16) & 15;
                const float sh = s_scale[kt][0], sl = s_scale[kt][1];
                const float2* gI = reinterpret_cast<const float2*>(L.mom) + d->mom_off + d->pair_off[sp];
                for (int i = tid; i < K3; i += nth) sI[i] = ArithFF::scaled(__ldg(gI + i), 0.0, sh, sl);
                __syncthreads();
                stages12_op<N>(tu, tv, sI, sB, 0, N, tid, nth);
                __syncthreads();
                if (tid < ncombo) {
                    float2 b[K];
#pragma unroll
                    for (int q = 0; q < K; ++q) b[q] = sB[(size_t)tid * K + q];
                    switch (tw) {
                    case 0: stage3_acc<N, 0>(b, acc); break;
                    case 1: stage3_acc<N, 1>(b, acc); break;
                    case 2: stage3_acc<N, 2>(b, acc); break;
                    default: stage3_acc<N, 3>(b, acc); break;
                    }
                }
                __syncthreads();
            }
        }
        // the element's rows (m1, n1, p1) = mn N + p1 and columns (m2, n2, p2) into the staged tile
        if (tid < ncombo) {
            const int mn = tid / MJ, mj = tid - mn * MJ, m2 = mj / N, n2 = mj - m2 * N;
#pragma unroll
            for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                for (int p2 = 0; p2 < N; ++p2)
                    s_x[((mn * N + p1) * N + m2) * P + n2 * N + p2] = ArithFF::finish(acc[p1][p2]);
        }
        const int e = cu.e, i = e % ms.nx, j = (e / ms.nx) % ms.ny, k = e / (ms.nx * ms.ny);
        asm_element_tables<N>(ms, i, j, k, s_base, s_cvw, s_rank, tid, nth);
        __syncthreads();
        asm_pass_a_shared<N, true>(s_x, coef, tid, nth);
        __syncthreads();
        asm_passes_bcd<N, true>(s_x, coef, tid, nth);
        asm_scatter<N, true>(s_x, s_base, s_cvw, s_rank, ms.values, tid, nth);
        __syncthreads();  // s_cu, the tile and the tables are reused by the next unit
    }
}

template <int N>
cudaError_t set_attr_asm() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_opn_assemble<N>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_opn_assemble<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

template <int N>
cudaError_t set_attr_op() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_contract_opn<N>);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_contract_opn<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

}  // namespace

#define P2S_OPN_CASES(X) X(2) X(3) X(4) X(5) X(6)

cudaError_t contract_opn_upload(const void* runs, size_t bytes) {
    cudaError_t e = cudaMemcpyToSymbol(c_runs, runs, bytes);
    if (e != cudaSuccess) return e;
    for (cudaError_t r : {set_attr_op<2>(), set_attr_op<3>(), set_attr_op<4>(), set_attr_op<5>(), set_attr_op<6>(),
                          set_attr_asm<2>(), set_attr_asm<3>(), set_attr_asm<4>()})
        if (r != cudaSuccess) return r;
    return cudaSuccess;
}

size_t opn_assemble_smem_bytes(int N) {
    const int K = 2 * N - 1, NN = N * N, n = NN * N;
    return sizeof(float2) * ((size_t)K * K * K + (size_t)NN * NN * K + (size_t)n * N * (NN | 1)) +
           sizeof(int64_t) * n + sizeof(int2) * n + sizeof(int) * 3 * NN;
}

cudaError_t launch_opn_assemble(int N, const ContractLaunch& L, const AsmMeshDev& ms, const AsmCoef& coef, int grid,
                                int threads, size_t smem, cudaStream_t s) {
    switch (N) {
    case 2: k_opn_assemble<2><<<grid, threads, smem, s>>>(L, ms, coef); break;
    case 3: k_opn_assemble<3><<<grid, threads, smem, s>>>(L, ms, coef); break;
    case 4: k_opn_assemble<4><<<grid, threads, smem, s>>>(L, ms, coef); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int opn_assemble_blocks_per_sm(int N, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_opn_assemble<2>, threads, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_opn_assemble<3>, threads, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_opn_assemble<4>, threads, smem); break;
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_contract_opn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (N) {
#define X(n) case n: k_contract_opn<n><<<grid, threads, smem, s>>>(L); break;
        P2S_OPN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int contract_opn_blocks_per_sm(int N, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
#define X(n) case n: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_contract_opn<n>, threads, smem); break;
        P2S_OPN_CASES(X)
#undef X
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

}  // namespace p2s
