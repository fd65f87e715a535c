// Mixed-precision contraction (step a4, Eq. (4) of arXiv:1703.09619) specialised at
// compile time on the order N (2..6) of a batch whose components all have N on every
// axis, and on the product type.
//
// Same work units and results as k_contract<ArithFF> (contract.cu); what changes:
//   - the Eq. (3) coefficient runs are resolved at compile time: for Legendre products
//     every coefficient is positive (Adams' formula has positive terms and P'_m is a
//     positive combination of P_j), so the nonzero k of P^(d1)_a P^(d2)_b are exactly
//         vv: |a-b| .. a+b,       dv (a>0): max(b-a+1, (a-1-b) mod 2) .. a+b-1,
//         dd (a,b>0): (a-b) mod 2 .. a+b-2,      vd(a,b) = dv(b,a),   step 2;
//     the host checks these runs against its table before enabling this kernel;
//   - the coefficient values sit in __constant__ memory at compile-time offsets;
//   - stages 1 and 2 run per thread on one (m1, m2, q) column held in registers;
//   - stage 3 gives each thread one (m1, n1, m2, n2) and all N x N (p1, p2) results in
//     registers, and stores them straight from registers in both orientations: N
//     consecutive doubles of a row of M_t(gi,gj) per p1 (consecutive threads write
//     consecutive chunks, so a warp's stores are contiguous), and N consecutive doubles
//     of a row of the transposed partner block per p2.  No shared-memory tile.
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

namespace {

constexpr int kSpec = 8;     // coefficient table extent
constexpr int kSpecMax = 6;  // largest specialised order (N^2 FP64 results per thread in registers)
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

// Stage 3 and both write-outs for one (m1, n1, m2, n2) combination per thread.
// Mt points at (row rbase, column col0) of M_t; Mp (or nullptr) at (row col0, column
// rbase) of the partner block; n is the row stride of the element's matrices.
// Streaming 256-bit store of four doubles (a whole 32-byte sector; p 32-byte aligned).  Two
// 16-byte stores per sector would send each sector to L2 in two halves.
__device__ __forceinline__ void st_cs_v4(double* p, double a, double b, double c, double d) {
    asm volatile("st.global.cs.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}

template <int N, int TT>
__device__ __forceinline__ void stage3(const float2* __restrict__ sB, int m1n, int tid, int nth, double* Mt,
                                       double* Mp, int64_t n, bool vec, bool vec4) {
    constexpr int K = 2 * N - 1, MJ = N * N;
    const int ncombo = m1n * N * MJ;
    for (int c = tid; c < ncombo; c += nth) {
        const int mn = c / MJ, mj = c - mn * MJ;  // mn = im1 * N + n1, mj = m2 * N + n2
        float2 b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) b[q] = sB[(size_t)c * K + q];
        double v[N][N];
#pragma unroll
        for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2) {
                const int q0 = run_kmin(TT, p1, p2), qc = run_cnt(TT, p1, p2);
                float2 acc = qc > 0 ? ArithFF::mul(c_runs[TT][p1][p2][0], b[q0]) : ArithFF::zero();
#pragma unroll
                for (int r = 1; r < N; ++r)
                    if (r < qc) ArithFF::fma_acc(acc, c_runs[TT][p1][p2][r], b[q0 + 2 * r]);
                v[p1][p2] = ArithFF::to_double_fast(ArithFF::finish(acc));
            }
        double* r1 = Mt + (int64_t)(mn * N) * n + mj * N;  // row (m1,n1,p1=0), column (m2,n2,p2=0)
        if (N == 4 && vec4) {  // one whole 32-byte sector per store
#pragma unroll
            for (int p1 = 0; p1 < N; ++p1) st_cs_v4(r1 + p1 * n, v[p1][0], v[p1][1], v[p1][2], v[p1][3]);
        } else if (vec) {
#pragma unroll
            for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                for (int p2 = 0; p2 < N; p2 += 2)
                    __stcs(reinterpret_cast<double2*>(r1 + p1 * n + p2), make_double2(v[p1][p2], v[p1][p2 + 1]));
        } else {
#pragma unroll
            for (int p1 = 0; p1 < N; ++p1)
#pragma unroll
                for (int p2 = 0; p2 < N; ++p2) __stcs(r1 + p1 * n + p2, v[p1][p2]);
        }
        if (Mp) {
            double* r2 = Mp + (int64_t)(mj * N) * n + mn * N;  // partner row (m2,n2,p2=0), column (m1,n1,p1=0)
            if (N == 4 && vec4) {
#pragma unroll
                for (int p2 = 0; p2 < N; ++p2) st_cs_v4(r2 + p2 * n, v[0][p2], v[1][p2], v[2][p2], v[3][p2]);
            } else if (vec) {
#pragma unroll
                for (int p2 = 0; p2 < N; ++p2)
#pragma unroll
                    for (int p1 = 0; p1 < N; p1 += 2)
                        __stcs(reinterpret_cast<double2*>(r2 + p2 * n + p1), make_double2(v[p1][p2], v[p1 + 1][p2]));
            } else {
#pragma unroll
                for (int p2 = 0; p2 < N; ++p2)
#pragma unroll
                    for (int p1 = 0; p1 < N; ++p1) __stcs(r2 + p2 * n + p1, v[p1][p2]);
            }
        }
    }
}

__device__ __forceinline__ int type_slot_ff(uint32_t mask, int t) { return __popc(mask & ((1u << t) - 1u)); }

__device__ __forceinline__ const float2* unit_moments(const ContractLaunch& L, const ContractUnit& u) {
    const ElemDesc* d = L.desc + u.e;
    return reinterpret_cast<const float2*>(L.mom) + d->mom_off + d->pair_off[pair_index(u.gi, u.gj, d->n_comp)];
}

// Persistent CTAs take units from the queue.  Thread 0 keeps the current and the next unit in
// shared slots indexed by iteration parity.  While stage 3 of the current unit runs (it reads
// no moments), every thread holds its share of the next unit's moments in registers (N <= 4;
// larger orders load them after stage 3), and stores them once stage 3 is done: two barriers
// per unit and the moment load off the critical path.
template <int N>
__global__ void __launch_bounds__(512) k_contract_ffn(ContractLaunch L) {
    constexpr int K = 2 * N - 1, K3 = K * K * K;
    constexpr int kPre = N <= 4 ? (K3 + 127) / 128 : 1;  // prefetch registers per thread (>= 128 threads)
    extern __shared__ __align__(16) unsigned char smraw[];
    float2* sI = reinterpret_cast<float2*>(smraw);
    float2* sB = sI + L.a_cap;
    __shared__ ContractUnit s_cu[2], s_nx[2];  // e = -1: no unit
    const int tid = threadIdx.x, nth = blockDim.x;
    const unsigned long long nu = (unsigned long long)L.n_units;
    const bool out_aligned = (reinterpret_cast<uintptr_t>(L.out) & 15) == 0;
    const bool out_aligned32 = (reinterpret_cast<uintptr_t>(L.out) & 31) == 0;
    const bool pre = N <= 4 && kPre * nth >= K3;

    if (tid == 0) {
        ContractUnit none{};
        none.e = -1;
        const unsigned long long a = atomicAdd(L.counter, 1ull), b = atomicAdd(L.counter, 1ull);
        s_cu[0] = a < nu ? L.units[a] : none;
        s_nx[0] = b < nu ? L.units[b] : none;
    }
    __syncthreads();
    if (s_cu[0].e >= 0) {
        const float2* gI = unit_moments(L, s_cu[0]);
        for (int i = tid; i < K3; i += nth) sI[i] = __ldg(gI + i);
    }
    __syncthreads();
    for (int iter = 0;; ++iter) {
        const int par = iter & 1;
        const ContractUnit cu = s_cu[par];
        if (cu.e < 0) break;
        const ElemDesc* d = L.desc + cu.e;
        const int gi = cu.gi, gj = cu.gj, t = cu.t, m1a = cu.m1a, m1n = cu.m1n;
        const int64_t n = d->n;
        switch (t) {
        case 0: stages12<N, 0>(sI, sB, m1a, m1n, tid, nth); break;
        case 1: stages12<N, 1>(sI, sB, m1a, m1n, tid, nth); break;
        case 2: stages12<N, 2>(sI, sB, m1a, m1n, tid, nth); break;
        default: stages12<N, 3>(sI, sB, m1a, m1n, tid, nth); break;
        }
        __syncthreads();  // stage-2 results complete; the moment buffer is free
        const ContractUnit nx = s_nx[par];
        const float2* gN = nx.e >= 0 ? unit_moments(L, nx) : nullptr;
        float2 pf[kPre];
        if (pre && gN) {
#pragma unroll
            for (int j = 0; j < kPre; ++j) {
                const int i = tid + j * nth;
                if (i < K3) pf[j] = __ldg(gN + i);
            }
        }
        // the unit's results are rows [rbase, rbase + m1n N^2) x columns [col0, col0 + N^3)
        const int rbase = d->dof_off[gi] + m1a * N * N;
        const int col0 = d->dof_off[gj];
        const bool vec = out_aligned && (N % 2 == 0) && (n % 2 == 0) && (col0 % 2 == 0) && (rbase % 2 == 0);
        // every 4-double segment 32-byte aligned: base, row stride, block corner, segment starts
        const bool vec4 = out_aligned32 && (n % 4 == 0) && (col0 % 4 == 0) && (rbase % 4 == 0) &&
                          ((d->out_off + (int64_t)type_slot_ff(L.types_mask, t) * n * n) % 4 == 0);
        double* Mt = L.out + d->out_off + type_slot_ff(L.types_mask, t) * n * n + rbase * n + col0;
        double* Mp = cu.tp >= 0 ? L.out + d->out_off + type_slot_ff(L.types_mask, cu.tp) * n * n + col0 * n + rbase
                                : nullptr;
        switch (t) {
        case 0: stage3<N, 0>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4); break;
        case 1: stage3<N, 1>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4); break;
        case 2: stage3<N, 2>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4); break;
        default: stage3<N, 3>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4); break;
        }
        if (tid == 0) {  // the unit after next, into the other slot
            ContractUnit none{};
            none.e = -1;
            const unsigned long long c = atomicAdd(L.counter, 1ull);
            s_cu[par ^ 1] = nx;
            s_nx[par ^ 1] = c < nu ? L.units[c] : none;
        }
        if (gN) {
            if (pre) {
#pragma unroll
                for (int j = 0; j < kPre; ++j) {
                    const int i = tid + j * nth;
                    if (i < K3) sI[i] = pf[j];
                }
            } else {
                for (int i = tid; i < K3; i += nth) sI[i] = __ldg(gN + i);
            }
        }
        __syncthreads();  // the next unit's moments in place; the stage-2 buffer free
    }
}

// ---------------------------------------------------------------------------------------------
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

template <int N>
cudaError_t set_attr() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_contract_ffn<N>);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_contract_ffn<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

}  // namespace

bool contract_ff_runs_match(const HostTables& T) {
    for (int t = 0; t < 4; ++t)
        for (int a = 0; a < kSpec; ++a)
            for (int b = 0; b < kSpec; ++b) {
                const int32_t li = T.lin_idx[lin_slot(t, a, b)];
                const int cnt = lin_cnt(li);
                if (cnt != run_cnt(t, a, b)) return false;
                if (cnt && lin_kmin(li) != run_kmin(t, a, b)) return false;
            }
    return true;
}

cudaError_t contract_ff_upload(const HostTables& T) {
    static float2 h[4][kSpec][kSpec][kSpec];
    for (int t = 0; t < 4; ++t)
        for (int a = 0; a < kSpec; ++a)
            for (int b = 0; b < kSpec; ++b)
                for (int r = 0; r < kSpec; ++r) {
                    const int32_t li = T.lin_idx[lin_slot(t, a, b)];
                    h[t][a][b][r] = r < lin_cnt(li)
                                        ? make_float2(T.lin_coef_ff[2 * (lin_off(li) + r)], T.lin_coef_ff[2 * (lin_off(li) + r) + 1])
                                        : make_float2(0.f, 0.f);
                }
    cudaError_t e = cudaMemcpyToSymbol(c_runs, h, sizeof(h));
    if (e != cudaSuccess) return e;
    for (cudaError_t r : {set_attr<2>(), set_attr<3>(), set_attr<4>(), set_attr<5>(), set_attr<6>(), set_attr_op<2>(),
                          set_attr_op<3>(), set_attr_op<4>(), set_attr_op<5>(), set_attr_op<6>()})
        if (r != cudaSuccess) return r;
    return cudaSuccess;
}

int contract_ff_max_order() { return kSpecMax; }

void contract_ff_shape(int N, int m1n, size_t& a_cap, size_t& b_cap, size_t& tile_cap, int& combos) {
    const int K = 2 * N - 1;
    a_cap = (size_t)K * K * K;
    b_cap = (size_t)m1n * N * N * N * K;
    tile_cap = 0;
    combos = m1n * N * N * N;
}

#define P2S_FFN_CASES(X) X(2) X(3) X(4) X(5) X(6)

cudaError_t launch_contract_ffn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (N) {
#define X(n) case n: k_contract_ffn<n><<<grid, threads, smem, s>>>(L); break;
        P2S_FFN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_contract_opn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (N) {
#define X(n) case n: k_contract_opn<n><<<grid, threads, smem, s>>>(L); break;
        P2S_FFN_CASES(X)
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
        P2S_FFN_CASES(X)
#undef X
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

int contract_ffn_blocks_per_sm(int N, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (N) {
#define X(n) case n: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_contract_ffn<n>, threads, smem); break;
        P2S_FFN_CASES(X)
#undef X
    default: break;
    }
    return e == cudaSuccess ? nb : 0;
}

}  // namespace p2s
