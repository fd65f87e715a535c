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
#include "contract_ff_stages.cuh"

namespace p2s {
namespace {

// Rows p1 in [P1A, P1A + NP) of one combination: v[i][p2] = sum_q C_TT[p1,p2,q] b[q], p1 = P1A + i.
template <int N, int TT, int P1A, int NP>
__device__ __forceinline__ void stage3_rows(const float2 (&b)[2 * N - 1], double (&v)[NP][N]) {
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int p2 = 0; p2 < N; ++p2) {
            const int p1 = P1A + i;
            const int q0 = run_kmin(TT, p1, p2), qc = run_cnt(TT, p1, p2);
            float2 acc = qc > 0 ? ArithFF::mul(c_runs[TT][p1][p2][0], b[q0]) : ArithFF::zero();
#pragma unroll
            for (int r = 1; r < N; ++r)
                if (r < qc) ArithFF::fma_acc(acc, c_runs[TT][p1][p2][r], b[q0 + 2 * r]);
            v[i][p2] = ArithFF::to_double_fast(ArithFF::finish(acc));
        }
}

// Store rows [P1A, P1A + NP) of one combination in both orientations.
template <int N, int P1A, int NP>
__device__ __forceinline__ void stage3_store(const double (&v)[NP][N], double* r1, double* r2, int64_t n, bool vec,
                                             bool vec4) {
    if (N == 4 && NP == 4 && vec4) {  // one whole 32-byte sector per store
#pragma unroll
        for (int i = 0; i < NP; ++i) st_cs_v4(r1 + (P1A + i) * n, v[i][0], v[i][1 % N], v[i][2 % N], v[i][3 % N]);
    } else if (vec) {
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int p2 = 0; p2 < N; p2 += 2)
                __stcs(reinterpret_cast<double2*>(r1 + (P1A + i) * n + p2), make_double2(v[i][p2], v[i][(p2 + 1) % N]));
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2) __stcs(r1 + (P1A + i) * n + p2, v[i][p2]);
    }
    if (r2) {
        if (N == 4 && NP == 4 && vec4) {
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2)
                st_cs_v4(r2 + p2 * n, v[0][p2], v[1 % NP][p2], v[2 % NP][p2], v[3 % NP][p2]);
        } else if (vec && P1A % 2 == 0 && NP % 2 == 0) {
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2)
#pragma unroll
                for (int i = 0; i < NP; i += 2)
                    __stcs(reinterpret_cast<double2*>(r2 + p2 * n + P1A + i), make_double2(v[i][p2], v[(i + 1) % NP][p2]));
        } else {
#pragma unroll
            for (int p2 = 0; p2 < N; ++p2)
#pragma unroll
                for (int i = 0; i < NP; ++i) __stcs(r2 + p2 * n + P1A + i, v[i][p2]);
        }
    }
}

// Stage 3 and both write-outs; one (m1, n1, m2, n2) combination per item.  Orders N >= 7 split
// each combination's p1 rows over two items (halves of ceil(N/2) and floor(N/2) rows), so a
// thread holds at most ceil(N/2) x N results in registers.
// Mt points at (row rbase, column col0) of M_t; Mp (or nullptr) at (row col0, column
// rbase) of the partner block; n is the row stride of the element's matrices.
template <int N, int TT>
__device__ __forceinline__ void stage3_split(const float2* __restrict__ sB, int m1n, int tid, int nth, double* Mt,
                                             double* Mp, int64_t n, bool vec, bool vec4) {
    constexpr int K = 2 * N - 1, MJ = N * N, H = N >= 7 ? 2 : 1, P0 = (N + H - 1) / H, P1 = N - P0;
    const int ncombo = m1n * N * MJ;
    for (int it = tid; it < ncombo * H; it += nth) {
        const int c = H == 2 ? it >> 1 : it, h = H == 2 ? it & 1 : 0;
        const int mn = c / MJ, mj = c - mn * MJ;  // mn = im1 * N + n1, mj = m2 * N + n2
        float2 b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) b[q] = sB[(size_t)c * K + q];
        double* r1 = Mt + (int64_t)(mn * N) * n + mj * N;                // row (m1,n1,p1=0), column (m2,n2,p2=0)
        double* r2 = Mp ? Mp + (int64_t)(mj * N) * n + mn * N : nullptr;  // partner row (m2,n2,p2=0)
        if (h == 0) {
            double v[P0][N];
            stage3_rows<N, TT, 0, P0>(b, v);
            stage3_store<N, 0, P0>(v, r1, r2, n, vec, vec4);
        } else if constexpr (P1 > 0) {
            double v[P1 > 0 ? P1 : 1][N];
            stage3_rows<N, TT, P0, (P1 > 0 ? P1 : 1)>(b, v);
            stage3_store<N, P0, (P1 > 0 ? P1 : 1)>(v, r1, r2, n, vec, vec4);
        }
    }
}

// Orders up to 6 keep all N x N results of a combination in one thread (stage3_full).
template <int N, int TT>
__device__ __forceinline__ void stage3_full(const float2* __restrict__ sB, int m1n, int tid, int nth, double* Mt,
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

template <int N, int TT>
__device__ __forceinline__ void stage3(const float2* __restrict__ sB, int m1n, int tid, int nth, double* Mt,
                                       double* Mp, int64_t n, bool vec, bool vec4) {
    if constexpr (N >= 7) stage3_split<N, TT>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4);
    else stage3_full<N, TT>(sB, m1n, tid, nth, Mt, Mp, n, vec, vec4);
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
    static double h64[4][kSpec][kSpec][kSpec];
    for (int t = 0; t < 4; ++t)
        for (int a = 0; a < kSpec; ++a)
            for (int b = 0; b < kSpec; ++b)
                for (int r = 0; r < kSpec; ++r) {
                    const int32_t li = T.lin_idx[lin_slot(t, a, b)];
                    h[t][a][b][r] = r < lin_cnt(li)
                                        ? make_float2(T.lin_coef_ff[2 * (lin_off(li) + r)], T.lin_coef_ff[2 * (lin_off(li) + r) + 1])
                                        : make_float2(0.f, 0.f);
                    h64[t][a][b][r] = r < lin_cnt(li) ? T.lin_coef[lin_off(li) + r] : 0.0;
                }
    cudaError_t e = cudaMemcpyToSymbol(c_runs, h, sizeof(h));
    if (e != cudaSuccess) return e;
    for (cudaError_t r : {set_attr<2>(), set_attr<3>(), set_attr<4>(), set_attr<5>(), set_attr<6>(), set_attr<7>(),
                          set_attr<8>()})
        if (r != cudaSuccess) return r;
    e = contract_opn_upload(h, sizeof(h));
    if (e != cudaSuccess) return e;
    return contract_ffb_upload(h, sizeof(h), &h64[0][0][0][0], sizeof(h64));
}

int contract_ff_max_order() { return kSpecMax; }
int contract_opn_max_order() { return kSpecOpMax; }

void contract_ff_shape(int N, int m1n, size_t& a_cap, size_t& b_cap, size_t& tile_cap, int& combos) {
    const int K = 2 * N - 1;
    a_cap = (size_t)K * K * K;
    b_cap = (size_t)m1n * N * N * N * K;
    tile_cap = 0;
    combos = m1n * N * N * N;
}

#define P2S_FFN_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

cudaError_t launch_contract_ffn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s) {
    switch (N) {
#define X(n) case n: k_contract_ffn<n><<<grid, threads, smem, s>>>(L); break;
        P2S_FFN_CASES(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
