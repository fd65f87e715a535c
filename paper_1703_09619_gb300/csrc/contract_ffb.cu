// Contraction (step a4, Eq. (4) of arXiv:1703.09619) for batches whose per-axis orders are at
// most 8, uniform or not, in either arithmetic (FP64 or float-float).
//
// Same work units and the same arithmetic, operation for operation, as k_contract<A>
// (contract.cu), so the two give identical bits.  The orders are run-time values here, but
// the loops over the v- and w-axis indices are unrolled to the bound 8 with warp-uniform
// guards, which makes n2 and (p1, p2) compile-time constants in the unrolled bodies:
//   - the Eq. (3) coefficient runs of stages 2 and 3 come from the closed forms of
//     contract_ff_stages.cuh (checked by the host against its table), their values from
//     __constant__ memory (a float-float and an FP64 copy);
//   - stage 1 takes one (m1, m2, l, q) per thread and stage 2 one (n1, m1, m2, q) column
//     per thread over every n2, both through shared memory, so that either stage keeps
//     most of the CTA busy between its barriers;
//   - stage 3 gives each thread one (m1, n1, m2, n2) combination and up to 4 x 8 (p1, p2)
//     results in registers (2 x 8 in FP64; further p1 rows in later passes), stored straight
//     from registers in both orientations: no shared-memory tile and no write-out pass.
// The next unit's moments arrive in shared memory by cp.async while stages 2 and 3 run, and
// units of elements whose mask entry is 0 (optional) are skipped.
#include <type_traits>

#include "contract_ff_stages.cuh"

namespace p2s {
namespace {

constexpr int kB = kSpecMax;      // largest order per axis (8)
constexpr int kKB = 2 * kB - 1;  // largest moment count per axis
__constant__ double c_runs64[4][kSpec][kSpec][kSpec];  // FP64 values of c_runs

// Coefficient r of the run of (t, a, b) in the arithmetic's own type (compile-time indices).
template <class A>
__device__ __forceinline__ typename A::C run_coef(int t, int a, int b, int r);
template <>
__device__ __forceinline__ float2 run_coef<ArithFF>(int t, int a, int b, int r) { return c_runs[t][a][b][r]; }
template <>
__device__ __forceinline__ double run_coef<ArithF64>(int t, int a, int b, int r) { return c_runs64[t][a][b][r]; }

// The run-time shape of one unit: block (gi, gj) orders and derived extents.
struct FfbShape {
    int Nu_i, Nv_i, Nw_i, Nu_j, Nv_j, Nw_j;
    int Kv, Kw, Kwp, mjn;
};

__device__ __forceinline__ FfbShape ffb_shape(const ElemDesc* d, int gi, int gj) {
    FfbShape s;
    s.Nu_i = d->ord[gi][0];
    s.Nv_i = d->ord[gi][1];
    s.Nw_i = d->ord[gi][2];
    s.Nu_j = d->ord[gj][0];
    s.Nv_j = d->ord[gj][1];
    s.Nw_j = d->ord[gj][2];
    s.Kv = s.Nv_i + s.Nv_j - 1;
    s.Kw = s.Nw_i + s.Nw_j - 1;
    s.Kwp = s.Kw | 1;  // odd stage-2 row stride: stage 3's row reads spread over the banks
    s.mjn = s.Nu_j * s.Nv_j;
    return s;
}

__device__ __forceinline__ int unit_moment_count(const ElemDesc* d, int gi, int gj) {
    int v = 1;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) v *= d->ord[gi][ax] + d->ord[gj][ax] - 1;
    return v;
}

// First moment (8-byte word) of the unit's component pair.
__device__ __forceinline__ size_t ffb_moments(const ContractLaunch& L, const ContractUnit& u) {
    const ElemDesc* d = L.desc + u.e;
    return (size_t)d->mom_off + d->pair_off[pair_index(u.gi, u.gj, d->n_comp)];
}

// Stage 1 of one unit (any type; runs from the table): items (im1, m2, l, q),
//   A[im1][m2][l][q] = sum_k C[m1,m2,k] I[k][l][q].
template <class A>
__device__ __forceinline__ void ffb_stage1(const ContractLaunch& L, int t, const typename A::T* __restrict__ sI,
                                           typename A::T* __restrict__ sA, const FfbShape& s, int m1a, int m1n,
                                           int tid, int nth) {
    using T = typename A::T;
    const int KvKw = s.Kv * s.Kw;
    const int items = m1n * s.Nu_j * KvKw;
    const float rKvKw = 1.f / (float)KvKw, rNuj = 1.f / (float)s.Nu_j;
    for (int it = tid; it < items; it += nth) {
        const int mm = div_small(it, KvKw, rKvKw), lq = it - mm * KvKw;
        const int im1 = div_small(mm, s.Nu_j, rNuj), m2 = mm - im1 * s.Nu_j;
        const int32_t li = __ldg(L.lin_idx + lin_slot(t, m1a + im1, m2));
        const int k0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
        const T* Ik = sI + k0 * KvKw + lq;
        T acc = cnt > 0 ? A::mul(A::load_coef(L.lin_coef, off), Ik[0]) : A::zero();
        for (int r = 1; r < cnt; ++r) A::fma_acc(acc, A::load_coef(L.lin_coef, off + r), Ik[2 * r * KvKw]);
        sA[it] = A::finish(acc);
    }
}

// Stage 2 of one unit, type TT: items (n1, im1, m2, q) with n1 outermost (the coefficient
// reads of a warp then share n1), every n2 < Nv_j unrolled:
//   Bt[(im1, n1, m2, n2)][q] = sum_l C[n1,n2,l] A[im1][m2][l][q].
template <class A, int TT>
__device__ __forceinline__ void ffb_stage2(const typename A::T* __restrict__ sA, typename A::T* __restrict__ sB,
                                           const FfbShape& s, int m1n, int tid, int nth) {
    using T = typename A::T;
    const int per_n1 = m1n * s.Nu_j * s.Kw;
    const int items = s.Nv_i * per_n1;
    const float rper = 1.f / (float)per_n1, rKw = 1.f / (float)s.Kw, rNuj = 1.f / (float)s.Nu_j;
    for (int it = tid; it < items; it += nth) {
        const int n1 = div_small(it, per_n1, rper), rest = it - n1 * per_n1;
        const int mm = div_small(rest, s.Kw, rKw), q = rest - mm * s.Kw;
        const int im1 = div_small(mm, s.Nu_j, rNuj), m2 = mm - im1 * s.Nu_j;
        const T* a = sA + (size_t)mm * s.Kv * s.Kw + q;  // A[im1][m2][l][q] at a[l Kw]
        // combination (im1, n1, m2, n2) = ((im1 Nv_i + n1) Nu_j + m2) Nv_j + n2
        T* dst = sB + ((size_t)((im1 * s.Nv_i + n1) * s.Nu_j + m2) * s.Nv_j) * s.Kwp + q;
        // n1 is a run-time index here; it is outermost in the item order, so the constant-memory
        // reads of a warp mostly share one address
#pragma unroll
        for (int n2 = 0; n2 < kB; ++n2) {
            if (n2 >= s.Nv_j) break;
            const int l0 = run_kmin(TT, n1, n2), lc = run_cnt(TT, n1, n2);
            T acc = lc > 0 ? A::mul(run_coef<A>(TT, n1, n2, 0), a[l0 * s.Kw]) : A::zero();
            // bounded by the longest run of (TT, ., n2), a constant in this unrolled body, so
            // the multiply-adds no n1 can reach are not issued
#pragma unroll
            for (int r = 1; r < kB; ++r) {
                if (r >= max_run_over_a(TT, n2)) break;
                if (r < lc) A::fma_acc(acc, run_coef<A>(TT, n1, n2, r), a[(l0 + 2 * r) * s.Kw]);
            }
            dst[n2 * s.Kwp] = A::finish(acc);
        }
    }
}

// Streaming store of one or two consecutive doubles; the pair goes as one 16-byte store
// when its address allows.
__device__ __forceinline__ void st_one_or_two(double* p, double a, double b, bool two) {
    if (two && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));
    } else {
        __stcs(p, a);
        if (two) __stcs(p + 1, b);
    }
}

// Stage 3 for rows p1 in [P1A, P1A + 4) of combination c of the unit, and both write-outs.
// Mt points at (row rbase, column col0) of M_t; Mp (or nullptr) at (row col0, column rbase)
// of the partner block; n is the row stride of the element's matrices.
template <class A, int TT, int P1A, int NP>
__device__ __forceinline__ void ffb_stage3_rows(const typename A::T* __restrict__ sB, const FfbShape& s, int c,
                                                float rmjn, double* Mt, double* Mp, int64_t n) {
    static_assert(NP % 2 == 0, "row pairs");
    using T = typename A::T;
    const int mn = div_small(c, s.mjn, rmjn), mj = c - mn * s.mjn;  // mn = im1 Nv_i + n1, mj = m2 Nv_j + n2
    T b[kKB];
    const T* brow = sB + (size_t)c * s.Kwp;
#pragma unroll
    for (int q = 0; q < kKB; ++q) b[q] = q < s.Kw ? brow[q] : A::zero();
    double v[NP][kB];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int p2 = 0; p2 < kB; ++p2) {
            const int p1 = P1A + i;
            if (p1 < s.Nw_i && p2 < s.Nw_j) {
                const int q0 = run_kmin(TT, p1, p2), qc = run_cnt(TT, p1, p2);
                T acc = qc > 0 ? A::mul(run_coef<A>(TT, p1, p2, 0), b[q0]) : A::zero();
#pragma unroll
                for (int r = 1; r < kB; ++r)
                    if (r < qc) A::fma_acc(acc, run_coef<A>(TT, p1, p2, r), b[q0 + 2 * r]);
                v[i][p2] = A::to_double_fast(A::finish(acc));
            } else {
                v[i][p2] = 0.0;
            }
        }
    // rows (mn, p1) of M_t: Nw_j consecutive doubles each, at column mj Nw_j
    double* r1 = Mt + (int64_t)(mn * s.Nw_i + P1A) * n + mj * s.Nw_j;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (P1A + i >= s.Nw_i) break;
#pragma unroll
        for (int p2 = 0; p2 < kB; p2 += 2) {
            if (p2 >= s.Nw_j) break;
            st_one_or_two(r1 + i * n + p2, v[i][p2], v[i][p2 + 1], p2 + 1 < s.Nw_j);
        }
    }
    // rows (mj, p2) of the partner block: the unit's p1 values are consecutive columns
    if (Mp) {
        double* r2 = Mp + (int64_t)(mj * s.Nw_j) * n + mn * s.Nw_i + P1A;
#pragma unroll
        for (int p2 = 0; p2 < kB; ++p2) {
            if (p2 >= s.Nw_j) break;
#pragma unroll
            for (int i = 0; i < NP; i += 2) {
                if (P1A + i >= s.Nw_i) break;
                st_one_or_two(r2 + p2 * n + i, v[i][p2], v[i + 1][p2], P1A + i + 1 < s.Nw_i);
            }
        }
    }
}

// Stage 3 of the unit: rows p1 < 4 of every combination, then (Nw_i > 4) rows 4..7.  (One
// flat list of (half, combination) items measured slower on the uneven-order batch.)
// Rows per pass: 4 in float-float; 2 in FP64, whose DFMA chains keep more registers in flight
// (4 rows spill there).
template <class A>
constexpr int ffb_rows() { return std::is_same<typename A::T, double>::value ? 2 : 4; }

template <class A, int TT>
__device__ __forceinline__ void ffb_stage3(const typename A::T* __restrict__ sB, const FfbShape& s, int ncombo,
                                           int tid, int nth, double* Mt, double* Mp, int64_t n, float rmjn) {
    constexpr int NP = ffb_rows<A>();
    for (int c = tid; c < ncombo; c += nth) ffb_stage3_rows<A, TT, 0, NP>(sB, s, c, rmjn, Mt, Mp, n);
    if (s.Nw_i > NP)
        for (int c = tid; c < ncombo; c += nth) ffb_stage3_rows<A, TT, NP, NP>(sB, s, c, rmjn, Mt, Mp, n);
    if constexpr (NP == 2) {
        if (s.Nw_i > 4)
            for (int c = tid; c < ncombo; c += nth) ffb_stage3_rows<A, TT, 4, NP>(sB, s, c, rmjn, Mt, Mp, n);
        if (s.Nw_i > 6)
            for (int c = tid; c < ncombo; c += nth) ffb_stage3_rows<A, TT, 6, NP>(sB, s, c, rmjn, Mt, Mp, n);
    }
}

__device__ __forceinline__ int type_slot_ffb(uint32_t mask, int t) { return __popc(mask & ((1u << t) - 1u)); }

// Persistent CTAs take units from the queue.  The stages are software-pipelined over units:
// one interval between two CTA barriers runs stage 2 of unit u while the moments of unit u+1
// arrive by cp.async (into the moment buffer, free once stage 1 of u is done), and the next
// interval runs stage 3 of unit u and stage 1 of unit u+1 together (they touch different
// buffers), so a unit costs two barriers and threads with no stage-3 combination go on to
// the next unit's stage 1.  Thread 0 keeps the units in a ring of three shared slots (the
// unit of iteration i in slot i mod 3) and fetches unit u+2 during iteration u.  Shared
// memory: moments (a_cap), stage 1 (s1_cap), stage 2 (b_cap), in 8-byte words (FP64 values
// or (hi, lo) FP32 pairs).  Units of elements whose mask entry is 0 (elem_mask, optional) are
// taken from the queue and skipped.  Every entry is computed by the same operations in the
// same order as in the unpipelined loop.
template <class A>
__global__ void __launch_bounds__(512) k_contract_ffb(ContractLaunch L) {
    using T = typename A::T;
    static_assert(sizeof(T) == 8, "8-byte words");
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sI = reinterpret_cast<T*>(smraw);  // moments of the unit's pair, [k][l][q]
    T* sA = sI + L.a_cap;                  // stage 1, [im1][m2][l][q]
    T* sB = sA + L.s1_cap;                 // stage 2, [combination][q] (odd stride)
    __shared__ ContractUnit s_u[3];        // e = -1: no unit
    const int tid = threadIdx.x, nth = blockDim.x;
    const unsigned long long nu = (unsigned long long)L.n_units;
    auto fetch = [&](ContractUnit& slot) {
        ContractUnit none{};
        none.e = -1;
        const unsigned long long a = atomicAdd(L.counter, 1ull);
        slot = a < nu ? L.units[a] : none;
    };
    auto skipped = [&](const ContractUnit& u) { return L.elem_mask && !L.elem_mask[u.e]; };
    auto stage1 = [&](const ContractUnit& u) {
        const ElemDesc* d = L.desc + u.e;
        ffb_stage1<A>(L, u.t, sI, sA, ffb_shape(d, u.gi, u.gj), u.m1a, u.m1n, tid, nth);
    };

    if (tid == 0) {
        fetch(s_u[0]);
        fetch(s_u[1]);
    }
    __syncthreads();
    {  // prologue: moments and stage 1 of the first unit
        const ContractUnit u = s_u[0];
        if (u.e >= 0) {
            const size_t m0 = ffb_moments(L, u);
            const int cnt = unit_moment_count(L.desc + u.e, u.gi, u.gj);
            for (int i = tid; i < cnt; i += nth) sI[i] = A::load_moment(L.mom, m0 + i);
        }
        __syncthreads();
        if (u.e >= 0 && !skipped(u)) stage1(u);
        __syncthreads();
    }
    for (int iter = 0;; ++iter) {
        const ContractUnit cu = s_u[iter % 3];
        if (cu.e < 0) break;
        const ContractUnit nx = s_u[(iter + 1) % 3];
        const ElemDesc* d = L.desc + cu.e;
        const int gi = cu.gi, gj = cu.gj, t = cu.t, m1a = cu.m1a, m1n = cu.m1n;
        const FfbShape s = ffb_shape(d, gi, gj);
        const int64_t n = d->n;
        const bool skip = skipped(cu);  // uniform: cu is shared
        // the next unit's moments into the moment buffer (stage 1 of cu is done)
        if (nx.e >= 0) {
            const T* gN = reinterpret_cast<const T*>(L.mom) + ffb_moments(L, nx);
            const int cnt = unit_moment_count(L.desc + nx.e, nx.gi, nx.gj);
            for (int i = tid; i < cnt; i += nth) cp_async8(sI + i, gN + i);
        }
        if (!skip) {
            switch (t) {
            case 0: ffb_stage2<A, 0>(sA, sB, s, m1n, tid, nth); break;
            case 1: ffb_stage2<A, 1>(sA, sB, s, m1n, tid, nth); break;
            case 2: ffb_stage2<A, 2>(sA, sB, s, m1n, tid, nth); break;
            default: ffb_stage2<A, 3>(sA, sB, s, m1n, tid, nth); break;
            }
        }
        if (tid == 0) fetch(s_u[(iter + 2) % 3]);  // that slot held unit iter - 1, finished
        cp_async_wait_all();
        __syncthreads();  // stage 2 of cu complete; the moments of nx in place
        // the unit's results are rows [rbase, rbase + m1n Nv_i Nw_i) x columns [col0, col0 + n_j)
        const int rbase = d->dof_off[gi] + m1a * s.Nv_i * s.Nw_i;
        const int col0 = d->dof_off[gj];
        double* Mt = L.out + d->out_off + (int64_t)type_slot_ffb(L.types_mask, t) * n * n + (int64_t)rbase * n + col0;
        double* Mp = cu.tp >= 0 ? L.out + d->out_off + (int64_t)type_slot_ffb(L.types_mask, cu.tp) * n * n +
                                      (int64_t)col0 * n + rbase
                                : nullptr;
        const int ncombo = skip ? 0 : m1n * s.Nv_i * s.mjn;
        const float rmjn = 1.f / (float)s.mjn;
        switch (t) {
        case 0: ffb_stage3<A, 0>(sB, s, ncombo, tid, nth, Mt, Mp, n, rmjn); break;
        case 1: ffb_stage3<A, 1>(sB, s, ncombo, tid, nth, Mt, Mp, n, rmjn); break;
        case 2: ffb_stage3<A, 2>(sB, s, ncombo, tid, nth, Mt, Mp, n, rmjn); break;
        default: ffb_stage3<A, 3>(sB, s, ncombo, tid, nth, Mt, Mp, n, rmjn); break;
        }
        if (nx.e >= 0 && !skipped(nx)) stage1(nx);  // into the stage-1 buffer, read by stage 2 above already
        __syncthreads();  // stage 1 of nx complete; the stage-2 and moment buffers free
    }
}

}  // namespace

bool contract_ffb_fits(const int8_t* Ni, const int8_t* Nj) {
    for (int ax = 0; ax < 3; ++ax)
        if (Ni[ax] < 1 || Ni[ax] > kB || Nj[ax] < 1 || Nj[ax] > kB) return false;
    return true;
}

void contract_ffb_shape(const int8_t* Ni, const int8_t* Nj, int m1n, size_t& a_cap, size_t& s1_cap, size_t& b_cap,
                        int& combos) {
    const int Ku = Ni[0] + Nj[0] - 1, Kv = Ni[1] + Nj[1] - 1, Kw = Ni[2] + Nj[2] - 1;
    a_cap = (size_t)Ku * Kv * Kw;
    s1_cap = (size_t)m1n * Nj[0] * Kv * Kw;
    combos = m1n * Ni[1] * Nj[0] * Nj[1];
    b_cap = (size_t)combos * (Kw | 1);
}

template <class A>
cudaError_t ffb_set_attr() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_contract_ffb<A>);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_contract_ffb<A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

cudaError_t contract_ffb_upload(const void* runs_ff, size_t bytes_ff, const double* runs64, size_t bytes64) {
    if (bytes_ff != sizeof(c_runs) || bytes64 != sizeof(c_runs64)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbol(c_runs, runs_ff, bytes_ff);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_runs64, runs64, bytes64);
    if (e == cudaSuccess) e = ffb_set_attr<ArithFF>();
    if (e == cudaSuccess) e = ffb_set_attr<ArithF64>();
    return e;
}

cudaError_t launch_contract_ffb(int precision, const ContractLaunch& L, int grid, int threads, size_t smem,
                                cudaStream_t s) {
    if (threads < 32 || threads > 512 || threads % 32) return cudaErrorInvalidValue;
    if (precision == P2S_MIXED)
        k_contract_ffb<ArithFF><<<grid, threads, smem, s>>>(L);
    else
        k_contract_ffb<ArithF64><<<grid, threads, smem, s>>>(L);
    return cudaGetLastError();
}

int contract_ffb_blocks_per_sm(int precision, int threads, size_t smem) {
    int nb = 0;
    const cudaError_t e =
        precision == P2S_MIXED ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_contract_ffb<ArithFF>, threads, smem)
                               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_contract_ffb<ArithF64>, threads, smem);
    return e == cudaSuccess ? nb : 0;
}

}  // namespace p2s
