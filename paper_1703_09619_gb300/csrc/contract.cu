// Step a4: the product-to-sum contraction of Eq. (4) of arXiv:1703.09619,
//   M_t[(m1,n1,p1),(m2,n2,p2)] = sum_{k,l,q} C_t[m1,m2,k] C_t[n1,n2,l] C_t[p1,p2,q] I[k,l,q],
// with the Eq. (3) linearisation coefficients C_t stored as runs k = kmin, kmin+2, ...
// Three sparse mode products, one warp per work unit (element, block (gi,gj), type t,
// test index m1):
//   stage 1  A[m2][l][q]  = sum_k C_t[m1,m2,k] I[k][l][q]           (moments read from L2)
//   stage 2  Bt[m2][n2][q] = sum_l C_t[n1,n2,l] A[m2][l][q]          (per n1)
//   stage 3  M[(m1,n1,p1),(m2,n2,p2)] = sum_q C_t[p1,p2,q] Bt[m2][n2][q]
// Stage 3 gives each lane one (m2,n2) and walks (p1,p2) in the same order on every lane,
// so the coefficient runs are warp-uniform; a lane's Nw_j outputs of a row go through a
// per-warp staging row and leave as one contiguous, coalesced span.
// Plain path: every operation in FP64.
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kWarpsPerCta = 8;

__device__ __forceinline__ int type_slot(uint32_t mask, int t) { return __popc(mask & ((1u << t) - 1u)); }

__global__ void __launch_bounds__(kWarpsPerCta * 32) k_contract_fp64(ContractLaunch L) {
    extern __shared__ double sm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t wd = contract_warp_doubles(L.nmax, L.kmax);
    double* A = sm + wid * wd;
    double* Bt = A + (size_t)L.nmax * L.kmax * L.kmax;
    double* stg = Bt + (size_t)L.nmax * L.nmax * L.kmax;
    const int32_t* __restrict__ lidx = L.lin_idx;
    const double* __restrict__ lcoef = L.lin_coef;

    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(L.counter, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= (unsigned long long)L.n_units) break;
        const ContractUnit cu = L.units[u];
        const ElemDesc* d = L.desc + cu.e;
        const int gi = cu.gi, gj = cu.gj, t = cu.t, m1 = cu.m1;
        const int Nv_i = d->ord[gi][1], Nw_i = d->ord[gi][2];
        const int Nu_j = d->ord[gj][0], Nv_j = d->ord[gj][1], Nw_j = d->ord[gj][2];
        const int Kv = Nv_i + Nv_j - 1, Kw = Nw_i + Nw_j - 1;
        const int n = d->n;
        const double* __restrict__ I = L.mom + d->mom_off + d->pair_off[pair_index(gi, gj, d->n_comp)];
        double* Mt = L.out + d->out_off + (int64_t)type_slot(L.types_mask, t) * n * n;

        // stage 1
        const int KvKw = Kv * Kw;
        for (int idx = lane; idx < Nu_j * KvKw; idx += 32) {
            const int m2 = idx / KvKw, lq = idx - m2 * KvKw;
            const int32_t li = __ldg(lidx + lin_slot(t, m1, m2));
            const int k0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
            double acc = 0.0;
            for (int r = 0; r < cnt; ++r) acc = fma(__ldg(lcoef + off + r), __ldg(I + (k0 + 2 * r) * KvKw + lq), acc);
            A[idx] = acc;
        }
        __syncwarp();
        const int NvKw = Nv_j * Kw;
        const int ncombo = Nu_j * Nv_j;
        for (int n1 = 0; n1 < Nv_i; ++n1) {
            // stage 2
            for (int idx = lane; idx < Nu_j * NvKw; idx += 32) {
                const int m2 = idx / NvKw, r2 = idx - m2 * NvKw, n2 = r2 / Kw, q = r2 - n2 * Kw;
                const int32_t li = __ldg(lidx + lin_slot(t, n1, n2));
                const int l0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
                const double* a = A + (m2 * Kv + l0) * Kw + q;
                double acc = 0.0;
                for (int r = 0; r < cnt; ++r) acc = fma(__ldg(lcoef + off + r), a[2 * r * Kw], acc);
                Bt[idx] = acc;
            }
            __syncwarp();
            // stage 3
            for (int p1 = 0; p1 < Nw_i; ++p1) {
                const int row = d->dof_off[gi] + (m1 * Nv_i + n1) * Nw_i + p1;
                double* rowp = Mt + (int64_t)row * n + d->dof_off[gj];
                for (int cb = 0; cb < ncombo; cb += 32) {
                    const int combo = cb + lane;
                    if (combo < ncombo) {
                        const double* bt = Bt + combo * Kw;
                        for (int p2 = 0; p2 < Nw_j; ++p2) {
                            const int32_t li = __ldg(lidx + lin_slot(t, p1, p2));
                            const int q0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
                            double acc = 0.0;
                            for (int r = 0; r < cnt; ++r) acc = fma(__ldg(lcoef + off + r), bt[q0 + 2 * r], acc);
                            stg[lane * Nw_j + p2] = acc;
                        }
                    }
                    __syncwarp();
                    const int span = min(32, ncombo - cb) * Nw_j;
                    double* dst = rowp + cb * Nw_j;
                    for (int x = lane; x < span; x += 32) dst[x] = stg[x];
                    __syncwarp();
                }
            }
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_contract_fp64(const ContractLaunch& L, int grid, int warps_per_cta, size_t smem, cudaStream_t s) {
    if (warps_per_cta < 1 || warps_per_cta > kWarpsPerCta) return cudaErrorInvalidValue;
    k_contract_fp64<<<grid, warps_per_cta * 32, smem, s>>>(L);
    return cudaGetLastError();
}

int contract_max_warps_per_cta() { return kWarpsPerCta; }

int contract_blocks_per_sm(int warps, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_contract_fp64, warps * 32, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t contract_init_attributes() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_contract_fp64);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_contract_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace p2s
