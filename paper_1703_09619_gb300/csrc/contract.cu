// Step a4: the product-to-sum contraction of Eq. (4) of arXiv:1703.09619,
//   M_t[(m1,n1,p1),(m2,n2,p2)] = sum_{k,l,q} C_t[m1,m2,k] C_t[n1,n2,l] C_t[p1,p2,q] I[k,l,q],
// with the Eq. (3) linearisation coefficients C_t stored as runs k = kmin, kmin+2, ...
//
// One CTA per work unit = (element, block (gi,gj), type t, m1-slab, n1-slab):
//   stage 1  A[m1][m2][l][q]        = sum_k C_t[m1,m2,k] I[k][l][q]
//   stage 2  Bt[m1][n1][m2][n2][q]  = sum_l C_t[n1,n2,l] A[m1][m2][l][q]
//   stage 3  tile[(m1,n1,p1)][(m2,n2,p2)] = sum_q C_t[p1,p2,q] Bt[m1][n1][m2][n2][q]
// Stage 3 takes items (p1, combination (m1,n1,m2,n2)) with p1 outermost, so the lanes of a
// warp share p1 and walk p2 in step: the coefficient runs are uniform across the warp.  The
// tile is staged in shared memory with the columns of a row ordered p2-major (consecutive
// lanes store consecutive doubles; odd strides keep the write-out reads conflict-free), and
// it leaves twice, both times as contiguous row segments:
//   - as rows of M_t(gi,gj), and
//   - transposed, as rows of the partner block M_t'(gj,gi) = M_t(gi,gj)^T, where
//     t' = t for vv and dd (alpha symmetric) and t' = vd for t = dv.
// The host builds the unit list so that every block is computed once and written to
// both places.
//
// Two arithmetics share the structure:
//   FP64   - every operation in FP64;
//   mixed  - float-float (hi + lo FP32 pairs) products and sums with exact FMA product
//            errors and TwoSum accumulation; moments arrive as (hi, lo) pairs; the FP64
//            output bits are assembled from (hi, lo) with integer operations, so the hot
//            loop issues no FP64 instruction (FP64 runs at 1/58 of FP32 on this part).
#include <type_traits>

#include "arith.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

__device__ __forceinline__ int type_slot(uint32_t mask, int t) { return __popc(mask & ((1u << t) - 1u)); }

template <class A>
__global__ void __launch_bounds__(512) k_contract(ContractLaunch L) {
    using T = typename A::T;
    constexpr bool kFP64 = sizeof(T) == sizeof(double) && alignof(T) == alignof(double) &&
                           !std::is_same<T, float2>::value;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sA = reinterpret_cast<T*>(smraw);
    T* sB = sA + L.a_cap;
    double* tile = reinterpret_cast<double*>(smraw + L.tile_off);
    uint32_t* s_cmb = reinterpret_cast<uint32_t*>(smraw + L.combo_off);  // im1 | in1 << 8 | m2 << 16 | n2 << 24
    int32_t* s_cli = reinterpret_cast<int32_t*>(s_cmb + L.combo_cap);     // stage-2 run of (n1, n2)
    __shared__ ContractUnit cu;
    __shared__ unsigned long long unit_id;
    __shared__ int32_t s_lin[kMaxOrder * kMaxOrder];
    __shared__ int16_t s_col[kMaxOrder * kMaxOrder * kMaxOrder];  // tile offset of output column c
    __shared__ typename A::C s_coef[kMaxOrder * kMaxOrder * kMaxOrder];  // stage-3 runs, [p1][p2][r]
    const int tid = threadIdx.x, nth = blockDim.x;
    const int32_t* __restrict__ lidx = L.lin_idx;
    const void* lcoef = L.lin_coef;

    for (;;) {
        if (tid == 0) {
            unit_id = atomicAdd(L.counter, 1ull);
            if (unit_id < (unsigned long long)L.n_units) cu = L.units[unit_id];
        }
        __syncthreads();
        if (unit_id >= (unsigned long long)L.n_units) break;
        if (L.elem_mask && !L.elem_mask[cu.e]) {  // every thread reads cu before tid 0 refills it
            __syncthreads();
            continue;
        }
        const ElemDesc* d = L.desc + cu.e;
        const int gi = cu.gi, gj = cu.gj, t = cu.t;
        const int m1a = cu.m1a, m1n = cu.m1n, n1a = cu.n1a, n1n = cu.n1n;
        const int Nv_i = d->ord[gi][1], Nw_i = d->ord[gi][2];
        const int Nu_j = d->ord[gj][0], Nv_j = d->ord[gj][1], Nw_j = d->ord[gj][2];
        const int Kv = Nv_i + Nv_j - 1, Kw = Nw_i + Nw_j - 1;
        const int Kwp = Kw | 1;  // stage-2 row stride: odd, so stage 3's row reads spread over banks
        const int Nwm = max(Nw_i, Nw_j);  // s_coef run stride
        const int n = d->n;
        const int nj = Nu_j * Nv_j * Nw_j;
        const int mjp = contract_mj_stride(Nu_j * Nv_j);
        const int ld = contract_tile_ld(Nu_j * Nv_j, Nw_j);  // padded tile row stride (doubles)
        const float rNwj = 1.f / (float)Nw_j, rNwm = 1.f / (float)Nwm;
        for (int c = tid; c < nj; c += nth) {
            const int mj = div_small(c, Nw_j, rNwj);
            s_col[c] = (int16_t)((c - mj * Nw_j) * mjp + mj);
        }
        // every combination (m1, n1, m2, n2) of the unit, decoded once: c = mn * mjn + mj with
        // mn = im1 * n1n + in1, mj = m2 * Nv_j + n2
        const int ncombo = m1n * n1n * Nu_j * Nv_j;
        const int mjn = Nu_j * Nv_j;
        {
            const float rmjn = 1.f / (float)mjn, rn1n = 1.f / (float)n1n, rNvj = 1.f / (float)Nv_j;
            for (int c = tid; c < ncombo; c += nth) {
                const int mn = div_small(c, mjn, rmjn), mj = c - mn * mjn;
                const int im1 = div_small(mn, n1n, rn1n), in1 = mn - im1 * n1n;
                const int m2 = div_small(mj, Nv_j, rNvj), n2 = mj - m2 * Nv_j;
                s_cmb[c] = (uint32_t)im1 | ((uint32_t)in1 << 8) | ((uint32_t)m2 << 16) | ((uint32_t)n2 << 24);
            }
        }
        // The terms summed into this block: the single uniform type t, or the operator's list
        // (per-axis types, coupling entry, scale); each term is stages 1-3 with its own runs,
        // stage 3 adding its share to the staged tile.
        const bool op = L.op_terms != nullptr;
        const int bslot = 2 * (3 * gi + gj);
        const int term0 = op ? L.op_block[bslot] : 0, n_terms = op ? L.op_block[bslot + 1] : 1;
        const int Kvm = op ? d->kax[1] : Kv, Kwm = op ? d->kax[2] : Kw;  // moment tensor extents
        const int KvKwm = Kvm * Kwm;
        for (int kt = 0; kt < n_terms; ++kt) {
            int tu = t, tv = t, tw = t, sp = pair_index(gi, gj, d->n_comp);
            double scale = 1.0;
            if (op) {
                const int32_t pk = __ldg(L.op_terms + term0 + kt);
                const int sa = pk & 15, sb = (pk >> 4) & 15;
                tu = (pk >> 8) & 15;
                tv = (pk >> 12) & 15;
                tw = (pk >> 16) & 15;
                sp = pair_index(sa, sb, L.op_nalpha);
                scale = __ldg(L.op_scales + term0 + kt);
            }
            const size_t moff = d->mom_off + d->pair_off[sp];
            // the scale, tested and split once per term (FP64 work runs on a narrow pipe)
            const bool rescale = op && scale != 1.0;
            const float scale_hi = (float)scale, scale_lo = (float)(scale - (double)scale_hi);
            // the term's stage-3 coefficient runs (type tw) and stage-2 runs per combination (tv)
            if (tid < Nw_i * Nw_j) {
                const int p1 = div_small(tid, Nw_j, rNwj);
                s_lin[tid] = __ldg(lidx + lin_slot(tw, p1, tid - p1 * Nw_j));
            }
            for (int i = tid; i < Nw_i * Nw_j * Nwm; i += nth) {  // the runs' coefficient values
                const int pp = div_small(i, Nwm, rNwm), r = i - pp * Nwm;
                const int p1 = div_small(pp, Nw_j, rNwj);
                const int32_t li = __ldg(lidx + lin_slot(tw, p1, pp - p1 * Nw_j));
                if (r < lin_cnt(li)) s_coef[i] = A::load_coef(lcoef, lin_off(li) + r);
            }
            for (int c = tid; c < ncombo; c += nth) {
                const uint32_t w = s_cmb[c];
                s_cli[c] = __ldg(lidx + lin_slot(tv, n1a + (int)((w >> 8) & 0xffu), (int)(w >> 24)));
            }

            // stage 1: A[m1][m2][l][q], m1 in the slab
            const int KvKw = Kv * Kw;
            const int nA = m1n * Nu_j * KvKw;
            const float rKvKw = 1.f / (float)KvKw, rNuj = 1.f / (float)Nu_j, rKw1 = 1.f / (float)Kw;
            for (int idx = tid; idx < nA; idx += nth) {
                const int mm = div_small(idx, KvKw, rKvKw), lq = idx - mm * KvKw;
                const int im1 = div_small(mm, Nu_j, rNuj), m2 = mm - im1 * Nu_j;
                const int l = div_small(lq, Kw, rKw1), q = lq - l * Kw;
                const int32_t li = __ldg(lidx + lin_slot(tu, m1a + im1, m2));
                const int k0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
                const size_t mb = moff + (size_t)k0 * KvKwm + (size_t)l * Kwm + q;
                T acc = cnt > 0 ? A::mul(A::load_coef(lcoef, off), A::load_moment(L.mom, mb)) : A::zero();
                for (int r = 1; r < cnt; ++r)
                    A::fma_acc(acc, A::load_coef(lcoef, off + r), A::load_moment(L.mom, mb + (size_t)(2 * r) * KvKwm));
                sA[idx] = A::finish(acc);
            }
            __syncthreads();
            // stage 2: Bt[m1][n1][m2][n2][q], (m1, n1) in the slab
            const int nB = ncombo * Kw;
            const float rKw = 1.f / (float)Kw;
            for (int idx = tid; idx < nB; idx += nth) {
                const int c = div_small(idx, Kw, rKw), q = idx - c * Kw;
                const uint32_t w = s_cmb[c];
                const int im1 = w & 0xffu, m2 = (w >> 16) & 0xffu;
                const int32_t li = s_cli[c];
                const int l0 = lin_kmin(li), cnt = lin_cnt(li), off = lin_off(li);
                const T* a = sA + ((im1 * Nu_j + m2) * Kv + l0) * Kw + q;
                T acc = cnt > 0 ? A::mul(A::load_coef(lcoef, off), a[0]) : A::zero();
                for (int r = 1; r < cnt; ++r) A::fma_acc(acc, A::load_coef(lcoef, off + r), a[2 * r * Kw]);
                sB[c * Kwp + q] = A::finish(acc);
            }
            __syncthreads();
            // stage 3: items (p1, combination (m1, n1, m2, n2)); each walks p2
            const float rncombo = 1.f / (float)ncombo;
            for (int it = tid; it < ncombo * Nw_i; it += nth) {
                const int p1 = div_small(it, ncombo, rncombo), c = it - p1 * ncombo;
                const uint32_t w = s_cmb[c];
                const int mn = (int)(w & 0xffu) * n1n + (int)((w >> 8) & 0xffu);       // im1 * n1n + in1
                const int mj = (int)((w >> 16) & 0xffu) * Nv_j + (int)(w >> 24);      // m2 * Nv_j + n2
                const T* bt = sB + (size_t)c * Kwp;
                double* trow = tile + (size_t)(mn * Nw_i + p1) * ld + mj;
                const int32_t* lrow = s_lin + p1 * Nw_j;
                const typename A::C* crow = s_coef + p1 * Nw_j * Nwm;
                for (int p2 = 0; p2 < Nw_j; ++p2) {
                    const int32_t li = lrow[p2];
                    const int q0 = lin_kmin(li), cnt = lin_cnt(li);
                    const typename A::C* cf = crow + p2 * Nwm;
                    T acc = cnt > 0 ? A::mul(cf[0], bt[q0]) : A::zero();
                    for (int r = 1; r < cnt; ++r) A::fma_acc(acc, cf[r], bt[q0 + 2 * r]);
                    if (!op) {
                        trow[p2 * mjp] = A::to_double_fast(A::finish(acc));
                    } else if constexpr (kFP64) {  // operator terms: FP64 sums in the tile
                        const double v = A::finish(acc);
                        trow[p2 * mjp] = kt == 0 ? scale * v : fma(scale, v, trow[p2 * mjp]);
                    } else {  // float-float: the terms add in the tile, converted once at the end
                        T* tr = reinterpret_cast<T*>(trow + p2 * mjp);
                        T v = A::finish(acc);
                        if (rescale) v = A::scaled(v, scale, scale_hi, scale_lo);
                        *tr = kt == 0 ? v : A::add(*tr, v);
                    }
                }
            }
            __syncthreads();
        }
        // The slabs the host builds are either full in n1 or a single m1, so the tile's rows
        // (m1, n1, p1) are consecutive dofs: rows [rbase, rbase + rows) of block (gi, gj).
        const int rows = m1n * n1n * Nw_i;
        if (n_terms == 0) {  // an operator block without terms is zero
            for (int i = tid; i < rows * ld; i += nth) tile[i] = 0.0;
            __syncthreads();
        } else if (op && !kFP64 && !L.out_ff) {  // the summed terms to FP64, once per entry, in place
            const T* tT = reinterpret_cast<const T*>(tile);
            for (int i = tid; i < rows * ld; i += nth) tile[i] = A::to_double_fast(tT[i]);
            __syncthreads();
        }
        const int rbase = d->dof_off[gi] + (m1a * Nv_i + n1a) * Nw_i;
        const int col0 = d->dof_off[gj];
        const int warp = tid >> 5, lane = tid & 31, nwarp = nth >> 5;
        // write-out 1: one warp per tile row, lanes along the row of M_t(gi, gj)
        double* Mt = L.out + d->out_off + (int64_t)type_slot(L.types_mask, t) * n * n + col0;
        for (int r = warp; r < rows; r += nwarp) {
            double* dst = Mt + (int64_t)(rbase + r) * n;
            const double* src = tile + (size_t)r * ld;
            for (int c = lane; c < nj; c += 32) __stcs(dst + c, src[s_col[c]]);
        }
        // write-out 2: the transpose, one warp per row of the partner block (gj, gi)
        if (cu.tp >= 0) {
            double* Mp = L.out + d->out_off + (int64_t)type_slot(L.types_mask, cu.tp) * n * n + rbase;
            for (int c = warp; c < nj; c += nwarp) {
                double* dst = Mp + (int64_t)(col0 + c) * n;
                const double* src = tile + s_col[c];
                for (int r = lane; r < rows; r += 32) __stcs(dst + r, src[(size_t)r * ld]);
            }
        }
        __syncthreads();
    }
}

cudaError_t set_max_smem(const void* f) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace

ContractShape contract_shape(const int8_t* Ni, const int8_t* Nj, int m1n, int n1n) {
    ContractShape s;
    const int Kv = Ni[1] + Nj[1] - 1, Kw = Ni[2] + Nj[2] - 1;
    s.a = (size_t)m1n * Nj[0] * Kv * Kw;
    s.b = (size_t)m1n * n1n * Nj[0] * Nj[1] * (Kw | 1);
    s.tile = (size_t)m1n * n1n * Ni[2] * contract_tile_ld(Nj[0] * Nj[1], Nj[2]);
    s.combos = m1n * n1n * Nj[0] * Nj[1];
    return s;
}

size_t contract_tile_offset(int precision, size_t a_cap, size_t b_cap) {
    size_t el = precision == P2S_MIXED ? sizeof(float2) : sizeof(double);
    return ((a_cap + b_cap) * el + 15) & ~(size_t)15;
}

size_t contract_combo_offset(int precision, size_t a_cap, size_t b_cap, size_t tile_cap) {
    return contract_tile_offset(precision, a_cap, b_cap) + tile_cap * sizeof(double);
}

size_t contract_smem_bytes(int precision, size_t a_cap, size_t b_cap, size_t tile_cap, size_t combo_cap) {
    return contract_combo_offset(precision, a_cap, b_cap, tile_cap) + 2 * sizeof(uint32_t) * combo_cap;
}

cudaError_t launch_contract(int precision, const ContractLaunch& L, int grid, int threads, size_t smem,
                            cudaStream_t s) {
    if (threads < 32 || threads > 512 || threads % 32) return cudaErrorInvalidValue;
    if (precision == P2S_MIXED)
        k_contract<ArithFF><<<grid, threads, smem, s>>>(L);
    else
        k_contract<ArithF64><<<grid, threads, smem, s>>>(L);
    return cudaGetLastError();
}

int contract_blocks_per_sm(int precision, int threads, size_t smem) {
    int n = 0;
    cudaError_t e = precision == P2S_MIXED
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_contract<ArithFF>, threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_contract<ArithF64>, threads, smem);
    return e == cudaSuccess ? n : 0;
}

cudaError_t contract_init_attributes() {
    cudaError_t e = set_max_smem((const void*)k_contract<ArithF64>);
    if (e != cudaSuccess) return e;
    return set_max_smem((const void*)k_contract<ArithFF>);
}

}  // namespace p2s
