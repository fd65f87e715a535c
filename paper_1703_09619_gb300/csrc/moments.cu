// Steps a1 + a2: coupling factor at the Gauss-Legendre points and the moment tensors
//   I_s[k,l,q] = sum_{a,b,c} w_a w_b w_c P_k(u_a) P_l(v_b) P_q(w_c) alpha_s(u_a,v_b,w_c)
// of Eq. (4) of arXiv:1703.09619 ("starting-point" integrals; Eq. (19) is the 2-D case),
// sum-factorised as three mode products with B[k][a] = w_a P_k(x_a):
//   T1[k][b]   = sum_a B[k][a] alpha[a,b,c]        (per w-plane c, in chunks of b)
//   T2[k][l]  += sum_b B[l][b] T1[k][b]
//   I[k][l][q] += B[q][c] T2[k][l]
// alpha (Eq. (2) coupling factor) is evaluated in shared memory chunk by chunk and never
// reaches global memory.  One CTA owns one element at a time (persistent loop).
// Plain path: every operation in FP64.
#include <cmath>

#include "alpha.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;  // alpha points per chunk
constexpr int kNB = 16;      // max b-rows per chunk: min(G, 256/G) <= 16
constexpr int kGeo = 48;

__device__ __forceinline__ void pair_comps(int s, int n_comp, int& gi, int& gj) {
    if (n_comp == 1) { gi = gj = 0; return; }
    const int tgi[6] = {0, 0, 0, 1, 1, 2}, tgj[6] = {0, 1, 2, 1, 2, 2};
    gi = tgi[s];
    gj = tgj[s];
}

struct Smem {
    double *B, *xq, *t0, *t1, *t2, *alpha, *T1, *T2, *Iacc, *geo;
};

__device__ __forceinline__ Smem carve(double* sm, int n_pairs, int kb, int gmax, int iacc_cap) {
    Smem S;
    S.B = sm;
    S.xq = S.B + kb * (gmax | 1);  // B rows padded to an odd stride (bank spread)
    S.t0 = S.xq + gmax;
    S.t1 = S.t0 + gmax;
    S.t2 = S.t1 + gmax;
    S.alpha = S.t2 + gmax;
    S.T1 = S.alpha + n_pairs * kChunk;
    S.T2 = S.T1 + n_pairs * kb * kNB;
    S.Iacc = S.T2 + n_pairs * kb * kb;
    S.geo = S.Iacc + iacc_cap;
    return S;
}

// One element's moments (kPart false), or one part of them (kPart true): the w-planes c in
// [part G / nparts, (part + 1) G / nparts).  Whole elements, and parts with slot == nullptr
// (nparts 1), store the pairs' sub-tensors in L.mom and write the element status; otherwise the
// accumulator of every pair goes to slot[pair * slot_stride + i] for the split reduction, and a
// Jacobian failure only raises the error flag.  tid is threadIdx.x, gstride the B rows' stride
// (gmax | 1), bad_jac the CTA's shared Jacobian flag.
template <bool kPart>
__device__ __forceinline__ void element_moments(const MomentLaunch& L, const Smem& S, int64_t e, int part, int nparts,
                                                double* slot, int64_t slot_stride, const int tid, const int gstride,
                                                int& bad_jac) {
    const ElemDesc& d = L.desc[e];
    const int G = d.G, nc = d.n_comp, np = (nc == 1) ? 1 : 6;
    const int Ku = d.kax[0], Kv = d.kax[1], Kw = d.kax[2];
    const int Kb = max(Ku, max(Kv, Kw));
    if (tid == 0) bad_jac = 0;
    // 1-D tables: nodes, B[k][a] = w_a P_k(x_a), per-axis factors
    if (tid < G) {
        double x = L.gl_x[G * kMaxG + tid], w = L.gl_w[G * kMaxG + tid];
        S.xq[tid] = x;
        double p0 = 1.0, p1 = x;
        S.B[0 * gstride + tid] = w;
        if (Kb > 1) S.B[1 * gstride + tid] = w * x;
        for (int k = 1; k + 1 < Kb; ++k) {
            double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
            S.B[(k + 1) * gstride + tid] = w * p2;
            p0 = p1;
            p1 = p2;
        }
        const double* p = L.params + 4 * e;
        if (L.kind == P2S_ALPHA_SCALAR) {
            const double pi = 3.141592653589793;
            S.t0[tid] = p[0] * sin(pi * (x + p[1]));
            S.t1[tid] = cos(pi * (x + p[2]));
            S.t2[tid] = exp(p[3] * x);
        } else {
            double sx, cx;
            sincos(1.5707963267948966 * x, &sx, &cx);
            S.t0[tid] = cx;
            S.t1[tid] = sx;
        }
    }
    if (L.kind == P2S_ALPHA_METRIC_EPS && tid < 3) {
        // trilinear coefficients of coordinate i: x_i = sum_j c_ij * (1,u,v,w,uv,uw,vw,uvw)_j
        const double* X = L.nodes + 24 * e;
        double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int nd = 0; nd < 8; ++nd) {
            double su = (nd & 1) ? 1.0 : -1.0, sv = (nd & 2) ? 1.0 : -1.0, sw = (nd & 4) ? 1.0 : -1.0;
            double xv = 0.125 * X[3 * nd + tid];
            c[0] += xv; c[1] += su * xv; c[2] += sv * xv; c[3] += sw * xv;
            c[4] += su * sv * xv; c[5] += su * sw * xv; c[6] += sv * sw * xv; c[7] += su * sv * sw * xv;
        }
        for (int j = 0; j < 8; ++j) S.geo[8 * tid + j] = c[j];
        const double* bg = L.bulge ? L.bulge + 4 * e : nullptr;
        S.geo[24 + tid] = bg ? bg[0] * bg[1 + tid] : 0.0;
    }
    __syncthreads();
    if (L.kind == P2S_ALPHA_METRIC_EPS && tid < 8) {
        const double* p = L.params + 4 * e;
        // phase theta = k . x as trilinear coefficients plus k . (a b) for the bulge
        S.geo[31 + tid] = p[1] * S.geo[tid] + p[2] * S.geo[8 + tid] + p[3] * S.geo[16 + tid];
        if (tid == 0) {
            S.geo[27] = p[0];
            S.geo[39] = p[1] * S.geo[24] + p[2] * S.geo[25] + p[3] * S.geo[26];
        }
    }
    __syncthreads();

    const int per_pair = Ku * Kv * Kw;
    const int ppg = max(1, min(np, L.iacc_cap / per_pair));
    const int nb = max(1, min(G, kChunk / G));
    const int c_begin = kPart ? part * G / nparts : 0, c_end = kPart ? (part + 1) * G / nparts : G;
    for (int s0 = 0; s0 < np; s0 += ppg) {
        const int ns = min(np, s0 + ppg) - s0;
        for (int i = tid; i < ns * per_pair; i += kThreads) S.Iacc[i] = 0.0;
        for (int c = c_begin; c < c_end; ++c) {
            for (int i = tid; i < ns * Ku * Kv; i += kThreads) S.T2[i] = 0.0;
            for (int b0 = 0; b0 < G; b0 += nb) {
                const int nbc = min(nb, G - b0);
                const int npts = nbc * G;
                // phase A: alpha at (a, b0 + bb, c)
                if (tid < npts) {
                    const int bb = tid / G, a = tid - bb * G, b = b0 + bb;
                    if (L.kind == P2S_ALPHA_SCALAR) {
                        S.alpha[tid] = fma(S.t0[a] * S.t1[b], S.t2[c], 1.0);
                    } else {
                        double K[6];
                        bool ok = metric_alpha(S.geo, S.xq[a], S.xq[b], S.xq[c], S.t0[a], S.t1[a], S.t0[b],
                                               S.t1[b], S.t0[c], S.t1[c], K);
                        if (!ok) bad_jac = 1;
                        for (int s = 0; s < ns; ++s) S.alpha[s * kChunk + tid] = K[s0 + s];
                    }
                }
                __syncthreads();
                // phase B: T1[s][bb][k] = sum_a B[k][a] alpha[s][bb*G + a]; k fastest across
                // threads, so the alpha reads are broadcasts and the B rows (odd stride) spread
                for (int i = tid; i < ns * nbc * Ku; i += kThreads) {
                    const int sb = i / Ku, k = i - sb * Ku, s = sb / nbc, bb = sb - s * nbc;
                    const double* al = S.alpha + s * kChunk + bb * G;
                    const double* Bk = S.B + k * gstride;
                    double acc = 0.0;
                    for (int a = 0; a < G; ++a) acc = fma(Bk[a], al[a], acc);
                    S.T1[(s * kNB + bb) * Kb + k] = acc;
                }
                __syncthreads();
                // phase C: T2[s][k][l] += sum_bb B[l][b0+bb] T1[s][bb][k]
                for (int i = tid; i < ns * Ku * Kv; i += kThreads) {
                    const int s = i / (Ku * Kv), r = i - s * Ku * Kv, k = r / Kv, l = r - k * Kv;
                    const double* t1 = S.T1 + s * kNB * Kb + k;
                    const double* Bl = S.B + l * gstride + b0;
                    double acc = S.T2[i];
                    for (int bb = 0; bb < nbc; ++bb) acc = fma(Bl[bb], t1[bb * Kb], acc);
                    S.T2[i] = acc;
                }
                __syncthreads();
            }
            // phase D: I[s][k][l][q] += B[q][c] T2[s][k][l]
            for (int i = tid; i < ns * per_pair; i += kThreads) {
                const int skl = i / Kw, q = i - skl * Kw;
                S.Iacc[i] = fma(S.B[q * gstride + c], S.T2[skl], S.Iacc[i]);
            }
            __syncthreads();
        }
        if (kPart && slot) {  // a part of a split element: its whole accumulator, summed later
            for (int i = tid; i < ns * per_pair; i += kThreads) {
                const int s = i / per_pair;
                slot[(int64_t)(s0 + s) * slot_stride + (i - s * per_pair)] = S.Iacc[i];
            }
        } else {
            // store each pair's own sub-tensor (K_axis = N_i + N_j - 1 <= element-wide K)
            for (int s = 0; s < ns; ++s) {
                int gi, gj;
                pair_comps(s0 + s, nc, gi, gj);
                const int ku = d.ord[gi][0] + d.ord[gj][0] - 1, kv = d.ord[gi][1] + d.ord[gj][1] - 1,
                          kw = d.ord[gi][2] + d.ord[gj][2] - 1;
                double* dst = L.mom + d.mom_off + d.pair_off[s0 + s];
                const double* src = S.Iacc + s * per_pair;
                for (int i = tid; i < ku * kv * kw; i += kThreads) {
                    const int k = i / (kv * kw), r = i - k * kv * kw, l = r / kw, q = r - l * kw;
                    const double v = src[(k * Kv + l) * Kw + q];
                    if (L.out_ff) {
                        const float hi = (float)v;
                        reinterpret_cast<float2*>(dst)[i] = make_float2(hi, (float)(v - (double)hi));
                    } else {
                        dst[i] = v;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (!(kPart && slot) && L.elem_status) L.elem_status[e] = bad_jac ? P2S_ERR_JACOBIAN : P2S_OK;
        if (bad_jac && L.err_flag) atomicCAS(L.err_flag, 0, P2S_ERR_JACOBIAN);
    }
}

__global__ void __launch_bounds__(kThreads) k_moments_fp64(MomentLaunch L) {
    extern __shared__ double sm[];
    const int tid = threadIdx.x;
    Smem S = carve(sm, L.n_pairs, L.kb, L.gmax, L.iacc_cap);
    __shared__ int bad_jac;
    const int gstride = L.gmax | 1;

    __shared__ long long s_elem;
    for (int64_t es = blockIdx.x;; es += gridDim.x) {
        int64_t e = es;
        if (L.counter) {  // dynamic element queue: the next element to whichever CTA is free
            __syncthreads();
            if (threadIdx.x == 0) s_elem = (long long)atomicAdd(L.counter, 1ull);
            __syncthreads();
            e = s_elem;
        }
        if (e < L.n_elem && L.order) e = L.order[e];
        if (e >= L.n_elem) break;
        if (L.elem_mask && !L.elem_mask[e]) continue;  // uniform across the CTA
        element_moments<false>(L, S, e, 0, 1, nullptr, 0, tid, gstride, bad_jac);
        __syncthreads();
    }
}

// Parts per listed element of a split launch: as many as keep every part on its own CTA,
// at most one w-plane each.  n * parts <= grid whenever parts > 1.
__device__ __forceinline__ int split_parts(int n, int grid, int gmax) { return max(1, min(gmax, grid / max(n, 1))); }

// The listed elements (Sp.list[0 .. *Sp.count)), each cut into split_parts() parts of its
// w-planes, one part per CTA: a few elements spread over the whole GPU instead of one CTA
// each.  With a single part per element the pairs' sub-tensors are stored directly.
__global__ void __launch_bounds__(kThreads) k_moments_fp64_split(MomentLaunch L, MomentSplit Sp) {
    extern __shared__ double sm[];
    Smem S = carve(sm, L.n_pairs, L.kb, L.gmax, L.iacc_cap);
    __shared__ int bad_jac;
    const int n = *Sp.count;
    if (n <= 0) return;
    const int P = split_parts(n, Sp.grid, L.gmax);
    const int64_t kb3 = (int64_t)L.kb * L.kb * L.kb;
    for (int64_t it = blockIdx.x; it < (int64_t)n * P; it += gridDim.x) {
        const int64_t k = it / P;
        const int part = (int)(it - k * P);
        const int64_t e = Sp.list[k];
        if (e < 0 || e >= L.n_elem) continue;  // uniform across the CTA
        double* slot = P > 1 ? Sp.part + it * L.n_pairs * kb3 : nullptr;
        element_moments<true>(L, S, e, part, P, slot, kb3, threadIdx.x, L.gmax | 1, bad_jac);
        __syncthreads();
    }
}

// Sum of each split element's parts, in part order, into the pairs' sub-tensors of L.mom
// (FP64).  Nothing to do when the launch kept whole elements.
__global__ void __launch_bounds__(256) k_moments_split_reduce(MomentLaunch L, MomentSplit Sp) {
    const int n = *Sp.count;
    if (n <= 0) return;
    const int P = split_parts(n, Sp.grid, L.gmax);
    if (P == 1) return;
    const int64_t kb3 = (int64_t)L.kb * L.kb * L.kb, per_elem = L.n_pairs * kb3;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (int64_t)n * per_elem;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = g / per_elem;
        const int64_t r = g - k * per_elem;
        const int s = (int)(r / kb3), i = (int)(r - s * kb3);
        const int64_t e = Sp.list[k];
        if (e < 0 || e >= L.n_elem) continue;
        const ElemDesc& d = L.desc[e];
        const int nc = d.n_comp, np = (nc == 1) ? 1 : 6;
        const int Kv = d.kax[1], Kw = d.kax[2];
        if (s >= np || i >= d.kax[0] * Kv * Kw) continue;
        const int kq = i / (Kv * Kw), rr = i - kq * Kv * Kw, l = rr / Kw, q = rr - l * Kw;
        int gi, gj;
        pair_comps(s, nc, gi, gj);
        const int ku = d.ord[gi][0] + d.ord[gj][0] - 1, kv = d.ord[gi][1] + d.ord[gj][1] - 1,
                  kw = d.ord[gi][2] + d.ord[gj][2] - 1;
        if (kq >= ku || l >= kv || q >= kw) continue;
        const double* src = Sp.part + (k * P * L.n_pairs + s) * kb3 + i;
        double v = 0.0;
        for (int p = 0; p < P; ++p) v += src[(int64_t)p * per_elem];
        L.mom[d.mom_off + d.pair_off[s] + (kq * kv + l) * kw + q] = v;
    }
}

}  // namespace

size_t moments_smem_bytes(int n_pairs, int kb, int gmax, int iacc_cap) {
    size_t d = (size_t)kb * (gmax | 1) + 4 * (size_t)gmax + (size_t)n_pairs * kChunk + (size_t)n_pairs * kb * kNB +
               (size_t)n_pairs * kb * kb + (size_t)iacc_cap + kGeo;
    return d * sizeof(double);
}

cudaError_t launch_moments_fp64(const MomentLaunch& L, int grid, size_t smem, cudaStream_t s) {
    k_moments_fp64<<<grid, kThreads, smem, s>>>(L);
    return cudaGetLastError();
}

size_t moments_split_part_doubles(int grid, int n_pairs, int kb) {
    return (size_t)grid * n_pairs * kb * kb * kb;
}

cudaError_t launch_moments_fp64_split(const MomentLaunch& L, const MomentSplit& Sp, size_t smem, cudaStream_t s) {
    if (L.out_ff || L.elem_status) return cudaErrorInvalidValue;  // FP64 moments, no per-element status
    k_moments_fp64_split<<<Sp.grid, kThreads, smem, s>>>(L, Sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_moments_split_reduce<<<Sp.grid, 256, 0, s>>>(L, Sp);
    return cudaGetLastError();
}

int moments_split_blocks_per_sm(size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_moments_fp64_split, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

int moments_threads() { return kThreads; }

int moments_blocks_per_sm(size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_moments_fp64, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t moments_init_attributes() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_moments_fp64);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_moments_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncGetAttributes(&fa, k_moments_fp64_split);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_moments_fp64_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)fa.sharedSizeBytes);
}

}  // namespace p2s
