// Steps a1 + a2 in double-word arithmetic for the mixed-precision path: the coupling
// factor alpha of Eq. (2) of arXiv:1703.09619 at the Gauss-Legendre points and the
// moment tensors I_s[k,l,q] of Eq. (4), with every per-point operation in float-float
// (hi + lo FP32 pairs, dw.cuh) and no FP64 instruction per point.  FP64 is used once per
// element to set up its constants (trilinear coefficients, 1-D node tables), which are
// then split into double words.
//
// Same sum factorisation and data flow as k_moments_fp64 (moments.cu).  For the metric
// kind, the parts of the Jacobian and of the phase k.x that do not depend on u are formed
// once per (v, w) row:
//   J_iu = B_i(v,w) + g_i dbeta/du,
//   J_iv = D_i(w) + u E_i(w) + g_i dbeta/dv,
//   J_iw = F_i(v) + u H_i(v) + g_i dbeta/dw,
//   k.x  = T0(v,w) + u T1(v,w) + kappa beta,   beta = cos(pi u/2) cos(pi v/2) cos(pi w/2).
// Output: the moment tensors as (hi, lo) FP32 pairs in the moment layout.
#include <cmath>

#include "alpha.cuh"
#include "dw.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;
constexpr int kNB = 16;
constexpr int kRow = 14;   // per-row constants: B_i, F_i, H_i (9), T0, T1, P1, P2, P3
constexpr int kPlane = 6;  // per-plane constants: D_i, E_i
constexpr int kGeoDW = 40;

struct SmemDW {
    dw *B, *xq, *t0, *t1, *t2, *alpha, *T1, *T2, *Iacc, *geo, *row, *plane;
    double* geo64;
};

// B-table rows are padded to an odd number of double-words so that threads reading the
// same column of different rows hit different banks.
__host__ __device__ __forceinline__ int padded_stride(int gmax) { return gmax | 1; }

__device__ __forceinline__ SmemDW carve_dw(unsigned char* sm, int n_pairs, int kb, int gmax, int iacc_cap) {
    SmemDW S;
    dw* p = reinterpret_cast<dw*>(sm);
    S.B = p;
    S.xq = S.B + kb * padded_stride(gmax);
    S.t0 = S.xq + gmax;
    S.t1 = S.t0 + gmax;
    S.t2 = S.t1 + gmax;
    S.alpha = S.t2 + gmax;
    S.T1 = S.alpha + n_pairs * kChunk;
    S.T2 = S.T1 + n_pairs * kb * kNB;
    S.Iacc = S.T2 + n_pairs * kb * kb;
    S.geo = S.Iacc + iacc_cap;
    S.row = S.geo + kGeoDW;
    S.plane = S.row + kNB * kRow;
    S.geo64 = reinterpret_cast<double*>(S.plane + kPlane);
    return S;
}

__device__ __forceinline__ void pair_comps_dw(int s, int n_comp, int& gi, int& gj) {
    if (n_comp == 1) { gi = gj = 0; return; }
    const int tgi[6] = {0, 0, 0, 1, 1, 2}, tgj[6] = {0, 1, 2, 1, 2, 2};
    gi = tgi[s];
    gj = tgj[s];
}

// alpha (metric kind) at one point from the row/plane constants; returns detJ > 0.
__device__ __forceinline__ bool metric_alpha_dw(const dw* geo, const dw* row, const dw* plane, dw u, dw Ca,
                                                dw Sa, dw* K) {
    const dw beta = dw_mul(Ca, row[11]);
    const dw dbu = dw_mul(Sa, row[11]);
    const dw dbv = dw_mul(Ca, row[12]);
    const dw dbw = dw_mul(Ca, row[13]);
    dw J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const dw g = geo[24 + i];
        J[i][0] = dw_fma(g, dbu, row[i]);
        J[i][1] = dw_fma(g, dbv, dw_fma(u, plane[3 + i], plane[i]));
        J[i][2] = dw_fma(g, dbw, dw_fma(u, row[6 + i], row[3 + i]));
    }
    const dw theta = dw_fma(geo[39], beta, dw_fma(u, row[10], row[9]));
    const dw eps = dw_add_f(dw_mul(geo[27], dw_sin(theta)), 1.f);
    dw C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            C[i][j] = dw_sub(dw_mul(J[i1][j1], J[i2][j2]), dw_mul(J[i1][j2], J[i2][j1]));
        }
    const dw det = dw_add(dw_mul(J[0][0], C[0][0]), dw_add(dw_mul(J[0][1], C[0][1]), dw_mul(J[0][2], C[0][2])));
    const dw sc = dw_div(eps, det);
    const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const int i = pi_[s], j = pj_[s];
        const dw g = dw_add(dw_mul(C[0][i], C[0][j]), dw_add(dw_mul(C[1][i], C[1][j]), dw_mul(C[2][i], C[2][j])));
        K[s] = dw_mul(sc, g);
    }
    return det.hi > 0.f;
}

__global__ void __launch_bounds__(kThreads) k_moments_dw(MomentLaunch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x;
    SmemDW S = carve_dw(smraw, L.n_pairs, L.kb, L.gmax, L.iacc_cap);
    __shared__ int bad_jac;
    const int gstride = padded_stride(L.gmax);
    const bool metric = L.kind == P2S_ALPHA_METRIC_EPS;

    for (int64_t e = blockIdx.x; e < L.n_elem; e += gridDim.x) {
        const ElemDesc& d = L.desc[e];
        const int G = d.G, nc = d.n_comp, np = (nc == 1) ? 1 : 6;
        const int Ku = d.kax[0], Kv = d.kax[1], Kw = d.kax[2];
        const int Kb = max(Ku, max(Kv, Kw));
        if (tid == 0) bad_jac = 0;
        const double* prm = L.params + 4 * e;
        if (tid < G) {  // 1-D tables, FP64 once per node, then split
            const double x = L.gl_x[G * kMaxG + tid], w = L.gl_w[G * kMaxG + tid];
            S.xq[tid] = dw_from_double(x);
            double p0 = 1.0, p1 = x;
            S.B[tid] = dw_from_double(w);
            if (Kb > 1) S.B[gstride + tid] = dw_from_double(w * x);
            for (int k = 1; k + 1 < Kb; ++k) {
                const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
                S.B[(k + 1) * gstride + tid] = dw_from_double(w * p2);
                p0 = p1;
                p1 = p2;
            }
            if (!metric) {
                const double pi = 3.141592653589793;
                S.t0[tid] = dw_from_double(prm[0] * sin(pi * (x + prm[1])));
                S.t1[tid] = dw_from_double(cos(pi * (x + prm[2])));
                S.t2[tid] = dw_from_double(exp(prm[3] * x));
            } else {
                double sx, cx;
                sincos(1.5707963267948966 * x, &sx, &cx);
                S.t0[tid] = dw_from_double(cx);                        // cos(pi x / 2)
                S.t1[tid] = dw_from_double(-1.5707963267948966 * sx);  // d/dx cos(pi x / 2)
            }
        }
        if (metric && tid == 0) metric_geo(L.nodes + 24 * e, L.bulge ? L.bulge + 4 * e : nullptr, prm, S.geo64);
        __syncthreads();
        if (metric && tid < kGeoDW) S.geo[tid] = dw_from_double(S.geo64[tid]);
        __syncthreads();

        const int per_pair = Ku * Kv * Kw;
        const int ppg = max(1, min(np, L.iacc_cap / per_pair));
        const int nb = max(1, min(G, kChunk / G));
        for (int s0 = 0; s0 < np; s0 += ppg) {
            const int ns = min(np, s0 + ppg) - s0;
            for (int i = tid; i < ns * per_pair; i += kThreads) S.Iacc[i] = dw_from_float(0.f);
            for (int c = 0; c < G; ++c) {
                for (int i = tid; i < ns * Ku * Kv; i += kThreads) S.T2[i] = dw_from_float(0.f);
                if (metric && tid < 3) {  // plane constants D_i, E_i (J_iv = D_i + u E_i + ...)
                    const dw* cf = S.geo + 8 * tid;
                    const dw w = S.xq[c];
                    S.plane[tid] = dw_fma(cf[6], w, cf[2]);
                    S.plane[3 + tid] = dw_fma(cf[7], w, cf[4]);
                }
                for (int b0 = 0; b0 < G; b0 += nb) {
                    const int nbc = min(nb, G - b0);
                    const int npts = nbc * G;
                    if (metric && tid < nbc) {  // row constants for (b0 + tid, c)
                        const int b = b0 + tid;
                        const dw v = S.xq[b], w = S.xq[c], vw = dw_mul(v, w);
                        dw* r = S.row + tid * kRow;
                        const dw* cf = S.geo;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            const dw* ci = cf + 8 * i;
                            r[i] = dw_fma(ci[7], vw, dw_fma(ci[5], w, dw_fma(ci[4], v, ci[1])));  // B_i
                            r[3 + i] = dw_fma(ci[6], v, ci[3]);                                  // F_i
                            r[6 + i] = dw_fma(ci[7], v, ci[5]);                                  // H_i
                        }
                        const dw* th = cf + 31;
                        r[9] = dw_fma(th[6], vw, dw_fma(th[3], w, dw_fma(th[2], v, th[0])));   // T0
                        r[10] = dw_fma(th[7], vw, dw_fma(th[5], w, dw_fma(th[4], v, th[1])));  // T1
                        r[11] = dw_mul(S.t0[b], S.t0[c]);  // cos cos      (beta / cos_u)
                        r[12] = dw_mul(S.t1[b], S.t0[c]);  // dcos_v cos_w
                        r[13] = dw_mul(S.t0[b], S.t1[c]);  // cos_v dcos_w
                    } else if (!metric && tid < nbc) {
                        S.row[tid * kRow] = dw_mul(S.t1[b0 + tid], S.t2[c]);
                    }
                    __syncthreads();
                    // phase A: alpha at (a, b0 + bb, c)
                    if (tid < npts) {
                        const int bb = tid / G, a = tid - bb * G;
                        if (!metric) {
                            S.alpha[tid] = dw_add_f(dw_mul(S.t0[a], S.row[bb * kRow]), 1.f);
                        } else {
                            dw K[6];
                            const bool ok = metric_alpha_dw(S.geo, S.row + bb * kRow, S.plane, S.xq[a], S.t0[a],
                                                            S.t1[a], K);
                            if (!ok) bad_jac = 1;
                            for (int s = 0; s < ns; ++s) S.alpha[s * kChunk + tid] = K[s0 + s];
                        }
                    }
                    __syncthreads();
                    // phase B: T1[s][bb][k] = sum_a B[k][a] alpha[s][bb*G + a]; k fastest across
                    // threads, so the alpha reads are broadcasts and the B rows (odd stride) spread
                    for (int i = tid; i < ns * nbc * Ku; i += kThreads) {
                        const int sb = i / Ku, k = i - sb * Ku, s = sb / nbc, bb = sb - s * nbc;
                        const dw* al = S.alpha + s * kChunk + bb * G;
                        const dw* Bk = S.B + k * gstride;
                        dw_acc acc;
                        for (int a = 0; a < G; ++a) acc.fma(Bk[a], al[a]);
                        S.T1[(s * kNB + bb) * Kb + k] = acc.value();
                    }
                    __syncthreads();
                    // phase C: T2[s][k][l] += sum_bb B[l][b0+bb] T1[s][bb][k]
                    for (int i = tid; i < ns * Ku * Kv; i += kThreads) {
                        const int s = i / (Ku * Kv), r = i - s * Ku * Kv, k = r / Kv, l = r - k * Kv;
                        const dw* t1 = S.T1 + s * kNB * Kb + k;
                        const dw* Bl = S.B + l * gstride + b0;
                        dw_acc acc;
                        acc.s = S.T2[i].hi;
                        acc.c = S.T2[i].lo;
                        for (int bb = 0; bb < nbc; ++bb) acc.fma(Bl[bb], t1[bb * Kb]);
                        S.T2[i] = acc.value();
                    }
                    __syncthreads();
                }
                // phase D: I[s][k][l][q] += B[q][c] T2[s][k][l]
                for (int i = tid; i < ns * per_pair; i += kThreads) {
                    const int skl = i / Kw, q = i - skl * Kw;
                    dw_acc acc;
                    acc.s = S.Iacc[i].hi;
                    acc.c = S.Iacc[i].lo;
                    acc.fma(S.B[q * gstride + c], S.T2[skl]);
                    S.Iacc[i] = acc.value();
                }
                __syncthreads();
            }
            for (int s = 0; s < ns; ++s) {
                int gi, gj;
                pair_comps_dw(s0 + s, nc, gi, gj);
                const int ku = d.ord[gi][0] + d.ord[gj][0] - 1, kv = d.ord[gi][1] + d.ord[gj][1] - 1,
                          kw = d.ord[gi][2] + d.ord[gj][2] - 1;
                float2* dst = reinterpret_cast<float2*>(L.mom + d.mom_off + d.pair_off[s0 + s]);
                const dw* src = S.Iacc + s * per_pair;
                for (int i = tid; i < ku * kv * kw; i += kThreads) {
                    const int k = i / (kv * kw), r = i - k * kv * kw, l = r / kw, q = r - l * kw;
                    const dw v = src[(k * Kv + l) * Kw + q];
                    dst[i] = make_float2(v.hi, v.lo);
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            if (L.elem_status) L.elem_status[e] = bad_jac ? P2S_ERR_JACOBIAN : P2S_OK;
            if (bad_jac && L.err_flag) atomicCAS(L.err_flag, 0, P2S_ERR_JACOBIAN);
        }
        __syncthreads();
    }
}

}  // namespace

size_t moments_dw_smem_bytes(int n_pairs, int kb, int gmax, int iacc_cap) {
    size_t d = (size_t)kb * padded_stride(gmax) + 4 * (size_t)gmax + (size_t)n_pairs * kChunk + (size_t)n_pairs * kb * kNB +
               (size_t)n_pairs * kb * kb + (size_t)iacc_cap + kGeoDW + kNB * kRow + kPlane;
    return d * sizeof(dw) + 48 * sizeof(double);
}

cudaError_t launch_moments_dw(const MomentLaunch& L, int grid, size_t smem, cudaStream_t s) {
    k_moments_dw<<<grid, kThreads, smem, s>>>(L);
    return cudaGetLastError();
}

int moments_dw_blocks_per_sm(size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_moments_dw, kThreads, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t moments_dw_init_attributes() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_moments_dw);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_moments_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

}  // namespace p2s
