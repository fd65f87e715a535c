// Learned quadrature order (not part of arXiv:1703.09619; it picks, per element, the
// Gauss-Legendre size G that the fill of Eq. (2)-(4) uses).
//
//   k_features      alpha (Eq. (2) coupling factor) at the 4 x 4 x 4 Gauss-Legendre points
//                   of the element, all 9 factors, divided by the mean of trace(alpha)/3:
//                   576 FP32 features per element.
//   k_mlp_predict   576 -> 64 -> 64 -> 6 ReLU MLP, FP16 weights in shared memory, FP32
//                   accumulation; class c -> G = {8, 12, 16, 24, 32, 48}[min(c + margin, 5)].
//   k_mlp_grad      training forward (same FP16-rounded weights) + softmax cross-entropy +
//                   backward for 32 samples per CTA; weight gradients reach the FP32
//                   gradient buffer with one atomic add per weight per CTA.
//   k_adam          Adam update of the FP32 master parameters.
//   k_elem_err      per element, max over product types of max|a - b| / max|b| (labels and
//                   the judge).
// Parameter layout (FP32, P2S_MLP_PARAMS values): W1 [576][64], b1 [64], W2 [64][64], b2 [64],
// W3 [64][6], b3 [6]; W[i][j] multiplies input i into output j.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "alpha_dw.cuh"
#include "dw.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kIn = P2S_MLP_IN, kH = P2S_MLP_HIDDEN, kC = P2S_MLP_CLASSES;
constexpr int oW1 = 0, oB1 = kIn * kH, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH * kC;
static_assert(oB3 + kC == P2S_MLP_PARAMS, "parameter layout");
constexpr int kS = 32;  // samples per CTA
constexpr int kThr = 256;
const int kClassG[kC] = {8, 12, 16, 24, 32, 48};
// Per-axis positions of the 4 x 4 x 4 coarse samples: two close pairs.  The close pairs
// (0.1 apart in u, about 0.05 in a unit-size element) see the local oscillation of the
// coupling factor without aliasing up to |k| ~ 60; the far pair sees its variation
// across the element.
__constant__ double c_coarse_x[4] = {-0.9, -0.8, 0.35, 0.45};

// ------------------------------------------------------------------ features
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Four elements per CTA, 64 threads (one coarse point each) per element.  The element
// constants (the geo[] layout of alpha.cuh) are formed in FP64 by 27 threads of each element,
// one trilinear coefficient or bulge entry each, then the phase coefficients by 10, and
// split into double words; each thread then forms its point's row and plane constants and
// the coupling factor in double words (alpha_dw.cuh, the moment kernel's arithmetic) on the
// FP32 pipe; the trace mean by warp shuffles in FP64.
constexpr int kFeatElems = 4;
__global__ void __launch_bounds__(64 * kFeatElems) k_features(const double* __restrict__ nodes,
                                                               const double* __restrict__ bulge,
                                                               const double* __restrict__ params, int64_t E,
                                                               float* __restrict__ feat, int32_t* __restrict__ bad) {
    const double* x4 = c_coarse_x;
    __shared__ double geo[kFeatElems][48];
    __shared__ dw geo_dw[kFeatElems][40];
    __shared__ double half_tr[kFeatElems][2];
    __shared__ dw xq[4], cs4[4], dc4[4];  // positions, cos(pi x / 2), d/dx cos(pi x / 2)
    const int sub = threadIdx.x >> 6, p = threadIdx.x & 63, warp = p >> 5, lane = p & 31;
    if (threadIdx.x < 4) {
        double sx, cx;
        sincos(1.5707963267948966 * x4[threadIdx.x], &sx, &cx);
        xq[threadIdx.x] = dw_from_double(x4[threadIdx.x]);
        cs4[threadIdx.x] = dw_from_double(cx);
        dc4[threadIdx.x] = dw_from_double(-1.5707963267948966 * sx);
    }
    for (int64_t e0 = (int64_t)blockIdx.x * kFeatElems; e0 < E; e0 += (int64_t)gridDim.x * kFeatElems) {
        const int64_t e = e0 + sub;
        const bool on = e < E;
        if (on && p < 24) {  // coefficient j of coordinate i: signed sum over the 8 nodes
            const int i = p >> 3, j = p & 7;
            const double* X = nodes + 24 * e;
            double c = 0.0;
            for (int nd = 0; nd < 8; ++nd) {
                const double su = (nd & 1) ? 1.0 : -1.0, sv = (nd & 2) ? 1.0 : -1.0, sw = (nd & 4) ? 1.0 : -1.0;
                const double sg = j == 0 ? 1.0 : j == 1 ? su : j == 2 ? sv : j == 3 ? sw
                                : j == 4 ? su * sv : j == 5 ? su * sw : j == 6 ? sv * sw : su * sv * sw;
                const double xv = 0.125 * X[3 * nd + i];
                c += j == 0 ? xv : sg * xv;
            }
            geo[sub][p] = c;
        } else if (on && p < 27) {
            geo[sub][p] = bulge ? bulge[4 * e] * bulge[4 * e + 1 + (p - 24)] : 0.0;
        }
        __syncthreads();
        if (on && p < 10) {
            const double* pr = params + 4 * e;
            const double* g = geo[sub];
            if (p < 8) geo[sub][31 + p] = pr[1] * g[p] + pr[2] * g[8 + p] + pr[3] * g[16 + p];
            else if (p == 8) geo[sub][39] = pr[1] * g[24] + pr[2] * g[25] + pr[3] * g[26];
            else geo[sub][27] = pr[0];
        }
        __syncthreads();
        if (on && p < 40) geo_dw[sub][p] = dw_from_double(p < 28 || p >= 31 ? geo[sub][p] : 0.0);
        __syncthreads();
        const int a = p & 3, b = (p >> 2) & 3, c = p >> 4;
        double K[6] = {0, 0, 0, 0, 0, 0};
        if (on) {
            // the row constants of (v, w) = (x_b, x_c) and the plane constants of w
            const dw* cf = geo_dw[sub];
            const dw v = xq[b], w = xq[c], vw = dw_mul_fast(v, w);
            dw row[14], plane[6];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const dw* ci = cf + 8 * i;
                row[i] = dw_fma_fast(ci[7], vw, dw_fma_fast(ci[5], w, dw_fma_fast(ci[4], v, ci[1])));
                row[3 + i] = dw_fma_fast(ci[6], v, ci[3]);
                row[6 + i] = dw_fma_fast(ci[7], v, ci[5]);
                plane[i] = dw_fma_fast(ci[6], w, ci[2]);
                plane[3 + i] = dw_fma_fast(ci[7], w, ci[4]);
            }
            const dw* th = cf + 31;
            row[9] = dw_fma_fast(th[6], vw, dw_fma_fast(th[3], w, dw_fma_fast(th[2], v, th[0])));
            row[10] = dw_fma_fast(th[7], vw, dw_fma_fast(th[5], w, dw_fma_fast(th[4], v, th[1])));
            row[11] = dw_mul_fast(cs4[b], cs4[c]);
            row[12] = dw_mul_fast(dc4[b], cs4[c]);
            row[13] = dw_mul_fast(cs4[b], dc4[c]);
            dw Kd[6];
            const bool ok = metric_alpha_dw(cf, row, plane, xq[a], cs4[a], dc4[a], Kd);
            if (!ok && bad) bad[e] = 1;
#pragma unroll
            for (int q = 0; q < 6; ++q) K[q] = dw_to_double(Kd[q]);
        }
        const double t = warp_sum_d((K[0] + K[3] + K[5]) / 3.0);
        if (lane == 0) half_tr[sub][warp] = t;
        __syncthreads();
        if (on) {
            const double inv = 64.0 / (half_tr[sub][0] + half_tr[sub][1]);
            const int map[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
            float* f = feat + (size_t)e * kIn + p * 9;
#pragma unroll
            for (int q = 0; q < 9; ++q) f[q] = (float)(K[map[q]] * inv);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ MLP forward (shared by both kernels)
struct MlpSmem {
    __half* W1;  // [576][64]
    float* W2;   // [64][64] (FP16-rounded values)
    float* W3;   // [64][6]
    float* b;    // b1[64] b2[64] b3[6]
    float* X;    // [32][576]
    float* H1;   // [32][64]
    float* H2;   // [32][64]
    float* Z;    // [32][6]
};
constexpr size_t kMlpSmem = sizeof(__half) * kIn * kH + sizeof(float) * (kH * kH + kH * kC + 2 * kH + kC + kS * kIn +
                                                                          2 * kS * kH + kS * kC);

// W1, then the row-major activations X, H1, H2 (each row 16-byte aligned for float4 reads),
// then W2 (8-byte pairs), W3, the biases and Z.
__device__ MlpSmem mlp_carve(unsigned char* sm) {
    MlpSmem S;
    S.W1 = reinterpret_cast<__half*>(sm);
    float* f = reinterpret_cast<float*>(sm + sizeof(__half) * kIn * kH);
    S.X = f;
    S.H1 = S.X + kS * kIn;
    S.H2 = S.H1 + kS * kH;
    S.W2 = S.H2 + kS * kH;
    S.W3 = S.W2 + kH * kH;
    S.b = S.W3 + kH * kC;
    S.Z = S.b + 2 * kH + kC;
    return S;
}

__device__ float half_round(float x) { return __half2float(__float2half_rn(x)); }

__device__ void mlp_load_weights(const float* __restrict__ P, MlpSmem& S) {
    for (int i = threadIdx.x; i < kIn * kH; i += blockDim.x) S.W1[i] = __float2half_rn(P[oW1 + i]);
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) S.W2[i] = half_round(P[oW2 + i]);
    for (int i = threadIdx.x; i < kH * kC; i += blockDim.x) S.W3[i] = half_round(P[oW3 + i]);
    for (int i = threadIdx.x; i < kH; i += blockDim.x) {
        S.b[i] = P[oB1 + i];
        S.b[kH + i] = P[oB2 + i];
    }
    if (threadIdx.x < kC) S.b[2 * kH + threadIdx.x] = P[oB3 + threadIdx.x];
}

// The features of samples e0 .. e0 + ns - 1 into S.X, zero rows after them.  Every thread
// issues all of its loads before its first store (18 float4 per thread when the rows are
// 16-byte aligned), so one memory latency covers the whole chunk even at one CTA per SM.
__device__ __forceinline__ void mlp_load_x(MlpSmem& S, const float* __restrict__ feat, int64_t e0, int ns) {
    static_assert((kS * kIn) % (4 * kThr) == 0, "feature chunk in whole float4 rounds");
    constexpr int kR = kS * kIn / (4 * kThr);
    const float* src = feat + e0 * kIn;
    const int lim = ns * kIn;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4 v[kR];
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int i = r * kThr + threadIdx.x;
            v[r] = 4 * i < lim ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float4* d4 = reinterpret_cast<float4*>(S.X);
#pragma unroll
        for (int r = 0; r < kR; ++r) d4[r * kThr + threadIdx.x] = v[r];
    } else {
        for (int i = threadIdx.x; i < kS * kIn; i += blockDim.x) S.X[i] = i < lim ? src[i] : 0.f;
    }
}

// H1, H2 (post-ReLU) and logits Z for the ns samples in S.X.  In the two hidden layers each
// thread owns two neighbouring outputs j = 2 jp, 2 jp + 1 of four samples sg + 8 k: per four
// inputs it reads four weight pairs and one float4 of each sample's row (the same row across
// a warp, a broadcast).  Every output still accumulates its inputs in order 0, 1, 2, ... with
// one FMA each, so the results do not depend on this blocking.
__device__ void mlp_forward(MlpSmem& S, int ns) {
    const int t = threadIdx.x;
    const int jp = t & 31, sg = t >> 5;  // 8 warps: samples sg, sg + 8, sg + 16, sg + 24
    static_assert(kThr == 256 && kS == 32 && kH == 64 && kIn % 4 == 0, "forward blocking");
    {
        const __half2* W1 = reinterpret_cast<const __half2*>(S.W1);  // [576][32] pairs
        float a0[4], a1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a0[k] = S.b[2 * jp];
            a1[k] = S.b[2 * jp + 1];
        }
        for (int i = 0; i < kIn; i += 4) {
            float2 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = __half22float2(W1[(i + u) * (kH / 2) + jp]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 x = *reinterpret_cast<const float4*>(S.X + (sg + 8 * k) * kIn + i);
                a0[k] = fmaf(x.x, w[0].x, a0[k]);
                a1[k] = fmaf(x.x, w[0].y, a1[k]);
                a0[k] = fmaf(x.y, w[1].x, a0[k]);
                a1[k] = fmaf(x.y, w[1].y, a1[k]);
                a0[k] = fmaf(x.z, w[2].x, a0[k]);
                a1[k] = fmaf(x.z, w[2].y, a1[k]);
                a0[k] = fmaf(x.w, w[3].x, a0[k]);
                a1[k] = fmaf(x.w, w[3].y, a1[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int sm = sg + 8 * k;
            *reinterpret_cast<float2*>(S.H1 + sm * kH + 2 * jp) =
                sm < ns ? make_float2(fmaxf(a0[k], 0.f), fmaxf(a1[k], 0.f)) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    {
        const float2* W2 = reinterpret_cast<const float2*>(S.W2);  // [64][32] pairs
        float a0[4], a1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a0[k] = S.b[kH + 2 * jp];
            a1[k] = S.b[kH + 2 * jp + 1];
        }
        for (int i = 0; i < kH; i += 4) {
            float2 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = W2[(i + u) * (kH / 2) + jp];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 h = *reinterpret_cast<const float4*>(S.H1 + (sg + 8 * k) * kH + i);
                a0[k] = fmaf(h.x, w[0].x, a0[k]);
                a1[k] = fmaf(h.x, w[0].y, a1[k]);
                a0[k] = fmaf(h.y, w[1].x, a0[k]);
                a1[k] = fmaf(h.y, w[1].y, a1[k]);
                a0[k] = fmaf(h.z, w[2].x, a0[k]);
                a1[k] = fmaf(h.z, w[2].y, a1[k]);
                a0[k] = fmaf(h.w, w[3].x, a0[k]);
                a1[k] = fmaf(h.w, w[3].y, a1[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int sm = sg + 8 * k;
            *reinterpret_cast<float2*>(S.H2 + sm * kH + 2 * jp) =
                sm < ns ? make_float2(fmaxf(a0[k], 0.f), fmaxf(a1[k], 0.f)) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    if (t < kS * kC) {
        const int s = t / kC, c = t % kC;
        float acc = S.b[2 * kH + c];
        for (int i = 0; i < kH; ++i) acc = fmaf(S.H2[s * kH + i], S.W3[i * kC + c], acc);
        S.Z[s * kC + c] = acc;
    }
    __syncthreads();
}

// The risk rule on class probabilities p (sum 1): the smallest class whose higher classes
// hold at most `risk`; the last class if none does.
__device__ __forceinline__ int risk_class(const float (&p)[kC], float risk) {
    float above = 1.f;  // probability of the classes above c
    for (int c = 0; c < kC; ++c) {
        above -= p[c];
        if (above <= risk) return c;
    }
    return kC - 1;
}

// An ensemble of n_nets > 1 networks (parameter sets P + m P2S_MLP_PARAMS): each sample's
// class probabilities are the mean of the networks' softmax outputs, summed in `acc` (the
// caller's logits array, [E][kC]) one network after the other, then the rule (risk > 0) or
// the argmax decides and acc receives the log of the mean probabilities.  Each thread of a
// CTA owns the same samples in every pass, so the sums need no synchronisation and are
// reproducible.
__device__ void mlp_predict_ensemble(const float* __restrict__ P, int n_nets, const float* __restrict__ feat,
                                     int64_t E, int margin, float risk, int32_t* __restrict__ npts,
                                     float* __restrict__ acc, MlpSmem& S) {
    const int G[kC] = {8, 12, 16, 24, 32, 48};
    for (int m = 0; m < n_nets; ++m) {
        __syncthreads();
        mlp_load_weights(P + (size_t)m * P2S_MLP_PARAMS, S);
        for (int64_t e0 = (int64_t)blockIdx.x * kS; e0 < E; e0 += (int64_t)gridDim.x * kS) {
            const int ns = (int)(E - e0 < kS ? E - e0 : kS);
            __syncthreads();
            mlp_load_x(S, feat, e0, ns);
            __syncthreads();
            mlp_forward(S, ns);
            if (threadIdx.x < ns) {
                const int s = threadIdx.x;
                float mx = S.Z[s * kC];
                for (int c = 1; c < kC; ++c) mx = fmaxf(mx, S.Z[s * kC + c]);
                float pr[kC], tot = 0.f;
                for (int c = 0; c < kC; ++c) tot += (pr[c] = expf(S.Z[s * kC + c] - mx));
                float* a = acc + (e0 + s) * kC;
                for (int c = 0; c < kC; ++c) a[c] = (m ? a[c] : 0.f) + pr[c] / tot;
            }
        }
    }
    for (int64_t e0 = (int64_t)blockIdx.x * kS; e0 < E; e0 += (int64_t)gridDim.x * kS) {
        const int ns = (int)(E - e0 < kS ? E - e0 : kS);
        if (threadIdx.x < ns) {
            float* a = acc + (e0 + threadIdx.x) * kC;
            float p[kC];
            int best = 0;
            for (int c = 0; c < kC; ++c) {
                p[c] = a[c] / (float)n_nets;
                if (p[c] > p[best]) best = c;
            }
            if (risk > 0.f) best = risk_class(p, risk);
            npts[e0 + threadIdx.x] = G[min(best + margin, kC - 1)];
            for (int c = 0; c < kC; ++c) a[c] = logf(p[c]);
        }
    }
}

// Decision: with risk > 0 the smallest class whose higher classes hold at most `risk`
// of the softmax probability; otherwise the argmax.  Then `margin` classes up.  With
// n_nets > 1, the mean probabilities of an ensemble decide (mlp_predict_ensemble).
__global__ void __launch_bounds__(kThr) k_mlp_predict(const float* __restrict__ P, int n_nets,
                                                      const float* __restrict__ feat, int64_t E, int margin,
                                                      float risk, int32_t* __restrict__ npts,
                                                      float* __restrict__ logits) {
    extern __shared__ __align__(16) unsigned char sm[];
    MlpSmem S = mlp_carve(sm);
    if (n_nets > 1) {
        mlp_predict_ensemble(P, n_nets, feat, E, margin, risk, npts, logits, S);
        return;
    }
    mlp_load_weights(P, S);
    const int G[kC] = {8, 12, 16, 24, 32, 48};
    for (int64_t e0 = (int64_t)blockIdx.x * kS; e0 < E; e0 += (int64_t)gridDim.x * kS) {
        const int ns = (int)(E - e0 < kS ? E - e0 : kS);
        __syncthreads();
        mlp_load_x(S, feat, e0, ns);
        __syncthreads();
        mlp_forward(S, ns);
        if (threadIdx.x < ns) {
            const int s = threadIdx.x;
            int best = 0;
            for (int c = 1; c < kC; ++c)
                if (S.Z[s * kC + c] > S.Z[s * kC + best]) best = c;
            if (risk > 0.f) {
                const float m = S.Z[s * kC + best];
                float pr[kC], tot = 0.f;
                for (int c = 0; c < kC; ++c) tot += (pr[c] = expf(S.Z[s * kC + c] - m));
                float above = 1.f;  // probability of the classes above c
                best = kC - 1;
                for (int c = 0; c < kC; ++c) {
                    above -= pr[c] / tot;
                    if (above <= risk) { best = c; break; }
                }
            }
            npts[e0 + s] = G[min(best + margin, kC - 1)];
            if (logits)
                for (int c = 0; c < kC; ++c) logits[(e0 + s) * kC + c] = S.Z[s * kC + c];
        }
    }
}

// ------------------------------------------------------------------ training
__global__ void __launch_bounds__(kThr) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ feat,
                                                   const int32_t* __restrict__ label, int64_t B,
                                                   const float* __restrict__ class_w, float* __restrict__ grad,
                                                   float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char sm[];
    MlpSmem S = mlp_carve(sm);
    __shared__ float dZ[kS * kC];
    __shared__ float lsum[kS];
    mlp_load_weights(P, S);
    const int64_t e0 = (int64_t)blockIdx.x * kS;
    const int ns = (int)(B - e0 < kS ? B - e0 : kS);
    mlp_load_x(S, feat, e0, ns);
    __syncthreads();
    mlp_forward(S, ns);
    const int t = threadIdx.x;
    const float invB = 1.0f / (float)B;
    if (t < kS) {
        float l = 0.f;
        if (t < ns) {
            const int y = label[e0 + t];
            float m = S.Z[t * kC];
            for (int c = 1; c < kC; ++c) m = fmaxf(m, S.Z[t * kC + c]);
            float se = 0.f;
            for (int c = 0; c < kC; ++c) se += expf(S.Z[t * kC + c] - m);
            const float w = class_w ? class_w[y] : 1.f;
            for (int c = 0; c < kC; ++c) {
                const float pc = expf(S.Z[t * kC + c] - m) / se;
                dZ[t * kC + c] = w * (pc - (c == y ? 1.f : 0.f)) * invB;
            }
            l = w * (logf(se) + m - S.Z[t * kC + y]) * invB;
        } else {
            for (int c = 0; c < kC; ++c) dZ[t * kC + c] = 0.f;
        }
        lsum[t] = l;
    }
    __syncthreads();
    if (t == 0) {
        float l = 0.f;
        for (int s = 0; s < kS; ++s) l += lsum[s];
        atomicAdd(loss, l);
    }
    // layer 3
    for (int k = t; k < kH * kC; k += blockDim.x) {
        const int i = k / kC, c = k % kC;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = fmaf(S.H2[s * kH + i], dZ[s * kC + c], acc);
        atomicAdd(grad + oW3 + k, acc);
    }
    if (t < kC) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += dZ[s * kC + t];
        atomicAdd(grad + oB3 + t, acc);
    }
    // dH2 (overwrites H2 after its last read above; synchronise first)
    float dh2[8];
    const int j = t & (kH - 1), g = t / kH;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int s = g + 4 * k;
        float acc = 0.f;
        for (int c = 0; c < kC; ++c) acc = fmaf(dZ[s * kC + c], S.W3[j * kC + c], acc);
        dh2[k] = S.H2[s * kH + j] > 0.f ? acc : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) S.H2[(g + 4 * k) * kH + j] = dh2[k];  // H2 now holds dH2
    __syncthreads();
    for (int k = t; k < kH * kH; k += blockDim.x) {
        const int i = k / kH, jj = k % kH;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = fmaf(S.H1[s * kH + i], S.H2[s * kH + jj], acc);
        atomicAdd(grad + oW2 + k, acc);
    }
    if (t < kH) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += S.H2[s * kH + t];
        atomicAdd(grad + oB2 + t, acc);
    }
    // dH1
    float dh1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int s = g + 4 * k;
        float acc = 0.f;
        for (int jj = 0; jj < kH; ++jj) acc = fmaf(S.H2[s * kH + jj], S.W2[j * kH + jj], acc);
        dh1[k] = S.H1[s * kH + j] > 0.f ? acc : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) S.H1[(g + 4 * k) * kH + j] = dh1[k];  // H1 now holds dH1
    __syncthreads();
    for (int k = t; k < kIn * kH; k += blockDim.x) {
        const int i = k / kH, jj = k % kH;
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc = fmaf(S.X[s * kIn + i], S.H1[s * kH + jj], acc);
        atomicAdd(grad + oW1 + k, acc);
    }
    if (t < kH) {
        float acc = 0.f;
        for (int s = 0; s < ns; ++s) acc += S.H1[s * kH + t];
        atomicAdd(grad + oB1 + t, acc);
    }
}

// Adam with decoupled weight decay (Loshchilov & Hutter, AdamW).
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float wd) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
    }
}

// ------------------------------------------------------------------ per-element errors
// |x| as the bit pattern of a non-negative double: such patterns order as the values, so the
// maxima below run on the integer pipe (FP64 min/max would share the FP64 unit with the
// subtraction, about 2 operations per clock per SM on this part).  A NaN entry orders above
// every number, so it makes the element's error NaN, which fails every tolerance.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One (element, type) per CTA of 256 threads, so that a few hundred judged elements still
// spread over every SM; at most 32 registers, so that the launch's 8 CTAs per SM are all
// resident (a persistent CTA that starts late holds up its later items); 16-byte loads
// (when both segments allow them) two deep per thread; one FP64 subtraction per entry,
// the maxima on bit patterns, reduced by warp shuffles.
__global__ void __launch_bounds__(256, 8) k_elem_err(const double* __restrict__ a, const int64_t* __restrict__ offa,
                                                     const double* __restrict__ b, const int64_t* __restrict__ offb,
                                                     int64_t E, int n_types, double* __restrict__ err) {
    // err[e] (zeroed by the launcher) takes the largest ratio of its types by an atomic
    // maximum on the bit patterns
    __shared__ unsigned long long sd[8], sm[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int64_t it = blockIdx.x; it < E * n_types; it += gridDim.x) {
        const int64_t e = it / n_types;
        const int t = (int)(it - e * n_types);
        const int64_t len = (offb[e + 1] - offb[e]) / n_types;
        const double* pa = a + offa[e] + t * len;
        const double* pb = b + offb[e] + t * len;
        unsigned long long d = 0, m = 0;
        if (((reinterpret_cast<uintptr_t>(pa) | reinterpret_cast<uintptr_t>(pb)) & 15) == 0) {
            const double2* qa = reinterpret_cast<const double2*>(pa);
            const double2* qb = reinterpret_cast<const double2*>(pb);
            const int64_t n2 = len / 2;
            int64_t i = tid;
            for (; i + 256 < n2; i += 512) {
                double2 va[2], vb[2];
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    va[j] = __ldcs(qa + i + 256 * j);
                    vb[j] = __ldcs(qb + i + 256 * j);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    d = max(d, max(abs_bits(va[j].x - vb[j].x), abs_bits(va[j].y - vb[j].y)));
                    m = max(m, max(abs_bits(vb[j].x), abs_bits(vb[j].y)));
                }
            }
            for (; i < n2; i += 256) {
                const double2 va = __ldcs(qa + i), vb = __ldcs(qb + i);
                d = max(d, max(abs_bits(va.x - vb.x), abs_bits(va.y - vb.y)));
                m = max(m, max(abs_bits(vb.x), abs_bits(vb.y)));
            }
            if ((len & 1) && tid == 0) {
                d = max(d, abs_bits(pa[len - 1] - pb[len - 1]));
                m = max(m, abs_bits(pb[len - 1]));
            }
        } else {
            for (int64_t i = tid; i < len; i += 256) {
                d = max(d, abs_bits(pa[i] - pb[i]));
                m = max(m, abs_bits(pb[i]));
            }
        }
        d = warp_max_u64(d);
        m = warp_max_u64(m);
        if (lane == 0) {
            sd[warp] = d;
            sm[warp] = m;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < 8; ++w) {
                d = max(d, sd[w]);
                m = max(m, sm[w]);
            }
            const double dd = __longlong_as_double((long long)d), mm = __longlong_as_double((long long)m);
            const double r = mm > 0.0 ? dd / mm : dd;
            atomicMax(reinterpret_cast<unsigned long long*>(err + e), (unsigned long long)__double_as_longlong(r));
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ judge selection
// Counter-based selection: element e is judged when splitmix64(seed + e * golden) falls
// below frac * 2^64 (splitmix64: Steele, Lea and Flood, OOPSLA 2014).
uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

cudaError_t set_mlp_smem() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
}

}  // namespace

cudaError_t learned_init_attributes() { return set_mlp_smem(); }

}  // namespace p2s

using namespace p2s;

#define P2S_LCUDA(call)                                                 \
    do {                                                                \
        cudaError_t ce_ = (call);                                       \
        if (ce_ != cudaSuccess) return fail(P2S_ERR_CUDA, #call, ce_);  \
    } while (0)

extern "C" {

int p2s_learned_npts(int cls) { return (cls >= 0 && cls < kC) ? kClassG[cls] : P2S_ERR_ARG; }

int p2s_coarse_features(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat, float* features,
                        void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || !geom || !mat) return fail(P2S_ERR_ARG, "p2s_coarse_features: NULL argument");
    if (mat->kind != P2S_ALPHA_METRIC_EPS) return fail(P2S_ERR_ARG, "p2s_coarse_features: needs the metric coupling kind");
    if (geom->n_elem == 0) return P2S_OK;
    if (!geom->nodes || !mat->params || !features) return fail(P2S_ERR_ARG, "p2s_coarse_features: NULL array");
    P2S_LCUDA(cudaSetDevice(T->device));
    const int grid = (int)std::min<int64_t>((geom->n_elem + kFeatElems - 1) / kFeatElems, (int64_t)T->sm_count * 8);
    k_features<<<grid, 64 * kFeatElems, 0, (cudaStream_t)stream>>>(geom->nodes, geom->bulge, mat->params, geom->n_elem, features,
                                                       nullptr);
    P2S_LCUDA(cudaGetLastError());
    return P2S_OK;
}

int p2s_mlp_predict_ensemble(p2s_ctx* ctx, const float* params, int n_nets, const float* features, int64_t n,
                             int margin, float risk, int32_t* npts, float* logits, void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || n < 0 || margin < 0 || !(risk >= 0.f) || risk >= 1.f || n_nets < 1 || n_nets > P2S_MLP_MAX_NETS)
        return fail(P2S_ERR_ARG, "p2s_mlp_predict: bad argument");
    if (n == 0) return P2S_OK;
    if (!params || !features || !npts || (n_nets > 1 && !logits))
        return fail(P2S_ERR_ARG, "p2s_mlp_predict: NULL array (an ensemble needs logits)");
    P2S_LCUDA(cudaSetDevice(T->device));
    const int grid = (int)std::min<int64_t>((n + kS - 1) / kS, (int64_t)T->sm_count);
    k_mlp_predict<<<grid, kThr, kMlpSmem, (cudaStream_t)stream>>>(params, n_nets, features, n, margin, risk, npts,
                                                                   logits);
    P2S_LCUDA(cudaGetLastError());
    return P2S_OK;
}

int p2s_mlp_predict(p2s_ctx* ctx, const float* params, const float* features, int64_t n, int margin, float risk,
                    int32_t* npts, float* logits, void* stream) {
    return p2s_mlp_predict_ensemble(ctx, params, 1, features, n, margin, risk, npts, logits, stream);
}

int p2s_mlp_grad(p2s_ctx* ctx, const float* params, const float* features, const int32_t* labels, int64_t batch,
                 const float* class_weight, float* grad, float* loss, void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || batch <= 0 || !params || !features || !labels || !grad || !loss)
        return fail(P2S_ERR_ARG, "p2s_mlp_grad: bad argument");
    P2S_LCUDA(cudaSetDevice(T->device));
    cudaStream_t s = (cudaStream_t)stream;
    P2S_LCUDA(cudaMemsetAsync(grad, 0, sizeof(float) * P2S_MLP_PARAMS, s));
    P2S_LCUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
    const int grid = (int)((batch + kS - 1) / kS);
    k_mlp_grad<<<grid, kThr, kMlpSmem, s>>>(params, features, labels, batch, class_weight, grad, loss);
    P2S_LCUDA(cudaGetLastError());
    return P2S_OK;
}

int p2s_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                 float eps, float weight_decay, int step, void* stream) {
    if (!params || !grad || !m || !v || n <= 0 || step < 1 || !(weight_decay >= 0.f))
        return fail(P2S_ERR_ARG, "p2s_mlp_adam: bad argument");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
    k_adam<<<grid, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2, weight_decay);
    P2S_LCUDA(cudaGetLastError());
    return P2S_OK;
}

int p2s_element_errors(p2s_ctx* ctx, const double* a, const int64_t* offsets_a, const double* b,
                       const int64_t* offsets_b, int64_t n_elem, int n_types, double* err, void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || n_elem < 0 || n_types < 1 || n_types > 4) return fail(P2S_ERR_ARG, "p2s_element_errors: bad argument");
    if (n_elem == 0) return P2S_OK;
    if (!a || !b || !offsets_a || !offsets_b || !err) return fail(P2S_ERR_ARG, "p2s_element_errors: NULL array");
    P2S_LCUDA(cudaSetDevice(T->device));
    const int grid = (int)std::min<int64_t>(n_elem * n_types, (int64_t)T->sm_count * 8);
    P2S_LCUDA(cudaMemsetAsync(err, 0, sizeof(double) * n_elem, (cudaStream_t)stream));
    k_elem_err<<<grid, 256, 0, (cudaStream_t)stream>>>(a, offsets_a, b, offsets_b, n_elem, n_types, err);
    P2S_LCUDA(cudaGetLastError());
    return P2S_OK;
}

int p2s_judge_select(int64_t n_elem, double frac, uint64_t seed, int8_t* judged) {
    if (n_elem < 0 || frac < 0.0 || frac > 1.0 || (n_elem > 0 && !judged)) return fail(P2S_ERR_ARG, "p2s_judge_select: bad argument");
    const double lim = frac * 18446744073709551616.0;
    for (int64_t e = 0; e < n_elem; ++e)
        judged[e] = (frac >= 1.0) || ((double)splitmix64(seed + (uint64_t)e * 0x9e3779b97f4a7c15ull) < lim);
    return P2S_OK;
}

}  // extern "C"

// ====================================================================== learned fill
// A learned plan holds: the main plan (the requested precision; every element's G is
// written into its descriptor from the prediction at fill time, so one plan serves every
// prediction), the judge subset (seeded, fixed at plan time) with its own FP64 plan at 48
// points, and device scratch for features, predictions, judge outputs and the report.
// A fill is asynchronous end to end: features -> prediction -> per-element G -> fill ->
// judge fill of the subset -> per-element comparison -> judged elements above the
// tolerance replaced in `out` by their 48-point FP64 fill (the plain method).
namespace p2s {
namespace {

__global__ void k_set_npts(ElemDesc* desc, const int32_t* npts, int64_t E, unsigned long long* cls_count) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int Gs[kC] = {8, 12, 16, 24, 32, 48};
        const int G = npts[e];
        desc[e].G = (int16_t)G;
        int c = 0;
        while (c < kC - 1 && Gs[c] != G) ++c;
        atomicAdd(cls_count + c, 1ull);
    }
}

// Queue order of the main fill's moment kernel: elements grouped by class, largest G first
// (the CTAs of an SM then mostly run the same specialised code, and the small elements fill
// the tail).  cls_count holds the class sizes; cursor (zeroed) the fill position per class.
__global__ void k_order_by_class(const int32_t* __restrict__ npts, int64_t E, const unsigned long long* cls_count,
                                 unsigned long long* cursor, int32_t* __restrict__ order) {
    const int Gs[kC] = {8, 12, 16, 24, 32, 48};
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int G = npts[e];
        int c = 0;
        while (c < kC - 1 && Gs[c] != G) ++c;
        unsigned long long off = 0;
        for (int c2 = c + 1; c2 < kC; ++c2) off += cls_count[c2];
        order[off + atomicAdd(cursor + c, 1ull)] = (int32_t)e;
    }
}

__global__ void k_gather_inputs(const double* __restrict__ nodes, const double* __restrict__ bulge,
                                const double* __restrict__ params, const int32_t* __restrict__ idx, int64_t nJ,
                                double* __restrict__ jn, double* __restrict__ jb, double* __restrict__ jp) {
    for (int64_t k = blockIdx.x; k < nJ; k += gridDim.x) {
        const int64_t e = idx[k];
        const int t = threadIdx.x;
        if (t < 24) jn[24 * k + t] = nodes[24 * e + t];
        else if (t < 28) jb[4 * k + t - 24] = bulge ? bulge[4 * e + t - 24] : 0.0;
        else if (t < 32) jp[4 * k + t - 28] = params[4 * e + t - 28];
    }
}

// The judged elements whose check failed: mask[k] = 1, and their indices in list[0 .. *count)
// (in no particular order; *count zeroed by the caller) for the split fallback moments.
__global__ void k_judge_mask(const double* __restrict__ err, int64_t nJ, double tol, int8_t* __restrict__ mask,
                             int32_t* __restrict__ list, int* __restrict__ count) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nJ; k += (int64_t)gridDim.x * blockDim.x) {
        const bool bad = !(err[k] <= tol);
        mask[k] = bad;
        if (bad) list[atomicAdd(count, 1)] = (int32_t)k;
    }
}

// report: [0] judged, [1] failed, [2..7] per class, [8] max judged error (double bits).
// Judged elements whose check failed (list[0 .. *count), from k_judge_mask) take their 48-point
// FP64 fill (jout): every CTA copies its share of each of them, so that a few failures still use
// the whole grid.
__global__ void k_judge_fix(double* __restrict__ out, const int64_t* __restrict__ off_main, const double* __restrict__ jout,
                            const int64_t* __restrict__ off_j, const double* __restrict__ err, int64_t nJ,
                            const int32_t* __restrict__ list, const int* __restrict__ count,
                            unsigned long long* report) {
    const int nf = *count;
    if (blockIdx.x == 0) {  // the report: block maximum of the error bits (non-negative doubles order as their bits)
        __shared__ unsigned long long wmax[32];
        unsigned long long mb = 0;
        for (int64_t k = threadIdx.x; k < nJ; k += blockDim.x)
            mb = max(mb, (unsigned long long)__double_as_longlong(err[k]));
        for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mb;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mb = max(mb, wmax[w]);
            report[0] = (unsigned long long)nJ;
            report[1] = (unsigned long long)nf;
            report[8] = mb;
        }
    }
    for (int f = 0; f < nf; ++f) {
        const int64_t k = list[f];
        const int64_t len = off_j[k + 1] - off_j[k];
        double* dst = out + off_main[k];
        const double* src = jout + off_j[k];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
            dst[i] = src[i];
    }
}

}  // namespace
}  // namespace p2s

struct p2s_learned_plan {
    p2s_ctx* ctx = nullptr;
    p2s_plan* main = nullptr;
    p2s_plan* judge = nullptr;     // judged subset, the learned fill's precision at 48 points
    p2s_plan* fallback = nullptr;  // judged subset, FP64 at 48 points (the plain method), masked
    int64_t E = 0, nJ = 0;
    int margin = 0;
    float risk = 0.f;
    double tol = 1e-9;
    int32_t* d_jidx = nullptr;
    int64_t* d_off_main = nullptr;  // [nJ+1] start of each judged element in the main output
    int64_t* d_off_j = nullptr;     // [nJ+1] start of each judged element in the judge output
    float* d_feat = nullptr;
    int32_t* d_npts = nullptr;
    double* d_jin = nullptr;  // gathered nodes [nJ][24], bulge [nJ][4], params [nJ][4]
    double* d_jout = nullptr;  // judge fill
    double* d_jfb = nullptr;   // plain-method fill of the judged elements that failed
    int8_t* d_mask = nullptr;  // [nJ] judged element failed
    int32_t* d_flist = nullptr;  // [nJ] the failed judged elements, and their number (d_fcount)
    int* d_fcount = nullptr;
    double* d_fpart = nullptr;   // partial moments of the split fallback (plan_split_part_doubles)
    double* d_jerr = nullptr;
    unsigned long long* d_report = nullptr;
    // the judge's 48-point fill runs on a side stream, forked from and joined to the caller's
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int32_t* order = nullptr;  // the main plan's moment-queue order (owned by the main plan)
    int n_nets = 1;              // networks of the prediction
    float* d_logits = nullptr;   // [E][6] probability sums of an ensemble's prediction
};

extern "C" {

void p2s_learned_plan_destroy(p2s_learned_plan* L) {
    if (!L) return;
    if (L->ctx) cudaSetDevice(context_tables(L->ctx)->device);
    p2s_plan_destroy(L->main);
    p2s_plan_destroy(L->judge);
    p2s_plan_destroy(L->fallback);
    cudaFree(L->d_jidx);
    cudaFree(L->d_off_main);
    cudaFree(L->d_off_j);
    cudaFree(L->d_feat);
    cudaFree(L->d_npts);
    cudaFree(L->d_jin);
    cudaFree(L->d_jout);
    cudaFree(L->d_jfb);
    cudaFree(L->d_mask);
    cudaFree(L->d_flist);
    cudaFree(L->d_fcount);
    cudaFree(L->d_fpart);
    cudaFree(L->d_jerr);
    cudaFree(L->d_report);
    cudaFree(L->d_logits);
    if (L->side) cudaStreamSynchronize(L->side);
    if (L->ev_fork) cudaEventDestroy(L->ev_fork);
    if (L->ev_join) cudaEventDestroy(L->ev_join);
    if (L->side) cudaStreamDestroy(L->side);
    delete L;
}

int p2s_learned_plan_create(p2s_ctx* ctx, int64_t E, const p2s_orders* orders, const p2s_learned_opts* opts,
                            p2s_learned_plan** out) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || !out || !orders || !opts) return fail(P2S_ERR_ARG, "p2s_learned_plan_create: NULL argument");
    *out = nullptr;
    if (orders->n_comp != 3) return fail(P2S_ERR_ARG, "p2s_learned_plan_create: the learned fill needs three components");
    if (opts->margin < 0 || opts->judge_frac < 0 || opts->judge_frac > 1 || !(opts->judge_tol >= 0) ||
        !(opts->risk >= 0.0) || opts->risk >= 1.0 || opts->n_nets < 0 || opts->n_nets > P2S_MLP_MAX_NETS)
        return fail(P2S_ERR_ARG, "p2s_learned_plan_create: bad margin, judge fraction, tolerance or network count");
    P2S_LCUDA(cudaSetDevice(T->device));
    p2s_learned_plan* L = new (std::nothrow) p2s_learned_plan();
    if (!L) return fail(P2S_ERR_OOM, "p2s_learned_plan_create: host allocation");
    L->ctx = ctx;
    L->E = E;
    L->margin = opts->margin;
    L->risk = (float)opts->risk;
    L->tol = opts->judge_tol;
    L->n_nets = opts->n_nets > 1 ? opts->n_nets : 1;
    p2s_quadrature q48 = {48, nullptr};
    p2s_fill_opts fo = {opts->precision, P2S_TYPES_ALL};
    int rc = p2s_plan_create(ctx, E, orders, &q48, &fo, &L->main);
    if (rc) { p2s_learned_plan_destroy(L); return rc; }
    L->order = plan_order(L->main);
    if (!L->order) { p2s_learned_plan_destroy(L); return fail(P2S_ERR_OOM, "p2s_learned_plan_create: element order"); }
    // judge subset
    std::vector<int8_t> sel((size_t)std::max<int64_t>(E, 1));
    p2s_judge_select(E, opts->judge_frac, opts->seed, sel.data());
    std::vector<int32_t> jidx;
    for (int64_t e = 0; e < E; ++e)
        if (sel[e]) jidx.push_back((int32_t)e);
    L->nJ = (int64_t)jidx.size();
    std::vector<int64_t> off_full((size_t)E + 1);
    p2s_output_entries(E, orders, P2S_TYPES_ALL, off_full.data());
    const size_t nc3 = 9;
    std::vector<int32_t> jord(std::max<size_t>(1, jidx.size() * nc3));
    std::vector<int64_t> off_main(jidx.size() + 1), off_j(jidx.size() + 1);
    for (size_t k = 0; k < jidx.size(); ++k) {
        std::memcpy(&jord[k * nc3], orders->orders + nc3 * jidx[k], sizeof(int32_t) * nc3);
        off_main[k] = off_full[jidx[k]];
    }
    off_main[jidx.size()] = off_full[E];
    p2s_orders jo = {3, jord.data()};
    p2s_fill_opts fj = {opts->precision, P2S_TYPES_ALL};
    rc = p2s_plan_create(ctx, L->nJ, &jo, &q48, &fj, &L->judge);
    if (rc) { p2s_learned_plan_destroy(L); return rc; }
    p2s_fill_opts ff = {P2S_FP64, P2S_TYPES_ALL};
    rc = p2s_plan_create(ctx, L->nJ, &jo, &q48, &ff, &L->fallback);
    if (rc) { p2s_learned_plan_destroy(L); return rc; }
    const int64_t jent = p2s_output_entries(L->nJ, &jo, P2S_TYPES_ALL, off_j.data());
    bool ok = (L->n_nets == 1 ||
               cudaMalloc(&L->d_logits, sizeof(float) * kC * std::max<int64_t>(E, 1)) == cudaSuccess) &&
              cudaMalloc(&L->d_feat, sizeof(float) * kIn * std::max<int64_t>(E, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_npts, sizeof(int32_t) * std::max<int64_t>(E, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_jidx, sizeof(int32_t) * std::max<int64_t>(L->nJ, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_off_main, sizeof(int64_t) * (L->nJ + 1)) == cudaSuccess &&
              cudaMalloc(&L->d_off_j, sizeof(int64_t) * (L->nJ + 1)) == cudaSuccess &&
              cudaMalloc(&L->d_jin, sizeof(double) * 32 * std::max<int64_t>(L->nJ, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_jout, sizeof(double) * std::max<int64_t>(jent, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_jfb, sizeof(double) * std::max<int64_t>(jent, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_mask, std::max<int64_t>(L->nJ, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_flist, sizeof(int32_t) * std::max<int64_t>(L->nJ, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_fcount, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&L->d_fpart, sizeof(double) * std::max<size_t>(plan_split_part_doubles(L->fallback), 1)) ==
                  cudaSuccess &&
              cudaMalloc(&L->d_jerr, sizeof(double) * std::max<int64_t>(L->nJ, 1)) == cudaSuccess &&
              cudaMalloc(&L->d_report, sizeof(unsigned long long) * 16) == cudaSuccess;
    if (!ok) { p2s_learned_plan_destroy(L); return fail(P2S_ERR_OOM, "p2s_learned_plan_create: device allocation"); }
    {
        cudaError_t ce = cudaStreamCreateWithFlags(&L->side, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&L->ev_fork, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&L->ev_join, cudaEventDisableTiming);
        if (ce != cudaSuccess) { p2s_learned_plan_destroy(L); return fail(P2S_ERR_CUDA, "p2s_learned_plan_create: stream", ce); }
    }
    if (L->nJ) {
        cudaError_t ce = cudaMemcpy(L->d_jidx, jidx.data(), sizeof(int32_t) * L->nJ, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(L->d_off_main, off_main.data(), sizeof(int64_t) * (L->nJ + 1), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(L->d_off_j, off_j.data(), sizeof(int64_t) * (L->nJ + 1), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) { p2s_learned_plan_destroy(L); return fail(P2S_ERR_CUDA, "p2s_learned_plan_create: upload", ce); }
    }
    *out = L;
    return P2S_OK;
}

int64_t p2s_learned_plan_output_entries(const p2s_learned_plan* L) {
    return L ? p2s_plan_output_entries(L->main) : P2S_ERR_ARG;
}

int p2s_learned_fill(p2s_learned_plan* L, const p2s_geometry* geom, const p2s_material* mat, const float* params,
                     double* out, int32_t* npts_out, void* stream) {
    if (!L || !geom || !mat || !params) return fail(P2S_ERR_ARG, "p2s_learned_fill: NULL argument");
    if (geom->n_elem != L->E) return fail(P2S_ERR_ARG, "p2s_learned_fill: n_elem differs from the plan");
    if (mat->kind != P2S_ALPHA_METRIC_EPS) return fail(P2S_ERR_ARG, "p2s_learned_fill: needs the metric coupling kind");
    const DeviceTables* T = context_tables(L->ctx);
    P2S_LCUDA(cudaSetDevice(T->device));
    cudaStream_t s = (cudaStream_t)stream;
    P2S_LCUDA(cudaMemsetAsync(L->d_report, 0, sizeof(unsigned long long) * 16, s));
    if (L->E == 0) return P2S_OK;
    double* jn = L->d_jin;
    double* jb = jn + 24 * L->nJ;
    double* jp = jb + 4 * L->nJ;
    const int gj = (int)std::min<int64_t>(std::max<int64_t>(L->nJ, 1), 4096);
    p2s_geometry g2 = {L->nJ, jn, jb};
    p2s_material m2 = {P2S_ALPHA_METRIC_EPS, jp};
    // The judge's 48-point fill does not depend on the prediction: it starts first, on the
    // side stream, and the main path's kernels fill the SMs its last elements leave idle.
    NvtxRange whole("p2s learned fill");
    if (L->nJ) {
        NvtxRange r("p2s learned: judge 48-point fill (side stream)");
        P2S_LCUDA(cudaEventRecord(L->ev_fork, s));
        P2S_LCUDA(cudaStreamWaitEvent(L->side, L->ev_fork, 0));
        k_gather_inputs<<<gj, 32, 0, L->side>>>(geom->nodes, geom->bulge, mat->params, L->d_jidx, L->nJ, jn, jb, jp);
        P2S_LCUDA(cudaGetLastError());
        int jrc = p2s_plan_fill(L->judge, &g2, &m2, L->d_jout, nullptr, L->side);
        P2S_LCUDA(cudaEventRecord(L->ev_join, L->side));
        if (jrc) {
            P2S_LCUDA(cudaStreamWaitEvent(s, L->ev_join, 0));
            return jrc;
        }
    }
    nvtxRangePushA("p2s learned: features, prediction, class order");
    int rc = p2s_coarse_features(L->ctx, geom, mat, L->d_feat, stream);
    if (rc == P2S_OK)
        rc = p2s_mlp_predict_ensemble(L->ctx, params, L->n_nets, L->d_feat, L->E, L->margin, L->risk, L->d_npts,
                                      L->d_logits, stream);
    if (rc == P2S_OK) {
        const int gs = (int)std::min<int64_t>((L->E + 255) / 256, 1024);
        k_set_npts<<<gs, 256, 0, s>>>(plan_desc(L->main), L->d_npts, L->E, L->d_report + 2);
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) {
            k_order_by_class<<<gs, 256, 0, s>>>(L->d_npts, L->E, L->d_report + 2, L->d_report + 9, L->order);
            ce = cudaGetLastError();
        }
        if (ce != cudaSuccess) rc = fail(P2S_ERR_CUDA, "p2s_learned_fill: k_set_npts / k_order_by_class", ce);
    }
    if (rc == P2S_OK && npts_out) {
        const cudaError_t ce = cudaMemcpyAsync(npts_out, L->d_npts, sizeof(int32_t) * L->E, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) rc = fail(P2S_ERR_CUDA, "p2s_learned_fill: npts copy", ce);
    }
    nvtxRangePop();
    if (rc == P2S_OK) rc = p2s_plan_fill(L->main, geom, mat, out, nullptr, stream);
    if (L->nJ) P2S_LCUDA(cudaStreamWaitEvent(s, L->ev_join, 0));  // joined on every path
    if (rc) return rc;
    if (L->nJ) {
        NvtxRange r("p2s learned: judge comparison and fallback");
        rc = p2s_element_errors(L->ctx, out, L->d_off_main, L->d_jout, L->d_off_j, L->nJ, 4, L->d_jerr, stream);
        if (rc) return rc;
        // judged elements above the tolerance: their plain-method fill, then the copy into out
        P2S_LCUDA(cudaMemsetAsync(L->d_fcount, 0, sizeof(int), s));
        k_judge_mask<<<(int)std::min<int64_t>((L->nJ + 255) / 256, 1024), 256, 0, s>>>(L->d_jerr, L->nJ, L->tol, L->d_mask,
                                                                                     L->d_flist, L->d_fcount);
        P2S_LCUDA(cudaGetLastError());
        rc = plan_fill_masked(L->fallback, &g2, &m2, L->d_jfb, L->d_mask, s, L->d_flist, L->d_fcount, L->d_fpart);
        if (rc) return rc;
        k_judge_fix<<<gj, 256, 0, s>>>(out, L->d_off_main, L->d_jfb, L->d_off_j, L->d_jerr, L->nJ, L->d_flist, L->d_fcount,
                                       L->d_report);
        P2S_LCUDA(cudaGetLastError());
    }
    return P2S_OK;
}

int p2s_learned_report_get(p2s_learned_plan* L, p2s_learned_report* rep, int8_t* judge_state, void* stream) {
    if (!L || !rep) return fail(P2S_ERR_ARG, "p2s_learned_report_get: NULL argument");
    P2S_LCUDA(cudaSetDevice(context_tables(L->ctx)->device));
    P2S_LCUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long h[16];
    P2S_LCUDA(cudaMemcpy(h, L->d_report, sizeof(h), cudaMemcpyDeviceToHost));
    rep->n_elem = L->E;
    rep->judged = (int64_t)h[0];
    rep->failed = (int64_t)h[1];
    for (int c = 0; c < kC; ++c) rep->per_class[c] = (int64_t)h[2 + c];
    long long bits = (long long)h[8];
    std::memcpy(&rep->max_judged_err, &bits, sizeof(double));
    if (judge_state) {
        std::memset(judge_state, 0, (size_t)L->E);
        if (L->nJ) {
            std::vector<int32_t> idx((size_t)L->nJ);
            std::vector<double> err((size_t)L->nJ);
            P2S_LCUDA(cudaMemcpy(idx.data(), L->d_jidx, sizeof(int32_t) * L->nJ, cudaMemcpyDeviceToHost));
            P2S_LCUDA(cudaMemcpy(err.data(), L->d_jerr, sizeof(double) * L->nJ, cudaMemcpyDeviceToHost));
            for (int64_t k = 0; k < L->nJ; ++k) judge_state[idx[k]] = (err[k] <= L->tol) ? 1 : 2;
        }
    }
    return P2S_OK;
}

}  // extern "C"
