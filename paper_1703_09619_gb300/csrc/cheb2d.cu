// The paper's own example (arXiv:1703.09619, Sec. III): element matrices of the 2-D curl-curl
// equation, Eq. (5), on curved quadrilaterals with the curl-conforming Chebyshev basis of Eq. (6)
//   E_u = U_m(u) T_n(v) (m < M, n <= N),   E_v = T_m(u) U_n(v) (m <= M, n < N),
// stiffness S and mass M of Eq. (7)-(15).  Two fills of the same matrices:
//
//  * product to sum (Sec. III, Eq. (16)-(19)): every product of two Chebyshev polynomials of one
//    variable becomes a sum of two, so each entry is a signed sum of four "starting-point"
//    integrals (Eq. (19)).  Four moment sets per element, one per coupling factor:
//      I_S [k][l] = sum_ab w_a w_b T^ns_k(u_a) T^ns_l(v_b) / (mu_r J)                 (S, all blocks)
//      I_uu[k][l] = ... T^ns_k(u) T_l(v)  eps_r (x_v^2 + y_v^2) / J                   (M_uu)
//      I_uv[k][l] = ... U_k(u)    U_l(v)  -eps_r (x_u x_v + y_u y_v) / J              (M_uv, M_vu)
//      I_vv[k][l] = ... T_k(u)    T^ns_l(v) eps_r (x_u^2 + y_u^2) / J                 (M_vv)
//    sum-factorised (u first, then v), then the entries (k_cheb2d_p2s);
//  * direct numerical integration, the paper's comparison method: every entry is its own 2-D
//    Gauss-Legendre sum of the basis products and the coupling factor (k_cheb2d_direct).
//
// Products (Eq. (16); the T.T and U.T lines carry a 1/2):
//   U_a U_b = T^ns_{|a-b|} - T^ns_{a+b+2},  T_a T_b = (T_{|a-b|} + T_{a+b}) / 2,
//   U_a T_b = (U_{a+b} + U_{a-b}) / 2 with U_{-1} = 0, U_{-j} = -U_{j-2},
// and T^ns_n (Eq. (17)) evaluated as -(U_{n-2} + U_{n-4} + ...), which equals the quotient of
// Eq. (17) without its cancellation near u = +-1 (T^ns_0 = T^ns_1 = 0).
//
// Geometry (Fig. 1): element (s_lo, s_hi, t_lo, t_hi) of the map X(s, t) = (s g(t), t f(s)),
// f(x) = 1 - 0.2 (x^2 - 1)^2, g(y) = 1 + 0.2 (y^2 - 1)^2; eps_r = 2 exp(x + y + 2) where the
// element's flag is set, else 1; mu_r = 1.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "arith.cuh"
#include "dw.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kC2Threads = 256;     // direct fill
constexpr int kC2P2SThreads = 512;  // product-to-sum fill
constexpr int kC2MaxOrder = P2S_CHEB2D_MAX_ORDER;
constexpr int kC2MaxG = P2S_CHEB2D_MAX_NPTS;
constexpr int kC2Chunk = 8;                   // v-columns of coupling factors per chunk

struct C2Launch {
    const double* params;  // [E][5]
    int64_t n_elem;
    int M, N, G;
    const double* gl_x;  // [kMaxG + 1][kMaxG]
    const double* gl_w;
    double* S;
    double* Mm;
    int* err_flag;
};

// Map of one element at (u, v): x, y and the Jacobian entries.
struct Geo {
    double x, y, xu, xv, yu, yv;
};
__device__ __forceinline__ Geo c2_geometry(const double* p, double u, double v) {
    const double hs = 0.5 * (p[1] - p[0]), ht = 0.5 * (p[3] - p[2]);
    const double s = p[0] + (u + 1.0) * hs, t = p[2] + (v + 1.0) * ht;
    const double s2 = s * s - 1.0, t2 = t * t - 1.0;
    const double f = 1.0 - 0.2 * s2 * s2, g = 1.0 + 0.2 * t2 * t2;
    const double df = -0.8 * s * s2, dg = 0.8 * t * t2;
    Geo r;
    r.x = s * g;
    r.y = t * f;
    r.xu = hs * g;
    r.xv = ht * s * dg;
    r.yu = hs * t * df;
    r.yv = ht * f;
    return r;
}

// The four coupling factors at (u, v): c[0] = 1/(mu J), c[1] = eps (x_v^2 + y_v^2)/J,
// c[2] = -eps (x_u x_v + y_u y_v)/J, c[3] = eps (x_u^2 + y_u^2)/J.  Returns false if J <= 0.
__device__ __forceinline__ bool c2_couplings(const double* p, double u, double v, double* c) {
    const Geo q = c2_geometry(p, u, v);
    const double J = q.xu * q.yv - q.xv * q.yu;
    const double eps = p[4] != 0.0 ? 2.0 * exp(q.x + q.y + 2.0) : 1.0;
    const double rJ = 1.0 / J, er = eps * rJ;
    c[0] = rJ;
    c[1] = er * (q.xv * q.xv + q.yv * q.yv);
    c[2] = -er * (q.xu * q.xv + q.yu * q.yv);
    c[3] = er * (q.xu * q.xu + q.yu * q.yu);
    return J > 0.0;
}

// 1-D tables at the G nodes for indices 0..K-1 (row stride gs): T_k, U_k and T^ns_k, multiplied
// by the weight w_a when `weighted` (a moment is then a plain sum of table x table x coupling),
// and the nodes sx[a] and weights sw[a].
__device__ void c2_tables(const C2Launch& L, int K, int gs, bool weighted, double* sT, double* sU, double* sN,
                          double* sx, double* sw) {
    const int G = L.G;
    for (int a = threadIdx.x; a < G; a += blockDim.x) {
        const double x = L.gl_x[G * kMaxG + a], w = L.gl_w[G * kMaxG + a], f = weighted ? w : 1.0;
        sx[a] = x;
        sw[a] = w;
        double t0 = 1.0, t1 = x, u0 = 1.0, u1 = 2.0 * x;
        double ne = 0.0, no = 0.0;  // -(U_{k-2} + U_{k-4} + ...) for even / odd k
        for (int k = 0; k < K; ++k) {
            double tk, uk;
            if (k == 0) { tk = t0; uk = u0; }
            else if (k == 1) { tk = t1; uk = u1; }
            else {
                tk = 2.0 * x * t1 - t0;
                uk = 2.0 * x * u1 - u0;
                t0 = t1; t1 = tk;
                u0 = u1; u1 = uk;
            }
            sT[k * gs + a] = f * tk;
            sU[k * gs + a] = f * uk;
            double ns = 0.0;
            if (k >= 2) {
                if (k % 2 == 0) ns = (ne -= sU[(k - 2) * gs + a]);
                else ns = (no -= sU[(k - 2) * gs + a]);
            }
            sN[k * gs + a] = ns;  // carries the weight factor f through the U rows
        }
    }
}

// Sum-factorised moments of one element: I_s[k][l] = sum_a sum_b X_s[k][a] Y_s[l][b] c_s(a, b)
// with (X, Y) = (T^ns, T^ns), (T^ns, T), (U, U), (T, T^ns) for s = 0..3 (weights in the tables).
// Ku, Kv: moment counts per axis; Im[s] at s * Ku * Kv.  Returns false if some J <= 0.
__device__ bool c2_moments(const C2Launch& L, const double* p, int Ku, int Kv, int gs, const double* sT,
                           const double* sU, const double* sN, const double* sx, double* sc, double* sY,
                           double* Im, int* bad) {
    const int G = L.G;
    for (int i = threadIdx.x; i < 4 * Ku * Kv; i += blockDim.x) Im[i] = 0.0;
    for (int b0 = 0; b0 < G; b0 += kC2Chunk) {
        const int nb = min(kC2Chunk, G - b0);
        // coupling factors at (a, b0 + bb): sc[s][bb][a]
        for (int i = threadIdx.x; i < nb * G; i += blockDim.x) {
            const int bb = i / G, a = i - bb * G;
            double c[4];
            if (!c2_couplings(p, sx[a], sx[b0 + bb], c)) *bad = 1;
#pragma unroll
            for (int s = 0; s < 4; ++s) sc[(s * kC2Chunk + bb) * G + a] = c[s];
        }
        __syncthreads();
        // Y[s][bb][k] = sum_a X_s[k][a] c_s(a, b0 + bb)
        for (int i = threadIdx.x; i < 4 * nb * Ku; i += blockDim.x) {
            const int s = i / (nb * Ku), r = i - s * nb * Ku, bb = r / Ku, k = r - bb * Ku;
            const double* X = (s == 2 ? sU : (s == 3 ? sT : sN)) + k * gs;
            const double* c = sc + (s * kC2Chunk + bb) * G;
            double acc = 0.0;
            for (int a = 0; a < G; ++a) acc = fma(X[a], c[a], acc);
            sY[(s * kC2Chunk + bb) * Ku + k] = acc;
        }
        __syncthreads();
        // I[s][k][l] += sum_bb Y_s[l][b0 + bb] Y[s][bb][k]
        for (int i = threadIdx.x; i < 4 * Ku * Kv; i += blockDim.x) {
            const int s = i / (Ku * Kv), r = i - s * Ku * Kv, k = r / Kv, l = r - k * Kv;
            const double* Yt = (s == 2 ? sU : (s == 1 ? sT : sN)) + l * gs + b0;
            const double* y = sY + s * kC2Chunk * Ku + k;
            double acc = Im[i];
            for (int bb = 0; bb < nb; ++bb) acc = fma(Yt[bb], y[bb * Ku], acc);
            Im[i] = acc;
        }
        __syncthreads();
    }
    return true;
}

// One axis of a product-to-sum entry: up to two (moment index, coefficient) terms.  The
// coefficients are integers up to 24^2 or halves, exact in FP32 as in FP64.
template <typename C>
struct Axis2 {
    int k0, k1;
    C c0, c1;
};
// U_a U_b (a, b >= -1; U_{-1} = 0) -> T^ns_{|a-b|} - T^ns_{a+b+2}
template <typename C>
__device__ __forceinline__ Axis2<C> ax_uu(int a, int b, C scale) {
    Axis2<C> r;
    if (a < 0 || b < 0) { r.k0 = r.k1 = 0; r.c0 = r.c1 = C(0); return r; }
    r.k0 = abs(a - b);
    r.k1 = a + b + 2;
    r.c0 = scale;
    r.c1 = -scale;
    return r;
}
// T_a T_b -> (T_{|a-b|} + T_{a+b}) / 2
template <typename C>
__device__ __forceinline__ Axis2<C> ax_tt(int a, int b) {
    Axis2<C> r;
    r.k0 = abs(a - b);
    r.k1 = a + b;
    r.c0 = C(0.5);
    r.c1 = C(0.5);
    return r;
}
// U_a T_b -> (U_{a+b} + U_{a-b}) / 2, U_{-1} = 0, U_{-j} = -U_{j-2}
template <typename C>
__device__ __forceinline__ Axis2<C> ax_ut(int a, int b) {
    Axis2<C> r;
    r.k0 = a + b;
    r.c0 = C(0.5);
    const int d = a - b;
    if (d >= 0) { r.k1 = d; r.c1 = C(0.5); }
    else if (d == -1) { r.k1 = 0; r.c1 = C(0); }
    else { r.k1 = -d - 2; r.c1 = C(-0.5); }
    return r;
}

// u-axis and v-axis factors of each (row block, column block) pair, blocks 0 = E_u, 1 = E_v
// (Eq. (8)-(15) through Eq. (16)).  The curl scales of S are split so that every factor of m lies
// on the u side and every factor of n on the v side.
template <typename C>
__device__ __forceinline__ Axis2<C> s_axis_u(int rb, int cb, int m1, int m2) {
    if (rb == 0) return cb == 0 ? ax_uu<C>(m1, m2, C(1)) : ax_uu<C>(m1, m2 - 1, C(m2));
    return cb == 0 ? ax_uu<C>(m1 - 1, m2, C(-m1)) : ax_uu<C>(m1 - 1, m2 - 1, C(m1 * m2));
}
template <typename C>
__device__ __forceinline__ Axis2<C> s_axis_v(int rb, int cb, int n1, int n2) {
    if (rb == 0) return cb == 0 ? ax_uu<C>(n1 - 1, n2 - 1, C(n1 * n2)) : ax_uu<C>(n1 - 1, n2, C(-n1));
    return cb == 0 ? ax_uu<C>(n1, n2 - 1, C(n2)) : ax_uu<C>(n1, n2, C(1));
}
template <typename C>
__device__ __forceinline__ Axis2<C> m_axis_u(int rb, int cb, int m1, int m2) {
    if (rb == 0) return cb == 0 ? ax_uu<C>(m1, m2, C(1)) : ax_ut<C>(m1, m2);
    return cb == 0 ? ax_ut<C>(m2, m1) : ax_tt<C>(m1, m2);
}
template <typename C>
__device__ __forceinline__ Axis2<C> m_axis_v(int rb, int cb, int n1, int n2) {
    if (rb == 0) return cb == 0 ? ax_tt<C>(n1, n2) : ax_ut<C>(n2, n1);
    return cb == 0 ? ax_ut<C>(n1, n2) : ax_uu<C>(n1, n2, C(1));
}

// An axis factor as c (V[o0] + sgn V[o1]): the two coefficients of Eq. (16) are equal, opposite
// or (U_{-1}) zero, so one scaling and one signed sum per entry.  Offsets premultiplied by the
// row stride of V.
template <typename C>
struct Fac {
    int o0, o1;
    C c, sgn;
};
template <typename C>
__device__ __forceinline__ Fac<C> to_fac(Axis2<C> a, int stride) {
    Fac<C> f;
    f.o0 = a.k0 * stride;
    f.o1 = a.k1 * stride;
    f.c = a.c0;
    f.sgn = a.c1 == C(0) ? C(0) : (a.c1 == a.c0 ? C(1) : C(-1));
    return f;
}
// A float that holds a small integer or a half, as a double, by integer operations on its bits
// (sign, exponent rebiased from 127 to 1023, mantissa widened): exact for zero and normal floats.
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
    const uint64_t d = sign | ((uint64_t)(((b >> 23) & 0xffu) + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
// FP64: the sign by selection, then one DADD and one DMUL (FP64 arithmetic is the scarce pipe)
__device__ __forceinline__ double c2_combine(const double* V, Fac<float> f) {
    const double y = V[f.o1];
    const double t = f.sgn == 0.f ? 0.0 : (f.sgn > 0.f ? y : -y);
    return f2d_exact(f.c) * (V[f.o0] + t);
}
__device__ __forceinline__ dw c2_combine_dw(const float2* V, Fac<float> f) {
    const float2 x = V[f.o0], y = V[f.o1];
    return dw_mul_f(dw_add_fast(dw{x.x, x.y}, dw{f.sgn * y.x, f.sgn * y.y}), f.c);
}
// A factor in one int (o0, o1 < 2^15; the sign as 0, 1 = +1, 2 = -1 in bits 30-31) and its scale.
__device__ __forceinline__ int pack_fac(Fac<float> f) {
    return f.o0 | (f.o1 << 15) | ((f.sgn == 0.f ? 0 : (f.sgn > 0.f ? 1 : 2)) << 30);
}
__device__ __forceinline__ Fac<float> unpack_fac(int p, float c) {
    Fac<float> f;
    f.o0 = p & 0x7fff;
    f.o1 = (p >> 15) & 0x7fff;
    const int g = (p >> 30) & 3;
    f.c = c;
    f.sgn = g == 0 ? 0.f : (g == 1 ? 1.f : -1.f);
    return f;
}
__device__ __forceinline__ double c2_combine(const float2* V, Fac<float> f) {
    const dw r = c2_combine_dw(V, f);
    return ArithFF::to_double_fast(make_float2(r.hi, r.lo));
}

// Product-to-sum fill: one CTA per element (grid-stride).  After the moments, the rows are taken
// in groups of one row block and one n1 (the M or M+1 rows m1 of the group share n1): for each
// column block and matrix the v-axis sums V[ku][n2] = c (I[ku][kv_0] + sgn I[ku][kv_1]) are formed
// once for the group, so each entry is c' (V[ku_0][n2] + sgn' V[ku_1][n2]).  Warps take (row,
// column block) items, lanes along the row (coalesced streaming stores, columns stepped without
// divisions).  kFF: the moments are rounded to float-float pairs once per element and V and the
// entries are formed in float-float on the FP32 pipe (FP64 arithmetic issues at a small fraction
// of its rate); each entry reaches FP64 by integer operations.
template <bool kFF>
__global__ void __launch_bounds__(kC2P2SThreads, 2) k_cheb2d_p2s(C2Launch L) {
    using VT = typename std::conditional<kFF, float2, double>::type;
    using CT = float;  // factor coefficients: exact in FP32
    extern __shared__ double sm[];
    const int M = L.M, N = L.N, G = L.G;
    const int Ku = 2 * M + 1, Kv = 2 * N + 1, K = max(Ku, Kv), gs = G | 1;
    double* sT = sm;
    double* sU = sT + K * gs;
    double* sN = sU + K * gs;
    double* sx = sN + K * gs;
    double* sc = sx + G;
    double* sY = sc + 4 * kC2Chunk * G;
    double* Im = sY + 4 * kC2Chunk * K;
    double* sw = Im + 4 * Ku * Kv;
    VT* sV = reinterpret_cast<VT*>(sw + G);  // [matrix S, M][column block][ku][n2], n2 < N + 1
    const VT* IV = reinterpret_cast<const VT*>(Im);
    __shared__ int bad;
    const int nu = M * (N + 1), n = nu + (M + 1) * N, VB = Ku * (N + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    c2_tables(L, K, gs, true, sT, sU, sN, sx, sw);
    for (int64_t e = blockIdx.x; e < L.n_elem; e += gridDim.x) {
        const double* p = L.params + 5 * e;
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        c2_moments(L, p, Ku, Kv, gs, sT, sU, sN, sx, sc, sY, Im, &bad);
        if (kFF) {  // moments to (hi, lo) pairs in place
            for (int i = threadIdx.x; i < 4 * Ku * Kv; i += blockDim.x) {
                const double v = Im[i];
                const float hi = (float)v;
                reinterpret_cast<float2*>(Im)[i] = make_float2(hi, (float)(v - (double)hi));
            }
            __syncthreads();
        }
        double* Se = L.S + e * (int64_t)n * n;
        double* Me = L.Mm + e * (int64_t)n * n;
        for (int grp = 0; grp < 2 * N + 1; ++grp) {
            const int rb = grp <= N ? 0 : 1, n1 = rb == 0 ? grp : grp - (N + 1);
            const int rows = rb == 0 ? M : M + 1, rw = rb == 0 ? N + 1 : N, rbase = rb == 0 ? 0 : nu;
            // V for (S, M) x (column block 0, 1)
            for (int i = threadIdx.x; i < 4 * VB; i += blockDim.x) {
                const int tb = i / VB, r = i - tb * VB, ku = r / (N + 1), n2 = r - ku * (N + 1);
                const int mat = tb >> 1, cb = tb & 1;
                if (cb == 1 && n2 >= N) continue;
                const Fac<CT> f = to_fac(mat == 0 ? s_axis_v<CT>(rb, cb, n1, n2) : m_axis_v<CT>(rb, cb, n1, n2), 1);
                const VT* I = IV + (mat == 0 ? 0 : (rb == cb ? (rb == 0 ? 1 : 3) : 2)) * Ku * Kv + ku * Kv;
                if constexpr (kFF) {
                    const dw v = c2_combine_dw(I, f);
                    sV[i] = make_float2(v.hi, v.lo);
                } else {
                    sV[i] = c2_combine(I, f);
                }
            }
            __syncthreads();
            for (int item = warp; item < 2 * rows; item += nwarp) {
                const int m1 = item >> 1, cb = item & 1;
                const int r = rbase + m1 * rw + n1, cw = cb == 0 ? N + 1 : N;
                const int count = cb == 0 ? nu : n - nu, c0 = cb == 0 ? 0 : nu;
                const float rc = 1.0f / (float)cw;
                const int sm2 = div_small(32, cw, rc), sn2 = 32 - sm2 * cw;
                int m2 = div_small(lane, cw, rc), n2 = lane - m2 * cw;
                double* Srow = Se + (int64_t)r * n + c0;
                double* Mrow = Me + (int64_t)r * n + c0;
                const VT* VS = sV + (0 * 2 + cb) * VB;
                const VT* VM = sV + (1 * 2 + cb) * VB;
                // the row's u-axis factors for every m2, lane m2 holding those of m2 (m2 <= M <= 24);
                // each entry takes its own by two shuffles per matrix (uniform trip counts below)
                int pS = 0, pM = 0;
                float cS = 0.f, cM = 0.f;
                if (lane <= M) {
                    const Fac<CT> fs = to_fac(s_axis_u<CT>(rb, cb, m1, lane), N + 1);
                    const Fac<CT> fm = to_fac(m_axis_u<CT>(rb, cb, m1, lane), N + 1);
                    pS = pack_fac(fs);
                    cS = fs.c;
                    pM = pack_fac(fm);
                    cM = fm.c;
                }
                for (int j0 = 0; j0 < count; j0 += 32) {
                    const int j = j0 + lane, src = min(m2, M);
                    const Fac<CT> fs = unpack_fac(__shfl_sync(0xffffffffu, pS, src), __shfl_sync(0xffffffffu, cS, src));
                    const Fac<CT> fm = unpack_fac(__shfl_sync(0xffffffffu, pM, src), __shfl_sync(0xffffffffu, cM, src));
                    if (j < count) {
                        __stcs(Srow + j, c2_combine(VS + n2, fs));
                        __stcs(Mrow + j, c2_combine(VM + n2, fm));
                    }
                    m2 += sm2;
                    n2 += sn2;
                    if (n2 >= cw) { n2 -= cw; ++m2; }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && bad && L.err_flag) atomicCAS(L.err_flag, 0, P2S_ERR_JACOBIAN);
        __syncthreads();
    }
}

// Direct numerical integration (the paper's comparison method): every entry of S and M is its own
// sum over the G x G points, S_rc = sum_ab w_a w_b phi_r phi_c / (mu J) with the curl factors and
// M_rc the same with the block's mass coupling; the coupling factors of the element are staged in
// shared memory once, the 1-D values in tables.  One thread per (row, column) entry pair.
__global__ void __launch_bounds__(kC2Threads) k_cheb2d_direct(C2Launch L) {
    extern __shared__ double sm[];
    const int M = L.M, N = L.N, G = L.G;
    const int K = max(M, N) + 1, gs = G | 1;
    double* sT = sm;           // T_k(x_a)
    double* sU = sT + K * gs;  // U_k(x_a)
    double* sN = sU + K * gs;  // T^ns_k(x_a) (not used by this method)
    double* sx = sN + K * gs;
    double* sw = sx + G;
    double* sc = sw + G;       // [4][G][G]: w_a w_b c_s(a, b) at (b * G + a)
    __shared__ int bad;
    const int nu = M * (N + 1), n = nu + (M + 1) * N;
    c2_tables(L, K, gs, false, sT, sU, sN, sx, sw);
    for (int64_t e = blockIdx.x; e < L.n_elem; e += gridDim.x) {
        const double* p = L.params + 5 * e;
        if (threadIdx.x == 0) bad = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < G * G; i += blockDim.x) {
            const int b = i / G, a = i - b * G;
            double c[4];
            if (!c2_couplings(p, sx[a], sx[b], c)) bad = 1;
            const double ww = sw[a] * sw[b];
#pragma unroll
            for (int s = 0; s < 4; ++s) sc[s * G * G + i] = ww * c[s];
        }
        __syncthreads();
        double* Se = L.S + e * (int64_t)n * n;
        double* Me = L.Mm + e * (int64_t)n * n;
        for (int64_t i = threadIdx.x; i < (int64_t)n * n; i += blockDim.x) {
            const int r = (int)(i / n), c = (int)(i - (int64_t)r * n);
            const bool ru = r < nu, cu = c < nu;
            const int rr = ru ? r : r - nu, rw = ru ? N + 1 : N, cc = cu ? c : c - nu, cw = cu ? N + 1 : N;
            const int m1 = rr / rw, n1 = rr - m1 * rw, m2 = cc / cw, n2 = cc - m2 * cw;
            // per axis: the S factors (U_{.} or U_{.-1} with the curl scale) and the M factors
            // (U or T), as table rows; a negative index is the zero polynomial U_{-1}
            int su1, su2, sv1, sv2, mu1, mu2, mv1, mv2;
            const double *SU1, *SU2, *SV1, *SV2, *MU1, *MU2, *MV1, *MV2;
            double sscale;
            const double* cM;
            if (ru) { su1 = m1; sv1 = n1 - 1; SU1 = sU; SV1 = sU; mu1 = m1; mv1 = n1; MU1 = sU; MV1 = sT; }
            else { su1 = m1 - 1; sv1 = n1; SU1 = sU; SV1 = sU; mu1 = m1; mv1 = n1; MU1 = sT; MV1 = sU; }
            if (cu) { su2 = m2; sv2 = n2 - 1; SU2 = sU; SV2 = sU; mu2 = m2; mv2 = n2; MU2 = sU; MV2 = sT; }
            else { su2 = m2 - 1; sv2 = n2; SU2 = sU; SV2 = sU; mu2 = m2; mv2 = n2; MU2 = sT; MV2 = sU; }
            sscale = (ru ? -(double)n1 : (double)m1) * (cu ? -(double)n2 : (double)m2);
            cM = sc + (ru && cu ? 1 : (!ru && !cu ? 3 : 2)) * G * G;
            const bool szero = su1 < 0 || su2 < 0 || sv1 < 0 || sv2 < 0;
            double accS = 0.0, accM = 0.0;
            for (int b = 0; b < G; ++b) {
                const double vs = szero ? 0.0 : SV1[sv1 * gs + b] * SV2[sv2 * gs + b];
                const double vm = MV1[mv1 * gs + b] * MV2[mv2 * gs + b];
                const double* cSb = sc + b * G;
                const double* cMb = cM + b * G;
                for (int a = 0; a < G; ++a) {
                    const double us = szero ? 0.0 : SU1[su1 * gs + a] * SU2[su2 * gs + a];
                    const double um = MU1[mu1 * gs + a] * MU2[mu2 * gs + a];
                    accS = fma(us * vs, cSb[a], accS);
                    accM = fma(um * vm, cMb[a], accM);
                }
            }
            Se[i] = sscale * accS;
            Me[i] = accM;
        }
        if (threadIdx.x == 0 && bad && L.err_flag) atomicCAS(L.err_flag, 0, P2S_ERR_JACOBIAN);
        __syncthreads();
    }
}

size_t p2s_smem_bytes(int M, int N, int G) {
    const int Ku = 2 * M + 1, Kv = 2 * N + 1, K = std::max(Ku, Kv), gs = G | 1;
    return sizeof(double) * ((size_t)3 * K * gs + G + 4 * kC2Chunk * G + 4 * kC2Chunk * K + 4 * (size_t)Ku * Kv + G +
                             4 * (size_t)Ku * (N + 1));
}
size_t direct_smem_bytes(int M, int N, int G) {
    const int K = std::max(M, N) + 1, gs = G | 1;
    return sizeof(double) * ((size_t)3 * K * gs + 2 * G + 4 * (size_t)G * G);
}

}  // namespace
}  // namespace p2s

using namespace p2s;

extern "C" {

int64_t p2s_cheb2d_dofs(int M, int N) {
    if (M < 1 || N < 1 || M > kC2MaxOrder || N > kC2MaxOrder) return P2S_ERR_ORDER;
    return (int64_t)M * (N + 1) + (int64_t)(M + 1) * N;
}

int p2s_cheb2d_fill(p2s_ctx* ctx, int64_t n_elem, const double* params, int M, int N, int npts, int method,
                    int precision, double* S, double* Mass, void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T) return fail(P2S_ERR_ARG, "p2s_cheb2d_fill: NULL context");
    if (n_elem < 0 || (n_elem > 0 && (!params || !S || !Mass)))
        return fail(P2S_ERR_ARG, "p2s_cheb2d_fill: bad element count or NULL buffer");
    if (method != P2S_CHEB2D_P2S && method != P2S_CHEB2D_DIRECT) return fail(P2S_ERR_ARG, "p2s_cheb2d_fill: method");
    if (precision != P2S_FP64 && (precision != P2S_MIXED || method != P2S_CHEB2D_P2S))
        return fail(P2S_ERR_ARG, "p2s_cheb2d_fill: precision (mixed is a product-to-sum option)");
    if (p2s_cheb2d_dofs(M, N) < 0 || npts < 1 || npts > kC2MaxG)
        return fail(P2S_ERR_ORDER, "p2s_cheb2d_fill: M, N outside 1..24 or npts outside 1..48");
    if (n_elem == 0) return P2S_OK;
    P2S_CUDA(cudaSetDevice(T->device));
    C2Launch L;
    L.params = params;
    L.n_elem = n_elem;
    L.M = M;
    L.N = N;
    L.G = npts;
    L.gl_x = T->gl_x;
    L.gl_w = T->gl_w;
    L.S = S;
    L.Mm = Mass;
    L.err_flag = T->err;
    const bool p2s = method == P2S_CHEB2D_P2S;
    const size_t smem = p2s ? p2s_smem_bytes(M, N, npts) : direct_smem_bytes(M, N, npts);
    if (smem > T->smem_optin) return fail(P2S_ERR_ORDER, "p2s_cheb2d_fill: tables exceed shared memory");
    const bool ff = precision == P2S_MIXED;
    const void* kern = p2s ? (ff ? (const void*)k_cheb2d_p2s<true> : (const void*)k_cheb2d_p2s<false>)
                           : (const void*)k_cheb2d_direct;
    P2S_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    const int threads = p2s ? kC2P2SThreads : kC2Threads;
    P2S_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    const int grid = (int)std::min<int64_t>(n_elem, (int64_t)std::max(1, per_sm) * T->sm_count);
    if (p2s && ff) k_cheb2d_p2s<true><<<grid, threads, smem, (cudaStream_t)stream>>>(L);
    else if (p2s) k_cheb2d_p2s<false><<<grid, threads, smem, (cudaStream_t)stream>>>(L);
    else k_cheb2d_direct<<<grid, kC2Threads, smem, (cudaStream_t)stream>>>(L);
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}

}  // extern "C"
