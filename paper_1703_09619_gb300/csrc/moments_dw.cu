// Steps a1 + a2 in double-word arithmetic for the mixed-precision path: the coupling
// factor alpha of Eq. (2) of arXiv:1703.09619 at the Gauss-Legendre points and the
// moment tensors I_s[k,l,q] of Eq. (4), with every per-point operation in float-float
// (hi + lo FP32 pairs, dw.cuh) and no FP64 instruction per point.  FP64 is used once per
// element to set up its constants (trilinear coefficients, 1-D node tables), which are
// then split into double words.
//
// Same sum factorisation as k_moments_fp64 (moments.cu): per chunk of up to 256 points
// (rows b0 .. b0+nbc-1 of plane c)
//   A: alpha at the chunk's points,
//   B: T1[s][b][k] = sum_a B[k][a] alpha[s][b][a],
//   C: T2_c[s][k][l] (+)= sum_b B[l][b] T1[s][b][k],
//   D: after the last chunk of plane c, I[s][k][l][q] (+)= B[q][c] T2_c[s][k][l].
// The steps are software-pipelined over the chunks of an element: in one interval between
// two CTA barriers the threads compute the row constants of chunk t+1, A of chunk t, B of
// chunk t-1, C of chunk t-2 and D of the plane whose last chunk was t-3, on double buffers
// (row constants, alpha and T1 by chunk parity, T2 by plane parity), so an element of T
// chunks takes T + 3 barriers and the B/C/D work is one balanced list over all threads.
//
// For the metric kind, the parts of the Jacobian and of the phase k.x that do not depend on
// u are formed once per (v, w) row:
//   J_iu = B_i(v,w) + g_i dbeta/du,
//   J_iv = D_i(w) + u E_i(w) + g_i dbeta/dv,
//   J_iw = F_i(v) + u H_i(v) + g_i dbeta/dw,
//   k.x  = T0(v,w) + u T1(v,w) + kappa beta,   beta = cos(pi u/2) cos(pi v/2) cos(pi w/2).
// Output: the moment tensors as (hi, lo) FP32 pairs in the moment layout.
#include <cmath>

#include "alpha.cuh"
#include "alpha_dw.cuh"
#include "dw.cuh"
#include "dw2.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;
constexpr int kNB = 16;
constexpr int kRow = 14;   // per-row constants: B_i, F_i, H_i (9), T0, T1, P1, P2, P3
constexpr int kPlane = 6;  // per-plane constants: D_i, E_i
constexpr int kGeoDW = 40;

// The B table, the alpha, T1 and T2 buffers and the moment accumulator hold coupling pairs
// in pair slots: slot sp carries pairs 2 sp and 2 sp + 1 as one dw2 (lanes x and y), so that
// phases B, C and D advance both pairs with one packed instruction per FP32 operation.  The B
// table entries are duplicated into both lanes.  A group with an odd number of pairs leaves
// lane y of its last slot zero and never stores it.
struct SmemDW {
    dw2 *B, *alpha, *T1, *T2, *Iacc;
    dw *xq, *t0, *t1, *t2, *geo, *row, *plane;
    double* geo64;
};

// B-table rows are padded to an odd number of double-words so that threads reading the
// same column of different rows hit different banks.
__host__ __device__ __forceinline__ int padded_stride(int gmax) { return gmax | 1; }

// Pair slots of n_pairs coupling pairs.
__host__ __device__ __forceinline__ int pair_slots(int n_pairs) { return (n_pairs + 1) / 2; }

// Sizes (16-byte pair-slot entries) of one buffer of each double-buffered array.
// Folded alpha of a chunk, per pair: the even part E[bb][p] = alpha(p) + alpha(G-1-p) and the
// odd part O[bb][p] = alpha(p) - alpha(G-1-p), p < H = ceil(G/2) (for odd G the middle point
// has E = alpha, O = 0), each in rows of odd stride (H | 1) so that phase-B reads of different
// rows fall in different banks.  nb * (H | 1) <= 160 for every G; the odd part starts 164
// entries (656 words: 16 banks) after the even one, so the two parities of a row do not collide.
constexpr int kFoldHalf = 164;
constexpr int kAlphaPair = 2 * kFoldHalf;
__host__ __device__ __forceinline__ int alpha_buf(int n_pairs) { return pair_slots(n_pairs) * kAlphaPair; }
__host__ __device__ __forceinline__ int t1_buf(int n_pairs, int kb) { return pair_slots(n_pairs) * kNB * kb; }
__host__ __device__ __forceinline__ int t2_buf(int n_pairs, int kb) { return pair_slots(n_pairs) * kb * kb; }

// iacc_cap counts double-words (two per pair-slot entry; even); the dw2 arrays come first, so
// every one starts on a 16-byte boundary.
__device__ __forceinline__ SmemDW carve_dw(unsigned char* sm, int n_pairs, int kb, int gmax, int iacc_cap) {
    SmemDW S;
    S.B = reinterpret_cast<dw2*>(sm);
    S.alpha = S.B + kb * padded_stride(gmax);
    S.T1 = S.alpha + 2 * alpha_buf(n_pairs);
    S.T2 = S.T1 + 2 * t1_buf(n_pairs, kb);
    S.Iacc = S.T2 + 2 * t2_buf(n_pairs, kb);
    S.xq = reinterpret_cast<dw*>(S.Iacc + iacc_cap / 2);
    S.t0 = S.xq + gmax;
    S.t1 = S.t0 + gmax;
    S.t2 = S.t1 + gmax;
    S.geo = S.t2 + gmax;
    S.row = S.geo + kGeoDW;
    S.plane = S.row + 2 * kNB * kRow;
    S.geo64 = reinterpret_cast<double*>(S.plane + 2 * kPlane);
    return S;
}

__device__ __forceinline__ void pair_comps_dw(int s, int n_comp, int& gi, int& gj) {
    if (n_comp == 1) { gi = gj = 0; return; }
    const int tgi[6] = {0, 0, 0, 1, 1, 2}, tgj[6] = {0, 1, 2, 1, 2, 2};
    gi = tgi[s];
    gj = tgj[s];
}

// Rows per chunk: as few chunks per plane as the 256 lanes allow
// (lr lanes per row), with the rows spread evenly over them (G = 24: 8 + 8 + 8 rather than
// 10 + 10 + 4; G = 48 keeps 5 rows, as 4 would add two chunks per plane).
__host__ __device__ constexpr int rows_per_chunk(int G, int lr) {
    const int cap = kChunk / lr < 1 ? 1 : (kChunk / lr < G ? kChunk / lr : G);
    const int ncp = (G + cap - 1) / cap;
    return (G + ncp - 1) / ncp;
}

// Chunk t of an element: plane c, first row b0, nbc rows.
struct Chunk {
    int c, b0, nbc;
};

// n / d with d a compile-time constant when D > 0 (a multiply-shift), else by the FP32
// reciprocal rd of the runtime d.
template <int D>
__device__ __forceinline__ int div_ct(int n, int d, float rd) {
    if constexpr (D > 0) return n / D;
    else return div_small(n, d, rd);
}

template <int NCP>
__device__ __forceinline__ Chunk chunk_of_ct(int t, int ncp, float rncp, int nb, int G) {
    Chunk ch;
    ch.c = div_ct<NCP>(t, ncp, rncp);
    ch.b0 = (t - ch.c * ncp) * nb;
    ch.nbc = min(nb, G - ch.b0);
    return ch;
}

// One task of the row/plane constants of a chunk (metric kind): tasks 4 bb + i (i < 3) form
// B_i, F_i, H_i of row bb, task 4 bb + 3 forms T0, T1 and the three cosine products of row
// bb, tasks 4 nbc + i form D_i and E_i of the chunk's plane.
__device__ __forceinline__ void metric_constants_task(const SmemDW& S, const Chunk& ch, int task, dw* row, dw* plane) {
    const dw* cf = S.geo;
    const dw w = S.xq[ch.c];
    if (task < 4 * ch.nbc) {
        const int bb = task >> 2, part = task & 3, b = ch.b0 + bb;
        const dw v = S.xq[b];
        dw* r = row + bb * kRow;
        if (part < 3) {
            const dw* ci = cf + 8 * part;
            r[part] = dw_fma_fast(ci[7], dw_mul_fast(v, w), dw_fma_fast(ci[5], w, dw_fma_fast(ci[4], v, ci[1])));  // B_i
            r[3 + part] = dw_fma_fast(ci[6], v, ci[3]);                                                         // F_i
            r[6 + part] = dw_fma_fast(ci[7], v, ci[5]);                                                         // H_i
        } else {
            const dw* th = cf + 31;
            const dw vw = dw_mul_fast(v, w);
            r[9] = dw_fma_fast(th[6], vw, dw_fma_fast(th[3], w, dw_fma_fast(th[2], v, th[0])));   // T0
            r[10] = dw_fma_fast(th[7], vw, dw_fma_fast(th[5], w, dw_fma_fast(th[4], v, th[1])));  // T1
            r[11] = dw_mul_fast(S.t0[b], S.t0[ch.c]);  // cos cos      (beta / cos_u)
            r[12] = dw_mul_fast(S.t1[b], S.t0[ch.c]);  // dcos_v cos_w
            r[13] = dw_mul_fast(S.t0[b], S.t1[ch.c]);  // cos_v dcos_w
        }
    } else {
        const int i = task - 4 * ch.nbc;  // plane constants D_i, E_i (J_iv = D_i + u E_i + ...)
        const dw* ci = cf + 8 * i;
        plane[i] = dw_fma_fast(ci[6], w, ci[2]);
        plane[3 + i] = dw_fma_fast(ci[7], w, ci[4]);
    }
}

// The pipelined steps and the moment write-out of one element (the 1-D tables and element
// constants are in shared memory).  GC, KC > 0 fix G and the moment count per axis (metric
// kind, Ku = Kv = Kw = KC, all six pairs in one group) at compile time, which turns the chunk
// shape, the item decoding and every loop bound into constants; GC = KC = 0 takes them from
// the element at run time.
template <int GC, int KC>
__device__ __forceinline__ void element_pipeline(const MomentLaunch& L, const SmemDW& S, const ElemDesc& d, int Grt,
                                                 bool metric_rt, int gstride, int aS, int t1S, int t2S, int* bad_jac,
                                                 int* item_ctr) {
    constexpr bool kSpec = GC > 0 && KC > 0;
    const int tid = threadIdx.x;
    const int G = kSpec ? GC : Grt;
    const bool metric = kSpec ? true : metric_rt;
    const int nc = d.n_comp, np = kSpec ? 6 : ((nc == 1) ? 1 : 6);
    const int Ku = kSpec ? KC : d.kax[0], Kv = kSpec ? KC : d.kax[1], Kw = kSpec ? KC : d.kax[2];
    const int Kb = kSpec ? KC : max(Ku, max(Kv, Kw));
    constexpr int KCs = kSpec ? KC : 0;
    constexpr int HC = kSpec ? (GC + 1) / 2 : 0, LRC = 2 * HC;
    constexpr int NBC = kSpec ? rows_per_chunk(GC, LRC) : 0;
    constexpr int NCPC = kSpec ? (GC + NBC - 1) / NBC : 0;
    const int per_pair = Ku * Kv * Kw;
    // pairs per group: whole pair slots of the accumulator (the host sizes it for at least
    // one slot, so groups of several pairs start at even pairs)
    const int ppg = kSpec ? 6 : max(1, min(np, 2 * (L.iacc_cap / (2 * per_pair))));
    const int H = (G + 1) / 2, LR = 2 * H, Hs = H | 1;  // folded half, lanes per row, row stride
    const float rKu = 1.f / (float)Ku, rKv = 1.f / (float)Kv, rLR = 1.f / (float)LR;
    const int nb = kSpec ? NBC : rows_per_chunk(G, LR);
    const int ncp = kSpec ? NCPC : (G + nb - 1) / nb;  // chunks per plane
    const float rncp = 1.f / (float)ncp;
    const int T = G * ncp;
    for (int s0 = 0; s0 < np; s0 += ppg) {
        const int ns = min(np, s0 + ppg) - s0, nsp = pair_slots(ns);
        for (int step = -1; step < T + 3; ++step) {
            // row / plane constants of chunk step + 1 (tasks on the highest threads)
            if (step + 1 < T) {
                const int t = step + 1;
                const Chunk ch = chunk_of_ct<NCPC>(t, ncp, rncp, nb, G);
                dw* row = S.row + (t & 1) * kNB * kRow;
                const int task = kThreads - 1 - tid;
                if (metric) {
                    if (task < 4 * ch.nbc + 3) metric_constants_task(S, ch, task, row, S.plane + (t & 1) * kPlane);
                } else if (task < ch.nbc) {
                    row[task * kRow] = dw_mul_fast(S.t1[ch.b0 + task], S.t2[ch.c]);
                }
            }
            // A: alpha of chunk step, at mirrored points in neighbouring lanes: lane pair
            // (2 i, 2 i + 1) of row bb takes points p and G-1-p (p = i mod H), swaps values
            // with one shuffle per word and stores the folded E (even lane) and O (odd lane)
            if (step >= 0 && step < T) {
                const Chunk ch = chunk_of_ct<NCPC>(step, ncp, rncp, nb, G);
                const dw* row = S.row + (step & 1) * kNB * kRow;
                dw2* al = S.alpha + (step & 1) * aS;
                const bool lane_on = tid < ch.nbc * LR;
                const int bb = div_ct<LRC>(tid, LR, rLR), r = tid - bb * LR, p = r >> 1, side = r & 1;
                const bool middle = 2 * p + 1 == G;  // odd G: its middle point, taken by the even lane
                const bool active = lane_on && !(middle && side);
                const int a = side ? G - 1 - p : p;
                dw K[6];
#pragma unroll
                for (int s = 0; s < 6; ++s) K[s] = dw_from_float(0.f);
                if (active) {
                    if (!metric) {
                        K[0] = dw_add_f(dw_mul_fast(S.t0[a], row[bb * kRow]), 1.f);
                    } else {
                        const bool ok = metric_alpha_dw(S.geo, row + bb * kRow, S.plane + (step & 1) * kPlane,
                                                        S.xq[a], S.t0[a], S.t1[a], K);
                        if (!ok) *bad_jac = 1;
                    }
                }
                const int ia = (side ? kFoldHalf : 0) + bb * Hs + p;
                // pairs sa and sa + 1 in one slot (s0 is even whenever a group holds several pairs)
#pragma unroll
                for (int sa = 0; sa < 6; sa += 2) {
                    if (sa >= s0 && sa < s0 + ns) {  // uniform across the CTA: every lane shuffles
                        const dw2 k2 = dw2_make(K[sa], sa + 1 < s0 + ns ? K[sa + 1] : dw_from_float(0.f));
                        const dw2 o = dw2{f2{__shfl_xor_sync(0xffffffffu, k2.hi.v, 1)},
                                          f2{__shfl_xor_sync(0xffffffffu, k2.lo.v, 1)}};
                        // even lane K + o, odd lane o + (-K) (dw_add_fast / dw_sub_fast per pair)
                        dw2 f = dw2_add_fast(side ? o : k2, side ? dw2_neg(k2) : o);
                        if (side && middle) f = dw2_zero();
                        if (lane_on) al[((sa - s0) >> 1) * kAlphaPair + ia] = f;
                    }
                }
            }
            // B of chunk step - 1, C of chunk step - 2, D of the plane whose last chunk is step - 3
            const int tb = step - 1, tc = step - 2, td = step - 3;
            Chunk cb{0, 0, 0}, cc{0, 0, 0};
            int nB = 0, nC = 0, nD = 0, pd = -1;
            if (tb >= 0 && tb < T) {
                cb = chunk_of_ct<NCPC>(tb, ncp, rncp, nb, G);
                nB = nsp * cb.nbc * Ku;
            }
            if (tc >= 0 && tc < T) {
                cc = chunk_of_ct<NCPC>(tc, ncp, rncp, nb, G);
                nC = nsp * Ku * Kv;
            }
            if (td >= 0 && td < T) {
                const int pt = div_ct<NCPC>(td, ncp, rncp);
                if (td - pt * ncp == ncp - 1) pd = pt;
            }
            if (pd >= 0) {
                nD = nsp * Ku * Kv;
            }
            // items run on pair slots sp: both pairs of a slot advance together
            const dw2* alB = S.alpha + (tb & 1) * aS;
            dw2* t1B = S.T1 + (tb & 1) * t1S;
            const dw2* t1C = S.T1 + (tc & 1) * t1S;
            dw2* t2C = S.T2 + (cc.c & 1) * t2S;
            const dw2* t2D = S.T2 + (pd & 1) * t2S;
            const float r_nbc = 1.f / (float)max(cb.nbc, 1);
            // The items go to warps as they come free (a warp takes 32 at a time from the
            // step's counter), so the threads without a point in this chunk, and those done
            // with alpha first, take more of them.  The counters alternate with the step;
            // thread 0 clears the one the next step uses, which no thread touches in this one.
            const int nItems = nB + nC + nD;
            int* ctr = item_ctr + (step & 1);
            if (tid == 0) item_ctr[(step + 1) & 1] = 0;
            for (;;) {
                int base = nItems;
                if ((tid & 31) == 0 && nItems > 0) base = atomicAdd(ctr, 32);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= nItems) break;
                const int j = base + (tid & 31);
                if (j < nItems) {
                    if (j < nB) {
                        // T1[s][bb][k] = sum_a B[k][a] alpha[s][bb][a]
                        //              = sum_{p<H} B[k][p] (k even ? E : O)[s][bb][p],
                        // since B[k][G-1-p] = (-1)^k B[k][p] on the symmetric rule; k fastest
                        // across threads, so the folded reads are near-broadcasts and the B rows
                        // (odd stride) spread
                        const int sb = div_ct<KCs>(j, Ku, rKu), k = j - sb * Ku;
                        const int sp = div_small(sb, cb.nbc, r_nbc), bb = sb - sp * cb.nbc;
                        const dw2* al = alB + sp * kAlphaPair + (k & 1) * kFoldHalf + bb * Hs;
                        const dw2* Bk = S.B + k * gstride;
                        dw2_acc acc;
#pragma unroll 4
                        for (int p = 0; p < H; ++p) acc.fma(Bk[p], al[p]);
                        t1B[(sp * kNB + bb) * Kb + k] = acc.value();
                    } else if (j < nB + nC) {
                        // T2[s][k][l] (+)= sum_bb B[l][b0 + bb] T1[s][bb][k]
                        const int i = j - nB;
                        const int sk = div_ct<KCs>(i, Kv, rKv), l = i - sk * Kv;
                        const int sp = div_ct<KCs>(sk, Ku, rKu), k = sk - sp * Ku;
                        const dw2* t1 = t1C + sp * kNB * Kb + k;
                        const dw2* Bl = S.B + l * gstride + cc.b0;
                        dw2_acc acc;
                        if (cc.b0 > 0) {
                            acc.s = t2C[i].hi;
                            acc.c = t2C[i].lo;
                        }
                        for (int bb = 0; bb < cc.nbc; ++bb) acc.fma(Bl[bb], t1[bb * Kb]);
                        t2C[i] = acc.value();
                    } else {
                        // I[s][k][l][q] (+)= B[q][c] T2_c[s][k][l] for all q of one (s, k, l)
                        const int skl = j - nB - nC;
                        const dw2 t2 = t2D[skl];
                        dw2* I = S.Iacc + skl * Kw;
#pragma unroll
                        for (int q = 0; q < (kSpec ? KC : Kw); ++q) {
                            dw2_acc acc;
                            if (pd > 0) {
                                acc.s = I[q].hi;
                                acc.c = I[q].lo;
                            }
                            acc.fma(S.B[q * gstride + pd], t2);
                            I[q] = acc.value();
                        }
                    }
                }
            }
            __syncthreads();
        }
        for (int s = 0; s < ns; ++s) {
            int gi, gj;
            pair_comps_dw(s0 + s, nc, gi, gj);
            const int ku = d.ord[gi][0] + d.ord[gj][0] - 1, kv = d.ord[gi][1] + d.ord[gj][1] - 1,
                      kw = d.ord[gi][2] + d.ord[gj][2] - 1;
            float2* dst = reinterpret_cast<float2*>(L.mom + d.mom_off + d.pair_off[s0 + s]);
            const dw2* src = S.Iacc + (s >> 1) * per_pair;
            for (int i = tid; i < ku * kv * kw; i += kThreads) {
                const int k = i / (kv * kw), r = i - k * kv * kw, l = r / kw, q = r - l * kw;
                const dw2 v2 = src[(k * Kv + l) * Kw + q];
                const dw v = (s & 1) ? dw2_y(v2) : dw2_x(v2);
                dst[i] = make_float2(v.hi, v.lo);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_moments_dw(MomentLaunch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int tid = threadIdx.x;
    SmemDW S = carve_dw(smraw, L.n_pairs, L.kb, L.gmax, L.iacc_cap);
    __shared__ int bad_jac;
    const int gstride = padded_stride(L.gmax);
    const bool metric = L.kind == P2S_ALPHA_METRIC_EPS;
    const int aS = alpha_buf(L.n_pairs), t1S = t1_buf(L.n_pairs, L.kb), t2S = t2_buf(L.n_pairs, L.kb);

    __shared__ long long s_elem;
    __shared__ int s_item[2];  // per-step item counters of the element pipeline
    __shared__ int s_tabG, s_tabK;  // G and K of the 1-D tables in shared memory (-1: none yet)
    if (tid == 0) {
        s_tabG = -1;
        s_tabK = -1;
    }
    __syncthreads();
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
        if (L.elem_mask && !L.elem_mask[e]) continue;
        const ElemDesc& d = L.desc[e];
        const int G = d.G, nc = d.n_comp, np = (nc == 1) ? 1 : 6;
        const int Ku = d.kax[0], Kv = d.kax[1], Kw = d.kax[2];
        const int Kb = max(Ku, max(Kv, Kw));
        if (tid == 0) bad_jac = 0;
        const double* prm = L.params + 4 * e;
        // the 1-D tables depend on G and K alone for the metric kind: kept while consecutive
        // elements of this CTA share them (the queue hands out elements grouped by G)
        const bool keep = metric && s_tabG == G && s_tabK == Kb;
        if (tid < G && !keep) {  // 1-D tables, FP64 once per node, then split
            const double x = L.gl_x[G * kMaxG + tid], w = L.gl_w[G * kMaxG + tid];
            S.xq[tid] = dw_from_double(x);
            double p0 = 1.0, p1 = x;
            S.B[tid] = dw2_dup(dw_from_double(w));
            if (Kb > 1) S.B[gstride + tid] = dw2_dup(dw_from_double(w * x));
            for (int k = 1; k + 1 < Kb; ++k) {
                const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
                S.B[(k + 1) * gstride + tid] = dw2_dup(dw_from_double(w * p2));
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
        if (metric) {  // trilinear coefficients, one (coordinate, monomial) per thread, then the rest
            const double* X = L.nodes + 24 * e;
            if (tid < 24) {
                const int i = tid >> 3, j = tid & 7;
                double c = 0.0;
                for (int nd = 0; nd < 8; ++nd) {
                    const double su = (nd & 1) ? 1.0 : -1.0, sv = (nd & 2) ? 1.0 : -1.0, sw = (nd & 4) ? 1.0 : -1.0;
                    const double sgn = j == 0 ? 1.0 : j == 1 ? su : j == 2 ? sv : j == 3 ? sw
                                     : j == 4 ? su * sv : j == 5 ? su * sw : j == 6 ? sv * sw : su * sv * sw;
                    c += sgn * (0.125 * X[3 * nd + i]);
                }
                S.geo64[tid] = c;
            } else if (tid < 27) {
                const double* bg = L.bulge ? L.bulge + 4 * e : nullptr;
                S.geo64[tid] = bg ? bg[0] * bg[1 + (tid - 24)] : 0.0;
            }
        }
        __syncthreads();
        if (metric && tid < kGeoDW) {
            // geo layout: 0..23 coefficients of x, y, z; 24..26 bulge vector; 27 eps amplitude;
            // 31..38 coefficients of the phase k.x; 39 the phase of the bulge
            double g = 0.0;
            if (tid < 27) g = S.geo64[tid];
            else if (tid == 27) g = prm[0];
            else if (tid >= 31 && tid < 39) g = prm[1] * S.geo64[tid - 31] + prm[2] * S.geo64[tid - 23] + prm[3] * S.geo64[tid - 15];
            else if (tid == 39) g = prm[1] * S.geo64[24] + prm[2] * S.geo64[25] + prm[3] * S.geo64[26];
            S.geo[tid] = dw_from_double(g);
        }
        if (tid == 0) {
            s_tabG = metric ? G : -1;
            s_tabK = Kb;
        }
        __syncthreads();

        const bool spec = metric && np == 6 && Ku == 7 && Kv == 7 && Kw == 7 && L.iacc_cap >= 6 * 343;
        switch (spec ? G : 0) {
        case 8: element_pipeline<8, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        case 12: element_pipeline<12, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        case 16: element_pipeline<16, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        case 24: element_pipeline<24, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        case 32: element_pipeline<32, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        case 48: element_pipeline<48, 7>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
        default: element_pipeline<0, 0>(L, S, d, G, metric, gstride, aS, t1S, t2S, &bad_jac, s_item); break;
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
    const size_t e2 = (size_t)kb * padded_stride(gmax) + 2 * (size_t)alpha_buf(n_pairs) +
                      2 * (size_t)t1_buf(n_pairs, kb) + 2 * (size_t)t2_buf(n_pairs, kb);  // dw2 entries
    const size_t d = 2 * e2 + (size_t)iacc_cap + 4 * (size_t)gmax + kGeoDW + 2 * kNB * kRow + 2 * kPlane;
    return d * sizeof(dw) + 48 * sizeof(double);
}

// Accumulator of the double-word kernel in double-words: whole pair slots (two pairs each),
// at least one, for pairs of up to max_pair moments.
int moments_dw_iacc_words(int n_pairs, int max_pair) { return 2 * pair_slots(n_pairs) * max_pair; }

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
