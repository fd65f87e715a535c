// The first mode product of the sum-factorised moments (Eq. (4) of arXiv:1703.09619, the
// a-axis sum T[r][k] = sum_a B[k][a] x[r][a] with B[k][a] = w_a P_k(u_a) on the G-point
// Gauss-Legendre rule, k < 7) on rows of double-word samples, in two forms:
//
//   SIMT  (k_mode1_simt): the moment kernel's own phase B -- parity fold of the row
//         (E[p] = x[p] + x[G-1-p], O[p] = x[p] - x[G-1-p], p < G/2; even k take E, odd k O)
//         and double-word dot products on the FP32 pipe.
//   TC    (k_mode1_tc): the same fold, then split-precision tensor-core products.  Each
//         folded row is scaled by a power of two (its bound 2^e) and cut into S slices of
//         b = 8 bits, x ~ 2^e sum_i s_i 2^(-8(i+1)) with integer s_i, |s_0| <= 256 and
//         |s_i| <= 128 (i > 0), exact in FP16; the B table is cut the same way per column
//         k (host, FP64).  One tcgen05.mma chain (kind::f16, FP32 accumulation in TMEM,
//         M = 128 rows, K = slices x points) produces, per k, the level sums
//         D_L = sum_{i+j=L} sum_p s_i w_j for L < S: integers below 2^24, so the FP32
//         accumulation is exact.  The epilogue reads D from TMEM (tcgen05.ld) and forms
//         T = 2^(e+f_k-16) sum_L D_L 2^(-8L) as a double word.  Products with i + j >= S
//         are dropped: the relative error is about 2^(-8S) of max|B| max|x| per term.
//
// One CTA of 128 threads takes tiles of 128 rows (one row per thread, TMEM lane = row);
// the B images reach shared memory once per CTA by a bulk asynchronous copy (TMA) that
// completes on an mbarrier; thread 0 issues the MMAs and commits them to a second mbarrier
// that every thread waits on (each wait bounded by a clock budget: on expiry the kernel sets
// an error flag and leaves its tiles).
// Operands live in shared memory in the no-swizzle K-major layout: 8 x 16-byte core
// matrices, k-adjacent core matrices 128 B apart (LBO), 8-row groups KA/8 x 128 B apart
// (SBO).  Rows x come from a source array of n_src rows, row r reading source row r mod
// n_src, so that a small source can stay in L2; both forms stage each tile of 128 rows in
// shared memory with coalesced loads (the fused moment kernel holds its samples there too),
// so that the kernels' arithmetic is what is timed.  This is a measurement of the tensor-core form against the SIMT form on the
// same work (p2s_mode1_product); the fused moment kernel keeps the SIMT form.
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda_fp16.h>

#include "dw.cuh"
#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int kM1Threads = 128;
constexpr int kM1K = 7;       // moments per axis (N = 4)
constexpr int kBits = 8;      // bits per slice
constexpr int kMaxS = 5;      // slices
constexpr int kMaxH = 24;     // G <= 48
constexpr int kMaxKA = 128;   // K extent of one operand (slices x padded points)
constexpr int kNE = 32;       // D columns of the even-k part (levels x 4), padded to 32
constexpr int kNO = 16;       // D columns of the odd-k part (levels x 3), padded to 16
constexpr uint32_t kTmemCols = 64;

constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
__host__ __device__ constexpr int padded_h(int G) { return round_up(G / 2, 8); }
__host__ __device__ constexpr int ka_of(int G, int S) { return round_up(S * padded_h(G), 16); }

// Operand images of the TC form (B side, host-built) and the SIMT form's table.
__device__ __align__(128) unsigned char g_m1_bimg[(kNE + kNO) * kMaxKA * 2];
__constant__ float2 c_m1_B[kM1K][kMaxH];  // B[k][p], p < G/2, as (hi, lo)
__constant__ int c_m1_fexp[kM1K];         // column exponents f_k of the TC slices

// Byte offset of element (row, k) of a K-major no-swizzle operand with KA columns.
__host__ __device__ __forceinline__ int umma_off(int row, int k, int KA) {
    return (((row >> 3) * (KA >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, LBO, SBO (bytes, 16-byte units), version 1,
// no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D F32, A and B F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait for phase `parity` of an mbarrier: false if the clock budget ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// x * 2^k for a power-of-two scale built from its exponent (|k| < 126).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

template <int G>
__device__ __forceinline__ void load_pair(const float2* row, int p, dw& a, dw& b) {
    const float2 u = row[p], v = row[G - 1 - p];
    a = dw{u.x, u.y};
    b = dw{v.x, v.y};
}

// Row stride (float2) of a staged tile: odd, so that a warp's row-per-thread reads spread
// over the banks.
__host__ __device__ constexpr int tile_ld(int G) { return G + 1; }

// The 128 rows of tile t into shared memory, coalesced (consecutive threads take
// consecutive samples); rows past n_rows are zero.  As in the fused moment kernel, the
// samples a thread works on then come from shared memory.
template <int G>
__device__ __forceinline__ void stage_tile(const float2* __restrict__ x, int64_t n_rows, int64_t n_src, int64_t t,
                                           float2* sX) {
    for (int i = threadIdx.x; i < 128 * G; i += kM1Threads) {
        const int rr = i / G, a = i - rr * G;
        const int64_t r = t * 128 + rr;
        sX[rr * tile_ld(G) + a] = r < n_rows ? __ldg(x + (r % n_src) * G + a) : make_float2(0.f, 0.f);
    }
}

template <int G>
__global__ void __launch_bounds__(kM1Threads) k_mode1_simt(const float2* __restrict__ x, int64_t n_rows,
                                                           int64_t n_src, float2* __restrict__ out) {
    constexpr int H = G / 2;
    extern __shared__ __align__(16) unsigned char sm_simt[];
    float2* sX = reinterpret_cast<float2*>(sm_simt);
    const int64_t tiles = (n_rows + kM1Threads - 1) / kM1Threads;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        stage_tile<G>(x, n_rows, n_src, t, sX);
        __syncthreads();
        const int64_t r = t * kM1Threads + threadIdx.x;
        if (r < n_rows) {
            const float2* row = sX + threadIdx.x * tile_ld(G);
            dw_acc acc[kM1K];
#pragma unroll 4
            for (int p = 0; p < H; ++p) {
                dw a, b;
                load_pair<G>(row, p, a, b);
                const dw E = dw_add_fast(a, b), O = dw_sub_fast(a, b);
#pragma unroll
                for (int k = 0; k < kM1K; ++k) {
                    const float2 bk = c_m1_B[k][p];
                    acc[k].fma(dw{bk.x, bk.y}, (k & 1) ? O : E);
                }
            }
            float4* o = reinterpret_cast<float4*>(out + r * 8);
            dw v[8];
#pragma unroll
            for (int k = 0; k < kM1K; ++k) v[k] = acc[k].value();
            v[7] = dw{0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = make_float4(v[2 * q].hi, v[2 * q].lo, v[2 * q + 1].hi, v[2 * q + 1].lo);
        }
        __syncthreads();  // the tile buffer is free
    }
}

// Slices of one scaled double word (|y| < 2^8 after the first scaling): s_i = rint(y),
// y = (y - s_i) 2^8, renormalised.
template <int S>
__device__ __forceinline__ void cut(dw y, float* s) {
#pragma unroll
    for (int i = 0; i < S; ++i) {
        s[i] = rintf(y.hi);
        const dw r = fast_two_sum(y.hi - s[i], y.lo);
        y = dw{r.hi * 256.f, r.lo * 256.f};
    }
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int G, int S>
__global__ void __launch_bounds__(kM1Threads) k_mode1_tc(const float2* __restrict__ x, int64_t n_rows,
                                                         int64_t n_src, float2* __restrict__ out, int* err) {
    constexpr int H = G / 2, HP = padded_h(G), KA = ka_of(G, S);
    static_assert(G % 2 == 0 && H <= kMaxH && KA <= kMaxKA, "shape");
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* sAE = sm;                         // 128 x KA fp16, even part
    unsigned char* sAO = sAE + 128 * KA * 2;         // odd part
    unsigned char* sBE = sAO + 128 * KA * 2;         // kNE x KA
    unsigned char* sBO = sBE + kNE * KA * 2;         // kNO x KA
    float2* sX = reinterpret_cast<float2*>(sBO + kNO * KA * 2);  // 128 x tile_ld(G) samples
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;

    // zero A (its padding stays 0); the B images (host-built, K-major layout) arrive by one
    // bulk asynchronous copy (TMA, untiled) completing on s_tma
    for (int i = tid; i < 2 * 128 * KA * 2 / 16; i += kM1Threads) reinterpret_cast<uint4*>(sAE)[i] = make_uint4(0, 0, 0, 0);
    __shared__ __align__(8) unsigned long long s_tma;
    constexpr uint32_t kBBytes = (kNE + kNO) * KA * 2;  // a multiple of 16 (KA is)
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_tma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&s_tma)), "r"(kBBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sBE)),
            "l"(reinterpret_cast<uint64_t>(g_m1_bimg)), "r"(kBBytes), "r"(smem_u32(&s_tma))
            : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem, tE = tmem, tO = tmem + kNE;
    const uint32_t bar = smem_u32(&s_bar);
    const long long budget = 2000000000ll;  // about a second at the running clock
    if (!mbar_wait(smem_u32(&s_tma), 0, budget)) {  // the B images in place
        if (tid == 0) atomicExch(err, P2S_ERR_TIMEOUT);
        s_fail = 1;
    }
    __syncthreads();
    const uint32_t sbo = (KA / 8) * 128;
    const uint32_t aE = smem_u32(sAE), aO = smem_u32(sAO), bE = smem_u32(sBE), bO = smem_u32(sBO);
    constexpr uint32_t idE = idesc_f16(128, kNE), idO = idesc_f16(128, kNO);

    const int64_t tiles = (n_rows + 127) / 128;
    uint32_t phase = 0;
    for (int64_t t = s_fail ? tiles : blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t r = t * 128 + tid;
        const bool live = r < n_rows;
        stage_tile<G>(x, n_rows, n_src, t, sX);
        __syncthreads();
        const float2* row = sX + tid * tile_ld(G);
        // bound of the folded row: max_p |x_p| + |x_q| >= max(|E_p|, |O_p|)
        float m = 0.f;
#pragma unroll 4
        for (int p = 0; p < H; ++p) {
            const float2 u = row[p], v = row[G - 1 - p];
            m = fmaxf(m, fabsf(u.x) + fabsf(v.x));
        }
        int e = 0;
        if (m > 1e-30f) {
            frexpf(m * 1.0000002f, &e);  // m (1 + 2^-22) < 2^e
        }
        const float sc = live && m > 1e-30f ? pow2f(kBits - e) : 0.f;  // rows below 1e-30 give 0
        // fold, scale, cut; 8 points (one 16-byte core-matrix row per slice) at a time
#pragma unroll 1
        for (int g = 0; g < HP / 8; ++g) {
            uint32_t pe[S][4], po[S][4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float se[2][S], so[2][S];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int p = g * 8 + j + h;
                    dw E{0.f, 0.f}, O{0.f, 0.f};
                    if (p < H) {
                        dw a, b;
                        load_pair<G>(row, p, a, b);
                        E = dw_add_fast(a, b);
                        O = dw_sub_fast(a, b);
                    }
                    cut<S>(dw{E.hi * sc, E.lo * sc}, se[h]);
                    cut<S>(dw{O.hi * sc, O.lo * sc}, so[h]);
                }
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    pe[i][j / 2] = pack_h2(se[0][i], se[1][i]);
                    po[i][j / 2] = pack_h2(so[0][i], so[1][i]);
                }
            }
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const int k0 = i * HP + g * 8;
                *reinterpret_cast<uint4*>(sAE + umma_off(tid, k0, KA)) = make_uint4(pe[i][0], pe[i][1], pe[i][2], pe[i][3]);
                *reinterpret_cast<uint4*>(sAO + umma_off(tid, k0, KA)) = make_uint4(po[i][0], po[i][1], po[i][2], po[i][3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int j = 0; j < KA / 16; ++j) {
                mma_f16(tE, umma_desc(aE + j * 256, 128, sbo), umma_desc(bE + j * 256, 128, sbo), idE, j > 0);
                mma_f16(tO, umma_desc(aO + j * 256, 128, sbo), umma_desc(bO + j * 256, 128, sbo), idO, j > 0);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
        }
        const bool ok = mbar_wait(bar, phase, budget);
        phase ^= 1;
        if (!ok) {
            if (tid == 0) atomicExch(err, P2S_ERR_TIMEOUT);
            s_fail = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (s_fail) break;  // uniform: written before the barrier
        float de[kNE], dO[kNO];
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        tmem_ld16(tE + lane_base, de);
        tmem_ld16(tE + lane_base + 16, de + 16);
        tmem_ld16(tO + lane_base, dO);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (live) {
            dw v[8];
#pragma unroll
            for (int k = 0; k < kM1K; ++k) {
                const float* D = (k & 1) ? dO : de;
                const int j = k >> 1, cs = (k & 1) ? 3 : 4;
                // sum_L D_L 2^(-8L): the two leading levels exactly, the rest into the low word
                const dw h = two_sum(D[j], D[cs + j] * (1.f / 256.f));
                float lo = h.lo;
                float w = 1.f / 65536.f;
#pragma unroll
                for (int L = 2; L < S; ++L) {
                    lo = fmaf(D[cs * L + j], w, lo);
                    w *= 1.f / 256.f;
                }
                const dw s = fast_two_sum(h.hi, lo);
                const float f = pow2f(e + c_m1_fexp[k] - 2 * kBits);
                v[k] = dw{s.hi * f, s.lo * f};
            }
            v[7] = dw{0.f, 0.f};
            float4* o = reinterpret_cast<float4*>(out + r * 8);
#pragma unroll
            for (int i = 0; i < 4; ++i) o[i] = make_float4(v[2 * i].hi, v[2 * i].lo, v[2 * i + 1].hi, v[2 * i + 1].lo);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();  // every thread's TMEM reads done before the next tile's MMAs
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

template <int G, int S>
size_t tc_smem() {
    return (size_t)(2 * 128 + kNE + kNO) * ka_of(G, S) * 2 + sizeof(float2) * 128 * tile_ld(G);
}

// Host tables of one rule: B[k][p] (p < G/2) and the TC images with their column exponents.
struct M1Tables {
    float2 B[kM1K][kMaxH];
    int fexp[kM1K];
    unsigned char img[(kNE + kNO) * kMaxKA * 2];
};

void build_tables(int G, int S, M1Tables& T) {
    std::memset(&T, 0, sizeof(T));
    const HostTables& H = host_tables();
    const int h = G / 2, HP = padded_h(G), KA = ka_of(G, S);
    double Bk[kM1K][kMaxH];
    for (int p = 0; p < h; ++p) {
        const double u = H.gl_x[G][p], w = H.gl_w[G][p];
        double p0 = 1.0, p1 = u;
        Bk[0][p] = w;
        Bk[1][p] = w * u;
        for (int k = 1; k + 1 < kM1K; ++k) {
            const double p2 = ((2 * k + 1) * u * p1 - k * p0) / (k + 1);
            Bk[k + 1][p] = w * p2;
            p0 = p1;
            p1 = p2;
        }
    }
    for (int k = 0; k < kM1K; ++k) {
        double mx = 0.0;
        for (int p = 0; p < h; ++p) {
            const float hi = (float)Bk[k][p];
            T.B[k][p] = make_float2(hi, (float)(Bk[k][p] - (double)hi));
            mx = std::fmax(mx, std::fabs(Bk[k][p]));
        }
        int f = 0;
        std::frexp(mx * (1.0 + 1e-12), &f);
        T.fexp[k] = f;
        // slices w_j of B[k][p] 2^(8-f), 8 bits each; even k: column 4 L + k/2 of the even
        // part, odd k: column 3 L + (k-1)/2 of the odd part
        const bool odd = k & 1;
        const int jcol = k >> 1, cstride = odd ? 3 : 4;
        for (int p = 0; p < h; ++p) {
            double y = std::ldexp(Bk[k][p], kBits - f);
            double wj[kMaxS];
            for (int j = 0; j < S; ++j) {
                wj[j] = std::nearbyint(y);
                y = (y - wj[j]) * 256.0;
            }
            // column c = 4 L + jcol of the part, K index i HP + p carries w_{L-i}
            for (int L = 0; L < S; ++L)
                for (int i = 0; i <= L; ++i) {
                    const int c = cstride * L + jcol, kk = i * HP + p;
                    unsigned char* base = odd ? T.img + kNE * KA * 2 : T.img;
                    const __half v = __double2half(wj[L - i]);
                    std::memcpy(base + umma_off(c, kk, KA), &v, 2);
                }
        }
    }
}

std::mutex g_m1_mutex;

template <int G, int S>
cudaError_t launch_tc(const float2* x, int64_t n_rows, int64_t n_src, float2* out, int* err, int sms, cudaStream_t s) {
    const size_t smem = tc_smem<G, S>();
    cudaError_t e = cudaFuncSetAttribute(k_mode1_tc<G, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // CTAs per SM: as many as shared memory holds (about 220 KB per SM), at most 4 (4 x 64
    // TMEM columns of 512), so that several CTAs' serial phases overlap
    const int per = (int)std::max<size_t>(1, std::min<size_t>(4, (220u << 10) / (smem + 2048)));
    const int64_t tiles = (n_rows + 127) / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * per));
    k_mode1_tc<G, S><<<grid, kM1Threads, smem, s>>>(x, n_rows, n_src, out, err);
    return cudaGetLastError();
}

template <int G>
cudaError_t launch_simt(const float2* x, int64_t n_rows, int64_t n_src, float2* out, int sms, cudaStream_t s) {
    const size_t smem = sizeof(float2) * 128 * tile_ld(G);
    cudaError_t e = cudaFuncSetAttribute(k_mode1_simt<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per = (int)std::max<size_t>(1, std::min<size_t>(16, (220u << 10) / (smem + 1024)));
    const int64_t tiles = (n_rows + kM1Threads - 1) / kM1Threads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * per));
    k_mode1_simt<G><<<grid, kM1Threads, smem, s>>>(x, n_rows, n_src, out);
    return cudaGetLastError();
}

template <int G>
cudaError_t launch_g(int method, int S, const float2* x, int64_t n_rows, int64_t n_src, float2* out, int* err,
                     int sms, cudaStream_t s) {
    if (method == P2S_MODE1_SIMT) return launch_simt<G>(x, n_rows, n_src, out, sms, s);
    if (S == 4) return launch_tc<G, 4>(x, n_rows, n_src, out, err, sms, s);
    return launch_tc<G, 5>(x, n_rows, n_src, out, err, sms, s);
}

}  // namespace

int mode1_product(const DeviceTables& T, int method, int G, int slices, const float* x, int64_t n_src, int64_t n_rows,
                  float* out, cudaStream_t s) {
    if (method != P2S_MODE1_SIMT && method != P2S_MODE1_TC) return fail(P2S_ERR_ARG, "p2s_mode1_product: method");
    if (G != 8 && G != 12 && G != 16 && G != 24 && G != 32 && G != 48)
        return fail(P2S_ERR_ORDER, "p2s_mode1_product: G must be 8, 12, 16, 24, 32 or 48");
    if (method == P2S_MODE1_TC && slices != 4 && slices != 5) return fail(P2S_ERR_ARG, "p2s_mode1_product: slices 4 or 5");
    if (n_rows < 0 || n_src < 1 || !x || (!out && n_rows)) return fail(P2S_ERR_ARG, "p2s_mode1_product: sizes or NULL");
    if (n_rows == 0) return P2S_OK;
    std::lock_guard<std::mutex> lock(g_m1_mutex);  // the tables below are per call
    static M1Tables tab;
    build_tables(G, method == P2S_MODE1_TC ? slices : 4, tab);
    P2S_CUDA(cudaMemcpyToSymbolAsync(c_m1_B, tab.B, sizeof(tab.B), 0, cudaMemcpyHostToDevice, s));
    P2S_CUDA(cudaMemcpyToSymbolAsync(c_m1_fexp, tab.fexp, sizeof(tab.fexp), 0, cudaMemcpyHostToDevice, s));
    P2S_CUDA(cudaMemcpyToSymbolAsync(g_m1_bimg, tab.img, sizeof(tab.img), 0, cudaMemcpyHostToDevice, s));
    const float2* xx = reinterpret_cast<const float2*>(x);
    float2* oo = reinterpret_cast<float2*>(out);
    cudaError_t e = cudaErrorInvalidValue;
    switch (G) {
    case 8: e = launch_g<8>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    case 12: e = launch_g<12>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    case 16: e = launch_g<16>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    case 24: e = launch_g<24>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    case 32: e = launch_g<32>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    case 48: e = launch_g<48>(method, slices, xx, n_rows, n_src, oo, T.err, T.sm_count, s); break;
    }
    // the host tables must outlive the asynchronous copies above
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_mode1_product: launch", e);
    return P2S_OK;
}

}  // namespace p2s
