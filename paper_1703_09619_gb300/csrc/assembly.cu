// Global assembly on a conforming structured mesh: the step after the fill (the "total" time of
// arXiv:1703.09619, Sec. V), for one scalar field with N modes per axis.
//
// Basis.  The fill computes element matrices in the Legendre basis P_m of Eq. (2)-(4).  A
// conforming (C0) space needs the hierarchic basis
//     l_0 = (P_0 - P_1)/2,  l_1 = (P_0 + P_1)/2,  l_k = (P_k - P_{k-2}) / sqrt(2 (2k-1))  (k >= 2),
// vertex functions of the two ends and the normalised integrated Legendre bubbles.  Each l_k has
// two Legendre coefficients, so with T the N x N transform and Tk = T (x) T (x) T the element
// matrix in the hierarchic basis is Tk M Tk^T: 64 products per entry.
//
// Numbering.  On a structured mesh of aligned elements the global space is the tensor product of
// 1-D C0 spaces.  Axis dof g: vertex i (0..n_el), then bubble k of interval i at
// n_el + 1 + i (N-2) + k - 2; global row (gu Ngv + gv) Ngw + gw.  The CSR columns of row
// (gu, gv, gw) are the tensor product of the 1-D neighbour lists (the axis dofs sharing an
// interval), in increasing order, so the position of a coupling inside its row is
//     (ru cnt_v(gv) + rv) cnt_w(gw) + rw
// from the 1-D ranks r and neighbour counts cnt: small tables, no per-element maps.
//
// Scatter.  Elements are processed in 8 colours (parities of i, j, k): two elements of one colour
// share no dof, so each colour's launch adds into the values without atomics, and the sums are
// the same on every run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "asm_stages.cuh"

namespace p2s {
namespace {

constexpr int kAsmThreads = 256;

// one axis of the mesh: interval count, global axis dofs, neighbour counts [ng], ranks
// [n_el][N][N] (rank of g(i, b) among the sorted neighbours of g(i, a))
struct Axis1D {
    int n_el = 0, N = 0, ng = 0;
    std::vector<int32_t> cnt;
    std::vector<int32_t> rank;
    int g(int i, int m) const { return m == 0 ? i : (m == 1 ? i + 1 : n_el + 1 + i * (N - 2) + (m - 2)); }
};

void build_axis(Axis1D& A, int n_el, int N) {
    A.n_el = n_el;
    A.N = N;
    A.ng = n_el + 1 + n_el * (N - 2);
    std::vector<std::vector<int>> nb((size_t)A.ng);
    for (int i = 0; i < n_el; ++i)
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) nb[A.g(i, a)].push_back(A.g(i, b));
    A.cnt.assign((size_t)A.ng, 0);
    for (int g = 0; g < A.ng; ++g) {
        std::sort(nb[g].begin(), nb[g].end());
        nb[g].erase(std::unique(nb[g].begin(), nb[g].end()), nb[g].end());
        A.cnt[g] = (int32_t)nb[g].size();
    }
    A.rank.assign((size_t)n_el * N * N, 0);
    for (int i = 0; i < n_el; ++i)
        for (int a = 0; a < N; ++a) {
            const std::vector<int>& v = nb[A.g(i, a)];
            for (int b = 0; b < N; ++b)
                A.rank[((size_t)i * N + a) * N + b] =
                    (int32_t)(std::lower_bound(v.begin(), v.end(), A.g(i, b)) - v.begin());
        }
}

struct AsmLaunch {
    const double* emat;  // [E][n n] Legendre-basis element matrices (read only)
    double* work;        // [E][n n] scratch, used when the matrices are not staged in shared memory
    AsmMeshDev mesh;
    AsmCoef coef;
    int N, colour;
};

// y = T x on the N values X[base + k s] (in place): y_0 = (x_0 - x_1)/2, y_1 = (x_0 + x_1)/2,
// y_k = c_k (x_k - x_{k-2}); one thread per line, the N values held in registers.  Line
// `line` starts at base = hi s N + lo with (hi, lo) = divmod(line, s), stepped without
// divisions.  Lines are disjoint, so src == X is allowed.
__device__ __forceinline__ void hier_lines(const double* src, double* X, int s, int nn, const AsmLaunch& L) {
    const int N = L.N, lines = nn / N;
    const int step_hi = div_small((int)blockDim.x, s, 1.0f / (float)s), step_lo = (int)blockDim.x - step_hi * s;
    int hi = div_small((int)threadIdx.x, s, 1.0f / (float)s), lo = (int)threadIdx.x - hi * s;
    for (int line = threadIdx.x; line < lines; line += blockDim.x) {
        const int base = hi * s * N + lo;
        double* p = X + base;
        double x[kMaxOrder];
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k)
            if (k < N) x[k] = src[base + k * s];
        p[0] = 0.5 * (x[0] - x[1]);
        p[s] = 0.5 * (x[0] + x[1]);
#pragma unroll
        for (int k = 2; k < kMaxOrder; ++k)
            if (k < N) p[k * s] = L.coef.ck[k] * (x[k] - x[k - 2]);
        hi += step_hi;
        lo += step_lo;
        if (lo >= s) { lo -= s; ++hi; }
    }
}

__host__ __device__ inline size_t asm_table_bytes(int N) {
    const int n = N * N * N;
    return sizeof(int64_t) * n + sizeof(int2) * n + sizeof(int) * n + sizeof(int) * 3 * N * N;
}

// Element matrices staged in shared memory, order N (2..5) known at compile time.  Layout of the
// staged matrix: entry (r, c), c = m2 N^2 + j, at (r N + m2) P + j with P = N^2 rounded up to
// odd, so rows of N^2 trial entries start on distinct banks.  Four passes, each holding its
// values in registers:
//   A  test u: read from HBM (coalesced along c and the other test axes), T, store;
//   B  test v and w of one (m, c): N^2 values, stride P N between p;
//   C  trial u of one (r, j): N values, stride P;
//   D  trial v and w of one (r, m2): the N^2 contiguous values of a padded row;
// then every entry is added to its CSR position (tables as in k_assemble).  kFF: the input holds
// float-float pairs and the passes run in float-float on the FP32 pipe (FP64 arithmetic runs at
// a small fraction of the FP32 rate), the entries going to FP64 by integer operations at the end.
// The additions into the values are L2 reductions (red.global.add.f64): within one colour every
// position receives at most one, so the sums are the same on every run.
// Element matrices staged in shared memory, order N (2..5) known at compile time (layout and
// passes in asm_stages.cuh): pass A (test u) reads the matrix from HBM, passes B, C, D finish the
// change of basis, and every entry is added to its CSR position.  kFF: the input holds
// float-float pairs and the passes run in float-float on the FP32 pipe (FP64 arithmetic runs at
// a small fraction of the FP32 rate), the entries going to FP64 by integer operations at the end.
// The additions into the values are L2 reductions (red.global.add.f64): within one colour every
// position receives at most one, so the sums are the same on every run.
template <int N, bool kFF>
__global__ void __launch_bounds__(kAsmThreads, N <= 4 ? 4 : 1) k_assemble_staged(AsmLaunch L) {
    constexpr int NN = N * N, n = NN * N, nn = n * n, P = NN | 1, G = n * N;
    using M = typename AsmVal<kFF>::M;
    extern __shared__ __align__(16) unsigned char s_raw[];
    M* s_x = reinterpret_cast<M*>(s_raw);  // [G][P]
    int64_t* s_base = reinterpret_cast<int64_t*>(s_x + G * P);
    int2* s_cvw = reinterpret_cast<int2*>(s_base + n);
    int* s_rank = reinterpret_cast<int*>(s_cvw + n);
    const int tid = threadIdx.x;
    const AsmMeshDev& ms = L.mesh;
    const int cx = L.colour & 1, cy = (L.colour >> 1) & 1, cz = (L.colour >> 2) & 1;
    const int hx = (ms.nx - cx + 1) / 2, hy = (ms.ny - cy + 1) / 2, hz = (ms.nz - cz + 1) / 2;
    const int64_t count = (int64_t)hx * hy * hz;
    for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int qi = (int)(q % hx), qj = (int)((q / hx) % hy), qk = (int)(q / ((int64_t)hx * hy));
        const int i = 2 * qi + cx, j = 2 * qj + cy, k = 2 * qk + cz;
        const double* __restrict__ src = L.emat + (((int64_t)k * ms.ny + j) * ms.nx + i) * (int64_t)nn;
        asm_element_tables<N>(ms, i, j, k, s_base, s_cvw, s_rank, tid, kAsmThreads);
        asm_pass_a_global<N, kFF>(src, s_x, L.coef, tid, kAsmThreads);
        __syncthreads();
        asm_passes_bcd<N, kFF>(s_x, L.coef, tid, kAsmThreads);
        asm_scatter<N, kFF>(s_x, s_base, s_cvw, s_rank, ms.values, tid, kAsmThreads);
        __syncthreads();  // the staged matrix and the tables are reused by the next element
    }
}
constexpr int kMaxStagedOrder = 5;
using AsmKernel = void (*)(AsmLaunch);
template <bool kFF>
AsmKernel staged_kernel(int N) {
    switch (N) {
        case 2: return k_assemble_staged<2, kFF>;
        case 3: return k_assemble_staged<3, kFF>;
        case 4: return k_assemble_staged<4, kFF>;
        default: return k_assemble_staged<5, kFF>;
    }
}


// Any order (used for N >= 6, whose n^2 doubles do not fit in shared memory): one CTA per element
// of the colour (grid-stride).  Tk M Tk^T by sum factorisation in the assembly's scratch: T along
// the three test axes and the three trial axes of the n x n matrix, 2 products per entry and
// pass; then every entry is added to its CSR position.
__global__ void __launch_bounds__(kAsmThreads, 4) k_assemble(AsmLaunch L) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    const int N = L.N, NN = N * N, n = NN * N, nn = n * n;
    int64_t* s_base = reinterpret_cast<int64_t*>(s_raw);
    int2* s_cvw = reinterpret_cast<int2*>(s_base + n);
    int* s_dec = reinterpret_cast<int*>(s_cvw + n);
    int* s_rank = s_dec + n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const int m = r / NN, nv = (r / N) % N, p = r % N;
        s_dec[r] = m | (nv << 8) | (p << 16);
    }
    // (r, c) of entry t = r n + c, stepped by blockDim
    const int step_r = (int)blockDim.x / n, step_c = (int)blockDim.x - step_r * n;
    const int r0 = (int)threadIdx.x / n, c0 = (int)threadIdx.x - r0 * n;
    const int cx = L.colour & 1, cy = (L.colour >> 1) & 1, cz = (L.colour >> 2) & 1;
    const int hx = (L.mesh.nx - cx + 1) / 2, hy = (L.mesh.ny - cy + 1) / 2, hz = (L.mesh.nz - cz + 1) / 2;
    const int64_t count = (int64_t)hx * hy * hz;
    __syncthreads();
    for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int qi = (int)(q % hx), qj = (int)((q / hx) % hy), qk = (int)(q / ((int64_t)hx * hy));
        const int i = 2 * qi + cx, j = 2 * qj + cy, k = 2 * qk + cz;
        const int64_t e = ((int64_t)k * L.mesh.ny + j) * L.mesh.nx + i;
        const double* src = L.emat + e * (int64_t)nn;
        double* X = L.work + e * (int64_t)nn;
        // the element's tables (the previous element's scatter ended at a barrier)
        for (int t = threadIdx.x; t < 3 * NN; t += blockDim.x) {
            const int a = t / NN, xy = t - a * NN;
            const int el = a == 0 ? i : (a == 1 ? j : k);
            s_rank[t] = L.mesh.ax[a].rank[el * NN + xy];
        }
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const int d = s_dec[r];
            const int gu = axis_g(L.mesh.ax[0], i, d & 0xff), gv = axis_g(L.mesh.ax[1], j, (d >> 8) & 0xff),
                      gw = axis_g(L.mesh.ax[2], k, d >> 16);
            s_base[r] = L.mesh.row_ptr[((int64_t)gu * L.mesh.ax[1].ng + gv) * L.mesh.ax[2].ng + gw];
            s_cvw[r] = make_int2(L.mesh.ax[1].cnt[gv], L.mesh.ax[2].cnt[gw]);
        }
        // test u, v, w (strides n N^2, n N, n), then trial u, v, w (N^2, N, 1); the first pass
        // reads the input
#pragma unroll 1
        for (int pass = 0, st = n * NN; pass < 6; ++pass, st = pass == 3 ? NN : st / N) {
            hier_lines(pass == 0 ? src : X, X, st, nn, L);
            __syncthreads();
        }
        // scatter: one L2 reduction per entry (at most one per position within a colour)
        int r = r0, c = c0;
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int dr = s_dec[r], dc = s_dec[c];
            const int ru = s_rank[(dr & 0xff) * N + (dc & 0xff)];
            const int rv = s_rank[NN + ((dr >> 8) & 0xff) * N + ((dc >> 8) & 0xff)];
            const int rw = s_rank[2 * NN + (dr >> 16) * N + (dc >> 16)];
            const int2 cvw = s_cvw[r];
            atomicAdd(L.mesh.values + s_base[r] + ((ru * cvw.x + rv) * cvw.y + rw), X[t]);
            r += step_r;
            c += step_c;
            if (c >= n) { c -= n; ++r; }
        }
        __syncthreads();  // X and the tables are reused by the next element
    }
}

}  // namespace
}  // namespace p2s

using namespace p2s;

struct p2s_assembly {
    p2s_ctx* ctx = nullptr;
    int nx = 0, ny = 0, nz = 0, N = 0;
    p2s_plan* plan = nullptr;  // the operator fill of the mesh's elements
    Axis1D ax[3];
    std::vector<int64_t> row_ptr;
    int64_t rows = 0, nnz = 0;
    double* d_emat = nullptr;
    int64_t* d_row_ptr = nullptr;
    int32_t* d_axis = nullptr;  // cnt and rank tables of the three axes, back to back
    AxisDev dev[3];
    bool staged = false;  // element matrices staged in shared memory (k_assemble_staged<N>)
    bool ff = false;      // the fill writes float-float pairs, transformed in float-float
    void (*kernel)(AsmLaunch) = nullptr;       // p2s_assembly_add: FP64 element matrices
    void (*kernel_fill)(AsmLaunch) = nullptr;  // p2s_assembly_fill: the plan's own output
    size_t smem = 0;      // dynamic shared memory of k_assemble
    int grid = 1;     // CTAs of a colour launch: the resident capacity of the device
    // fused operator fill + assembly (mixed, N <= 4, the plan on the specialised operator path):
    // the elements as whole-element units, colour by colour
    bool fused = false;
    ContractUnit* d_units = nullptr;
    int64_t colour_off[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int fused_threads = 0, fused_grid = 0;
    size_t fused_smem = 0;
};

namespace {

int build_structure(int nx, int ny, int nz, int N, Axis1D* ax, std::vector<int64_t>& row_ptr, int64_t& rows,
                    int64_t& nnz) {
    if (nx < 1 || ny < 1 || nz < 1 || N < 2 || N > kMaxOrder) return fail(P2S_ERR_ARG, "assembly: mesh size >= 1 and 2 <= N <= 12");
    if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return fail(P2S_ERR_ARG, "assembly: too many elements");
    build_axis(ax[0], nx, N);
    build_axis(ax[1], ny, N);
    build_axis(ax[2], nz, N);
    rows = (int64_t)ax[0].ng * ax[1].ng * ax[2].ng;
    row_ptr.assign((size_t)rows + 1, 0);
    int64_t r = 0;
    for (int gu = 0; gu < ax[0].ng; ++gu)
        for (int gv = 0; gv < ax[1].ng; ++gv)
            for (int gw = 0; gw < ax[2].ng; ++gw, ++r)
                row_ptr[r + 1] = row_ptr[r] + (int64_t)ax[0].cnt[gu] * ax[1].cnt[gv] * ax[2].cnt[gw];
    nnz = row_ptr[rows];
    if (rows >= ((int64_t)1 << 31)) return fail(P2S_ERR_ARG, "assembly: more than 2^31 - 1 rows (int32 columns)");
    return P2S_OK;
}

}  // namespace

extern "C" {

int p2s_assembly_structure_host(int nx, int ny, int nz, int order, int64_t* rows, int64_t* nnz, int64_t* row_ptr,
                                int32_t* col_idx) {
    Axis1D ax[3];
    std::vector<int64_t> rp;
    int64_t R = 0, Z = 0;
    int rc = build_structure(nx, ny, nz, order, ax, rp, R, Z);
    if (rc) return rc;
    if (rows) *rows = R;
    if (nnz) *nnz = Z;
    if (row_ptr) std::memcpy(row_ptr, rp.data(), sizeof(int64_t) * (size_t)(R + 1));
    if (col_idx) {
        // the columns of every row: the tensor product of the sorted 1-D neighbour lists
        std::vector<std::vector<int>> nb[3];
        for (int a = 0; a < 3; ++a) {
            nb[a].assign((size_t)ax[a].ng, {});
            for (int i = 0; i < ax[a].n_el; ++i)
                for (int x = 0; x < order; ++x)
                    for (int y = 0; y < order; ++y) nb[a][ax[a].g(i, x)].push_back(ax[a].g(i, y));
            for (auto& v : nb[a]) {
                std::sort(v.begin(), v.end());
                v.erase(std::unique(v.begin(), v.end()), v.end());
            }
        }
        int64_t pos = 0;
        for (int gu = 0; gu < ax[0].ng; ++gu)
            for (int gv = 0; gv < ax[1].ng; ++gv)
                for (int gw = 0; gw < ax[2].ng; ++gw)
                    for (int a : nb[0][gu])
                        for (int b : nb[1][gv])
                            for (int c : nb[2][gw]) col_idx[pos++] = (int32_t)(((int64_t)a * ax[1].ng + b) * ax[2].ng + c);
    }
    return P2S_OK;
}

void p2s_assembly_destroy(p2s_assembly* A) {
    if (!A) return;
    if (A->ctx) cudaSetDevice(context_tables(A->ctx)->device);
    p2s_plan_destroy(A->plan);
    cudaFree(A->d_emat);
    cudaFree(A->d_units);
    cudaFree(A->d_row_ptr);
    cudaFree(A->d_axis);
    delete A;
}

int p2s_assembly_create(p2s_ctx* ctx, int nx, int ny, int nz, int order, int npts, int precision, int kind,
                        const p2s_term* terms, int n_terms, p2s_assembly** out) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || !out) return fail(P2S_ERR_ARG, "p2s_assembly_create: NULL context or out");
    *out = nullptr;
    for (int k = 0; k < n_terms && terms; ++k)
        if (terms[k].gi != 0 || terms[k].gj != 0) return fail(P2S_ERR_ARG, "p2s_assembly_create: one scalar field (gi = gj = 0)");
    p2s_assembly* A = new (std::nothrow) p2s_assembly();
    if (!A) return fail(P2S_ERR_OOM, "p2s_assembly_create: host allocation");
    A->ctx = ctx;
    A->nx = nx;
    A->ny = ny;
    A->nz = nz;
    A->N = order;
    int rc = build_structure(nx, ny, nz, order, A->ax, A->row_ptr, A->rows, A->nnz);
    if (rc) { p2s_assembly_destroy(A); return rc; }
    const int64_t E = (int64_t)nx * ny * nz;
    std::vector<int32_t> ord((size_t)E * 3, order);
    p2s_orders o = {1, ord.data()};
    p2s_quadrature q = {npts, nullptr};
    rc = p2s_operator_plan_create(ctx, E, &o, &q, precision, kind, terms, n_terms, nullptr, &A->plan);
    if (rc) { p2s_assembly_destroy(A); return rc; }
    if (cudaSetDevice(T->device) != cudaSuccess) { p2s_assembly_destroy(A); return fail(P2S_ERR_CUDA, "p2s_assembly_create: device"); }
    size_t ntab = 0;
    for (int a = 0; a < 3; ++a) ntab += A->ax[a].cnt.size() + A->ax[a].rank.size();
    const int64_t n = (int64_t)order * order * order;
    // the fused path keeps no element matrices: it needs a mixed plan on the specialised operator
    // kernel with whole-element units (N^4 <= 256) and the launch must fit
    if (precision == P2S_MIXED && order <= 4 && plan_spec_op(A->plan) == order) {
        const size_t fsmem = opn_assemble_smem_bytes(order);
        const int fthreads = (order * order * order * order + 31) / 32 * 32;
        const int per_sm = fsmem <= T->smem_optin ? opn_assemble_blocks_per_sm(order, fthreads, fsmem) : 0;
        if (per_sm >= 1) {
            std::vector<ContractUnit> units;
            units.reserve((size_t)E);
            for (int c = 0; c < 8; ++c) {
                A->colour_off[c] = (int64_t)units.size();
                for (int k = (c >> 2) & 1; k < nz; k += 2)
                    for (int j = (c >> 1) & 1; j < ny; j += 2)
                        for (int i = c & 1; i < nx; i += 2) {
                            ContractUnit u{};
                            u.e = (int32_t)(((int64_t)k * ny + j) * nx + i);
                            u.tp = -1;
                            u.m1n = (int8_t)order;
                            u.n1n = (int8_t)order;
                            units.push_back(u);
                        }
            }
            A->colour_off[8] = (int64_t)units.size();
            if (cudaMalloc(&A->d_units, sizeof(ContractUnit) * std::max<size_t>(1, units.size())) != cudaSuccess) {
                p2s_assembly_destroy(A);
                return fail(P2S_ERR_OOM, "p2s_assembly_create: device allocation");
            }
            if (cudaMemcpy(A->d_units, units.data(), sizeof(ContractUnit) * units.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
                p2s_assembly_destroy(A);
                return fail(P2S_ERR_CUDA, "p2s_assembly_create: upload");
            }
            A->fused = true;
            A->fused_smem = fsmem;
            A->fused_threads = fthreads;
            A->fused_grid = per_sm * T->sm_count;
        }
    }
    bool ok = (A->fused || cudaMalloc(&A->d_emat, sizeof(double) * std::max<int64_t>(1, E * n * n)) == cudaSuccess) &&
              cudaMalloc(&A->d_row_ptr, sizeof(int64_t) * (A->rows + 1)) == cudaSuccess &&
              cudaMalloc(&A->d_axis, sizeof(int32_t) * ntab) == cudaSuccess;
    if (!ok) { p2s_assembly_destroy(A); return fail(P2S_ERR_OOM, "p2s_assembly_create: device allocation"); }
    cudaError_t ce = cudaMemcpy(A->d_row_ptr, A->row_ptr.data(), sizeof(int64_t) * (A->rows + 1), cudaMemcpyHostToDevice);
    size_t off = 0;
    for (int a = 0; a < 3 && ce == cudaSuccess; ++a) {
        const Axis1D& X = A->ax[a];
        AxisDev& D = A->dev[a];
        D.n_el = X.n_el;
        D.N = X.N;
        D.ng = X.ng;
        D.cnt = A->d_axis + off;
        ce = cudaMemcpy(A->d_axis + off, X.cnt.data(), sizeof(int32_t) * X.cnt.size(), cudaMemcpyHostToDevice);
        off += X.cnt.size();
        D.rank = A->d_axis + off;
        if (ce == cudaSuccess) ce = cudaMemcpy(A->d_axis + off, X.rank.data(), sizeof(int32_t) * X.rank.size(), cudaMemcpyHostToDevice);
        off += X.rank.size();
    }
    if (ce != cudaSuccess) { p2s_assembly_destroy(A); return fail(P2S_ERR_CUDA, "p2s_assembly_create: upload", ce); }
    int per_sm = 0;
    A->staged = order <= kMaxStagedOrder && staged_smem_bytes(order) <= T->smem_optin;
    // a mixed fill hands its float-float pairs to the staged kernel without converting them
    A->ff = A->staged && precision == P2S_MIXED;
    if (A->ff && (rc = plan_set_output_ff(A->plan, true)) != P2S_OK) { p2s_assembly_destroy(A); return rc; }
    A->kernel = A->staged ? staged_kernel<false>(order) : k_assemble;
    A->kernel_fill = A->ff ? staged_kernel<true>(order) : A->kernel;
    A->smem = A->staged ? staged_smem_bytes(order) : asm_table_bytes(order);
    ce = cudaFuncSetAttribute(A->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A->smem);
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(A->kernel_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A->smem);
    if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, A->kernel, kAsmThreads, A->smem);
    if (ce != cudaSuccess) { p2s_assembly_destroy(A); return fail(P2S_ERR_CUDA, "p2s_assembly_create: kernel attributes", ce); }
    A->grid = std::max(1, per_sm) * T->sm_count;
    *out = A;
    return P2S_OK;
}

int64_t p2s_assembly_rows(const p2s_assembly* A) { return A ? A->rows : P2S_ERR_ARG; }
int64_t p2s_assembly_nnz(const p2s_assembly* A) { return A ? A->nnz : P2S_ERR_ARG; }
int p2s_assembly_fused(const p2s_assembly* A) { return A ? (A->fused ? 1 : 0) : P2S_ERR_ARG; }

int p2s_assembly_use_graph(p2s_assembly* A, int enable) {
    if (!A) return fail(P2S_ERR_ARG, "p2s_assembly_use_graph: NULL assembly");
    return p2s_plan_use_graph(A->plan, enable);
}

}  // extern "C"

namespace {

// The device views of the mesh (into `values`) and of the bubble normalisation.
void mesh_views(const p2s_assembly* A, double* values, AsmMeshDev& ms, AsmCoef& coef) {
    ms.values = values;
    ms.row_ptr = A->d_row_ptr;
    for (int a = 0; a < 3; ++a) ms.ax[a] = A->dev[a];
    ms.nx = A->nx;
    ms.ny = A->ny;
    ms.nz = A->nz;
    for (int k = 0; k < kMaxOrder; ++k) {
        coef.ck[k] = k >= 2 ? 1.0 / std::sqrt(2.0 * (2 * k - 1)) : 0.0;
        coef.ckf[2 * k] = (float)coef.ck[k];
        coef.ckf[2 * k + 1] = (float)(coef.ck[k] - (double)coef.ckf[2 * k]);
    }
}

// The fused path: 8 colour launches of the operator contraction + assembly over the moments in the
// plan's scratch.
int assemble_fused(p2s_assembly* A, double* values, cudaStream_t s) {
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    ContractLaunch C;
    int rc = plan_op_launch(A->plan, C);
    if (rc) return rc;
    AsmMeshDev ms;
    AsmCoef coef;
    mesh_views(A, values, ms, coef);
    for (int c = 0; c < 8; ++c) {
        const int64_t cnt = A->colour_off[c + 1] - A->colour_off[c];
        if (cnt == 0) continue;
        P2S_CUDA(cudaMemsetAsync(C.counter, 0, sizeof(unsigned long long), s));
        C.units = A->d_units + A->colour_off[c];
        C.n_units = cnt;
        const int grid = (int)std::min<int64_t>(cnt, A->fused_grid);
        P2S_CUDA(launch_opn_assemble(A->N, C, ms, coef, grid, A->fused_threads, A->fused_smem, s));
    }
    return P2S_OK;
}

// The 8 colour launches of `kernel` over the element matrices `emat`.
int assemble_colours(p2s_assembly* A, AsmKernel kernel, const double* emat, double* values, cudaStream_t s) {
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    AsmLaunch L;
    L.emat = emat;
    L.work = A->d_emat;
    mesh_views(A, values, L.mesh, L.coef);
    L.N = A->N;
    for (int c = 0; c < 8; ++c) {  // colours one after the other: no two elements in flight share a dof
        L.colour = c;
        const int64_t cnt = (int64_t)((A->nx - (c & 1) + 1) / 2) * ((A->ny - ((c >> 1) & 1) + 1) / 2) *
                            ((A->nz - ((c >> 2) & 1) + 1) / 2);
        if (cnt == 0) continue;
        const int grid = (int)std::min<int64_t>(cnt, A->grid);
        kernel<<<grid, kAsmThreads, A->smem, s>>>(L);
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

}  // namespace

extern "C" {

int p2s_assembly_add(p2s_assembly* A, const double* emat, double* values, void* stream) {
    if (!A || !emat || !values) return fail(P2S_ERR_ARG, "p2s_assembly_add: NULL assembly, matrices or values");
    return assemble_colours(A, A->kernel, emat, values, (cudaStream_t)stream);
}

int p2s_assembly_reassemble(p2s_assembly* A, double* values, void* stream) {
    if (!A || !values) return fail(P2S_ERR_ARG, "p2s_assembly_reassemble: NULL assembly or values");
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    P2S_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * A->nnz, (cudaStream_t)stream));
    if (A->fused) return assemble_fused(A, values, (cudaStream_t)stream);  // from the kept moments
    return assemble_colours(A, A->kernel_fill, A->d_emat, values, (cudaStream_t)stream);
}

int p2s_assembly_fill(p2s_assembly* A, const p2s_geometry* geom, const p2s_material* mat, double* values, void* stream) {
    if (!A || !values) return fail(P2S_ERR_ARG, "p2s_assembly_fill: NULL assembly or values");
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    int rc = A->fused ? plan_run_moments(A->plan, geom, mat, (cudaStream_t)stream)
                      : p2s_plan_fill(A->plan, geom, mat, A->d_emat, nullptr, stream);
    if (rc) return rc;
    return p2s_assembly_reassemble(A, values, stream);
}

}  // extern "C"
