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

#include "p2s_internal.h"

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

// Device view of one axis.
struct AxisDev {
    int n_el, N, ng;
    const int32_t* cnt;
    const int32_t* rank;
};

__device__ __forceinline__ int axis_g(const AxisDev& A, int i, int m) {
    return m == 0 ? i : (m == 1 ? i + 1 : A.n_el + 1 + i * (A.N - 2) + (m - 2));
}

struct AsmLaunch {
    const double* emat;      // [E][n n] Legendre-basis element matrices (read only)
    double* work;            // [E][n n] scratch, used when the matrices are not staged in shared memory
    double* values;          // CSR values
    const int64_t* row_ptr;  // [rows + 1]
    AxisDev ax[3];
    double ck[kMaxOrder];    // 1 / sqrt(2 (2k - 1)): the bubble normalisation
    int nx, ny, nz, N, colour;
};

// y = T x on the N values X[base + k s] (in place): y_0 = (x_0 - x_1)/2, y_1 = (x_0 + x_1)/2,
// y_k = c_k (x_k - x_{k-2}); one thread per line, the N values held in registers.
// Lines are disjoint, so src == X is allowed.
__device__ __forceinline__ void hier_lines(const double* src, double* X, int s, int nn, const AsmLaunch& L) {
    const int N = L.N, lines = nn / N;
    for (int line = threadIdx.x; line < lines; line += blockDim.x) {
        const int lo = line % s, hi = line / s;
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
            if (k < N) p[k * s] = L.ck[k] * (x[k] - x[k - 2]);
    }
}

// One CTA per element of the colour (grid-stride).  Tk M Tk^T by sum factorisation: T along the
// three test axes and the three trial axes of the n x n matrix, 2 products per entry and pass;
// then every entry is added to its CSR position.  kSmem: the matrix is staged in shared memory
// (n^2 doubles); otherwise it is transformed in place in the fill's scratch.
template <bool kSmem>
__global__ void __launch_bounds__(kAsmThreads, 4) k_assemble(AsmLaunch L) {
    extern __shared__ double s_mat[];
    const int N = L.N, n = N * N * N, nn = n * n;
    const int cx = L.colour & 1, cy = (L.colour >> 1) & 1, cz = (L.colour >> 2) & 1;
    const int hx = (L.nx - cx + 1) / 2, hy = (L.ny - cy + 1) / 2, hz = (L.nz - cz + 1) / 2;
    const int64_t count = (int64_t)hx * hy * hz;
    for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
        const int qi = (int)(q % hx), qj = (int)((q / hx) % hy), qk = (int)(q / ((int64_t)hx * hy));
        const int i = 2 * qi + cx, j = 2 * qj + cy, k = 2 * qk + cz;
        const int64_t e = ((int64_t)k * L.ny + j) * L.nx + i;
        const double* src = L.emat + e * (int64_t)nn;
        double* X = kSmem ? s_mat : L.work + e * (int64_t)nn;
        // test u, v, w (strides n N^2, n N, n), then trial u, v, w (N^2, N, 1); the first pass
        // reads the input
#pragma unroll 1
        for (int pass = 0, st = n * N * N; pass < 6; ++pass, st = pass == 3 ? N * N : st / N) {
            hier_lines(pass == 0 ? src : X, X, st, nn, L);
            __syncthreads();
        }
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            const int r = t / n, c = t - r * n;
            const int m = r / (N * N), nv = (r / N) % N, p = r % N;
            const int m2 = c / (N * N), n2 = (c / N) % N, p2 = c % N;
            const int gu = axis_g(L.ax[0], i, m), gv = axis_g(L.ax[1], j, nv), gw = axis_g(L.ax[2], k, p);
            const int64_t row = ((int64_t)gu * L.ax[1].ng + gv) * L.ax[2].ng + gw;
            const int ru = L.ax[0].rank[(i * N + m) * N + m2];
            const int rv = L.ax[1].rank[(j * N + nv) * N + n2];
            const int rw = L.ax[2].rank[(k * N + p) * N + p2];
            const int64_t pos = L.row_ptr[row] + ((int64_t)ru * L.ax[1].cnt[gv] + rv) * L.ax[2].cnt[gw] + rw;
            L.values[pos] += X[t];
        }
        __syncthreads();  // X is reused by the next element
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
    size_t smem = 0;  // > 0: element matrices staged in shared memory (n^2 doubles)
    int grid = 1;     // CTAs of a colour launch: the resident capacity of the device
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
    bool ok = cudaMalloc(&A->d_emat, sizeof(double) * std::max<int64_t>(1, E * n * n)) == cudaSuccess &&
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
    const size_t mat_bytes = sizeof(double) * (size_t)(n * n);
    int per_sm = 0;
    if (mat_bytes <= T->smem_optin) {
        A->smem = mat_bytes;
        ce = cudaFuncSetAttribute(k_assemble<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mat_bytes);
        if (ce == cudaSuccess) ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assemble<true>, kAsmThreads, mat_bytes);
    } else {
        ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_assemble<false>, kAsmThreads, 0);
    }
    if (ce != cudaSuccess) { p2s_assembly_destroy(A); return fail(P2S_ERR_CUDA, "p2s_assembly_create: kernel attributes", ce); }
    A->grid = std::max(1, per_sm) * T->sm_count;
    *out = A;
    return P2S_OK;
}

int64_t p2s_assembly_rows(const p2s_assembly* A) { return A ? A->rows : P2S_ERR_ARG; }
int64_t p2s_assembly_nnz(const p2s_assembly* A) { return A ? A->nnz : P2S_ERR_ARG; }
p2s_plan* p2s_assembly_plan(p2s_assembly* A) { return A ? A->plan : nullptr; }

int p2s_assembly_add(p2s_assembly* A, const double* emat, double* values, void* stream) {
    if (!A || !emat || !values) return fail(P2S_ERR_ARG, "p2s_assembly_add: NULL assembly, matrices or values");
    cudaStream_t s = (cudaStream_t)stream;
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    AsmLaunch L;
    L.emat = emat;
    L.work = A->d_emat;
    L.values = values;
    L.row_ptr = A->d_row_ptr;
    for (int a = 0; a < 3; ++a) L.ax[a] = A->dev[a];
    L.nx = A->nx;
    L.ny = A->ny;
    L.nz = A->nz;
    L.N = A->N;
    for (int k = 0; k < kMaxOrder; ++k) L.ck[k] = k >= 2 ? 1.0 / std::sqrt(2.0 * (2 * k - 1)) : 0.0;
    for (int c = 0; c < 8; ++c) {  // colours one after the other: no two elements in flight share a dof
        L.colour = c;
        const int64_t cnt = (int64_t)((A->nx - (c & 1) + 1) / 2) * ((A->ny - ((c >> 1) & 1) + 1) / 2) *
                            ((A->nz - ((c >> 2) & 1) + 1) / 2);
        if (cnt == 0) continue;
        const int grid = (int)std::min<int64_t>(cnt, A->grid);
        if (A->smem) k_assemble<true><<<grid, kAsmThreads, A->smem, s>>>(L);
        else k_assemble<false><<<grid, kAsmThreads, 0, s>>>(L);
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

int p2s_assembly_fill(p2s_assembly* A, const p2s_geometry* geom, const p2s_material* mat, double* values, void* stream) {
    if (!A || !values) return fail(P2S_ERR_ARG, "p2s_assembly_fill: NULL assembly or values");
    P2S_CUDA(cudaSetDevice(context_tables(A->ctx)->device));
    int rc = p2s_plan_fill(A->plan, geom, mat, A->d_emat, nullptr, stream);
    if (rc) return rc;
    P2S_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * A->nnz, (cudaStream_t)stream));
    return p2s_assembly_add(A, A->d_emat, values, stream);
}

}  // extern "C"
