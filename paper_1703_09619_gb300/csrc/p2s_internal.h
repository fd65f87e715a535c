// Internal declarations shared by the CUDA translation units of libp2s.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "p2s.h"

namespace p2s {

// NVTX range over a scope of host code (the enqueue of one stage of the path); a profiler
// that records NVTX shows the stages by name, and without one the calls cost nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxOrder = P2S_MAX_ORDER;       // N per axis
constexpr int kMaxK = 2 * kMaxOrder - 1;       // moments per axis
constexpr int kMaxG = P2S_MAX_NPTS;            // Gauss-Legendre points per axis
constexpr int kNumTypes = 4;                   // vv, dv, vd, dd

// Unique component pairs (gi <= gj) of a three-component field, in storage order.
__host__ __device__ inline int pair_index(int gi, int gj, int n_comp) {
    if (n_comp == 1) return 0;
    int a = gi < gj ? gi : gj, b = gi < gj ? gj : gi;
    // (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5
    return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// One element of a plan (device copy built by the host).
struct ElemDesc {
    int64_t out_off;      // first output entry of the element
    int64_t mom_off;      // first moment entry of the element
    int32_t n;            // dofs of the element
    int32_t pair_off[6];  // moment offset of pair s relative to mom_off
    int32_t dof_off[3];   // first dof of component g
    int16_t G;            // quadrature points per axis
    int8_t n_comp;
    int8_t n_types;       // selected product types
    int8_t ord[3][3];     // [component][axis] = N
    int8_t kax[3];        // element-wide moment count per axis (max over pairs)
};

// One CTA work item of the contraction: element, block (gi, gj), type t, the partner type
// tp whose block (gj, gi) receives the transpose (-1: none), and the m1/n1 slab.
struct ContractUnit {
    int32_t e;
    int8_t gi, gj, t, tp;
    int8_t m1a, m1n, n1a, n1n;
    int32_t pad;
};

// Packed linearisation index: kmin | cnt << 8 | off << 16 into the coefficient array.
__host__ __device__ inline int lin_kmin(int32_t v) { return v & 0xff; }
__host__ __device__ inline int lin_cnt(int32_t v) { return (v >> 8) & 0xff; }
__host__ __device__ inline int lin_off(int32_t v) { return (v >> 16) & 0xffff; }
__host__ __device__ inline int lin_slot(int t, int m1, int m2) {
    return (t * kMaxOrder + m1) * kMaxOrder + m2;
}

// Host-side tables (tables.cpp).
struct HostTables {
    double gl_x[kMaxG + 1][kMaxG];  // gl_x[G][a], ascending nodes
    double gl_w[kMaxG + 1][kMaxG];
    int32_t lin_idx[kNumTypes * kMaxOrder * kMaxOrder];
    double lin_coef[kNumTypes * kMaxOrder * kMaxOrder * kMaxOrder];
    int n_coef;
    float lin_coef_ff[2 * kNumTypes * kMaxOrder * kMaxOrder * kMaxOrder];  // (hi, lo) pairs
};
const HostTables& host_tables();

// Launch parameters shared by the kernels' host wrappers.
struct MomentLaunch {
    const ElemDesc* desc;
    int64_t n_elem;
    int kind;
    const double* params;
    const double* nodes;
    const double* bulge;
    const double* gl_x;  // device [kMaxG+1][kMaxG]
    const double* gl_w;
    double* mom;
    int32_t* elem_status;
    int* err_flag;
    int n_pairs;        // 1 or 6
    int kb;             // max moments per axis over the plan
    int gmax;           // max G over the plan
    int iacc_cap;       // doubles of the moment accumulator in shared memory
    int out_ff;         // 1: store moments as (hi, lo) FP32 pairs (mixed path)
    const int8_t* elem_mask;  // optional: elements with mask 0 are skipped (FP64 kernel)
    unsigned long long* counter;  // element queue (zeroed before the launch), or nullptr: static
    const int32_t* order;         // queue position -> element (optional; identity without it)
};
size_t moments_smem_bytes(int n_pairs, int kb, int gmax, int iacc_cap);
cudaError_t launch_moments_fp64(const MomentLaunch& L, int grid, size_t smem, cudaStream_t s);
// FP64 moments of a device-side list of elements (*count of them), each cut into parts of its
// w-planes so that a few elements still occupy `grid` CTAs; the parts' accumulators go to `part`
// (moments_split_part_doubles(grid, ...) doubles) and a second kernel sums them in part order.
// The launch needs elem_status == nullptr and FP64 moments (out_ff == 0).
struct MomentSplit {
    const int32_t* list;
    const int* count;
    double* part;
    int grid;
};
size_t moments_split_part_doubles(int grid, int n_pairs, int kb);
int moments_split_blocks_per_sm(size_t smem);
cudaError_t launch_moments_fp64_split(const MomentLaunch& L, const MomentSplit& Sp, size_t smem, cudaStream_t s);
// moments_dw.cu: the same step in double-word arithmetic (mixed path; writes (hi, lo) pairs)
size_t moments_dw_smem_bytes(int n_pairs, int kb, int gmax, int iacc_cap);
int moments_dw_iacc_words(int n_pairs, int max_pair);
cudaError_t launch_moments_dw(const MomentLaunch& L, int grid, size_t smem, cudaStream_t s);
int moments_dw_blocks_per_sm(size_t smem);

struct ContractLaunch {
    const ElemDesc* desc;
    const ContractUnit* units;
    int64_t n_units;
    const void* mom;       // FP64 moments, or (hi, lo) FP32 pairs for the mixed path
    const int32_t* lin_idx;
    const void* lin_coef;  // double, or float2 pairs for the mixed path
    double* out;
    unsigned long long* counter;  // zeroed before the launch
    uint32_t types_mask;
    int a_cap, b_cap;      // elements of the stage-1 / stage-2 buffers
    int tile_off;          // byte offset of the FP64 tile in shared memory
    int combo_off;         // general kernel: byte offset of the per-unit combination tables
    int combo_cap;         // entries of each combination table
    int s1_cap;            // bounded-order kernel: float2 entries of the stage-1 buffer
    const int8_t* elem_mask;  // optional: units of elements with mask 0 are skipped (generic kernel)
    // operator mode (general kernel; op_terms == nullptr: the four uniform types): the terms of
    // block (gi, gj) are op_terms[op_block[2 (3 gi + gj)] + k], k < op_block[2 (3 gi + gj) + 1],
    // each packed as sa | sb << 4 | tu << 8 | tv << 12 | tw << 16 (per-axis product types),
    // with op_scales alongside; the moments of every pair then have kax[] entries per axis.
    const int32_t* op_terms;
    const double* op_scales;
    const int32_t* op_block;
    int op_nalpha;            // 3 (metric kind) or 1
    int out_ff;               // operator mode, mixed precision: write each entry's (hi, lo) FP32 pair
                              // into its 8-byte slot instead of converting it to FP64
};
struct ContractShape {
    size_t a, b, tile;
    int combos;
};
#ifdef __CUDACC__
// n / d for 0 <= n < 2^20 and d >= 1, from the FP32 reciprocal rd of d: the product is
// within 1/8 of n / d, so one correction step gives the exact quotient (an integer
// division by a runtime divisor is a long dependent sequence).
__device__ __forceinline__ int div_small(int n, int d, float rd) {
    int q = __float2int_rz(__int2float_rn(n) * rd);
    const int r = n - q * d;
    q += (r >= d) - (r < 0);
    return q;
}
#endif

// Staged contraction tile: within a row, output column (m2, n2, p2) sits at p2 * mjp + mj
// (mj = m2 * Nv_j + n2, mjp = mjn rounded up to odd) and rows have an odd stride, so the
// stage-3 stores (consecutive mj), the row reads (stride mjp) and the column reads (stride
// ld) of the write-outs are all free of bank conflicts.
__host__ __device__ __forceinline__ int contract_mj_stride(int mjn) { return mjn | 1; }
__host__ __device__ __forceinline__ int contract_tile_ld(int mjn, int nw) { return (nw * contract_mj_stride(mjn)) | 1; }
ContractShape contract_shape(const int8_t* Ni, const int8_t* Nj, int m1n, int n1n);
size_t contract_tile_offset(int precision, size_t a_cap, size_t b_cap);
// Shared memory of the general contraction: stage-1/2 buffers, the tile, then two 4-byte
// tables of combo_cap entries (packed combination indices, stage-2 run descriptors).
size_t contract_smem_bytes(int precision, size_t a_cap, size_t b_cap, size_t tile_cap, size_t combo_cap = 0);
size_t contract_combo_offset(int precision, size_t a_cap, size_t b_cap, size_t tile_cap);
cudaError_t launch_contract(int precision, const ContractLaunch& L, int grid, int threads, size_t smem,
                            cudaStream_t s);
int contract_blocks_per_sm(int precision, int threads, size_t smem);
int moments_threads();
int moments_blocks_per_sm(size_t smem);
// contract_ff.cu: mixed contraction specialised for uniform orders 2..8
bool contract_ff_runs_match(const HostTables& T);
cudaError_t contract_ff_upload(const HostTables& T);
int contract_ff_max_order();
int contract_opn_max_order();
void contract_ff_shape(int N, int m1n, size_t& a_cap, size_t& b_cap, size_t& tile_cap, int& combos);
cudaError_t launch_contract_ffn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s);
int contract_ffn_blocks_per_sm(int N, int threads, size_t smem);
// contract_ffb.cu: contraction for per-axis orders at most 8, FP64 or mixed.  Units hold full
// n1 ranges; a_cap / s1_cap / b_cap of the launch are the moment, stage-1 and stage-2 buffer
// sizes in 8-byte words.
bool contract_ffb_fits(const int8_t* Ni, const int8_t* Nj);
void contract_ffb_shape(const int8_t* Ni, const int8_t* Nj, int m1n, size_t& a_cap, size_t& s1_cap, size_t& b_cap,
                        int& combos);
// the coefficient runs ([4][8][8][8]) as (hi, lo) FP32 pairs and as FP64 values
cudaError_t contract_ffb_upload(const void* runs_ff, size_t bytes_ff, const double* runs64, size_t bytes64);
cudaError_t launch_contract_ffb(int precision, const ContractLaunch& L, int grid, int threads, size_t smem,
                                cudaStream_t s);
int contract_ffb_blocks_per_sm(int precision, int threads, size_t smem);
// operator plans of one component and uniform order N (2..6), mixed precision (contract_opn.cu)
cudaError_t launch_contract_opn(int N, const ContractLaunch& L, int grid, int threads, size_t smem, cudaStream_t s);
int contract_opn_blocks_per_sm(int N, int threads, size_t smem);
// fills contract_opn.cu's copy of the coefficient runs ([4][8][8][8] (hi, lo) pairs)
cudaError_t contract_opn_upload(const void* runs, size_t bytes);
// fused operator fill + global assembly, N = 2..4 (contract_opn.cu; mesh views in asm_stages.cuh)
struct AsmMeshDev;
struct AsmCoef;
size_t opn_assemble_smem_bytes(int N);
cudaError_t launch_opn_assemble(int N, const ContractLaunch& L, const AsmMeshDev& ms, const AsmCoef& coef, int grid,
                                int threads, size_t smem, cudaStream_t s);
int opn_assemble_blocks_per_sm(int N, int threads, size_t smem);
cudaError_t init_kernel_attributes();

// ------------------------------------------------------------------ plan building (api.cu)
// Device-resident tables of a context and the device facts the launch shapes need.
struct DeviceTables {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    double* gl_x = nullptr;
    double* gl_w = nullptr;
    int32_t* lin_idx = nullptr;
    double* lin_coef = nullptr;
    float2* lin_coef_ff = nullptr;
    int* err = nullptr;
    bool spec_ok = false;  // the compile-time coefficient runs match the table (contract_ff.cu)
};

// Everything a fill needs besides device buffers: sizes and launch shapes.
// Tile configuration of the contraction (the p2s_tile_config of the C ABI, defaults filled in).
struct TileParams {
    int combo_target = 256;             // stage-3 combinations per work unit
    size_t unit_bytes = 100 * 1024;     // shared memory of one unit (generic kernel)
    int threads = 0;                    // CTA size; 0: one thread per combination of the largest unit
    int kernel = 0;                     // 0: library choice, 1: general, 2: bounded-order kernel
};

struct PlanLayout {
    int64_t n_elem = 0;
    int n_comp = 0;
    uint32_t types_mask = 0;
    int precision = 0;
    int64_t out_entries = 0, mom_entries = 0, n_units = 0;
    int n_pairs = 1, kb = 1, gmax = 1, iacc_cap = 0;
    size_t mom_smem = 0;
    int mom_grid = 1;
    int split_grid = 0;  // FP64 plans: resident CTAs of the split moment kernel on the whole GPU
    size_t a_cap = 1, b_cap = 1, tile_cap = 1, combo_cap = 1, s1_cap = 0;
    int con_threads = 256;
    size_t con_smem = 0, tile_off = 0;
    int con_grid = 1;
    int spec_n = 0;  // > 0: the mixed contraction specialised for uniform order N
    int op = 0;      // 1: an operator plan (term list), one n x n matrix per element
    int out_ff = 0;  // operator plans, mixed precision: entries written as (hi, lo) FP32 pairs
    int spec_op = 0; // > 0: an operator plan of one component and uniform order spec_op (k_contract_opn)
    int ffb = 0;     // 1: the contraction for orders <= 8 (k_contract_ffb)
    TileParams tile;  // the tile configuration in effect
};

// Destination of the contraction work list: a growing vector, or a fixed array that
// reports overflow instead of growing.
struct UnitSink {
    std::vector<ContractUnit>* vec = nullptr;
    ContractUnit* buf = nullptr;
    int64_t cap = 0;
    int64_t n = 0;
    void push(const ContractUnit& u) {
        if (vec) vec->push_back(u);
        else if (buf && n < cap) buf[n] = u;
        ++n;
    }
    bool overflow() const { return buf && n > cap; }
};

// Record a failure for p2s_last_error and return `code`.
int fail(int code, const char* where, cudaError_t ce = cudaSuccess);
// Run a CUDA call; on failure record it and return P2S_ERR_CUDA from the caller.
#define P2S_CUDA(call)                                                 \
    do {                                                               \
        cudaError_t ce_ = (call);                                      \
        if (ce_ != cudaSuccess) return fail(P2S_ERR_CUDA, #call, ce_); \
    } while (0)
// TileParams from a p2s_tile_config (NULL or zero fields: defaults); P2S_ERR_ARG if out of range.
int tile_params_from(const p2s_tile_config* c, TileParams& tp);
// Validate the arguments and fill desc[0..E) (host), the work list and the layout.
// The first call with units.buf == nullptr && units.vec == nullptr only counts units.
int build_layout(const DeviceTables& T, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                 const p2s_fill_opts* opts, ElemDesc* desc, UnitSink& units, PlanLayout& L,
                 const TileParams& tile = TileParams(), bool moments_only = false);
// `counter` (device, one word, optional): the moment kernel's element queue; with it CTAs take
// elements dynamically, which balances batches of uneven per-element cost.
// `order` (device [E], optional): the order in which the queue hands out elements.
int run_moments(const DeviceTables& T, const PlanLayout& L, const ElemDesc* d_desc, const p2s_geometry* geom,
                const p2s_material* mat, void* moments, int32_t* elem_status, cudaStream_t s,
                unsigned long long* counter, const int8_t* elem_mask = nullptr, const int32_t* order = nullptr,
                const MomentSplit* split = nullptr);
// Device arrays of an operator plan's term list (see ContractLaunch).
struct OpArrays {
    const int32_t* terms;
    const double* scales;
    const int32_t* block;
    int nalpha;
};
// Looks up the allocation-free fill's fixed scratch array for `device` (current), once per
// device; p2s_create calls it so that the fill itself never triggers the array's load.
int noalloc_prepare(int device);
// Throughput probes behind p2s_measure_peaks (peaks.cu).
int measure_peaks(const DeviceTables& T, int64_t write_bytes, p2s_peaks* out, cudaStream_t s);
// First mode product behind p2s_mode1_product (mode1_tc.cu).
int mode1_product(const DeviceTables& T, int method, int G, int slices, const float* x, int64_t n_src, int64_t n_rows,
                  float* out, cudaStream_t s);
int run_contract(const DeviceTables& T, const PlanLayout& L, const ElemDesc* d_desc, const ContractUnit* d_units,
                 unsigned long long* d_counter, const void* moments, double* out, cudaStream_t s,
                 const int8_t* elem_mask = nullptr, const OpArrays* op = nullptr);
}  // namespace p2s
struct p2s_ctx;
struct p2s_plan;
namespace p2s {
const DeviceTables* context_tables(const p2s_ctx* c);
ElemDesc* plan_desc(p2s_plan* p);
// The plan's element order for the moment kernel's queue (device [E], allocated on the first
// call; from then on the plan's moment launches follow it).  nullptr on allocation failure.
int32_t* plan_order(p2s_plan* p);
// Fill of a plan restricted to the elements with mask != 0 (FP64 plans only; the others
// are left untouched in `out`).
// Operator plans of mixed precision only: write each output entry as its (hi, lo) FP32 pair
// (float2 in the entry's 8 bytes) rather than the FP64 value, for a consumer that continues in
// float-float.  P2S_ERR_ARG for other plans.
int plan_set_output_ff(p2s_plan* p, bool on);
// operator plans: the order of the specialised path (0: none); the moments of a fill into the
// plan's scratch; the contraction launch parameters over that scratch
int plan_spec_op(const p2s_plan* p);
int plan_run_moments(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, cudaStream_t s);
int plan_op_launch(p2s_plan* p, ContractLaunch& C);
unsigned long long* plan_counter(p2s_plan* p);
// With `list` and `count` (device: the masked elements and their number) and `part` (device,
// plan_split_part_doubles(p) doubles), the moments of the masked elements run split over the
// whole GPU (launch_moments_fp64_split) rather than one CTA per element.
int plan_fill_masked(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* out,
                     const int8_t* mask, cudaStream_t s, const int32_t* list = nullptr, const int* count = nullptr,
                     double* part = nullptr);
size_t plan_split_part_doubles(const p2s_plan* p);
cudaError_t learned_init_attributes();

}  // namespace p2s
