// Internal declarations shared by the CUDA translation units of libp2s.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "p2s.h"

namespace p2s {

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
};
size_t moments_smem_bytes(int n_pairs, int kb, int gmax, int iacc_cap);
cudaError_t launch_moments_fp64(const MomentLaunch& L, int grid, size_t smem, cudaStream_t s);

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
};
struct ContractShape {
    size_t a, b, tile;
    int combos;
};
ContractShape contract_shape(const int8_t* Ni, const int8_t* Nj, int m1n, int n1n);
size_t contract_tile_offset(int precision, size_t a_cap, size_t b_cap);
size_t contract_smem_bytes(int precision, size_t a_cap, size_t b_cap, size_t tile_cap);
cudaError_t launch_contract(int precision, const ContractLaunch& L, int grid, int threads, size_t smem,
                            cudaStream_t s);
int contract_blocks_per_sm(int precision, int threads, size_t smem);
int moments_threads();
int moments_blocks_per_sm(size_t smem);
cudaError_t init_kernel_attributes();

}  // namespace p2s
