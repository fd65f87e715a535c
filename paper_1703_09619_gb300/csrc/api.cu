// C ABI of libp2s (declared in include/p2s.h): contexts, plans, launches, error reporting.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "p2s_internal.h"

namespace p2s {
cudaError_t moments_init_attributes();
cudaError_t contract_init_attributes();
cudaError_t init_kernel_attributes() {
    cudaError_t e = moments_init_attributes();
    if (e != cudaSuccess) return e;
    return contract_init_attributes();
}
}  // namespace p2s

using namespace p2s;

struct p2s_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    double* d_gl_x = nullptr;
    double* d_gl_w = nullptr;
    int32_t* d_lin_idx = nullptr;
    double* d_lin_coef = nullptr;
    float2* d_lin_coef_ff = nullptr;
    int* d_err = nullptr;
};

struct p2s_plan {
    p2s_ctx* ctx = nullptr;
    int64_t n_elem = 0;
    int n_comp = 0;
    uint32_t types_mask = 0;
    int precision = 0;
    int64_t out_entries = 0;
    int64_t mom_entries = 0;
    int64_t n_units = 0;
    ElemDesc* d_desc = nullptr;
    ContractUnit* d_units = nullptr;
    unsigned long long* d_counter = nullptr;
    double* d_mom = nullptr;  // scratch for p2s_plan_fill
    // launch shapes
    int n_pairs = 1, kb = 1, gmax = 1;
    int iacc_cap = 0;
    size_t mom_smem = 0;
    int mom_grid = 1;
    size_t a_cap = 1, b_cap = 1, tile_cap = 1;
    int con_threads = 256;
    size_t con_smem = 0, tile_off = 0;
    int con_grid = 1;
};

namespace {

thread_local char g_last_error[256] = "";

int fail(int code, const char* where, cudaError_t ce = cudaSuccess) {
    if (ce != cudaSuccess)
        std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorString(ce),
                      cudaGetErrorName(ce));
    else
        std::snprintf(g_last_error, sizeof(g_last_error), "%s", where);
    return code;
}

// Run a CUDA call; on failure record it and return P2S_ERR_CUDA from the caller.
#define P2S_CUDA(call)                                                   \
    do {                                                                 \
        cudaError_t ce_ = (call);                                        \
        if (ce_ != cudaSuccess) return fail(P2S_ERR_CUDA, #call, ce_);   \
    } while (0)

int set_device(int dev) {
    cudaError_t e = cudaSetDevice(dev);
    return e == cudaSuccess ? P2S_OK : fail(P2S_ERR_CUDA, "cudaSetDevice", e);
}

int check_orders(int64_t E, const p2s_orders* o) {
    if (E < 0 || !o || (o->n_comp != 1 && o->n_comp != 3) || (E > 0 && !o->orders)) return P2S_ERR_ARG;
    for (int64_t i = 0; i < E * 3 * o->n_comp; ++i)
        if (o->orders[i] < 1 || o->orders[i] > kMaxOrder) return P2S_ERR_ORDER;
    return P2S_OK;
}

int64_t elem_ndof(const int32_t* ord, int nc) {
    int64_t n = 0;
    for (int g = 0; g < nc; ++g) n += (int64_t)ord[3 * g] * ord[3 * g + 1] * ord[3 * g + 2];
    return n;
}

int ntypes(uint32_t m) { return __builtin_popcount(m & 0xFu); }

void pair_of(int s, int nc, int& gi, int& gj) {
    static const int tgi[6] = {0, 0, 0, 1, 1, 2}, tgj[6] = {0, 1, 2, 1, 2, 2};
    if (nc == 1) { gi = gj = 0; return; }
    gi = tgi[s];
    gj = tgj[s];
}

int64_t elem_moments(const int32_t* ord, int nc) {
    int np = nc == 1 ? 1 : 6;
    int64_t m = 0;
    for (int s = 0; s < np; ++s) {
        int gi, gj;
        pair_of(s, nc, gi, gj);
        int64_t v = 1;
        for (int ax = 0; ax < 3; ++ax) v *= ord[3 * gi + ax] + ord[3 * gj + ax] - 1;
        m += v;
    }
    return m;
}


// Contraction work list of one element.  Symmetry of the coupling factor
// (alpha_{gi gj} = alpha_{gj gi}) and of the Eq. (3) coefficients gives
//   vv(gj,gi) = vv(gi,gj)^T,  dd(gj,gi) = dd(gi,gj)^T,  vd(gj,gi) = dv(gi,gj)^T,
// so each such pair of blocks is computed once and written twice.  Slabs of m1 and n1
// keep one unit's shared-memory tile small and its thread count near one per
// stage-3 combination.
constexpr int kComboTarget = 256;
constexpr size_t kUnitBytesTarget = 100 * 1024;

void slab_sizes(const ElemDesc& d, int gi, int gj, int& m1n, int& n1n) {
    const int8_t* Ni = d.ord[gi];
    const int8_t* Nj = d.ord[gj];
    n1n = Ni[1];
    m1n = 1;
    auto bytes = [&](int a, int b) {
        ContractShape s = contract_shape(Ni, Nj, a, b);
        return (s.a + s.b + s.tile) * sizeof(double);
    };
    while (n1n > 1 && (bytes(1, n1n) > kUnitBytesTarget || contract_shape(Ni, Nj, 1, n1n).combos > 2 * kComboTarget))
        --n1n;
    if (n1n == Ni[1])
        while (m1n < Ni[0] && contract_shape(Ni, Nj, m1n + 1, n1n).combos <= kComboTarget &&
               bytes(m1n + 1, n1n) <= kUnitBytesTarget)
            ++m1n;
}

void push_block(const ElemDesc& d, int32_t e, int gi, int gj, int t, int tp, std::vector<ContractUnit>& units) {
    int m1n, n1n;
    slab_sizes(d, gi, gj, m1n, n1n);
    const int Nu = d.ord[gi][0], Nv = d.ord[gi][1];
    for (int m1a = 0; m1a < Nu; m1a += m1n)
        for (int n1a = 0; n1a < Nv; n1a += n1n) {
            ContractUnit u;
            u.e = e;
            u.gi = (int8_t)gi;
            u.gj = (int8_t)gj;
            u.t = (int8_t)t;
            u.tp = (int8_t)tp;
            u.m1a = (int8_t)m1a;
            u.m1n = (int8_t)std::min(m1n, Nu - m1a);
            u.n1a = (int8_t)n1a;
            u.n1n = (int8_t)std::min(n1n, Nv - n1a);
            u.pad = 0;
            units.push_back(u);
        }
}

void add_units(const ElemDesc& d, uint32_t mask, int32_t e, std::vector<ContractUnit>& units) {
    const int nc = d.n_comp;
    for (int t : {0, 3}) {  // vv, dd: upper blocks, transposed into the lower ones
        if (!(mask & (1u << t))) continue;
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = gi; gj < nc; ++gj) push_block(d, e, gi, gj, t, gi == gj ? -1 : t, units);
    }
    const bool dv = mask & 2u, vd = mask & 4u;
    if (dv || vd) {  // dv(gi,gj) and its transpose vd(gj,gi)
        const int t = dv ? 1 : 2, tp = (dv && vd) ? 2 : -1;
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = 0; gj < nc; ++gj) push_block(d, e, gi, gj, t, tp, units);
    }
}

}  // namespace

extern "C" {

const char* p2s_last_error(void) { return g_last_error; }

const char* p2s_error_string(int code) {
    switch (code) {
    case P2S_OK: return "ok";
    case P2S_ERR_ARG: return "invalid argument";
    case P2S_ERR_ORDER: return "order or quadrature size out of range";
    case P2S_ERR_JACOBIAN: return "detJ <= 0 at a quadrature point";
    case P2S_ERR_OOM: return "out of memory";
    case P2S_ERR_CUDA: return "CUDA error";
    case P2S_ERR_TIMEOUT: return "device wait timed out";
    case P2S_ERR_BUFFER: return "buffer too small";
    }
    return "unknown error";
}

int p2s_gauss_legendre(int G, double* x, double* w) {
    if (G < 1 || G > kMaxG || !x || !w) return P2S_ERR_ARG;
    const HostTables& T = host_tables();
    std::memcpy(x, T.gl_x[G], sizeof(double) * G);
    std::memcpy(w, T.gl_w[G], sizeof(double) * G);
    return P2S_OK;
}

int p2s_linearisation(int t, int m1, int m2, int kmax, double* C) {
    if (t < 0 || t > 3 || m1 < 0 || m2 < 0 || m1 >= kMaxOrder || m2 >= kMaxOrder || kmax < 0 || !C)
        return P2S_ERR_ARG;
    const HostTables& T = host_tables();
    for (int k = 0; k <= kmax; ++k) C[k] = 0.0;
    int32_t li = T.lin_idx[lin_slot(t, m1, m2)];
    for (int r = 0; r < lin_cnt(li); ++r) {
        int k = lin_kmin(li) + 2 * r;
        if (k <= kmax) C[k] = T.lin_coef[lin_off(li) + r];
    }
    return P2S_OK;
}

static int ctx_init(p2s_ctx* c, int device) {
    c->device = device;
    cudaDeviceProp prop;
    P2S_CUDA(cudaGetDeviceProperties(&prop, device));
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    const HostTables& T = host_tables();
    size_t glb = sizeof(double) * (kMaxG + 1) * kMaxG;
    P2S_CUDA(cudaMalloc(&c->d_gl_x, glb));
    P2S_CUDA(cudaMalloc(&c->d_gl_w, glb));
    P2S_CUDA(cudaMalloc(&c->d_lin_idx, sizeof(T.lin_idx)));
    P2S_CUDA(cudaMalloc(&c->d_lin_coef, sizeof(double) * std::max(1, T.n_coef)));
    P2S_CUDA(cudaMalloc(&c->d_lin_coef_ff, sizeof(float2) * std::max(1, T.n_coef)));
    P2S_CUDA(cudaMalloc(&c->d_err, sizeof(int)));
    P2S_CUDA(cudaMemcpy(c->d_gl_x, T.gl_x, glb, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(c->d_gl_w, T.gl_w, glb, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(c->d_lin_idx, T.lin_idx, sizeof(T.lin_idx), cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(c->d_lin_coef, T.lin_coef, sizeof(double) * T.n_coef, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(c->d_lin_coef_ff, T.lin_coef_ff, sizeof(float2) * T.n_coef, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    P2S_CUDA(init_kernel_attributes());
    return P2S_OK;
}

int p2s_create(p2s_ctx** out, int device) {
    if (!out) return fail(P2S_ERR_ARG, "p2s_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess) return fail(P2S_ERR_CUDA, "cudaGetDeviceCount", ce);
    if (device < 0 || device >= ndev) return fail(P2S_ERR_ARG, "p2s_create: no such device");
    if (set_device(device)) return P2S_ERR_CUDA;
    p2s_ctx* c = new (std::nothrow) p2s_ctx();
    if (!c) return fail(P2S_ERR_OOM, "p2s_create: host allocation");
    int rc = ctx_init(c, device);
    if (rc) {
        p2s_destroy(c);
        return rc;
    }
    *out = c;
    return P2S_OK;
}

void p2s_destroy(p2s_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->d_gl_x);
    cudaFree(c->d_gl_w);
    cudaFree(c->d_lin_idx);
    cudaFree(c->d_lin_coef);
    cudaFree(c->d_lin_coef_ff);
    cudaFree(c->d_err);
    delete c;
}

int64_t p2s_output_entries(int64_t n_elem, const p2s_orders* orders, uint32_t types_mask, int64_t* offsets) {
    int rc = check_orders(n_elem, orders);
    if (rc) return rc;
    if ((types_mask & 0xFu) == 0 || (types_mask & ~0xFu)) return P2S_ERR_ARG;
    int nt = ntypes(types_mask);
    int64_t off = 0;
    for (int64_t e = 0; e < n_elem; ++e) {
        if (offsets) offsets[e] = off;
        int64_t n = elem_ndof(orders->orders + 3 * orders->n_comp * e, orders->n_comp);
        off += nt * n * n;
    }
    if (offsets) offsets[n_elem] = off;
    return off;
}

int64_t p2s_moment_entries(int64_t n_elem, const p2s_orders* orders, int64_t* offsets) {
    int rc = check_orders(n_elem, orders);
    if (rc) return rc;
    int64_t off = 0;
    for (int64_t e = 0; e < n_elem; ++e) {
        if (offsets) offsets[e] = off;
        off += elem_moments(orders->orders + 3 * orders->n_comp * e, orders->n_comp);
    }
    if (offsets) offsets[n_elem] = off;
    return off;
}

void p2s_plan_destroy(p2s_plan* p) {
    if (!p) return;
    if (p->ctx) cudaSetDevice(p->ctx->device);
    cudaFree(p->d_desc);
    cudaFree(p->d_units);
    cudaFree(p->d_counter);
    cudaFree(p->d_mom);
    delete p;
}

int p2s_plan_create(p2s_ctx* ctx, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                    const p2s_fill_opts* opts, p2s_plan** out) {
    if (!ctx || !out || !quad || !opts) return P2S_ERR_ARG;
    *out = nullptr;
    int rc = check_orders(E, orders);
    if (rc) return rc;
    if ((opts->types_mask & 0xFu) == 0 || (opts->types_mask & ~0xFu)) return P2S_ERR_ARG;
    if (opts->precision != P2S_FP64 && opts->precision != P2S_MIXED) return P2S_ERR_ARG;
    if (quad->npts_uniform < 0 || quad->npts_uniform > kMaxG) return P2S_ERR_ORDER;
    if (quad->npts_uniform == 0 && E > 0 && !quad->npts) return P2S_ERR_ARG;
    if (set_device(ctx->device)) return P2S_ERR_CUDA;

    const int nc = orders->n_comp;
    std::vector<ElemDesc> desc((size_t)std::max<int64_t>(E, 1));
    std::vector<ContractUnit> units;
    p2s_plan* p = new (std::nothrow) p2s_plan();
    if (!p) return P2S_ERR_OOM;
    p->ctx = ctx;
    p->n_elem = E;
    p->n_comp = nc;
    p->types_mask = opts->types_mask;
    p->precision = opts->precision;
    p->n_pairs = nc == 1 ? 1 : 6;
    const int nt = ntypes(opts->types_mask);
    int64_t out_off = 0, mom_off = 0;
    int max_pair = 1, max_elem_mom = 1;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ord = orders->orders + 3 * nc * e;
        ElemDesc& d = desc[e];
        std::memset(&d, 0, sizeof(d));
        int G = quad->npts_uniform ? quad->npts_uniform : quad->npts[e];
        if (G < 1 || G > kMaxG) { delete p; return P2S_ERR_ORDER; }
        d.G = (int16_t)G;
        d.n_comp = (int8_t)nc;
        d.n_types = (int8_t)nt;
        int dof = 0;
        for (int g = 0; g < nc; ++g) {
            d.dof_off[g] = dof;
            for (int ax = 0; ax < 3; ++ax) d.ord[g][ax] = (int8_t)ord[3 * g + ax];
            dof += ord[3 * g] * ord[3 * g + 1] * ord[3 * g + 2];
        }
        d.n = dof;
        for (int ax = 0; ax < 3; ++ax) {
            int mx = 0;
            for (int g = 0; g < nc; ++g) mx = std::max(mx, (int)ord[3 * g + ax]);
            d.kax[ax] = (int8_t)(2 * mx - 1);
            p->kb = std::max(p->kb, 2 * mx - 1);
        }
        int po = 0;
        for (int s = 0; s < p->n_pairs; ++s) {
            int gi, gj;
            pair_of(s, nc, gi, gj);
            d.pair_off[s] = po;
            int v = 1;
            for (int ax = 0; ax < 3; ++ax) v *= ord[3 * gi + ax] + ord[3 * gj + ax] - 1;
            po += v;
        }
        d.out_off = out_off;
        d.mom_off = mom_off;
        out_off += (int64_t)nt * dof * dof;
        mom_off += po;
        max_pair = std::max(max_pair, d.kax[0] * d.kax[1] * d.kax[2]);
        max_elem_mom = std::max(max_elem_mom, p->n_pairs * d.kax[0] * d.kax[1] * d.kax[2]);
        p->gmax = std::max(p->gmax, G);
        add_units(d, opts->types_mask, (int32_t)e, units);
    }
    p->out_entries = out_off;
    p->mom_entries = mom_off;
    p->n_units = (int64_t)units.size();

    // moments launch shape: the accumulator takes what shared memory leaves, at least one pair
    size_t base = moments_smem_bytes(p->n_pairs, p->kb, p->gmax, 0);
    size_t limit = std::min<size_t>(ctx->smem_optin, 227 * 1024) - 1024;  // room for static shared memory
    if (base + sizeof(double) * max_pair > limit) { delete p; return P2S_ERR_ORDER; }
    p->iacc_cap = (int)std::min<size_t>((limit - base) / sizeof(double), (size_t)max_elem_mom);
    // prefer two CTAs per SM when everything fits in half the shared memory
    size_t half = limit / 2 - 1024;
    if (base + sizeof(double) * max_elem_mom <= half) p->iacc_cap = max_elem_mom;
    p->mom_smem = moments_smem_bytes(p->n_pairs, p->kb, p->gmax, p->iacc_cap);
    int per_sm = moments_blocks_per_sm(p->mom_smem);
    if (per_sm < 1) { delete p; return fail(P2S_ERR_ORDER, "p2s_plan_create: moment kernel does not fit"); }
    p->mom_grid = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)ctx->sm_count * per_sm));

    // contraction launch shape: buffers sized for the largest unit, one thread per
    // stage-3 combination of the largest unit (rounded to whole warps)
    int max_combos = 1;
    for (const ContractUnit& u : units) {
        const ElemDesc& d = desc[u.e];
        ContractShape sh = contract_shape(d.ord[u.gi], d.ord[u.gj], u.m1n, u.n1n);
        p->a_cap = std::max(p->a_cap, sh.a);
        p->b_cap = std::max(p->b_cap, sh.b);
        p->tile_cap = std::max(p->tile_cap, sh.tile);
        max_combos = std::max(max_combos, sh.combos);
    }
    p->con_threads = std::min(512, std::max(64, (max_combos + 31) / 32 * 32));
    p->tile_off = contract_tile_offset(p->precision, p->a_cap, p->b_cap);
    p->con_smem = contract_smem_bytes(p->precision, p->a_cap, p->b_cap, p->tile_cap);
    if (p->con_smem > limit) { delete p; return fail(P2S_ERR_ORDER, "p2s_plan_create: contraction tile too large"); }
    int con_per_sm = contract_blocks_per_sm(p->precision, p->con_threads, p->con_smem);
    if (con_per_sm < 1) { delete p; return fail(P2S_ERR_ORDER, "p2s_plan_create: contraction kernel does not fit"); }
    p->con_grid = ctx->sm_count * con_per_sm;

    bool ok = cudaMalloc(&p->d_desc, sizeof(ElemDesc) * desc.size()) == cudaSuccess &&
              cudaMalloc(&p->d_units, sizeof(ContractUnit) * std::max<size_t>(1, units.size())) == cudaSuccess &&
              cudaMalloc(&p->d_counter, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&p->d_mom, sizeof(double) * std::max<int64_t>(1, p->mom_entries)) == cudaSuccess;
    if (!ok) { p2s_plan_destroy(p); return P2S_ERR_OOM; }
    if (cudaMemcpy(p->d_desc, desc.data(), sizeof(ElemDesc) * desc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (units.size() && cudaMemcpy(p->d_units, units.data(), sizeof(ContractUnit) * units.size(),
                                    cudaMemcpyHostToDevice) != cudaSuccess)) {
        p2s_plan_destroy(p);
        return P2S_ERR_CUDA;
    }
    *out = p;
    return P2S_OK;
}

int64_t p2s_plan_output_entries(const p2s_plan* p) { return p ? p->out_entries : P2S_ERR_ARG; }
int64_t p2s_plan_moment_entries(const p2s_plan* p) { return p ? p->mom_entries : P2S_ERR_ARG; }

int p2s_plan_moments(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* moments,
                     int32_t* elem_status, void* stream) {
    if (!p || !geom || !mat) return fail(P2S_ERR_ARG, "p2s_plan_moments: NULL plan, geometry or material");
    if (geom->n_elem != p->n_elem) return fail(P2S_ERR_ARG, "p2s_plan_moments: n_elem differs from the plan");
    if (p->n_elem == 0) return P2S_OK;
    if (!moments || !mat->params) return fail(P2S_ERR_ARG, "p2s_plan_moments: NULL moments or params");
    if (mat->kind == P2S_ALPHA_SCALAR) {
        if (p->n_comp != 1) return P2S_ERR_ARG;
    } else if (mat->kind == P2S_ALPHA_METRIC_EPS) {
        if (p->n_comp != 3 || !geom->nodes) return P2S_ERR_ARG;
    } else {
        return P2S_ERR_ARG;
    }
    if (set_device(p->ctx->device)) return P2S_ERR_CUDA;
    MomentLaunch L;
    L.desc = p->d_desc;
    L.n_elem = p->n_elem;
    L.kind = mat->kind;
    L.params = mat->params;
    L.nodes = geom->nodes;
    L.bulge = geom->bulge;
    L.gl_x = p->ctx->d_gl_x;
    L.gl_w = p->ctx->d_gl_w;
    L.mom = moments;
    L.elem_status = elem_status;
    L.err_flag = p->ctx->d_err;
    L.n_pairs = p->n_pairs;
    L.kb = p->kb;
    L.gmax = p->gmax;
    L.iacc_cap = p->iacc_cap;
    L.out_ff = p->precision == P2S_MIXED;
    P2S_CUDA(launch_moments_fp64(L, p->mom_grid, p->mom_smem, (cudaStream_t)stream));
    return P2S_OK;
}

int p2s_plan_contract(p2s_plan* p, const double* moments, double* out, void* stream) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_contract: NULL plan");
    if (p->n_units == 0) return P2S_OK;
    if (!moments || !out) return fail(P2S_ERR_ARG, "p2s_plan_contract: NULL moments or out");
    if (set_device(p->ctx->device)) return P2S_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    P2S_CUDA(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), s));
    ContractLaunch L;
    L.desc = p->d_desc;
    L.units = p->d_units;
    L.n_units = p->n_units;
    L.mom = moments;
    L.lin_idx = p->ctx->d_lin_idx;
    L.lin_coef = p->precision == P2S_MIXED ? (const void*)p->ctx->d_lin_coef_ff : (const void*)p->ctx->d_lin_coef;
    L.out = out;
    L.counter = p->d_counter;
    L.types_mask = p->types_mask;
    L.a_cap = (int)p->a_cap;
    L.b_cap = (int)p->b_cap;
    L.tile_off = (int)p->tile_off;
    P2S_CUDA(launch_contract(p->precision, L, p->con_grid, p->con_threads, p->con_smem, s));
    return P2S_OK;
}

int p2s_plan_fill(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* out,
                  int32_t* elem_status, void* stream) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_fill: NULL plan");
    if (!out && p->n_units) return fail(P2S_ERR_ARG, "p2s_plan_fill: NULL out");
    int rc = p2s_plan_moments(p, geom, mat, p->d_mom, elem_status, stream);
    if (rc) return rc;
    return p2s_plan_contract(p, p->d_mom, out, stream);
}

int p2s_fill_elements(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat, const p2s_orders* orders,
                      const p2s_quadrature* quad, const p2s_fill_opts* opts, double* out, int32_t* elem_status,
                      void* stream) {
    if (!geom) return P2S_ERR_ARG;
    p2s_plan* p = nullptr;
    int rc = p2s_plan_create(ctx, geom->n_elem, orders, quad, opts, &p);
    if (rc) return rc;
    rc = p2s_plan_fill(p, geom, mat, out, elem_status, stream);
    if (rc == P2S_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = P2S_ERR_CUDA;
    p2s_plan_destroy(p);
    return rc;
}

int p2s_sync_status(p2s_ctx* ctx, void* stream) {
    if (!ctx) return P2S_ERR_ARG;
    if (set_device(ctx->device)) return P2S_ERR_CUDA;
    P2S_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    P2S_CUDA(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) P2S_CUDA(cudaMemset(ctx->d_err, 0, sizeof(int)));
    return h;
}

}  // extern "C"
