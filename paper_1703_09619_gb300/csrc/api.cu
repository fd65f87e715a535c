// C ABI of libp2s (declared in include/p2s.h): contexts, plans, launches, error reporting.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "p2s_internal.h"

namespace p2s {
cudaError_t moments_init_attributes();
cudaError_t moments_dw_init_attributes();
cudaError_t contract_init_attributes();
cudaError_t init_kernel_attributes() {
    cudaError_t e = moments_init_attributes();
    if (e != cudaSuccess) return e;
    e = moments_dw_init_attributes();
    if (e != cudaSuccess) return e;
    return contract_init_attributes();
}

namespace {
thread_local char g_last_error[256] = "";
}

int fail(int code, const char* where, cudaError_t ce) {
    // a failed allocation also sets the runtime's last-error state; clear it, or the error
    // check after the next kernel launch on this thread would report it as that launch's
    if (code == P2S_ERR_OOM) (void)cudaGetLastError();
    if (ce != cudaSuccess)
        std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorString(ce),
                      cudaGetErrorName(ce));
    else
        std::snprintf(g_last_error, sizeof(g_last_error), "%s", where);
    return code;
}

}  // namespace p2s

using namespace p2s;

struct p2s_ctx {
    DeviceTables T;
};

struct p2s_plan {
    p2s_ctx* ctx = nullptr;
    PlanLayout L;
    ElemDesc* d_desc = nullptr;
    ContractUnit* d_units = nullptr;
    unsigned long long* d_counter = nullptr;  // [0] contraction unit queue, [1] moment element queue
    double* d_mom = nullptr;  // moment scratch of p2s_plan_fill
    int32_t* d_order = nullptr;  // optional element order of the moment queue
    // moment view: an operator plan computes its moments on a virtual element (every coupling
    // entry at the element's largest K); other plans alias L and d_desc
    PlanLayout Lm;
    ElemDesc* d_mdesc = nullptr;
    // operator plans: terms grouped by block, packed (see ContractLaunch), their scales, and
    // the (start, count) of each block (gi, gj) at 2 (3 gi + gj)
    int32_t* d_op_terms = nullptr;
    double* d_op_scales = nullptr;
    int32_t* d_op_block = nullptr;
    int op_nalpha = 0;
    // CUDA-graph replay of p2s_plan_fill: the launch sequence (queue reset, moments,
    // contraction) captured on a private stream, re-captured when the arguments change
    bool use_graph = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int gkind = -1;
    int64_t gn = -1;
};


namespace {

int set_device(int dev) {
    cudaError_t e = cudaSetDevice(dev);
    return e == cudaSuccess ? P2S_OK : fail(P2S_ERR_CUDA, "cudaSetDevice", e);
}

int check_orders(int64_t E, const p2s_orders* o) {
    if (E < 0 || !o || (o->n_comp != 1 && o->n_comp != 3) || (E > 0 && !o->orders))
        return fail(P2S_ERR_ARG, "orders: bad count, component number or NULL array");
    for (int64_t i = 0; i < E * 3 * o->n_comp; ++i)
        if (o->orders[i] < 1 || o->orders[i] > kMaxOrder) return fail(P2S_ERR_ORDER, "orders: value outside 1..12");
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
// m1 slab of the bounded-order kernel: full n1, as many m1 as keep the unit's stage-3
// combinations within the target (at least one)
int ffb_m1_slab(const int8_t* Ni, const int8_t* Nj, const TileParams& tp) {
    const int per_m1 = Ni[1] * Nj[0] * Nj[1];
    int m1n = 1;
    while (m1n < Ni[0] && (m1n + 1) * per_m1 <= tp.combo_target) ++m1n;
    return m1n;
}

void slab_sizes(const ElemDesc& d, int gi, int gj, int& m1n, int& n1n, int spec_n, const TileParams& tp,
                bool ffb = false) {
    const int kComboTarget = tp.combo_target;
    const size_t kUnitBytesTarget = tp.unit_bytes;
    const int8_t* Ni = d.ord[gi];
    const int8_t* Nj = d.ord[gj];
    n1n = Ni[1];
    m1n = 1;
    if (spec_n) {  // specialised kernel: full n1, one thread per stage-3 combination
        const int n3 = spec_n * spec_n * spec_n;
        while (m1n < spec_n && (m1n + 1) * n3 <= kComboTarget) ++m1n;
        return;
    }
    if (ffb) {
        m1n = ffb_m1_slab(Ni, Nj, tp);
        return;
    }
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

void push_block(const ElemDesc& d, int32_t e, int gi, int gj, int t, int tp, UnitSink& units, int spec_n,
                const TileParams& tile, bool ffb = false) {
    int m1n, n1n;
    slab_sizes(d, gi, gj, m1n, n1n, spec_n, tile, ffb);
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
            units.push(u);
        }
}

void add_units(const ElemDesc& d, uint32_t mask, int32_t e, UnitSink& units, int spec_n, const TileParams& tile,
               bool ffb) {
    const int nc = d.n_comp;
    for (int t : {0, 3}) {  // vv, dd: upper blocks, transposed into the lower ones
        if (!(mask & (1u << t))) continue;
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = gi; gj < nc; ++gj)
                push_block(d, e, gi, gj, t, gi == gj ? -1 : t, units, spec_n, tile, ffb);
    }
    const bool dv = mask & 2u, vd = mask & 4u;
    if (dv || vd) {  // dv(gi,gj) and its transpose vd(gj,gi)
        const int t = dv ? 1 : 2, tp = (dv && vd) ? 2 : -1;
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = 0; gj < nc; ++gj) push_block(d, e, gi, gj, t, tp, units, spec_n, tile, ffb);
    }
}

// Launch shape of the bounded-order mixed contraction (contract_ffb.cu) for a batch: moment
// and stage-2 buffers sized for the largest unit, one thread per stage-3 combination of the
// largest unit (rounded to whole warps) unless the tile configuration fixes the CTA size.
// False when an order passes the kernel's bound or the buffers or the CTA do not fit.
struct FfbLaunch {
    size_t a_cap = 1, s1_cap = 1, b_cap = 1, smem = 0;
    int combos = 1, threads = 0, grid = 0;
};
bool ffb_launch_shape(const DeviceTables& T, int64_t E, const p2s_orders* orders, const TileParams& tile,
                      size_t limit, int precision, FfbLaunch& F) {
    const int nc = orders->n_comp;
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ord = orders->orders + 3 * nc * e;
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = 0; gj < nc; ++gj) {
                int8_t Ni[3], Nj[3];
                for (int ax = 0; ax < 3; ++ax) {
                    Ni[ax] = (int8_t)ord[3 * gi + ax];
                    Nj[ax] = (int8_t)ord[3 * gj + ax];
                }
                if (!contract_ffb_fits(Ni, Nj)) return false;
                size_t a, s1, b;
                int combos;
                contract_ffb_shape(Ni, Nj, ffb_m1_slab(Ni, Nj, tile), a, s1, b, combos);
                F.a_cap = std::max(F.a_cap, a);
                F.s1_cap = std::max(F.s1_cap, s1);
                F.b_cap = std::max(F.b_cap, b);
                F.combos = std::max(F.combos, combos);
            }
    }
    F.threads = tile.threads ? tile.threads : std::min(512, std::max(64, (F.combos + 31) / 32 * 32));
    F.smem = (F.a_cap + F.s1_cap + F.b_cap) * sizeof(double);  // 8-byte words in either precision
    if (F.smem > limit) return false;
    const int per_sm = contract_ffb_blocks_per_sm(precision, F.threads, F.smem);
    if (per_sm < 1) return false;
    F.grid = T.sm_count * per_sm;
    return true;
}

}  // namespace

namespace p2s {

// Launch shape of the general contraction for E elements with nc field components: the
// buffers sized for the largest unit, one thread per stage-3 combination of the largest unit
// (rounded to whole warps) unless the tile configuration fixes the CTA size.  With `check`
// the shared memory must fit (`limit`) and at least one CTA per SM.
int general_contract_shape(const DeviceTables& T, int64_t E, const ElemDesc* desc, int nc, const TileParams& tile,
                           bool check, size_t limit, PlanLayout& L) {
    int max_combos = 1;
    for (int64_t e = 0; e < E; ++e) {
        const ElemDesc& d = desc[e];
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = 0; gj < nc; ++gj) {
                int m1n, n1n;
                slab_sizes(d, gi, gj, m1n, n1n, 0, tile);
                ContractShape sh = contract_shape(d.ord[gi], d.ord[gj], m1n, n1n);
                L.a_cap = std::max(L.a_cap, sh.a);
                L.b_cap = std::max(L.b_cap, sh.b);
                L.tile_cap = std::max(L.tile_cap, sh.tile);
                max_combos = std::max(max_combos, sh.combos);
            }
    }
    L.tile = tile;
    L.con_threads = tile.threads ? tile.threads : std::min(512, std::max(64, (max_combos + 31) / 32 * 32));
    L.combo_cap = (size_t)max_combos;
    L.tile_off = contract_tile_offset(L.precision, L.a_cap, L.b_cap);
    L.con_smem = contract_smem_bytes(L.precision, L.a_cap, L.b_cap, L.tile_cap, L.combo_cap);
    if (check) {
        if (L.con_smem > limit) return fail(P2S_ERR_ORDER, "plan: contraction tile too large");
        int con_per_sm = contract_blocks_per_sm(L.precision, L.con_threads, L.con_smem);
        if (con_per_sm < 1) return fail(P2S_ERR_ORDER, "plan: contraction kernel does not fit");
        L.con_grid = T.sm_count * con_per_sm;
    }
    return P2S_OK;
}

int tile_params_from(const p2s_tile_config* c, TileParams& tp) {
    tp = TileParams();
    if (!c) return P2S_OK;
    if (c->combo_target < 0 || c->combo_target > 4096 || c->unit_kbytes < 0 || c->unit_kbytes > 227 ||
        c->threads < 0 || c->threads > 512 || (c->threads && (c->threads < 64 || c->threads % 32)))
        return fail(P2S_ERR_ARG, "tile config: combo_target 0..4096, unit_kbytes 0..227, threads 0 or 64..512 in steps of 32");
    if (c->kernel < 0 || c->kernel > 2) return fail(P2S_ERR_ARG, "tile config: kernel 0, 1 or 2");
    if (c->combo_target) tp.combo_target = c->combo_target;
    if (c->unit_kbytes) tp.unit_bytes = (size_t)c->unit_kbytes * 1024;
    tp.threads = c->threads;
    tp.kernel = c->kernel;
    return P2S_OK;
}

int build_layout(const DeviceTables& T, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                 const p2s_fill_opts* opts, ElemDesc* desc, UnitSink& units, PlanLayout& L, const TileParams& tile,
                 bool moments_only) {
    if (!quad || !opts) return fail(P2S_ERR_ARG, "plan: NULL quadrature or options");
    int rc = check_orders(E, orders);
    if (rc) return rc;
    if ((opts->types_mask & 0xFu) == 0 || (opts->types_mask & ~0xFu)) return fail(P2S_ERR_ARG, "plan: bad types_mask");
    if (opts->precision != P2S_FP64 && opts->precision != P2S_MIXED) return fail(P2S_ERR_ARG, "plan: bad precision");
    if (quad->npts_uniform < 0 || quad->npts_uniform > kMaxG) return fail(P2S_ERR_ORDER, "plan: npts outside 1..64");
    if (quad->npts_uniform == 0 && E > 0 && !quad->npts) return fail(P2S_ERR_ARG, "plan: NULL npts array");

    const int nc = orders->n_comp;
    L = PlanLayout();
    L.n_elem = E;
    L.n_comp = nc;
    L.types_mask = opts->types_mask;
    L.precision = opts->precision;
    L.n_pairs = nc == 1 ? 1 : 6;
    const int nt = ntypes(opts->types_mask);
    int64_t out_off = 0, mom_off = 0;
    int max_pair = 1, max_elem_mom = 1;
    // the kernels specialised on the coefficient runs, once the compile-time runs are verified
    // against the table: for mixed precision with every order of the batch equal to one N in
    // 2..8 the per-order kernel (contract_ff.cu), else with every order at most 8 the
    // bounded-order kernel (contract_ffb.cu, either precision), unless the tile configuration
    // names a kernel
    const size_t limit = std::min<size_t>(T.smem_optin, 227 * 1024) - 1024;  // room for static shared memory
    int spec_n = 0;
    bool ffb = false;
    FfbLaunch ffl;
    if (tile.kernel == 2 && E > 0 && !moments_only) {
        if (!(T.spec_ok && ffb_launch_shape(T, E, orders, tile, limit, L.precision, ffl)))
            return fail(P2S_ERR_ORDER, "plan: the bounded-order kernel needs orders <= 8 and a fitting unit");
        ffb = true;
    } else if (T.spec_ok && E > 0 && tile.kernel == 0 && !moments_only) {
        if (L.precision == P2S_MIXED) {
            const int N = orders->orders[0];
            bool uniform = N >= 2 && N <= contract_ff_max_order();
            for (int64_t i = 0; uniform && i < E * 3 * nc; ++i) uniform = orders->orders[i] == N;
            if (uniform) spec_n = N;
        }
        if (!spec_n) ffb = ffb_launch_shape(T, E, orders, tile, limit, L.precision, ffl);
    }
    for (int64_t e = 0; e < E; ++e) {
        const int32_t* ord = orders->orders + 3 * nc * e;
        ElemDesc& d = desc[e];
        std::memset(&d, 0, sizeof(d));
        int G = quad->npts_uniform ? quad->npts_uniform : quad->npts[e];
        if (G < 1 || G > kMaxG) return fail(P2S_ERR_ORDER, "plan: npts outside 1..64");
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
            L.kb = std::max(L.kb, 2 * mx - 1);
        }
        int po = 0;
        for (int s = 0; s < L.n_pairs; ++s) {
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
        max_elem_mom = std::max(max_elem_mom, L.n_pairs * d.kax[0] * d.kax[1] * d.kax[2]);
        L.gmax = std::max(L.gmax, G);
        if (!moments_only) add_units(d, opts->types_mask, (int32_t)e, units, spec_n, tile, ffb);
    }
    L.out_entries = out_off;
    L.mom_entries = mom_off;
    L.n_units = units.n;
    // The specialised contraction compiles one code path per product type; units taken in
    // element order interleave the four, and CTAs running different paths on one SM starve
    // on instruction fetch.  Within chunks of kTypeChunk elements (whose moments stay in L2
    // across the passes) the units are ordered by type, elements in order within a type.
    if ((spec_n || ffb) && !units.overflow()) {
        ContractUnit* first = units.vec ? units.vec->data() : units.buf;
        if (first) {
            constexpr int32_t kTypeChunk = 1024;
            std::stable_sort(first, first + units.n, [](const ContractUnit& a, const ContractUnit& b) {
                const int32_t ca = a.e / kTypeChunk, cb = b.e / kTypeChunk;
                return ca != cb ? ca < cb : a.t < b.t;
            });
        }
    }

    // moments launch shape: the accumulator takes what shared memory leaves, at least one pair
    // the mixed path evaluates alpha and the moments in double-word arithmetic (moments_dw.cu)
    const bool dwm = L.precision == P2S_MIXED;
    auto msmem = [&](int cap) {
        return dwm ? moments_dw_smem_bytes(L.n_pairs, L.kb, L.gmax, cap) : moments_smem_bytes(L.n_pairs, L.kb, L.gmax, cap);
    };
    // (the double-word kernel's accumulator holds whole pair slots: two pairs each, at least one)
    const size_t need_min = dwm ? 2 * (size_t)max_pair : (size_t)max_pair;
    const size_t need_all = dwm ? (size_t)moments_dw_iacc_words(L.n_pairs, max_pair) : (size_t)max_elem_mom;
    size_t base = msmem(0);
    if (base + sizeof(double) * need_min > limit) return fail(P2S_ERR_ORDER, "plan: moment accumulator too large");
    L.iacc_cap = (int)std::min<size_t>((limit - base) / sizeof(double), need_all);
    if (dwm) L.iacc_cap &= ~1;
    size_t half = limit / 2 - 1024;  // two CTAs per SM when everything fits in half
    if (base + sizeof(double) * need_all <= half) L.iacc_cap = (int)need_all;
    L.mom_smem = msmem(L.iacc_cap);
    int per_sm = dwm ? moments_dw_blocks_per_sm(L.mom_smem) : moments_blocks_per_sm(L.mom_smem);
    if (per_sm < 1) return fail(P2S_ERR_ORDER, "plan: moment kernel does not fit");
    L.mom_grid = (int)std::max<int64_t>(1, std::min<int64_t>(E, (int64_t)T.sm_count * per_sm));
    L.split_grid = dwm ? 0 : T.sm_count * std::max(1, moments_split_blocks_per_sm(L.mom_smem));

    // contraction launch shape of the general kernel (a specialised kernel's shape replaces it below)
    if (moments_only) return P2S_OK;
    rc = general_contract_shape(T, E, desc, nc, tile, !spec_n && !ffb, limit, L);
    if (rc) return rc;
    if (ffb) {
        L.ffb = 1;
        L.a_cap = ffl.a_cap;
        L.s1_cap = ffl.s1_cap;
        L.b_cap = ffl.b_cap;
        L.tile_cap = 0;
        L.combo_cap = (size_t)ffl.combos;
        L.tile_off = ffl.smem;
        L.con_smem = ffl.smem;
        L.con_threads = ffl.threads;
        L.con_grid = ffl.grid;
    }

    if (spec_n) {
        int m1n, n1n;
        slab_sizes(desc[0], 0, 0, m1n, n1n, spec_n, tile);
        size_t a, bcap, tl;
        int combos;
        contract_ff_shape(spec_n, m1n, a, bcap, tl, combos);
        // default CTA: one thread per stage-3 combination up to 128 (two combinations per thread
        // beyond); eight 128-thread CTAs per SM keep more barrier groups in flight than four of
        // 256 (c5 at N = 4: 6.89 against 7.88 ms; c2 at N = 6: 27.3 against 28.2 ms)
        const int threads = tile.threads ? tile.threads : std::min(128, std::max(64, (combos + 31) / 32 * 32));
        const size_t smem = (a + bcap) * sizeof(float2);
        const int per_sm = smem <= limit ? contract_ffn_blocks_per_sm(spec_n, threads, smem) : 0;
        if (per_sm < 1) return fail(P2S_ERR_ORDER, "plan: specialised contraction kernel does not fit");
        L.spec_n = spec_n;
        L.a_cap = a;
        L.b_cap = bcap;
        L.tile_cap = 0;
        L.tile_off = smem;
        L.con_smem = smem;
        L.con_threads = threads;
        L.con_grid = T.sm_count * per_sm;
    }
    return P2S_OK;
}

int run_moments(const DeviceTables& T, const PlanLayout& PL, const ElemDesc* d_desc, const p2s_geometry* geom,
                const p2s_material* mat, void* moments, int32_t* elem_status, cudaStream_t s,
                unsigned long long* counter, const int8_t* elem_mask, const int32_t* order, const MomentSplit* split) {
    if (elem_mask && PL.precision != P2S_FP64) return fail(P2S_ERR_ARG, "moments: element masks need an FP64 plan");
    if (split && (PL.precision != P2S_FP64 || elem_status || !split->list || !split->count || !split->part ||
                  split->grid < 1))
        return fail(P2S_ERR_ARG, "moments: split launches need an FP64 plan, an element list and part buffers");
    if (!geom || !mat) return fail(P2S_ERR_ARG, "moments: NULL geometry or material");
    if (geom->n_elem != PL.n_elem) return fail(P2S_ERR_ARG, "moments: n_elem differs from the plan");
    if (PL.n_elem == 0) return P2S_OK;
    if (!moments || !mat->params) return fail(P2S_ERR_ARG, "moments: NULL moments or params");
    if (mat->kind == P2S_ALPHA_SCALAR) {
        if (PL.n_comp != 1) return fail(P2S_ERR_ARG, "moments: scalar coupling needs one component");
    } else if (mat->kind == P2S_ALPHA_METRIC_EPS) {
        if (PL.n_comp != 3 || !geom->nodes) return fail(P2S_ERR_ARG, "moments: metric coupling needs 3 components and nodes");
    } else {
        return fail(P2S_ERR_ARG, "moments: unknown coupling kind");
    }
    MomentLaunch M;
    M.desc = d_desc;
    M.n_elem = PL.n_elem;
    M.kind = mat->kind;
    M.params = mat->params;
    M.nodes = geom->nodes;
    M.bulge = geom->bulge;
    M.gl_x = T.gl_x;
    M.gl_w = T.gl_w;
    M.mom = reinterpret_cast<double*>(moments);
    M.elem_status = elem_status;
    M.err_flag = T.err;
    M.n_pairs = PL.n_pairs;
    M.kb = PL.kb;
    M.gmax = PL.gmax;
    M.iacc_cap = PL.iacc_cap;
    M.out_ff = PL.precision == P2S_MIXED;
    M.elem_mask = elem_mask;
    M.counter = counter;
    M.order = order;
    NvtxRange range(M.out_ff ? "p2s moments a1+a2 (double word)" : "p2s moments a1+a2 (FP64)");
    if (split) {
        P2S_CUDA(launch_moments_fp64_split(M, *split, PL.mom_smem, s));
        return P2S_OK;
    }
    if (counter) P2S_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    if (M.out_ff)
        P2S_CUDA(launch_moments_dw(M, PL.mom_grid, PL.mom_smem, s));
    else
        P2S_CUDA(launch_moments_fp64(M, PL.mom_grid, PL.mom_smem, s));
    return P2S_OK;
}

int run_contract(const DeviceTables& T, const PlanLayout& PL, const ElemDesc* d_desc, const ContractUnit* d_units,
                 unsigned long long* d_counter, const void* moments, double* out, cudaStream_t s,
                 const int8_t* elem_mask, const OpArrays* op) {
    if (elem_mask && (PL.precision != P2S_FP64 || PL.spec_n))
        return fail(P2S_ERR_ARG, "contract: element masks need an FP64 plan");
    if (PL.n_units == 0) return P2S_OK;
    if (!moments || !out) return fail(P2S_ERR_ARG, "contract: NULL moments or out");
    NvtxRange range("p2s contraction a4");
    P2S_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s));
    ContractLaunch C;
    C.desc = d_desc;
    C.units = d_units;
    C.n_units = PL.n_units;
    C.mom = moments;
    C.lin_idx = T.lin_idx;
    C.lin_coef = PL.precision == P2S_MIXED ? (const void*)T.lin_coef_ff : (const void*)T.lin_coef;
    C.out = out;
    C.counter = d_counter;
    C.types_mask = PL.types_mask;
    C.a_cap = (int)PL.a_cap;
    C.b_cap = (int)PL.b_cap;
    C.tile_off = (int)PL.tile_off;
    C.combo_off = (int)contract_combo_offset(PL.precision, PL.a_cap, PL.b_cap, PL.tile_cap);
    C.combo_cap = (int)PL.combo_cap;
    C.s1_cap = (int)PL.s1_cap;
    C.elem_mask = elem_mask;
    C.op_terms = op ? op->terms : nullptr;
    C.op_scales = op ? op->scales : nullptr;
    C.op_block = op ? op->block : nullptr;
    C.op_nalpha = op ? op->nalpha : 0;
    C.out_ff = op ? PL.out_ff : 0;
    if (PL.spec_op)
        P2S_CUDA(launch_contract_opn(PL.spec_op, C, PL.con_grid, PL.con_threads, PL.con_smem, s));
    else if (PL.spec_n)
        P2S_CUDA(launch_contract_ffn(PL.spec_n, C, PL.con_grid, PL.con_threads, PL.con_smem, s));
    else if (PL.ffb)
        P2S_CUDA(launch_contract_ffb(PL.precision, C, PL.con_grid, PL.con_threads, PL.con_smem, s));
    else
        P2S_CUDA(launch_contract(PL.precision, C, PL.con_grid, PL.con_threads, PL.con_smem, s));
    return P2S_OK;
}

}  // namespace p2s

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
    if (G < 1 || G > kMaxG || !x || !w) return fail(P2S_ERR_ARG, "p2s_gauss_legendre: bad G or NULL");
    const HostTables& T = host_tables();
    std::memcpy(x, T.gl_x[G], sizeof(double) * G);
    std::memcpy(w, T.gl_w[G], sizeof(double) * G);
    return P2S_OK;
}

int p2s_linearisation(int t, int m1, int m2, int kmax, double* C) {
    if (t < 0 || t > 3 || m1 < 0 || m2 < 0 || m1 >= kMaxOrder || m2 >= kMaxOrder || kmax < 0 || !C)
        return fail(P2S_ERR_ARG, "p2s_linearisation: bad type, index or NULL");
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
    DeviceTables& D = c->T;
    D.device = device;
    cudaDeviceProp prop;
    P2S_CUDA(cudaGetDeviceProperties(&prop, device));
    D.sm_count = prop.multiProcessorCount;
    D.smem_optin = prop.sharedMemPerBlockOptin;
    const HostTables& T = host_tables();
    size_t glb = sizeof(double) * (kMaxG + 1) * kMaxG;
    P2S_CUDA(cudaMalloc(&D.gl_x, glb));
    P2S_CUDA(cudaMalloc(&D.gl_w, glb));
    P2S_CUDA(cudaMalloc(&D.lin_idx, sizeof(T.lin_idx)));
    P2S_CUDA(cudaMalloc(&D.lin_coef, sizeof(double) * std::max(1, T.n_coef)));
    P2S_CUDA(cudaMalloc(&D.lin_coef_ff, sizeof(float2) * std::max(1, T.n_coef)));
    P2S_CUDA(cudaMalloc(&D.err, sizeof(int)));
    P2S_CUDA(cudaMemcpy(D.gl_x, T.gl_x, glb, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(D.gl_w, T.gl_w, glb, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(D.lin_idx, T.lin_idx, sizeof(T.lin_idx), cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(D.lin_coef, T.lin_coef, sizeof(double) * T.n_coef, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemcpy(D.lin_coef_ff, T.lin_coef_ff, sizeof(float2) * T.n_coef, cudaMemcpyHostToDevice));
    P2S_CUDA(cudaMemset(D.err, 0, sizeof(int)));
    P2S_CUDA(init_kernel_attributes());
    P2S_CUDA(learned_init_attributes());
    D.spec_ok = contract_ff_runs_match(T);
    if (D.spec_ok) P2S_CUDA(contract_ff_upload(T));
    return noalloc_prepare(device);
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
    cudaSetDevice(c->T.device);
    cudaDeviceSynchronize();
    cudaFree(c->T.gl_x);
    cudaFree(c->T.gl_w);
    cudaFree(c->T.lin_idx);
    cudaFree(c->T.lin_coef);
    cudaFree(c->T.lin_coef_ff);
    cudaFree(c->T.err);
    delete c;
}

int64_t p2s_output_entries(int64_t n_elem, const p2s_orders* orders, uint32_t types_mask, int64_t* offsets) {
    int rc = check_orders(n_elem, orders);
    if (rc) return rc;
    if ((types_mask & 0xFu) == 0 || (types_mask & ~0xFu)) return fail(P2S_ERR_ARG, "p2s_output_entries: bad types_mask");
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
    if (p->ctx) cudaSetDevice(p->ctx->T.device);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    cudaFree(p->d_desc);
    cudaFree(p->d_units);
    cudaFree(p->d_counter);
    cudaFree(p->d_order);
    if (p->d_mdesc && p->d_mdesc != p->d_desc) cudaFree(p->d_mdesc);
    cudaFree(p->d_op_terms);
    cudaFree(p->d_op_scales);
    cudaFree(p->d_op_block);
    cudaFree(p->d_mom);
    delete p;
}

int p2s_plan_create(p2s_ctx* ctx, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                    const p2s_fill_opts* opts, p2s_plan** out) {
    return p2s_plan_create_tuned(ctx, E, orders, quad, opts, nullptr, out);
}

int p2s_plan_create_tuned(p2s_ctx* ctx, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                          const p2s_fill_opts* opts, const p2s_tile_config* tile, p2s_plan** out) {
    if (!ctx || !out) return fail(P2S_ERR_ARG, "p2s_plan_create: NULL context or out");
    *out = nullptr;
    if (E < 0) return fail(P2S_ERR_ARG, "p2s_plan_create: negative n_elem");
    TileParams tp;
    int trc = tile_params_from(tile, tp);
    if (trc) return trc;
    if (set_device(ctx->T.device)) return P2S_ERR_CUDA;
    std::vector<ElemDesc> desc((size_t)std::max<int64_t>(E, 1));
    std::vector<ContractUnit> units;
    UnitSink sink;
    sink.vec = &units;
    p2s_plan* p = new (std::nothrow) p2s_plan();
    if (!p) return fail(P2S_ERR_OOM, "p2s_plan_create: host allocation");
    p->ctx = ctx;
    int rc = build_layout(ctx->T, E, orders, quad, opts, desc.data(), sink, p->L, tp);
    if (rc) {
        delete p;
        return rc;
    }
    bool ok = cudaMalloc(&p->d_desc, sizeof(ElemDesc) * desc.size()) == cudaSuccess &&
              cudaMalloc(&p->d_units, sizeof(ContractUnit) * std::max<size_t>(1, units.size())) == cudaSuccess &&
              cudaMalloc(&p->d_counter, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&p->d_mom, sizeof(double) * std::max<int64_t>(1, p->L.mom_entries)) == cudaSuccess;
    if (!ok) {
        p2s_plan_destroy(p);
        return fail(P2S_ERR_OOM, "p2s_plan_create: device allocation");
    }
    cudaError_t ce = cudaMemcpy(p->d_desc, desc.data(), sizeof(ElemDesc) * desc.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && units.size())
        ce = cudaMemcpy(p->d_units, units.data(), sizeof(ContractUnit) * units.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        p2s_plan_destroy(p);
        return fail(P2S_ERR_CUDA, "p2s_plan_create: upload", ce);
    }
    // elements of several quadrature sizes: the moment queue hands them out grouped by G,
    // largest first (concurrent CTAs then run the same specialised code; small ones fill the tail)
    bool mixed_g = false;
    for (int64_t e = 1; e < E && !mixed_g; ++e) mixed_g = desc[e].G != desc[0].G;
    if (mixed_g) {
        std::vector<int32_t> ord((size_t)E);
        for (int64_t e = 0; e < E; ++e) ord[e] = (int32_t)e;
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return desc[a].G > desc[b].G; });
        int32_t* d_ord = plan_order(p);
        ce = d_ord ? cudaMemcpy(d_ord, ord.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice) : cudaErrorMemoryAllocation;
        if (ce != cudaSuccess) {
            p2s_plan_destroy(p);
            return fail(P2S_ERR_CUDA, "p2s_plan_create: element order", ce);
        }
    }
    p->Lm = p->L;
    p->d_mdesc = p->d_desc;
    *out = p;
    return P2S_OK;
}

int64_t p2s_plan_output_entries(const p2s_plan* p) { return p ? p->L.out_entries : P2S_ERR_ARG; }
int64_t p2s_plan_moment_entries(const p2s_plan* p) { return p ? p->Lm.mom_entries : P2S_ERR_ARG; }

int p2s_plan_moments(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* moments,
                     int32_t* elem_status, void* stream) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_moments: NULL plan");
    if (set_device(p->ctx->T.device)) return P2S_ERR_CUDA;
    return run_moments(p->ctx->T, p->Lm, p->d_mdesc, geom, mat, moments, elem_status, (cudaStream_t)stream,
                       p->d_counter + 1, nullptr, p->d_order);
}

int p2s_plan_contract(p2s_plan* p, const double* moments, double* out, void* stream) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_contract: NULL plan");
    if (set_device(p->ctx->T.device)) return P2S_ERR_CUDA;
    OpArrays op{p->d_op_terms, p->d_op_scales, p->d_op_block, p->op_nalpha};
    return run_contract(p->ctx->T, p->L, p->d_desc, p->d_units, p->d_counter, moments, out, (cudaStream_t)stream,
                        nullptr, p->L.op ? &op : nullptr);
}

int p2s_plan_tile_config(const p2s_plan* p, p2s_tile_config* out) {
    if (!p || !out) return fail(P2S_ERR_ARG, "p2s_plan_tile_config: NULL plan or out");
    out->combo_target = p->L.tile.combo_target;
    out->unit_kbytes = (int)(p->L.tile.unit_bytes / 1024);
    out->threads = p->L.con_threads;
    out->kernel = p->L.tile.kernel;
    return P2S_OK;
}

int p2s_plan_use_graph(p2s_plan* p, int enable) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_use_graph: NULL plan");
    if (set_device(p->ctx->T.device)) return P2S_ERR_CUDA;
    if (enable && !p->cap_stream) P2S_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    p->use_graph = enable != 0;
    return P2S_OK;
}

// Capture the plan's launch sequence for these arguments on the private stream and make
// p->gexec replay it (instantiated once, then updated in place when the arguments change).
static int plan_capture(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* out,
                        int32_t* elem_status) {
    cudaStream_t cs = p->cap_stream;
    P2S_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = run_moments(p->ctx->T, p->Lm, p->d_mdesc, geom, mat, p->d_mom, elem_status, cs, p->d_counter + 1, nullptr,
                         p->d_order);
    OpArrays op{p->d_op_terms, p->d_op_scales, p->d_op_block, p->op_nalpha};
    if (rc == P2S_OK)
        rc = run_contract(p->ctx->T, p->L, p->d_desc, p->d_units, p->d_counter, p->d_mom, out, cs, nullptr,
                          p->L.op ? &op : nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_plan_fill: graph capture", ce);
    if (p->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(p->gexec, g, &info) != cudaSuccess) {
            cudaGetLastError();  // an update that does not fit is not an error: instantiate anew
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
    }
    if (!p->gexec) ce = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        p->gexec = nullptr;
        return fail(P2S_ERR_CUDA, "p2s_plan_fill: graph instantiate", ce);
    }
    p->gkey[0] = geom ? geom->nodes : nullptr;
    p->gkey[1] = geom ? geom->bulge : nullptr;
    p->gkey[2] = mat ? mat->params : nullptr;
    p->gkey[3] = out;
    p->gkey[4] = elem_status;
    p->gkey[5] = p->d_mom;
    p->gkind = mat ? mat->kind : -1;
    p->gn = geom ? geom->n_elem : -1;
    return P2S_OK;
}

int p2s_plan_fill(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* out,
                  int32_t* elem_status, void* stream) {
    if (!p) return fail(P2S_ERR_ARG, "p2s_plan_fill: NULL plan");
    if (!out && p->L.n_units) return fail(P2S_ERR_ARG, "p2s_plan_fill: NULL out");
    if (p->use_graph && p->L.n_elem > 0) {
        if (set_device(p->ctx->T.device)) return P2S_ERR_CUDA;
        if (!geom || !mat) return fail(P2S_ERR_ARG, "p2s_plan_fill: NULL geometry or material");
        const bool same = p->gexec && p->gkey[0] == geom->nodes && p->gkey[1] == geom->bulge &&
                          p->gkey[2] == mat->params && p->gkey[3] == out && p->gkey[4] == elem_status &&
                          p->gkind == mat->kind && p->gn == geom->n_elem;
        if (!same) {
            int rc = plan_capture(p, geom, mat, out, elem_status);
            if (rc) return rc;
        }
        P2S_CUDA(cudaGraphLaunch(p->gexec, (cudaStream_t)stream));
        return P2S_OK;
    }
    int rc = p2s_plan_moments(p, geom, mat, p->d_mom, elem_status, stream);
    if (rc) return rc;
    return p2s_plan_contract(p, p->d_mom, out, stream);
}

int p2s_fill_elements(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat, const p2s_orders* orders,
                      const p2s_quadrature* quad, const p2s_fill_opts* opts, double* out, int32_t* elem_status,
                      void* stream) {
    if (!geom) return fail(P2S_ERR_ARG, "p2s_fill_elements: NULL geometry");
    p2s_plan* p = nullptr;
    int rc = p2s_plan_create(ctx, geom->n_elem, orders, quad, opts, &p);
    if (rc) return rc;
    rc = p2s_plan_fill(p, geom, mat, out, elem_status, stream);
    if (rc == P2S_OK) {
        cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
        if (ce != cudaSuccess) rc = fail(P2S_ERR_CUDA, "p2s_fill_elements: stream", ce);
    }
    p2s_plan_destroy(p);
    return rc;
}

int p2s_operator_plan_create(p2s_ctx* ctx, int64_t E, const p2s_orders* orders, const p2s_quadrature* quad,
                             int precision, int kind, const p2s_term* terms, int n_terms,
                             const p2s_tile_config* tile, p2s_plan** out) {
    if (!ctx || !out || !orders || !quad || (n_terms > 0 && !terms)) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: NULL argument");
    *out = nullptr;
    if (E < 0 || n_terms < 1 || n_terms > 4096) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: n_elem < 0 or n_terms outside 1..4096");
    const int nc = orders->n_comp;
    if (nc < 1 || nc > 3 || (E > 0 && !orders->orders)) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: 1..3 field components");
    for (int64_t i = 0; i < E * 3 * nc; ++i)
        if (orders->orders[i] < 1 || orders->orders[i] > kMaxOrder) return fail(P2S_ERR_ORDER, "orders: value outside 1..12");
    if (kind != P2S_ALPHA_SCALAR && kind != P2S_ALPHA_METRIC_EPS) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: bad kind");
    if (precision != P2S_FP64 && precision != P2S_MIXED) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: bad precision");
    const int na = kind == P2S_ALPHA_METRIC_EPS ? 3 : 1;
    for (int k = 0; k < n_terms; ++k) {
        const p2s_term& tm = terms[k];
        bool ok = tm.gi >= 0 && tm.gi < nc && tm.gj >= 0 && tm.gj < nc && tm.sa >= 0 && tm.sa < na && tm.sb >= 0 &&
                  tm.sb < na && std::isfinite(tm.scale);
        for (int x = 0; x < 3; ++x) ok = ok && (tm.d_test[x] == 0 || tm.d_test[x] == 1) && (tm.d_trial[x] == 0 || tm.d_trial[x] == 1);
        if (!ok) return fail(P2S_ERR_ARG, "p2s_operator_plan_create: term out of range");
    }
    TileParams tp;
    int rc = tile_params_from(tile, tp);
    if (rc) return rc;
    if (set_device(ctx->T.device)) return P2S_ERR_CUDA;

    // moments: a virtual element whose na components all have the field's largest order per
    // axis, so every coupling entry (sa, sb) is a moment pair with K = 2 N_max - 1 per axis
    const int nv = na;
    std::vector<int32_t> vord((size_t)std::max<int64_t>(E, 1) * 3 * nv);
    for (int64_t e = 0; e < E; ++e)
        for (int x = 0; x < 3; ++x) {
            int mx = 1;
            for (int g = 0; g < nc; ++g) mx = std::max(mx, (int)orders->orders[(e * nc + g) * 3 + x]);
            for (int g = 0; g < nv; ++g) vord[(e * nv + g) * 3 + x] = mx;
        }
    p2s_orders vo = {nv, vord.data()};
    p2s_fill_opts fo = {precision, 1u};
    std::vector<ElemDesc> mdesc((size_t)std::max<int64_t>(E, 1));
    UnitSink count_only;
    PlanLayout Lm;
    rc = build_layout(ctx->T, E, &vo, quad, &fo, mdesc.data(), count_only, Lm, tp, true);
    if (rc) return rc;

    // contraction: the field's own components and orders, one n x n matrix per element
    std::vector<ElemDesc> cdesc(mdesc);
    int64_t out_off = 0;
    for (int64_t e = 0; e < E; ++e) {
        ElemDesc& d = cdesc[e];
        d.n_comp = (int8_t)nc;
        d.n_types = 1;
        int dof = 0;
        for (int g = 0; g < 3; ++g)
            for (int x = 0; x < 3; ++x) d.ord[g][x] = g < nc ? (int8_t)orders->orders[(e * nc + g) * 3 + x] : 0;
        for (int g = 0; g < nc; ++g) {
            d.dof_off[g] = dof;
            dof += d.ord[g][0] * d.ord[g][1] * d.ord[g][2];
        }
        d.n = dof;
        d.out_off = out_off;
        out_off += (int64_t)dof * dof;
    }
    // terms grouped by block; a list closed under (gi,gj,sa,sb,d,e,scale) -> (gj,gi,sb,sa,e,d,scale)
    // gives M = M^T (alpha is symmetric), so only blocks gi <= gj are computed and the others
    // written as their transposes
    auto packed = [](const p2s_term& tm) {
        const int tu = tm.d_test[0] + 2 * tm.d_trial[0], tv = tm.d_test[1] + 2 * tm.d_trial[1],
                  tw = tm.d_test[2] + 2 * tm.d_trial[2];
        return (int32_t)(tm.sa | (tm.sb << 4) | (tu << 8) | (tv << 12) | (tw << 16));
    };
    std::vector<int32_t> h_terms;
    std::vector<double> h_scales;
    std::vector<int32_t> h_block(18, 0);
    for (int gi = 0; gi < 3; ++gi)
        for (int gj = 0; gj < 3; ++gj) {
            h_block[2 * (3 * gi + gj)] = (int32_t)h_terms.size();
            for (int k = 0; k < n_terms; ++k)
                if (terms[k].gi == gi && terms[k].gj == gj) {
                    h_terms.push_back(packed(terms[k]));
                    h_scales.push_back(terms[k].scale);
                }
            h_block[2 * (3 * gi + gj) + 1] = (int32_t)h_terms.size() - h_block[2 * (3 * gi + gj)];
        }
    std::vector<bool> used((size_t)n_terms, false);
    bool symmetric = true;
    for (int k = 0; k < n_terms && symmetric; ++k) {
        const p2s_term& a = terms[k];
        bool found = false;
        for (int j = 0; j < n_terms && !found; ++j) {
            const p2s_term& b = terms[j];
            if (used[j]) continue;
            const bool alpha_match = (a.sa == b.sb && a.sb == b.sa) || (a.sa == b.sa && a.sb == b.sb && a.sa == a.sb);
            bool m = b.gi == a.gj && b.gj == a.gi && alpha_match && b.scale == a.scale;
            for (int x = 0; x < 3; ++x) m = m && b.d_test[x] == a.d_trial[x] && b.d_trial[x] == a.d_test[x];
            if (m) {
                used[j] = true;
                found = true;
            }
        }
        symmetric = found;
    }
    // one component of uniform order N <= 6, mixed precision: the specialised operator kernel
    // (compile-time runs; units are m1 slabs of at most 256 stage-3 combinations)
    int spec_op = 0;
    if (precision == P2S_MIXED && nc == 1 && E > 0 && ctx->T.spec_ok && !tile) {
        const int N0 = cdesc[0].ord[0][0];
        bool uni = N0 >= 2 && N0 <= contract_opn_max_order();
        for (int64_t e = 0; e < E && uni; ++e)
            for (int x = 0; x < 3; ++x) uni = uni && cdesc[e].ord[0][x] == N0;
        if (uni) spec_op = N0;
    }
    std::vector<ContractUnit> units;
    UnitSink sink;
    sink.vec = &units;
    const int m1s = spec_op ? std::max(1, std::min(spec_op, 256 / (spec_op * spec_op * spec_op))) : 0;
    for (int64_t e = 0; e < E; ++e) {
        if (spec_op) {
            for (int m1a = 0; m1a < spec_op; m1a += m1s) {
                ContractUnit u{};
                u.e = (int32_t)e;
                u.tp = -1;
                u.m1a = (int8_t)m1a;
                u.m1n = (int8_t)std::min(m1s, spec_op - m1a);
                u.n1n = (int8_t)spec_op;
                sink.push(u);
            }
            continue;
        }
        for (int gi = 0; gi < nc; ++gi)
            for (int gj = symmetric ? gi : 0; gj < nc; ++gj)
                push_block(cdesc[e], (int32_t)e, gi, gj, 0, (symmetric && gi != gj) ? 0 : -1, sink, 0, tp);
    }
    PlanLayout L = Lm;  // moment fields for reference; the contraction fields are set below
    L.n_comp = nc;
    L.types_mask = 1u;
    L.out_entries = out_off;
    L.n_units = (int64_t)units.size();
    L.spec_n = 0;
    L.ffb = 0;
    L.op = 1;
    L.a_cap = L.b_cap = L.tile_cap = L.combo_cap = 1;
    const size_t limit = std::min<size_t>(ctx->T.smem_optin, 227 * 1024) - 1024;
    rc = general_contract_shape(ctx->T, E, cdesc.data(), nc, tp, true, limit, L);
    if (rc) return rc;
    if (spec_op) {
        size_t a, bcap, tl;
        int combos;
        contract_ff_shape(spec_op, m1s, a, bcap, tl, combos);
        const int threads = (combos + 31) / 32 * 32;
        const size_t smem = (a + bcap) * sizeof(float2);
        const int per_sm = smem <= limit ? contract_opn_blocks_per_sm(spec_op, threads, smem) : 0;
        if (per_sm >= 1) {
            L.spec_op = spec_op;
            L.a_cap = a;
            L.b_cap = bcap;
            L.tile_cap = 0;
            L.con_smem = smem;
            L.con_threads = threads;
            L.con_grid = ctx->T.sm_count * per_sm;
        } else {  // does not fit: the general kernel's units instead
            units.clear();
            sink.n = 0;
            for (int64_t e = 0; e < E; ++e)
                push_block(cdesc[e], (int32_t)e, 0, 0, 0, -1, sink, 0, tp);
            L.n_units = (int64_t)units.size();
        }
    }

    p2s_plan* p = new (std::nothrow) p2s_plan();
    if (!p) return fail(P2S_ERR_OOM, "p2s_operator_plan_create: host allocation");
    p->ctx = ctx;
    p->L = L;
    p->Lm = Lm;
    p->op_nalpha = na;
    const size_t nd = cdesc.size();
    bool ok = cudaMalloc(&p->d_desc, sizeof(ElemDesc) * nd) == cudaSuccess &&
              cudaMalloc(&p->d_mdesc, sizeof(ElemDesc) * nd) == cudaSuccess &&
              cudaMalloc(&p->d_units, sizeof(ContractUnit) * std::max<size_t>(1, units.size())) == cudaSuccess &&
              cudaMalloc(&p->d_counter, 2 * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&p->d_mom, sizeof(double) * std::max<int64_t>(1, Lm.mom_entries)) == cudaSuccess &&
              cudaMalloc(&p->d_op_terms, sizeof(int32_t) * h_terms.size()) == cudaSuccess &&
              cudaMalloc(&p->d_op_scales, sizeof(double) * h_scales.size()) == cudaSuccess &&
              cudaMalloc(&p->d_op_block, sizeof(int32_t) * h_block.size()) == cudaSuccess;
    if (!ok) {
        p2s_plan_destroy(p);
        return fail(P2S_ERR_OOM, "p2s_operator_plan_create: device allocation");
    }
    cudaError_t ce = cudaMemcpy(p->d_desc, cdesc.data(), sizeof(ElemDesc) * nd, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_mdesc, mdesc.data(), sizeof(ElemDesc) * nd, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && units.size())
        ce = cudaMemcpy(p->d_units, units.data(), sizeof(ContractUnit) * units.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_op_terms, h_terms.data(), sizeof(int32_t) * h_terms.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_op_scales, h_scales.data(), sizeof(double) * h_scales.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_op_block, h_block.data(), sizeof(int32_t) * h_block.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        p2s_plan_destroy(p);
        return fail(P2S_ERR_CUDA, "p2s_operator_plan_create: upload", ce);
    }
    bool mixed_g = false;
    for (int64_t e = 1; e < E && !mixed_g; ++e) mixed_g = mdesc[e].G != mdesc[0].G;
    if (mixed_g) {  // the moment queue grouped by G, largest first (as for ordinary plans)
        std::vector<int32_t> ord((size_t)E);
        for (int64_t e = 0; e < E; ++e) ord[e] = (int32_t)e;
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return mdesc[a].G > mdesc[b].G; });
        int32_t* d_ord = plan_order(p);
        ce = d_ord ? cudaMemcpy(d_ord, ord.data(), sizeof(int32_t) * E, cudaMemcpyHostToDevice) : cudaErrorMemoryAllocation;
        if (ce != cudaSuccess) {
            p2s_plan_destroy(p);
            return fail(P2S_ERR_CUDA, "p2s_operator_plan_create: element order", ce);
        }
    }
    *out = p;
    return P2S_OK;
}

int p2s_sync_status(p2s_ctx* ctx, void* stream) {
    if (!ctx) return fail(P2S_ERR_ARG, "p2s_sync_status: NULL context");
    if (set_device(ctx->T.device)) return P2S_ERR_CUDA;
    P2S_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    P2S_CUDA(cudaMemcpy(&h, ctx->T.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) P2S_CUDA(cudaMemset(ctx->T.err, 0, sizeof(int)));
    return h;
}

int p2s_measure_peaks(p2s_ctx* ctx, int64_t write_bytes, p2s_peaks* out, void* stream) {
    if (!ctx) return fail(P2S_ERR_ARG, "p2s_measure_peaks: NULL context");
    if (set_device(ctx->T.device)) return P2S_ERR_CUDA;
    return measure_peaks(ctx->T, write_bytes, out, (cudaStream_t)stream);
}

int p2s_mode1_product(p2s_ctx* ctx, int method, int G, int slices, const float* x, int64_t n_src, int64_t n_rows,
                      float* out, void* stream) {
    if (!ctx) return fail(P2S_ERR_ARG, "p2s_mode1_product: NULL context");
    if (set_device(ctx->T.device)) return P2S_ERR_CUDA;
    return mode1_product(ctx->T, method, G, slices, x, n_src, n_rows, out, (cudaStream_t)stream);
}

}  // extern "C"

namespace p2s {
const DeviceTables* context_tables(const p2s_ctx* c) { return c ? &c->T : nullptr; }
ElemDesc* plan_desc(p2s_plan* p) { return p ? p->d_desc : nullptr; }
int plan_spec_op(const p2s_plan* p) { return p ? p->L.spec_op : 0; }
unsigned long long* plan_counter(p2s_plan* p) { return p ? p->d_counter : nullptr; }
int plan_run_moments(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, cudaStream_t s) {
    if (!p || !p->L.op) return fail(P2S_ERR_ARG, "plan_run_moments: an operator plan is required");
    if (set_device(p->ctx->T.device)) return P2S_ERR_CUDA;
    return run_moments(p->ctx->T, p->Lm, p->d_mdesc, geom, mat, p->d_mom, nullptr, s, p->d_counter + 1, nullptr,
                       p->d_order);
}
int plan_op_launch(p2s_plan* p, ContractLaunch& C) {
    if (!p || !p->L.op) return fail(P2S_ERR_ARG, "plan_op_launch: an operator plan is required");
    const DeviceTables& T = p->ctx->T;
    const PlanLayout& PL = p->L;
    C = ContractLaunch{};
    C.desc = p->d_desc;
    C.units = p->d_units;
    C.n_units = PL.n_units;
    C.mom = p->d_mom;
    C.lin_idx = T.lin_idx;
    C.lin_coef = PL.precision == P2S_MIXED ? (const void*)T.lin_coef_ff : (const void*)T.lin_coef;
    C.counter = p->d_counter;
    C.types_mask = PL.types_mask;
    C.a_cap = (int)PL.a_cap;
    C.b_cap = (int)PL.b_cap;
    C.op_terms = p->d_op_terms;
    C.op_scales = p->d_op_scales;
    C.op_block = p->d_op_block;
    C.op_nalpha = p->op_nalpha;
    C.out_ff = PL.out_ff;
    return P2S_OK;
}
int plan_set_output_ff(p2s_plan* p, bool on) {
    if (!p || !p->L.op || p->L.precision != P2S_MIXED || p->L.spec_n)
        return fail(P2S_ERR_ARG, "plan_set_output_ff: a mixed-precision operator plan is required");
    p->L.out_ff = on ? 1 : 0;
    p->gkey[3] = nullptr;  // a captured replay has the old setting: capture again on the next fill
    return P2S_OK;
}
int32_t* plan_order(p2s_plan* p) {
    if (!p) return nullptr;
    if (!p->d_order && cudaMalloc(&p->d_order, sizeof(int32_t) * std::max<int64_t>(1, p->L.n_elem)) != cudaSuccess) {
        p->d_order = nullptr;
        return nullptr;
    }
    return p->d_order;
}

int plan_fill_masked(p2s_plan* p, const p2s_geometry* geom, const p2s_material* mat, double* out,
                     const int8_t* mask, cudaStream_t s, const int32_t* list, const int* count, double* part) {
    if (!p) return fail(P2S_ERR_ARG, "plan_fill_masked: NULL plan");
    MomentSplit sp = {list, count, part, p->Lm.split_grid};
    int rc = run_moments(p->ctx->T, p->Lm, p->d_mdesc, geom, mat, p->d_mom, nullptr, s, p->d_counter + 1, mask,
                         p->d_order, list ? &sp : nullptr);
    if (rc) return rc;
    return run_contract(p->ctx->T, p->L, p->d_desc, p->d_units, p->d_counter, p->d_mom, out, s, mask);
}

size_t plan_split_part_doubles(const p2s_plan* p) {
    return p ? moments_split_part_doubles(p->Lm.split_grid, p->Lm.n_pairs, p->Lm.kb) : 0;
}
}  // namespace p2s
