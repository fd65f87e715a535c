// Autotuner of the contraction's tile configuration (the launch shape of step a4, the
// product-to-sum contraction of Eq. (4) of arXiv:1703.09619).
//
// The contraction splits each (element, block, type) into work units of m1/n1 slabs.  How
// many stage-3 combinations a unit holds, how much shared memory it may stage and how many
// threads a CTA has trade occupancy against barrier count and redundant stage-1/2 work, and
// the best point depends on the batch's order mix; the kernel itself is a candidate too (the
// library's choice or the bounded-order kernel).  The tuner builds one plan per candidate
// on a leading sample of the batch, computes the sample's moments once (the moment layout
// does not depend on the tiles), times each candidate's contraction with CUDA events on the
// caller's stream and returns the fastest.  Every candidate computes the same entries with
// the same arithmetic in the same order, so the choice changes speed, never results.
// Built on the public entry points only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "p2s.h"

namespace {

struct Candidate {
    int combo, kbytes, threads, kernel;
};

// combo targets x shared-memory budgets, each with the derived CTA size (one thread per
// combination of the largest unit) and with fixed 128- and 256-thread CTAs, with the library's
// kernel choice, and the bounded-order kernel (no shared-memory tile, so no budget) at each
// combo target and CTA size
std::vector<Candidate> candidates() {
    std::vector<Candidate> c;
    const int combos[] = {64, 128, 256, 512};
    const int kbytes[] = {24, 48, 100};
    const int threads[] = {0, 128, 256};
    for (int co : combos)
        for (int kb : kbytes)
            for (int th : threads) c.push_back({co, kb, th, 0});
    for (int co : combos)
        for (int th : threads) c.push_back({co, 0, th, 2});
    return c;
}

}  // namespace

extern "C" int p2s_autotune_tiles(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat,
                                  const p2s_orders* orders, const p2s_quadrature* quad, const p2s_fill_opts* opts,
                                  int64_t sample, int reps, p2s_tile_config* best, double* best_ms, int* n_tried,
                                  void* stream) {
    if (!ctx || !geom || !mat || !orders || !quad || !opts || !best) return P2S_ERR_ARG;
    if (geom->n_elem <= 0 || reps < 1 || reps > 100) return P2S_ERR_ARG;
    const int64_t S = (sample <= 0 || sample > geom->n_elem) ? geom->n_elem : sample;
    p2s_geometry g = *geom;
    g.n_elem = S;  // the leading S elements: the same pointers, a shorter batch
    cudaStream_t s = (cudaStream_t)stream;

    p2s_plan* base = nullptr;
    int rc = p2s_plan_create(ctx, S, orders, quad, opts, &base);
    if (rc) return rc;
    const int64_t n_out = p2s_plan_output_entries(base), n_mom = p2s_plan_moment_entries(base);
    double *mom = nullptr, *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = cudaMalloc(&mom, sizeof(double) * std::max<int64_t>(1, n_mom)) == cudaSuccess &&
              cudaMalloc(&out, sizeof(double) * std::max<int64_t>(1, n_out)) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (!ok) rc = P2S_ERR_OOM;
    if (!rc) rc = p2s_plan_moments(base, &g, mat, mom, nullptr, stream);
    p2s_plan_destroy(base);

    double best_t = 1e300;
    int tried = 0;
    for (const Candidate& c : candidates()) {
        if (rc) break;
        p2s_tile_config cfg{c.combo, c.kbytes, c.threads, c.kernel};
        p2s_plan* p = nullptr;
        if (p2s_plan_create_tuned(ctx, S, orders, quad, opts, &cfg, &p) != P2S_OK) continue;  // does not fit
        int r = p2s_plan_contract(p, mom, out, stream);  // warm-up
        std::vector<float> ts;
        for (int i = 0; i < reps && r == P2S_OK; ++i) {
            cudaEventRecord(e0, s);
            r = p2s_plan_contract(p, mom, out, stream);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = P2S_ERR_CUDA;
            ts.push_back(ms);
        }
        if (r == P2S_OK) {
            std::sort(ts.begin(), ts.end());
            const double t = ts[ts.size() / 2];
            ++tried;
            if (t < best_t) {
                best_t = t;
                p2s_plan_tile_config(p, best);  // the configuration in effect, threads resolved
            }
        } else {
            rc = r;
        }
        p2s_plan_destroy(p);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(mom);
    cudaFree(out);
    if (rc) return rc;
    if (tried == 0) return P2S_ERR_ORDER;
    if (best_ms) *best_ms = best_t;
    if (n_tried) *n_tried = tried;
    return P2S_OK;
}
