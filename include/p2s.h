/*
 * p2s.h -- C ABI of the GB300 product-to-sum element-matrix fill.
 *
 * Method: E. Khodapanah, "A Product to Sum Approach for Matrix Filling in a
 * Hierarchical Finite-Element Method", arXiv:1703.09619, Sec. II.
 *   Eq. (1)  hierarchical basis A^{mnp}_g = P_m(u) Q_n(v) R_p(w) per field component g;
 *   Eq. (2)  matrix entries as 3-D integrals of basis/derivative products times a
 *            coupling factor alpha (Jacobian and material);
 *   Eq. (3)  product-to-sum (linearisation) of every same-variable product;
 *   Eq. (4)  entries as triple sums of linearisation coefficients times the
 *            "starting-point" moments  I_klq = iiint P_k(u) P_l(v) P_q(w) alpha.
 * This library evaluates Eq. (4) on the GPU: alpha at Gauss-Legendre points,
 * sum-factorised moments, and three sparse mode products that write M.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Basis: Legendre P_m with P_m(1) = 1, m = 0..N-1, on the reference element [-1,1]^3.
 * Product types t (bit t of a types mask):  0 vv, 1 dv, 2 vd, 3 dd, where the first
 *   letter is the test function (row) and the second the trial function (column), "d"
 *   meaning the first derivative on all three axes and "v" the value.
 * Output layout (one element): the selected types in the order vv, dv, vd, dd, each an
 *   n x n row-major FP64 matrix, n = sum_g Nu_g Nv_g Nw_g; dof index = (offset of
 *   component g) + (m Nv_g + n) Nw_g + p, rows = test (g_i, m1, n1, p1), columns = trial
 *   (g_j, m2, n2, p2).  Elements follow each other without padding; element e starts at
 *   entry offsets[e] as returned by p2s_output_entries.
 * Moment layout (one element): the unique component pairs (gi <= gj) in the order
 *   (0,0),(0,1),(0,2),(1,1),(1,2),(2,2) (three components) or (0,0) (one component),
 *   each a row-major Ku x Kv x Kw FP64 tensor, K_axis = N_axis(gi) + N_axis(gj) - 1.
 * Coupling factor kinds (p2s_material.kind), parameters [E][4] FP64:
 *   P2S_ALPHA_SCALAR (one component): p = (A, phi, psi, c),
 *       alpha = 1 + A sin(pi (u + phi)) cos(pi (v + psi)) exp(c w)   (reference coordinates);
 *   P2S_ALPHA_METRIC_EPS (three components): p = (A, kx, ky, kz),
 *       eps(x) = 1 + A sin(k . x),  alpha_{gi gj} = eps detJ (J^-1 J^-T)_{gi gj},
 *       J = dx/d(u,v,w) of the trilinear-plus-bulge map below.
 * Geometry (metric kind): nodes [E][8][3] FP64, node index iu + 2 iv + 4 iw (iu = 0 at
 *   u = -1); bulge [E][4] FP64 = (a, bx, by, bz):
 *       x(u,v,w) = sum_n N_n(u,v,w) X_n + a b cos(pi u/2) cos(pi v/2) cos(pi w/2).
 * Memory: every pointer named "device" is caller-owned device memory, "host" is
 *   caller-owned host memory.  The library never frees caller memory.  Contexts and plans
 *   own the library's own tables and scratch.
 * Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *   Entry points that launch work are asynchronous on that stream; their return value
 *   reports argument and launch errors only.  Device-side errors (detJ <= 0, a wait that
 *   gave up) are written to elem_status (if given) and to a per-context flag that
 *   p2s_sync_status reads.
 * Errors: every int-returning entry point returns P2S_OK (0) or a negative P2S_ERR_* code.
 */
#ifndef P2S_H
#define P2S_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define P2S_OK 0
#define P2S_ERR_ARG (-1)      /* bad pointer, size, kind or mask                         */
#define P2S_ERR_ORDER (-2)    /* an order or quadrature size outside the supported range */
#define P2S_ERR_JACOBIAN (-3) /* detJ <= 0 at a quadrature point of some element          */
#define P2S_ERR_OOM (-4)      /* a library allocation failed                              */
#define P2S_ERR_CUDA (-5)     /* a CUDA runtime call or launch failed                     */
#define P2S_ERR_TIMEOUT (-6)  /* a bounded device wait gave up                            */
#define P2S_ERR_BUFFER (-7)   /* a caller buffer is too small                             */

#define P2S_MAX_ORDER 12 /* N per axis and component: 1..12            */
#define P2S_MAX_NPTS 64  /* Gauss-Legendre points per axis: 1..64       */

#define P2S_ALPHA_SCALAR 0
#define P2S_ALPHA_METRIC_EPS 1

#define P2S_FP64 0  /* every step in FP64                                          */
#define P2S_MIXED 1 /* reduced-precision moments and contraction, FP64 output       */

#define P2S_TYPE_VV 1u
#define P2S_TYPE_DV 2u
#define P2S_TYPE_VD 4u
#define P2S_TYPE_DD 8u
#define P2S_TYPES_ALL 15u

typedef struct p2s_ctx p2s_ctx;
typedef struct p2s_plan p2s_plan;

typedef struct {
    int64_t n_elem;      /* E                                                   */
    const double* nodes; /* device [E][8][3]; may be NULL for P2S_ALPHA_SCALAR  */
    const double* bulge; /* device [E][4];  may be NULL (no bulge)              */
} p2s_geometry;

typedef struct {
    int kind;             /* P2S_ALPHA_SCALAR or P2S_ALPHA_METRIC_EPS */
    const double* params; /* device [E][4]                           */
} p2s_material;

typedef struct {
    int n_comp;            /* 1 (scalar kind) or 3 (metric kind)            */
    const int32_t* orders; /* host [E][n_comp][3] = (Nu, Nv, Nw), 1..12    */
} p2s_orders;

typedef struct {
    int npts_uniform;    /* G for every element, or 0 to use npts[]        */
    const int32_t* npts; /* host [E], each 1..64 (read when npts_uniform=0) */
} p2s_quadrature;

typedef struct {
    int precision;       /* P2S_FP64 or P2S_MIXED        */
    uint32_t types_mask; /* subset of P2S_TYPES_ALL, != 0 */
} p2s_fill_opts;

/* Create a context on CUDA device `device` (uploads the Gauss-Legendre and
 * linearisation tables).  *out receives the context.  Returns P2S_OK,
 * P2S_ERR_ARG, P2S_ERR_CUDA or P2S_ERR_OOM. */
int p2s_create(p2s_ctx** out, int device);

/* Release a context and everything it owns (waits for its device work). */
void p2s_destroy(p2s_ctx* ctx);

/* Output size: total FP64 entries for E elements with the given orders and types
 * (4 n^2 per element for all types).  If offsets (host, E+1) is non-NULL, it
 * receives the first entry of every element and the total.  Returns the total,
 * or a negative P2S_ERR_* code. */
int64_t p2s_output_entries(int64_t n_elem, const p2s_orders* orders, uint32_t types_mask,
                           int64_t* offsets);

/* Moment scratch size: total FP64 moment entries for E elements (layout above).
 * If offsets (host, E+1) is non-NULL it receives the per-element starts. */
int64_t p2s_moment_entries(int64_t n_elem, const p2s_orders* orders, int64_t* offsets);

/* Build a plan: per-element descriptors, the contraction work list and the launch
 * shapes for a batch of E elements with these orders, quadrature sizes and options.
 * A plan is reusable for any geometry/material of the same shape, and owns device
 * scratch for the moments (p2s_plan_moment_entries doubles).  Orders and npts are
 * read only during this call.  Errors: P2S_ERR_ARG, P2S_ERR_ORDER, P2S_ERR_OOM,
 * P2S_ERR_CUDA. */
int p2s_plan_create(p2s_ctx* ctx, int64_t n_elem, const p2s_orders* orders,
                    const p2s_quadrature* quad, const p2s_fill_opts* opts, p2s_plan** out);
void p2s_plan_destroy(p2s_plan* plan);
int64_t p2s_plan_output_entries(const p2s_plan* plan);
int64_t p2s_plan_moment_entries(const p2s_plan* plan);

/* Steps a1+a2 (coupling factor at the G^3 points, Eq. (2); moments of Eq. (4)):
 * writes the moment tensors of every element to `moments` (device, layout above,
 * p2s_plan_moment_entries doubles).  alpha is never stored.  elem_status (device
 * [E], optional) receives 0 or P2S_ERR_JACOBIAN per element. */
int p2s_plan_moments(p2s_plan* plan, const p2s_geometry* geom, const p2s_material* mat,
                     double* moments, int32_t* elem_status, void* stream);

/* Step a4 (Eq. (3)-(4)): M = C^u x1 C^v x2 C^w x3 I for every element, block and
 * selected type, from moment tensors in the layout above; writes `out` (device,
 * p2s_plan_output_entries doubles).  Uses the plan's precision. */
int p2s_plan_contract(p2s_plan* plan, const double* moments, double* out, void* stream);

/* Steps a1-a4 in one call, moments kept in the plan's scratch. */
int p2s_plan_fill(p2s_plan* plan, const p2s_geometry* geom, const p2s_material* mat, double* out,
                  int32_t* elem_status, void* stream);

/* ------------------------------------------------------------------------------------
 * Tile shapes and launch replay of a plan (batches of uneven per-axis orders).  Not part
 * of the paper.  The contraction of step a4 splits each (element, block, type) into work
 * units of m1/n1 slabs that a persistent kernel takes from a queue; these calls choose
 * the unit shape and replay a plan's launches from a CUDA graph.  Neither changes any
 * computed value: every unit shape computes each entry with the same operations in the
 * same order.
 *
 * p2s_tile_config (zero fields take the library default):
 *   combo_target  stage-3 (m1, n1, m2, n2) combinations per work unit: slabs grow until
 *                 they would pass it (default 256; 1..4096);
 *   unit_kbytes   shared memory of one work unit in KiB, stage-1/2 buffers plus the staged
 *                 output tile (general kernel only; default 100; up to 227);
 *   threads       threads per CTA of the contraction, 64..512 in steps of 32 (default:
 *                 one per combination of the largest unit, at most 128 for the kernel
 *                 compiled per uniform order);
 *   kernel        which contraction kernel (every one computes each entry with the same
 *                 operations in the same order):
 *                 0 (default) the library's choice: with every order <= 8 a kernel
 *                   specialised on the coefficient runs (mixed precision with uniform
 *                   orders: one compiled per order; otherwise the bounded-order kernel, in
 *                   either precision), else the general kernel;
 *                 1 the general kernel;
 *                 2 the bounded-order kernel (every order <= 8; plan creation fails with
 *                   P2S_ERR_ORDER otherwise). */
typedef struct {
    int combo_target;
    int unit_kbytes;
    int threads;
    int kernel;
} p2s_tile_config;

/* p2s_plan_create with a tile configuration (NULL: defaults).  Errors as
 * p2s_plan_create; P2S_ERR_ARG for a field out of range, P2S_ERR_ORDER when a unit of
 * the batch does not fit the shared-memory budget. */
int p2s_plan_create_tuned(p2s_ctx* ctx, int64_t n_elem, const p2s_orders* orders,
                          const p2s_quadrature* quad, const p2s_fill_opts* opts,
                          const p2s_tile_config* tile, p2s_plan** out);

/* The tile configuration a plan uses, defaults and the CTA size resolved (host out). */
int p2s_plan_tile_config(const p2s_plan* plan, p2s_tile_config* out);

/* Autotuner: builds a plan per candidate configuration (combo targets 64..512 x budgets
 * 24/48/100 KiB x derived/128/256-thread CTAs with the library's kernel choice, and the
 * bounded-order kernel at each combo target and CTA size) on the first
 * `sample` elements of the batch
 * (<= 0: all), computes their moments once, times `reps` contractions of each candidate
 * with CUDA events on `stream` (median) and writes the fastest to *best (host), its time
 * in ms to *best_ms and the number of candidates that fit to *n_tried (both optional).
 * Synchronises `stream`; allocates device scratch for the sample's moments and output.
 * Geometry, material, orders and quadrature are those of the whole batch (the sample is
 * its leading elements).  Errors: P2S_ERR_ARG, P2S_ERR_OOM, P2S_ERR_CUDA, P2S_ERR_ORDER
 * (no candidate fits). */
int p2s_autotune_tiles(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat,
                       const p2s_orders* orders, const p2s_quadrature* quad,
                       const p2s_fill_opts* opts, int64_t sample, int reps,
                       p2s_tile_config* best, double* best_ms, int* n_tried, void* stream);

/* Replay p2s_plan_fill from a CUDA graph (enable != 0) or launch directly (0, the
 * default).  With replay on, the first fill captures the plan's launch sequence (queue
 * reset, moment kernel, contraction kernel) on a private stream and each later fill
 * launches the captured graph on the caller's stream as one unit; a fill whose
 * geometry, material, out or elem_status pointers or kind differ from the captured ones
 * re-captures and updates the graph in place.  The other plan calls are unaffected. */
int p2s_plan_use_graph(p2s_plan* plan, int enable);

/* ------------------------------------------------------------------------------------
 * Operators given as term lists: Eq. (2) in full generality.  Each term adds to the block
 * (gi, gj) of an element matrix
 *
 *   scale * int P^(d_test[0])_{m1}(u) P^(d_trial[0])_{m2}(u) * (same in v) * (same in w)
 *                 * alpha_{sa sb}(u, v, w) du dv dw
 *
 * (Gauss-Legendre quadrature of the plan's G), so the value/derivative choice may differ per
 * axis and several coupling-factor entries may sum into one matrix.  alpha is the coupling
 * factor of the material kind: P2S_ALPHA_METRIC_EPS gives the 3 x 3 matrix
 * eps detJ J^-1 J^-T (sa, sb < 3, for any number of field components), P2S_ALPHA_SCALAR the
 * scalar (sa = sb = 0).  Example: the diffusion stiffness sum_ab alpha_ab d_a phi_i d_b phi_j
 * of one scalar field is nine terms (a, b) with d_test = e_a, d_trial = e_b.
 * The moments of Eq. (4) are computed once per element for every coupling entry at the
 * element's largest K per axis and shared by all terms; the product-to-sum contraction runs
 * the terms of a block one after the other into one staged tile.  A term list closed under
 * the mirror (gi,gj,sa,sb,d_test,d_trial,scale) -> (gj,gi,sb,sa,d_trial,d_test,scale) gives a
 * symmetric matrix: then only the blocks gi <= gj are computed and written twice.
 * Output per element: one n x n row-major matrix (n = sum_g Nu_g Nv_g Nw_g, rows test dofs,
 * columns trial dofs, dof numbering as above); blocks without terms are zero. */
typedef struct {
    int32_t gi, gj;      /* test / trial field component of the block the term adds to    */
    int32_t sa, sb;      /* coupling-factor entry alpha[sa][sb]                            */
    int32_t d_test[3];   /* derivative order (0 or 1) of the test function on u, v, w      */
    int32_t d_trial[3];  /* derivative order (0 or 1) of the trial function on u, v, w     */
    double scale;
} p2s_term;

/* Plan an operator fill of E elements: orders of the field (1..3 components, host),
 * quadrature, precision (P2S_FP64 or P2S_MIXED), material kind, n_terms terms (host, read
 * during the call), optional tile configuration.  The plan works with p2s_plan_fill,
 * p2s_plan_moments / p2s_plan_contract (moments in the plan's own layout, sized by
 * p2s_plan_moment_entries), p2s_plan_output_entries, p2s_plan_use_graph and
 * p2s_plan_tile_config; the material passed to the fill must have `kind`.  Errors:
 * P2S_ERR_ARG (NULL, term out of range, n_terms outside 1..4096), P2S_ERR_ORDER,
 * P2S_ERR_OOM, P2S_ERR_CUDA. */
int p2s_operator_plan_create(p2s_ctx* ctx, int64_t n_elem, const p2s_orders* orders,
                             const p2s_quadrature* quad, int precision, int kind,
                             const p2s_term* terms, int n_terms, const p2s_tile_config* tile,
                             p2s_plan** out);

/* One-shot fill: plan, fill, release.  Same arguments and errors as the plan calls;
 * `out` must hold p2s_output_entries(...) doubles. */
int p2s_fill_elements(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat,
                      const p2s_orders* orders, const p2s_quadrature* quad,
                      const p2s_fill_opts* opts, double* out, int32_t* elem_status,
                      void* stream);

/* Fill without allocating.  The paper has no counterpart to this entry point: it
 * computes exactly what p2s_fill_elements computes, and only moves the fill's scratch
 * (moments, element descriptors, work list, queue counter) into one fixed array of
 * 18.3 MiB that the library reserves in device memory on every GPU that loads it, for
 * the life of the process.  It is meant for callers that must not call cudaMalloc or
 * cudaFree while they run -- for instance a solver whose own memory pool has taken all
 * free device memory, a service held to a fixed device-memory budget, or a loop that
 * cannot pay for the synchronisation an allocation or free may trigger.  Such a caller
 * creates the context once beforehand (p2s_create allocates its small tables).
 *   Arguments, layouts and results are those of p2s_fill_elements; `out` (device) and
 *   `elem_status` (device, optional) are caller-owned.  The call is asynchronous on
 *   `stream` (it does not synchronise, unlike p2s_fill_elements).
 *   Limits per call: at most 2048 elements, 2,097,152 moment entries and 131,072
 *   contraction work units; larger requests return P2S_ERR_BUFFER with a message in
 *   p2s_last_error and launch nothing -- split the batch.  (Three-component N = 6
 *   elements fit 262 per call, N = 4 elements 1019.)
 *   Set-up: p2s_create looks up the array's device address for its device (that look-up
 *   may load the library's module for the array, which places the array in device
 *   memory), so this call itself loads nothing and allocates nothing.
 *   Sharing: every call uses the same array, which keeps the previous call's contents
 *   (each call rewrites what it reads, and clears its counter).  Calls whose kernels
 *   overlap on the GPU -- on different streams or from different threads without
 *   ordering -- race on the array and give wrong results; order them on one stream.
 *   It calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: as p2s_fill_elements, plus P2S_ERR_BUFFER. */
int p2s_fill_elements_noalloc(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat,
                              const p2s_orders* orders, const p2s_quadrature* quad,
                              const p2s_fill_opts* opts, double* out, int32_t* elem_status,
                              void* stream);

/* ------------------------------------------------------------------------------------
 * Learned quadrature order.  Not part of the paper: a small network picks, per element,
 * the Gauss-Legendre size G of the fill (Eq. (2)-(4)); a seeded share of the elements is
 * re-filled at 48 points (in the learned fill's precision) to judge the choice, and judged
 * elements that miss the tolerance are replaced by their 48-point FP64 fill (the plain
 * method).  Three-component metric coupling only.
 *
 * Network: 576 inputs (alpha on the 4 x 4 x 4 grid with per-axis reference positions
 * {-0.9, -0.8, 0.35, 0.45}, all 9 factors alpha_{gi gj}, point index (c*4 + b)*4 + a,
 * factor index 3 gi + gj, divided by the element's mean of trace(alpha)/3) -> 64 -> 64 -> 6 classes, ReLU, weights used in
 * FP16 with FP32 accumulation.  Class c means G = {8, 12, 16, 24, 32, 48}[c].
 * Parameters: one FP32 device array of P2S_MLP_PARAMS values in the order
 * W1 [576][64], b1 [64], W2 [64][64], b2 [64], W3 [64][6], b3 [6] (W[i][j]: input i to
 * output j). */
#define P2S_MLP_IN 576
#define P2S_MLP_HIDDEN 64
#define P2S_MLP_CLASSES 6
#define P2S_MLP_PARAMS 41478
#define P2S_MLP_MAX_NETS 8  /* networks of an ensemble */

/* G of class cls (0..5), or P2S_ERR_ARG. */
int p2s_learned_npts(int cls);

/* The 576 features of every element (device [E][576] FP32). */
int p2s_coarse_features(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat, float* features,
                        void* stream);

/* Inference: npts (device [n]) = G of the chosen class + margin (capped at class 5);
 * logits (device [n][6], optional).  The chosen class is the argmax when risk = 0, else the
 * smallest class c whose higher classes c+1..5 hold at most `risk` (0 < risk < 1) of the
 * softmax probability. */
int p2s_mlp_predict(p2s_ctx* ctx, const float* params, const float* features, int64_t n, int margin, float risk,
                    int32_t* npts, float* logits, void* stream);

/* Inference by an ensemble of n_nets (1..P2S_MLP_MAX_NETS) networks, whose parameter sets
 * follow one another in params (device [n_nets][P2S_MLP_PARAMS]).  A sample's class
 * probabilities are the mean of the networks' softmax outputs; the class is chosen from
 * them as in p2s_mlp_predict (argmax, or the risk rule), then `margin` is added.  With
 * n_nets > 1, logits (device [n][6]) is required: it holds the running sums and receives the
 * log of the mean probabilities.  n_nets = 1 is p2s_mlp_predict. */
int p2s_mlp_predict_ensemble(p2s_ctx* ctx, const float* params, int n_nets, const float* features, int64_t n,
                             int margin, float risk, int32_t* npts, float* logits, void* stream);

/* Training step, forward and backward on `batch` samples: mean softmax cross-entropy
 * (each sample weighted by class_weight[label], device [6], optional) into *loss (device)
 * and its gradient with respect to the FP32 parameters into grad (device
 * [P2S_MLP_PARAMS]); both are overwritten.  The forward uses the FP16-rounded weights of
 * inference; the gradient passes the rounding straight through. */
int p2s_mlp_grad(p2s_ctx* ctx, const float* params, const float* features, const int32_t* labels, int64_t batch,
                 const float* class_weight, float* grad, float* loss, void* stream);

/* Adam update (Kingma & Ba) with decoupled weight decay (AdamW) of n FP32 parameters in
 * place; m, v are the moment buffers (device, start at 0), step counts from 1. */
int p2s_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                 float beta2, float eps, float weight_decay, int step, void* stream);

/* err[k] (device [n]) = max over the n_types product types of max|a - b| / max|b| over
 * element k's matrices, a starting at offsets_a[k] and b at offsets_b[k]..offsets_b[k+1]
 * (device arrays, offsets_b of length n+1); max|a - b| itself where b is zero throughout.
 * A NaN in either array makes err[k] NaN, which no tolerance accepts.  Used for the labels
 * and by the judge. */
int p2s_element_errors(p2s_ctx* ctx, const double* a, const int64_t* offsets_a, const double* b,
                       const int64_t* offsets_b, int64_t n, int n_types, double* err, void* stream);

/* Seeded judge selection (host): judged[e] = 1 for the elements re-filled by the judge.
 * Element e is chosen when splitmix64(seed + e * 0x9e3779b97f4a7c15) < frac * 2^64. */
int p2s_judge_select(int64_t n_elem, double frac, uint64_t seed, int8_t* judged);

typedef struct p2s_learned_plan p2s_learned_plan;
typedef struct {
    int margin;        /* classes added to every prediction (0: as predicted)      */
    double risk;       /* 0: argmax; else the risk rule of p2s_mlp_predict          */
    int precision;     /* precision of the learned fill: P2S_MIXED or P2S_FP64     */
    double judge_frac; /* share of elements re-filled at 48 points in FP64          */
    uint64_t seed;     /* judge selection seed                                     */
    double judge_tol;  /* largest accepted relative difference (metric of p2s_element_errors) */
    int n_nets;        /* networks in the parameters of p2s_learned_fill (0 or 1: one; up to
                          P2S_MLP_MAX_NETS: an ensemble, p2s_mlp_predict_ensemble)          */
} p2s_learned_opts;
typedef struct {
    int64_t n_elem;
    int64_t judged;            /* elements re-filled by the judge                   */
    int64_t failed;            /* judged elements above judge_tol, replaced         */
    int64_t per_class[6];      /* elements filled with each G class                 */
    double max_judged_err;     /* largest relative difference the judge saw         */
} p2s_learned_report;

/* Plan a learned fill of E elements (three components, host orders, all four types).
 * Allocates the fill's scratch, the judge subset, its 48-point plan and its 48-point FP64
 * fallback plan. */
int p2s_learned_plan_create(p2s_ctx* ctx, int64_t n_elem, const p2s_orders* orders, const p2s_learned_opts* opts,
                            p2s_learned_plan** out);
void p2s_learned_plan_destroy(p2s_learned_plan* plan);
int64_t p2s_learned_plan_output_entries(const p2s_learned_plan* plan);

/* Learned fill, asynchronous on `stream`: features, prediction, fill at the predicted G,
 * judge fill at 48 points and comparison, FP64 fill of the judged elements that failed and
 * their replacement in `out` (when few fail, each one's moment sums over w-planes are split
 * over several CTAs and added in a fixed order: the FP64 48-point fill up to rounding).  npts_out (device [E], optional) receives the G used per
 * element before any replacement.  The judge's 48-point fill, which does not depend on the
 * prediction, runs on a stream of the plan that is forked from `stream` when the call
 * starts and joined to it before the comparison: work queued on `stream` after the call
 * sees the whole fill.  Calls with one plan must be ordered (one stream, or synchronised). */
int p2s_learned_fill(p2s_learned_plan* plan, const p2s_geometry* geom, const p2s_material* mat, const float* params,
                     double* out, int32_t* npts_out, void* stream);

/* Wait for `stream` and read the last learned fill's report; judge_state (host [E],
 * optional) receives 0 (not judged), 1 (judged, kept) or 2 (judged, replaced). */
int p2s_learned_report_get(p2s_learned_plan* plan, p2s_learned_report* report, int8_t* judge_state, void* stream);

/* ------------------------------------------------------------------------------------
 * Global assembly on a conforming structured mesh (the "total" step after the fill,
 * Sec. V).  The mesh has nx x ny x nz hexahedra, element (i, j, k) at (k ny + j) nx + i, and
 * shares vertices with its lattice neighbours (geometry: its 8 corners in the order of
 * p2s_geometry); one scalar field of order N on every axis.  The element matrices of the
 * fill (Legendre basis) are changed to the hierarchic C0 basis
 *   l_0 = (P_0 - P_1)/2, l_1 = (P_0 + P_1)/2, l_k = (P_k - P_{k-2}) / sqrt(2 (2k - 1)),
 * (vertex functions of u = -1 and +1, then integrated-Legendre bubbles) and summed into one
 * global CSR matrix.  Axis dof numbering: vertex i (0..n_el), then bubble k of interval i at
 * n_el + 1 + i (N - 2) + k - 2; global dof (gu Ngv + gv) Ngw + gw, Ng = n_el (N - 1) + 1.
 * Row r holds the columns coupled to r in increasing order.  The sums are deterministic:
 * elements are added in 8 colours of lattice parity, so within one colour every position
 * receives at most one addition.  A mixed-precision assembly (N <= 5) keeps the fill's
 * float-float values through the basis change and rounds each to FP64 once before adding. */
typedef struct p2s_assembly p2s_assembly;

/* CSR structure of the global matrix (host, no device needed): *rows, *nnz, and, where
 * non-NULL, row_ptr [rows + 1] and col_idx [nnz] (caller-owned host arrays).  Errors:
 * P2S_ERR_ARG (a mesh size < 1, N outside 2..12, or 2^31 rows or more). */
int p2s_assembly_structure_host(int nx, int ny, int nz, int order, int64_t* rows, int64_t* nnz,
                                int64_t* row_ptr, int32_t* col_idx);

/* Plan the assembly: an operator plan of the mesh's elements (npts-point rule, precision,
 * material kind, n_terms terms of field component 0, host, read during the call), the CSR
 * row pointers and 1-D rank tables on the device, and scratch for the element matrices
 * (E N^6 doubles; none on the fused path, see p2s_assembly_fused).  Errors: as
 * p2s_operator_plan_create and p2s_assembly_structure_host. */
int p2s_assembly_create(p2s_ctx* ctx, int nx, int ny, int nz, int order, int npts, int precision,
                        int kind, const p2s_term* terms, int n_terms, p2s_assembly** out);
void p2s_assembly_destroy(p2s_assembly* A);
int64_t p2s_assembly_rows(const p2s_assembly* A);
int64_t p2s_assembly_nnz(const p2s_assembly* A);
/* Replay the element fill of p2s_assembly_fill from a CUDA graph (as p2s_plan_use_graph; no
 * effect on the fused path). */
int p2s_assembly_use_graph(p2s_assembly* A, int enable);

/* 1 if the assembly runs fused: mixed precision, N <= 4, where each element's matrix goes from the
 * operator contraction's registers through the basis change into the CSR values in one kernel
 * (launched per colour), with no element-matrix scratch; 0 for the two-step path (fill into E N^6
 * doubles of scratch, then the assembly kernel); P2S_ERR_ARG for NULL. */
int p2s_assembly_fused(const p2s_assembly* A);

/* Add element matrices to a global matrix: emat (device [E][n][n], n = N^3, Legendre basis,
 * row-major, element order above; read only) is changed to the hierarchic basis and added
 * into values (device, p2s_assembly_nnz doubles, CSR order above; not zeroed first).  emat
 * may be the output of any fill with these orders (one field component).  Asynchronous on
 * `stream`; uses the assembly's scratch, so calls on one assembly must not overlap.
 * Errors: P2S_ERR_ARG (NULL), P2S_ERR_CUDA. */
int p2s_assembly_add(p2s_assembly* A, const double* emat, double* values, void* stream);

/* Fill the element matrices (device inputs as for p2s_plan_fill, E elements) and assemble:
 * values (device, p2s_assembly_nnz doubles) is overwritten with the global matrix in the
 * CSR order above.  Asynchronous on `stream`; Jacobian failures set the context's error
 * flag (p2s_sync_status).  Errors: P2S_ERR_ARG, P2S_ERR_CUDA, those of p2s_plan_fill. */
int p2s_assembly_fill(p2s_assembly* A, const p2s_geometry* geom, const p2s_material* mat,
                      double* values, void* stream);

/* Assemble the element matrices of the most recent p2s_assembly_fill on this assembly again:
 * values (device, p2s_assembly_nnz doubles) is overwritten.  Stream-ordered after that fill.  On
 * the fused path the element matrices are formed again from the moments the fill kept.
 * Errors: P2S_ERR_ARG, P2S_ERR_CUDA. */
int p2s_assembly_reassemble(p2s_assembly* A, double* values, void* stream);

/* ------------------------------------------------------------------------------------
 * The paper's 2-D example (Sec. III): stiffness and mass element matrices of the curl-curl
 * equation (Eq. (5)) on curved quadrilaterals, curl-conforming Chebyshev basis (Eq. (6))
 *   E_u = U_m(u) T_n(v) (m < M, n <= N), E_v = T_m(u) U_n(v) (m <= M, n < N),
 * S and M of Eq. (7)-(15) with mu_r = 1.  Geometry (Fig. 1): element e is the image of the
 * cell [s_lo, s_hi] x [t_lo, t_hi] under X(s, t) = (s g(t), t f(s)), f(x) = 1 - 0.2 (x^2 - 1)^2,
 * g(y) = 1 + 0.2 (y^2 - 1)^2; params (device [E][5]) = (s_lo, s_hi, t_lo, t_hi, filled), and
 * eps_r = 2 exp(x + y + 2) where filled != 0, else 1.  Dofs per element: n = M (N+1) + (M+1) N,
 * the E_u functions (m, n) at m (N+1) + n, then the E_v functions at M (N+1) + m N + n.  S and Mass
 * (device, caller-owned, [E][n][n] row-major each, rows = testing functions) are overwritten.
 * method P2S_CHEB2D_P2S: the product-to-sum fill (Eq. (16)-(19)): four moment sets per element
 * then every entry as a signed sum of four moments; P2S_CHEB2D_DIRECT: direct numerical
 * integration of every entry over the npts x npts Gauss-Legendre points (the paper's
 * comparison method).  Both use the same rule, so they agree to rounding.  precision: P2S_FP64,
 * or P2S_MIXED for the product-to-sum method (moments and v-axis sums in FP64, each entry formed
 * in double-word FP32 arithmetic and rounded to FP64 once: relative error ~1e-14).  Asynchronous
 * on `stream`; J <= 0 at a point sets the context's error flag (p2s_sync_status).  Errors:
 * P2S_ERR_ARG (NULL, method, precision), P2S_ERR_ORDER (M, N outside 1..24, npts outside 1..48),
 * P2S_ERR_CUDA. */
#define P2S_CHEB2D_MAX_ORDER 24
#define P2S_CHEB2D_MAX_NPTS 48
#define P2S_CHEB2D_P2S 0
#define P2S_CHEB2D_DIRECT 1
int64_t p2s_cheb2d_dofs(int M, int N);
int p2s_cheb2d_fill(p2s_ctx* ctx, int64_t n_elem, const double* params, int M, int N, int npts, int method,
                    int precision, double* S, double* Mass, void* stream);

/* Wait for `stream`, then return and clear the context's device error flag:
 * P2S_OK, P2S_ERR_JACOBIAN, P2S_ERR_TIMEOUT, or P2S_ERR_CUDA if the stream failed. */
int p2s_sync_status(p2s_ctx* ctx, void* stream);

/* Host copies of the library's tables (for inspection and tests).
 * p2s_linearisation: C[0..kmax] with P^{(d1)}_{m1} P^{(d2)}_{m2} = sum_k C[k] P_k for
 *   type t (d1 = t&1, d2 = t>>1), Eq. (3); Adams-Neumann products plus the expansion
 *   P'_m = sum_{j=m-1,m-3,..} (2j+1) P_j.  Entries beyond the product's degree are 0.
 * p2s_gauss_legendre: the G-point rule the kernels use (x ascending). */
int p2s_linearisation(int t, int m1, int m2, int kmax, double* C);
int p2s_gauss_legendre(int G, double* x, double* w);

/* Device throughput probes.  The paper measures on a CPU and has no counterpart; these
 * are the denominators of the roofline fractions that a fill's kernels are reported
 * against (FP64 pipe, FP32 pipe, store-only HBM stream).
 *   fp64_fma_tflops / fp32_fma_tflops: independent FMA chains on 2048 threads per SM,
 *     2 flop per FMA, best of 5 timed launches (CUDA events) after one warm-up launch;
 *   hbm_write_gbs: 16-byte streaming stores over a device buffer of write_bytes
 *     (>= 1 MiB; use several times the L2 size), best of 5.
 * fp32_ms, fp64_ms, write_ms: the kept launch times; write_bytes: the buffer used.
 * The call allocates and frees a device buffer of write_bytes, runs on `stream` and
 * synchronises it.  Errors: P2S_ERR_ARG, P2S_ERR_OOM, P2S_ERR_CUDA. */
typedef struct {
    double fp64_fma_tflops;
    double fp32_fma_tflops;
    double hbm_write_gbs;
    double fp64_ms, fp32_ms, write_ms;
    int64_t write_bytes;
} p2s_peaks;
int p2s_measure_peaks(p2s_ctx* ctx, int64_t write_bytes, p2s_peaks* out, void* stream);

/* First mode product of the sum-factorised moments (Eq. (4): the a-axis sum of the
 * starting-point integrals) on rows of double-word samples, by one of two methods; a
 * measurement of the tensor-core form against the SIMT form on the same work (the fill's
 * moment kernel uses the SIMT form, fused with the coupling factor).
 *   T[r][k] = sum_{a<G} B[k][a] x[r][a],  B[k][a] = w_a P_k(u_a) (the G-point
 *   Gauss-Legendre rule of the fill), k < 7 (order 4).
 * method: P2S_MODE1_SIMT -- parity fold and double-word dot products (FP32 pipe);
 *         P2S_MODE1_TC   -- parity fold, per-row power-of-two scaling, `slices` (4 or 5)
 *           8-bit integer slices of the samples and of B in FP16, tcgen05.mma with FP32
 *           accumulation in tensor memory (exact: every level sum is an integer below
 *           2^24), level sums recombined into a double word; error about 2^(-8 slices)
 *           of max|B| max|x| per term.
 * x: device, n_src rows of G (hi, lo) FP32 pairs ([n_src][G][2] floats); row r of the
 *    product reads source row r mod n_src.  G in {8, 12, 16, 24, 32, 48}.
 * out: device, [n_rows][8][2] floats: T[r][k] as (hi, lo) for k < 7, slot 7 zero.
 * Synchronises `stream`.  A tensor-core wait that exceeds its clock budget sets the
 * context's flag to P2S_ERR_TIMEOUT (p2s_sync_status).  Errors: P2S_ERR_ARG,
 * P2S_ERR_ORDER, P2S_ERR_CUDA. */
#define P2S_MODE1_SIMT 0
#define P2S_MODE1_TC 1
int p2s_mode1_product(p2s_ctx* ctx, int method, int G, int slices, const float* x, int64_t n_src, int64_t n_rows,
                      float* out, void* stream);

/* Static description of an error code. */
const char* p2s_error_string(int code);

/* Text of the most recent failure recorded on the calling host thread (the CUDA call
 * and its error, or the argument check that failed); "" if none.  The pointer stays
 * valid until the thread's next failing call. */
const char* p2s_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* P2S_H */
