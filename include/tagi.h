/*
 * tagi.h -- C ABI of the treecode-accelerated Green Iteration hot path
 * (arXiv:2003.01833): the discrete convolution sums of Green Iteration with
 * the modified-Helmholtz (Yukawa) kernel and the Coulomb kernel, both with
 * singularity subtraction, evaluated by a barycentric Lagrange treecode.
 *
 * Conventions shared by every entry point
 *   - Pointers marked [dev] are CUDA device pointers, [host] are host
 *     pointers.  The caller owns every buffer it passes; the library never
 *     frees or keeps them, except that tagi_tree_build copies xyz and w.
 *   - Point arrays are in the caller's order.  Coordinates are structure of
 *     arrays: xyz[0..n) = x, xyz[n..2n) = y, xyz[2n..3n) = z, all float64.
 *     Field arrays are row-major (nf, n) float64.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).  Entry points that return host values
 *     (tagi_green_step, tagi_tree_info) synchronise the stream.
 *   - No exception crosses the ABI.  Every call returns a tagi_status; on
 *     failure tagi_last_error() gives a message (thread-local, valid until
 *     the next call on the same thread).
 *   - Kernel convention: G_k(r) = exp(-k r) / (4 pi r), so the paper's
 *     Green's function (Eq. Hemlholtz_Greens_Function) is -2 G_k with
 *     k = sqrt(-2 eps); G_C(r) = 1 / r (Eq. Coulomb).
 */
#ifndef TAGI_H
#define TAGI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TAGI_OK = 0,
    TAGI_ERR_INVALID_ARG = 1, /* a size, parameter or input value is out of range */
    TAGI_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    TAGI_ERR_OOM = 3,         /* device or host allocation failed */
    TAGI_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    TAGI_ERR_STATE = 5        /* the object is not in a state that allows the call */
} tagi_status;

typedef enum {
    TAGI_FP64 = 0,  /* plain form: every sum and every kernel value in float64 */
    TAGI_FP32C = 1  /* float32 kernel sums, per-target two-float (compensated)
                       accumulation, float64 singularity-subtraction epilogue */
} tagi_precision;

/* Treecode parameters (Section 5; Eq. MAC; Algorithm 3) and one tile shape
 * of the near/far kernel.
 *   theta      MAC parameter, 0 <= theta < 1.  theta = 0 never approximates,
 *              so the treecode reduces to the direct sum of Eq. direct-sum.
 *   degree     interpolation degree n, 1 <= n <= 9; (n+1)^3 proxies per cluster.
 *   leaf_size  maximum leaf size N_L >= 1.
 *   batch_size maximum batch size N_B; must equal leaf_size (the batches are
 *              the leaves, Section 5.1) or be 0 (taken as leaf_size).
 *   prec       TAGI_FP64 or TAGI_FP32C.
 *   ss         1: singularity subtraction (Eq. yukawa-conv-ss, coulomb-conv-ss); 0: none.
 *   alpha      Gaussian width of the Coulomb subtraction (Eq. coulomb-conv-ss), > 0.
 *   segment    sources per work item of the near/far kernel (a batch's 256
 *              targets against a run of its interaction list), 1024 <= segment
 *              <= 65536, or 0 for 8192.  Longer segments mean fewer partial
 *              sums, shorter ones a finer balance of the work; the float32
 *              sums of the FP32C form are grouped by segment. */
typedef struct {
    double theta;
    int degree;
    int leaf_size;
    int batch_size;
    int prec;
    int ss;
    double alpha;
    int segment;
} tagi_params;

typedef struct tagi_tree tagi_tree; /* opaque, owned by the library */

/* Sizes of a built tree (host struct filled by tagi_tree_info). */
typedef struct {
    int64_t n_points;
    int32_t n_clusters;
    int32_t n_leaves;       /* = number of target batches */
    int32_t depth;          /* number of levels below the root */
    int32_t n_far_clusters; /* clusters approximated by at least one batch */
    int64_t n_list_entries; /* batch-cluster entries after near-field leaf expansion */
    int64_t n_items;        /* work items of the near/far kernel */
    int64_t near_pairs;     /* sum over batches |B| * (sources in near entries) */
    int64_t far_pairs;      /* sum over batches |B| * (proxies in far entries) */
    int32_t degree;         /* interpolation degree n */
    int32_t n_proxies;      /* (n+1)^3 proxies per cluster */
    int64_t near_pairs_nogauss; /* near pairs in entries whose boxes are >= sqrt(42) alpha apart */
    int64_t far_pairs_nogauss;  /* far pairs likewise: there exp(-r^2/alpha^2) <= 2^-60 */
    int64_t ant_points;         /* sum over approximated clusters of their points (anterpolation work) */
} tagi_tree_stats;

/* Build the source-cluster tree and target batches (Algorithm 3 line 1,
 * Section 5.1), the per-batch interaction lists of Algorithm 3's
 * ComputePotential under the MAC of Eq. MAC, the proxy grid of every cluster
 * that some batch approximates (Chebyshev points of the second kind,
 * Section 5.2) and the anterpolated quadrature weights w^ of those clusters.
 *   xyz [dev] 3*n float64, w [dev] n float64 (quadrature weights, finite).
 *   n >= 1.  params [host].  out [host] receives the new tree.
 * Tree rules where the paper is silent: root = minimal bounding box; a
 * cluster is a leaf iff it holds <= leaf_size points; the dimensions split
 * are those whose extent e satisfies e*sqrt(2) >= the largest extent; the cut
 * is at (lo+hi)*0.5 of the shrunk box, a point with x >= mid goes up; empty
 * children are dropped.  Errors: TAGI_ERR_INVALID_ARG for n < 1, bad params,
 * non-finite xyz or w, or a tree deeper than 64 levels. */
tagi_status tagi_tree_build(const double* xyz, const double* w, int64_t n, const tagi_params* params,
                            void* stream, tagi_tree** out);

/* Free the tree and every device buffer it owns.  NULL is accepted. */
tagi_status tagi_tree_destroy(tagi_tree* tree);

/* Fill *stats [host] (synchronises the stream used at build). */
tagi_status tagi_tree_info(const tagi_tree* tree, tagi_tree_stats* stats);

/* Copy the tree's integer structure and boxes out for inspection.
 *   perm [host] n int32: tree position -> caller index.
 *   begin, end [host] n_clusters int32 each: the cluster owns positions [begin, end).
 *   lo, hi [host] 3*n_clusters float64 (x, y, z per cluster).
 *   parent, nchild [host] n_clusters int32; child [host] 8*n_clusters int32.
 *   Any pointer may be NULL to skip that array. */
tagi_status tagi_tree_export(const tagi_tree* tree, int32_t* perm, int32_t* begin, int32_t* end,
                             double* lo, double* hi, int32_t* parent, int32_t* nchild,
                             int32_t* child);

/* Copy the interaction lists out: for every list entry (in batch order)
 * batch cluster id, source cluster id and kind (0 = direct sum, Eq.
 * direct-sum_2; 1 = approximation, Eq. particle-cluster-approx-rearranged).
 * Direct entries are expanded to the leaves under the cluster Algorithm 3
 * named.  cap: capacity of each host array; *count receives the total. */
tagi_status tagi_tree_lists(const tagi_tree* tree, int64_t cap, int32_t* batch, int32_t* cluster,
                            int32_t* kind, int64_t* count);

/* Proxy weights of Eq. particle-cluster-approx-rearranged,
 *   qh[c][j][k] = sum_{i in cluster c} L_k1(x_i) L_k2(y_i) L_k3(z_i) q[j][i],
 * for EVERY cluster c of the tree (not only the approximated ones), with the
 * barycentric basis of Eq. Lagrange_polynomials / barycentric_weights on the
 * cluster's Chebyshev points of the second kind.
 *   q [dev] nq*n float64 charges in the caller's order; nq >= 1.
 *   qh [dev] n_clusters*nq*(degree+1)^3 float64, caller-owned.
 * The arithmetic is the tree's, as its Green steps anterpolate their fields:
 *   TAGI_FP64: float64 throughout;
 *   TAGI_FP32C: charges rounded to float32, the basis evaluated in float64 on
 *     the float32-rounded nodes (where that form's proxies sit) and rounded to
 *     float32, products on the tensor cores in split precision (3xTF32) with
 *     float32 accumulation over 64 points, partial sums added in float64.
 *     Relative error about 1e-7 of a cluster's largest weight.
 * Synchronises the stream.  TAGI_ERR_TIMEOUT if a bounded wait of the
 * tensor-core kernel gave up. */
tagi_status tagi_anterpolate(tagi_tree* tree, const double* q, int nq, double* qh, void* stream);

/* Yukawa convolution for nf fields with their own decay rates:
 *   u[o][i] = sum_{j, r_ij != 0} G_{k_o}(r_ij) (f[o][j] - f[o][i]) w_j + f[o][i] / k_o^2   (ss = 1)
 *   u[o][i] = sum_{j, r_ij != 0} G_{k_o}(r_ij) f[o][j] w_j                                (ss = 0)
 * evaluated by the treecode (Eq. direct-sum, yukawa-conv-ss, Algorithm 3).
 *   f [dev] nf*n float64; k [host] nf float64, each finite and > 0;
 *   u [dev] nf*n float64, caller-owned.  nf >= 1. */
tagi_status tagi_yukawa_conv(tagi_tree* tree, const double* f, const double* k, int nf, double* u,
                             void* stream);

/* Coulomb (Hartree) convolution by the treecode (Eq. Coulomb, coulomb-conv-ss):
 *   vh[i] = sum_{j, r != 0} (rho_j - rho_i exp(-r^2/alpha^2)) w_j / r + 2 pi alpha^2 rho_i  (ss = 1)
 *   vh[i] = sum_{j, r != 0} rho_j w_j / r                                                  (ss = 0)
 *   rho [dev] n float64; vh [dev] n float64, caller-owned. */
tagi_status tagi_coulomb_conv(tagi_tree* tree, const double* rho, double* vh, void* stream);

/* The convolutions of one Green iteration in a single pass over the
 * geometry (one kernel launch per group of up to 8 fields): nf_y Yukawa
 * fields with their own k, as tagi_yukawa_conv computes them, and, when rho
 * is non-NULL, the Coulomb field of tagi_coulomb_conv.
 *   f [dev] nf_y*n float64 (may be NULL if nf_y = 0); k [host] nf_y, each
 *   finite and > 0; rho [dev] n or NULL; u [dev] nf_y*n and vh [dev] n,
 *   caller-owned.  1 <= nf_y + (rho != NULL) <= 128. */
tagi_status tagi_fields_conv(tagi_tree* tree, const double* f, const double* k, int nf_y, const double* rho,
                             double* u, double* vh, void* stream);

/* One Green iteration for nw orbitals at once (Algorithm 2 lines 3-6):
 *   f_o = (veff + vshift) psi_o, k_o = sqrt(-2 (eps_o + vshift))  (Eq. gauge-shift)
 *   psi~_o = -2 * Yukawa_{k_o}[f_o]                               (Eq. Yukawa)
 *   eps'_o <- eps'_o - <f_o, psi_o - psi~_o> / <psi~_o, psi~_o>   (Eq. gradient-free, shifted eps' = eps + vshift)
 *   modified Gram-Schmidt of psi~ in index order, then normalisation,
 * with every inner product weighted by the quadrature, <a, b> = sum a_i b_i w_i.
 * With rho non-NULL the Hartree potential is computed in the same pass
 * (tagi_coulomb_conv's formula) into vh, and E_H = 1/2 sum vh rho w
 * (Eq. quadrature-example) into *eh.
 *   veff [dev] n; psi [dev] nw*n, in: current orbitals, out: new orbitals;
 *   eps [host] nw, in: current unshifted eigenvalues, out: updated ones;
 *   rho [dev] n or NULL; vh [dev] n or NULL (required when rho is given);
 *   resid [host] nw or NULL: ||psi_new - psi_old||_w; eh [host] or NULL.
 * Errors: TAGI_ERR_INVALID_ARG when eps_o + vshift >= 0 (no decay, Section 3.3).
 * Synchronises the stream. */
tagi_status tagi_green_step(tagi_tree* tree, const double* veff, double vshift, double* psi,
                            double* eps, int nw, const double* rho, double* vh, double* resid,
                            double* eh, void* stream);

/* ------------------------------------------------------------------------
 * The Green step split over target batches, one process per GPU.  Batches
 * are independent once the tree, lists and proxy weights exist (Section 5.5;
 * the paper's multi-GPU runs share the batches out, Section 5.6).  Each
 * process builds the same tree from the same inputs (the build is
 * deterministic), forms and anterpolates every field itself, and computes
 * the convolutions for its own batches only; each target's sums are then
 * bit for bit those of the whole step.  The processes exchange the results
 * (every target is written by exactly one of them) and apply
 * tagi_green_reduce to the full fields.
 * ------------------------------------------------------------------------ */

/* Per batch, in the tree's fixed batch order (0 .. n_leaves-1): size [host]
 * n_leaves targets, cost [host] n_leaves interactions per field
 * (|B| x (near sources + far proxies)).  Either may be NULL.  Synchronises
 * the tree's stream. */
tagi_status tagi_tree_batches(const tagi_tree* tree, int32_t* size, int64_t* cost);

/* tagi_fields_conv for the targets of the listed batches only: u and vh are
 * written at those targets and left untouched elsewhere.
 *   batches [host] nb distinct batch indices (0 <= b < n_leaves); nb = 0 is
 *   a no-op.  Synchronises the stream. */
tagi_status tagi_fields_conv_batches(tagi_tree* tree, const double* f, const double* k, int nf_y, const double* rho,
                                     double* u, double* vh, const int32_t* batches, int nb, void* stream);

/* The convolutions of tagi_green_step for the targets of the listed batches:
 * f_o = (veff + vshift) psi_o, k_o = sqrt(-2 (eps_o + vshift)) (Eq.
 * gauge-shift); u[o] = Yukawa_{k_o}[f_o] (so psi~ = -2 u, Eq. Yukawa) and,
 * with rho, vh = the Hartree potential, both written at the batches' targets
 * only.  veff [dev] n, psi [dev] nw*n (not modified), eps [host] nw
 * unshifted; u [dev] nw*n, vh [dev] n.  Errors: TAGI_ERR_INVALID_ARG when
 * eps_o + vshift >= 0.  Synchronises the stream. */
tagi_status tagi_green_conv_batches(tagi_tree* tree, const double* veff, double vshift, const double* psi,
                                    const double* eps, int nw, const double* rho, double* u, double* vh,
                                    const int32_t* batches, int nb, void* stream);

/* Algorithm 2 lines 4-6 of tagi_green_step given the full convolution
 * results u (nw*n, as tagi_green_conv_batches writes them; not modified):
 * the gradient-free eigenvalue update, modified Gram-Schmidt in index
 * order, normalisation, residuals, and with rho E_H = 1/2 sum vh rho w.
 * psi [dev] in: the orbitals the convolutions used, out: the new ones;
 * eps [host] in/out; resid [host] nw or NULL; eh [host] or NULL.
 * Synchronises the stream. */
tagi_status tagi_green_reduce(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps, int nw,
                              const double* u, const double* rho, const double* vh, double* resid, double* eh,
                              void* stream);

/* Diagnostics (no counterpart in the paper).
 * tagi_kernel_launches: number of CUDA kernels this library has launched in
 * this process so far (monotonic; differences bracket a region of interest).
 * tagi_profile_enable: on != 0 starts CUDA-event timing of the phases of
 * every call (and clears earlier totals); 0 stops it.  Timing adds two event
 * records per phase on the call's stream.
 * tagi_profile_read: total milliseconds and number of timed phases so far for
 * one group: 0 = tree, lists and items (tagi_tree_build), 1 = field
 * preparation and anterpolation, 2 = near/far interaction kernel(s),
 * 3 = SS epilogue, 4 = Green-step reductions.  Synchronises the recorded
 * events.  ms, count [host], either may be NULL. */
int64_t tagi_kernel_launches(void);

/* Device memory of trees and calls comes from a caching allocator: blocks a
 * tree or a call gives back are kept for later calls on the same stream.
 * tagi_trim_cache synchronises the device and returns every cached block to
 * the CUDA driver (call it after destroying trees to shrink the footprint). */
tagi_status tagi_trim_cache(void);

/* Mean relative bias of the float32 kernel values of the TAGI_FP32C path on
 * the current device, weighted as in the singularity-subtraction integrals:
 * *beta_yukawa for exp(-k r)/r (weight r e^{-k r}), *beta_gauss for
 * exp(-r^2/alpha^2)/r (weight r e^{-r^2/alpha^2}).  Measured once per device
 * and process by a deterministic kernel (first FP32C call); the SS epilogue
 * scales the analytic terms f/k^2 and 2 pi alpha^2 rho by (1 + beta) so the
 * subtraction cancels against the float32 sums.  Outputs [host], may be NULL. */
tagi_status tagi_fp32_bias(double* beta_yukawa, double* beta_gauss, void* stream);
tagi_status tagi_profile_enable(int on);
tagi_status tagi_profile_read(int group, double* ms, int64_t* count);

/* Measured throughput of the units that bound the near/far kernel, in thread
 * operations per SM per SM clock (median over SMs; one CTA of 1024 threads
 * per SM runs independent operations in a loop and reads clock64 at both
 * ends):  rates[0] FP32 FMA (fma.rn.f32), rates[1] FP32 FMA issued as packed
 * f32x2 pairs (counted per FMA), rates[2] ex2.approx.ftz.f32, rates[3]
 * rsqrt.approx.ftz.f32, rates[4] FP64 FMA.  rates [host] n_rates >= 5.
 * Takes a few milliseconds; synchronises the stream. */
tagi_status tagi_unit_rates(double* rates, int n_rates, void* stream);

/* Direct-sum Yukawa convolution that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library call cudaMalloc -- host frameworks that hand out every
 * device byte from their own memory pool (a second allocator would fragment
 * it or exceed its budget), and latency-critical loops in which an
 * allocation's implicit device synchronisation would stall other streams.
 * It computes, in float64, the same sum as tagi_yukawa_conv with singularity
 * subtraction on a tree with theta = 0:
 *   u[o][i] = sum_{j, r_ij != 0} G_{k_o}(r_ij) (f[o][j] - f[o][i]) w_j + f[o][i] / k_o^2,
 * G_k(r) = exp(-k r) / (4 pi r), over all n points (O(n^2) work).
 *   xyz [dev] 3*n float64 (structure of arrays), w [dev] n, f [dev] nf*n,
 *   k [host] nf (finite, > 0), u [dev] nf*n, caller-owned; 1 <= nf <= 16.
 * Scratch: one file-scope device array of 2^20 float64 values (8 MiB), held
 * by every GPU that loads the library until the process exits.  Calls with
 * n * nf > 1048576 are rejected with TAGI_ERR_INVALID_ARG.  All calls share
 * that array and it keeps the last call's contents: two calls whose work
 * overlaps on the GPU (different streams, or different host threads on the
 * same device) race and give wrong results.  The caller's stream must be the
 * only one using this entry point on its device until the call's work has
 * completed.  Each call writes every scratch value it reads, so stale
 * contents are never used.
 * Set-up: the first call on each device (and after a cudaDeviceReset, the
 * first call in the new context) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Enqueued on `stream`, asynchronous. */
tagi_status tagi_yukawa_direct_noalloc(const double* xyz, const double* w, const double* f, const double* k,
                                       int nf, int64_t n, double* u, void* stream);

/* A whole Green iteration (tagi_green_step's computation) captured as a CUDA
 * graph, for loops of Green iterations on a fixed tree (FP32C only).  Every
 * per-iteration value lives in device memory, so a replay reads the current
 * eigenvalues, updates the orbitals and eigenvalues in place, and writes the
 * residuals (and E_H) without any host synchronisation.
 *   create: veff [dev] n; psi [dev] nw*n, in/out on every replay; eps [dev]
 *     nw, unshifted, in/out; rho [dev] n or NULL; vh [dev] n (with rho);
 *     resid [dev] nw, out; eh [dev] 1, out (with rho).  1 <= nw < 128.
 *     Runs one eager iteration on private copies of psi and eps (sizing every
 *     buffer, checking eps + vshift < 0), then captures the sequence on
 *     `stream`, which must be a created stream (not NULL or a default stream).  The pointers are baked into the graph: keep the buffers and
 *     the tree alive until the graph is destroyed, and do not call other
 *     entry points on the same tree while replays are in flight.
 *   launch: enqueue one Green iteration on `stream` (asynchronous).
 *   check: synchronise `stream` and report TAGI_ERR_INVALID_ARG if a replay
 *     met eps + vshift >= 0 (Section 3.3).
 *   destroy: waits for the device; NULL is accepted. */
typedef struct tagi_green_graph tagi_green_graph;
tagi_status tagi_green_graph_create(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps,
                                    int nw, const double* rho, double* vh, double* resid, double* eh, void* stream,
                                    tagi_green_graph** out);
tagi_status tagi_green_graph_launch(tagi_green_graph* graph, void* stream);
tagi_status tagi_green_graph_check(tagi_green_graph* graph, void* stream);
tagi_status tagi_green_graph_destroy(tagi_green_graph* graph);

/* Green Iteration to convergence (Algorithm 2) for nw orbitals at once, with
 * Anderson mixing of the eigenpairs x = (eps, psi) under the inner product
 * (x1, x2) = eps1 eps2 + sum psi1 psi2 w (Section 4.3, "Wavefunction Mixing").
 * Each step applies, to every orbital not yet converged, the Green step of
 * tagi_green_step (G(eps) psi, the gradient-free eigenvalue update, then
 * modified Gram-Schmidt in index order against every lower-index orbital --
 * the new iterate of an active one, the stored pair of a converged one -- and
 * normalisation), giving g(x) = (eps', psi') and the residual
 * r = ||psi' - psi||_w (Algorithm 2 line 7).  Then:
 *   r < tol_gi: the orbital is converged and keeps the input of that step,
 *     (eps^(n), psi^(n)), as Algorithm 2 stores it -- or, with store_output,
 *     the step's output g(x) -- and it is not convolved again;
 *   else, before mixing starts: x <- g(x);
 *   else (mixing, which starts once r < mix_tol and stays on): Anderson update
 *     of the last history+1 pairs (x_j, F_j = g(x_j) - x_j): with
 *     D_j = F_n - F_{n-j}, theta solves the normal equations of
 *     min ||F_n - sum_j theta_j D_j||, and
 *     x <- x_n - sum theta_j (x_n - x_{n-j}) + beta (F_n - sum theta_j D_j).
 *     A Gram matrix with a pivot below 1e-13 of its largest diagonal entry
 *     takes theta = 0 (simple mixing) for that step.
 * The loop ends when every orbital has converged or after max_iter steps.
 *   veff [dev] n; psi [dev] nw*n in/out; eps [host] nw in/out (unshifted);
 *   resid [host] nw or NULL: each orbital's last residual;
 *   iters [host] nw or NULL: the step at which each orbital converged, -1 if
 *     it did not;  stats [host] or NULL.
 * Errors: TAGI_ERR_INVALID_ARG for bad parameters, or when eps_o + vshift >= 0
 * at the start or at any step (no decay, Section 3.3); psi and eps then hold
 * the last completed step.  Synchronises the stream once per step. */
typedef struct {
    double tol_gi;   /* convergence tolerance, >= 0 */
    int max_iter;    /* >= 1 */
    double beta;     /* mixing parameter, in (0, 1]; the paper uses 0.5 */
    int history;     /* 0..8 past pairs besides the newest (0: simple mixing) */
    double mix_tol;  /* mixing starts once r < mix_tol (INFINITY: at once; 0: never) */
    int store_output;/* 0: a converged orbital keeps its step input (Algorithm 2);
                        1: its step output (inside an SCF iteration the stored
                        input stops following V_eff once V_eff moves the orbital
                        by less than tol_gi in one step) */
} tagi_gi_params;
typedef struct {
    int steps;            /* Green steps taken */
    int n_converged;      /* orbitals converged */
    int64_t field_steps;  /* sum over steps of the orbitals convolved */
} tagi_gi_stats;
tagi_status tagi_green_iterate(tagi_tree* tree, const double* veff, double vshift, double* psi, double* eps,
                               int nw, const tagi_gi_params* gp, double* resid, int* iters, tagi_gi_stats* stats,
                               void* stream);

/* One SCF iteration (Algorithm 1 lines 2-7) on a fixed mesh (the tree):
 *   line 2: V_eff = V_ext + V_H[rho_in] + V_xc[rho_in] (Eq. effective-potential;
 *           V_H by the treecode Coulomb sum with SS, V_xc the spin-unpolarised
 *           LDA of Section 2: Slater exchange, Perdew-Zunger correlation,
 *           zero where rho <= 1e-30);
 *   line 3: eigenpairs by tagi_green_iterate, warm-started from (eps, psi),
 *           with tol_gi from the schedule below; then each psi_i is
 *           normalised, sum psi_i^2 w = 1;
 *   line 4: Fermi energy mu with 2 sum f_i = N_e, f_i = 1/(e^{(eps_i - mu)/kT} + 1)
 *           (Eq. Fermi), by bisection to the resolution of float64;
 *   line 5: rho_out = 2 sum f_i psi_i^2 (Eq. density-construction);
 *   line 6: residual ||rho_out - rho_in||_w;
 *   line 7: rho_next by Anderson mixing of the density under <a, b> = sum a b w
 *           (tagi_green_iterate's update without the eigenvalue component),
 *           from the pairs (rho_in, rho_out - rho_in) of this and earlier steps.
 * Energy, gradient-free (Eq. total-energy-gradient-free), double-counting
 * terms from rho_in:  E = 2 sum f_i eps_i - E_H + E_xc - <V_xc, rho_in> + E_ZZ,
 * E_H = 1/2 <V_H, rho_in>, E_xc = <eps_xc, rho_in>.
 * tol_gi schedule (Section 6): tol_gi_first on SCF step 0, then geometric
 * steps to tol_gi_final over the next tol_gi_ramp steps, then tol_gi_final.
 * Green Iteration mixing starts at once from step 1 on; on step 0 it starts
 * once an orbital's residual is below gi_mix_tol_first (Section 4.3).
 * The tagi_scf object keeps the density-mixing history and the step count;
 * it refers to the tree, which must outlive it. */
typedef struct {
    double n_electrons;     /* N_e, 0 < N_e <= 2 nw (2 nw: every state filled) */
    double kT;              /* k_B T in Ha, > 0 (Section 6: T = 200 K) */
    double e_zz;            /* nuclear repulsion E_ZZ (Eq. electrostatics) */
    double beta;            /* density mixing parameter, in (0, 1] */
    int history;            /* density mixing depth, 0..8 */
    double tol_gi_first;    /* > 0 */
    double tol_gi_final;    /* > 0 */
    int tol_gi_ramp;        /* >= 0 */
    int gi_max_iter;        /* >= 1 */
    double gi_beta;         /* eigenpair mixing parameter, in (0, 1] */
    int gi_history;         /* 0..8 */
    double gi_mix_tol_first;/* >= 0, INFINITY allowed */
    int gi_store_output;    /* tagi_gi_params.store_output of every Green Iteration */
} tagi_scf_params;
typedef struct {
    int step;               /* index of the SCF step just taken (0-based) */
    double tol_gi;          /* Green Iteration tolerance it used */
    double mu;              /* Fermi energy */
    double residual;        /* ||rho_out - rho_in||_w */
    double e_band, e_hartree, e_xc, e_vxc, e_zz, e_total;
    tagi_gi_stats gi;       /* the Green Iteration of this step */
} tagi_scf_report;
typedef struct tagi_scf tagi_scf;
tagi_status tagi_scf_create(tagi_tree* tree, const tagi_scf_params* params, tagi_scf** out);
/*   vext [dev] n; rho [dev] n, in: rho_in, out: rho_next; psi [dev] nw*n in/out;
 *   eps [host] nw in/out (unshifted); occ [host] nw out or NULL;
 *   rho_out [dev] n out or NULL; report [host] or NULL.
 * Errors: as tagi_green_iterate, and TAGI_ERR_INVALID_ARG for N_e outside
 * (0, 2 nw].  Synchronises the stream. */
tagi_status tagi_scf_step(tagi_scf* scf, const double* vext, double vshift, double* rho, double* psi, double* eps,
                          int nw, double* occ, double* rho_out, tagi_scf_report* report, void* stream);
tagi_status tagi_scf_destroy(tagi_scf* scf);

/* ------------------------------------------------------------------------
 * Learned warm start (an addition to the paper's method, whose SCF runs
 * start from superposed atomic data, Section 6).  A per-point MLP maps the
 * features of a mesh point to a relative correction y of the normalised
 * superposition start s: psi = s (1 + y), normalised in the quadrature
 * norm.  Trained on converged orbitals of this solver's SCF runs; plain
 * Green Iteration measures its error.
 *
 * Model: F = 8 features, two tanh layers of H = 32 or H = 64 units, one
 * output.  Parameters (H F + H^2 + 3 H + 1 float64 values: 1377 for H = 32,
 * 4801 for H = 64; this order): W1 (H x F row-major), b1 (H), W2 (H x H
 * row-major), b2 (H), W3 (H), b3 (1).  Weights enter the products rounded to
 * bfloat16 (nearest, ties to even); biases as float32; Adam (Kingma and Ba,
 * 2015) updates float64 master weights.
 *   H = 32: the arithmetic of a point is float32 (SIMT kernels); gradients
 *     are summed over points in float64 in a fixed order.
 *   H = 64: the three products of a point (W1 x, W2 h1, and dz2 W2 in the
 *     gradient) and the weight-gradient sums over points run on the tensor
 *     cores (tcgen05.mma kind::f16, bfloat16 operands, float32 accumulation),
 *     so the second layer's input bf16(h1) and the gradient's dz2, dz1, dy
 *     and h2 enter those products rounded to bfloat16; sums over at most 1024
 *     points in float32, then in float64 in a fixed order.  TAGI_ERR_TIMEOUT
 *     if a bounded wait of these kernels gave up.
 * Both are deterministic on a given device.
 *
 * A tagi_mlp holds its weights, Adam moments and scratch: use it from one
 * stream at a time.
 *
 * Features of a point (float64, then rounded to bfloat16, stored as (n, 8)
 * uint16 encodings, row-major, 16-byte aligned): with r1 <= r2 the
 * distances to the two nearest nuclei (lower index first on ties) and R the
 * distance between those two nuclei,
 *   [e^-r1, e^-r2, tanh r1, tanh r2, (r2 - r1)/R, tanh((r1 + r2)/R - 1),
 *    R - 1.5, e^-(r1 + r2 - R)]
 * (with per-nucleus decay rates z1, z2 the first two are e^-(z1 r1) and
 * e^-(z2 r2): tagi_mlp_features_scaled).
 * ------------------------------------------------------------------------ */
typedef struct tagi_mlp tagi_mlp;
typedef struct {
    double lr;     /* step size, >= 0 */
    double beta1;  /* in [0, 1) */
    double beta2;  /* in [0, 1) */
    double eps;    /* > 0 */
} tagi_adam_params;

/* params [host] n_params finite values (1377 for hidden = 32, 4801 for
 * hidden = 64); n_features must be 8 and hidden 32 or 64.  Synchronous
 * (default stream).  Adam's moments start at zero. */
tagi_status tagi_mlp_create(int n_features, int hidden, const double* params, int64_t n_params, tagi_mlp** out);
/* Master weights into params [host] (the model's n_params values).
 * Synchronises stream. */
tagi_status tagi_mlp_get_params(const tagi_mlp* mlp, double* params, int64_t n_params, void* stream);
/* xyz [dev] 3*n (structure of arrays); nuclei [host] n_nuclei*3 positions
 * (2..16, distinct); feat [dev] n*8 uint16 out. */
tagi_status tagi_mlp_features(const double* xyz, int64_t n, const double* nuclei, int n_nuclei, uint16_t* feat,
                              void* stream);
/* The same features with the two nuclei of a heteronuclear pair in list
 * order: r1 is the distance to nuclei[0..2], r2 to nuclei[3..5] (no
 * sorting by distance), so a point's features say which atom it is near.
 * nuclei [host] 2*3 positions, distinct. */
tagi_status tagi_mlp_features_ordered(const double* xyz, int64_t n, const double* nuclei, uint16_t* feat,
                                      void* stream);
/* The features with a decay rate per nucleus in the first two: e^-(z1 r1)
 * and e^-(z2 r2), z1 and z2 the rates of the nuclei at distances r1 and r2
 * (all 1: tagi_mlp_features / _ordered, bit for bit).  A rate near the
 * Slater exponent of a heavier atom's 1s shell resolves its core, where the
 * rate-1 exponentials are nearly flat.  scale [host] n_nuclei rates, finite
 * and > 0; ordered: 0 (two nearest, 2..16 nuclei) or 1 (list order, 2
 * nuclei).  TAGI_ERR_INVALID_ARG for a NULL scale or a bad rate. */
tagi_status tagi_mlp_features_scaled(const double* xyz, int64_t n, const double* nuclei, const double* scale,
                                     int n_nuclei, int ordered, uint16_t* feat, void* stream);
/* y [dev] n float32 out: the network's output for each point. */
tagi_status tagi_mlp_forward(const tagi_mlp* mlp, const uint16_t* feat, int64_t n, float* y, void* stream);
/* Loss L = sum_p wt_p (y_p - t_p)^2 and dL/dparams of the current master
 * weights (the gradient of a rounded weight is applied to its master value):
 * target, wt [dev] n float32; grad [host] n_params out; loss [host] out.
 * Synchronises stream. */
tagi_status tagi_mlp_gradient(tagi_mlp* mlp, const uint16_t* feat, const float* target, const float* wt, int64_t n,
                              double* grad, double* loss, void* stream);
/* One full-batch Adam step on L; loss [host] (L before the step) or NULL
 * (then nothing synchronises). */
tagi_status tagi_mlp_train_step(tagi_mlp* mlp, const uint16_t* feat, const float* target, const float* wt,
                                int64_t n, const tagi_adam_params* adam, double* loss, void* stream);
/* psi [dev] n out = s (1 + y) / ||s (1 + y)||_w with s, w [dev] n. */
tagi_status tagi_mlp_warm_start(const tagi_mlp* mlp, const uint16_t* feat, const double* s, const double* w,
                                int64_t n, double* psi, void* stream);
tagi_status tagi_mlp_destroy(tagi_mlp* mlp);

/* Message of the last failing call on this thread ("" if none). */
const char* tagi_last_error(void);

/* Library version string. */
const char* tagi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TAGI_H */
