/*
 * fmm_layered.h -- C ABI of the GB300 layered-media Helmholtz FMM.
 *
 * Computes, for N_t targets and N_s wave sources embedded in a medium of
 * L+1 horizontal layers, the potentials
 *
 *     Phi(t_i) = sum_j q_j G(t_i, s_j)
 *
 * with G the layered-media Green's function of the Helmholtz equation
 * (Wang, Zhang & Cai, "Fast multipole method for 3-D Helmholtz equation in
 * layered media", Sec. 3.1 eqs. domaingreenfn-totaldensity and the sum of
 * eq. totalinteraction): the free-space part e^{ik_l r}/(4 pi r) for source
 * and target in the same layer l (skipped when the two points are bitwise
 * identical, the paper's j != i), plus the reaction components u^{ab}_{l l'}
 * for every source (self image included).  Interface conditions: [u] = 0 and
 * [eps du/dz] = 0 across every interface.
 *
 * Layers are numbered 0..L from top to bottom; interfaces d_0 > ... > d_{L-1};
 * layer l is d_l < z < d_{l-1}.
 *
 * Memory and threading: the caller owns every buffer passed in.  The library
 * owns the handle and its device workspace (grown on demand, freed by
 * fmm_layered_destroy).  A handle must not be used by two threads at once.
 * Device buffers must be on the device that was current at create time.
 *
 * Errors: every int-returning call returns 0 (FMM_OK) or a negative code;
 * fmm_layered_last_error() then describes the last failure of that handle.
 */
#ifndef FMM_LAYERED_H
#define FMM_LAYERED_H

#ifdef __cplusplus
extern "C" {
#endif

#define FMM_OK                 0
#define FMM_ERR_ARG           -1   /* invalid argument (sizes, order, layers) */
#define FMM_ERR_ON_INTERFACE  -2   /* a point lies exactly on an interface    */
#define FMM_ERR_NONFINITE     -3   /* a coordinate or charge is NaN or Inf    */
#define FMM_ERR_CUDA          -4   /* a CUDA call failed                      */
#define FMM_ERR_OOM           -5   /* device allocation failed                */
#define FMM_ERR_TIMEOUT       -6   /* a bounded device wait expired (the kernel
                                       released its resources; the context
                                       stays usable)                          */
#define FMM_ERR_UNSUPPORTED   -7   /* beyond the compiled limits              */

/* flags for fmm_layered_create */
#define FMM_PLAIN_FP64   0u   /* every stage in FP64 (default)                 */
#define FMM_NORM_PAPER   1u   /* scale results for targets in layer l by
                                 4 pi / (i k_l): the paper's h_0 normalization
                                 with the factor i k_l / 4 pi omitted (eq.
                                 totalinteraction)                             */
#define FMM_MIXED        2u   /* M2L translations on the tensor cores: FP16
                                 hi/lo split operands with power-of-two
                                 scaling, FP32 accumulation (3 products);
                                 free-space near field in FP32 with a
                                 compensated sum; in the reaction near field
                                 the real-axis tail of the Sommerfeld
                                 quadrature in FP32 with a compensated sum;
                                 expansions, operators, the rest of the
                                 reaction near field and all sums over
                                 translations stay FP64.  Relative error of
                                 the potentials below 1e-5.                    */
#define FMM_SURROGATE    4u   /* once fmm_layered_surrogate_train has run: the
                                 reaction components of the near field and of
                                 fmm_layered_direct come from the learned
                                 surrogate wherever its held-out check passed
                                 (quadrature elsewhere)                        */
#define FMM_TREE_COUNTS  8u   /* reaction trees refined by the point counts
                                 alone: without it a reaction-tree box that
                                 touches the interface is refined while it
                                 holds any point, which separates every
                                 target leaf from every image leaf, so the
                                 reaction components run entirely through
                                 M2L.  With it, target leaves next to the
                                 interface meet image leaves in their U, W
                                 and X lists and those pairs are evaluated
                                 directly (Sommerfeld quadrature of eq.
                                 generalcomponentsimag, or the surrogate)    */
#define FMM_TABLES      16u   /* reaction M2L operators from tabulated
                                 Sommerfeld integrals (Sec. 3.5, eqs.
                                 M2Ltable, metoletableform): at create, the
                                 integrals S_{q,t,mu,nu} of every reaction
                                 component are computed on the 40 rays of
                                 M2L classes (box centres (jt + 1/2) w and
                                 (js + 1/2) w from the interface, jt, js in
                                 {0, 1}, horizontal offset w sqrt(dx^2+dy^2))
                                 for k_max w in [2^-8, 2^1.5] and kept at 12
                                 Chebyshev points per panel of log2(k_max w);
                                 an evaluation interpolates them instead of
                                 integrating, so a new geometry costs no
                                 quadrature.  Classes outside that range use
                                 the quadrature.  The reaction near field
                                 takes its kernel from a second table, of
                                 R u~ on 10 x 16 x 8 Chebyshev points per
                                 panel in (log2(k_max R), atan(rho/H), zt/H),
                                 R = |(rho, H)|, H = zt + zs, k_max R in
                                 [2^-7, 2^3], rho <= 6 H (quadrature outside;
                                 the surrogate, when trained and attached,
                                 comes first).  p <= 12 (FMM_ERR_UNSUPPORTED
                                 otherwise).  Cost at create, per reaction
                                 component: about 36 ms and 52 MB at p = 8
                                 (16 components of three layers: 0.58 s,
                                 830 MB); memory grows with the number of
                                 tables, 351 at p = 8, 519 at p = 10           */
#define FMM_TEST_STALL_TC (1u << 30) /* test only, with FMM_MIXED: every
                                 stage of the tensor-core M2L waits for 16
                                 bytes more than it copies, so its bounded
                                 waits expire (about 1 s each); the kernel
                                 then releases its resources and the
                                 evaluation returns FMM_ERR_TIMEOUT            */

typedef struct fmm_layered fmm_layered_t;

typedef struct {
  int    n_components;     /* FMMs in the last evaluation (free + reaction)  */
  int    n_boxes;          /* boxes over all component trees                 */
  int    max_level;        /* deepest tree level                             */
  long   n_v_pairs;        /* M2L translations                               */
  long   n_u_pairs;        /* near-field (U, W, X) source-target pairs       */
  int    n_quad_near;      /* complex contour nodes of the quadrature rule   */
  int    n_quad_total;     /* all contour nodes currently held               */
  double ms_setup;         /* last fmm_layered_create, host wall clock       */
  double ms_tree;          /* last evaluation: classification, keys, sort,
                              levels and lists (host wall clock, synchronous) */
  double ms_operators;     /* translation operators                          */
  double ms_eval;          /* upward, downward, near field and sum           */
  /* device time of each stage of the last evaluation (CUDA events on the
     evaluation's stream) */
  double gpu_ms_tree, gpu_ms_operators, gpu_ms_upward, gpu_ms_m2l, gpu_ms_l2p,
         gpu_ms_near_free, gpu_ms_near_reac, gpu_ms_sum, gpu_ms_total;
  long   n_free_pairs;     /* free-space near-field pairs evaluated          */
  long   n_reac_pairs;     /* reaction near-field pairs evaluated            */
  long   n_reac_nodes;     /* quadrature nodes summed over reaction pairs    */
  long   n_reac_tail_nodes;/* ... of which on the real-axis tail             */
  long   n_reac_classes;   /* reaction M2L radial integrals computed         */
  long   n_free_ops;       /* free-space translation operators built         */
  long   n_reac_T_nodes;   /* quadrature nodes summed over those integrals   */
  long   n_v_pairs_reac;   /* ... of n_v_pairs, in reaction components        */
  long   n_launches;       /* kernels of this library launched by the last
                              evaluation (its own sort and scan included)    */
  double gpu_ms_m2l_gemm;  /* device time of the M2L translation products
                              alone (CUDA events around those launches)      */
  double m2l_gemm_flops;   /* their algorithmic flops: 8 per complex
                              multiply-add of operator entry and expansion
                              coefficient over all V-list translations       */
  double m2l_tensor_flops; /* FMM_MIXED: flops the tensor cores executed for
                              them (3 real products per tile, padding
                              included); 0 in the FP64 path                  */
  double m2l_tc_bytes;     /* FMM_MIXED: algorithmic bytes of those products:
                              the FP16 hi/lo tiles of the gathered columns
                              and of each operator used, read once, and the
                              FP64 translated columns written once           */
  long   n_reac_surr_pairs;/* of n_reac_pairs, those the learned surrogate
                              evaluated (FMM_SURROGATE)                      */
  double reac_near_rho_max;/* the box of (rho, zt, zs) the reaction near-field
                              pairs of the last evaluation needed: largest
                              horizontal distance, smallest and largest
                              distance of target or image to the interface
                              (all 0 without reaction near-field pairs); the
                              box to train the surrogate on                  */
  double reac_near_z_min, reac_near_z_max;
  double ms_tables;        /* FMM_TABLES: device time of the table build at
                              create (CUDA events)                           */
  double table_bytes;      /* FMM_TABLES: device memory of the tables        */
  long   n_reac_table_classes; /* reaction M2L radial operators of the last
                              evaluation interpolated from the tables        */
  long   n_reac_table_pairs;   /* FMM_TABLES: of n_reac_pairs, those whose
                              kernel came from the near-field table          */
  /* M2L tile autotuner: on the first evaluation with free-space translations
     (rotation form, p >= 5) the handle times every candidate column tile and
     block size of that kernel on the evaluation's own translations and keeps
     the fastest; 0 until then */
  int    tune_zrot_kc;         /* chosen column tile (translations per CTA)  */
  int    tune_zrot_threads;    /* chosen threads per CTA                     */
  int    tune_zrot_candidates; /* candidates timed                           */
  double tune_zrot_ms;         /* device time of the chosen candidate        */
  double tune_zrot_rule_ms;    /* ... of the fixed rule (the default tile,
                                  128 threads), for comparison              */
} fmm_stats_t;

/*
 * Create a solver for a layered medium (Sec. 3.1).
 *   n_layers    L+1 >= 1 (at most 8)
 *   k           [L+1] wave numbers k_l > 0, top to bottom (host)
 *   interfaces  [L] d_0 > d_1 > ... (host; NULL when L = 0)
 *   eps         [L+1] material coefficients > 0 in the transmission
 *               condition [eps du/dz] = 0 (host; NULL means all 1)
 *   p           expansion order, 1 <= p <= 16 (terms n = 0..p)
 *   leaf        maximum number of sources or targets in a leaf box, >= 1
 *   flags       FMM_PLAIN_FP64 | FMM_NORM_PAPER | FMM_MIXED | FMM_SURROGATE |
 *               FMM_TREE_COUNTS
 *   out         receives the handle (NULL on failure)
 * Builds the contour quadrature rule and the reaction densities sigma at its
 * nodes on the current device.  Returns FMM_ERR_ARG for invalid input.
 */
int fmm_layered_create(int n_layers, const double* k, const double* interfaces,
                       const double* eps, int p, int leaf, unsigned flags,
                       fmm_layered_t** out);

/* Release the handle and all device memory it owns.  NULL is accepted. */
void fmm_layered_destroy(fmm_layered_t* h);

/* Message of the handle's last failure ("" if none); valid until the next
 * call on the handle.  With h == NULL: message of the last failed create. */
const char* fmm_layered_last_error(const fmm_layered_t* h);

/*
 * FMM evaluation (Algorithm 1 for every component, summed as in eq.
 * totalinteraction).
 *   src_xyz   [n_src*3] row-major x,y,z (device)
 *   charges   [2*n_src] interleaved complex128 (device)
 *   tgt_xyz   [n_tgt*3] (device)
 *   out       [2*n_tgt] interleaved complex128 potentials (device, written)
 *   stream    cudaStream_t to run on (NULL: legacy default stream)
 * The call returns after the result is complete on `stream` (it synchronizes
 * the stream while building the trees).  n_src or n_tgt may be 0.
 * FMM_ERR_ON_INTERFACE if a point has z equal to an interface;
 * FMM_ERR_NONFINITE for NaN/Inf input.
 */
int fmm_layered_eval(fmm_layered_t* h, long n_src, const double* src_xyz,
                     const double* charges, long n_tgt, const double* tgt_xyz,
                     double* out, void* stream);

/*
 * Batched evaluation of n independent problems (the components of different
 * problems never interact, as the components of one problem are summed only
 * at the end: eq. totalinteraction).  Problem i uses handle hs[i] (its own
 * medium, p and leaf size) and the device buffers src_xyz[i], charges[i],
 * tgt_xyz[i], out[i] laid out as in fmm_layered_eval, with n_src[i] sources
 * and n_tgt[i] targets.  The handles must be distinct: a handle holds the
 * workspace of one problem at a time.
 * The problems run concurrently, each on a stream of its own handle that
 * first waits for the work already queued on `stream` (the inputs); when
 * the call returns, `stream` is ordered after every problem that succeeded.
 * Results are identical to n separate fmm_layered_eval calls.
 * Returns FMM_OK, FMM_ERR_ARG (bad arrays or a repeated handle, nothing
 * run), or the code of the first failed problem (in index order); the
 * message of each failed problem is fmm_layered_last_error(hs[i]), and the
 * outputs of the problems that did not fail are valid.
 */
int fmm_layered_eval_batched(int n, fmm_layered_t* const* hs, const long* n_src,
                             const double* const* src_xyz, const double* const* charges,
                             const long* n_tgt, const double* const* tgt_xyz,
                             double* const* out, void* stream);

/*
 * Learned surrogate of the reaction components (the form that replaces the
 * Sommerfeld quadrature of eq. generalcomponentsimag in the near field).
 * For every reaction component (l, l', a, b) of the medium, draws
 * samples_per_component points (rounded up to a multiple of 512) uniformly in
 * the box rho in [0, rho_max], zt, zs in [z_min, z_max] (zt: target distance
 * to the component's reference interface, zs: image depth), stratified over
 * the cells of an 8 x 8 x 8 grid, plus 1/8 as many held-out points (seeded
 * counter-based generator), evaluates the component there with the
 * library's quadrature, and trains one network per component on
 * y = 4 pi R u, R = sqrt(rho^2 + (zt + zs)^2): hidden layers 3 -> 64 -> 64 ->
 * 64 (GELU) by Adam for `steps` steps on the standardized outputs (BF16
 * weights and layer inputs, FP32 accumulation, FP32 master weights,
 * minibatch 1024, cosine learning-rate decay), then a linear output layer
 * 64 -> 2 per cell by least squares over the cell's samples (FP64 normal
 * equations).  Inference carries weights and layer inputs as BF16 hi/lo
 * pairs with FP32 accumulation.  The held-out relative RMS error is measured
 * on each cell; the surrogate is used (with FMM_SURROGATE) only in cells
 * within `bound`, and the quadrature everywhere else and outside the box.
 * Retraining replaces the previous networks.  Runs on `stream` and returns
 * when done.  FMM_ERR_ARG for a single layer or invalid box/sizes.
 */
int fmm_layered_surrogate_train(fmm_layered_t* h, double rho_max, double z_min,
                                double z_max, long samples_per_component,
                                int steps, double bound, unsigned long long seed,
                                void* stream);

/* Re-judge the cells of the last training against a new bound (no
 * retraining; synchronous).  FMM_ERR_ARG if untrained or bound <= 0. */
int fmm_layered_surrogate_set_bound(fmm_layered_t* h, double bound);

/* Held-out verdict of the last training: cell_err[slot * 512 + cell] (relative
 * RMS error, -1 where not judged) and cell_ok (1 where used), slot =
 * ((l (L+1) + l') 2 + a) 2 + b, cell = (c_rho 8 + c_zt) 8 + c_zs; arrays of
 * 4 (L+1)^2 512 entries (host, either may be NULL).  FMM_ERR_ARG if untrained. */
int fmm_layered_surrogate_report(const fmm_layered_t* h, double* cell_err,
                                 unsigned char* cell_ok);

/*
 * Gradient of the surrogate's training loss over one minibatch, computed by
 * the training kernels of fmm_layered_surrogate_train (forward and backward
 * with weights and layer inputs rounded to BF16, FP32 accumulation, the
 * per-CTA partial gradients added in the order of the Adam step).  Exists to
 * check those kernels against an independent implementation.
 *   params  [FMM_SURR_NPARAM] FP32 parameters: W1 [64][3], b1 [64],
 *           W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [2][64], b4 [2]
 *           (row-major, output index first; host)
 *   x       [1024][3] network inputs (host)
 *   y       [1024][2] targets (host)
 *   grad    [FMM_SURR_NPARAM] written: gradient of
 *           (1/1024) sum_s |net(x_s) - y_s|^2 (host)
 * Runs on the current device (allocates and frees its own buffers; legacy
 * default stream, synchronous).  FMM_ERR_ARG for NULL pointers.
 */
#define FMM_SURR_NPARAM 8706
#define FMM_SURR_BATCH 1024
int fmm_layered_surrogate_grad(const float* params, const float* x, const float* y, float* grad);

/* Same as fmm_layered_eval with HOST buffers: copies inputs to the device,
 * evaluates and copies the potentials back (all on `stream`). */
int fmm_layered_eval_host(fmm_layered_t* h, long n_src, const double* src_xyz,
                          const double* charges, long n_tgt, const double* tgt_xyz,
                          double* out, void* stream);

/*
 * Direct O(N_s N_t) evaluation of the same sum on the GPU: free-space kernel
 * and the reaction part as one Sommerfeld integral per pair on the library's
 * contour (eq. generalcomponents summed over the four types).  Arguments as
 * fmm_layered_eval (device buffers).
 */
int fmm_layered_direct(fmm_layered_t* h, long n_src, const double* src_xyz,
                       const double* charges, long n_tgt, const double* tgt_xyz,
                       double* out, void* stream);

/*
 * Allocation-free direct sum.  The paper has no counterpart: this exists for
 * callers that cannot allocate device memory when they need the potentials,
 * for example code running inside another framework's memory manager (whose
 * caching allocator holds the free device memory) or an inner solver loop
 * that must not call cudaMalloc/cudaFree (they synchronize the device).
 * Computes exactly what fmm_layered_direct computes (same arguments, device
 * buffers, result on `stream`) but keeps its scratch -- the per-node reaction
 * coefficients, interface-distance reductions and error flags -- in one
 * file-scope device array of FMM_NOALLOC_SCRATCH_BYTES, held by every GPU
 * that loads the library until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call shares the one array and the array keeps the last call's
 *     contents (the call clears what must start at zero): calls that overlap
 *     on the GPU (several streams or threads at once) race; serialize them.
 *   - Limit: the coefficient table needs 64 * n_layers^2 * Q bytes (Q = nodes
 *     of the handle's quadrature rule); larger tables are rejected with
 *     FMM_ERR_UNSUPPORTED and a message, as is a geometry whose points lie so
 *     close to an interface that the rule would have to grow (run
 *     fmm_layered_direct or fmm_layered_eval once on that geometry first).
 */
#define FMM_NOALLOC_SCRATCH_BYTES (4 * 1024 * 1024)
int fmm_layered_direct_noalloc(fmm_layered_t* h, long n_src, const double* src_xyz,
                               const double* charges, long n_tgt, const double* tgt_xyz,
                               double* out, void* stream);

/*
 * Splitting one problem's components over several GPUs.  The free-space and
 * reaction components are independent FMMs whose potentials are summed at
 * the end (eq. totalinteraction; Sec. 4 notes that they can run in
 * parallel).  Component order: free-space layers 0..L that hold points, then
 * reaction (l, l', a, b) lexicographically, arrow up = 0 (as reported by
 * fmm_layered_component_info after an evaluation of all components).
 *   fmm_layered_set_components: later evaluations of the handle compute only
 *     components [first, first + count) of that order (count < 0: all from
 *     `first`; ranges past the end are clipped, an empty range gives zero
 *     potentials); fmm_layered_eval then returns their sum.  The component
 *     export reports the evaluated components only.  FMM_ERR_ARG if first < 0.
 *   fmm_layered_component_work: work estimate of each component of the last
 *     evaluation (FP64-equivalent flops: M2L translations in the form the
 *     library runs, near-field pairs -- reaction pairs weighted by their
 *     contour nodes -- and P2M/L2P per point); writes work[0 .. nc-1] (host)
 *     and returns nc, or FMM_ERR_ARG if n < nc.  Evaluate all components once
 *     to split them by this estimate.
 *   fmm_layered_add_components: out += the potentials of the components of
 *     the last evaluation, added one component after the other in their
 *     order -- the same additions, in the same order, as the final sum of
 *     fmm_layered_eval.  A device buffer holding the sum of the components
 *     before `first` (computed the same way) therefore becomes bit-identical
 *     to the all-component result once every later range has been added in
 *     turn.  Runs on `stream`; FMM_ERR_UNSUPPORTED with FMM_NORM_PAPER (the
 *     scaling applies to the final sum only).
 */
int fmm_layered_set_components(fmm_layered_t* h, int first, int count);
int fmm_layered_component_work(const fmm_layered_t* h, double* work, int n);
int fmm_layered_add_components(fmm_layered_t* h, double* out, void* stream);

/*
 * Throughput of dependent FP64 fused multiply-adds on the current device
 * (GFLOP/s, 2 flops per FMA), measured by a short kernel; the denominator of
 * the FP64 roofline.  Returns FMM_OK and writes *gflops.
 */
int fmm_layered_measure_fp64_peak(double* gflops);

/*
 * Let handle h use the device workspace of `owner` (the scratch arrays of an
 * evaluation: sorted points, trees, lists, expansions, M2L work arrays),
 * releasing its own if no other handle shares it.  Handles that share a
 * workspace must not be evaluated at the same time: fmm_layered_eval_batched
 * runs the problems of such handles one after the other on one stream, so
 * that a batch of many problems holds as many workspaces as there are
 * groups instead of one per problem.  Each handle keeps its own operators,
 * tables and statistics; the tree export and fmm_layered_add_components
 * describe the last evaluation made in the shared workspace.  Both handles
 * must belong to the same device (FMM_ERR_ARG otherwise).  Synchronizes the
 * device.  The paper has no counterpart (it evaluates one problem at a time).
 */
int fmm_layered_share_workspace(fmm_layered_t* h, fmm_layered_t* owner);

/* Statistics of the last create/evaluation. */
int fmm_layered_stats(const fmm_layered_t* h, fmm_stats_t* stats);

/*
 * One radial reaction M2L operator interpolated from the tables of a handle
 * created with FMM_TABLES (Sec. 3.5, eq. metoletableform: the entries
 * I_{nm,n'm'} as sums of the tabulated S integrals, with the phases and
 * signs of eq. me2lesimplified; the azimuthal factor e^{i(m'-m)phi} is not
 * included).  The class is the reaction component (l, l', a, b) (a, b: 0 up,
 * 1 down) at box width w, target box centre (jt + 1/2) w and image box centre
 * (js + 1/2) w from the interface (jt, js in {0, 1}) and horizontal distance
 * w sqrt(R2[r]), R2 = {0, 1, 2, 4, 5, 8, 9, 10, 13, 18}, r in 0..9.
 *   out  host, [(p+1)^2][(p+1)^2] complex128 interleaved, row (n, m) =
 *        output coefficient, column (n', m') = input coefficient, flat index
 *        n^2 + n + m (caller-owned)
 * Synchronous on the default stream.  FMM_ERR_ARG without tables, for an
 * absent component or a width outside the tables.
 */
int fmm_layered_table_operator(fmm_layered_t* h, int l, int lp, int a, int b, double w, int jt, int js, int r,
                               double* out);

/*
 * Export of the trees and interaction lists of the last evaluation, for
 * checking them against an independent implementation.
 *   fmm_layered_component_info: for component c (0 <= c < n_components, in the
 *     order: free-space layers 0..L, then reaction (l, l', a, b) in
 *     lexicographic order with arrow up = 0, down = 1) writes
 *     info[0..9] = kind (0 free, 1 reaction), l, l', a, b, n_src, n_tgt,
 *     n_boxes, n_levels, 0 and root[0..3] = centre x, y, z and half-width.
 *   fmm_layered_tree_export: host arrays sized by component_info; boxes are
 *     numbered per component by (level, key prefix):
 *       level[nb], prefix[nb] (uint64 as long long), src_begin[nb],
 *       src_end[nb], tgt_begin[nb], tgt_end[nb], parent[nb] (component-local
 *       positions; -1 for the root),
 *       src_perm[n_src], tgt_perm[n_tgt]: original index (within the
 *       component's layer) of each sorted point,
 *       list_off[4][nb+1], list_idx[4][*]: CSR of the V, U, W, X lists
 *       (list_idx arrays sized by list_off[..][nb]; pass NULL list_idx to only
 *       read the offsets).
 */
int fmm_layered_num_components(const fmm_layered_t* h);
int fmm_layered_component_info(const fmm_layered_t* h, int c, long long* info, double* root);
int fmm_layered_tree_export(const fmm_layered_t* h, int c, int* level, long long* prefix,
                            int* src_begin, int* src_end, int* tgt_begin, int* tgt_end,
                            int* parent, int* src_perm, int* tgt_perm,
                            int* list_off, int* v_idx, int* u_idx, int* w_idx, int* x_idx);

#ifdef __cplusplus
}
#endif
#endif
