/*
 * ds.h -- C ABI of the GB300 (sm_103a) library for third-order directionally
 * split exponential integrators on Kronecker-sum matrices
 * (Cassini, "Efficient third order tensor-oriented directional splitting for
 * exponential integrators", arXiv 2310.07551).
 *
 * What the library computes
 *   The stiff linear part is K = A_d (+) ... (+) A_1 (Section 1, eq. kronsum).
 *   phi_l(tau K) v is replaced by the directional splits of Section 2
 *   (Table 1 real coefficients for d = 2, Table 3 for d = 3 and 4, the
 *   second eta scaled by 2^(d-3) as Section 2.3 prescribes), each realised
 *   as Tucker operators, i.e. chained mu-mode products (Section 2,
 *   eq. krontomu).  These drive the exponential Runge-Kutta scheme EXPRK3
 *   (Section 2.4, eq. exprk3), i.e. EXPRK3DS_REAL of Algorithms 1 and 2, on
 *   the two-component block system of Section 3 (eq. twocompdisc).
 *
 * Conventions shared by every entry point
 *   - Tensors: FP64, mode 1 fastest (column-stacking vec of Section 2):
 *     element (i_1, ..., i_d) sits at i_1 + n_1 (i_2 + n_2 (...)).
 *     A two-component state is the u tensor followed by the v tensor.
 *   - Matrices: FP64, column-major, n_mu x n_mu.
 *   - Device pointers are CUDA device (or managed) addresses on the current
 *     device; host pointers are ordinary host addresses.
 *   - Ownership: the caller owns every tensor and matrix it passes; the
 *     library owns the objects it creates (phi-sets, plans) and their device
 *     workspaces, and frees them only in the matching *_destroy call.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls enqueue work and return without waiting,
 *     except where stated.
 *   - Errors: every call returns a ds_status; on failure nothing is
 *     launched, and ds_last_error() gives a message (thread-local).  No C++
 *     exception crosses the ABI.  There is no CPU fallback: a missing or
 *     non-sm_103 GPU gives DS_ERR_UNSUPPORTED or DS_ERR_CUDA.
 *   - Device-side failures (a bounded wait that gave up) are recorded in the
 *     plan and reported by ds_plan_sync as DS_ERR_TIMEOUT.
 */
#ifndef DS3_DS_H
#define DS3_DS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DS_OK = 0,
    DS_ERR_INVALID_ARG = 1,   /* bad pointer, size, tau, model, ... */
    DS_ERR_UNSUPPORTED = 2,   /* valid request outside the library's shapes/precisions */
    DS_ERR_OOM = 3,           /* device allocation failed */
    DS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    DS_ERR_NONFINITE = 5,     /* NaN/Inf found in the state */
    DS_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} ds_status;

/* Arithmetic of the mu-mode contractions.
 *   DS_PREC_F64    : FP64 everywhere (FP64 FMA pipe).
 *   DS_PREC_F32    : FP32 mode products on the CUDA cores (FP32 FMA, FP32
 *                    intermediates and stage sums), FP64 state -- the
 *                    design of the paper's single-precision GPU runs.
 *   DS_PREC_BF16X6 : each FP32-class operand x is split into three BF16
 *                    parts x = x0 + x1 + x2; the six partial products of
 *                    weight >= 2^-16 run on the tcgen05 tensor cores with FP32
 *                    accumulation in tensor memory.  The state u_{n+1}, the
 *                    stage sums and the phi-matrices stay FP64.
 *   DS_PREC_BF16X6C: DS_PREC_BF16X6 with compensated accumulation: the main
 *                    product x0 y0 and the five cross products accumulate in
 *                    two tensor-memory accumulators, added with
 *                    round-to-nearest.  The tensor core's accumulation
 *                    truncates; this keeps its bias about six times smaller
 *                    (128-column tiles, same arithmetic otherwise).
 *   DS_PREC_F16X10 : the Tucker group on F (the stiff, large right-hand side
 *                    of Algorithm 1/2) with ~35-bit operands on the tensor
 *                    cores; the groups on D2, D3 as DS_PREC_BF16X6.  F and
 *                    every intermediate of that group are held as four FP16
 *                    parts x = 2^E (h + s1 + s2 + s3) with a fixed-point head
 *                    h (a multiple of 16, |h| <= 2^11 nominally) and a
 *                    fixed-point s1 (a multiple of 2^-7), E one exponent per
 *                    tensor set; each phi-matrix row has its own exponent.
 *                    Ten partial products run on the tensor cores, summed in
 *                    four FP32 tensor-memory accumulators by weight class
 *                    (head x head, where the sum is exact; the two products
 *                    with s1; the three of weight ~2^-16; the four below)
 *                    and combined in double-float, so the accumulators'
 *                    truncation acts on small partial sums only.
 *                    F = K U + g(U) is formed in double-float.  A plan sets
 *                    each E from the largest magnitude the previous step
 *                    wrote, never more than 10 below the largest E since the
 *                    state's calibrating step (a tensor that settles far
 *                    below its early size keeps a precision floor instead of
 *                    following it down); the first step on a state pointer
 *                    (of ds_step, ds_integrate or a batch) is that
 *                    calibrating step: it measures every tensor before
 *                    writing it.  The parts stay exact up to 2^16 times 2^E,
 *                    so a tensor may grow ~32x within one step (beyond 16x
 *                    its head products lose their exact sum for that step);
 *                    a value beyond the FP16 range of its parts makes
 *                    ds_plan_sync report DS_ERR_NONFINITE.  d = 2 or 3,
 *                    fewer than 2^31 points.
 *   DS_PREC_F16X13 : the FX operands of DS_PREC_F16X10 for all three Tucker
 *                    groups (F, D2, D3), with thirteen partial products (the
 *                    ten above plus s1 s3', s3 s1' and s2 s2' in the fourth
 *                    accumulator), every stage increment kept as a
 *                    double-float (the FP32 value plus its rounding residual)
 *                    and the stage differences g(U_s) - g(U) and the final
 *                    update formed in double-float (separate stage kernels;
 *                    the D planes are FX tensors with their own exponents).
 *                    For problems whose dynamics amplify every rounding
 *                    (Turing growth), where the FP32-class parts of
 *                    DS_PREC_F16X10 dominate. */
typedef enum {
    DS_PREC_F64 = 0,
    DS_PREC_BF16X6 = 1,
    DS_PREC_F32 = 2,
    DS_PREC_BF16X6C = 3,
    DS_PREC_F16X10 = 4,
    DS_PREC_F16X13 = 5
} ds_precision;

/* Reaction term g of the two-component systems (Section 3).
 *   DS_SCHNAKENBERG, p = (gamma, a, b):
 *       g_u = gamma (a - u + u^2 v),  g_v = gamma (b - u^2 v)   (Sect. 3.1)
 *   DS_FHN (FitzHugh-Nagumo), p = (eps, alpha1, alpha0):
 *       g_u = u - u^3 - v,            g_v = eps (u - alpha1 v - alpha0)
 *       (the Section 3.2 model with the reaction written in this form)
 *   DS_LINEAR: g = 0 (pure linear problem; used to check against exp(tau K)). */
typedef enum { DS_SCHNAKENBERG = 0, DS_FHN = 1, DS_LINEAR = 2 } ds_model;

/* Grid: d in {2, 3, 4}; n[0] = n_1 (fastest) ... n[d-1] = n_d; n_mu >= 2. */
typedef struct {
    int32_t d;
    int64_t n[4];
} ds_grid;

typedef struct {
    int32_t model;   /* ds_model */
    double p[8];     /* model parameters, see ds_model */
} ds_params;

/* Time-stepping scheme of a phi-set (and of the plans built on it).
 *   DS_EXPRK3DS_REAL: third-order EXPRK3 (Section 2.4, eq. exprk3) with the
 *     Table 1 (d = 2) / Table 3 (d = 3, 4) splits -- Algorithms 1 and 2.
 *   DS_ETD2RKDS: second-order ETD2RK (Section 1, eq. ETD2RK) with the
 *     second-order split phi_l(tau K) ~ l!^(d-1) (x)_mu phi_l(tau A_mu)
 *     (Section 2, eq. secondord); FP64 plans only.
 *   DS_EXPRK3DS_CPLX: EXPRK3 with the complex two-term split of Table 2
 *     (Section 2.2, Algorithm 1); each split action is complex and its real
 *     part is the increment; phi of complex multiples of A via the real
 *     2n x 2n embedding [[Re, -Im], [Im, Re]]; FP64 plans only.
 *   DS_EXPRK3_DENSE: the unsplit EXPRK3 (Section 2.4, eq. exprk3) that the
 *     splits approximate: K_c = A_{c,d} (+) ... (+) A_{c,1} is assembled as a
 *     dense N x N matrix (N = prod n_mu <= 4096) and phi_l(c tau K_c) is
 *     formed densely (same Taylor + modified squaring), so a run of it next
 *     to an EXPRK3DS_REAL run measures the splitting error; FP64 plans only,
 *     no adjoint.  ds_phi_get/_ex return the N x N matrix of (c, slot) with
 *     term = mu = 0. */
typedef enum { DS_EXPRK3DS_REAL = 0, DS_ETD2RKDS = 1, DS_EXPRK3DS_CPLX = 2, DS_EXPRK3_DENSE = 3 } ds_scheme;

typedef struct ds_phi_set ds_phi_set;
typedef struct ds_plan ds_plan;

/* ds_phi_setup -- the "Needed phi-functions" block of Algorithms 1 and 2.
 *   For component c in {0, 1}, direction mu, term i (k = 2 terms for d = 2,
 *   3 for d >= 3) it forms, in FP64 on the GPU (scheme DS_EXPRK3DS_REAL; see
 *   ds_phi_setup_ex for the others),
 *     P_{i,2}^{(1)}{mu} = phi_{l_i}(tau/3  alpha_{i,mu}^{(1)} A_{c,mu})
 *     P_{i,3}^{(l)}{mu} = phi_{l_i}(2tau/3 alpha_{i,mu}^{(l)} A_{c,mu}), l = 1, 2
 *     P_{i,f}^{(l)}{mu} = phi_{l_i}(tau    alpha_{i,mu}^{(l)} A_{c,mu}), l = 1, 2
 *   with the coefficients of Table 1 (real, "+" sign, d = 2) or Table 3
 *   (d >= 3, eta_2 times 2^(d-3)) (Section 2.4 fixes the "+" choice), by scaling, a degree-16
 *   Taylor series and the modified squaring of Skaflestad & Wright
 *   (the paper's [SW09]; Section 2.4 uses it with a Pade core).
 *   A: for c = 0, 1 and mu = 0..d-1, in that order, the column-major
 *      n_mu x n_mu matrix A_{c,mu}, concatenated (2 sum_mu n_mu^2 doubles).
 *      a_on_device = 0: host memory; 1: device memory.
 *   tau: time step, > 0.
 *   *out: receives a library-owned phi-set (device FP64 matrices plus a copy
 *      of A).  Synchronous: returns after the set is complete.
 *   Errors: DS_ERR_INVALID_ARG (d, n, tau, NULL), DS_ERR_NONFINITE (A has
 *   NaN/Inf), DS_ERR_OOM, DS_ERR_CUDA. */
ds_status ds_phi_setup(const ds_grid *grid, const double *A, int a_on_device,
                       double tau, ds_phi_set **out, void *stream);

/* ds_phi_setup_ex -- ds_phi_setup for a given ds_scheme.  For
 * DS_ETD2RKDS the set holds, per component and direction, slot 0 =
 * phi_1(tau A_{c,mu}) and slot 1 = phi_2(tau A_{c,mu}) (one "term" each);
 * a plan on it performs
 *   U2 = U + tau T(F, {phi_1}),  U <- U2 + tau 2^(d-1) T(g(U2) - g(U), {phi_2}). */
ds_status ds_phi_setup_ex(const ds_grid *grid, const double *A, int a_on_device, double tau,
                          int scheme, ds_phi_set **out, void *stream);

/* Release a phi-set (NULL is accepted).  Plans created from it must be
 * destroyed first. */
ds_status ds_phi_set_destroy(ds_phi_set *set);

/* Copy one phi-matrix to host memory (column-major n_mu x n_mu), for
 * inspection and tests.  slot: 0 = P_{i,2}^{(1)}, 1 = P_{i,3}^{(1)},
 * 2 = P_{i,3}^{(2)}, 3 = P_{i,f}^{(1)}, 4 = P_{i,f}^{(2)}.  Synchronous. */
ds_status ds_phi_get(const ds_phi_set *set, int c, int slot, int term, int mu,
                     double *host_out);

/* ds_phi_get_ex -- as ds_phi_get, choosing the part: 0 = the phi-matrix
 * (real part for DS_EXPRK3DS_CPLX), 1 = imaginary part (complex scheme only),
 * 2 = its derivative d/ds phi_l(s Z) at s = 1 (real schemes).  Synchronous. */
ds_status ds_phi_get_ex(const ds_phi_set *set, int c, int slot, int term, int mu, int part,
                        double *host_out);

/* ds_tucker -- Tucker operator Y = X x_1 L_1 x_2 ... x_d L_d (Section 2,
 * eq. krontomu: equals (L_d (x) ... (x) L_1) vec(X)).
 *   X, Y: device FP64 tensors of grid's sizes; may not overlap.
 *   L: host array of d device pointers to column-major n_mu x n_mu FP64
 *      matrices (L[0] is L_1).
 *   transpose = 1 uses L_mu^T instead of L_mu (the adjoint operator).
 *   precision: DS_PREC_F64, DS_PREC_F32, DS_PREC_BF16X6, DS_PREC_BF16X6C or
 *      DS_PREC_F16X10 (the last three need n_1 % 8 == 0 and n_mu >= 8; with
 *      BF16X6/BF16X6C the intermediates and the last product are FP32, with
 *      F16X10 the intermediates are FX parts scaled by their exact largest
 *      magnitude and the last product is formed in double-float).  Y is
 *      written in FP64.
 *   Temporary device memory is allocated per call and released before the
 *   call returns (stream-ordered).
 *   Errors: DS_ERR_INVALID_ARG, DS_ERR_UNSUPPORTED (precision/shape),
 *   DS_ERR_OOM, DS_ERR_CUDA. */
ds_status ds_tucker(const ds_grid *grid, const double *X, double *Y,
                    const double *const *L, int transpose, int precision, void *stream);

/* ds_tucker_static -- the FP64 Tucker operator of ds_tucker (same result,
 * same kernels) for callers that cannot allocate device memory when they
 * need it: code running inside an allocator or memory-pool callback, hosts
 * that forbid allocation after start-up, plugins whose framework owns the
 * device heap.  The paper has no counterpart; this is a property of the
 * library, not of the method.
 *   It allocates nothing.  Its two intermediate tensors live in one fixed
 *   device array inside the library (16 MiB: two FP64 tensors of up to
 *   1,048,576 points), which every GPU that loads the library holds until
 *   the process exits.  Grids with more than 1,048,576 points are rejected
 *   with DS_ERR_INVALID_ARG; use ds_tucker for them.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it for the
 *   life of the process; make that first call before any stream capture on
 *   the device.  The kept address belongs to the device's context: after a
 *   cudaDeviceReset of a device, do not call ds_tucker_static on it again in
 *   the same process.
 *   All calls on a device share the array and it keeps the last call's
 *   contents; every intermediate is fully overwritten, so nothing needs
 *   clearing.  Calls whose work overlaps on the GPU (different streams,
 *   or host threads without ordering) race on the array and must be
 *   serialised by the caller.
 *   Arguments, layouts and the other errors are those of ds_tucker with
 *   precision DS_PREC_F64 (DS_ERR_UNSUPPORTED on a device other than
 *   sm_103).  Asynchronous on `stream`. */
ds_status ds_tucker_static(const ds_grid *grid, const double *X, double *Y,
                           const double *const *L, int transpose, void *stream);

/* ds_kronsum -- Y = K x = vec(sum_mu X x_mu A_mu) (Section 2.4,
 * eq. kronsumv), FP64, for component c of a phi-set's A.  Tridiagonal A
 * run as a (2d+1)-point stencil, others as dense mode products. */
ds_status ds_kronsum(const ds_phi_set *set, int c, const double *X, double *Y, void *stream);

/* ds_plan_create -- bind a phi-set, the reaction model and a precision into
 * a stepping plan with its device workspace.  Synchronous.
 *   Errors: DS_ERR_INVALID_ARG (grid does not match the set, unknown model),
 *   DS_ERR_UNSUPPORTED (precision for this grid: BF16X6 needs n_1 % 8 == 0
 *   and n_mu >= 16), DS_ERR_OOM. */
ds_status ds_plan_create(const ds_grid *grid, const ds_params *params,
                         const ds_phi_set *set, int precision, ds_plan **out);

/* ds_step -- one EXPRK3DS_REAL step (Algorithm 1 for d = 2, Algorithm 2
 * for d = 3 and its d = 4 extension):
 *   G = g(U), F = K(U) + G
 *   U2 = U + tau/3 S_2^{(1)}(F),  D2 = g(U2) - G
 *   U3 = U + 2tau/3 S_3^{(1)}(F) + 4tau/3 S_3^{(2)}(D2),  D3 = g(U3) - G
 *   U <- U + tau S_f^{(1)}(F) + 3tau/2 S_f^{(2)}(D3)
 * with S_s^{(l)}(X) = sum_i eta_i^{(l)} T(X, {P_{i,s}^{(l)}{mu}}).
 *   U: device FP64 two-component state (2 N doubles), updated in place.
 *   The time argument of g is not used (autonomous models). */
ds_status ds_step(ds_plan *plan, double *U, void *stream);

/* ds_integrate -- nsteps >= 0 steps of ds_step.  The step is captured once
 * into a CUDA graph (per U pointer) and replayed, so the loop makes no host
 * round trips.  Asynchronous. */
ds_status ds_integrate(ds_plan *plan, double *U, int64_t nsteps, void *stream);

/* ds_integrate_ckpt -- ds_integrate with checkpoints for reverse mode: after
 * every ckpt_every steps the state is copied (device to device, on stream)
 * into ckpt + j * 2 N, j = 0, 1, ..., i.e. checkpoint j is the state after
 * (j + 1) ckpt_every steps, for every such count <= nsteps.  ckpt: caller-
 * owned device buffer of floor(nsteps / ckpt_every) * 2 N doubles (may be
 * NULL when nsteps < ckpt_every).  ckpt_every <= 0 gives
 * DS_ERR_INVALID_ARG.  Asynchronous. */
ds_status ds_integrate_ckpt(ds_plan *plan, double *U, int64_t nsteps, int64_t ckpt_every, double *ckpt,
                            void *stream);

/* ds_step_backward -- adjoint (reverse mode) of one ds_step, for FP64
 * plans.  The paper has no adjoint; this is the exact transpose of the step
 * of Algorithms 1/2.  From U = U_n it recomputes F, U2, D2, U3 and, with
 * lam = dL/dU_{n+1}, forms
 *   lam_F  = tau S_f^{(1)T}(lam),  lam_D3 = 3tau/2 S_f^{(2)T}(lam),
 *   lam_U3 = J_g(U3)^T lam_D3,
 *   lam_F += 2tau/3 S_3^{(1)T}(lam_U3),  lam_D2 = 4tau/3 S_3^{(2)T}(lam_U3),
 *   lam_U2 = J_g(U2)^T lam_D2,  lam_F += tau/3 S_2^{(1)T}(lam_U2),
 *   lam_n  = lam + lam_U3 + lam_U2 + K^T lam_F + J_g(U)^T (lam_F - lam_D2 - lam_D3),
 * where S^T uses the transposed phi-matrices (T(X, P)^T = T(X, P^T)) and
 * J_g is the 2x2 pointwise Jacobian of the reaction.
 *   U, lam, lam_n: device FP64 two-component tensors (2 N doubles); lam_n
 *     must not alias U or lam.
 *   dparams: NULL, or a device array of 3 doubles to which dL/dp[0..2] of
 *     the model parameters is added (atomically; zero it before the sweep):
 *     (dg/dp)(U)^T (lam_F - lam_D2 - lam_D3) + (dg/dp)(U2)^T lam_D2
 *     + (dg/dp)(U3)^T lam_D3, summed over the grid.
 *   dscale: NULL, or a device array of 2 doubles to which dL/ds_c is added,
 *     s_c a relative scaling of component c's matrices (A_{c,mu} -> s_c
 *     A_{c,mu} at s_c = 1; for A = delta_c D, dL/d delta_c = dL/ds_c /
 *     delta_c).  It flows through K (<lam_F, K U>) and through every
 *     phi-matrix: d/ds phi_l(s Z) = phi_{l-1}(Z) - l phi_l(Z) (from the
 *     power series), formed once by ds_phi_setup.  Costs d extra Tucker
 *     operators per Tucker operator of the step.
 *   Errors: DS_ERR_INVALID_ARG, DS_ERR_UNSUPPORTED (non-FP64 plan), DS_ERR_OOM
 *   (first call allocates a 24 N-double workspace). */
ds_status ds_step_backward(ds_plan *plan, const double *U, const double *lam, double *lam_n,
                           double *dparams, double *dscale, void *stream);

/* ds_plan_sync -- wait for the plan's work and report device-side errors:
 * DS_ERR_TIMEOUT if a bounded wait gave up, DS_ERR_NONFINITE if check_state
 * is non-zero and U (may be NULL) holds NaN/Inf. */
ds_status ds_plan_sync(ds_plan *plan, const double *U, int check_state);

/* Number of the library's own kernel launches enqueued by the last ds_step
 * (graph replays count the kernels inside the graph). */
int64_t ds_plan_kernels_per_step(const ds_plan *plan);

/* ds_plan_profile -- when enable != 0, every later ds_step (not the graph
 * replay of ds_integrate) records a CUDA event pair around each of the
 * library's kernel launches, on the stream the kernel is launched on.  The
 * events add a few microseconds per launch. */
ds_status ds_plan_profile(ds_plan *plan, int enable);

/* ds_plan_profile_read -- wait for the recorded events and return, per
 * launch kind k (0 = tensor-core mode products, 1 = FP64 mode products,
 * 2 = pointwise kernels), the summed device time ms[k] (milliseconds), the
 * launch count launches[k] and the useful floating-point operations
 * flops[k] (2 N n_mu per mode product, FP32-class or FP64 as the kind
 * says).  Arrays have 3 entries each.  Clears the records. */
ds_status ds_plan_profile_read(ds_plan *plan, double *ms, int64_t *launches, double *flops);

/* ds_plan_profile_read_ex -- ds_plan_profile_read plus bytes[k], the summed
 * algorithmic DRAM bytes of kind k: every distinct input read once, every
 * output written once (for a split-BF16 mode product: its distinct input
 * planes, its phi-matrix planes, its output; for a pointwise kernel: the
 * state, increments and planes it touches).  Split-K partials and re-reads
 * are not counted, so measured traffic above bytes[k] is waste.  bytes may be
 * NULL; kinds without a byte model report 0. */
ds_status ds_plan_profile_read_ex(ds_plan *plan, double *ms, int64_t *launches, double *flops,
                                  double *bytes);

/* ds_plan_profile_kinds -- as ds_plan_profile_read_ex with nkinds (1..4)
 * entries per array, the tensor-core launches split by operand format:
 * kind 0 = split-BF16 mode products (six BF16 products per FP32-class
 * product), 1 = FP64 mode products, 2 = pointwise kernels, 3 = FX mode
 * products of DS_PREC_F16X10 plans (ten FP16 products per product).  The
 * three-kind reads above count kind 3 under kind 0.  flops are the useful
 * 2 N n_mu per product; bytes may be NULL.  Clears the records. */
ds_status ds_plan_profile_kinds(ds_plan *plan, int nkinds, double *ms, int64_t *launches, double *flops,
                                double *bytes);

/* ds_plan_tuning -- what the autotuner chose for the split-BF16 plan's mode
 * product launch of group (0 = the F group, 1 = D2, 2 = D3) and mode mu: the
 * split-K factor (0: stream-K, see ds_plan_streamk_times), the number of
 * output tiles, and the measured time (ms, fastest of five) of each
 * candidate factor 1..8 at the chosen tile width (0 = not tried).
 * Synchronous; DS_ERR_UNSUPPORTED for other precisions. */
ds_status ds_plan_tuning(const ds_plan *plan, int group, int mu, int *ksplit, int64_t *tiles,
                         float *times_ms);

/* ds_plan_tuning_ex -- ds_plan_tuning plus the chosen output tile width
 * tile_n (256 or 128 columns; the tiles have 128 rows) and times_ms[16]:
 * [w * 8 + k - 1] for width w (0: 256, 1: 128) and split factor k. */
ds_status ds_plan_tuning_ex(const ds_plan *plan, int group, int mu, int *ksplit, int64_t *tiles, int *tile_n,
                            float *times_ms);

/* ds_plan_streamk_times -- times_ms[2]: the measured time of the launch's
 * stream-K candidate at 256- and 128-column tiles (0 = not tried).  In
 * stream-K form one CTA per SM takes an equal contiguous share of the
 * launch's (tile, K chunk) iterations; a tile shared by several CTAs is
 * summed from their FP32 partials, in CTA order, by the last CTA to deliver
 * one, which then runs the tile's epilogue (no CTA waits for another). */
ds_status ds_plan_streamk_times(const ds_plan *plan, int group, int mu, float *times_ms);

/* ds_plan_tile_order -- the order in which the CTAs of a launch take its
 * output tiles.  Mode-1 launches (mu = 0): 0 row tiles fastest, then the
 * stacked phi-matrices, then column tiles, so that neighbouring CTAs share a
 * tile of the data; 1 column tiles fastest, so that they share a stripe of a
 * phi-matrix.  Other modes: 0 column tiles fastest (neighbouring CTAs share
 * a data tile), 1 row tiles fastest (they share a phi-matrix column block).
 * times_ms[2]: the tuner's time of each order with the chosen tile width and
 * K decomposition (0 = not tried).  Without stream-K the order changes no
 * result; with it, it moves where K sums are cut. */
ds_status ds_plan_tile_order(const ds_plan *plan, int group, int mu, int *order, float *times_ms);

/* ds_plan_set_tile_order -- override that order (0 or 1; DS_ERR_INVALID_ARG
 * otherwise).  Waits for the plan's stream and drops its captured graphs. */
ds_status ds_plan_set_tile_order(ds_plan *plan, int group, int mu, int order);

/* ds_plan_set_tiles -- override the autotuner for one launch: output tile
 * width tile_n (256 or 128) and split-K factor (1 .. the largest factor the
 * tuner considered for that width, or 0 for stream-K where the tuner offered
 * it; DS_ERR_INVALID_ARG otherwise).  The tile width does not change any
 * element's summation order; the split factor and stream-K do.  Waits for
 * the plan's stream and drops its captured graphs. */
ds_status ds_plan_set_tiles(ds_plan *plan, int group, int mu, int tile_n, int ksplit);

/* ds_plan_fusion -- for the split-BF16 plan's group (0 = F, 1 = D2, 2 = D3):
 * whether its last mode product runs with the fused epilogue (the stage
 * difference g(U_s) - G, or the final update of U, computed as the
 * contraction's output is drained) or as a plain product followed by a
 * separate stage kernel; the plan creation times both (fastest of five
 * launches, milliseconds; 0 when the choice came from DS_TUNE_CACHE) and
 * keeps the faster.  Both give the same values.  DS_ERR_UNSUPPORTED for other
 * precisions. */
ds_status ds_plan_fusion(const ds_plan *plan, int group, int *fused, float *ms_fused, float *ms_separate);

/* ds_plan_set_fusion -- override that choice for group (fused != 0: fused
 * epilogue).  Waits for the plan's stream and drops its captured graphs.
 * DS_ERR_UNSUPPORTED for precisions other than split-BF16. */
ds_status ds_plan_set_fusion(ds_plan *plan, int group, int fused);

ds_status ds_plan_destroy(ds_plan *plan);

/* Batches of independent instances (uneven grids, parameters, tau).
 * ds_batch_create -- one phi-set and plan per instance (as ds_phi_setup
 *   with host A and ds_plan_create).  grids, A, tau, params: arrays of
 *   ninst entries; A[i] is the host pointer of instance i's packed matrices
 *   (layout of ds_phi_setup).  Synchronous.
 * ds_batch_integrate -- nsteps steps of every instance; U: host array of
 *   ninst device pointers to the instances' FP64 states.  The steps are
 *   captured into CUDA graphs (up to 10 steps each, cached per set of U
 *   pointers).  Split-BF16 batches (all instances of one d): per step, each
 *   instance's F = K U + g(U) runs on its own captured stream, then each of
 *   the 3 d mode products of all instances runs as one grouped persistent
 *   launch (the instances' tiles in one work list, their arguments in a
 *   device table; 128-column tiles, with two accumulators for
 *   DS_PREC_BF16X6C; no split-K; each group's last mode with the fused
 *   epilogue or, where that timed slower, followed by one grouped stage
 *   kernel: see ds_batch_fusion).  Other precisions: each
 *   instance's steps on its own captured stream.  Asynchronous.
 * ds_batch_sync -- wait and report the first instance's device-side error.
 * ds_batch_kernels_per_step -- library kernel launches per batch step.
 * The paper has no batching; the instances are independent problems. */
typedef struct ds_batch ds_batch;
ds_status ds_batch_create(int ninst, const ds_grid *grids, const double *const *A, const double *tau,
                          const ds_params *params, int precision, ds_batch **out);
ds_status ds_batch_integrate(ds_batch *batch, double *const *U, int64_t nsteps, void *stream);
ds_status ds_batch_sync(ds_batch *batch);
int64_t ds_batch_kernels_per_step(const ds_batch *batch);

/* ds_batch_fusion -- for the grouped launches of the most recently captured
 * split-BF16 batch graph: whether group g's (0 = F, 1 = D2, 2 = D3) last
 * mode product runs with the fused epilogue or as the plain grouped product
 * followed by one grouped stage kernel over all instances' points.  Building
 * the first graph of a batch shape times both on scratch states (fastest of
 * five, milliseconds; later graphs replay the choice; 0 when it came from
 * DS_TUNE_CACHE or ds_batch_set_fusion) and keeps the faster.  Both give the same values.  DS_ERR_UNSUPPORTED before the
 * first ds_batch_integrate or for other precisions. */
ds_status ds_batch_fusion(const ds_batch *batch, int group, int *fused, float *ms_fused, float *ms_separate);

/* ds_batch_tile_order -- the tile order (as ds_plan_tile_order) of the
 * grouped mode-1 product of group g in the most recently captured
 * split-BF16 batch graph; building the first graph of a batch shape times
 * both orders (times_ms, fastest of five; 0 when replayed) and keeps the
 * faster.  DS_ERR_UNSUPPORTED before the first ds_batch_integrate or for
 * other precisions. */
ds_status ds_batch_tile_order(const ds_batch *batch, int group, int *order, float *times_ms);

/* ds_batch_set_fusion -- fix that choice for group g in graphs built from now
 * on: fused = 1 fused epilogue, 0 separate stage kernel, -1 timed (default).
 * Waits for the batch's stream and drops its captured graphs. */
ds_status ds_batch_set_fusion(ds_batch *batch, int group, int fused);
ds_status ds_batch_destroy(ds_batch *batch);

/* Message of the last failed call on this thread ("" if none). */
const char *ds_last_error(void);

/* Library version string. */
const char *ds_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DS3_DS_H */
