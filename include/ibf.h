/*
 * ibf.h -- C ABI of the GB300 (sm_103a) interpolative butterfly factorization.
 *
 * The library builds and applies the preliminary interpolative butterfly
 * factorization (IBF) of Li & Yang, arXiv 1605.03616, Sec. 3, of the
 * complementary low-rank kernel K(x, xi) = exp(2 pi i Phi(x, xi)) on
 *   X     = N points in [0,1)        (eq. X: x_j = j/N, or caller-given points),
 *   Omega = {xi_k = k - N/2 : k = 0..N-1}  (eq. Omega),
 * so that  u = K g  (eq. DFIO: u(x) = sum_{xi in Omega} K(x, xi) g(xi))  costs
 * O(r^2 N log N) instead of O(N^2).  The factorization is
 *   K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^1)^* (V^0)^*       (Sec. 3)
 * with L = log2 N levels, switch level h = floor(L/2), and r Chebyshev points
 * per box (Sec. 2.1).  All computation happens in CUDA kernels on the current
 * device; there is no CPU fallback.
 *
 * Conventions shared by every call:
 *   - Return value: IBF_OK (0) or one of the IBF_ERR_* codes below.  No call
 *     aborts the process.  ibf_get_last_error() returns a message for the last
 *     failure of the calling thread.
 *   - Complex vectors are interleaved (re, im).  Their element type follows the
 *     plan's dtype: complex128 (two doubles) for IBF_C128, complex64 (two
 *     floats) for IBF_C64_FP32, IBF_C64_TF32X3 and IBF_C64_BF16X3.
 *   - Multi-vector arguments are column-major: column c of an n x nrhs array
 *     starts at element n*c.
 *   - Streams are CUDA streams (cudaStream_t); NULL is the legacy default
 *     stream.  Apply calls are asynchronous on that stream and do not
 *     synchronize the host; they allocate nothing, except the first
 *     ibf_apply_host call on a plan (its staging buffers, see there).
 */
#ifndef IBF_GB300_H
#define IBF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle; identical to cudaStream_t. */
typedef struct CUstream_st* ibf_stream_t;

/* Opaque plan.  Owns all device memory of the factorization and the
 * workspace used by the apply calls. */
typedef struct ibf_plan ibf_plan;

enum ibf_status {
    IBF_OK = 0,
    IBF_ERR_INVALID = 1,     /* bad argument (sizes, pointers, ids)             */
    IBF_ERR_OOM = 2,         /* device allocation failed                         */
    IBF_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed      */
    IBF_ERR_UNSUPPORTED = 4, /* valid request this build does not implement      */
    IBF_ERR_TIMEOUT = 5      /* a bounded device-side wait expired               */
};

/* Phase functions Phi(x, xi) (Assumption 1.1: homogeneous of degree 1 in xi). */
enum ibf_phase {
    IBF_PHASE_NUFFT = 0,        /* Phi = x . xi  (Sec. 6.1, eq. 1D-FT with K = e(+x xi))  */
    IBF_PHASE_FIO1D = 1,        /* Phi = x xi + c(x)|xi|, c = (2 + sin 2 pi x)/8
                                   (Sec. 6.2, eq. 1D-FIO-kernal)                       */
    IBF_PHASE_FIO2D = 2,        /* Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2) with
                                   c1 = (2 + sin 2 pi x1 sin 2 pi x2)/16,
                                   c2 = (2 + cos 2 pi x1 cos 2 pi x2)/16 (Sec. 6.3's
                                   form; the paper prints /32).  d = 2 only.
                                   IBF_PHASE_NUFFT and IBF_PHASE_SEPARABLE also
                                   have 2D forms: x.xi and 0.75 sin(2 pi x1)
                                   cos(2 pi x2) + 0.125|xi| + 0.3 sin(0.1 xi1 -
                                   0.07 xi2).                                         */
    IBF_PHASE_FIO1D_SERIES = 4, /* Phi = x xi + c(x)|xi| with a caller-given
                                   coefficient c(x) = sum_{m<M} a_m cos(2 pi m x)
                                   + b_m sin(2 pi m x) (ibf_options.phase_coef,
                                   phase_ncoef): the 1D FIOs of Assumption 1.1
                                   with a smooth periodic c; Sec. 6.2's phase is
                                   a_0 = 1/4, b_1 = 1/8.  d = 1 only.              */
    IBF_PHASE_FIO2D_SERIES = 5, /* Phi = x.xi + sqrt(c1^2 xi1^2 + c2^2 xi2^2), the
                                   generalized-Radon form of Sec. 6.3 (Sec. 1 names
                                   the class), with caller-given coefficients
                                   c_d(x) = sum_{t<M} al_{d,t} cos(2 pi (p_t x1 + q_t x2))
                                   + be_{d,t} sin(2 pi (p_t x1 + q_t x2)), d = 1, 2
                                   (ibf_options.phase_coef, phase_ncoef).  Each c_d
                                   must be bounded away from zero by its terms: the
                                   sum of al_{d,t} over the terms with p_t = q_t = 0
                                   must exceed the sum of |al_{d,t}| + |be_{d,t}|
                                   over the others (then Phi is smooth in xi away
                                   from 0, Assumption 1.1), else IBF_ERR_INVALID.
                                   Sec. 6.3's c1, c2 (constants /16) are the rows
                                   (0, 0, 1/8, 0, 1/8, 0), (1, -1, 1/32, 0, 1/32, 0),
                                   (1, 1, -1/32, 0, 1/32, 0).  d = 2 only.        */
    IBF_PHASE_SEPARABLE = 100   /* test phase f(x) + h(xi), f = 0.75 sin 2 pi x,
                                   h = 0.125|xi| + 0.3 sin(0.1 xi); the remainder
                                   R^{AB} of eq. RAB vanishes, so the IBF is exact    */
};

/* Arithmetic of the apply. */
enum ibf_dtype {
    IBF_C128 = 0,       /* complex128 in and out, FP64 factors and FP64 arithmetic  */
    IBF_C64_FP32 = 1,   /* complex64 in and out, FP32 factors, FP32 arithmetic      */
    IBF_C64_BF16X3 = 2, /* complex64 in and out, three-term split-BF16 tensor-core
                           products with FP32 accumulation: not built -- plan
                           creation returns IBF_ERR_UNSUPPORTED (IBF_C64_TF32X3
                           is the tensor-core form that is built)                */
    IBF_C64_TF32X3 = 3  /* complex64 in and out, FP32 factors (structured form,
                           d = 1); the transfer products of the G-form levels
                           (forward G levels, adjoint H levels) of 32-column
                           tiles run on the tensor cores (tcgen05, kind::tf32)
                           with both operands split in two TF32 terms and three
                           products kept, FP32 accumulation in tensor memory;
                           everything else as IBF_C64_FP32                       */
};

/* Storage form of the factors. */
enum ibf_form {
    IBF_FORM_AUTO = 0,       /* EXPLICIT for IBF_C128, STRUCTURED otherwise             */
    IBF_FORM_EXPLICIT = 1,   /* every r x r block of V^0, H^l, M^h, G^l, U^L stored
                                as in Sec. 3; one kernel per level (the plain form).
                                IBF_C128, or IBF_C64_FP32: built in FP64, stored and
                                applied in FP32 (also for the optimal forms)          */
    IBF_FORM_STRUCTURED = 2, /* each butterfly block stored as diag * T_c * diag with
                                the two universal real Lagrange transfer matrices T_c
                                and the diagonal phases of adjacent levels merged;
                                several levels fused per kernel                       */
    IBF_FORM_OPTIMAL = 3,    /* the optimal IBF after the sweep-out stage of Sec. 4.2:
                                the explicit factors compressed from the middle level
                                outward (eqs. KeqUCMRV, GC, HR) to blocks of rank
                                ibf_options.rank by truncated SVDs, applied like the
                                explicit form.  IBF_C128 or IBF_C64_FP32 (the
                                compression runs in FP64 either way), d = 1, r <= 12. */
    IBF_FORM_OPTIMAL_IN = 4  /* IBF_FORM_OPTIMAL followed by the sweep-in stage of
                                Sec. 4.3 (eq. IBFin): the outer factors compressed
                                toward the middle, each block to the number of points
                                its boxes hold (capped at the rank), so the operator is
                                unchanged to rounding and the outer levels shrink
                                (1 x 1 leaf factors with one point per leaf).  Same
                                limits as IBF_FORM_OPTIMAL.                           */
};

/* Optional plan parameters; zero-initialise and set what you need. */
typedef struct ibf_options {
    int form;              /* enum ibf_form                                         */
    int h;                 /* switch level in [1, L-1]; <= 0 means floor(L/2)        */
    int max_nrhs;          /* columns of the apply workspace; larger nrhs is
                              processed in slices of max_nrhs.  <= 0: 64 for the
                              structured form, 8 for the explicit and optimal
                              forms.                                               */
    int levels_per_launch; /* structured form: butterfly levels fused per kernel
                              (1..10); <= 0 lets the autotuner choose              */
    int rhs_tile;          /* structured form: right-hand sides per CTA (1..64,
                              power of two); <= 0 lets the autotuner choose        */
    int rank;              /* optimal form: rank r0 of every compressed block,
                              1..r (the paper's r0); ignored by the other forms    */
    const double* phase_coef; /* IBF_PHASE_FIO1D_SERIES: 2 M host doubles, a_0..a_{M-1}
                              then b_0..b_{M-1}.  IBF_PHASE_FIO2D_SERIES: 6 M host
                              doubles, rows (p_t, q_t, al_{1,t}, be_{1,t}, al_{2,t},
                              be_{2,t}).  Copied at creation; all finite.         */
    int phase_ncoef;       /* the series phases: M, 1..16                          */
} ibf_options;

/*
 * ibf_plan_create -- build the preliminary IBF (Sec. 3) for the uniform grid
 * X = {j/N} (eq. X) and Omega = {k - N/2} (eq. Omega).
 *   phase_id : enum ibf_phase.
 *   d        : dimension, 1 or 2.  d = 2 builds the multiscale IBF of
 *              Sec. 5.2 on the n x n grids X = {(n1, n2)/n} and
 *              Omega = {(k1 - n/2, k2 - n/2)}, N = n^2: the frequency square is
 *              split into corona rings -- ring t is the 12 outer boxes (side
 *              n/2^(t+2)) of the 4 x 4 partition of [-n/2^(t+1), n/2^(t+1))^2
 *              -- down to a 16 x 16 centre that is summed directly; every box
 *              gets a 2D butterfly of depth log2(side) switching at
 *              ceil(depth/2) (Sec. 5.1).  2D plans: structured form, r in
 *              {5, 7, 9}, the grid X only (x = NULL); apply and adjoint.
 *              Vectors are n x n row-major in (n1, n2) and (k1, k2).
 *   N        : number of points, a power of two, 4 <= N <= 2^24 (d = 1), or
 *              n^2 with n a power of two, 32 <= n <= 2048 (d = 2).
 *   r        : Chebyshev points per box (the paper's r_eps), 3 <= r <= 16;
 *              the structured form supports r in {5, 7, 9, 11}.
 *   dtype    : enum ibf_dtype.
 *   out      : receives the plan; *out is NULL on failure.
 * Construction evaluates every phase in FP64 on the current device and
 * stream 0, and synchronizes before returning.  The caller owns the plan and
 * frees it with ibf_plan_destroy.
 */
int ibf_plan_create(int phase_id, int d, int64_t N, int r, int dtype, ibf_plan** out);

/*
 * ibf_plan_create_ex -- as ibf_plan_create, with caller-given target points.
 *   x   : host array of N doubles in [0,1) (the rows of K, in the caller's
 *         order; they need not be sorted and a leaf box may hold any number of
 *         them, Sec. 2.2), or NULL for the uniform grid.  Copied; the caller
 *         keeps ownership.
 *   opt : options, or NULL for the defaults.
 */
int ibf_plan_create_ex(int phase_id, int d, int64_t N, int r, int dtype, const double* x,
                       const ibf_options* opt, ibf_plan** out);

/*
 * ibf_apply -- u = K g with the IBF factors (Sec. 3: V^0, H^1..H^h, M^h,
 * G^h..G^{L-1}, U^L in that order).
 *   g    : device array, N x nrhs column-major; column c holds g(xi_k) at
 *          element k + N c, xi_k = k - N/2.
 *   u    : device array, N x nrhs column-major, in the caller's x order.
 *          Overwritten.  Must not overlap g.
 *   nrhs : number of columns, >= 1.
 * Both pointers must be aligned to their element size.  Asynchronous on
 * `stream`; uses the plan's workspace, so calls on one plan must be ordered
 * (same stream or explicit synchronisation).
 */
int ibf_apply(ibf_plan* plan, const void* g, void* u, int nrhs, ibf_stream_t stream);

/*
 * ibf_apply_adjoint -- g = K^* y, the conjugate-transposed factors in reverse
 * order: V^0 H^1 ... H^h (M^h)^* (G^h)^* ... (G^{L-1})^* (U^L)^*.  The paper
 * gives only the forward product (Sec. 3); this is its exact adjoint.  For a
 * 2D plan it is the adjoint of the multiscale sum (Sec. 5.2): the direct
 * centre sum transposed, and per corona box its butterfly steps transposed,
 * each box writing its own frequencies of g.
 *   y : device array N x nrhs (rows in the caller's x order).
 *   g : device array N x nrhs (rows xi_k).  Overwritten.
 * Same layout, alignment and stream rules as ibf_apply.
 */
int ibf_apply_adjoint(ibf_plan* plan, const void* y, void* g, int nrhs, ibf_stream_t stream);

/*
 * ibf_apply_host -- u = K g or g = K^* y (bit 0 of `flags`, IBF_HOST_ADJOINT) with
 * both vectors in host memory (same column-major layouts as ibf_apply and
 * ibf_apply_adjoint).  The paper applies the factors to resident vectors; this
 * is the transfer-overlapped form of the same apply for data that lives on
 * the host.  The columns are processed in chunks of the plan's rhs tile
 * (16 for 2D and explicit plans): while chunk j is applied on `stream`,
 * chunk j+1 is copied in and chunk j-1 copied out on two copy streams owned
 * by the plan, ordered by events.
 *   in_host, out_host : host arrays N x nrhs; page-locked memory
 *          (cudaHostAlloc / cudaHostRegister) lets the copies run
 *          asynchronously and overlap, pageable memory works but serialises.
 *          Must stay valid and untouched until `stream` has completed.
 * The first call on a plan creates its staging buffers (4 N chunk elements on
 * the device), copy streams and events: make it outside stream capture.
 * Returns once the work is queued; out_host is complete when `stream` is.
 * Calls on one plan must be ordered on `stream`.  Errors as ibf_apply;
 * IBF_ERR_OOM if the staging buffers cannot be allocated, IBF_ERR_INVALID
 * for unknown flag bits.
 *   flags : IBF_HOST_ADJOINT (1) applies K^*; IBF_HOST_PIPELINE (2) declares
 *          that in_host is written only by the host (no earlier work queued
 *          on `stream` produces it).  Without it the first copy-in waits for
 *          all earlier work on `stream`; with it the copy-in of a chunk waits
 *          only until its staging buffer is free (the previous call's last
 *          apply that read it, and that call's copy-outs when its out_host
 *          overlaps this call's in_host), so back-to-back calls overlap the
 *          copy-in of one with the last apply of the other.  `stream` still
 *          completes only after every copy-out of the call.
 *          IBF_HOST_DEFER (4), for a stream of calls: `stream` is not made to
 *          wait for this call's copy-outs, so the last chunk's copy-out runs
 *          under the next call's applies.  out_host is then complete once
 *          `stream` has completed after a later call on the plan without the
 *          flag, or after ibf_host_flush; a later call's applies wait for the
 *          copy-outs still reading the staging buffer they write.
 */
enum { IBF_HOST_ADJOINT = 1, IBF_HOST_PIPELINE = 2, IBF_HOST_DEFER = 4 };
int ibf_apply_host(ibf_plan* plan, const void* in_host, void* out_host, int nrhs, int flags,
                   ibf_stream_t stream);

/*
 * ibf_host_flush -- orders `stream` after every copy-out of the plan's
 * host applies still outstanding (those of calls made with IBF_HOST_DEFER):
 * their out_host arrays are complete once `stream` has completed.  No effect
 * when nothing is outstanding.  IBF_ERR_INVALID for a NULL plan.
 */
int ibf_host_flush(ibf_plan* plan, ibf_stream_t stream);

/*
 * ibf_apply_amplitude -- u = A g (adjoint = 0) or g = A^* y (adjoint = 1) for
 * the kernel with a non-unit amplitude, A(x, xi) = a(x, xi) exp(2 pi i
 * Phi(x, xi)) (eq. FIO).  The paper sets a = 1 after noting that a smooth
 * amplitude is numerically low rank jointly on X x Omega (Sec. 1); the
 * caller supplies that low-rank form, a(x, xi) = sum_{t<q} alpha_t(x)
 * beta_t(xi), and
 *   A   = sum_t diag(alpha_t) K diag(beta_t),
 *   A^* = sum_t diag(conj beta_t) K^* diag(conj alpha_t),
 * with K the plan's phase-only operator, applied by ibf_apply /
 * ibf_apply_adjoint (any form, 1D or 2D).
 *   alpha : device array N x q column-major; column t holds alpha_t at the
 *           points in the caller's x order.
 *   beta  : device array N x q column-major; column t holds beta_t(xi_k).
 *   in, out : as ibf_apply (adjoint = 0: g -> u) or ibf_apply_adjoint
 *           (adjoint = 1: y -> g).  out is overwritten.
 *   work  : caller-owned device scratch of work_elems elements of the plan's
 *           element type, work_elems >= 2 N nrhs.  The terms are processed in
 *           passes of m = min(q, floor(work_elems / (2 N nrhs))) terms: per
 *           pass one scaling kernel, the phase-only apply on m nrhs columns,
 *           one accumulation kernel.  2 N q nrhs elements take one pass.
 * Allocates nothing; asynchronous on `stream`; calls on one plan must be
 * ordered.  Errors: IBF_ERR_INVALID for a NULL plan or pointer, q < 1,
 * nrhs < 1, a pointer not aligned to the element size, work_elems below
 * 2 N nrhs, m nrhs above INT_MAX, out overlapping in, alpha or beta, or the
 * used part of work overlapping any other argument; otherwise as ibf_apply.
 */
int ibf_apply_amplitude(ibf_plan* plan, const void* alpha, const void* beta, int q, const void* in, void* out,
                        int nrhs, int adjoint, void* work, int64_t work_elems, ibf_stream_t stream);

/*
 * ibf_apply_static_scratch -- u = K g like ibf_apply, for callers that may
 * not allocate device memory once their plans exist (for example a plug-in
 * whose host application owns the device heap and forbids further cudaMalloc
 * calls, or a server whose memory budget was fixed when its plans were
 * built).  The paper has no counterpart: this is an operational variant of
 * the structured-form apply.
 *
 * It allocates nothing.  Its two Lambda buffers live in one file-scope
 * device array of 256 MiB (two halves of 128 MiB); the plan's own workspace
 * is not used, so a plan created with max_nrhs = 1 still applies many
 * columns per launch here.  Creating a 1D structured plan sets this entry
 * point up on the plan's device: it looks up the array's device address
 * (cudaGetSymbolAddress, which makes that device commit the 256 MiB, held
 * until the process exits) and copies the transfer weights for the plan's r
 * and precision.  A call on a device where no 1D structured plan of that r
 * and precision was created does this set-up itself, with synchronous CUDA
 * calls: make such a call before any stream capture.  The set-up is guarded
 * by a lock.  Every call shares the array and it keeps the last call's
 * contents; no part of it needs to start at zero because each launch writes
 * every element the next launch reads.  Calls that overlap on the GPU (other
 * streams, or other threads) race on the array: order them.
 *   plan : a 1D structured-form plan (IBF_FORM_STRUCTURED, d = 1); a 2D plan
 *          or another form returns IBF_ERR_UNSUPPORTED before any CUDA call.
 *   g, u, nrhs, stream : as ibf_apply.
 * Size limit: N * r * (element size) must not exceed 128 MiB (one Lambda
 * column per half), else IBF_ERR_INVALID with a message naming the limit;
 * e.g. complex64 with r = 9 allows N <= 2^20, complex128 N <= 2^19.  The
 * columns are processed in chunks of as many as one half holds.
 */
int ibf_apply_static_scratch(const ibf_plan* plan, const void* g, void* u, int nrhs, ibf_stream_t stream);

/*
 * Batched apply of many plans of uneven size in few launches.  The paper
 * applies one IBF at a time (Sec. 3); a batch runs the same factor products
 * for many independent plans together.
 *
 * ibf_batch_create binds `count` structured-form plans (same dtype and r),
 * their right-hand-side counts nrhs[b] >= 1 and device buffers in[b] (input,
 * N_b x nrhs[b] column-major: g for the forward apply, y for the adjoint) and
 * out[b] (output, same shape, overwritten); adjoint != 0 makes the batch
 * compute K_b^* y_b instead of K_b g_b.  The batch owns a workspace of
 * sum_b 2 N_b r nrhs[b] complex elements and a launch table; the plans and
 * buffers must outlive it.  Synchronizes the device before returning.
 *
 * ibf_batch_apply runs the whole batch on `stream`: one launch runs fused
 * chunk p of every plan with the same level kind, rhs tile width (1, 2, ...,
 * 32) and fusion depth, so the number of launches (IBF_BQ_LAUNCHES) is
 * bounded by the number of distinct (kind, tile, depth) shapes per chunk
 * index times the largest number of chunks of any plan, independent of the
 * number of plans.  It copies nothing from the host and
 * allocates nothing, so it may be captured in a CUDA graph.  Calls on one
 * batch must be ordered.
 */
typedef struct ibf_batch ibf_batch;
int ibf_batch_create(ibf_plan* const* plans, int count, const int* nrhs, const void* const* in, void* const* out,
                     int adjoint, ibf_batch** batch);
int ibf_batch_apply(const ibf_batch* batch, ibf_stream_t stream);
enum ibf_batch_query_key { IBF_BQ_LAUNCHES = 0, IBF_BQ_WORKSPACE_BYTES = 1, IBF_BQ_COUNT = 2,
                           IBF_BQ_PERSIST_ITEMS = 3 };
int ibf_batch_query(const ibf_batch* batch, int what, int64_t* value);

/*
 * ibf_batch_apply_persistent -- the same batch in ONE launch.  Persistent CTAs
 * take work items (a CTA-sized block of one fused chunk of one plan) from a
 * device counter in chunk-major order; an item of chunk c of a plan first
 * waits until every item of that plan's chunk c-1 has finished (a device
 * counter, polled with a bounded number of spins).  Items are handed out in
 * dependency order to running CTAs only, so the waits cannot deadlock.  The
 * call resets its counters with stream-ordered memsets and launches one
 * kernel, so it can be captured in a CUDA graph.  Results equal
 * ibf_batch_apply's.
 *
 * ibf_batch_status synchronizes with the device and returns IBF_ERR_TIMEOUT
 * if a wait of the last persistent apply ran out of spins (every CTA then
 * stops early and the outputs are incomplete), else IBF_OK.
 * ibf_batch_set_wait_limit sets the spin limit (default 2^21, about a second).
 * ibf_batch_test_withhold(batch, plan, 1) is a test hook: it makes the wait of
 * that plan's second chunk unsatisfiable, so that a test can check that the
 * kernel returns with IBF_ERR_TIMEOUT instead of hanging; (..., 0) restores it.
 */
int ibf_batch_apply_persistent(const ibf_batch* batch, ibf_stream_t stream);
int ibf_batch_status(const ibf_batch* batch);
int ibf_batch_set_wait_limit(ibf_batch* batch, long long spins);
int ibf_batch_test_withhold(ibf_batch* batch, int plan, int withhold);
int ibf_batch_destroy(ibf_batch* batch);   /* NULL-safe; synchronizes the device */

/*
 * ibf_plan_autotune -- choose the structured form's launch shape (levels
 * fused per launch, right-hand sides per CTA) for applies with `nrhs`
 * columns by timing every candidate on scratch buffers (allocated and freed
 * here) on `stream`, and store the fastest in the plan (it then behaves as if
 * ibf_options.levels_per_launch / rhs_tile had been set).  Reports the choice
 * and its time per apply in milliseconds through the optional out pointers.
 * Structured plans only (else IBF_ERR_UNSUPPORTED).  Synchronizes.
 */
int ibf_plan_autotune(ibf_plan* plan, int nrhs, ibf_stream_t stream, int* levels_per_launch, int* rhs_tile,
                      float* ms);

/* Free the plan and all its device memory; NULL is accepted.  Synchronizes
 * the device first. */
int ibf_plan_destroy(ibf_plan* plan);

/* Plan facts for measurement and bookkeeping. */
enum ibf_query {
    IBF_Q_N = 0,
    IBF_Q_L = 1,
    IBF_Q_H = 2,
    IBF_Q_R = 3,
    IBF_Q_DTYPE = 4,
    IBF_Q_FORM = 5,
    IBF_Q_FACTOR_BYTES = 6,    /* device bytes of all stored factors              */
    IBF_Q_WORKSPACE_BYTES = 7, /* device bytes of the apply workspace             */
    IBF_Q_MAX_NRHS = 8,
    IBF_Q_NNZ = 9,             /* entries of the explicit factors (complex)       */
    IBF_Q_LAUNCHES = 10,       /* kernels one apply of one slice launches         */
    IBF_Q_LEVELS_PER_LAUNCH = 11,
    IBF_Q_RHS_TILE = 12,
    IBF_Q_RANK = 13            /* block rank the apply uses: r0 for the optimal
                                  form, r otherwise                               */
};
int ibf_plan_query(const ibf_plan* plan, int what, int64_t* value);

/*
 * ibf_plan_status -- the plan's sticky status, read and cleared.  Apply calls
 * are asynchronous, and a persistent batch reports an expired device-side
 * wait only through ibf_batch_status; the plan keeps the first such failure
 * so that a caller holding only the plan sees it.  Recorded: any error of an
 * apply call on this plan (ibf_apply, ibf_apply_adjoint, ibf_apply_host,
 * ibf_apply_amplitude, ibf_apply_static_scratch) returned after its
 * arguments were accepted (CUDA launch or copy failures), and
 * IBF_ERR_TIMEOUT when ibf_batch_status finds an expired wait in a batch
 * holding the plan, or when a bounded device-side wait of the plan's own
 * kernels expired (the tensor-core levels of an IBF_C64_TF32X3 plan, the
 * bulk-copy levels of a complex64 explicit or optimal plan).  Argument
 * errors are returned by the call itself and are not recorded.  Returns that
 * status (IBF_OK if none) and resets it to IBF_OK; IBF_ERR_INVALID for a
 * NULL plan.  No CUDA call except, for the plans named above, one
 * synchronous read (and reset) of the device status word.
 */
int ibf_plan_status(ibf_plan* plan);

/*
 * Per-launch timing for measurement tools.  ibf_plan_profile_begin(plan, cap)
 * makes the following apply calls record a CUDA event on their stream before
 * the first kernel and after every kernel, for up to `cap` kernels in total.
 * ibf_plan_profile_end waits for those events, writes the duration of each
 * recorded kernel in milliseconds to ms[] and its kind to kind[] (enum
 * ibf_kernel_kind), at most `cap_out` entries, stores the number of recorded
 * kernels in *count, and stops recording.  Recording adds two event records
 * per kernel and no synchronisation to the apply calls.
 */
enum ibf_kernel_kind {
    IBF_K_EXPLICIT_INIT = 0, IBF_K_EXPLICIT_LEVEL = 1, IBF_K_EXPLICIT_SWITCH = 2, IBF_K_EXPLICIT_TERM = 3,
    IBF_K_FUSED_H = 4, IBF_K_FUSED_G = 5, IBF_K_2D = 6
};
int ibf_plan_profile_begin(ibf_plan* plan, int cap);
int ibf_plan_profile_end(ibf_plan* plan, float* ms, int* kind, int cap_out, int* count);

/* Copy the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns the last status code. */
int ibf_get_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* IBF_GB300_H */
