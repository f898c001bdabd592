/*
 * rs.h — C ABI of the range-separated (RS) canonical/Tucker Newton-potential library.
 *
 * The library assembles and evaluates the N-particle Newton potential sum
 *     P(x) = sum_nu Z_nu / |x - x_nu|,      x, x_nu in [-b, b]^3            (Sec. 1, Eq. (1.1))
 * on an n x n x n grid with the range-separated tensor format of Benner, Khoromskaia and
 * Khoromskij (arXiv:1606.09218):
 *   - a sinc-quadrature Gaussian sum gives the rank-R reference canonical tensor P_R
 *     (Sec. 2.2, Eqs. (2.5)-(2.10));
 *   - P_R is split into R_l long-range and R_s short-range terms (Sec. 2.3, Eqs. (2.11)-(2.12));
 *   - the long-range sum of the N shifted references (Sec. 3.2, Eq. (3.5)) is compressed to a
 *     Tucker tensor by the reduced HOSVD (Sec. 6, Def. 6.1, Eqs. (6.1)-(6.3));
 *   - the short-range part is kept as a cumulated canonical tensor of local windows
 *     (Sec. 3.3, Defs. 3.4 and 3.6);
 *   - the RS-Tucker tensor (Def. 3.9, Eq. (3.11)) is evaluated on the full grid and at the
 *     particles, giving the interaction energy of Sec. 4.2, Eq. (4.7) / Lemma 4.1.
 *
 * Conventions common to every call:
 *   - Grid: vertex grid x_i = -b + i*h, i = 0..n-1, h = 2b/(n-1); n must be odd.
 *   - Output grid layout: C order, P[i1][i2][i3] at offset (i1*n + i2)*n + i3 (i3 fastest).
 *   - Every call returns an rs_status; nothing aborts or exits.  Negative values are errors,
 *     RS_OK is success, positive values are warnings whose results are valid.
 *   - Work is asynchronous on the stream given to rs_create, except where a call says it
 *     synchronises.  Device pointers belong to the caller unless stated otherwise.
 *   - A context is not thread-safe; use one context per host thread or serialise calls.
 *
 * Typical sequence:
 *     rs_create(&cfg, stream, &ctx);                       // workspace for cfg, once
 *     rs_solve(ctx, N, xyz, Z, RS_POTENTIAL | RS_ENERGY, 0.0, P);   // per particle set
 *     rs_energy(ctx, &E);                                  // synchronises
 *     rs_report(ctx, &stats);                              // ranks, eps bound, status
 *     rs_tucker_als(ctx, 1, RS_POTENTIAL | RS_ENERGY, P);  // optional: lower ranks, same eps
 *     rs_destroy(ctx);
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RS_OK = 0,
    RS_RANK_CAPPED = 1,        /* warning: rank_cap (or the subspace width) bound before eps was met;
                                  the result is valid and rs_report gives the achieved error */
    RS_ERR_INVALID_ARG = -1,   /* bad size, null pointer, even n, R_s >= R, ... */
    RS_ERR_OUTSIDE_BOX = -2,   /* a centre outside [-b,b]^3 or a non-finite coordinate/charge */
    RS_ERR_SEPARATION = -3,    /* RS_VALIDATE_SEPARATION: two centres closer than min_sep */
    RS_ERR_OOM = -4,           /* device allocation failed */
    RS_ERR_CUDA = -5,          /* a CUDA runtime call failed; rs_last_error has the message */
    RS_ERR_TIMEOUT = -6,       /* a bounded device wait ran out */
    RS_ERR_NOT_READY = -7,     /* result requested before a successful rs_solve */
    RS_ERR_CAPACITY = -8       /* N above the context's max_particles, or more than 256 windows
                                  per round reach one 8x16x64 output tile */
} rs_status;

typedef enum {
    RS_FP64 = 0,        /* every stage in FP64 (the plain RS path) */
    RS_FP32_SPLIT = 1,  /* eigen stage in FP64-level arithmetic (double-float sums and products on
                           the FP32 units, FP32 Jacobi rotations); FP32 bulk: the core contraction
                           and the grid assembly on the tensor cores with FP16 hi/lo operands, FP32
                           accumulation folded into compensated pairs and 64-bit fixed-point sums */
    RS_FP32 = 2         /* as RS_FP32_SPLIT (serving tolerance 1e-4 against the oracle) */
} rs_precision;

/* Method parameters (Sec. 2.2-2.3, Sec. 6).  All lengths in the units of the coordinates. */
typedef struct {
    double b;            /* half-width of the box [-b,b]^3 */
    int    n;            /* grid points per axis (odd, >= 5) */
    int    R;            /* rank of the reference canonical tensor P_R (number of sinc nodes) */
    int    R_s;          /* short-range terms; the long part has R_l = R - R_s */
    double h_q;          /* sinc step: t_k = exp(u0 + k*h_q), a_k = (2/sqrt(pi)) h_q t_k */
    double u0;           /* sinc offset */
    double eps;          /* Tucker tolerance (relative Frobenius error of the long-range part) */
    int    rank_cap;     /* 0: none; otherwise the maximal Tucker rank per mode */
    int    max_rank;     /* 0: default 128; upper bound on Tucker ranks (sets workspace size) */
    double delta_rel;    /* window cut-off delta = delta_rel * P_R(0) (Sec. 2.3, criterion (A)) */
    int    precision;    /* rs_precision */
    int    snap;         /* 1: centres are moved to their nearest grid point (Sec. 3.2) */
    int    max_particles;/* capacity of the context */
} rs_config;

/* rs_solve flags */
#define RS_INPUT_HOST          1   /* xyz and Z are host pointers (copied in on the stream) */
#define RS_POTENTIAL           2   /* write the full-grid potential into potential_out */
#define RS_ENERGY              4   /* compute the interaction energy (read with rs_energy) */
#define RS_FORCES              8   /* compute the forces (read with rs_forces) */
#define RS_VALIDATE_SEPARATION 16  /* check that no two centres are closer than min_sep */
#define RS_FORCES_PAIR         32  /* with RS_FORCES: the long part of the forces from the
                                      untruncated pair kernel instead of the discrete gradient */

typedef struct rs_ctx rs_ctx;

/* Per-solve report (rs_report synchronises). */
typedef struct {
    int    N, N_nonzero;
    int    ranks[3];            /* Tucker ranks r_1, r_2, r_3 */
    int    subspace[3];         /* width of the subspace the ranks were chosen from */
    int    gamma;               /* window half-width in grid steps (n_s = 2*gamma + 1) */
    double tail_rel[3];         /* discarded side-matrix energy / total, per mode */
    double eps_bound;           /* sqrt(sum_l tail_rel[l]): the error bound used for eps */
    double P_R0, P_Rl0;         /* P_R and P_{R_l} at the origin (self-interaction terms) */
    double energy;              /* last energy (if computed) */
    int    status;              /* status of the last solve (rs_status) */
    int    kernel_launches;     /* CUDA kernels the last rs_solve (or rs_tucker_als after it) enqueued */
} rs_stats;

/* Pipeline stages timed by rs_profile_read (in this order). */
#define RS_NSTAGE 9
/* 0 factors (Sec. 2.2)       1 particles (snap, aggregate)  2 gram (Sec. 3.2 / Sec. 6 (I))
 * 3 eigen (Sec. 6 (I))       4 core (Sec. 6 (II))           5 bins (window lists)
 * 6 reconstruct (Eq. (2.3))  7 windows (Defs. 3.4, 3.6)     8 energy (Eq. (4.7)) */

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*; NULL = default
 * stream).  Allocates all device workspace for cfg (sizes grow with n^2, max_rank^3,
 * max_particles).  Errors: RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA. */
rs_status rs_create(const rs_config* cfg, void* cuda_stream, rs_ctx** out);

/* Free the context and all its device memory.  Safe on NULL. */
void rs_destroy(rs_ctx* ctx);

/* Workspace bytes a context for cfg would allocate (no allocation). */
size_t rs_workspace_bytes(const rs_config* cfg);

/* Run the whole method for N particles (Sec. 3.2-3.3 and Sec. 6):
 *   xyz (N x 3, row-major, float64) and Z (N, float64): device pointers, or host pointers
 *   with RS_INPUT_HOST;
 *   potential_out: with RS_POTENTIAL a 16-byte aligned device buffer of n^3 elements (double
 *   for RS_FP64, float otherwise), written in C order; ignored otherwise.
 * Enqueues the work on the context stream and returns without waiting (inputs must stay
 * valid until the stream reaches the solve).  Device-side input errors (outside the box,
 * non-finite values) are reported by rs_report / rs_energy.  min_sep is used only with
 * RS_VALIDATE_SEPARATION. */
rs_status rs_solve(rs_ctx* ctx, int N, const double* xyz, const double* Z, int flags,
                   double min_sep, void* potential_out);

/* Interaction energy of the last solve (Eq. (4.7) applied to the RS-Tucker tensor:
 * E = 1/2 sum_j z_j (A(x_j) - z_j P_R(0)), A the RS tensor at the particle's grid point).
 * Synchronises the stream.  RS_ERR_NOT_READY if the last solve did not ask for RS_ENERGY. */
rs_status rs_energy(rs_ctx* ctx, double* E);

/* Forces of the last solve (Sec. 4.3), F_j = -z_j grad_{x_j} of the potential of the other
 * particles at x_j, with the charged centres at their grid points:
 *   default: the discrete gradient of the RS-Tucker tensor (Eq. (4.9)): the long-range Tucker
 *     part differentiated by a one-dimensional difference operator D_h applied to its bases (the
 *     centred formula of order 8 in the interior, the same nine points shifted into the grid near
 *     its ends), the particle's own long-range term taken out, plus the windows of the other
 *     particles (Defs. 3.4, 3.6) differentiated term by term with the derivatives of the
 *     Galerkin factors.  This is the gradient of the tensor whose energy rs_energy returns;
 *     O(N r^2) work.  It differs from the gradient of the untruncated long-range sum by
 *     O(eps / h) (the difference operator weighs the discarded directions) and by the
 *     difference formula's error (below 1e-7 of the forces on the bundled workloads).
 *   with RS_FORCES_PAIR: the long part from the untruncated long-range pair kernel, grad P_l(x_j) =
 *     sum_{nu != j} z_nu sum_{k long} grad (p_k x p_k x p_k)(x_j - x_nu) (exact for P_l, O(N^2 R_l)
 *     work), the windows as above.
 * F: N x 3 row-major float64, a device pointer, or a host pointer with to_host != 0; particles
 * with zero charge get zero force.  Synchronises the stream.  RS_ERR_NOT_READY if the last solve
 * did not ask for RS_FORCES; device-side input errors as for rs_energy. */
rs_status rs_forces(rs_ctx* ctx, double* F, int to_host);

/* Synchronise and fill *st for the last solve; returns that solve's status. */
rs_status rs_report(rs_ctx* ctx, rs_stats* st);

/* Device pointers to the RS-Tucker long-range part of the last solve (valid until the next
 * rs_solve or rs_destroy; synchronises to read the ranks):
 *   V[l]: n x ld_V column block, row-major (V[l][i*ld_V + a], a < ranks[l]), orthonormal columns;
 *   beta: core, beta[(a*ld_b + b)*ld_b + c];  dtype double for RS_FP64, float otherwise. */
rs_status rs_get_tucker(rs_ctx* ctx, int ranks[3], int* ld_V, int* ld_b,
                        const void* V[3], const void** beta);

/* Device pointers to the short-range part of the RS-Tucker tensor of the last solve
 * (Def. 3.9): the uniform cumulated canonical tensor of Def. 3.6, one local reference tensor of
 * R_s canonical terms on a window of n_s = 2 gamma + 1 grid points per axis (Def. 3.4, the window
 * width of Sec. 2.3, criterion (A)), shifted to every centre and weighted by its charge:
 *   W[i1][i2][i3] = sum_nu z_nu sum_{k < R_s} f_k[i1 - j1 + gamma] f_k[i2 - j2 + gamma] f_k[i3 - j3 + gamma]
 * over the centres nu with |i_l - j_l| <= gamma in every mode (j = the centre's grid indices).
 * Together with rs_get_tucker this is the whole RS-Tucker state (storage r1 r2 r3 + 3 n r +
 * R_s n_s + 4 N numbers).  Outputs (valid until the next rs_solve or rs_destroy; synchronises to
 * read gamma):
 *   *n_s, *R_s: window width and number of short-range terms;  *N: centres of the last solve;
 *   factors: FP64 table of R_s rows, row k at factors + k * (*ld_f), entries n_s: the Galerkin
 *            factors p_k (Eq. (2.5)) of the R_s short-range sinc nodes at the offsets
 *            -gamma..gamma (in every precision);
 *   grid_idx: int32 N x 3 row-major, the snapped grid indices of the centres (Sec. 3.2);
 *   charges: FP64 N, the charges as given (zero charges add nothing).
 * The buffers belong to the context.  Errors: RS_ERR_INVALID_ARG (null pointer),
 * RS_ERR_NOT_READY (no solve), RS_ERR_CUDA. */
rs_status rs_get_windows(rs_ctx* ctx, int* n_s, int* R_s, int* N, const double** factors, int* ld_f,
                         const int** grid_idx, const double** charges);

/* Evaluate the RS-Tucker tensor of the last solve at M grid multi-indices (Lemma 3.10):
 * idx: device int32 array (M x 3), out: device double array (M).  Asynchronous. */
rs_status rs_eval_points(rs_ctx* ctx, int M, const int* idx, double* out);

/* RS-canonical form (Def. 3.7) of the last solve: its long-range Tucker part converted to a
 * canonical tensor sum_k xi_k u1_k (x) u2_k (x) u3_k by the singular value decomposition of every
 * mode-1 slice of the core, beta[a,:,:] = sum_m s x y^T (FP64 one-sided Jacobi, one CTA per
 * slice), with the smallest s^2 discarded while their sum stays <= eps^2 ||beta||_F^2 and
 * u1 = V1[:, a], u2 = V2 x, u3 = V3 y, xi = s for the rest (the Frobenius error of the long part
 * is then at most eps ||beta||_F = eps ||P_l^T||_F).  Sec. 3 reports RS-canonical ranks after
 * such a Tucker-to-canonical step; the slice SVD is this library's reading of its algorithm.
 * eps >= 0; *rank receives R*.  The first call allocates the form's device memory
 * (3 n r1 r3 + O(rmax^3) doubles), kept until rs_destroy.  Ranks above RS_CANONICAL_RMAX or
 * r1 r3 above RS_CANONICAL_TERMS give RS_ERR_CAPACITY; before a solve RS_ERR_NOT_READY.
 * Synchronises.  The form is valid until the next rs_solve. */
#define RS_CANONICAL_RMAX 112
#define RS_CANONICAL_TERMS 16384
rs_status rs_canonical(rs_ctx* ctx, double eps, int* rank);

/* Point values of the RS-canonical tensor (Lemma 3.8): the canonical long part at M grid
 * multi-indices (3 R* products each) plus the windows of the neighbours.  idx: device int32
 * (M x 3, clamped to the grid), out: device double (M).  Needs rs_canonical after the last
 * solve (else RS_ERR_NOT_READY).  Asynchronous. */
rs_status rs_canonical_eval_points(rs_ctx* ctx, int M, const int* idx, double* out);

/* Device pointers to the RS-canonical form (valid until the next rs_solve or rs_canonical):
 * xi (R*), U: three side matrices, U[(l*n + i)*ld + k] for mode l, grid index i, term k < R*. */
rs_status rs_get_canonical(rs_ctx* ctx, int* rank, const double** xi, const double** U, int* ld);

/* ALS refinement of the canonical-to-Tucker transform of the last solve (Sec. 6, steps (III)-(V)).
 * It starts from the RHOSVD bases.  Each sweep updates the modes in the order l = 1, 2, 3.  Mode l
 * takes the dominant left singular vectors of M_{U_l}: the long-range canonical tensor projected
 * onto the current bases of the other two modes and reshaped to n x (r_l' r_l'').  The new rank
 * r_l is the eps rule of rs_solve applied to the singular values of M_{U_l} (the eps-truncation
 * variant of the algorithm), capped by rank_cap and max_rank.  The core is then formed from the
 * final bases (step (V)).  The mode matrices and their Gram matrices M M^T are FP64 in every
 * precision.  The eigenvectors come from the eigen stage of rs_solve, and the core from its core
 * contraction.
 *   sweeps: 1..RS_ALS_MAX_SWEEPS.  A second call continues from the refined form.
 *   flags: RS_POTENTIAL writes the refined full-grid RS-Tucker potential into potential_out (as for
 *   rs_solve).  RS_ENERGY recomputes the energy; it needs a solve that computed one.  Without
 *   RS_ENERGY, rs_energy returns RS_ERR_NOT_READY until the next solve (the old energy belonged to
 *   the RHOSVD tensor).  Forces are unchanged (they use the untruncated long-range kernel).
 * Afterwards rs_report (ranks, tail_rel of the mode matrices), rs_get_tucker, rs_eval_points and
 * rs_canonical see the refined tensor, and an earlier RS-canonical form is invalidated.
 * Synchronises: once per mode update to read the ranks, and at the end, where a device-side
 * error of the refinement (RS_ERR_TIMEOUT of a bounded wait) is returned; warnings such as
 * RS_RANK_CAPPED are left to rs_report.  The first call allocates
 * 8 (3 n R_l rmax + n rmax^2 + n K_c + K_c rmax^2) bytes of device memory (rmax the context's
 * rank bound, K_c = min(n R_l, 2^24 / rmax^2) rows of one chunk, so the last term is at most
 * 128 MiB), kept until rs_destroy.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_NOT_READY (no solve, or RS_ENERGY without a solve energy),
 * the status of a failed solve, RS_ERR_OOM (nothing changed), RS_ERR_CUDA (the solve's results are
 * withdrawn: later calls return RS_ERR_NOT_READY until the next rs_solve). */
#define RS_ALS_MAX_SWEEPS 8
rs_status rs_tucker_als(rs_ctx* ctx, int sweeps, int flags, void* potential_out);

/* Stage timing (tracing): with enable != 0, each rs_solve records one CUDA event per stage
 * boundary on the context stream (ring of 512 solves).  Errors: RS_ERR_CUDA. */
rs_status rs_profile_enable(rs_ctx* ctx, int enable);

/* Synchronise and return, per stage, the device time in milliseconds summed over the solves
 * recorded since the last read (ms: RS_NSTAGE doubles), and how many solves that was
 * (*nsolves); then restart the accumulation.  RS_ERR_NOT_READY if profiling is off. */
rs_status rs_profile_read(rs_ctx* ctx, double* ms, int* nsolves);

/* Inspection hook for tests: device pointer and size in bytes of an internal buffer of the
 * last solve ("pk64" factors R x (2n-1), "F", "G" Gram matrices 3 x n x n, "C" aggregated
 * weights 3 x n, "Q" subspace 3 x n x ksub, "T" Rayleigh quotients 3 x ksub x ksub, "Z64"
 * Tucker bases, "beta64", "Qp", "T1", "T2").  Synchronises.  RS_ERR_INVALID_ARG for an
 * unknown name.  The buffers stay owned by the context. */
rs_status rs_debug_buffer(rs_ctx* ctx, const char* name, void** ptr, size_t* bytes);

/* Static name of a stage (NULL outside [0, RS_NSTAGE)). */
const char* rs_stage_name(int stage);

/* Allocation-free Gram matrices (no counterpart in the paper; an interface for callers that
 * cannot allocate device memory).  Some callers cannot call cudaMalloc: a host application
 * that has reserved all device memory and forbids further allocation, a latency-critical
 * path where an allocation (which may synchronise the device) is not acceptable, or a
 * plug-in that may only use the memory it is given.  This call allocates nothing.  It
 * computes, on the given stream, the three n x n FP64 Gram matrices of the long-range side
 * matrices, G_l = U^(l) U^(l)^T (the same values as the context path's eigen-stage input),
 * for centres snapped to the grid of cfg (only b, n, R, R_s, h_q, u0, delta_rel are used):
 *   xyz (N x 3) and Z (N): device pointers, float64;   G: device output, 3 x n x n, C order.
 * Scratch: a fixed 16 MiB device array inside the library, held by every GPU that loads the
 * library until the process exits; problems that do not fit (n above 513, or more centres than
 * the message states) are rejected with RS_ERR_CAPACITY and a message in rs_last_error(NULL).
 * Every call looks up the array's device address (cudaGetSymbolAddress, which allocates
 * nothing) for the current device.  Every call reuses the same array, so calls that overlap on
 * the GPU (different streams, or several host threads) race: serialise them.  The call
 * synchronises the stream at its end to read the status word of the particle kernels: a centre
 * outside [-b,b]^3 or a non-finite coordinate or charge gives RS_ERR_OUTSIDE_BOX (G is then not
 * the Gram matrix of the input).  Errors: RS_ERR_INVALID_ARG, RS_ERR_OUTSIDE_BOX, RS_ERR_CAPACITY,
 * RS_ERR_CUDA. */
rs_status rs_gram_noalloc(const rs_config* cfg, int N, const double* xyz, const double* Z,
                          double* G, void* cuda_stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of solves of different N and n (no counterpart in the paper, whose
 * experiments are single solves).  rs_submit queues a request (its inputs are copied); a worker
 * thread admits queued requests to slots — a slot is a context with its own CUDA stream, kept for
 * later requests of the same configuration — when an idle slot of the configuration exists or a
 * new slot fits hbm_budget (the sum of the slots' rs_workspace_bytes, idle slots of other
 * configurations are released to make room) and at most max_slots slots exist; admitted requests
 * run concurrently.  The queue is scanned in arrival order; a request that cannot be admitted
 * yet does not hold back later ones that can.  Results match a solve of the same request alone
 * (separate workspaces and a fixed order of every floating-point sum: bit for bit). */
typedef struct rs_server rs_server;

typedef struct {
    rs_config cfg;          /* configuration; N <= cfg.max_particles */
    int    N;
    const double* xyz;      /* host, N x 3 row-major; copied by rs_submit */
    const double* Z;        /* host, N; copied by rs_submit */
    int    flags;           /* RS_ENERGY and/or RS_POTENTIAL */
    void*  potential_out;   /* with RS_POTENTIAL: caller-owned 16-byte aligned device buffer of
                               n^3 elements, valid until rs_wait returns */
} rs_request;

typedef struct {
    int    status;          /* rs_status of the solve (RS_RANK_CAPPED is a warning) */
    double energy;          /* with RS_ENERGY */
    double latency_ms;      /* rs_submit -> completion observed by the worker */
    double queue_ms;        /* rs_submit -> launch */
    int    ranks[3];
    int    slot;            /* slot index that ran the request */
    char   message[128];    /* with a negative status: the error text, NUL-terminated */
} rs_result;

/* Start a server on the current device.  Errors: RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA. */
rs_status rs_server_create(size_t hbm_budget, int max_slots, rs_server** out);
/* Queue one request; *ticket identifies it for rs_wait.  RS_ERR_CAPACITY if N > max_particles. */
rs_status rs_submit(rs_server* srv, const rs_request* req, unsigned long long* ticket);
/* Wait up to timeout_ms for a request; fills *out and releases the ticket.  RS_ERR_TIMEOUT if
 * it is not done in time (the ticket stays valid); RS_ERR_INVALID_ARG for an unknown ticket. */
rs_status rs_wait(rs_server* srv, unsigned long long ticket, int timeout_ms, rs_result* out);
/* Slots, workspace bytes held and queued requests (any pointer may be NULL). */
rs_status rs_server_info(rs_server* srv, int* slots, size_t* bytes_in_use, int* queued);
/* Finish queued and running requests, free every slot and stop the worker.  Safe on NULL. */
void rs_server_destroy(rs_server* srv);

/* ---------------------------------------------------------------- plain-method GPU paths
 * The potential of the last solve's particles (snapped centres x_nu = -b + j_nu h, charges
 * Z_nu) on the same grid without the RS format: the comparisons of the RS path on one GPU.
 *   rs_plain_direct:    P[i] = sum_nu Z_nu / |x_i - x_nu| (Sec. 1, Eq. (1.1)); terms with
 *                       x_i = x_nu are skipped.  n^3 N pair terms; n <= 640.
 *   rs_plain_canonical: the full-rank canonical sum P_0[i] = sum_nu Z_nu sum_{k<R}
 *                       p_k[i1-j1] p_k[i2-j2] p_k[i3-j3] with the context's Galerkin factors
 *                       (Eqs. (2.5), (3.4); no split, no truncation).  2 n^3 N R operations;
 *                       n <= 1280 and R (2n-1) factors within one CTA's shared memory.
 * out: caller-owned device buffer of n^3 float32 (C order, i3 fastest).  Products and square
 * roots in FP32, each output's sum compensated (two-sum of 32-term chunks).  Asynchronous on the
 * context stream.  Errors: RS_ERR_NOT_READY without a solve, RS_ERR_INVALID_ARG for a null or
 * misaligned out, RS_ERR_CAPACITY for a grid beyond the limits above.  The paper has no GPU
 * counterpart; these are the plain methods its RS format is measured against. */
rs_status rs_plain_direct(rs_ctx* ctx, float* out);
rs_status rs_plain_canonical(rs_ctx* ctx, float* out);

/* ---------------------------------------------------------------- RS interaction matrix
 * Matrix-vector product with the RS interaction matrix of the n^3 grid points (Sec. 4.1,
 * problem (B), case (A): the point set is the grid, N = n^3):
 *   A = sum_{k long} T_k (x) T_k (x) T_k + sum_{k short} T_k^g (x) T_k^g (x) T_k^g,
 * with T_k[i][i'] = p_k[i - i'] the symmetric Toeplitz matrix of the Galerkin factor vector p_k
 * (Eq. (2.5)) and T_k^g the same inside the window |i - i'| <= gamma only (Def. 3.4), so that
 * A applied to the charges embedded in the grid is the long-range canonical sum plus the windows
 * (the RS tensor before the Tucker truncation).  Each Kronecker term is applied as three mode
 * products by 1-D FFT convolutions of the fibres (circulant embedding of size M, the power of
 * two >= 2n - 2): O(R n^3 log n) work, 3R kernel launches.
 *   X, Y: distinct device buffers of n^3 elements (double for RS_FP64, float otherwise), C order,
 *         8-byte aligned; Y is overwritten.
 *   flags: RS_MATVEC_LONG and/or RS_MATVEC_SHORT select the terms (neither = both);
 *          RS_MATVEC_OFFDIAG subtracts diag(A) X (diag A = sum of p_k[0]^3 over the selected
 *          terms), the matrix A - diag A of Eq. (4.6).
 * Needs no solve (the factors depend only on the configuration).  The first call allocates
 * 2 n^3 elements of scratch and the symbols (R M + M elements), kept until rs_destroy.
 * Asynchronous on the context stream.  Errors: RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA.
 * The products run in the precision of the context (FFT rounding: about 1e-7 of the result's
 * norm per mode product in FP32). */
#define RS_MATVEC_LONG    1
#define RS_MATVEC_SHORT   2
#define RS_MATVEC_OFFDIAG 4
rs_status rs_matvec(rs_ctx* ctx, const void* X, void* Y, int flags);

/* Interaction energy of the last solve's charges through the interaction matrix,
 * E_N = 1/2 <(A - diag A) z, z> (Sec. 4.2, Eq. (4.6)), z the charges embedded in the grid at
 * their snapped grid points and A as for rs_matvec (long and short terms): the energy of the RS
 * tensor without the Tucker truncation, computed without forming the RS-Tucker tensor.  The first
 * call allocates 2 n^3 more elements (the charge grid and its product).  Synchronises.
 * Errors: RS_ERR_NOT_READY without a solve, RS_ERR_OOM, RS_ERR_CUDA, and the device-side input
 * errors of the solve. */
rs_status rs_energy_matvec(rs_ctx* ctx, double* E);

/* Energy and forces of N centres anywhere in the box (not snapped) with the RS kernel of the
 * context in pair form: E = 1/2 sum_{j != nu} Z_j Z_nu K_h(x_j - x_nu), K_h(r) =
 * sum_{k<R} p_k(r1) p_k(r2) p_k(r3) with the Galerkin factors p_k continued to any offset (cell
 * averages of a_k^{1/3} exp(-t_k^2 x^2), Eq. (2.10); on grid offsets the kernel of the RS grid
 * tensor), and F_j = -dE/dx_j (Secs. 4.2, 4.3; no factor 1/2).  All pairs and all R terms, so E
 * is smooth in the centres and F is its exact gradient.  xyz (N x 3), Z (N): device float64;
 * E: device pointer to one float64; F: device N x 3 float64, or NULL for the energy alone.
 * Factors in FP32, sums in FP64.  Asynchronous on the context stream; needs no prior solve.
 * Errors: RS_ERR_INVALID_ARG, RS_ERR_CAPACITY for N > max_particles.  The paper evaluates
 * off-grid energies through the RS tensor; this is the reading used for centres off the grid. */
rs_status rs_pair_energy_forces(rs_ctx* ctx, int N, const double* xyz, const double* Z, double* E, double* F);

/* Text of the last error of this context (or of rs_create when ctx is NULL). */
const char* rs_last_error(rs_ctx* ctx);

/* Library version string. */
const char* rs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RS_H */
