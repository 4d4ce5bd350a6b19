/*
 * libfock -- lattice core-Hamiltonian eigensolver on one GB300 (sm_103a).
 *
 * C ABI.  Plain pointers and sizes only; no exceptions cross it; every
 * function returns a fock_status (0 = success).  All host pointers are
 * owned by the caller and read (or written) only during the call.  Device
 * memory used by a context is owned by the context and released by
 * fock_destroy.
 *
 * The problem (struct fock_problem) follows the paper's statement of the
 * method (Sec. 2.1-2.3, Sec. 3.3): an L1 x L2 x L3 lattice of unit cells
 * of size b0, each holding M0 nuclei (charges Z, positions as cell
 * fractions) and m0 separable Gaussian (GTO) basis functions; a uniform
 * grid of step h = b0/n0 with N_l nodes per axis; a rank-R Gaussian-sum
 * quadrature of the Newton kernel (Eqs. 2.6-2.7).  The discrete operator is
 * H = A/2 - V (Eqs. 2.4-2.5) with A, S the Galerkin Laplacian and mass
 * matrices of the P1-interpolated GTOs (Eqs. 2.15-2.17) and V the Galerkin
 * matrix of the lattice-summed P0 potential (Lemma 2.1, Eq. 2.13, Eq. 3.6);
 * the eigenproblem is H C = S C Lambda.
 *
 * Grid conventions (identical in the oracle and the kernels):
 *   periodic axis:  N = L*n0 nodes at x_i = (i + 1/2) h, period N h;
 *   Dirichlet axis: N nodes at x_i = (i + 1) h, walls at 0 and (N+1) h,
 *                   lattice origin X0 = (pad + 1/2) h, pad = (N - L n0) / 2
 *                   (integer division), N >= L n0.
 * Basis index a = kbar*m0 + mu, kbar = (k1*L2 + k2)*L3 + k3.
 */
#ifndef FOCK_H
#define FOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FOCK_OK = 0,
  FOCK_EINVAL = -1,    /* malformed problem or argument */
  FOCK_ENOMEM = -2,    /* the request does not fit the context's HBM budget */
  FOCK_ENOCONV = -3,   /* iterative solve hit maxit; best estimates returned */
  FOCK_ETIMEOUT = -4,  /* a bounded wait ran out */
  FOCK_EAGAIN = -5,    /* result not ready yet (serving poll) */
  FOCK_ECUDA = -6      /* a CUDA call failed; see fock_last_error */
} fock_status;

enum { FOCK_FP64 = 0, FOCK_MIXED = 1, FOCK_MIXED_F32 = 2 };
enum { FOCK_ANG_S = 0, FOCK_ANG_PX = 1, FOCK_ANG_PY = 2, FOCK_ANG_PZ = 3 };
enum { FOCK_OP_H = 0, FOCK_OP_S = 1 };

/* Substitution of nucleus `nucleus` of lattice cell `cell` by charge newZ
 * (newZ = 0: vacancy; the basis functions stay).  Only the defect's own
 * rank-R kernel is added (no lattice window, no replication).  The paper
 * only motivates defects (Sec. 1, Sec. 2.3 item (B)); supported on chains
 * (at most one axis with L > 1). */
typedef struct {
  int cell[3];
  int nucleus;
  double newZ;
} fock_defect;

typedef struct {
  int L[3];              /* lattice cells per axis, >= 1 */
  int periodic[3];       /* 1 periodic, 0 Dirichlet */
  int N[3];              /* grid nodes per axis (periodic: L*n0) */
  int n0;                /* nodes per cell, h = b0 / n0 */
  double b0;             /* cell size (bohr) */
  int M0;                /* nuclei per cell */
  const double* Z;       /* [M0] charges */
  const double* frac;    /* [M0][3] positions as fractions of the cell */
  int m0;                /* GTOs per cell, 1..32 */
  const double* exps;    /* [m0] exponents alpha > 0 */
  const int* ang;        /* [m0] FOCK_ANG_* */
  const int* centre;     /* [m0] nucleus index of each GTO */
  int R;                 /* quadrature rank, 3..64 */
  const double* sinc_t;  /* [R] Gaussian parameters t_q, or NULL: default rule */
  const double* sinc_c;  /* [R] weights c_q, or NULL: default rule */
  double eps_support;    /* GTO support cut-off (<= 0: 1e-14) */
  int ndef;              /* number of defects */
  const fock_defect* defects;
  int k_eig;             /* box / defect solves: eigenpairs wanted (0: 16) */
  int box_potential;     /* box chains: 0 = the central cell's lattice-summed potential
                            replicated over the box (reading R1, Sec. 2.3 (A), Eq. 3.6);
                            1 = the plain sum over the box's cells, each nucleus once with
                            its full charge (Sec. 2.3 case (B)): the difference is added as
                            blocks on every pair of cells whose functions meet */
  int precision;         /* FOCK_FP64; FOCK_MIXED: the quadrature contractions of the
                            assembly and the dense products of the block iteration (Gram
                            matrices, basis updates) run on the tensor cores as exact split
                            products (fock_split_dgemm, near-FP64); Rayleigh-Ritz, matvecs,
                            preconditioner and Fourier-block eigensolves FP64;
                            FOCK_MIXED_F32: as FOCK_MIXED, and box / defect solves run the
                            preconditioner, and their matvecs until the residual falls
                            below 1e-5, in FP32 */
} fock_problem;

/* Output slot of one problem in a batched solve. */
typedef struct {
  double* evals;    /* [n_evals]: periodic: all |L|*m0 eigenvalues; box/defect:
                       the k_eig lowest; ascending.  Host or device memory
                       (see `outputs_on_device`). */
  int* block_of;    /* optional [n_evals] (periodic only): linear Fourier index
                       jbar = (j1*L2 + j2)*L3 + j3 of each eigenvalue, else NULL */
  int n_evals;      /* out: number written */
  int iters;        /* out: iterations of the box eigensolver (0 periodic) */
  double resid;     /* out: max relative residual |Hx - lSx| / (|l| |Sx|) */
  int status;       /* out: fock_status of this problem */
} fock_output;

typedef struct fock_ctx fock_ctx;
typedef struct fock_blocks fock_blocks;

/* Context: owns device memory (a growable arena) and one CUDA stream.
 * device: CUDA ordinal.  hbm_budget_bytes: cap on the arena (0: 90% of the
 * free memory at creation).  stream: a cudaStream_t to run on, or NULL to
 * create a private one.  Errors: FOCK_EINVAL, FOCK_ECUDA. */
int fock_create(fock_ctx** ctx, int device, size_t hbm_budget_bytes, void* stream);
/* Frees the context; every fock_blocks / fock_plan made from it must be
 * freed first (they use its stream). */
void fock_destroy(fock_ctx* ctx);
const char* fock_last_error(const fock_ctx* ctx);
int fock_synchronize(fock_ctx* ctx);

/* Default quadrature rule (Eq. 2.7 read as a sinc rule in u = log t with a
 * tail node, (u_lo, u_hi) tuned on [zmin, zmax]); writes t[R], c[R] and the
 * measured maximum relative error.  Host only. */
int fock_sinc_table(int R, double zmin, double zmax, double* t, double* c, double* err);
/* The default z-range of a problem (zmin = h/100, zmax = twice a bound on
 * the nucleus-node distance over the lattice window). */
int fock_default_range(const fock_problem* p, double* zmin, double* zmax);
/* Checks a problem as every solve entry point does, on the host only (no
 * device, no context).  On success writes *kind (0: periodic, solved
 * through its Fourier blocks, Thm. 3.3; 1: box chain or problem with
 * defects, solved for the lowest k_eig by the structured iteration,
 * Remark 3.2) and *n_evals (|L|*m0, or k_eig) when the pointers are not
 * NULL.  On FOCK_EINVAL writes the reason, NUL-terminated and truncated to
 * why_cap bytes, into `why` (may be NULL). */
int fock_problem_check(const fock_problem* p, int* kind, int* n_evals, char* why, int why_cap);
/* The block structure the planner lays out for one problem, on the host
 * only (no device, no context), as fock_plan_problem_sizes reports it for a
 * planned batch: *Nb = |L|*m0; box chains and problems with defects
 * (Remark 3.2, Sec. 2.3): *D = reach of the Toeplitz generators T_d
 * (|d| <= D), *mcirc = size of the circulant embedding, and the cell pairs
 * (Ek[e], Em[e]) of the blocks E added to the banded Toeplitz part, sorted
 * by (row, column), with Ekind[e] = 0 wall block, 1 wrap-around block of a
 * periodic chain, 2 defect block, 3 wall block stored as the transpose of
 * its mirror (E(k,m) = E(m,k)^T); at most `cap` entries are written (the
 * pointers may be NULL), *nbound = their full number.  Periodic problems:
 * *mcirc = |L|, *D = *nbound = 0.  FOCK_EINVAL for a malformed problem. */
int fock_problem_layout(const fock_problem* p, int* Nb, int* mcirc, int* D, int* nbound, int* Ek,
                        int* Em, int* Ekind, int cap);

/* Batched solve (stages (a)+(b) for periodic problems, (a)+(c) for box
 * chains and problems with defects).  nprob problems, outs[nprob].
 * Evals pointers are device pointers when outputs_on_device != 0.
 * Returns the first non-zero per-problem status, or FOCK_OK.  Errors:
 * FOCK_EINVAL (no problems, a malformed problem: see fock_problem_check),
 * FOCK_ENOMEM (the batch exceeds the context's budget), FOCK_ECUDA; per
 * problem, out->status FOCK_ENOCONV when the block iteration hit its cap
 * (best estimates written).  The block iteration stops at a relative
 * residual of 1e-10 (or its rounding floor) or after FOCK_DEFAULT_MAXIT
 * iterations. */
#define FOCK_DEFAULT_MAXIT 1000
int fock_solve(fock_ctx* ctx, int nprob, const fock_problem* probs, fock_output* outs,
               int outputs_on_device);

/* Stage (a) for one problem: separable rank-R assembly of the generator
 * blocks (Lemma 2.1, Prop. 2.2, Lemma 3.4).  The handle keeps the per-axis
 * factor tensors and (box) the Toeplitz generators, the embedding Fourier
 * blocks and the boundary perturbation resident on the device; it is owned
 * by the caller and freed by fock_blocks_free before fock_destroy.
 * Errors: FOCK_EINVAL, FOCK_ENOMEM, FOCK_ECUDA. */
int fock_assemble(fock_ctx* ctx, const fock_problem* p, fock_blocks** out);
void fock_blocks_free(fock_blocks* b);

/* Sizes of an assembled handle: N_b, the number of generator blocks
 * written by fock_blocks_copy_generators, of boundary blocks, and the
 * circulant size used by the matvec (|L| periodic; M >= L + D box). */
int fock_blocks_info(const fock_blocks* b, int* Nb, int* ngen, int* nbound, int* mcirc);

/* Copies generators to host memory, layout [g][mu][nu] row-major.
 * Periodic: the |L| generators A_k = block (row cell k, column cell 0) in
 * kbar order (ngen = |L|).  Box chain: T_d = block (k+d, k) of an interior
 * cell for d = -D..D (ngen = 2D+1, d = g - D), and the boundary blocks E
 * with their (row cell, column cell) in bound_rc[2*nbound] such that
 * H = BToepl(T) + E.  Any output pointer may be NULL. */
int fock_blocks_copy_generators(const fock_blocks* b, double* H, double* S, double* EH,
                                double* ES, int* bound_rc);

/* Periodic eigenvalues by FFT block-diagonalisation (Lemma 3.1, Thm 3.3,
 * Eqs. 3.11-3.12): evals[|L|*m0] ascending (host), block_of optional.
 * evecs (optional, host, |L|*m0*m0 complex values as interleaved re, im
 * doubles): the Fourier-block eigenvectors y, evecs[((j*m0 + i)*m0 + mu)]
 * = component mu of the i-th eigenvector (ascending within block j) of the
 * pencil (Hbar_j, Sbar_j), y^H Sbar_j y = 1; removed directions give zero
 * vectors (last).  The lattice eigenvector is u[(k, mu)] = f_j[k] y[mu] with
 * f_j[k] = exp(+2 pi i j.k / L) / sqrt(|L|) (Prop. A.1; fock_bloch_vectors
 * forms it on the device). */
int fock_circulant_eig(fock_ctx* ctx, const fock_blocks* b, double* evals, int* block_of, double* evecs);
/* The same for the Fourier indices jbar in [j0, j1) only: evals[(j1-j0)*m0]
 * ascending (ties by Fourier index), block_of optional.  The blocks are
 * independent (Thm. 3.3), so ranks that each take a contiguous range and
 * merge the sorted parts obtain exactly fock_circulant_eig's output.
 * Errors: FOCK_EINVAL (not periodic, range outside 0..|L|), FOCK_ECUDA. */
int fock_circulant_eig_range(fock_ctx* ctx, const fock_blocks* b, int j0, int j1, double* evals,
                             int* block_of);

/* Lattice eigenvectors of a periodic problem (Prop. A.1: the inverse DFT
 * over the lattice index of block eigenvectors, U = (F^* (x) I) Ubar) for
 * nsel eigenpairs given by their Fourier index jbar[c] (block_of of
 * fock_circulant_eig) and rank[c] within that block (0 = lowest): U is host
 * memory of nsel columns of N_b complex values (interleaved re, im),
 * U[c][(kbar*m0 + mu)] = f_j[k] y[mu]; S-orthonormal, H u = lambda S u.  The
 * needed blocks are solved again (with vectors) and the back-transform runs
 * on the device (k_bloch_vectors).  Errors: FOCK_EINVAL (not periodic, index
 * out of range), FOCK_ECUDA. */
int fock_bloch_vectors(fock_ctx* ctx, const fock_blocks* b, int nsel, const int* jbar, const int* rank,
                       double* U);

/* y = H x or y = S x (which = FOCK_OP_H / FOCK_OP_S) for an assembled box
 * chain or problem with defects, by the block-circulant embedding FFT
 * matvec plus the boundary/defect blocks (Remark 3.2, Sec. 2.3).  x, y:
 * N_b x nvec, column-major; device pointers when on_device != 0, else
 * host.  Errors: FOCK_EINVAL (a periodic handle -- its operator is applied
 * through its Fourier blocks -- null pointers, `which`, nvec < 1, device x
 * and y that overlap), FOCK_ENOMEM, FOCK_ECUDA. */
int fock_toeplitz_matvec(fock_ctx* ctx, const fock_blocks* b, int which, const double* x,
                         double* y, int nvec, int on_device);

/* Same product as fock_toeplitz_matvec (device x, y only), for callers that
 * cannot allocate device memory: real-time loops that forbid allocator calls
 * (and the synchronisation a free implies) once running, and hosts whose own
 * allocator owns the device.  The paper has no counterpart; it is a
 * deployment variant.  All work arrays and launch descriptors live in one
 * fixed device array of FOCK_NOALLOC_SCRATCH_BYTES per device, held until
 * the process exits; requires 2*M*m0*nvec*16 + 4096 <= that size (M =
 * circulant size from fock_blocks_info), else FOCK_EINVAL with a message;
 * x and y must not overlap (FOCK_EINVAL).  The first call on a device looks
 * the array's address up (make that first call before any stream capture);
 * the address is kept for the life of the device's primary context.  Calls
 * share the array: two calls whose work overlaps on the GPU race; the array
 * keeps the last call's contents and every part a call reads is written
 * earlier in the same call.  The caller's current device is left as it was.
 * Synchronous on the context's stream. */
#define FOCK_NOALLOC_SCRATCH_BYTES (16u << 20)
int fock_toeplitz_matvec_noalloc(fock_ctx* ctx, const fock_blocks* b, int which, const double* x,
                                 double* y, int nvec);

/* Lowest k eigenpairs of (H, S) by preconditioned block iteration
 * (Sec. 2.3, "structured iteration on subspace"; LOBPCG with the embedding's
 * shifted inverse as preconditioner).  evals[k] host; evecs[N_b x k]
 * (host, column-major, S-orthonormal) or NULL; iters out.  Returns
 * FOCK_ENOCONV (with the best estimates written: Ritz values, each above
 * the eigenvalue it approximates) when maxit is reached; FOCK_EINVAL for a
 * periodic handle or k above the problem's k_eig; FOCK_ECUDA. */
int fock_box_eig(fock_ctx* ctx, const fock_blocks* b, int k, double tol, int maxit,
                 double* evals, double* evecs, int* iters);

/* ---- device-resident batched execution ----
 * fock_plan_create validates and plans nprob problems, allocates their device
 * memory and uploads every input (parameters, index maps, descriptors) once.
 * fock_plan_execute runs the whole hot path -- stage (a) for all, (b) for
 * periodic problems, (c) for box chains -- on the context's stream; results
 * stay on the device until fock_plan_outputs copies them (host or device
 * destinations).  A plan may be executed any number of times. */
typedef struct fock_plan fock_plan;
int fock_plan_create(fock_ctx* ctx, int nprob, const fock_problem* probs, fock_plan** out);
/* tol <= 0: 1e-10; maxit <= 0: FOCK_DEFAULT_MAXIT */
int fock_plan_execute(fock_plan* plan, double tol, int maxit);
int fock_plan_outputs(fock_plan* plan, fock_output* outs, int outputs_on_device);
/* bytes uploaded by fock_plan_create, bytes of device memory held, and the
 * number of eigenvalues the plan returns in total */
int fock_plan_info(const fock_plan* plan, size_t* upload_bytes, size_t* device_bytes, size_t* n_evals);
/* Launch machinery of a plan (no counterpart in the paper; its batching):
 * fft_cc = columns per CTA of the embedded FFT chosen by the plan's tuner
 * (timed on the first execution, once per largest embedding size and column
 * count per context; 0 before), graph_nodes = kernels of the block iteration's
 * body captured as two CUDA graphs (split at the Rayleigh-Ritz launch) and
 * replayed from its second pass on (0: not
 * captured -- before the second pass, with the kernel timers on, or when the
 * capture was refused and the launches stayed eager).  Either pointer may be
 * NULL.  FOCK_EINVAL for a NULL plan. */
int fock_plan_tuning(const fock_plan* plan, int* fft_cc, int* graph_nodes);
/* Periodic problem i of a plan, after an execution: n_eig = the Fourier blocks
 * (conjugate pairs once) whose overlap had a direction at or below the
 * dependency cut, or could not be certified free of one, and so were solved
 * through the overlap's eigendecomposition instead of its Cholesky factor
 * (Prop. A.1; the cut of reading G16).  0 for other problems.  Synchronous.
 * FOCK_EINVAL for a NULL plan or pointer or i out of range. */
int fock_plan_block_routes(const fock_plan* plan, int i, int* n_eig);
/* Sizes of problem i of a plan: N_b, circulant size M (box: M >= L + D;
 * periodic: |L|), generator reach D in cells (box) and boundary blocks. */
int fock_plan_problem_sizes(const fock_plan* plan, int i, int* Nb, int* mcirc, int* D, int* nbound);
/* Convergence history of problem i of a plan after its last execution: the
 * largest relative residual of the wanted pairs at each iteration of the
 * block iteration (box chains and problems with defects; 0 entries for
 * periodic problems).  Writes min(n, cap) values to res (may be NULL) and
 * returns n, or FOCK_EINVAL. */
int fock_plan_history(const fock_plan* plan, int i, double* res, int cap);
/* Tensor-core work of one execution of a plan's mixed-form assembly
 * (fock_split_dgemm products of its gram tasks): the BF16 multiply-add
 * flops the MMAs execute (128 x 64 output tiles, 64-long chunks, 28 digit
 * pairs, 4 MMAs of K = 16 each) and the FP64 flops they stand for (2 M N K).
 * Zero for a plan without mixed problems. */
int fock_plan_split_work(const fock_plan* plan, double* tensor_flops, double* fp64_flops);
void fock_plan_free(fock_plan* plan);

/* ---- kernel timers (CUDA events recorded on the context's stream) ----
 * While enabled, every kernel launch of the library is bracketed by events;
 * fock_profile_read synchronizes and returns, per kernel name, the number of
 * launches and the summed device time.  names: buffer of `cap` entries of
 * 32 chars.  Returns the number of distinct kernels written. */
int fock_profile_enable(fock_ctx* ctx, int on);
int fock_profile_reset(fock_ctx* ctx);
int fock_profile_read(fock_ctx* ctx, int cap, char* names, int* launches, double* ms);

/* C = alpha A B + beta C in FP64 on the tensor cores: the exact split
 * products (base-128 digits of the 53-bit mantissas, BF16 x BF16 -> FP32
 * tcgen05 products, integer level sums combined in FP64) that the mixed
 * form uses for the quadrature contractions of stage (a) (Lemma 2.1
 * display; X_t = sum_r P_t[r] Z[r]).  A: M x K with element (m, k) at
 * A[m*a_m + k*a_k]; B: K x N, (k, n) at B[k*b_k + n*b_n]; C: (m, n) at
 * C[m*c_m + n*c_n]; all device pointers, strides in elements.  Each product
 * carries a relative error below ~2^-46 of |row max of A| |column max of B|
 * per summand.  ksplit (1..1024): the summation is split into that many
 * ranges computed by separate CTAs and added in a fixed order (a work array
 * is allocated for them); sym != 0 (M = N): C is taken as symmetric, its
 * upper triangle computed and mirrored (the Gram products of the block
 * iteration).  Synchronous on the context's stream.  Errors: FOCK_EINVAL,
 * FOCK_ETIMEOUT (a tensor-core completion wait ran out; C not written),
 * FOCK_ECUDA. */
int fock_split_dgemm(fock_ctx* ctx, int M, int N, int K, const double* A, long long a_m, long long a_k,
                     const double* B, long long b_k, long long b_n, double* C, long long c_m, long long c_n,
                     double alpha, double beta, int ksplit, int sym);

/* Measured FP64 and FP32 fused-multiply-add throughput of CUDA device
 * `device` in TFLOP/s (best of three timed launches of independent FMA
 * chains on every SM, after a warm-up): the denominators of the FP64- and
 * FP32-pipe roofline fractions.  Allocates a small output buffer; the
 * caller's current device is left as it was.  Errors: FOCK_EINVAL,
 * FOCK_ECUDA. */
int fock_measure_peaks(int device, double* fp64_tflops, double* fp32_tflops);

/* ---- serving: continuous batching of lattice problems on one GPU ----
 *
 * The paper solves one lattice at a time; this layer serves a stream of
 * problems (different L, m0, periodic or box chains).  A server owns
 * `slots` worker threads, each with a private CUDA stream, and one
 * stream-ordered device memory pool.  Submitted problems are deep-copied,
 * validated and sized, and queued in arrival order; a free worker admits
 * the queue's head problem and, in queue order, the later problems of the
 * same kind (periodic: one pass; box chains and defects: an iteration)
 * while the device bytes of the batches already in flight plus theirs stay
 * within hbm_budget_bytes (and at most max_batch of them), solves them as
 * one batch (fock_solve's path) and publishes one result per ticket.  Problems that arrive while batches
 * run are admitted by the next free worker, so their kernels overlap with
 * the batches in flight.  Each result equals the result of solving that
 * problem alone (per-problem reduction orders and start vectors are fixed).
 */
typedef struct fock_server fock_server;
typedef struct {
  int slots;                /* concurrent batches (worker threads/streams); 0: 2, at most 16 */
  int max_batch;            /* problems per batch; 0: 256 */
  size_t hbm_budget_bytes;  /* device bytes for all batches in flight; 0: 80% of free memory */
  double tol;               /* box eigensolver relative residual; <= 0: 1e-10 */
  int maxit;                /* box eigensolver iteration cap; <= 0: FOCK_DEFAULT_MAXIT */
} fock_serve_config;
/* One request's result.  evals/block_of point into library-owned host
 * memory that stays valid until fock_result_release(ticket) or
 * fock_serve_stop.  Times are nanoseconds since fock_serve_start. */
typedef struct {
  const double* evals;      /* [n_evals] ascending (periodic: all |L| m0, +inf for removed
                               directions; box: the k_eig lowest) */
  const int* block_of;      /* [n_evals] Fourier index of each eigenvalue (periodic), else NULL */
  int n_evals;
  int status;               /* fock_status of this problem */
  int iters;                /* box eigensolver iterations (0 periodic) */
  double resid;             /* box: max relative residual */
  int64_t t_submit_ns, t_admit_ns, t_done_ns;
  int batch_id, batch_size; /* the batch the request was solved in */
} fock_result;
typedef struct {
  uint64_t completed, pending, batches;
  int inflight, max_inflight;            /* batches on the device now / at most so far */
  size_t reserved_bytes, peak_reserved_bytes, budget_bytes;
} fock_serve_stats_t;
/* Starts the workers on CUDA device `device`.  cfg may be NULL (defaults).
 * Errors: FOCK_EINVAL, FOCK_ECUDA. */
int fock_serve_start(int device, const fock_serve_config* cfg, fock_server** out);
/* Queues a copy of *p (the caller may free p at once) and returns its ticket.
 * Errors: FOCK_EINVAL (malformed problem, server stopping; message in
 * fock_serve_last_error), FOCK_ENOMEM (the problem alone exceeds the budget).
 * Thread-safe. */
int fock_serve_submit(fock_server* s, const fock_problem* p, uint64_t* ticket);
/* Waits up to timeout_ms (< 0: no limit, 0: no wait) for the ticket's result.
 * A periodic request's result is ready when its batch ends; a structured
 * request's (box chains, defects) as soon as it leaves the block iteration,
 * while the rest of its batch may still run (the values are the same either
 * way; t_done_ns records which).
 * FOCK_OK: *out filled (the problem's own status in out->status);
 * FOCK_EAGAIN: not finished yet; FOCK_EINVAL: unknown ticket.  Thread-safe. */
int fock_serve_poll(fock_server* s, uint64_t ticket, fock_result* out, int timeout_ms);
/* Frees a finished ticket's result (FOCK_EAGAIN if it is still running); a
 * finished structured request may be freed while its batch still runs. */
int fock_result_release(fock_server* s, uint64_t ticket);
int fock_serve_stats(fock_server* s, fock_serve_stats_t* out);
const char* fock_serve_last_error(const fock_server* s);
/* Finishes every queued problem, joins the workers, frees all device memory
 * and every unreleased result. */
int fock_serve_stop(fock_server* s);

#ifdef __cplusplus
}
#endif
#endif /* FOCK_H */
