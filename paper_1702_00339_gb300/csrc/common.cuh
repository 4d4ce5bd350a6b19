// Internal descriptors and device helpers of libfock (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include <mutex>

// Raises a kernel's dynamic shared memory limit, once per process, to the
// device's opt-in maximum minus the kernel's static shared memory.  The
// attribute is a per-function upper bound (a launch still occupies only the
// bytes it asks for); setting it per batch instead would let concurrent
// batches on other streams lower it under a launch in flight.
#define FOCK_SMEM_OPTIN(kernel)                                                       \
  do {                                                                                \
    static std::once_flag fock_optin_flag_;                                           \
    std::call_once(fock_optin_flag_, [] {                                             \
      int dev = 0, mx = 0;                                                            \
      cudaGetDevice(&dev);                                                            \
      cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);      \
      cudaFuncAttributes fa;                                                          \
      if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) mx -= (int)fa.sharedSizeBytes; \
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);  \
    });                                                                               \
  } while (0)

namespace fock {

constexpr int MAXM0 = 32;
constexpr int MAXR = 64;
constexpr int MAXRADIX = 16;   // radix factors of a circulant size

// Numerically singular overlap directions (reading G16 of the pencil
// H C = S C Lambda, Eqs. 2.4-2.5 and 3.11-3.12).  B[mu nu] = sum over lattice
// offsets d of |S_d[mu nu]| bounds every entry of every Fourier block and every
// block row of the lattice overlap (||S||_2 <= ||B||_F).  The lattice overlap is
// an N_b x N_b matrix (N_b = |L| m0); the usual rank tolerance of a matrix of
// that order, N_b * eps * ||S|| (eps = 2^-52; the tolerance of LAPACK-based
// numerical rank decisions), sets tau = N_b * eps * ||B||_F: an overlap
// direction (of a Fourier block Sbar_j, whose eigen-directions are the
// lattice overlap's, or of the cell overlap T_S[0] of a chain, repeated on
// every cell) with eigenvalue at most tau is removed; nothing else is.
__host__ __device__ inline double null_tau(double normB_F, double nb) { return nb * 0x1p-52 * normB_F; }

// Modes of a 1D Galerkin form along one axis (gram task):
//   RING - periodic axis: nodes 0..N-1 with wrap-around, potential tiled;
//   VIRT - Toeplitz generator of a chain axis: unbounded node line, no walls,
//          potential tiled with period n0 (what an interior cell sees);
//   WALL - Dirichlet axis as it is: nodes -pad..N-pad-1, zero outside,
//          potential replicated with the cell index clamped to 0..L-1.
enum GramMode { RING = 0, VIRT = 1, WALL = 2 };

struct AxisDev {
  int N, L, per, pad;
  int jlo, W;           // reference-cell function window: j in [jlo, jlo + W)
  int rlo, nr;          // potential table: reduced node r in [rlo, rlo + nr)
  int smin, slen;       // support of the reference-cell functions: virtual nodes [smin, smin + slen)
  double* g;            // [m0][W]   nodal GTO factors of the reference cell
  double* p;            // [T][nr]   window-summed P0 Gaussian integrals
};

struct ProbDev {
  int m0, M0, R, T, nF; // T = M0*R potential terms, nF = T + 2 factors
  int n0;
  double b0, h, eps;
  AxisDev ax[3];
  const double* alpha;  // [m0]
  const int* ang;       // [m0]
  const int* centre;    // [m0]
  const double* Z;      // [M0]
  const double* frac;   // [M0*3]
  const double* tq;     // [R]
  const double* cq;     // [R]
};

// One 1D Galerkin form: X[f][mu][nu] = sum_rho g_{a,mu}(rho) [W_f g_{b,nu}](rho)
// for f = 0 (mass S1), 1 (stiffness A1), 2 + t (potential term t).
struct GramTask {
  int prob, axis, mode;
  int a, b;             // cells of the row / column function
  int rho0, rho1;       // node range [rho0, rho1) (RING: 0..N)
  int ptab;             // -1: the lattice potential table of the axis; >= 0: a
                        //     defect table index (no replication, direct nodes)
  double* X;            // out [nF][m0*m0]
  double* Zs;           // scratch [nfold][m0*m0] (folded pair products)
  int nfold;            // number of reduced nodes of the fold
  int foldlo;           // first reduced node
  int split;            // 1: the potential contraction runs on the tensor cores (k_split_gemm)
};

// A defect table: single-nucleus Gaussian integrals e[q][i] on the grid of
// one axis (no window, no replication), scaled into the defect term.
struct DefTab {
  int prob, axis, N, pad;
  double pos;           // nucleus coordinate in lattice units relative to X0 (h units)
  double* e;            // [R][N]
  // mode 1 (box potential read as the plain lattice sum, Sec. 2.3 case (B), on
  // a chain's axis 0): e[q][i] = sum over the L cells k of the Gaussian cell
  // integral of the nucleus at pos + k n0, minus the replicated table of the
  // same term (prep[t][r(rho) - rlo], t = nu R + q, r the reduced node)
  int mode, L, nu, nr, rlo;
  const double* prep;
};

// Defect field of a chain (reading R-DEF): F[rho][mu nu] = sum over defects d
// and quadrature terms q of dZ_d c_q D1_d[q][mu nu] D2_d[q][mu nu] e_d[q][rho],
// with e_d the defect's axis-0 single-nucleus table and D1_d, D2_d its
// transverse forms (the chain's transverse axes hold one cell, so these do
// not depend on the block pair).
struct DefRef {
  const double* e;      // [R][N0] axis-0 table
  const double* D1;     // [R][m0*m0] transverse forms (axis 1)
  const double* D2;     // [R][m0*m0] transverse forms (axis 2)
  double dz;            // newZ - Z
};
struct DefField {
  int prob, N, ndef;
  const DefRef* refs;   // [ndef]
  double* F;            // [N][m0*m0]
};
// One defect block: out_H[mu nu] = -sum_rho g_{a mu}(rho) g_{b nu}(rho) F[rho][mu nu]
// over the pair's node range (axis 0, WALL or RING), out_S = 0.
struct DefBlock {
  int prob, mode, a, b, rho0, rho1, pad;
  const double* F;
  double* outH; double* outS;
};

struct __align__(16) cplx { double x, y; };

__host__ __device__ inline cplx cmk(double a, double b) { cplx r; r.x = a; r.y = b; return r; }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) {
  return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline cplx cmulc(cplx a, cplx b) {  // a * conj(b)
  return cmk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ inline cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__host__ __device__ inline cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
// acc + a b, acc + a conj(b), and c - a conj(b) - d conj(e), each real part
// and imaginary part as a chain of fused multiply-adds (the FP64 pipe issues 4
// or 8 instructions instead of 6 or 12 for products followed by sums)
__host__ __device__ inline cplx cfma(cplx a, cplx b, cplx acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ inline cplx cfmac(cplx a, cplx b, cplx acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y); acc.y = fma(-a.x, b.y, acc.y);
  return acc;
}
__host__ __device__ inline cplx crank2(cplx c, cplx a, cplx b, cplx d, cplx e) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x); c.x = fma(-d.x, e.x, c.x); c.x = fma(-d.y, e.y, c.x);
  c.y = fma(-a.y, b.x, c.y); c.y = fma(a.x, b.y, c.y); c.y = fma(-d.y, e.x, c.y); c.y = fma(d.x, e.y, c.y);
  return c;
}

__device__ inline int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
__device__ inline int posmod(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }

// Circulant (FFT) plan of one problem's block lattice index.
struct CircDev {
  int M;                // circulant size
  int nfac;             // radix factors of M
  int fac[MAXRADIX];
  cplx* tw;             // [M] exp(-2 pi i t / M)
};

// ---- task descriptors shared by the host planner and the kernels ----
struct SegDesc { int prob, axis, count; };

struct CombineTask {
  int prob;
  const double* X0; const double* X1; const double* X2;   // [nF][m0*m0]
  const double* subH; const double* subS; int subT;        // generator to subtract (transposed?)
  const double* D0; const double* D1; const double* D2;    // defect forms [R][m0*m0] or null
  double dZ;
  double* outH; double* outS;
  double* outHT; double* outST;        // optional: the transposed block as well (mirror entry)
};

struct DftTask {
  int prob, L, noff;
  const int* offs;        // [noff] lattice offsets d
  const double* X;        // [noff][nF][m0*m0]
  cplx* Xh;               // [L][nF][m0*m0]
};

struct FBlockTask {
  int prob, source, nj;          // Fourier indices handled: j in [j0, j0 + nj)
  int j0;                        // first Fourier index (outputs are indexed from 0)
  int L[3];                      // lattice (FACTORS)
  const cplx* Xh[3];             // per-axis DFT'd factors [L_l][nF][m0*m0] (FACTORS)
  int M, D;                      // circulant size and generator reach (TOEPLITZ)
  const double* TH;              // [D+1][m0*m0] generators T_d of H (TOEPLITZ)
  const double* TS;              // [D+1][m0*m0] of S
  cplx* outH;                    // optional [nj][m0*m0]: store Hbar_j
  cplx* outS;                    // optional [nj][m0*m0]: store Sbar_j
  int want;                      // 0: no eigenvalues, 1: all, 2: only the lowest
  double* ev;                    // [nj*m0] (want 1) or [nj] (want 2)
  int* blk;                      // optional [nj*m0] Fourier index of each eigenvalue
  int* fail;                     // set to 1 if a block's Sbar is not positive definite
  const double* tau;             // FACTORS: the problem's dependency cut (k_null_tau); TOEPLITZ:
                                 // null, the cut is formed from TS in the block kernel
  cplx* vecs;                    // optional [nj][m0][m0] (want 1): eigenvector i of block j at
                                 // [j][i][mu], Sbar_j-orthonormal, ascending; removed directions zero
  int* neig;                     // optional: counts the blocks solved by the overlap's
                                 // eigendecomposition (the Cholesky certificate failed)
};

// Dependency cut of a periodic problem: B[mu nu] = prod over axes of the sum
// over that axis's offsets of |X_a[o][0][mu nu]| (the per-axis mass forms; the
// overlap blocks are their Hadamard products, Lemma 3.4), tau = null_tau(||B||_F).
struct NullTask {
  int m0, nF;
  int nb;                        // N_b = |L| m0, the order of the lattice overlap
  const double* X[3];            // [noff][nF][m0*m0] per axis
  int noff[3];
  double* tau;                   // out
};

struct PrecTask {
  int prob, M;
  const double* emin;    // [M] lowest eigenvalue of each embedding block
  double* sigma;         // out
  const cplx* CH; const cplx* CS;   // [M][m0*m0]
  cplx* K;               // out [M][m0*m0]
  double rel_shift;
};

struct SortTask { int n; double* v; int* idx; };

struct FftTask {
  int prob, L, m0, ncol;          // block rows L, block size m0, vectors ncol
  const CircDev* circ;
  const double* x; int ldx;       // forward input (real, N_b x ncol, col-major)
  cplx* X;                        // [M][m0*ncol]
  double* y; int ldy;             // inverse output
  double beta;                    // y = beta*y + Re(.)/M
  int cc;                         // columns per CTA
  const int* mode;                // null: FP64 only; else the problem's mode (0 FP64, 1 FP32)
  const int* active;              // null: always; else skipped once the problem has converged
};

struct BmulTask {
  int prob, M, m0, ncol;
  const cplx* B1; const cplx* B2;  // [M][m0*m0] (B2 optional)
  const cplx* X;                   // [M][m0*ncol]
  cplx* Y1; cplx* Y2;
  const int* mode;                 // as FftTask::mode
  const int* active;               // as FftTask::active
};

struct EApplyTask {
  int prob, m0, ncol, nrows;
  const int* rows;      // [nrows] block-row ids
  const int* rowptr;    // [nrows+1] into cols/vals
  const int* cols;      // block-column ids
  const double* vals;   // [nnz][m0*m0]
  const double* x; int ldx;
  double* y; int ldy;
  const int* mode;      // null: always; else only while *mode == 0 (image refresh lists)
  const int* active;    // as FftTask::active
  const double* vals2;  // optional second operator on the same x (S beside H), into y2 (ldy)
  double* y2;
};

struct InitTask { int n, k, ld; uint64_t seed; double* X; };

struct GemmTask {
  const int* active;           // skip when *active == 0
  int n, a, b;                 // TN: G[a x b] = A[n x a]^T B[n x b];  NN: C[n x b] = A[n x a] B[a x b]
  const double* A; int lda;
  const double* B; int ldb;
  double* C; int ldc;
  double alpha, beta;
  int sym;                     // TN with a symmetric result: upper tiles computed, mirrored
  int tile;                    // TN output tile: 20 when the problem's block size is a multiple of 20, else 16
  int split;                   // 1: computed by k_split_gemm instead (mixed form)
};

struct ResidTask {
  const int* active;
  int n, k, ld;
  const double* X; const double* HX; const double* SX;
  double* lam;        // Rayleigh quotients (recomputed from X, HX, SX)
  double* R;          // [n x k]
  double* res;        // [k] relative residual
};

// pivot columns per block of the Rayleigh-Ritz step's triangular substitutions
// (its shared-memory staging: 2 kRRBlock ld doubles)
constexpr int kRRBlock = 8;
// CTAs of the cluster that runs one large Rayleigh-Ritz step (k_rr_cl)
constexpr int kRRCluster = 8;
// extra doubles of staging a shared-memory Rayleigh-Ritz step needs beyond its
// 3 ld^2 (none when its first working matrix, ld^2 doubles, can hold it)
__host__ __device__ inline int rr_stage_extra(int ld) { return (ld * ld >= 2 * kRRBlock * ld) ? 0 : 2 * kRRBlock * ld; }

struct RRTask {
  const int* active;
  int nb, k, ld;          // current basis size, wanted pairs, leading dim of G / C
  double* GH; double* GS; // [nb x nb] (ld), destroyed
  double* work;           // [7 * ld * ld] scratch: C, V, Z (global when they do not fit
                          //   shared memory), then 4 ld^2 for the tridiagonal eigensolver
  double* lam;            // out [k]
  double* Cc;             // out [nb x 2k] (ld): [C | C with the first k rows zeroed]
  int* fail;              // out: 1 if Y^T S Y was not numerically positive definite
  const int* mode;        // mixed form: 1 while the images are FP32 (coarser drop threshold)
  int big;                // 1: the working matrices (3 ld^2 doubles) exceed shared memory; the
                          //    problem runs on a cluster of 512-thread CTAs (k_rr_cl), else in
                          //    the 256-thread k_rr (a property of the problem alone, so results
                          //    are batch-invariant)
};

struct CopyTask { const int* active; int n, ncols; const double* src; int lds; double* dst; int ldd; };

// One piece of a batch's results gathered into a contiguous staging buffer
// (4-byte words) for a single device-to-host copy.
struct GatherSeg { const uint32_t* src; unsigned int words; unsigned int dst; };

struct BandTask {
  int m0, L, D, k, n;
  const double* TH; const double* TS;      // [D+1][m0*m0]
  int nE;
  const int* Ek; const int* Em;            // boundary block positions
  const double* EH; const double* ES;      // [nE][m0*m0]
  const double* sigma0;                    // shift from the embedding
  double* band;                            // [L][D+1][m0*m0]
  double* sigma_used;                      // out
  int* fail;                               // out: 1 if every attempt broke down
  const double* R; double* W; int ld;      // solve: W = A^-1 R (n x k, ld)
  const int* active;
  int fp32;                                // 1: solve in FP32 arithmetic (mixed form)
};

// Cell basis of a chain on the structured path: Xc (m0 x m0, row-major
// Xc[mu][j]) = Q_K diag(s_K)^-1/2 from the eigenpairs of the cell overlap
// T_S[0] with s > tau (the dependency cut, common.cuh); columns j >= the kept
// count are zero.  Then every block B becomes Xc^T B Xc: an exact change of
// basis when nothing is removed.
struct CanonTask {
  int m0, D, nE;
  const double* TH; const double* TS;     // original generators [D+1][m0*m0]
  const double* EH; const double* ES;     // original boundary blocks [nE][m0*m0]
  double* Xc;                             // out [m0*m0]
  int* kept;                              // out: kept directions
  double* THc; double* TSc;               // out transformed generators
  double* EHc; double* ESc;               // out transformed boundary blocks
  const int* Epart;                       // [nE] index of the transposed partner block
                                          // (self on the diagonal, -1 if none)
  int nb;                                 // N_b = L m0, the order of the chain's overlap
  int ring_full;                          // 1: T_d, d = 0..D, are every ring offset once (a periodic
                                          //    chain planned as its whole circulant), so the scale B of
                                          //    the dependency cut is sum_d |T_S[d]|; 0: sum_d of
                                          //    |T_S[d]| + |T_S[d]|^T over d >= 1, plus |T_S[0]|
};

// One FP64 product C = alpha A B + beta C computed on the tensor cores by
// exact split products (k_split.cu): A is M x K with A(m, k) at
// A[m * a_m + k * a_k], B is K x N with B(k, n) at B[k * b_k + n * b_n],
// C(m, n) at C[m * c_m + n * c_n].
struct SplitTask {
  const int* active;           // skip when *active == 0 (null: always)
  int M, N, K;
  const double* A; long long a_m, a_k;
  const double* B; long long b_k, b_n;
  double* C; long long c_m, c_n;
  double alpha, beta;
  int ksplit;                  // K ranges computed by separate CTAs (>= 1)
  double* work;                // null: C written directly; else [ksplit][M][N] partial sums,
                               // reduced in a fixed order by k_split_reduce
  int sym;                     // (with work) C is symmetric: the upper triangle is reduced, mirrored
};

// Device pointers and sizes the matvec of an assembled box chain needs.
struct MatvecView {
  int Lc, m0, M, nE, nErows;
  const CircDev* circ;
  const cplx *CH, *CS;
  const int *Erows, *Erowptr, *Ecols;
  const double *EH, *ES;
  cudaStream_t stream;
  int device;
};

// ---- FP64 with few FP64-pipe instructions ----
// On this part a warp-wide FP64 instruction holds a sub-partition's FP64
// unit for ~64 cycles whether 1 or 32 lanes are active; an IEEE FP64
// division takes ~440 cycles and a square root ~690 (measured).  Reciprocal
// and inverse square root below: an FP32 seed refined by two Newton-Raphson
// steps in FP64 (quadratic convergence, relative error 2^-22 -> 2^-44 ->
// rounding level), 4 and 8 FP64 instructions.  Arguments outside
// [2^-100, 2^100] in magnitude (where the FP32 seed could over- or
// underflow) take the IEEE operation; the test is on the exponent bits.
__device__ inline bool nr_range(double x) {
  const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return ex > 1023 - 100 && ex < 1023 + 100;
}
__device__ inline double rcp_nr(double x) {
  if (!nr_range(x)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
// x > 0
__device__ inline double rsqrt_nr(double x) {
  if (!nr_range(x)) return 1.0 / sqrt(x);
  double r = (double)__frsqrt_rn((float)x);
  // Newton for r^-2 = x: r <- r + (r / 2)(1 - x r^2)
  double e = fma(-x * r, r, 1.0);
  r = fma(0.5 * r, e, r);
  e = fma(-x * r, r, 1.0);
  return fma(0.5 * r, e, r);
}
// |x| as a bit pattern: orders like |x| (integer compare, no FP64 pipe)
__device__ inline long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFll; }
// ordering key for "largest non-negative value" searches: non-negative
// finite values order by their bit pattern; negative, infinite and NaN
// values map below all of them
__device__ inline long long pivot_key(double x) {
  const long long b = __double_as_longlong(x);
  return (b < 0 || (b & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) ? -1ll : b;
}

// ---- symmetric tridiagonal (d[0..m), e[0..m-1)) helpers ----
// Number of eigenvalues of the symmetric tridiagonal (d, e) below x, from
// FP32 copies df = d and e2f = e^2 (Kahan's recurrence of the pivots of
// T - x I; a pivot below pivmin in magnitude counts as negative).
__device__ inline int sturm_count_f32(const float* df, const float* e2f, int m, float x, float pivmin) {
  int cnt = 0;
  float q = df[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  cnt += (q < 0.0f);
  for (int i = 1; i < m; ++i) {
    q = (df[i] - x) - __fdividef(e2f[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0f);
  }
  return cnt;
}

// Number of eigenvalues below x in FP64 without divisions: the sign changes
// of the leading principal minors p_0 = 1, p_1 = d_0 - x,
// p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2} (Sturm sequence).  A minor
// leaving [2^-500, 2^500] in magnitude rescales the last two minors by a
// power of two (exact); an exactly zero minor takes the sign opposite to its
// predecessor.  Three FP64 instructions per row; signs and exponents are
// tested on the bit patterns.
__device__ inline int sturm_count_minors(const double* d, const double* e2, int m, double x) {
  double pm = 1.0, p = d[0] - x;
  int cnt = 0;
  long long sp = 0;   // sign bit of the previous minor
  for (int i = 0;; ++i) {
    long long b = __double_as_longlong(p);
    if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) {        // zero minor
      p = pm * -0x1p-200;
      b = __double_as_longlong(p);
    }
    const long long sb = (long long)((unsigned long long)b >> 63);
    cnt += (int)(sb ^ sp);
    sp = sb;
    if (i + 1 >= m) break;
    const int ex = max((int)((b >> 52) & 0x7FF), (int)((__double_as_longlong(pm) >> 52) & 0x7FF));
    if (ex > 1023 + 500 || ex < 1023 - 500) {      // rescale both by 2^(1023 - the larger exponent)
      const double sc = __longlong_as_double((long long)(2046 - min(ex, 2046)) << 52);
      p *= sc;
      pm *= sc;
    }
    const double pn = fma(d[i + 1] - x, p, -e2[i] * pm);
    pm = p;
    p = pn;
  }
  return cnt;
}

// idx-th (0-based, ascending) eigenvalue of the symmetric tridiagonal of
// order m given by FP32 copies (df, e2f) and FP64 (d, e2 = e^2), with tnf a
// Gershgorin bound of its spectral radius: FP32 bisection to ~1e-7 of the
// spectral radius, then (fp64) a bracket around that value verified by FP64
// Sturm counts (widened up to three times, else the Gershgorin interval)
// and FP64 bisection inside it to 2 u |lambda|, or to rtol (1 + |lambda|)
// when that is wider (shifts and bounds that need no more).
__device__ inline double tridiag_eig_fast(const float* df, const float* e2f, const double* d, const double* e2,
                                          int m, int idx, double rtol) {
  float lo = FLT_MAX, hi = -FLT_MAX, emax2 = 0.0f;
  for (int i = 0; i < m; ++i) {
    const float r = (i > 0 ? sqrtf(e2f[i - 1]) : 0.0f) + (i + 1 < m ? sqrtf(e2f[i]) : 0.0f);
    lo = fminf(lo, df[i] - r);
    hi = fmaxf(hi, df[i] + r);
    if (i + 1 < m) emax2 = fmaxf(emax2, e2f[i]);
  }
  const float tnf = fmaxf(fabsf(lo), fabsf(hi));
  const float pivmin = FLT_MIN * fmaxf(1.0f, emax2);
  const float glo = lo - (4.0f * FLT_EPSILON * tnf + pivmin), ghi = hi + (4.0f * FLT_EPSILON * tnf + pivmin);
  lo = glo; hi = ghi;
  for (int it = 0; it < 64; ++it) {
    const float mid = 0.5f * (lo + hi);
    if (hi - lo <= 2.0f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + pivmin || mid <= lo || mid >= hi) break;
    if (sturm_count_f32(df, e2f, m, mid, pivmin) > idx) hi = mid; else lo = mid;
  }
  const double g = 0.5 * ((double)lo + (double)hi);
  const double pivmin64 = DBL_MIN * fmax(1.0, (double)emax2);
  double w = 8.0 * (double)FLT_EPSILON * (double)tnf + (double)pivmin;
  double dlo = g - w, dhi = g + w;
  bool ok = false;
  for (int t = 0; t < 3 && !ok; ++t) {
    ok = sturm_count_minors(d, e2, m, dlo) <= idx && sturm_count_minors(d, e2, m, dhi) > idx;
    if (!ok) { w *= 16.0; dlo = g - w; dhi = g + w; }
  }
  if (!ok) { dlo = (double)glo - w; dhi = (double)ghi + w; }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (dlo + dhi);
    const double am = fmax(fabs(dlo), fabs(dhi));
    if (dhi - dlo <= fmax(2.0 * DBL_EPSILON * am + pivmin64, rtol * (1.0 + am)) || mid <= dlo || mid >= dhi) break;
    if (sturm_count_minors(d, e2, m, mid) > idx) dhi = mid; else dlo = mid;
  }
  return 0.5 * (dlo + dhi);
}
}  // namespace fock
