// Stage (c): preconditioned block iteration for the lowest k eigenpairs of
// the box pencil (H, S) -- the paper's "structured iteration on subspace"
// (Sec. 2.3), read as LOBPCG (Knyazev 2001) with basis Y = [X | P | W],
// W = K (H X - S X Lambda) and K the shifted inverse of the circulant
// embedding (a Fourier-block solve).  All dense work is FP64.
//
//  k_init_x     deterministic pseudo-random start X (splitmix64 counter hash), P = W = 0
//  k_gemm_tn    G = A^T B            (Gram blocks of the Rayleigh-Ritz step; 16- or 20-wide tiles)
//  k_gemm_nn    C = beta C + alpha A B
//  k_resid      R = HX - SX diag(lambda), relative residual norms, soft locking
//  k_rr         Rayleigh-Ritz: diagonal scaling, pivoted LDL^T of Y^T S Y (rank-revealing),
//               C = Delta^-1/2 L^-1 (Y^T H Y) L^-T Delta^-1/2, Householder tridiagonal,
//               FP32 multisection shifts, FP64 inverse iteration (clusters of shifts in turn),
//               Cholesky-QR twice and a Rayleigh-Ritz step in their span, back-transformation;
//               lowest k
//  k_colnorm    unit 2-norm columns (non-finite ones zeroed)
//  k_copy_cols  column-block copies
//  k_gather     results of a batch into one staging buffer
//  k_cell_canon / k_cell_transform / k_cell_back
//               canonical cell basis and the exactly symmetric transformed operator
#include <float.h>
#include "common.cuh"

namespace fock {

// eigenvalue given to the cell directions dropped by the canonical transform
constexpr double kDecoupledEig = 1e6;
// k_rr runs 256 threads when its working matrices fit shared memory, 512 when
// they live in global memory (bases of 3 k > ~80 columns): twice the warps in
// flight for the global loads that then bound it
constexpr int kRRMaxThreads = 512;



__device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}



__global__ void k_init_x(const InitTask* __restrict__ tasks) {
  const InitTask T = tasks[blockIdx.y];
  const int tot = T.n * 3 * T.k;   // X random in [-1, 1); P and W zero
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int i = it % T.n, c = it / T.n;
    double v = 0.0;
    if (c < T.k) {
      uint64_t h = splitmix64(T.seed ^ splitmix64(((uint64_t)c << 32) | (uint64_t)i));
      v = 2.0 * ((double)(h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    T.X[(size_t)i + (size_t)T.ld * c] = v;
  }
}



// G = alpha A^T B (+ beta G), one output per thread of a 16 x 16 tile.  With
// T.sym the result is symmetric: tiles below the diagonal are skipped and the
// tiles above also write their transposes (diagonal tiles are computed in
// full and not mirrored, so no entry has two writers).
#define TT 16
// C = alpha A^T B + beta C on TILE x TILE output tiles, one thread per
// output; TILE = 20 when the block sizes are multiples of 20 (less padding
// than 16 for the 3k x 3k Gram and the k x k projections at k = 20).
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_gemm_tn(const GemmTask* __restrict__ tasks) {
  const GemmTask T = tasks[blockIdx.z];
  if (T.split) return;                       // computed on the tensor cores (mixed form)
  if (T.tile != TILE) return;                // the other tile size's launch
  if (T.active && *T.active == 0) return;
  const int i0 = blockIdx.x * TILE, j0 = blockIdx.y * TILE;
  if (i0 >= T.a || j0 >= T.b) return;
  if (T.sym && j0 < i0) return;
  __shared__ double As[TILE][TILE + 1], Bs[TILE][TILE + 1];
  const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
  // blocked summation: a partial sum over 8 tiles (128 or 160 terms) is added
  // to the total, so the rounding error of a sum over n terms grows like
  // (8 TILE + n / (8 TILE)) u instead of n u (n = 16384 on the 512-cell chains,
  // where the Gram entries of nearly dependent directions decide the pivots of
  // the Rayleigh-Ritz step)
  double acc = 0.0, blk = 0.0;
  int cnt = 0;
  for (int n0 = 0; n0 < T.n; n0 += TILE) {
    int r = n0 + tx;
    As[ty][tx] = (r < T.n && i0 + ty < T.a) ? T.A[(size_t)r + (size_t)T.lda * (i0 + ty)] : 0.0;
    Bs[ty][tx] = (r < T.n && j0 + ty < T.b) ? T.B[(size_t)r + (size_t)T.ldb * (j0 + ty)] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TILE; ++q) blk = fma(As[tx][q], Bs[ty][q], blk);
    __syncthreads();
    if (++cnt == 8) { acc += blk; blk = 0.0; cnt = 0; }
  }
  acc += blk;
  // thread (tx, ty) holds G[i0+tx][j0+ty]
  if (i0 + tx < T.a && j0 + ty < T.b) {
    double* g = T.C + (size_t)(i0 + tx) + (size_t)T.ldc * (j0 + ty);
    const double v = (T.beta == 0.0) ? T.alpha * acc : T.beta * *g + T.alpha * acc;
    *g = v;
    if (T.sym && j0 > i0) T.C[(size_t)(j0 + ty) + (size_t)T.ldc * (i0 + tx)] = v;
  }
}

// amax, bmax: largest output dimensions; tiles: bit 0 = some task uses 16,
// bit 1 = some task uses 20 (one launch per tile size, each skipping the
// other's tasks, so a problem's products never depend on its batch)
void launch_gemm_tn(const GemmTask* t, int n, int amax, int bmax, int tiles, cudaStream_t st) {
  if (!n) return;
  if (tiles & 1) k_gemm_tn<16><<<dim3((amax + 15) / 16, (bmax + 15) / 16, n), 256, 0, st>>>(t);
  if (tiles & 2) k_gemm_tn<20><<<dim3((amax + 19) / 20, (bmax + 19) / 20, n), 400, 0, st>>>(t);
}

// C = alpha A B + beta C; a thread owns row i of four consecutive columns,
// so each load of A serves four FP64 FMAs.
__global__ void k_gemm_nn(const GemmTask* __restrict__ tasks) {
  const GemmTask T = tasks[blockIdx.y];
  if (T.split) return;                       // computed on the tensor cores (mixed form)
  if (T.active && *T.active == 0) return;
  const int nb4 = (T.b + 3) >> 2;
  const int tot = T.n * nb4;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    const int i = it % T.n, j0 = (it / T.n) * 4;
    const int nj = min(4, T.b - j0);
    const double* b0 = T.B + (size_t)T.ldb * j0;
    const double* b1 = b0 + (nj > 1 ? T.ldb : 0);
    const double* b2 = b0 + (nj > 2 ? 2 * (size_t)T.ldb : 0);
    const double* b3 = b0 + (nj > 3 ? 3 * (size_t)T.ldb : 0);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int q = 0; q < T.a; ++q) {
      const double x = T.A[(size_t)i + (size_t)T.lda * q];
      a0 = fma(x, b0[q], a0); a1 = fma(x, b1[q], a1); a2 = fma(x, b2[q], a2); a3 = fma(x, b3[q], a3);
    }
    const double acc[4] = {a0, a1, a2, a3};
    for (int c = 0; c < nj; ++c) {
      double* cp = T.C + (size_t)i + (size_t)T.ldc * (j0 + c);
      *cp = (T.beta == 0.0) ? T.alpha * acc[c] : T.beta * *cp + T.alpha * acc[c];
    }
  }
}

// Columns at or below lock_tol get R = 0 (soft locking).
__global__ void k_resid(const ResidTask* __restrict__ tasks, double lock_tol) {
  const ResidTask T = tasks[blockIdx.y];
  if (T.active && *T.active == 0) return;
  const int c = blockIdx.x;
  if (c >= T.k) return;
  __shared__ double r1[256], r2[256];
  __shared__ double s_l;
  // Rayleigh quotient of the column from its fresh images: x^T H x / x^T S x
  double xh = 0.0, xs = 0.0;
  for (int i = threadIdx.x; i < T.n; i += blockDim.x) {
    size_t o = (size_t)i + (size_t)T.ld * c;
    xh += T.X[o] * T.HX[o];
    xs += T.X[o] * T.SX[o];
  }
  r1[threadIdx.x] = xh;
  r2[threadIdx.x] = xs;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { r1[threadIdx.x] += r1[threadIdx.x + s]; r2[threadIdx.x] += r2[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    s_l = (r2[0] > 0.0) ? r1[0] / r2[0] : T.lam[c];
    T.lam[c] = s_l;
  }
  __syncthreads();
  const double l = s_l;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < T.n; i += blockDim.x) {
    size_t o = (size_t)i + (size_t)T.ld * c;
    double sx = T.SX[o];
    double r = T.HX[o] - l * sx;
    T.R[o] = r;
    a += r * r;
    b += sx * sx;
  }
  r1[threadIdx.x] = a;
  r2[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { r1[threadIdx.x] += r1[threadIdx.x + s]; r2[threadIdx.x] += r2[threadIdx.x + s]; }
    __syncthreads();
  }
  __shared__ int lock;
  if (threadIdx.x == 0) {
    double den = fmax(fabs(l), 1e-300) * sqrt(r2[0]);
    // a column with no S-image (zero or non-finite) is broken, never converged
    double rv = (den > 0.0) ? sqrt(r1[0]) / den : NAN;
    T.res[c] = rv;
    lock = (rv <= lock_tol);
  }
  __syncthreads();
  if (lock)   // converged column: no search direction (the Rayleigh-Ritz step drops it)
    for (int i = threadIdx.x; i < T.n; i += blockDim.x) T.R[(size_t)i + (size_t)T.ld * c] = 0.0;
}



// Parallel cyclic Jacobi on the symmetric n x n matrix a (row-major, stride
// ld >= n + 1), round-robin pairing, A' = J^T A J; eigenvectors accumulated
// in v.  Odd n is padded with a decoupled huge diagonal entry.  At exit the
// eigenvalues are on the diagonal of a (unsorted).
__device__ void cta_jacobi(double* a, double* v, int n, int ld) {
  __shared__ double rc[128], rs[128];
  __shared__ int rp[128], rq[128];
  __shared__ int nrot;
  __shared__ double red[32], s_thr;
  const int ne = n + (n & 1);
  // rotation threshold: |a_pq| <= 1e-14 ||A||_F leaves the pair alone (rounding level)
  double part = 0.0;
  for (int it = threadIdx.x; it < n * n; it += blockDim.x) {
    double x = a[(it / n) * ld + (it % n)];
    part += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    s_thr = 1e-14 * sqrt(t);
  }
  for (int it = threadIdx.x; it < ne * ne; it += blockDim.x) {
    int i = it / ne, j = it % ne;
    v[i * ld + j] = (i == j) ? 1.0 : 0.0;
    if (i == n || j == n) a[i * ld + j] = (i == j) ? 1e300 : 0.0;
  }
  __syncthreads();
  const double thr = s_thr;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) nrot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int pi = threadIdx.x; pi < ne / 2; pi += blockDim.x) {
        int x = (pi == 0) ? 0 : ((pi - 1 + rnd) % (ne - 1)) + 1;
        int y = ((ne - 2 - pi + rnd) % (ne - 1)) + 1;
        int p = min(x, y), q = max(x, y);
        double apq = a[p * ld + q], app = a[p * ld + p], aqq = a[q * ld + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > thr && apq * apq > 1e-34 * fabs(app * aqq)) {   // |a_pq| > 1e-17 sqrt|a_pp a_qq|
          // reciprocals and square roots by Newton-Raphson from FP32 seeds
          const double th = (aqq - app) * (0.5 * rcp_nr(apq));
          const double y = fma(th, th, 1.0);
          double t = rcp_nr(fabs(th) + y * rsqrt_nr(y));
          if (th < 0.0) t = -t;
          c = rsqrt_nr(fma(t, t, 1.0));
          s = t * c;
          atomicAdd(&nrot, 1);
        }
        rp[pi] = p; rq[pi] = q; rc[pi] = c; rs[pi] = s;
      }
      __syncthreads();
      const int np2 = ne / 2;
      for (int it = threadIdx.x; it < np2 * ne; it += blockDim.x) {   // rows p, q
        int pi = it / ne, jj = it % ne;
        double s = rs[pi];
        if (s == 0.0) continue;
        int p = rp[pi], q = rq[pi];
        double c = rc[pi];
        double ap = a[p * ld + jj], aq = a[q * ld + jj];
        a[p * ld + jj] = c * ap - s * aq;
        a[q * ld + jj] = s * ap + c * aq;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < np2 * ne; it += blockDim.x) {   // columns p, q and v
        int pi = it / ne, ii = it % ne;
        double s = rs[pi];
        if (s == 0.0) continue;
        int p = rp[pi], q = rq[pi];
        double c = rc[pi];
        double ap = a[ii * ld + p], aq = a[ii * ld + q];
        a[ii * ld + p] = c * ap - s * aq;
        a[ii * ld + q] = s * ap + c * aq;
        double vp = v[ii * ld + p], vq = v[ii * ld + q];
        v[ii * ld + p] = c * vp - s * vq;
        v[ii * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    int done = (nrot == 0);
    __syncthreads();
    if (done) break;
  }
}

// ---- lowest eigenpairs of a dense symmetric matrix (whole CTA) ----
//
// FP64 cost model of this part (measured): a warp-wide FP64 instruction
// holds a sub-partition's FP64 unit for ~64 cycles with 1 or 32 active lanes
// alike, a division ~440 cycles, a square root ~690.  The phases below keep
// FP64 work in right-looking (trailing-update) form spread over all warps,
// compare doubles by their bit patterns, take reciprocals and inverse square
// roots by Newton-Raphson from FP32 seeds, and locate eigenvalues by FP32
// multisection.
//
// Shifts closer than kShiftCluster ||T|| form a cluster.  The FP32
// multisection places a shift within a few FP32 units of ||T|| of its
// eigenvalue, so two shifts in one such window can both lie much nearer one
// of the two eigenvalues; inverse iteration then turns both vectors into that
// one eigenvector, the Cholesky-QR below meets a singular Gram matrix, and
// the Ritz basis built from it loses rank.  Exactly degenerate pairs (a ring
// with two identical, distant defects) split, as the block iteration
// converges, by about lambda res^2, which crosses that window.  A cluster's
// vectors are therefore computed by one thread in turn, each orthogonalised
// against the cluster's earlier vectors after every solve (the
// reorthogonalisation of LAPACK's inverse iteration, dstein).
constexpr double kShiftCluster = 32.0 * FLT_EPSILON;
// The multisection's own resolution is far finer than that bound wherever
// ||T|| is far above the wanted eigenvalues (the Rayleigh-Ritz matrices of
// box chains), and clusters of the bound's width there chain long runs of
// well separated shifts into one thread.  So clusters are first tight
// (shifts whose final brackets lie within twice their widths: the ones the
// multisection could not tell apart), and the wide clusters are taken only
// when the first Cholesky factor of the vectors' Gram matrix meets a pivot
// below kDepPivot (a unit vector within 1e-5 of the span of the earlier ones).
constexpr double kDepPivot = 1e-10;

// Whether shift q (> 0) joins the cluster of shift q - 1: tight (brackets lo,
// hi of the multisection) or wide (kShiftCluster ||T||, tnorm = ||T||).
__device__ inline bool shift_clustered(const double* lam, const float* lo, const float* hi, int q,
                                       float tnorm, bool wide) {
  const double gap = lam[q] - lam[q - 1];
  if (wide) return gap <= kShiftCluster * (double)tnorm;
  const double w = (double)(hi[q] - lo[q]) + (double)(hi[q - 1] - lo[q - 1]);
  return gap <= 2.0 * w + 4.0 * FLT_EPSILON * fmax(fabs(lam[q]), fabs(lam[q - 1]));
}

// One inverse-iteration vector of the symmetric tridiagonal (d, e) of order r
// for the shift lm into column c of z (rows 0..r-1, stride ld): LU with
// partial pivoting of T - lm I (pivots below eps raised to eps; ws: 5 r
// doubles of workspace), start vector from a counter hash of (row, c), three
// sweeps of solve and normalisation.  Columns c0..c-1 (the earlier vectors
// of c's cluster, orthonormal) are projected out after every solve; with
// c0 == c the vector is the plain inverse iteration.
__device__ void inverse_iteration(const double* d, const double* e, int r, double lm, double eps,
                                  double* ws, double* z, int ld, int c, int c0) {
  double* lv = ws;                                   // multipliers
  double* rp = lv + r;                               // reciprocal pivots
  double* u1 = rp + r;
  double* u2 = u1 + r;
  double* pvt = u2 + r;                              // row swap flags (bit pattern tested)
  const long long eps_bits = abs_bits(eps);
  // LU of T - lm I with partial pivoting between rows i and i+1, branch-free
  double a0 = d[0] - lm, a1 = (r > 1) ? e[0] : 0.0;
  for (int i = 0; i + 1 < r; ++i) {
    const double sub = e[i], dn = d[i + 1] - lm, sn = (i + 2 < r) ? e[i + 1] : 0.0;
    const bool sw = abs_bits(sub) > abs_bits(a0);
    double p0 = sw ? sub : a0;
    const double p1 = sw ? dn : a1, p2 = sw ? sn : 0.0;
    const double o0 = sw ? a0 : sub, o1 = sw ? a1 : dn, o2 = sw ? 0.0 : sn;
    if (abs_bits(p0) < eps_bits) p0 = (__double_as_longlong(p0) < 0) ? -eps : eps;   // tiny pivot raised to eps
    const double rq = rcp_nr(p0);
    const double m = o0 * rq;
    lv[i] = m; rp[i] = rq; u1[i] = p1; u2[i] = p2; pvt[i] = sw ? 1.0 : 0.0;
    a0 = fma(-m, p1, o1);
    a1 = fma(-m, p2, o2);
  }
  if (abs_bits(a0) < eps_bits) a0 = (__double_as_longlong(a0) < 0) ? -eps : eps;
  rp[r - 1] = rcp_nr(a0);
  u1[r - 1] = 0.0; u2[r - 1] = 0.0;
  if (r >= 2) u2[r - 2] = 0.0;
  // start vector: counter hash of (row, vector), uniform in [0.5, 1.5)
  for (int i = 0; i < r; ++i) {
    const uint32_t h = (uint32_t)(splitmix64(((uint64_t)(c + 1) << 32) | (uint64_t)(i + 1)) >> 40);
    z[i * ld + c] = 0.5 + (double)h * (1.0 / 16777216.0);
  }
  for (int sweep = 0; sweep < 3; ++sweep) {
    for (int i = 0; i + 1 < r; ++i) {                // P and L^-1
      const double zi = z[i * ld + c], zn = z[(i + 1) * ld + c];
      const bool sw = __double_as_longlong(pvt[i]) != 0;
      const double bi = sw ? zn : zi, bn = sw ? zi : zn;
      z[i * ld + c] = bi;
      z[(i + 1) * ld + c] = fma(-lv[i], bi, bn);
    }
    double nxt = 0.0, nxt2 = 0.0, nn = 0.0;          // U^-1, and the squared norm
    for (int i = r - 1; i >= 0; --i) {
      double s = fma(-u1[i], nxt, z[i * ld + c]);
      s = fma(-u2[i], nxt2, s);
      s *= rp[i];
      z[i * ld + c] = s;
      nn = fma(s, s, nn);
      nxt2 = nxt; nxt = s;
    }
    if (c0 < c) {                                    // the cluster's earlier vectors projected out
      for (int p = c0; p < c; ++p) {
        double dp = 0.0;
        for (int i = 0; i < r; ++i) dp = fma(z[i * ld + p], z[i * ld + c], dp);
        for (int i = 0; i < r; ++i) z[i * ld + c] = fma(-dp, z[i * ld + p], z[i * ld + c]);
      }
      nn = 0.0;
      for (int i = 0; i < r; ++i) nn = fma(z[i * ld + c], z[i * ld + c], nn);
    }
    const double inv = (nn > 0.0 && isfinite(nn)) ? rsqrt_nr(nn) : 0.0;
    for (int i = 0; i < r; ++i) z[i * ld + c] *= inv;
  }
}

// Householder reduction to a tridiagonal T = Q^T A Q (A symmetric, only its
// lower triangle is read or kept; reflectors stay below the subdiagonal of
// a); the kk lowest eigenvalues of T by FP32 Sturm multisection; one FP64
// inverse-iteration vector per eigenvalue (one thread per cluster of shifts,
// see kShiftCluster); Cholesky-QR applied twice to those vectors and a
// Rayleigh-Ritz step in their span (Jacobi of the kk x kk projection of T),
// which restores orthogonality between clusters of close eigenvalues; z = Q y
// (groups of 8 lanes per vector).
// Eigenvector c lands in column c of z (rows 0..r-1, stride ld), eigenvalue
// c in lam[c], ascending.  scr: 4 ld^2 doubles of scratch.  d, e, tau, pv:
// shared arrays of >= 256 entries; ord: shared ints, >= kk + 1 entries.
__device__ void cta_sym_lowest(double* a, double* z, int r, int ld, int kk, double* scr,
                               double* d, double* e, double* tau, double* pv, double* lam, int* ord) {
  __shared__ double s_tau, s_K;
  double (*s_pw)[64] = reinterpret_cast<double (*)[64]>(lam);   // lam is written only at the end
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto A = [&](int i, int j) -> double& { return i >= j ? a[i * ld + j] : a[j * ld + i]; };
  for (int k = 0; k + 2 < r; ++k) {
    const int n = r - k - 1;                     // order of the trailing block
    if (warp == 0) {                             // x = a[k+1.., k]: norm, reflector, tau
      double part = 0.0;
      for (int i = k + 1 + lane; i < r; i += 32) part = fma(a[i * ld + k], a[i * ld + k], part);
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) {
        const double s = part;
        const double x0 = a[(k + 1) * ld + k];
        const double xn = (s > 0.0) ? s * rsqrt_nr(s) : 0.0;
        const double alpha = (x0 > 0.0) ? -xn : xn;
        const double vtv = 2.0 * (s - x0 * alpha);
        d[k] = a[k * ld + k];
        e[k] = alpha;
        s_tau = (vtv > 0.0) ? 2.0 * rcp_nr(vtv) : 0.0;
        tau[k] = s_tau;
        a[(k + 1) * ld + k] = x0 - alpha;       // v, first entry (the rest of x is v already)
      }
    }
    __syncthreads();
    const double tk = s_tau;
    if (__double_as_longlong(tk) == 0) continue;
    // p = tau A22 v: thread (part q, row k+1+ri) sums over every 4th column
    if (n <= 64) {
      const int q = threadIdx.x >> 6, ri = threadIdx.x & 63;
      if (ri < n && q < 4) {
        const int i = k + 1 + ri;
        double acc = 0.0;
        for (int j = k + 1 + q; j < r; j += 4) acc = fma(A(i, j), a[j * ld + k], acc);
        s_pw[q][ri] = acc;
      }
      __syncthreads();
      for (int ri2 = threadIdx.x; ri2 < n; ri2 += blockDim.x)
        pv[k + 1 + ri2] = tk * ((s_pw[0][ri2] + s_pw[1][ri2]) + (s_pw[2][ri2] + s_pw[3][ri2]));
    } else {
      for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) {
        double acc = 0.0;
        for (int j = k + 1; j < r; ++j) acc = fma(A(i, j), a[j * ld + k], acc);
        pv[i] = tk * acc;
      }
    }
    __syncthreads();
    if (warp == 0) {                             // K = (tau / 2) v^T p
      double kp = 0.0;
      for (int i = k + 1 + lane; i < r; i += 32) kp = fma(a[i * ld + k], pv[i], kp);
      for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xffffffffu, kp, o);
      if (lane == 0) s_K = 0.5 * tk * kp;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) pv[i] = fma(-s_K, a[i * ld + k], pv[i]);   // w
    __syncthreads();
    // A22 -= v w^T + w v^T on the lower triangle: linear index over rows of
    // 1, 2, ..., n entries
    const int nt = n * (n + 1) / 2;
    for (int it = threadIdx.x; it < nt; it += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * (float)it + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= it) ++ii;
      while (ii * (ii + 1) / 2 > it) --ii;
      const int jj = it - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      a[i * ld + j] -= fma(a[i * ld + k], pv[j], pv[i] * a[j * ld + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (r >= 2) {
      d[r - 2] = a[(r - 2) * ld + (r - 2)];
      d[r - 1] = a[(r - 1) * ld + (r - 1)];
      e[r - 2] = a[(r - 1) * ld + (r - 2)];
      if (r >= 3) tau[r - 2] = 0.0;
    } else {
      d[0] = a[0];
    }
  }
  __syncthreads();
  float tnorm;                                   // Gershgorin bound of |T|, FP32
  __shared__ float s_lo[128], s_hi[128];         // final multisection brackets (kk <= 128)
  // ---- kk lowest eigenvalues of T: FP32 Sturm multisection ----
  // Eigenvalue c is assigned a group of g = blockDim / kk threads; each round
  // the group counts the eigenvalues below g interior points of its bracket
  // and keeps the sub-interval holding eigenvalue c (g + 1 times narrower).
  {
    __shared__ int s_cnt[kRRMaxThreads];
    float* df = reinterpret_cast<float*>(pv);    // pv is free here: d and e^2 in FP32
    float* e2f = df + 256;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      df[i] = (float)d[i];
      e2f[i] = (i + 1 < r) ? (float)(e[i] * e[i]) : 0.0f;
    }
    __syncthreads();
    float glo = FLT_MAX, ghi = -FLT_MAX, emax2 = 0.0f;   // Gershgorin bounds (every thread)
    for (int i = 0; i < r; ++i) {
      const float rad = (i > 0 ? sqrtf(e2f[i - 1]) : 0.0f) + (i + 1 < r ? sqrtf(e2f[i]) : 0.0f);
      glo = fminf(glo, df[i] - rad);
      ghi = fmaxf(ghi, df[i] + rad);
      if (i + 1 < r) emax2 = fmaxf(emax2, e2f[i]);
    }
    tnorm = fmaxf(fabsf(glo), fabsf(ghi));
    const float pivmin = FLT_MIN * fmaxf(1.0f, emax2);
    glo -= 4.0f * FLT_EPSILON * tnorm + pivmin;
    ghi += 4.0f * FLT_EPSILON * tnorm + pivmin;
    const int g = max(1, (int)blockDim.x / max(kk, 1));
    const int grp = threadIdx.x / g, mem = threadIdx.x % g;
    for (int c = threadIdx.x; c < kk; c += blockDim.x) { s_lo[c] = glo; s_hi[c] = ghi; }
    __syncthreads();
    for (int round = 0; round < 40; ++round) {
      float x = 0.0f;
      if (grp < kk) {
        const float lo = s_lo[grp], hi = s_hi[grp];
        x = lo + (hi - lo) * ((float)(mem + 1) / (float)(g + 1));
        int cnt = 0;
        float q = df[0] - x;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += (q < 0.0f);
        for (int i = 1; i < r; ++i) {
          q = (df[i] - x) - __fdividef(e2f[i - 1], q);
          if (fabsf(q) < pivmin) q = -pivmin;
          cnt += (q < 0.0f);
        }
        s_cnt[threadIdx.x] = cnt;
      }
      __syncthreads();
      int open = 0;
      if (grp < kk && mem == 0) {                // the group's new bracket
        const float lo = s_lo[grp], hi = s_hi[grp];
        float nlo = lo, nhi = hi;
        for (int m = 0; m < g; ++m) {
          const float xm = lo + (hi - lo) * ((float)(m + 1) / (float)(g + 1));
          if (s_cnt[grp * g + m] > grp) { nhi = fminf(nhi, xm); break; }
          nlo = fmaxf(nlo, xm);
        }
        if (!(nlo < nhi)) nhi = nlo;             // bracket collapsed to rounding
        s_lo[grp] = nlo;
        s_hi[grp] = nhi;
        open = (nhi - nlo > 2.0f * FLT_EPSILON * fmaxf(fabsf(nlo), fabsf(nhi)) + pivmin);
      }
      if (!__syncthreads_or(open)) break;
    }
    for (int c = threadIdx.x; c < kk; c += blockDim.x) lam[c] = 0.5 * ((double)s_lo[c] + (double)s_hi[c]);
    __syncthreads();
  }
  // ---- inverse iteration: one thread per cluster of shifts (workspace 5 r per thread in scr),
  // tight clusters first, wide ones when the Gram factor below finds a dependent vector ----
  const int nw = max(1, min(kk, min((4 * ld * ld) / (5 * r), (int)blockDim.x)));
  auto vectors = [&](bool wide) {
    if (threadIdx.x < nw) {
      double* ws = scr + (size_t)threadIdx.x * 5 * r;
      const double eps = DBL_EPSILON * fmax((double)tnorm, DBL_MIN);
      for (int c = threadIdx.x; c < kk; c += nw) {
        if (c > 0 && shift_clustered(lam, s_lo, s_hi, c, tnorm, wide)) continue;   // its cluster's first thread
        for (int q = c; q < kk && (q == c || shift_clustered(lam, s_lo, s_hi, q, tnorm, wide)); ++q)
          inverse_iteration(d, e, r, lam[q], eps, ws, z, ld, q, c);
      }
    }
    __syncthreads();
  };
  // ---- Cholesky-QR, twice: Z <- Z L^-T with Z^T Z = L L^T (G in scr[ld^2, 2 ld^2)) ----
  double* s_rl = pv;                             // reciprocal diagonal of the Gram factor
  double* G = scr + (size_t)ld * ld;
  __shared__ int s_dep;
  // the Gram of the (unit) vectors and its Cholesky factor; with `track`, s_dep
  // = 1 when a pivot falls below kDepPivot (a vector nearly in the span of the
  // earlier ones)
  auto gram_factor = [&](bool track) {
    for (int it = threadIdx.x; it < kk * kk; it += blockDim.x) {
      const int c1 = it / kk, c2 = it % kk;
      if (c2 > c1) continue;
      double s = 0.0;
      for (int i = 0; i < r; ++i) s = fma(z[i * ld + c1], z[i * ld + c2], s);
      G[c1 * kk + c2] = s;
    }
    if (threadIdx.x == 0) s_dep = 0;
    __syncthreads();
    for (int j = 0; j < kk; ++j) {               // right-looking Cholesky, reciprocal diagonal in s_rl
      if (threadIdx.x == 0) {
        if (track && !(G[j * kk + j] >= kDepPivot)) s_dep = 1;
        const double gjj = fmax(G[j * kk + j], DBL_MIN);
        const double rl = rsqrt_nr(gjj);
        s_rl[j] = rl;
        G[j * kk + j] = gjj * rl;
      }
      __syncthreads();
      const double rl = s_rl[j];
      for (int i = j + 1 + threadIdx.x; i < kk; i += blockDim.x) G[i * kk + j] *= rl;
      __syncthreads();
      const int nt = kk - j - 1;
      for (int it = threadIdx.x; it < nt * nt; it += blockDim.x) {
        const int i = j + 1 + it / nt, l = j + 1 + it % nt;
        if (l <= i) G[i * kk + l] = fma(-G[i * kk + j], G[l * kk + j], G[i * kk + l]);
      }
      __syncthreads();
    }
  };
  auto apply = [&]() {
    for (int i = threadIdx.x; i < r; i += blockDim.x)   // row i of Z times L^-T
      for (int c = 0; c < kk; ++c) {
        double s = z[i * ld + c];
        for (int q = 0; q < c; ++q) s = fma(-z[i * ld + q], G[c * kk + q], s);
        z[i * ld + c] = s * s_rl[c];
      }
    __syncthreads();
  };
  vectors(false);
  gram_factor(true);
  if (s_dep) {                                   // uniform: read after the factor's last barrier
    vectors(true);
    gram_factor(false);
  }
  apply();
  gram_factor(false);
  apply();
  // ---- Rayleigh-Ritz in span(Z): Tz = Z^T (T Z), Jacobi (stride kj = kk + 1) ----
  const int kj = kk + 1;
  double* Tz = scr + (size_t)2 * ld * ld;
  double* Qz = scr + (size_t)3 * ld * ld;
  double* tmp = scr;   // r x kk: T Z, then Z Qz
  for (int it = threadIdx.x; it < r * kk; it += blockDim.x) {
    const int i = it / kk, c = it % kk;
    double s = d[i] * z[i * ld + c];
    if (i > 0) s = fma(e[i - 1], z[(i - 1) * ld + c], s);
    if (i + 1 < r) s = fma(e[i], z[(i + 1) * ld + c], s);
    tmp[it] = s;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kk * kk; it += blockDim.x) {
    const int c1 = it / kk, c2 = it % kk;
    if (c2 > c1) continue;
    double s = 0.0;
    for (int i = 0; i < r; ++i) s = fma(z[i * ld + c1], tmp[i * kk + c2], s);
    Tz[c1 * kj + c2] = s;
    Tz[c2 * kj + c1] = s;
  }
  __syncthreads();
  cta_jacobi(Tz, Qz, kk, kj);
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {   // ascending order, ties by index, NaN last:
    double di = Tz[i * kj + i];                          // the ranks are always a permutation
    if (isnan(di)) di = DBL_MAX;
    int rank = 0;
    for (int j = 0; j < kk; ++j) {
      double dj = Tz[j * kj + j];
      if (isnan(dj)) dj = DBL_MAX;
      rank += (dj < di) || (dj == di && j < i);
    }
    ord[rank] = i;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < r * kk; it += blockDim.x) {
    const int i = it / kk, c = it % kk, oc = ord[c];
    double s = 0.0;
    for (int q = 0; q < kk; ++q) s = fma(z[i * ld + q], Qz[q * kj + oc], s);
    tmp[it] = s;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < r * kk; it += blockDim.x) z[(it / kk) * ld + (it % kk)] = tmp[it];
  for (int c = threadIdx.x; c < kk; c += blockDim.x) lam[c] = Tz[ord[c] * kj + ord[c]];
  __syncthreads();
  // ---- back-transformation z = H_0 ... H_{r-3} y ----
  // a group of 8 lanes per vector, lane q of the group owning rows = q mod 8:
  // the dot product needs 3 shuffles and no block barrier
  {
    const int grp = threadIdx.x >> 3, q = threadIdx.x & 7;
    for (int c0 = 0; c0 < kk; c0 += (int)(blockDim.x >> 3)) {
      const int c = c0 + grp;
      const bool act = c < kk;
      if (__all_sync(0xffffffffu, !act)) continue;      // whole warp idle
      for (int k = r - 3; k >= 0; --k) {
        const double tk = tau[k];
        if (__double_as_longlong(tk) == 0) continue;
        const int i0 = k + 1 + ((q - (k + 1)) & 7);      // first owned row > k
        double s = 0.0;
        if (act)
          for (int i = i0; i < r; i += 8) s = fma(a[i * ld + k], z[i * ld + c], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s *= tk;
        if (act)
          for (int i = i0; i < r; i += 8) z[i * ld + c] = fma(-s, a[i * ld + k], z[i * ld + c]);
      }
    }
  }
  __syncthreads();
}

// Rayleigh-Ritz on the basis Y (Gram matrices GH = Y^T H Y, GS = Y^T S Y):
// scale by D = diag(GS)^-1/2; LDL^T factorisation of D GS D with diagonal
// pivoting (right-looking, through a permutation, unit lower factor L and
// pivots delta), stopping when the largest remaining pivot falls below
// kDropRel (the remaining columns are numerically in the span of the kept
// ones and are dropped, as are zero columns); with the kept set K the
// reduced matrix is C = Delta^-1/2 L^-1 (D GH D)_KK L^-T Delta^-1/2, whose k
// lowest eigenpairs give the Ritz pairs.  Coefficients in the Y basis:
// D P [L^-T Delta^-1/2 w; 0].
__global__ void __launch_bounds__(kRRMaxThreads) k_rr(const RRTask* __restrict__ tasks, int smem_bytes, int big) {
  const RRTask T = tasks[blockIdx.x];
  if (T.big != big) return;                 // the other launch's problems
  if (T.active && *T.active == 0) return;
  extern __shared__ double rr_smem[];
  // basis directions whose S-independent part is below kDropRel are dropped:
  // 1e-10 with FP64 images, 1e-6 while the images are FP32 (their noise level)
  const double kDropRel = (T.mode && *T.mode) ? 1e-6 : 1e-10;
  const int ld = T.ld, k = T.k, nb = T.nb;
  // working matrices in shared memory when 3 ld^2 doubles fit, else global.
  // The substitutions' staging (2 kRRBlock ld doubles) is shared memory: the
  // first ld^2 of the working matrices (C, free while they run) when those are
  // in shared memory and large enough, else dynamic shared memory of its own
  // (after the matrices, or all of it for matrices in global memory)
  const int xs = rr_stage_extra(ld);
  const bool in_smem = !big && ((3 * ld * ld + xs) * (int)sizeof(double) <= smem_bytes);
  double* base = in_smem ? rr_smem : T.work;
  double* rr_blk = !in_smem ? rr_smem : (xs ? rr_smem + (size_t)3 * ld * ld : rr_smem);
  double* C = base;                          // scaled H-Gram, then the reduced matrix (lower)
  double* V = base + (size_t)ld * ld;        // work matrix, then the eigenvectors
  double* G = base + (size_t)2 * ld * ld;    // scaled S-Gram (lower, original indices), then L
  __shared__ double dsc[256], rl[256];
  __shared__ long long wkey[kRRMaxThreads / 32];
  __shared__ int perm[256], order[256], wpos[kRRMaxThreads / 32];
  __shared__ double tdd[256], tee[256], ttau[256], tpv[256], tlam[256];
  __shared__ int s_r;
  __shared__ double s_rd;
  double* colS = tlam;                       // column of the Schur complement (until the eigensolver)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double g = T.GS[(size_t)i * ld + i];
    dsc[i] = (g > 0.0) ? rsqrt_nr(g) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  // lower triangles (i >= j, original indices) of D GS D and D GH D
  for (int it = threadIdx.x; it < nb * nb; it += blockDim.x) {
    const int i = it / nb, j = it % nb;
    if (j > i) continue;
    const double gs = 0.5 * (T.GS[(size_t)i + (size_t)ld * j] + T.GS[(size_t)j + (size_t)ld * i]);
    const double gh = 0.5 * (T.GH[(size_t)i + (size_t)ld * j] + T.GH[(size_t)j + (size_t)ld * i]);
    const double sc = dsc[i] * dsc[j];
    G[i * ld + j] = gs * sc;
    C[i * ld + j] = gh * sc;
  }
  if (threadIdx.x == 0) s_r = nb;
  __syncthreads();
  // S(a, b) at positions a, b: the lower-triangle entry of the original indices
  auto GP = [&](int pa, int pb) -> double& { return pa >= pb ? G[pa * ld + pb] : G[pb * ld + pa]; };
  for (int j = 0; j < nb; ++j) {
    // pivot: the largest remaining diagonal over positions j..nb-1 (bit-pattern
    // keys, ties to the lower position)
    long long bk = -2;
    int bi = j;
    for (int i = j + threadIdx.x; i < nb; i += blockDim.x) {
      const long long kq = pivot_key(G[perm[i] * ld + perm[i]]);
      if (kq > bk) { bk = kq; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long ok = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ok > bk || (ok == bk && oi < bi)) { bk = ok; bi = oi; }
    }
    if (lane == 0) { wkey[warp] = bk; wpos[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nwarp; ++w)
        if (wkey[w] > wkey[0] || (wkey[w] == wkey[0] && wpos[w] < wpos[0])) { wkey[0] = wkey[w]; wpos[0] = wpos[w]; }
      const int piv = wpos[0];
      const double dj = G[perm[piv] * ld + perm[piv]];
      if (!(wkey[0] >= 0 && dj > kDropRel)) {  // the diagonal scale is 1: drop below kDropRel
        s_r = j;
      } else {
        const int t = perm[j]; perm[j] = perm[piv]; perm[piv] = t;
        s_rd = rcp_nr(dj);
        rl[j] = rsqrt_nr(dj);
      }
    }
    __syncthreads();
    if (s_r == j) break;
    const int pj = perm[j];
    const double rd = s_rd;
    // column j: L(a, j) = S(a, j) / delta_j (stored in place), S(a, j) kept in colS
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      double& sij = GP(perm[i], pj);
      colS[i] = sij;
      sij *= rd;
    }
    __syncthreads();
    // trailing update S(a, b) -= L(a, j) S(b, j), a >= b > j
    const int n = nb - j - 1, nt = n * (n + 1) / 2;
    for (int it = threadIdx.x; it < nt; it += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * (float)it + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= it) ++ii;
      while (ii * (ii + 1) / 2 > it) --ii;
      const int aa = j + 1 + ii, bb = j + 1 + (it - ii * (ii + 1) / 2);
      double& s = GP(perm[aa], perm[bb]);
      s = fma(-GP(perm[aa], pj), colS[bb], s);
    }
    __syncthreads();
  }
  const int r = s_r;
  if (r < k && threadIdx.x == 0 && T.fail) *T.fail = 1;
  // V = (D GH D) at the kept positions: A(a, b) = C(perm a, perm b), a >= b
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {
    const int aa = it / r, bb = it % r;
    if (bb > aa) continue;
    const int pa = perm[aa], pb = perm[bb];
    V[aa * ld + bb] = pa >= pb ? C[pa * ld + pb] : C[pb * ld + pa];
    V[bb * ld + aa] = V[aa * ld + bb];
  }
  __syncthreads();
  auto Lp = [&](int aa, int bb) -> double { return GP(perm[aa], perm[bb]); };   // unit lower factor, aa > bb
  // V <- L^-1 V (right-looking over rows), then the lower triangle of V L^-T,
  // both blocked by kRRBlock pivot columns: the block's columns of L and its
  // finished rows (columns) of V are staged in shared memory, then every entry
  // outside the block takes the block's updates in one pass.  Each entry gets
  // the same fma sequence, in the same order, as in the unblocked
  // substitution; global traffic per fma falls from three accesses to about
  // two per block.
  constexpr int RB = kRRBlock;
  double* sL = rr_blk;                         // sL[q ld + a] = L(a, i0 + q), a > i0 + q
  double* sV = rr_blk + (size_t)RB * ld;       // the block's finished rows / columns of V
  for (int i0 = 0; i0 < r; i0 += RB) {
    const int nbk = min(RB, r - i0);
    for (int it = threadIdx.x; it < nbk * r; it += blockDim.x) {
      const int q = it / r, aa = it % r;
      sL[q * ld + aa] = (aa > i0 + q) ? Lp(aa, i0 + q) : 0.0;
    }
    __syncthreads();
    for (int col = threadIdx.x; col < r; col += blockDim.x) {   // the block's rows
      double v[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        if (q < nbk) {
          double t = V[(i0 + q) * ld + col];
#pragma unroll
          for (int p = 0; p < q; ++p) t = fma(-sL[p * ld + i0 + q], v[p], t);
          v[q] = t;
          V[(i0 + q) * ld + col] = t;
          sV[q * ld + col] = t;
        }
      }
    }
    __syncthreads();
    const int a0 = i0 + nbk, na = r - a0;
    for (int it = threadIdx.x; it < na * r; it += blockDim.x) {   // rows below the block
      const int aa = a0 + it / r, col = it % r;
      double t = V[aa * ld + col];
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (q < nbk) t = fma(-sL[q * ld + aa], sV[q * ld + col], t);
      V[aa * ld + col] = t;
    }
    __syncthreads();
  }
  for (int i0 = 0; i0 < r; i0 += RB) {         // columns a > i, rows x >= a
    const int nbk = min(RB, r - i0);
    for (int it = threadIdx.x; it < nbk * r; it += blockDim.x) {
      const int q = it / r, aa = it % r;
      sL[q * ld + aa] = (aa > i0 + q) ? Lp(aa, i0 + q) : 0.0;
    }
    __syncthreads();
    for (int x = i0 + threadIdx.x; x < r; x += blockDim.x) {   // the block's columns, rows x >= column
      double w[RB];
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        const int c = i0 + q;
        if (q < nbk && x >= c) {
          double t = V[x * ld + c];
#pragma unroll
          for (int p = 0; p < q; ++p) t = fma(-sL[p * ld + c], w[p], t);
          w[q] = t;
          V[x * ld + c] = t;
          sV[q * ld + x] = t;
        }
      }
    }
    __syncthreads();
    const int a0 = i0 + nbk, na = r - a0;
    for (int it = threadIdx.x; it < na * na; it += blockDim.x) {   // columns right of the block
      const int x = a0 + it / na, aa = a0 + it % na;
      if (aa > x) continue;
      double t = V[x * ld + aa];
#pragma unroll
      for (int q = 0; q < RB; ++q)
        if (q < nbk) t = fma(-sL[q * ld + aa], sV[q * ld + x], t);
      V[x * ld + aa] = t;
    }
    __syncthreads();
  }
  // C = Delta^-1/2 V Delta^-1/2, lower triangle
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {
    const int aa = it / r, bb = it % r;
    if (bb > aa) continue;
    C[aa * ld + bb] = V[aa * ld + bb] * (rl[aa] * rl[bb]);
  }
  __syncthreads();
  // the kk lowest eigenpairs of C (ascending) into the columns of V
  const int kk = min(k, r);
  cta_sym_lowest(C, V, r, ld, kk, T.work + (size_t)3 * ld * ld, tdd, tee, ttau, tpv, tlam, order);
  for (int c = threadIdx.x; c < k; c += blockDim.x) T.lam[c] = (c < kk) ? tlam[c] : NAN;
  // coefficients: w = L^-T Delta^-1/2 v (right-looking over positions, in V)
  for (int it = threadIdx.x; it < r * kk; it += blockDim.x) {
    const int aa = it / kk, c = it % kk;
    V[aa * ld + c] *= rl[aa];
  }
  __syncthreads();
  for (int aa = r - 1; aa > 0; --aa) {
    for (int it = threadIdx.x; it < aa * kk; it += blockDim.x) {
      const int qq = it / kk, c = it % kk;
      V[qq * ld + c] = fma(-Lp(aa, qq), V[aa * ld + c], V[qq * ld + c]);
    }
    __syncthreads();
  }
  // z[perm a] = D w[a]; the second block is z with the first k rows zeroed
  for (int it = threadIdx.x; it < k * nb; it += blockDim.x) {
    const int c = it / nb, i = it % nb;
    T.Cc[(size_t)ld * c + i] = 0.0;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kk * r; it += blockDim.x) {
    const int c = it / r, aa = it % r;
    const int p = perm[aa];
    T.Cc[(size_t)ld * c + p] = V[aa * ld + c] * dsc[p];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < k * nb; it += blockDim.x) {
    const int c = it / nb, i = it % nb;
    T.Cc[(size_t)ld * (k + c) + i] = (i < k) ? 0.0 : T.Cc[(size_t)ld * c + i];
  }
}

// One CTA per (column, task): scale dst's column to unit 2-norm (zero
// columns stay zero, non-finite ones become zero).
__global__ void k_colnorm(const CopyTask* __restrict__ tasks) {
  const CopyTask T = tasks[blockIdx.y];
  if (T.active && *T.active == 0) return;
  const int c = blockIdx.x;
  if (c >= T.ncols) return;
  double* col = T.dst + (size_t)T.ldd * c;
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < T.n; i += blockDim.x) s += col[i] * col[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) tot += red[w];
    red[0] = tot;
  }
  __syncthreads();
  const double nrm = sqrt(red[0]);
  if (!isfinite(nrm)) {   // a non-finite search direction: zeroed, so the Rayleigh-Ritz step drops it
    for (int i = threadIdx.x; i < T.n; i += blockDim.x) col[i] = 0.0;
    return;
  }
  if (!(nrm > 0.0)) return;
  const double inv = 1.0 / nrm;
  for (int i = threadIdx.x; i < T.n; i += blockDim.x) col[i] *= inv;
}

// One CTA per segment: dst[seg.dst + w] = seg.src[w].
__global__ void k_gather(const GatherSeg* __restrict__ segs, uint32_t* __restrict__ dst) {
  const GatherSeg g = segs[blockIdx.x];
  for (unsigned int w = threadIdx.x; w < g.words; w += blockDim.x) dst[g.dst + w] = g.src[w];
}

__global__ void k_copy_cols(const CopyTask* __restrict__ tasks) {
  const CopyTask T = tasks[blockIdx.y];
  if (T.active && *T.active == 0) return;
  const int tot = T.n * T.ncols;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int i = it % T.n, c = it / T.n;
    T.dst[(size_t)i + (size_t)T.ldd * c] = T.src[(size_t)i + (size_t)T.lds * c];
  }
}

}  // namespace fock

namespace fock {

// One CTA per chain on the structured path: the cell basis.  Jacobi
// eigendecomposition T_S[0] = Q diag(s) Q^T of the cell overlap, kept set
// K = {s > tau} in ascending Jacobi index with tau the dependency cut
// (common.cuh) formed from B = sum over offsets of |T_S[d]|, and
// Xc = Q_K diag(s_K)^-1/2 (m0 x m0, the columns past |K| zero).  A removed
// cell direction v spans vectors e_k (x) v, one per cell, on which the
// chain's overlap form is at most tau: numerically singular directions.
__global__ void k_cell_canon(const CanonTask* __restrict__ tasks) {
  extern __shared__ double cs[];
  const CanonTask T = tasks[blockIdx.x];
  const int m0 = T.m0, ld = m0 + 1;
  double* G = cs;                 // ld x ld
  double* Q = cs + ld * ld;       // ld x ld
  __shared__ double sv[MAXM0 + 1];
  __shared__ int keep[MAXM0 + 1], s_r;
  __shared__ double red[32], s_tau;
  double part = 0.0;
  for (int it = threadIdx.x; it < m0 * m0; it += blockDim.x) {
    int i = it / m0, j = it % m0;
    G[i * ld + j] = 0.5 * (T.TS[i * m0 + j] + T.TS[j * m0 + i]);
    double b = fabs(T.TS[it]);
    for (int d = 1; d <= T.D; ++d)
      b += fabs(T.TS[(size_t)d * m0 * m0 + it]) + (T.ring_full ? 0.0 : fabs(T.TS[(size_t)d * m0 * m0 + j * m0 + i]));
    part += b * b;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    s_tau = null_tau(sqrt(t), (double)T.nb);
  }
  cta_jacobi(G, Q, m0, ld);
  if (threadIdx.x == 0) {
    int r = 0;
    for (int i = 0; i < m0; ++i)
      if (G[i * ld + i] > s_tau && G[i * ld + i] > 0.0) { keep[r] = i; sv[r] = G[i * ld + i]; ++r; }
    s_r = r;
    *T.kept = r;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < m0 * m0; it += blockDim.x) {
    int mu = it / m0, j = it % m0;
    T.Xc[it] = (j < s_r) ? Q[mu * ld + keep[j]] / sqrt(sv[j]) : 0.0;
  }
}

// One CTA per block: B' = Xc^T B Xc.  Blocks: [0, D] generators (H then S),
// then the boundary blocks (H then S).  The dropped directions of the cell
// (zero columns of Xc) get a decoupled diagonal in T_H[0], T_S[0]: H = big,
// S = 1, so their eigenvalue `big` stays above every wanted one.
// Transformed blocks Xc^T B Xc of the generators and boundary blocks, made
// exactly symmetric where the operator is: the zero-offset generators and the
// diagonal boundary blocks are replaced by the mean of the product and its
// transpose, and a boundary pair (k, m) / (m, k) is written by the block with
// k < m as the mean of its product and the transpose of its partner's, the
// partner receiving the bitwise transpose.  (Xc carries factors up to
// tau^{-1/2}; products computed independently differ by rounding amplified by
// that factor squared, which would make the structured operator slightly
// non-symmetric and the one-sided Gram products of the block iteration
// inconsistent.)
__global__ void k_cell_transform(const CanonTask* __restrict__ tasks) {
  extern __shared__ double ts[];
  const CanonTask T = tasks[blockIdx.y];
  const int m0 = T.m0, m2 = m0 * m0;
  const int nblk = 2 * (T.D + 1) + 2 * T.nE;
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const double* src; const double* srcp = nullptr; double* dst; double* dstp = nullptr;
  const int g = T.D + 1;
  bool sym = false;
  if (b < 2 * g) {
    const int d = b < g ? b : b - g;
    src = (b < g ? T.TH : T.TS) + (size_t)d * m2;
    dst = (b < g ? T.THc : T.TSc) + (size_t)d * m2;
    sym = (d == 0);
  } else {
    const bool hs = b < 2 * g + T.nE;
    const int e = hs ? b - 2 * g : b - 2 * g - T.nE;
    const int pe = T.Epart ? T.Epart[e] : -1;
    const double* E = hs ? T.EH : T.ES;
    double* Ec = hs ? T.EHc : T.ESc;
    if (pe >= 0 && pe < e) return;        // written by its partner
    src = E + (size_t)e * m2;
    dst = Ec + (size_t)e * m2;
    if (pe == e) sym = true;
    else if (pe > e) { srcp = E + (size_t)pe * m2; dstp = Ec + (size_t)pe * m2; }
  }
  double* X = ts;
  double* Y = ts + m2;
  double* Yp = ts + 2 * m2;
  for (int it = threadIdx.x; it < m2; it += blockDim.x) X[it] = T.Xc[it];
  __syncthreads();
  for (int it = threadIdx.x; it < m2; it += blockDim.x) {   // Y = B Xc (and the partner's)
    int mu = it / m0, j = it % m0;
    double acc = 0.0, accp = 0.0;
    for (int nu = 0; nu < m0; ++nu) acc += src[mu * m0 + nu] * X[nu * m0 + j];
    Y[it] = acc;
    if (srcp) {
      for (int nu = 0; nu < m0; ++nu) accp += srcp[mu * m0 + nu] * X[nu * m0 + j];
      Yp[it] = accp;
    }
  }
  __syncthreads();
  const int r = *T.kept;
  const double* Yt = srcp ? Yp : Y;         // the product whose transpose is averaged in
  for (int it = threadIdx.x; it < m2; it += blockDim.x) {   // dst = Xc^T Y
    int i = it / m0, j = it % m0;
    double acc = 0.0;
    for (int mu = 0; mu < m0; ++mu) acc += X[mu * m0 + i] * Y[mu * m0 + j];
    if (sym || srcp) {
      double acct = 0.0;                    // (Xc^T Yt)[j][i]
      for (int mu = 0; mu < m0; ++mu) acct += X[mu * m0 + j] * Yt[mu * m0 + i];
      acc = 0.5 * (acc + acct);
    }
    if ((b == 0 || b == g) && i == j && i >= r) acc = (b == 0) ? kDecoupledEig : 1.0;
    dst[it] = acc;
    if (dstp) dstp[j * m0 + i] = acc;
  }
}

// V (original basis) = (I_L (x) Xc) V' for n = L m0 rows, ncol columns.
__global__ void k_cell_back(const double* __restrict__ Xc, int m0, int L, int ncol, const double* Vr,
                            double* V, int ld) {
  const int tot = L * m0 * ncol;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int mu = it % m0, rest = it / m0, cell = rest % L, c = rest / L;
    double acc = 0.0;
    for (int j = 0; j < m0; ++j) acc += Xc[mu * m0 + j] * Vr[(size_t)(cell * m0 + j) + (size_t)ld * c];
    V[(size_t)(cell * m0 + mu) + (size_t)ld * c] = acc;
  }
}

void launch_gather(const GatherSeg* segs, int n, uint32_t* dst, cudaStream_t st) {
  if (n) k_gather<<<n, 128, 0, st>>>(segs, dst);
}

void launch_cell_canon(const CanonTask* t, int n, int maxm0, int maxblk, cudaStream_t st) {
  if (!n) return;
  size_t sm = (size_t)2 * (maxm0 + 1) * (maxm0 + 1) * sizeof(double);
  k_cell_canon<<<n, 256, sm, st>>>(t);
  k_cell_transform<<<dim3(maxblk, n), 256, (size_t)3 * maxm0 * maxm0 * sizeof(double), st>>>(t);
}

void launch_cell_back(const double* Xc, int m0, int L, int ncol, const double* Vr, double* V, int ld,
                      cudaStream_t st) {
  k_cell_back<<<64, 256, 0, st>>>(Xc, m0, L, ncol, Vr, V, ld);
}

}  // namespace fock

namespace fock {

// ---- Rayleigh-Ritz on a thread-block cluster (bases in global memory) ----
//
// A basis too large for one CTA's shared memory (3 ld^2 doubles > 160 KB) is
// handled by a cluster of kRRCluster CTAs of kRRMaxThreads threads, so that
// one problem's step uses kRRCluster SMs' FP64 pipes instead of one.  The
// phases are those of k_rr / cta_sym_lowest with every per-entry operation
// unchanged: work that is independent per entry, row, column or vector is
// divided among the CTAs; small sequential decisions (pivots, reflectors, the
// kk x kk Cholesky and Jacobi steps) are repeated in every CTA from the same
// data, so all CTAs take the same branches and the results equal the
// single-CTA kernel's bit for bit.  The working matrices stay in the problem's
// global work array (L2); a CTA's copies of the small arrays live in its own
// shared memory.


// Barrier of the cluster's CTAs: the hardware cluster barrier, whose arrive
// has release and whose wait has acquire semantics at cluster scope, so every
// global-memory write of the cluster before it is seen by every read after it.
// Every CTA of a cluster reaches the same sequence of barriers: each branch on
// the way is taken on values that every CTA computes alike from data that no
// CTA changes until the next barrier (checked on the GPU with a form of this
// barrier whose waits were bounded: no wait ran out, and the results were the
// same).
__device__ bool cl_sync() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  return true;
}

// [lo, hi) of 0..n-1 for CTA `rank` of the cluster (contiguous shares)
__device__ inline int cl_lo(int n, int rank) { return (int)(((long long)n * rank) / kRRCluster); }

// cta_sym_lowest on a cluster (same phases, same per-entry arithmetic).
// a, z: r x r and r x kk in global memory (stride ld); scr: 4 ld^2 doubles of
// global scratch shared by the cluster; priv: this CTA's dynamic shared
// memory, >= 2 (kk + 1)^2 doubles (private copies for the small factorisations);
// d, e, tau, pv, lam, ord: this CTA's shared arrays as in cta_sym_lowest.
// Returns false when a cluster barrier ran out.
__device__ bool cl_sym_lowest(double* a, double* z, int r, int ld, int kk, double* scr, double* priv,
                              double* d, double* e, double* tau, double* pv, double* lam, int* ord,
                              int rank) {
  __shared__ double s_tau, s_K, s_v1;
  __shared__ double s_pw[4][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* pg = scr + (size_t)3 * ld * ld;        // p of the current column, shared by the cluster
  auto A = [&](int i, int j) -> double { return i >= j ? a[i * ld + j] : a[j * ld + i]; };
  // v of column k: its first entry (row k + 1) is this CTA's s_v1 until the
  // reduction ends, the rest are the column's entries below it
  // ---- Householder reduction to tridiagonal form ----
  for (int k = 0; k + 2 < r; ++k) {
    const int n = r - k - 1;
    if (warp == 0) {                             // reflector of column k (every CTA alike)
      double part = 0.0;
      for (int i = k + 1 + lane; i < r; i += 32) part = fma(a[i * ld + k], a[i * ld + k], part);
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) {
        const double s = part;
        const double x0 = a[(k + 1) * ld + k];
        const double xn = (s > 0.0) ? s * rsqrt_nr(s) : 0.0;
        const double alpha = (x0 > 0.0) ? -xn : xn;
        const double vtv = 2.0 * (s - x0 * alpha);
        d[k] = a[k * ld + k];
        e[k] = alpha;
        s_tau = (vtv > 0.0) ? 2.0 * rcp_nr(vtv) : 0.0;
        tau[k] = s_tau;
        s_v1 = x0 - alpha;
      }
    }
    __syncthreads();
    const double tk = s_tau, v1 = s_v1;
    if (__double_as_longlong(tk) == 0) continue;   // the same in every CTA: x = 0 below row k + 1
    auto vv = [&](int j) -> double { return j == k + 1 ? v1 : a[j * ld + k]; };
    // p = tau A22 v for this CTA's rows of the trailing block, into pg
    const int rlo = cl_lo(n, rank), rhi = cl_lo(n, rank + 1);
    if (n <= 64) {
      const int q = threadIdx.x >> 6, ri = rlo + (threadIdx.x & 63);
      if (q < 4 && ri < rhi) {
        const int i = k + 1 + ri;
        double acc = 0.0;
        for (int j = k + 1 + q; j < r; j += 4) acc = fma(A(i, j), vv(j), acc);
        s_pw[q][ri - rlo] = acc;
      }
      __syncthreads();
      for (int ri2 = rlo + threadIdx.x; ri2 < rhi; ri2 += blockDim.x) {
        const int o = ri2 - rlo;
        pg[k + 1 + ri2] = tk * ((s_pw[0][o] + s_pw[1][o]) + (s_pw[2][o] + s_pw[3][o]));
      }
    } else {
      for (int i = k + 1 + rlo + threadIdx.x; i < k + 1 + rhi; i += blockDim.x) {
        double acc = 0.0;
        for (int j = k + 1; j < r; ++j) acc = fma(A(i, j), vv(j), acc);
        pg[i] = tk * acc;
      }
    }
    if (!cl_sync()) return false;
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) pv[i] = pg[i];
    __syncthreads();
    if (warp == 0) {                             // K = (tau / 2) v^T p (every CTA alike)
      double kp = 0.0;
      for (int i = k + 1 + lane; i < r; i += 32) kp = fma(vv(i), pv[i], kp);
      for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xffffffffu, kp, o);
      if (lane == 0) s_K = 0.5 * tk * kp;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < r; i += blockDim.x) pv[i] = fma(-s_K, vv(i), pv[i]);   // w
    __syncthreads();
    // A22 -= v w^T + w v^T on the lower triangle, this CTA's share of its entries
    const int nt = n * (n + 1) / 2, tlo = cl_lo(nt, rank), thi = cl_lo(nt, rank + 1);
    for (int it = tlo + threadIdx.x; it < thi; it += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * (float)it + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= it) ++ii;
      while (ii * (ii + 1) / 2 > it) --ii;
      const int jj = it - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      a[i * ld + j] -= fma(vv(i), pv[j], pv[i] * vv(j));
    }
    if (rank == 0 && threadIdx.x == 0) a[(k + 1) * ld + k] = v1;   // read again only by the back-transformation
    if (!cl_sync()) return false;
  }
  if (threadIdx.x == 0) {
    if (r >= 2) {
      d[r - 2] = a[(r - 2) * ld + (r - 2)];
      d[r - 1] = a[(r - 1) * ld + (r - 1)];
      e[r - 2] = a[(r - 1) * ld + (r - 2)];
      if (r >= 3) tau[r - 2] = 0.0;
    } else {
      d[0] = a[0];
    }
  }
  __syncthreads();
  float tnorm;                                   // Gershgorin bound of |T|, FP32
  __shared__ float s_lo[128], s_hi[128];         // final multisection brackets (kk <= 128)
  // ---- kk lowest eigenvalues of T: FP32 Sturm multisection (every CTA alike) ----
  {
    __shared__ int s_cnt[kRRMaxThreads];
    float* df = reinterpret_cast<float*>(pv);    // pv is free here: d and e^2 in FP32
    float* e2f = df + 256;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
      df[i] = (float)d[i];
      e2f[i] = (i + 1 < r) ? (float)(e[i] * e[i]) : 0.0f;
    }
    __syncthreads();
    float glo = FLT_MAX, ghi = -FLT_MAX, emax2 = 0.0f;
    for (int i = 0; i < r; ++i) {
      const float rad = (i > 0 ? sqrtf(e2f[i - 1]) : 0.0f) + (i + 1 < r ? sqrtf(e2f[i]) : 0.0f);
      glo = fminf(glo, df[i] - rad);
      ghi = fmaxf(ghi, df[i] + rad);
      if (i + 1 < r) emax2 = fmaxf(emax2, e2f[i]);
    }
    tnorm = fmaxf(fabsf(glo), fabsf(ghi));
    const float pivmin = FLT_MIN * fmaxf(1.0f, emax2);
    glo -= 4.0f * FLT_EPSILON * tnorm + pivmin;
    ghi += 4.0f * FLT_EPSILON * tnorm + pivmin;
    const int g = max(1, (int)blockDim.x / max(kk, 1));
    const int grp = threadIdx.x / g, mem = threadIdx.x % g;
    for (int c = threadIdx.x; c < kk; c += blockDim.x) { s_lo[c] = glo; s_hi[c] = ghi; }
    __syncthreads();
    for (int round = 0; round < 40; ++round) {
      float x = 0.0f;
      if (grp < kk) {
        const float lo = s_lo[grp], hi = s_hi[grp];
        x = lo + (hi - lo) * ((float)(mem + 1) / (float)(g + 1));
        int cnt = 0;
        float q = df[0] - x;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += (q < 0.0f);
        for (int i = 1; i < r; ++i) {
          q = (df[i] - x) - __fdividef(e2f[i - 1], q);
          if (fabsf(q) < pivmin) q = -pivmin;
          cnt += (q < 0.0f);
        }
        s_cnt[threadIdx.x] = cnt;
      }
      __syncthreads();
      int open = 0;
      if (grp < kk && mem == 0) {
        const float lo = s_lo[grp], hi = s_hi[grp];
        float nlo = lo, nhi = hi;
        for (int m = 0; m < g; ++m) {
          const float xm = lo + (hi - lo) * ((float)(m + 1) / (float)(g + 1));
          if (s_cnt[grp * g + m] > grp) { nhi = fminf(nhi, xm); break; }
          nlo = fmaxf(nlo, xm);
        }
        if (!(nlo < nhi)) nhi = nlo;
        s_lo[grp] = nlo;
        s_hi[grp] = nhi;
        open = (nhi - nlo > 2.0f * FLT_EPSILON * fmaxf(fabsf(nlo), fabsf(nhi)) + pivmin);
      }
      if (!__syncthreads_or(open)) break;
    }
    for (int c = threadIdx.x; c < kk; c += blockDim.x) lam[c] = 0.5 * ((double)s_lo[c] + (double)s_hi[c]);
    __syncthreads();
  }
  // ---- inverse iteration: the cluster of shifts led by vector c on CTA c mod kRRCluster,
  // workspace 5 r at scr + 5 r c; tight clusters first, wide ones when the Gram
  // factor below finds a dependent vector (every CTA decides alike: the copies
  // it factors are equal) ----
  const double eps_ii = DBL_EPSILON * fmax((double)tnorm, DBL_MIN);
  auto vectors = [&](bool wide) -> bool {
    for (int c = rank + kRRCluster * (int)threadIdx.x; c < kk; c += kRRCluster * (int)blockDim.x) {
      if (c > 0 && shift_clustered(lam, s_lo, s_hi, c, tnorm, wide)) continue;   // its cluster's first thread
      for (int q = c; q < kk && (q == c || shift_clustered(lam, s_lo, s_hi, q, tnorm, wide)); ++q)
        inverse_iteration(d, e, r, lam[q], eps_ii, scr + (size_t)q * 5 * r, z, ld, q, c);
    }
    return cl_sync();
  };
  // ---- Cholesky-QR, twice: Gram entries shared out, each CTA factors its own copy ----
  double* s_rl = pv;                             // reciprocal diagonal of the Gram factor
  double* Gg = scr + (size_t)ld * ld;            // the Gram, shared by the cluster
  double* Gp = priv;                             // this CTA's copy, factored in place
  const int zlo = cl_lo(r, rank), zhi = cl_lo(r, rank + 1);   // this CTA's rows of Z
  __shared__ int s_dep;
  auto gram_factor = [&](bool track) -> bool {
    for (int it = cl_lo(kk * kk, rank) + threadIdx.x; it < cl_lo(kk * kk, rank + 1); it += blockDim.x) {
      const int c1 = it / kk, c2 = it % kk;
      if (c2 > c1) continue;
      double s = 0.0;
      for (int i = 0; i < r; ++i) s = fma(z[i * ld + c1], z[i * ld + c2], s);
      Gg[c1 * kk + c2] = s;
    }
    if (!cl_sync()) return false;
    for (int it = threadIdx.x; it < kk * kk; it += blockDim.x) Gp[it] = Gg[it];
    if (threadIdx.x == 0) s_dep = 0;
    __syncthreads();
    for (int j = 0; j < kk; ++j) {               // right-looking Cholesky, reciprocal diagonal in s_rl
      if (threadIdx.x == 0) {
        if (track && !(Gp[j * kk + j] >= kDepPivot)) s_dep = 1;
        const double gjj = fmax(Gp[j * kk + j], DBL_MIN);
        const double rlj = rsqrt_nr(gjj);
        s_rl[j] = rlj;
        Gp[j * kk + j] = gjj * rlj;
      }
      __syncthreads();
      const double rlj = s_rl[j];
      for (int i = j + 1 + threadIdx.x; i < kk; i += blockDim.x) Gp[i * kk + j] *= rlj;
      __syncthreads();
      const int nt = kk - j - 1;
      for (int it = threadIdx.x; it < nt * nt; it += blockDim.x) {
        const int i = j + 1 + it / nt, l = j + 1 + it % nt;
        if (l <= i) Gp[i * kk + l] = fma(-Gp[i * kk + j], Gp[l * kk + j], Gp[i * kk + l]);
      }
      __syncthreads();
    }
    return true;
  };
  auto apply = [&]() -> bool {
    for (int i = zlo + threadIdx.x; i < zhi; i += blockDim.x)   // row i of Z times L^-T
      for (int c = 0; c < kk; ++c) {
        double s = z[i * ld + c];
        for (int q = 0; q < c; ++q) s = fma(-z[i * ld + q], Gp[c * kk + q], s);
        z[i * ld + c] = s * s_rl[c];
      }
    return cl_sync();
  };
  if (!vectors(false) || !gram_factor(true)) return false;
  if (s_dep) {                                   // the workspace overlays the shared Gram: every
    if (!cl_sync()) return false;                // CTA has copied it before the vectors are redone
    if (!vectors(true) || !gram_factor(false)) return false;
  }
  if (!apply() || !gram_factor(false) || !apply()) return false;
  // ---- Rayleigh-Ritz in span(Z): Tz = Z^T (T Z) shared out, Jacobi on each CTA's copy ----
  const int kj = kk + 1;
  double* Tz = scr + (size_t)2 * ld * ld;
  double* tmp = scr;   // r x kk: T Z, then Z Qz
  double* Tp = priv;                               // (kk + 1) x kj
  double* Qp = priv + (size_t)kj * kj;             // (kk + 1) x kj
  for (int it = cl_lo(r * kk, rank) + threadIdx.x; it < cl_lo(r * kk, rank + 1); it += blockDim.x) {
    const int i = it / kk, c = it % kk;
    double s = d[i] * z[i * ld + c];
    if (i > 0) s = fma(e[i - 1], z[(i - 1) * ld + c], s);
    if (i + 1 < r) s = fma(e[i], z[(i + 1) * ld + c], s);
    tmp[it] = s;
  }
  if (!cl_sync()) return false;
  for (int it = cl_lo(kk * kk, rank) + threadIdx.x; it < cl_lo(kk * kk, rank + 1); it += blockDim.x) {
    const int c1 = it / kk, c2 = it % kk;
    if (c2 > c1) continue;
    double s = 0.0;
    for (int i = 0; i < r; ++i) s = fma(z[i * ld + c1], tmp[i * kk + c2], s);
    Tz[c1 * kj + c2] = s;
    Tz[c2 * kj + c1] = s;
  }
  if (!cl_sync()) return false;
  for (int it = threadIdx.x; it < kk * kk; it += blockDim.x) Tp[(it / kk) * kj + it % kk] = Tz[(it / kk) * kj + it % kk];
  __syncthreads();
  cta_jacobi(Tp, Qp, kk, kj);
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {   // ascending order, ties by index, NaN last
    double di = Tp[i * kj + i];
    if (isnan(di)) di = DBL_MAX;
    int rk = 0;
    for (int j = 0; j < kk; ++j) {
      double dj = Tp[j * kj + j];
      if (isnan(dj)) dj = DBL_MAX;
      rk += (dj < di) || (dj == di && j < i);
    }
    ord[rk] = i;
  }
  __syncthreads();
  for (int it = zlo * kk + threadIdx.x; it < zhi * kk; it += blockDim.x) {   // this CTA's rows of Z Qz
    const int i = it / kk, c = it % kk, oc = ord[c];
    double s = 0.0;
    for (int q = 0; q < kk; ++q) s = fma(z[i * ld + q], Qp[q * kj + oc], s);
    tmp[it] = s;
  }
  __syncthreads();
  for (int it = zlo * kk + threadIdx.x; it < zhi * kk; it += blockDim.x) z[(it / kk) * ld + (it % kk)] = tmp[it];
  for (int c = threadIdx.x; c < kk; c += blockDim.x) lam[c] = Tp[ord[c] * kj + ord[c]];
  if (!cl_sync()) return false;
  // ---- back-transformation z = H_0 ... H_{r-3} y of this CTA's vectors (c = rank mod kRRCluster) ----
  {
    const int grp = threadIdx.x >> 3, q = threadIdx.x & 7;
    const int nown = (kk - rank + kRRCluster - 1) / kRRCluster;
    for (int m0 = 0; m0 < nown; m0 += (int)(blockDim.x >> 3)) {
      const int m = m0 + grp, c = rank + kRRCluster * m;
      const bool act = m < nown;
      if (__all_sync(0xffffffffu, !act)) continue;
      for (int k = r - 3; k >= 0; --k) {
        const double tk = tau[k];
        if (__double_as_longlong(tk) == 0) continue;
        const int i0 = k + 1 + ((q - (k + 1)) & 7);
        double s = 0.0;
        if (act)
          for (int i = i0; i < r; i += 8) s = fma(a[i * ld + k], z[i * ld + c], s);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s *= tk;
        if (act)
          for (int i = i0; i < r; i += 8) z[i * ld + c] = fma(-s, a[i * ld + k], z[i * ld + c]);
      }
    }
  }
  __syncthreads();
  return true;
}

// k_rr for the problems with big = 1, one cluster of kRRCluster CTAs per task
// (grid = tasks x kRRCluster).  Dynamic shared memory: the substitutions' staging and
// the private copies of cl_sym_lowest (rr_cl_smem doubles).  If a barrier
// reported failure (a bounded form of cl_sync), the CTA would leave NaN in its
// coefficient columns, so that the problem's next residual is not finite and
// the iteration reports it unconverged.
__global__ void __launch_bounds__(kRRMaxThreads) k_rr_cl(const RRTask* __restrict__ tasks) {
  const RRTask T = tasks[blockIdx.x / kRRCluster];
  const int rank = blockIdx.x % kRRCluster;
  if (T.big != 1) return;                   // the same for the whole cluster
  if (T.active && *T.active == 0) return;
  extern __shared__ double rr_smem[];
  const double kDropRel = (T.mode && *T.mode) ? 1e-6 : 1e-10;
  const int ld = T.ld, k = T.k, nb = T.nb;
  double* C = T.work;                        // scaled H-Gram, then the reduced matrix (lower)
  double* V = T.work + (size_t)ld * ld;      // work matrix, then the eigenvectors
  double* G = T.work + (size_t)2 * ld * ld;  // scaled S-Gram (lower, original indices), then L
  double* rr_blk = rr_smem;                  // substitution staging, 2 kRRBlock ld
  double* priv = rr_smem + (size_t)2 * kRRBlock * ld;
  __shared__ double dsc[256], rl[256], rdv[256], colS[256], colL[256], dg[256];
  __shared__ long long wkey[kRRMaxThreads / 32];
  __shared__ int perm[256], order[256], wpos[kRRMaxThreads / 32];
  __shared__ double tdd[256], tee[256], ttau[256], tpv[256], tlam[256];
  __shared__ int s_r;
  __shared__ double s_rd;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  bool ok = true;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double g = T.GS[(size_t)i * ld + i];
    dsc[i] = (g > 0.0) ? rsqrt_nr(g) : 0.0;
    perm[i] = i;
  }
  __syncthreads();
  for (int it = cl_lo(nb * nb, rank) + threadIdx.x; it < cl_lo(nb * nb, rank + 1); it += blockDim.x) {
    const int i = it / nb, j = it % nb;
    if (j > i) continue;
    const double gs = 0.5 * (T.GS[(size_t)i + (size_t)ld * j] + T.GS[(size_t)j + (size_t)ld * i]);
    const double gh = 0.5 * (T.GH[(size_t)i + (size_t)ld * j] + T.GH[(size_t)j + (size_t)ld * i]);
    const double sc = dsc[i] * dsc[j];
    G[i * ld + j] = gs * sc;
    C[i * ld + j] = gh * sc;
  }
  if (threadIdx.x == 0) s_r = nb;
  ok = cl_sync();
  auto GP = [&](int pa, int pb) -> double& { return pa >= pb ? G[pa * ld + pb] : G[pb * ld + pa]; };
  // this CTA's copy of the diagonal (original indices), kept up to date with the
  // same fma as the trailing update, so that the pivot search reads nothing
  // another CTA is writing
  for (int i = threadIdx.x; i < nb; i += blockDim.x) dg[i] = G[i * ld + i];
  __syncthreads();
  // ---- pivoted LDL^T: pivots in every CTA alike, the trailing update shared
  // out; column j keeps S(., j) until the factorisation ends (colL holds its
  // scaled copy for the update), then every column is scaled to L in one pass
  for (int j = 0; ok && j < nb; ++j) {
    long long bk = -2;
    int bi = j;
    for (int i = j + threadIdx.x; i < nb; i += blockDim.x) {
      const long long kq = pivot_key(dg[perm[i]]);
      if (kq > bk) { bk = kq; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long okk = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (okk > bk || (okk == bk && oi < bi)) { bk = okk; bi = oi; }
    }
    if (lane == 0) { wkey[warp] = bk; wpos[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nwarp; ++w)
        if (wkey[w] > wkey[0] || (wkey[w] == wkey[0] && wpos[w] < wpos[0])) { wkey[0] = wkey[w]; wpos[0] = wpos[w]; }
      const int piv = wpos[0];
      const double dj = dg[perm[piv]];
      if (!(wkey[0] >= 0 && dj > kDropRel)) {
        s_r = j;
      } else {
        const int t = perm[j]; perm[j] = perm[piv]; perm[piv] = t;
        s_rd = rcp_nr(dj);
        rl[j] = rsqrt_nr(dj);
        rdv[j] = s_rd;
      }
    }
    __syncthreads();
    if (s_r == j) break;                      // the same j in every CTA
    const int pj = perm[j];
    const double rd = s_rd;
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      const double sij = GP(perm[i], pj);
      colS[i] = sij;
      colL[i] = __dmul_rn(sij, rd);           // the value the single-CTA kernel stores as L(i, j)
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      const int pi = perm[i];
      dg[pi] = fma(-colL[i], colS[i], dg[pi]);
    }
    const int n = nb - j - 1, nt = n * (n + 1) / 2;
    for (int it = cl_lo(nt, rank) + threadIdx.x; it < cl_lo(nt, rank + 1); it += blockDim.x) {
      int ii = (int)((sqrtf(8.0f * (float)it + 1.0f) - 1.0f) * 0.5f);
      while ((ii + 1) * (ii + 2) / 2 <= it) ++ii;
      while (ii * (ii + 1) / 2 > it) --ii;
      const int aa = j + 1 + ii, bb = j + 1 + (it - ii * (ii + 1) / 2);
      double& s = GP(perm[aa], perm[bb]);
      s = fma(-colL[aa], colS[bb], s);
    }
    if (!(ok = cl_sync())) break;
  }
  const int r = s_r;
  if (ok) {
    // L(a, j) = S(a, j) / delta_j for the kept pivots j < r, rows a > j: this CTA's rows
    for (int aa = cl_lo(nb, rank) + threadIdx.x; aa < cl_lo(nb, rank + 1); aa += blockDim.x)
      for (int jj = 0; jj < min(aa, r); ++jj) {
        double& s = GP(perm[aa], perm[jj]);
        s *= rdv[jj];
      }
    ok = cl_sync();
  }
  if (rank == 0 && threadIdx.x == 0 && r < k && T.fail) *T.fail = 1;
  auto Lp = [&](int aa, int bb) -> double { return GP(perm[aa], perm[bb]); };   // unit lower factor, aa > bb
  constexpr int RB = kRRBlock;
  double* sL = rr_blk;
  double* sV = rr_blk + (size_t)RB * ld;
  if (ok) {
    // V = (D GH D) at the kept positions, this CTA's columns; V <- L^-1 V on them
    const int clo = cl_lo(r, rank), chi = cl_lo(r, rank + 1), nc = chi - clo;
    for (int it = threadIdx.x; it < r * nc; it += blockDim.x) {
      const int aa = it / nc, col = clo + it % nc;
      const int pa = perm[aa], pb = perm[col];
      V[aa * ld + col] = pa >= pb ? C[pa * ld + pb] : C[pb * ld + pa];
    }
    __syncthreads();
    for (int i0 = 0; i0 < r; i0 += RB) {
      const int nbk = min(RB, r - i0);
      for (int it = threadIdx.x; it < nbk * r; it += blockDim.x) {
        const int q = it / r, aa = it % r;
        sL[q * ld + aa] = (aa > i0 + q) ? Lp(aa, i0 + q) : 0.0;
      }
      __syncthreads();
      for (int col = clo + threadIdx.x; col < chi; col += blockDim.x) {
        double v[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          if (q < nbk) {
            double t = V[(i0 + q) * ld + col];
#pragma unroll
            for (int p = 0; p < q; ++p) t = fma(-sL[p * ld + i0 + q], v[p], t);
            v[q] = t;
            V[(i0 + q) * ld + col] = t;
            sV[q * ld + col] = t;
          }
        }
      }
      __syncthreads();
      const int a0 = i0 + nbk, na = r - a0;
      for (int it = threadIdx.x; it < na * nc; it += blockDim.x) {
        const int aa = a0 + it / nc, col = clo + it % nc;
        double t = V[aa * ld + col];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < nbk) t = fma(-sL[q * ld + aa], sV[q * ld + col], t);
        V[aa * ld + col] = t;
      }
      __syncthreads();
    }
    ok = cl_sync();
  }
  if (ok) {
    // the lower triangle of V L^-T on this CTA's rows x = rank + kRRCluster m,
    // then C = Delta^-1/2 V Delta^-1/2 on them
    const int nm = (r - rank + kRRCluster - 1) / kRRCluster;   // rows of this CTA
    for (int i0 = 0; i0 < r; i0 += RB) {
      const int nbk = min(RB, r - i0);
      for (int it = threadIdx.x; it < nbk * r; it += blockDim.x) {
        const int q = it / r, aa = it % r;
        sL[q * ld + aa] = (aa > i0 + q) ? Lp(aa, i0 + q) : 0.0;
      }
      __syncthreads();
      const int mb = (i0 > rank) ? (i0 - rank + kRRCluster - 1) / kRRCluster : 0;   // first row >= i0
      for (int m = mb + threadIdx.x; m < nm; m += blockDim.x) {
        const int x = rank + kRRCluster * m;
        double w[RB];
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          const int c = i0 + q;
          if (q < nbk && x >= c) {
            double t = V[x * ld + c];
#pragma unroll
            for (int p = 0; p < q; ++p) t = fma(-sL[p * ld + c], w[p], t);
            w[q] = t;
            V[x * ld + c] = t;
            sV[q * ld + x] = t;
          }
        }
      }
      __syncthreads();
      const int a0 = i0 + nbk, na = r - a0;
      const int ma = (a0 > rank) ? (a0 - rank + kRRCluster - 1) / kRRCluster : 0;  // first row >= a0
      const int nmr = max(nm - ma, 0);
      for (int it = threadIdx.x; it < nmr * na; it += blockDim.x) {
        const int x = rank + kRRCluster * (ma + it / na), aa = a0 + it % na;
        if (aa > x) continue;
        double t = V[x * ld + aa];
#pragma unroll
        for (int q = 0; q < RB; ++q)
          if (q < nbk) t = fma(-sL[q * ld + aa], sV[q * ld + x], t);
        V[x * ld + aa] = t;
      }
      __syncthreads();
    }
    for (int it = threadIdx.x; it < nm * r; it += blockDim.x) {
      const int x = rank + kRRCluster * (it / r), bb = it % r;
      if (bb > x) continue;
      C[x * ld + bb] = V[x * ld + bb] * (rl[x] * rl[bb]);
    }
    ok = cl_sync();
  }
  const int kk = min(k, r);
  if (ok) ok = cl_sym_lowest(C, V, r, ld, kk, T.work + (size_t)3 * ld * ld, priv, tdd, tee, ttau, tpv, tlam,
                             order, rank);
  const int nown_k = (k - rank + kRRCluster - 1) / kRRCluster;   // this CTA's columns c = rank + kRRCluster m < k
  if (!ok) {
    for (int it = threadIdx.x; it < nown_k; it += blockDim.x) {
      const int c = rank + kRRCluster * it;
      T.Cc[(size_t)ld * c] = NAN;
      T.Cc[(size_t)ld * (k + c)] = NAN;
    }
    if (threadIdx.x == 0 && T.fail) *T.fail = 2;
    return;
  }
  if (rank == 0)
    for (int c = threadIdx.x; c < k; c += blockDim.x) T.lam[c] = (c < kk) ? tlam[c] : NAN;
  // coefficients of this CTA's columns: w = L^-T Delta^-1/2 v (right-looking over positions)
  const int nown = (kk - rank + kRRCluster - 1) / kRRCluster;
  for (int it = threadIdx.x; it < r * nown; it += blockDim.x) {
    const int aa = it / nown, c = rank + kRRCluster * (it % nown);
    V[aa * ld + c] *= rl[aa];
  }
  __syncthreads();
  for (int aa = r - 1; aa > 0; --aa) {
    for (int it = threadIdx.x; it < aa * nown; it += blockDim.x) {
      const int qq = it / nown, c = rank + kRRCluster * (it % nown);
      V[qq * ld + c] = fma(-Lp(aa, qq), V[aa * ld + c], V[qq * ld + c]);
    }
    __syncthreads();
  }
  // z[perm a] = D w[a]; the second block is z with the first k rows zeroed
  for (int it = threadIdx.x; it < nown_k * nb; it += blockDim.x) {
    const int c = rank + kRRCluster * (it / nb), i = it % nb;
    T.Cc[(size_t)ld * c + i] = 0.0;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nown * r; it += blockDim.x) {
    const int c = rank + kRRCluster * (it / r), aa = it % r;
    const int p = perm[aa];
    T.Cc[(size_t)ld * c + p] = V[aa * ld + c] * dsc[p];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nown_k * nb; it += blockDim.x) {
    const int c = rank + kRRCluster * (it / nb), i = it % nb;
    T.Cc[(size_t)ld * (k + c) + i] = (i < k) ? 0.0 : T.Cc[(size_t)ld * c + i];
  }
}

// doubles of dynamic shared memory k_rr_cl needs for leading dimension ld and k
size_t rr_cl_smem(int ld, int k) {
  return ((size_t)2 * kRRBlock * ld + (size_t)2 * (k + 1) * (k + 1)) * sizeof(double);
}

}  // namespace fock
