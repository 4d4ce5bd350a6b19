// Stage (c): preconditioned block iteration for the lowest k eigenpairs of
// the box pencil (H, S) -- the paper's "structured iteration on subspace"
// (Sec. 2.3), read as LOBPCG (Knyazev 2001) with basis Y = [X | P | W],
// W = K (H X - S X Lambda) and K the shifted inverse of the circulant
// embedding (a Fourier-block solve).  All dense work is FP64.
//
//  k_init_x     deterministic pseudo-random start X (splitmix64 counter hash), P = W = 0
//  k_gemm_tn    G = A^T B            (Gram blocks of the Rayleigh-Ritz step)
//  k_gemm_nn    C = beta C + alpha A B
//  k_resid      R = HX - SX diag(lambda), relative residual norms
//  k_rr         Rayleigh-Ritz: diagonal scaling, Cholesky of Y^T S Y,
//               C = L^-1 (Y^T H Y) L^-T, parallel cyclic Jacobi, lowest k
//  k_copy_cols  column-block copies
#include <float.h>
#include "common.cuh"

namespace fock {


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



#define TT 16
__global__ void k_gemm_tn(const GemmTask* __restrict__ tasks) {
  const GemmTask T = tasks[blockIdx.z];
  if (T.active && *T.active == 0) return;
  const int i0 = blockIdx.x * TT, j0 = blockIdx.y * TT;
  if (i0 >= T.a || j0 >= T.b) return;
  __shared__ double As[TT][TT + 1], Bs[TT][TT + 1];
  const int tx = threadIdx.x % TT, ty = threadIdx.x / TT;
  double acc = 0.0;
  for (int n0 = 0; n0 < T.n; n0 += TT) {
    int r = n0 + tx;
    As[ty][tx] = (r < T.n && i0 + ty < T.a) ? T.A[(size_t)r + (size_t)T.lda * (i0 + ty)] : 0.0;
    Bs[ty][tx] = (r < T.n && j0 + ty < T.b) ? T.B[(size_t)r + (size_t)T.ldb * (j0 + ty)] : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TT; ++q) acc += As[tx][q] * Bs[ty][q];
    __syncthreads();
  }
  // thread (tx, ty) holds G[i0+tx][j0+ty]
  if (i0 + tx < T.a && j0 + ty < T.b) {
    double* g = T.C + (size_t)(i0 + tx) + (size_t)T.ldc * (j0 + ty);
    *g = (T.beta == 0.0) ? T.alpha * acc : T.beta * *g + T.alpha * acc;
  }
}

__global__ void k_gemm_nn(const GemmTask* __restrict__ tasks) {
  const GemmTask T = tasks[blockIdx.y];
  if (T.active && *T.active == 0) return;
  const int tot = T.n * T.b;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int i = it % T.n, j = it / T.n;
    double acc = 0.0;
    const double* bj = T.B + (size_t)T.ldb * j;
    for (int q = 0; q < T.a; ++q) acc += T.A[(size_t)i + (size_t)T.lda * q] * bj[q];
    double* c = T.C + (size_t)i + (size_t)T.ldc * j;
    *c = (T.beta == 0.0) ? T.alpha * acc : T.beta * *c + T.alpha * acc;
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
    double rv = (den > 0.0) ? sqrt(r1[0]) / den : 0.0;
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
        if (fabs(apq) > thr && fabs(apq) > 1e-17 * sqrt(fabs(app * aqq))) {
          double th = (aqq - app) / (2.0 * apq);
          double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
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

// Rayleigh-Ritz on the basis Y (Gram matrices GH = Y^T H Y, GS = Y^T S Y):
// scale by D = diag(GS)^-1/2, eigendecompose D GS D = Q diag(s) Q^T and keep
// the directions with s > kDropRel * max(s) (a numerically dependent basis
// loses its dependent directions instead of amplifying rounding), reduce
// B^T (D GH D) B with B = Q_kept diag(s)^-1/2, eigendecompose, keep the k
// lowest.  Coefficients in the Y basis: D B w.
__global__ void k_rr(const RRTask* __restrict__ tasks, int smem_bytes) {
  const RRTask T = tasks[blockIdx.x];
  if (T.active && *T.active == 0) return;
  const double kDropRel = 1e-10;
  extern __shared__ double rr_smem[];
  const int ld = T.ld, k = T.k, nb = T.nb;
  // working matrices in shared memory when 3 ld^2 doubles fit, else global
  const bool in_smem = (3 * ld * ld * (int)sizeof(double) <= smem_bytes);
  double* base = in_smem ? rr_smem : T.work;
  double* C = base;                          // scaled H-Gram / reduced matrix
  double* V = base + (size_t)ld * ld;        // eigenvectors / scratch
  double* G = base + (size_t)2 * ld * ld;    // scaled S-Gram, then B
  __shared__ double dsc[256], sv[256];
  __shared__ int keep[256], order[256];
  __shared__ int s_r;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    double g = T.GS[(size_t)i * ld + i];
    dsc[i] = (g > 0.0) ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nb * nb; it += blockDim.x) {
    int i = it / nb, j = it % nb;
    double gs = 0.5 * (T.GS[(size_t)i + (size_t)ld * j] + T.GS[(size_t)j + (size_t)ld * i]);
    double gh = 0.5 * (T.GH[(size_t)i + (size_t)ld * j] + T.GH[(size_t)j + (size_t)ld * i]);
    G[i * ld + j] = gs * dsc[i] * dsc[j];
    C[i * ld + j] = gh * dsc[i] * dsc[j];
  }
  __syncthreads();
  cta_jacobi(G, V, nb, ld);
  if (threadIdx.x == 0) {
    double smax = 0.0;
    for (int i = 0; i < nb; ++i) {
      double si = G[i * ld + i];
      if (si == si) smax = fmax(smax, si);
    }
    int r = 0;
    for (int i = 0; i < nb; ++i) {
      double si = G[i * ld + i];
      if (si == si && si > kDropRel * smax) { keep[r] = i; sv[r] = si; ++r; }
    }
    s_r = r;
    if (r < k && T.fail) *T.fail = 1;
  }
  __syncthreads();
  const int r = s_r;
  // B[i][c] = Q[i][keep c] / sqrt(s_c)  (into G)
  for (int it = threadIdx.x; it < nb * r; it += blockDim.x) {
    int i = it / r, c = it % r;
    G[i * ld + c] = V[i * ld + keep[c]] / sqrt(sv[c]);
  }
  __syncthreads();
  // V <- C B  (nb x r)
  for (int it = threadIdx.x; it < nb * r; it += blockDim.x) {
    int i = it / r, c = it % r;
    double acc = 0.0;
    for (int q = 0; q < nb; ++q) acc += C[i * ld + q] * G[q * ld + c];
    V[i * ld + c] = acc;
  }
  __syncthreads();
  // C <- B^T V  (r x r), symmetrised
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {
    int a = it / r, c = it % r;
    double acc = 0.0;
    for (int q = 0; q < nb; ++q) acc += G[q * ld + a] * V[q * ld + c];
    C[a * ld + c] = acc;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {
    int a = it / r, c = it % r;
    if (a < c) {
      double m = 0.5 * (C[a * ld + c] + C[c * ld + a]);
      C[a * ld + c] = m;
      C[c * ld + a] = m;
    }
  }
  __syncthreads();
  cta_jacobi(C, V, r, ld);
  // rank the eigenvalues (ties by index, NaN last), keep the k lowest
  for (int i = threadIdx.x; i < r; i += blockDim.x) order[i] = i;
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    double di = C[i * ld + i];
    if (isnan(di)) di = DBL_MAX;
    int rank = 0;
    for (int j = 0; j < r; ++j) {
      double dj = C[j * ld + j];
      if (isnan(dj)) dj = DBL_MAX;
      rank += (dj < di) || (dj == di && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  const int kk = min(k, r);
  for (int c = threadIdx.x; c < k; c += blockDim.x) T.lam[c] = (c < kk) ? C[order[c] * ld + order[c]] : NAN;
  // coefficients in the Y basis: D B w, and the P-update copy without the X rows
  for (int it = threadIdx.x; it < nb * k; it += blockDim.x) {
    int i = it % nb, c = it / nb;
    double acc = 0.0;
    if (c < kk) {
      int oc = order[c];
      for (int q = 0; q < r; ++q) acc += G[i * ld + q] * V[q * ld + oc];
      acc *= dsc[i];
    }
    T.Cc[(size_t)i + (size_t)ld * c] = acc;
    T.Cc[(size_t)i + (size_t)ld * (k + c)] = (i < k) ? 0.0 : acc;
  }
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
