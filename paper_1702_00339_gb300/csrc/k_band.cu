// Preconditioner of the box eigensolver: banded block Cholesky of H - sigma S.
//
// The box chain matrix is block banded: H = BToepl(T) + E with generators
// T_d = block (k+d, k), |d| <= D (Sec. 2.3, Remark 3.2) and the boundary blocks
// E.  A = H - sigma S, sigma below the spectrum (from the circulant
// embedding's Fourier blocks), is symmetric positive definite with the same
// band, so it factors as L L^T with L block lower banded (bandwidth D cells).
// W = A^-1 R is the shift-and-invert search direction of the block
// iteration.  Storage: band[J][d] = block (J+d, J) of A (then of L), d = 0..D.
//
//  k_band_factor  one CTA per problem: fill the band from T and E, factor it
//                 block column by block column; on a non-positive pivot lower
//                 sigma and start again (at most 4 attempts)
//                 (the diagonal slots then hold L_JJ^-1, which the solve
//                 applies as a mat-vec)
//  k_band_solve   forward and back substitution for the k columns of R:
//                 one CTA per problem, one warp per group of 4 columns; the
//                 next block row staged once per CTA in shared memory
//                 (double-buffered cp.async), solution rows in per-warp rings
#include "common.cuh"

namespace fock {



__device__ inline double* bblk(double* band, int D, int m2, int J, int d) {
  return band + ((size_t)J * (D + 1) + d) * m2;
}

__global__ void k_band_factor(const BandTask* __restrict__ tasks) {
  const BandTask T = tasks[blockIdx.x];
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L;
  __shared__ double inv[MAXM0 * MAXM0];
  __shared__ double rlv[MAXM0];              // reciprocal pivots of the diagonal block's factor
  __shared__ int bad, s_stop, s_nbis;
  __shared__ double s_sigma, s_ok, s_bad;
  if (threadIdx.x == 0) { s_sigma = *T.sigma0; s_ok = NAN; s_bad = NAN; s_nbis = 0; s_stop = 0; }
  __syncthreads();
  // Shift search: A = H - sigma S must be positive definite.  The first
  // sigma comes from the defect-free embedding; a bound state below that
  // band (a substituted nucleus) makes A indefinite.  Descend geometrically
  // until the factorisation succeeds, then bisect three times between the
  // last failing and the succeeding shift, which brackets lambda_min in
  // (ok, bad); the final shift is ok - (bad - ok), at least one bracket width
  // below lambda_min (close enough for a strong shift-invert preconditioner,
  // far enough for a well-conditioned factor), and the band holds its factor.
  for (int attempt = 0; attempt < 24; ++attempt) {
    const double sg = s_sigma;
    // fill: Toeplitz part, then the boundary blocks (lower band, k >= m)
    const int tot = L * (D + 1) * m2;
    for (int it = threadIdx.x; it < tot; it += blockDim.x) {
      int e = it % m2, d = (it / m2) % (D + 1);
      T.band[it] = T.TH[(size_t)d * m2 + e] - sg * T.TS[(size_t)d * m2 + e];
    }
    __syncthreads();
    for (int q = 0; q < T.nE; ++q) {           // entries of one block are disjoint
      int k = T.Ek[q], m = T.Em[q];
      if (k < m || k - m > D) continue;
      double* b = bblk(T.band, D, m2, m, k - m);
      for (int e = threadIdx.x; e < m2; e += blockDim.x)
        b[e] += T.EH[(size_t)q * m2 + e] - sg * T.ES[(size_t)q * m2 + e];
      __syncthreads();
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int J = 0; J < L; ++J) {
      double* Ajj = bblk(T.band, D, m2, J, 0);
      // Cholesky of the diagonal block (lower, in place)
      // (square roots and reciprocals by Newton-Raphson from FP32 seeds)
      for (int c = 0; c < m0; ++c) {
        if (threadIdx.x == 0) {
          double dv = Ajj[c * m0 + c];
          if (!(dv > 0.0)) { bad = 1; dv = 1.0; }
          const double rl = rsqrt_nr(dv);
          rlv[c] = rl;
          Ajj[c * m0 + c] = dv * rl;
        }
        __syncthreads();
        const double rl = rlv[c];
        for (int i = c + 1 + threadIdx.x; i < m0; i += blockDim.x) Ajj[i * m0 + c] *= rl;
        __syncthreads();
        const int nt = m0 - c - 1;
        for (int it = threadIdx.x; it < nt * nt; it += blockDim.x) {
          int i = c + 1 + it / nt, j = c + 1 + it % nt;
          if (j <= i) Ajj[i * m0 + j] -= Ajj[i * m0 + c] * Ajj[j * m0 + c];
        }
        __syncthreads();
      }
      if (bad) break;
      // L[J+d][J] = A[J+d][J] L_JJ^-T  (row-wise forward substitution)
      const int dmax = min(D, L - 1 - J);
      for (int it = threadIdx.x; it < dmax * m0; it += blockDim.x) {
        int d = 1 + it / m0, r = it % m0;
        double* b = bblk(T.band, D, m2, J, d) + r * m0;
        for (int c = 0; c < m0; ++c) {
          double s = b[c];
          for (int q = 0; q < c; ++q) s -= b[q] * Ajj[c * m0 + q];
          b[c] = s * rlv[c];
        }
      }
      __syncthreads();
      // L_JJ^-1 (lower) into the diagonal slot: column c by forward substitution
      for (int c = threadIdx.x; c < m0; c += blockDim.x) {
        for (int i = 0; i < m0; ++i) {
          double s = (i == c) ? 1.0 : 0.0;
          if (i >= c)
            for (int q = c; q < i; ++q) s -= Ajj[i * m0 + q] * inv[q * m0 + c];
          inv[i * m0 + c] = (i >= c) ? s * rlv[i] : 0.0;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < m2; e += blockDim.x) Ajj[e] = inv[e];
      // trailing update: block (J+d1, J+d2) -= L[J+d1][J] L[J+d2][J]^T, 1 <= d2 <= d1 <= dmax
      const int npair = dmax * (dmax + 1) / 2;
      for (int it = threadIdx.x; it < npair * m2; it += blockDim.x) {
        int pr = it / m2, e = it % m2, mu = e / m0, nu = e % m0;
        int d1 = (int)((sqrtf(8.0f * (float)pr + 1.0f) - 1.0f) * 0.5f);   // FP32: the loops below correct it
        while ((d1 + 1) * (d1 + 2) / 2 <= pr) ++d1;
        while (d1 * (d1 + 1) / 2 > pr) --d1;
        int d2 = pr - d1 * (d1 + 1) / 2;   // 0 <= d2 <= d1
        d1 += 1; d2 += 1;
        if (d1 == d2 && nu > mu) continue;  // diagonal block: lower triangle suffices
        const double* l1 = bblk(T.band, D, m2, J, d1) + mu * m0;
        const double* l2 = bblk(T.band, D, m2, J, d2) + nu * m0;
        double s = 0.0;
        for (int q = 0; q < m0; ++q) s += l1[q] * l2[q];
        bblk(T.band, D, m2, J + d2, d1 - d2)[e] -= s;
      }
      __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!bad) {
        s_ok = sg;
        if (isnan(s_bad) || s_nbis >= 3) s_stop = 1;
      } else {
        s_bad = sg;
      }
      if (!s_stop) {
        if (isnan(s_ok)) s_sigma = sg - 0.05 * (1.0 + fabs(sg)) * (double)(1 << min(attempt, 30));
        else if (s_nbis < 3) { s_sigma = 0.5 * (s_ok + s_bad); ++s_nbis; }
        else { s_sigma = s_ok - (s_bad - s_ok); s_nbis = 99; }   // refactor one bracket below
      }
    }
    __syncthreads();
    if (s_stop) break;
  }
  if (threadIdx.x == 0) {
    *T.sigma_used = s_sigma;
    if (!s_stop && T.fail) *T.fail = 1;
  }
}

// W = (L L^T)^-1 R.  blockIdx.y picks a group of kBandCols columns; a work
// item is (row mu of the block, column), and the nsplit threads of an item
// share its sum over the D off-diagonal blocks (partial sums reduced in
// shared memory).  The diagonal slots hold L_JJ^-1.  R = float: the same
// solve in FP32 arithmetic (mixed form: the preconditioner only shapes the
// search directions); each variant skips the tasks of the other.
constexpr int kBandCols = 4;

// 16-byte asynchronous global -> shared copies (L2 only), grouped per row
__device__ inline void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ inline void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ inline void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename R>
__global__ void __launch_bounds__(1024) k_band_solve(const BandTask* __restrict__ tasks, int stage, int ringd) {
  // One CTA per problem, one warp per group of kBandCols columns; lane l of
  // a warp owns the items l, l + 32, ... of a block row (item = (row mu,
  // column)).  A row's D-term sum and its diagonal-block product run inside
  // the warp.  When a block row of the band fits `stage` doubles (and m0 is
  // even, so blocks start on 16-byte boundaries), the CTA copies the next
  // row's blocks once into a shared-memory stage, for all its warps, while
  // they compute the current row (double-buffered cp.async), and each warp
  // keeps its last D + 1 solution rows in a shared-memory ring.
  extern __shared__ __align__(16) double bst[];
  const BandTask& T = tasks[blockIdx.x];
  if (T.active && *T.active == 0) return;
  if ((T.fp32 != 0) != (sizeof(R) == 4)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L, ld = T.ld;
  const int c0 = warp * kBandCols;
  const int nc = max(0, min(kBandCols, T.k - c0));
  const int items = m0 * nc;
  const double* band = T.band;
  double* W = T.W;
  const double* Rm = T.R;
  const int rw = m0 * kBandCols;              // one solution row of a warp's group
  const bool staged = stage > 0 && (m0 % 2 == 0) && (D + 1) * m2 <= stage && (D + 1) * rw <= ringd;
  double* buf0 = bst;
  double* buf1 = bst + stage;
  R* ring = reinterpret_cast<R*>(bst + 2 * (size_t)stage + (size_t)warp * ringd);
  R* tv = reinterpret_cast<R*>(bst + 2 * (size_t)stage + (size_t)(blockDim.x >> 5) * ringd) + warp * rw;
  const int ch = m2 / 2;   // 16-byte chunks per block
  // forward row J: slot d holds block (J, J - d) (d = 0: L_JJ^-1)
  auto fetch_fwd = [&](int J, double* dst) {
    const int nd = min(D, J) + 1;
    for (int it = threadIdx.x; it < nd * ch; it += blockDim.x) {
      const int d = it / ch, cq = it % ch;
      cp_async16(dst + d * m2 + 2 * cq, bblk(const_cast<double*>(band), D, m2, J - d, d) + 2 * cq);
    }
  };
  // backward row J: slot d holds block (J + d, J), stored contiguously from (J, 0)
  auto fetch_bwd = [&](int J, double* dst) {
    const int nd = min(D, L - 1 - J) + 1;
    const double* src = bblk(const_cast<double*>(band), D, m2, J, 0);
    for (int it = threadIdx.x; it < nd * ch; it += blockDim.x) cp_async16(dst + 2 * it, src + 2 * it);
  };
  // forward: y_J = L_JJ^-1 (r_J - sum_d L[J][J-d] y_{J-d})
  if (staged) { fetch_fwd(0, buf0); cp_async_commit(); }
  for (int J = 0; J < L; ++J) {
    const double* cur = nullptr;
    if (staged) {
      __syncthreads();                         // every warp is done with row J - 1's stage
      if (J + 1 < L) fetch_fwd(J + 1, (J & 1) ? buf0 : buf1);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();                         // row J's stage complete and visible
      cur = (J & 1) ? buf1 : buf0;
    }
    const int dmax = min(D, J);
    for (int i = lane; i < items; i += 32) {
      const int mu = i % m0, c = c0 + i / m0, cb = (i / m0) * m0;
      const double* Wc = W + (size_t)ld * c;
      R s = (R)Rm[(size_t)ld * c + J * m0 + mu];
      for (int d = 1; d <= dmax; ++d) {
        const double* l = (staged ? cur + d * m2 : bblk(const_cast<double*>(band), D, m2, J - d, d)) + mu * m0;
        if (staged) {
          const R* y = ring + ((J - d) % (D + 1)) * rw + cb;
          for (int q = 0; q < m0; ++q) s -= (R)l[q] * y[q];
        } else {
          const double* y = Wc + (size_t)((J - d) * m0);
          for (int q = 0; q < m0; ++q) s -= (R)l[q] * (R)y[q];
        }
      }
      tv[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < items; i += 32) {
      const int mu = i % m0, c = c0 + i / m0, cb = (i / m0) * m0;
      const double* iv = (staged ? cur : bblk(const_cast<double*>(band), D, m2, J, 0)) + mu * m0;
      R y = 0;
      for (int q = 0; q <= mu; ++q) y += (R)iv[q] * tv[cb + q];
      W[(size_t)ld * c + J * m0 + mu] = (double)y;
      if (staged) ring[(J % (D + 1)) * rw + cb + mu] = y;
    }
    __syncwarp();
  }
  if (staged) { cp_async_wait0(); __syncthreads(); }
  // backward: x_J = L_JJ^-T (y_J - sum_d L[J+d][J]^T x_{J+d})
  if (staged) { fetch_bwd(L - 1, buf0); cp_async_commit(); }
  for (int J = L - 1, step = 0; J >= 0; --J, ++step) {
    const double* cur = nullptr;
    if (staged) {
      __syncthreads();
      if (J > 0) fetch_bwd(J - 1, (step & 1) ? buf0 : buf1);
      cp_async_commit();
      cp_async_wait1();
      __syncthreads();
      cur = (step & 1) ? buf1 : buf0;
    }
    const int dmax = min(D, L - 1 - J);
    for (int i = lane; i < items; i += 32) {
      const int mu = i % m0, c = c0 + i / m0, cb = (i / m0) * m0;
      const double* Wc = W + (size_t)ld * c;
      R s = (R)Wc[(size_t)(J * m0 + mu)];
      for (int d = 1; d <= dmax; ++d) {
        const double* l = staged ? cur + d * m2 : bblk(const_cast<double*>(band), D, m2, J, d);   // block (J+d, J)
        if (staged) {
          const R* x = ring + ((J + d) % (D + 1)) * rw + cb;
          for (int q = 0; q < m0; ++q) s -= (R)l[q * m0 + mu] * x[q];
        } else {
          const double* x = Wc + (size_t)((J + d) * m0);
          for (int q = 0; q < m0; ++q) s -= (R)l[q * m0 + mu] * (R)x[q];
        }
      }
      tv[i] = s;
    }
    __syncwarp();
    for (int i = lane; i < items; i += 32) {
      const int mu = i % m0, c = c0 + i / m0, cb = (i / m0) * m0;
      const double* iv = staged ? cur : bblk(const_cast<double*>(band), D, m2, J, 0);
      R x = 0;
      for (int q = mu; q < m0; ++q) x += (R)iv[q * m0 + mu] * tv[cb + q];
      W[(size_t)ld * c + J * m0 + mu] = (double)x;
      if (staged) ring[(J % (D + 1)) * rw + cb + mu] = x;
    }
    __syncwarp();
  }
  if (staged) cp_async_wait0();
}

void launch_band_factor(const BandTask* t, int n, cudaStream_t st) {
  if (n) k_band_factor<<<n, 256, 0, st>>>(t);
}
// stage: doubles of the CTA's shared-memory stage (0: loads from global);
// ringrow: the largest (D + 1) m0 among the staged tasks (solution rings).
// One CTA per problem, one warp per kBandCols columns.
void launch_band_solve(const BandTask* t, int n, int kmax, int stage, int ringrow, cudaStream_t st, bool mixed) {
  if (!n) return;
  const int nwarp = (kmax + kBandCols - 1) / kBandCols;
  const int ringd = stage > 0 ? ((ringrow * kBandCols + 1) & ~1) : 0;   // doubles, even (16-byte stages)
  // stages, rings, and the per-warp row buffers (one row of a warp's group)
  const size_t sm = ((size_t)2 * stage + (size_t)nwarp * ringd) * sizeof(double) +
                    (size_t)nwarp * MAXM0 * kBandCols * sizeof(double);
  // (the 48 KB default covers static plus dynamic shared memory: always opt in)
  FOCK_SMEM_OPTIN(k_band_solve<double>);
  FOCK_SMEM_OPTIN(k_band_solve<float>);
  k_band_solve<double><<<n, nwarp * 32, sm, st>>>(t, stage, ringd);
  if (mixed) k_band_solve<float><<<n, nwarp * 32, sm, st>>>(t, stage, ringd);
}

// doubles of one band-solve stage for the largest block row among the tasks
// that can be staged (even m0), capped at 12 KB per stage
int band_stage_doubles(int maxrow) { return std::min(maxrow, 1536); }

}  // namespace fock
