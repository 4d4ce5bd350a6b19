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
//  k_band_solve   forward and back substitution for the k columns of R;
//                 the columns of a problem are spread over several CTAs
//                 (they are independent), the D-term sums over threads
#include "common.cuh"

namespace fock {



__device__ inline double* bblk(double* band, int D, int m2, int J, int d) {
  return band + ((size_t)J * (D + 1) + d) * m2;
}

__global__ void k_band_factor(const BandTask* __restrict__ tasks) {
  const BandTask T = tasks[blockIdx.x];
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L;
  __shared__ double inv[MAXM0 * MAXM0];
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
      for (int c = 0; c < m0; ++c) {
        if (threadIdx.x == 0) {
          double dv = Ajj[c * m0 + c];
          if (!(dv > 0.0)) { bad = 1; dv = 1.0; }
          Ajj[c * m0 + c] = sqrt(dv);
        }
        __syncthreads();
        double dc = Ajj[c * m0 + c];
        for (int i = c + 1 + threadIdx.x; i < m0; i += blockDim.x) Ajj[i * m0 + c] /= dc;
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
          b[c] = s / Ajj[c * m0 + c];
        }
      }
      __syncthreads();
      // L_JJ^-1 (lower) into the diagonal slot: column c by forward substitution
      for (int c = threadIdx.x; c < m0; c += blockDim.x) {
        for (int i = 0; i < m0; ++i) {
          double s = (i == c) ? 1.0 : 0.0;
          if (i >= c)
            for (int q = c; q < i; ++q) s -= Ajj[i * m0 + q] * inv[q * m0 + c];
          inv[i * m0 + c] = (i >= c) ? s / Ajj[i * m0 + i] : 0.0;
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < m2; e += blockDim.x) Ajj[e] = inv[e];
      // trailing update: block (J+d1, J+d2) -= L[J+d1][J] L[J+d2][J]^T, 1 <= d2 <= d1 <= dmax
      const int npair = dmax * (dmax + 1) / 2;
      for (int it = threadIdx.x; it < npair * m2; it += blockDim.x) {
        int pr = it / m2, e = it % m2, mu = e / m0, nu = e % m0;
        int d1 = (int)((sqrt(8.0 * pr + 1.0) - 1.0) * 0.5);
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

template <typename R>
__global__ void k_band_solve(const BandTask* __restrict__ tasks) {
  const BandTask T = tasks[blockIdx.x];
  if (T.active && *T.active == 0) return;
  if ((T.fp32 != 0) != (sizeof(R) == 4)) return;
  const int c0 = blockIdx.y * kBandCols;
  if (c0 >= T.k) return;
  const int nc = min(kBandCols, T.k - c0);
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L, ld = T.ld;
  const double* band = T.band;
  __shared__ R part[256];
  __shared__ R tv[MAXM0 * kBandCols];
  const int items = m0 * nc;
  const int nsplit = max(1, min((int)blockDim.x / items, 8));
  const int tid = threadIdx.x;
  const int item = tid % items, sp = tid / items;
  const bool on = sp < nsplit;
  const int mu = item % m0, c = c0 + item / m0;
  double* Wc = T.W + (size_t)ld * c;
  const double* Rc = T.R + (size_t)ld * c;
  // forward: y_J = L_JJ^-1 (r_J - sum_d L[J][J-d] y_{J-d})
  for (int J = 0; J < L; ++J) {
    R s = 0;
    if (on) {
      const int dmax = min(D, J);
      for (int d = 1 + sp; d <= dmax; d += nsplit) {
        const double* l = bblk(const_cast<double*>(band), D, m2, J - d, d) + mu * m0;   // block (J, J-d)
        const double* y = Wc + (size_t)((J - d) * m0);
        for (int q = 0; q < m0; ++q) s -= (R)l[q] * (R)y[q];
      }
      part[tid] = s;
    }
    __syncthreads();
    if (on && sp == 0) {
      R r = (R)Rc[(size_t)(J * m0 + mu)];
      for (int p2 = 0; p2 < nsplit; ++p2) r += part[p2 * items + item];
      tv[item] = r;
    }
    __syncthreads();
    if (on && sp == 0) {
      const double* iv = bblk(const_cast<double*>(band), D, m2, J, 0) + mu * m0;
      const int cb = (item / m0) * m0;
      R y = 0;
      for (int q = 0; q <= mu; ++q) y += (R)iv[q] * tv[cb + q];
      Wc[(size_t)(J * m0 + mu)] = (double)y;
    }
    __syncthreads();
  }
  // backward: x_J = L_JJ^-T (y_J - sum_d L[J+d][J]^T x_{J+d})
  for (int J = L - 1; J >= 0; --J) {
    R s = 0;
    if (on) {
      const int dmax = min(D, L - 1 - J);
      for (int d = 1 + sp; d <= dmax; d += nsplit) {
        const double* l = bblk(const_cast<double*>(band), D, m2, J, d);   // block (J+d, J): column mu
        const double* x = Wc + (size_t)((J + d) * m0);
        for (int q = 0; q < m0; ++q) s -= (R)l[q * m0 + mu] * (R)x[q];
      }
      part[tid] = s;
    }
    __syncthreads();
    if (on && sp == 0) {
      R r = (R)Wc[(size_t)(J * m0 + mu)];
      for (int p2 = 0; p2 < nsplit; ++p2) r += part[p2 * items + item];
      tv[item] = r;
    }
    __syncthreads();
    if (on && sp == 0) {
      const double* iv = bblk(const_cast<double*>(band), D, m2, J, 0);
      const int cb = (item / m0) * m0;
      R x = 0;
      for (int q = mu; q < m0; ++q) x += (R)iv[q * m0 + mu] * tv[cb + q];
      Wc[(size_t)(J * m0 + mu)] = (double)x;
    }
    __syncthreads();
  }
}

void launch_band_factor(const BandTask* t, int n, cudaStream_t st) {
  if (n) k_band_factor<<<n, 256, 0, st>>>(t);
}
void launch_band_solve(const BandTask* t, int n, int kmax, cudaStream_t st, bool mixed) {
  if (!n) return;
  const dim3 g(n, (kmax + kBandCols - 1) / kBandCols);
  k_band_solve<double><<<g, 256, 0, st>>>(t);
  if (mixed) k_band_solve<float><<<g, 256, 0, st>>>(t);
}

}  // namespace fock
