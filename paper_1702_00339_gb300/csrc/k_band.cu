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
//  k_band_solve   one CTA per problem: forward and back substitution for the
//                 k columns of R
#include "common.cuh"

namespace fock {



__device__ inline double* bblk(double* band, int D, int m2, int J, int d) {
  return band + ((size_t)J * (D + 1) + d) * m2;
}

__global__ void k_band_factor(const BandTask* __restrict__ tasks) {
  const BandTask T = tasks[blockIdx.x];
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L;
  __shared__ int bad;
  __shared__ double s_sigma;
  if (threadIdx.x == 0) s_sigma = *T.sigma0;
  __syncthreads();
  for (int attempt = 0; attempt < 4; ++attempt) {
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
    if (!bad) break;
    if (threadIdx.x == 0) s_sigma = sg - 0.05 * (1.0 + fabs(sg)) * (double)(1 << attempt);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *T.sigma_used = s_sigma;
    if (bad && T.fail) *T.fail = 1;
  }
}

// W = (L L^T)^-1 R for the k columns (thread per (row in block, column)).
__global__ void k_band_solve(const BandTask* __restrict__ tasks) {
  const BandTask T = tasks[blockIdx.x];
  if (T.active && *T.active == 0) return;
  const int m0 = T.m0, m2 = m0 * m0, D = T.D, L = T.L, k = T.k, ld = T.ld;
  double* band = const_cast<double*>(T.band);
  // forward: y_J = L_JJ^-1 (r_J - sum_d L[J][J-d] y_{J-d})
  for (int J = 0; J < L; ++J) {
    for (int it = threadIdx.x; it < m0 * k; it += blockDim.x) {
      int mu = it % m0, c = it / m0;
      double s = T.R[(size_t)(J * m0 + mu) + (size_t)ld * c];
      const int dmax = min(D, J);
      for (int d = 1; d <= dmax; ++d) {
        const double* l = bblk(band, D, m2, J - d, d) + mu * m0;   // block (J, J-d)
        const double* y = T.W + (size_t)((J - d) * m0) + (size_t)ld * c;
        for (int q = 0; q < m0; ++q) s += -l[q] * y[q];
      }
      T.W[(size_t)(J * m0 + mu) + (size_t)ld * c] = s;
    }
    __syncthreads();
    const double* Ljj = bblk(band, D, m2, J, 0);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      double* y = T.W + (size_t)(J * m0) + (size_t)ld * c;
      for (int mu = 0; mu < m0; ++mu) {
        double s = y[mu];
        for (int q = 0; q < mu; ++q) s -= Ljj[mu * m0 + q] * y[q];
        y[mu] = s / Ljj[mu * m0 + mu];
      }
    }
    __syncthreads();
  }
  // backward: x_J = L_JJ^-T (y_J - sum_d L[J+d][J]^T x_{J+d})
  for (int J = L - 1; J >= 0; --J) {
    for (int it = threadIdx.x; it < m0 * k; it += blockDim.x) {
      int mu = it % m0, c = it / m0;
      double s = T.W[(size_t)(J * m0 + mu) + (size_t)ld * c];
      const int dmax = min(D, L - 1 - J);
      for (int d = 1; d <= dmax; ++d) {
        const double* l = bblk(band, D, m2, J, d);   // block (J+d, J): column mu
        const double* x = T.W + (size_t)((J + d) * m0) + (size_t)ld * c;
        for (int q = 0; q < m0; ++q) s -= l[q * m0 + mu] * x[q];
      }
      T.W[(size_t)(J * m0 + mu) + (size_t)ld * c] = s;
    }
    __syncthreads();
    const double* Ljj = bblk(band, D, m2, J, 0);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      double* x = T.W + (size_t)(J * m0) + (size_t)ld * c;
      for (int mu = m0 - 1; mu >= 0; --mu) {
        double s = x[mu];
        for (int q = mu + 1; q < m0; ++q) s -= Ljj[q * m0 + mu] * x[q];
        x[mu] = s / Ljj[mu * m0 + mu];
      }
    }
    __syncthreads();
  }
}

void launch_band_factor(const BandTask* t, int n, cudaStream_t st) {
  if (n) k_band_factor<<<n, 256, 0, st>>>(t);
}
void launch_band_solve(const BandTask* t, int n, cudaStream_t st) {
  if (n) k_band_solve<<<n, 256, 0, st>>>(t);
}

}  // namespace fock
