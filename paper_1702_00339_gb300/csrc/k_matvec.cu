// Stage (c): the block-Toeplitz / block-circulant matvec by FFT over the
// lattice (block) index (Remark 3.2, Prop. A.1), plus the block-sparse
// boundary / defect perturbation E (Sec. 2.3 items (A), (B)).
//
//   y = C x (first L blocks) + E x,  C = sum_c pi^c (x) C_c of size M >= L + D,
//   xt_j = sum_{k<L} w^{jk} x_k,  yt_j = Chat_j xt_j,  y_k = (1/M) sum_j w^{-jk} yt_j,
//   w = exp(-2 pi i / M).
//
//  k_twiddle  table exp(-2 pi i t / M)
//  k_fft      batched mixed-radix Stockham FFT of the columns, two real
//             columns packed per complex transform (z = x1 + i x2); one CTA
//             holds a chunk of packed columns of one problem in shared memory
//  k_blockmul per Fourier index pair (j, M-j): m0 x m0 complex block times the
//             unpacked transforms of the real columns
//  k_eapply   y += E x over the block rows that carry boundary/defect blocks
#include <algorithm>

#include "common.cuh"

namespace fock {

__global__ void k_twiddle(CircDev* circs, int n) {
  const CircDev c = circs[blockIdx.y];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < c.M; t += gridDim.x * blockDim.x) {
    double s, co;
    sincospi(-2.0 * (double)t / (double)c.M, &s, &co);
    c.tw[t] = cmk(co, s);
  }
}



// dir = +1 forward (w), -1 inverse (conj w).
template <int DIR>
__global__ void k_fft(const FftTask* __restrict__ tasks) {
  extern __shared__ cplx sm[];
  const FftTask T = tasks[blockIdx.y];
  const CircDev C = *T.circ;
  const int M = C.M, CC = T.cc;
  const int npair = (T.ncol + 1) >> 1;    // two real columns per complex transform
  const int ncols = T.m0 * npair;
  const int c0 = blockIdx.x * CC;
  if (c0 >= ncols) return;
  const int ncc = min(CC, ncols - c0);
  cplx* A = sm;
  cplx* B = sm + (size_t)M * CC;
  // load
  for (int it = threadIdx.x; it < M * CC; it += blockDim.x) {
    int k = it / CC, cc = it % CC;
    cplx val = cmk(0.0, 0.0);
    if (cc < ncc) {
      int c = c0 + cc;
      if (DIR > 0) {
        if (k < T.L) {
          int mu = c % T.m0, p = c / T.m0;
          const double* xc = T.x + (size_t)(k * T.m0 + mu) + (size_t)T.ldx * (2 * p);
          val = cmk(xc[0], (2 * p + 1 < T.ncol) ? xc[T.ldx] : 0.0);
        }
      } else {
        val = T.X[(size_t)k * ncols + c];
      }
    }
    A[it] = val;
  }
  __syncthreads();
  int Ps = 1;
  for (int s = 0; s < C.nfac; ++s) {
    const int r = C.fac[s];
    const int Pn = Ps * r, m = M / Pn;
    const int nb = M / r;
    const int stepr = M / r;                 // w_r = tw[stepr]
    for (int it = threadIdx.x; it < nb * CC; it += blockDim.x) {
      const int b = it / CC, cc = it % CC;
      const int kp = b / Ps, j = b % Ps;
      // inputs times the stage twiddles w_{Pn}^{q j} = tw[q j m]
      cplx a[5];
      const int jm = j * m;
      for (int q = 0; q < r; ++q) {
        cplx x = A[(size_t)((kp + m * q) * Ps + j) * CC + cc];
        if (q) {
          cplx w = C.tw[(q * jm) % M];
          if (DIR < 0) w.y = -w.y;
          x = cmul(w, x);
        }
        a[q] = x;
      }
      cplx o[5];
      if (r == 2) {
        o[0] = cadd(a[0], a[1]);
        o[1] = csub(a[0], a[1]);
      } else if (r == 4) {
        cplx t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        cplx t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
        // multiply t3 by -i (forward) or +i (inverse)
        cplx t3r = (DIR > 0) ? cmk(t3.y, -t3.x) : cmk(-t3.y, t3.x);
        o[0] = cadd(t0, t2);
        o[2] = csub(t0, t2);
        o[1] = cadd(t1, t3r);
        o[3] = csub(t1, t3r);
      } else {   // r = 3 or 5: direct small DFT with the table's r-th roots
        for (int p = 0; p < r; ++p) {
          cplx acc = a[0];
          for (int q = 1; q < r; ++q) {
            cplx w = C.tw[((q * p) % r) * stepr];
            if (DIR < 0) w.y = -w.y;
            acc = cadd(acc, cmul(w, a[q]));
          }
          o[p] = acc;
        }
      }
      for (int p = 0; p < r; ++p) B[(size_t)(kp * Pn + j + Ps * p) * CC + cc] = o[p];
    }
    __syncthreads();
    cplx* t = A; A = B; B = t;
    Ps = Pn;
  }
  // store
  if (DIR > 0) {
    for (int it = threadIdx.x; it < M * CC; it += blockDim.x) {
      int k = it / CC, cc = it % CC;
      if (cc < ncc) T.X[(size_t)k * ncols + c0 + cc] = A[it];
    }
  } else {
    const double inv = 1.0 / (double)M;
    for (int it = threadIdx.x; it < T.L * CC; it += blockDim.x) {
      int k = it / CC, cc = it % CC;
      if (cc < ncc) {
        int c = c0 + cc, mu = c % T.m0, p = c / T.m0;
        size_t o = (size_t)(k * T.m0 + mu) + (size_t)T.ldy * (2 * p);
        double re = A[it].x * inv, im = A[it].y * inv;
        T.y[o] = (T.beta == 0.0) ? re : T.beta * T.y[o] + re;
        if (2 * p + 1 < T.ncol) {
          o += (size_t)T.ldy;
          T.y[o] = (T.beta == 0.0) ? im : T.beta * T.y[o] + im;
        }
      }
    }
  }
}



// Per Fourier index pair (j, M - j), j <= M/2.  X holds the transforms of
// column pairs packed as z = x1 + i x2, so X1_j = (Z_j + conj Z_{M-j}) / 2 and
// X2_j = -i (Z_j - conj Z_{M-j}) / 2.  With real generators
// Chat_{M-j} = conj(Chat_j), hence Y_{M-j} = conj(Y_j) for each real column,
// and the outputs are packed again as W = Y1 + i Y2 for the inverse transform.
__global__ void k_blockmul(const BmulTask* __restrict__ tasks) {
  extern __shared__ cplx sb[];
  const BmulTask T = tasks[blockIdx.y];
  const int j = blockIdx.x;
  if (2 * j > T.M) return;
  const int jm = (T.M - j) % T.M;
  const int m0 = T.m0, np = m0 * m0, nc = m0 * ((T.ncol + 1) >> 1);
  cplx* b1 = sb;
  cplx* b2 = sb + np;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    b1[pr] = T.B1[(size_t)j * np + pr];
    if (T.B2) b2[pr] = T.B2[(size_t)j * np + pr];
  }
  __syncthreads();
  const cplx* zj = T.X + (size_t)j * nc;
  const cplx* zm = T.X + (size_t)jm * nc;
  for (int it = threadIdx.x; it < nc; it += blockDim.x) {
    const int mu = it % m0, p = it / m0;
    cplx y1a = cmk(0.0, 0.0), y2a = cmk(0.0, 0.0), y1b = cmk(0.0, 0.0), y2b = cmk(0.0, 0.0);
    for (int nu = 0; nu < m0; ++nu) {
      const cplx a = zj[p * m0 + nu], b = zm[p * m0 + nu];
      const cplx x1 = cmk(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));    // (a + conj b) / 2
      const cplx x2 = cmk(0.5 * (a.y + b.y), -0.5 * (a.x - b.x));   // -i (a - conj b) / 2
      const cplx c1 = b1[mu * m0 + nu];
      y1a = cadd(y1a, cmul(c1, x1));
      y2a = cadd(y2a, cmul(c1, x2));
      if (T.B2) {
        const cplx c2 = b2[mu * m0 + nu];
        y1b = cadd(y1b, cmul(c2, x1));
        y2b = cadd(y2b, cmul(c2, x2));
      }
    }
    // W_j = Y1 + i Y2, W_{M-j} = conj(Y1) + i conj(Y2)
    T.Y1[(size_t)j * nc + it] = cmk(y1a.x - y2a.y, y1a.y + y2a.x);
    if (jm != j) T.Y1[(size_t)jm * nc + it] = cmk(y1a.x + y2a.y, -y1a.y + y2a.x);
    if (T.B2) {
      T.Y2[(size_t)j * nc + it] = cmk(y1b.x - y2b.y, y1b.y + y2b.x);
      if (jm != j) T.Y2[(size_t)jm * nc + it] = cmk(y1b.x + y2b.y, -y1b.y + y2b.x);
    }
  }
}

__global__ void k_eapply(const EApplyTask* __restrict__ tasks) {
  const EApplyTask T = tasks[blockIdx.y];
  const int m0 = T.m0, np = m0 * m0;
  const int tot = T.nrows * m0 * T.ncol;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int mu = it % m0, rest = it / m0;
    int ri = rest % T.nrows, v = rest / T.nrows;
    int row = T.rows[ri];
    double acc = 0.0;
    for (int e = T.rowptr[ri]; e < T.rowptr[ri + 1]; ++e) {
      const double* Eb = T.vals + (size_t)e * np + mu * m0;
      const double* xv = T.x + (size_t)T.cols[e] * m0 + (size_t)T.ldx * v;
      for (int nu = 0; nu < m0; ++nu) acc += Eb[nu] * xv[nu];
    }
    T.y[(size_t)row * m0 + mu + (size_t)T.ldy * v] += acc;
  }
}

// ---- launchers ----
void launch_twiddles(CircDev* circs, int n, cudaStream_t st) {
  if (n) k_twiddle<<<dim3(4, n), 256, 0, st>>>(circs, n);
}

size_t fft_smem(int M, int cc) { return (size_t)2 * M * cc * sizeof(cplx); }

void launch_fft(const FftTask* tasks, int ntask, int maxchunks, int maxM, int cc, int dir,
                cudaStream_t st) {
  if (!ntask) return;
  size_t sm = fft_smem(maxM, cc);
  if (dir > 0) {
    if (sm > 48 * 1024) FOCK_SMEM_OPTIN(k_fft<1>);
    k_fft<1><<<dim3(maxchunks, ntask), 256, sm, st>>>(tasks);
  } else {
    if (sm > 48 * 1024) FOCK_SMEM_OPTIN(k_fft<-1>);
    k_fft<-1><<<dim3(maxchunks, ntask), 256, sm, st>>>(tasks);
  }
}

void launch_blockmul(const BmulTask* tasks, int ntask, int maxM, int maxm0, cudaStream_t st) {
  if (!ntask) return;
  size_t sm = (size_t)2 * maxm0 * maxm0 * sizeof(cplx);
  if (sm > 48 * 1024) FOCK_SMEM_OPTIN(k_blockmul);
  k_blockmul<<<dim3(maxM / 2 + 1, ntask), 256, sm, st>>>(tasks);
}

// gx: CTAs per task, from the largest task's work (rows x m0 x columns / 256)
int eapply_grid(long long items) {
  long long g = (items + 255) / 256;
  return (int)std::min<long long>(2048, std::max<long long>(16, g));
}
void launch_eapply(const EApplyTask* tasks, int ntask, int gx, cudaStream_t st) {
  if (ntask) k_eapply<<<dim3(gx, ntask), 256, 0, st>>>(tasks);
}

}  // namespace fock
