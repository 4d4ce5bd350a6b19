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
//  k_blockmul per Fourier index: m0 x m0 complex block times the packed
//             columns (linear in them, so no unpacking is needed)
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



// Complex type of the working precision.
template <typename R> struct CT;
template <> struct CT<double> { using T = cplx; };
template <> struct CT<float> { using T = float2; };
template <typename C, typename R> __device__ inline C mkc(R a, R b) { C r; r.x = a; r.y = b; return r; }
template <typename C> __device__ inline C addc(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ inline C subc(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ inline C mulc(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// Does this launch variant handle the task?  mode null: FP64 only; else the
// problem's current precision (0 FP64, 1 FP32).
template <typename R> __device__ inline bool mode_match(const int* mode) {
  const int m = mode ? *mode : 0;
  return (sizeof(R) == 4) ? (m == 1) : (m == 0);
}

// dir = +1 forward (w), -1 inverse (conj w); R = double (FP64 form) or float
// (early iterations of the mixed form).  cc_arg > 0: columns per CTA for every
// task of the launch (a tuned width), else each task's own cc.  The arithmetic
// of a column does not depend on the width.
template <int DIR, typename R>
__global__ void k_fft(const FftTask* __restrict__ tasks, int cc_arg) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char fft_sbuf[];
  const FftTask T = tasks[blockIdx.y];
  if (!mode_match<R>(T.mode)) return;
  if (T.active && *T.active == 0) return;
  const CircDev Cd = *T.circ;
  const int M = Cd.M, CC = (cc_arg > 0) ? cc_arg : T.cc;
  const int npair = (T.ncol + 1) >> 1;    // two real columns per complex transform
  const int ncols = T.m0 * npair;
  const int c0 = blockIdx.x * CC;
  if (c0 >= ncols) return;
  const int ncc = min(CC, ncols - c0);
  C* A = reinterpret_cast<C*>(fft_sbuf);
  C* B = A + (size_t)M * CC;
  C* Xg = reinterpret_cast<C*>(T.X);
  // load
  for (int it = threadIdx.x; it < M * CC; it += blockDim.x) {
    int k = it / CC, cc = it % CC;
    C val = mkc<C, R>(0, 0);
    if (cc < ncc) {
      int c = c0 + cc;
      if (DIR > 0) {
        if (k < T.L) {
          int mu = c % T.m0, p = c / T.m0;
          const double* xc = T.x + (size_t)(k * T.m0 + mu) + (size_t)T.ldx * (2 * p);
          val = mkc<C, R>((R)xc[0], (2 * p + 1 < T.ncol) ? (R)xc[T.ldx] : (R)0);
        }
      } else {
        val = Xg[(size_t)k * ncols + c];
      }
    }
    A[it] = val;
  }
  __syncthreads();
  int Ps = 1;
  for (int s = 0; s < Cd.nfac; ++s) {
    const int r = Cd.fac[s];
    const int Pn = Ps * r, m = M / Pn;
    const int nb = M / r;
    for (int it = threadIdx.x; it < nb * CC; it += blockDim.x) {
      const int b = it / CC, cc = it % CC;
      const int kp = b / Ps, j = b % Ps;
      // inputs times the stage twiddles w_{Pn}^{q j} = tw[q j m]
      C a[5];
      const int jm = j * m;
      for (int q = 0; q < r; ++q) {
        C x = A[(size_t)((kp + m * q) * Ps + j) * CC + cc];
        if (q && j) {   // w^0 = 1 (the whole first stage)
          cplx w64 = Cd.tw[(q * jm) % M];
          C w = mkc<C, R>((R)w64.x, (R)(DIR < 0 ? -w64.y : w64.y));
          x = mulc(w, x);
        }
        a[q] = x;
      }
      C o[5];
      if (r == 2) {
        o[0] = addc(a[0], a[1]);
        o[1] = subc(a[0], a[1]);
      } else if (r == 4) {
        C t0 = addc(a[0], a[2]), t1 = subc(a[0], a[2]);
        C t2 = addc(a[1], a[3]), t3 = subc(a[1], a[3]);
        // multiply t3 by -i (forward) or +i (inverse)
        C t3r = (DIR > 0) ? mkc<C, R>(t3.y, -t3.x) : mkc<C, R>(-t3.y, t3.x);
        o[0] = addc(t0, t2);
        o[2] = subc(t0, t2);
        o[1] = addc(t1, t3r);
        o[3] = subc(t1, t3r);
      } else if (r == 3) {
        // o1,2 = a0 - (a1 + a2)/2 -/+ i sin(2pi/3) (a1 - a2) (forward; + / - inverse)
        const R h3 = (R)0.86602540378443864676;   // sin(2 pi / 3)
        C t1 = addc(a[1], a[2]);
        C t2 = mkc<C, R>(a[0].x - (R)0.5 * t1.x, a[0].y - (R)0.5 * t1.y);
        C d = subc(a[1], a[2]);
        C id = (DIR > 0) ? mkc<C, R>(h3 * d.y, -h3 * d.x) : mkc<C, R>(-h3 * d.y, h3 * d.x);
        o[0] = addc(a[0], t1);
        o[1] = addc(t2, id);
        o[2] = subc(t2, id);
      } else {   // r == 5
        const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;   // cos 2pi/5, cos 4pi/5
        const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;    // sin 2pi/5, sin 4pi/5
        C b1 = addc(a[1], a[4]), b2 = addc(a[2], a[3]);
        C d1 = subc(a[1], a[4]), d2 = subc(a[2], a[3]);
        C e1 = mkc<C, R>(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
        C e2 = mkc<C, R>(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
        C f1 = mkc<C, R>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);   // times -i (forward)
        C f2 = mkc<C, R>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        C g1 = (DIR > 0) ? mkc<C, R>(f1.y, -f1.x) : mkc<C, R>(-f1.y, f1.x);
        C g2 = (DIR > 0) ? mkc<C, R>(f2.y, -f2.x) : mkc<C, R>(-f2.y, f2.x);
        o[0] = addc(a[0], addc(b1, b2));
        o[1] = addc(e1, g1);
        o[4] = subc(e1, g1);
        o[2] = addc(e2, g2);
        o[3] = subc(e2, g2);
      }
      for (int p = 0; p < r; ++p) B[(size_t)(kp * Pn + j + Ps * p) * CC + cc] = o[p];
    }
    __syncthreads();
    C* t = A; A = B; B = t;
    Ps = Pn;
  }
  // store
  if (DIR > 0) {
    for (int it = threadIdx.x; it < M * CC; it += blockDim.x) {
      int k = it / CC, cc = it % CC;
      if (cc < ncc) Xg[(size_t)k * ncols + c0 + cc] = A[it];
    }
  } else {
    const double inv = 1.0 / (double)M;
    for (int it = threadIdx.x; it < T.L * CC; it += blockDim.x) {
      int k = it / CC, cc = it % CC;
      if (cc < ncc) {
        int c = c0 + cc, mu = c % T.m0, p = c / T.m0;
        size_t o = (size_t)(k * T.m0 + mu) + (size_t)T.ldy * (2 * p);
        double re = (double)A[it].x * inv, im = (double)A[it].y * inv;
        T.y[o] = (T.beta == 0.0) ? re : T.beta * T.y[o] + re;
        if (2 * p + 1 < T.ncol) {
          o += (size_t)T.ldy;
          T.y[o] = (T.beta == 0.0) ? im : T.beta * T.y[o] + im;
        }
      }
    }
  }
}

// Per Fourier index j: W_j = Chat_j Z_j on the packed columns.  A packed
// column is z = x1 + i x2 of two real columns; the operator is linear and the
// same for both, so Chat_j Z_j = Chat_j X1_j + i Chat_j X2_j, and the inverse
// transform returns y1 + i y2 with y1, y2 real (Chat_{M-j} = conj Chat_j).
template <typename R>
__global__ void k_blockmul(const BmulTask* __restrict__ tasks) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char bm_smem[];
  const BmulTask T = tasks[blockIdx.y];
  if (!mode_match<R>(T.mode)) return;
  if (T.active && *T.active == 0) return;
  const int j = blockIdx.x;
  if (j >= T.M) return;
  const int m0 = T.m0, np = m0 * m0, nc = m0 * ((T.ncol + 1) >> 1);
  // the blocks transposed in shared memory (b[nu][mu]): the lanes of a warp
  // take consecutive rows mu, so they read consecutive entries (a row-major copy
  // put all 32 lanes on the same banks for m0 = 32)
  C* b1 = reinterpret_cast<C*>(bm_smem);
  C* b2 = b1 + np;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    const int tr = (pr % m0) * m0 + pr / m0;
    cplx v = T.B1[(size_t)j * np + pr];
    b1[tr] = mkc<C, R>((R)v.x, (R)v.y);
    if (T.B2) { v = T.B2[(size_t)j * np + pr]; b2[tr] = mkc<C, R>((R)v.x, (R)v.y); }
  }
  __syncthreads();
  const C* zj = reinterpret_cast<const C*>(T.X) + (size_t)j * nc;
  C* Y1 = reinterpret_cast<C*>(T.Y1) + (size_t)j * nc;
  C* Y2 = reinterpret_cast<C*>(T.Y2) + (size_t)j * nc;
  for (int it = threadIdx.x; it < nc; it += blockDim.x) {
    const int mu = it % m0, p = it / m0;
    C a1 = mkc<C, R>(0, 0), a2 = mkc<C, R>(0, 0);
    // complex multiply-add as four fused multiply-adds (8 flops in 4 FP64
    // instructions, against 6 for a product then a sum)
    for (int nu = 0; nu < m0; ++nu) {
      const C x = zj[p * m0 + nu];
      const C u = b1[nu * m0 + mu];
      a1.x = fma(u.x, x.x, a1.x); a1.x = fma(-u.y, x.y, a1.x);
      a1.y = fma(u.x, x.y, a1.y); a1.y = fma(u.y, x.x, a1.y);
      if (T.B2) {
        const C w = b2[nu * m0 + mu];
        a2.x = fma(w.x, x.x, a2.x); a2.x = fma(-w.y, x.y, a2.x);
        a2.y = fma(w.x, x.y, a2.y); a2.y = fma(w.y, x.x, a2.y);
      }
    }
    Y1[it] = a1;
    if (T.B2) Y2[it] = a2;
  }
}

__global__ void k_eapply(const EApplyTask* __restrict__ tasks) {
  const EApplyTask T = tasks[blockIdx.y];
  if (T.mode && *T.mode != 0) return;
  if (T.active && *T.active == 0) return;
  const int m0 = T.m0, np = m0 * m0;
  const int tot = T.nrows * m0 * T.ncol;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int mu = it % m0, rest = it / m0;
    int ri = rest % T.nrows, v = rest / T.nrows;
    int row = T.rows[ri];
    double acc = 0.0, acc2 = 0.0;
    for (int e = T.rowptr[ri]; e < T.rowptr[ri + 1]; ++e) {
      const double* Eb = T.vals + (size_t)e * np + mu * m0;
      const double* xv = T.x + (size_t)T.cols[e] * m0 + (size_t)T.ldx * v;
      if (T.vals2) {   // H and S blocks on the same x: one pass over x
        const double* Eb2 = T.vals2 + (size_t)e * np + mu * m0;
        for (int nu = 0; nu < m0; ++nu) { acc += Eb[nu] * xv[nu]; acc2 += Eb2[nu] * xv[nu]; }
      } else {
        for (int nu = 0; nu < m0; ++nu) acc += Eb[nu] * xv[nu];
      }
    }
    T.y[(size_t)row * m0 + mu + (size_t)T.ldy * v] += acc;
    if (T.vals2) T.y2[(size_t)row * m0 + mu + (size_t)T.ldy * v] += acc2;
  }
}

// ---- launchers ----
void launch_twiddles(CircDev* circs, int n, cudaStream_t st) {
  if (n) k_twiddle<<<dim3(4, n), 256, 0, st>>>(circs, n);
}

size_t fft_smem(int M, int cc) { return (size_t)2 * M * cc * sizeof(cplx); }

// mixed: the batch has problems in the mixed form; their FP32 variant is
// launched too (each variant skips the tasks of the other precision).
static void fft_launch(const FftTask* tasks, int ntask, int maxchunks, int maxM, int cc, int dir,
                       cudaStream_t st, bool mixed, int cc_arg) {
  if (!ntask) return;
  size_t sm = fft_smem(maxM, cc);
  if (dir > 0) {
    FOCK_SMEM_OPTIN((k_fft<1, double>));
    k_fft<1, double><<<dim3(maxchunks, ntask), 256, sm, st>>>(tasks, cc_arg);
    if (mixed) {
      FOCK_SMEM_OPTIN((k_fft<1, float>));
      k_fft<1, float><<<dim3(maxchunks, ntask), 256, sm / 2, st>>>(tasks, cc_arg);
    }
  } else {
    FOCK_SMEM_OPTIN((k_fft<-1, double>));
    k_fft<-1, double><<<dim3(maxchunks, ntask), 256, sm, st>>>(tasks, cc_arg);
    if (mixed) {
      FOCK_SMEM_OPTIN((k_fft<-1, float>));
      k_fft<-1, float><<<dim3(maxchunks, ntask), 256, sm / 2, st>>>(tasks, cc_arg);
    }
  }
}

// columns per CTA from each task (cc: the largest, for the shared-memory size)
void launch_fft(const FftTask* tasks, int ntask, int maxchunks, int maxM, int cc, int dir,
                cudaStream_t st, bool mixed) {
  fft_launch(tasks, ntask, maxchunks, maxM, cc, dir, st, mixed, 0);
}

// every task with cc columns per CTA (the width chosen by the plan's tuner)
void launch_fft_cc(const FftTask* tasks, int ntask, int maxchunks, int maxM, int cc, int dir,
                   cudaStream_t st, bool mixed) {
  fft_launch(tasks, ntask, maxchunks, maxM, cc, dir, st, mixed, cc);
}

// largest columns per CTA whose two M-point buffers fit the opt-in shared memory
int fft_max_cc(int maxM) {
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_fft<1, double>) == cudaSuccess) mx -= (int)fa.sharedSizeBytes;
  int cc = 1;
  while (cc < 32 && fft_smem(maxM, 2 * cc) <= (size_t)mx) cc *= 2;
  return cc;
}

void launch_blockmul(const BmulTask* tasks, int ntask, int maxM, int maxm0, cudaStream_t st, bool mixed) {
  if (!ntask) return;
  size_t sm = (size_t)2 * maxm0 * maxm0 * sizeof(cplx);
  FOCK_SMEM_OPTIN(k_blockmul<double>);
  FOCK_SMEM_OPTIN(k_blockmul<float>);
  k_blockmul<double><<<dim3(maxM, ntask), 256, sm, st>>>(tasks);
  if (mixed) k_blockmul<float><<<dim3(maxM, ntask), 256, sm / 2, st>>>(tasks);
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
