// Stage (a): separable rank-R assembly (Lemma 2.1, Prop. 2.2, Lemma 3.4).
//
//  k_gref     nodal 1D GTO factors of the reference cell      (Sec. 2.4)
//  k_ptab_nodes / k_ptab
//             window-summed P0 Gaussian integrals per axis    (Eq. 2.13, Eq. 3.6);
//             k_ptab_nodes evaluates erfc once per cell endpoint (shared
//             memory), k_ptab (windows too wide for shared memory) per cell
//  k_deftab   one nucleus' P0 Gaussian integrals per axis     (defects)
//  k_gram_fold / k_gram_pot
//             1D Galerkin forms  X_f[mu][nu] = <g_{a,mu}, W_f g_{b,nu}>  with
//             W_f = S1, A1 or diag(p_t) (Lemma 2.1 display, Eqs. 2.16-2.17).
//             The potential of an interior node depends only on its node
//             modulo n0 (replicated cell), so the node sum folds first into
//             per-residue pair products Z[r][mu nu] and then contracts with
//             the n0-long potential rows: X_t = P_t . Z.
//  k_combine  Hadamard combine over the axes into m0 x m0 blocks
//             H = A/2 - V, S (Lemma 3.4, Eqs. 2.16-2.17); a wall block also
//             writes its transpose into the mirror entry (E(m,k) = E(k,m)^T).
//  k_axis_dft sparse DFT of the per-axis factors over the lattice offset
//             (Thm. 3.3: only 1D transforms of the factors are needed).
#include "common.cuh"

namespace fock {

// ---------------------------------------------------------------- K1 ----
// Segment = (problem, axis).  Items = m0*W (gref) or T*nr (ptab).


__global__ void k_gref(const ProbDev* __restrict__ probs, const SegDesc* __restrict__ segs) {
  const SegDesc sg = segs[blockIdx.y];
  const ProbDev& P = probs[sg.prob];
  const AxisDev& A = P.ax[sg.axis];
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < sg.count; it += gridDim.x * blockDim.x) {
    int mu = it / A.W, jj = it % A.W;
    int j = A.jlo + jj;
    double al = P.alpha[mu];
    int isp = (P.ang[mu] == sg.axis + 1);
    double f = P.frac[P.centre[mu] * 3 + sg.axis];
    double d = ((double)j + 0.5 - f * (double)P.n0) * P.h;
    if (A.per) {
      double period = (double)A.N * P.h;
      d = d - period * floor(d / period + 0.5);
    }
    double rcut = sqrt(log(1.0 / P.eps) / al);
    double v = 0.0;
    if (fabs(d) <= rcut) {
      double nrm = sqrt(sqrt(2.0 * al / 3.14159265358979323846));
      if (isp) nrm *= 2.0 * sqrt(al);
      v = nrm * exp(-al * d * d);
      if (isp) v *= d;
    }
    A.g[it] = v;
  }
}

// int_lo^hi exp(-t^2 s^2) ds, erfc in the tails.
__device__ inline double gauss_cell(double t, double lo, double hi) {
  double a = t * lo, b = t * hi, v;
  if (a >= 0.0) v = erfc(a) - erfc(b);
  else if (b <= 0.0) v = erfc(-b) - erfc(-a);
  else v = erf(b) - erf(a);
  return v * (0.88622692545275801365 / t);   // sqrt(pi)/2
}

__global__ void k_ptab(const ProbDev* __restrict__ probs, const SegDesc* __restrict__ segs) {
  const SegDesc sg = segs[blockIdx.y];
  const ProbDev& P = probs[sg.prob];
  const AxisDev& A = P.ax[sg.axis];
  const int L = A.L;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < sg.count; it += gridDim.x * blockDim.x) {
    int t = it / A.nr, rr = it % A.nr;
    int nu = t / P.R, q = t % P.R;
    double r = (double)(A.rlo + rr);
    double f = P.frac[nu * 3 + sg.axis];
    double tq = P.tq[q];
    double acc = 0.0;
    int hw = (L == 1) ? 0 : L / 2;
    // only window cells whose P0 integral exceeds the erfc(7) ~ 4e-23 tail:
    // the cell [u, u + h] must meet (-7/t, 7/t), u = (r - (k + f) n0) h
    const double reach = 7.0 / tq;
    const double cn = (double)P.n0 * P.h;
    const int klo = (int)fmax((double)-hw, floor((r * P.h - reach) / cn - f) - 1.0);
    const int khi = (int)fmin((double)hw, ceil((r * P.h + reach + P.h) / cn - f) + 1.0);
    for (int k = klo; k <= khi; ++k) {
      double w = (L > 1 && (L % 2 == 0) && (k == -hw || k == hw)) ? 0.5 : 1.0;
      double u = (r - ((double)k + f) * (double)P.n0) * P.h;   // lo - a, h units -> bohr
      acc += w * gauss_cell(tq, u, u + P.h);
    }
    A.p[it] = acc;
  }
}

// One CTA per (segment, potential term t): the erfc values at every cell
// endpoint of the window once (shared memory), then each reduced node's
// window sum from them.  Adjacent cells share endpoints, so each endpoint is
// evaluated once instead of twice per cell (and once for all the nodes whose
// windows meet there); the cell across the nucleus (endpoints of both
// signs) takes erf directly, as gauss_cell does.  Same cells and weights as
// k_ptab.
__global__ void k_ptab_nodes(const ProbDev* __restrict__ probs, const SegDesc* __restrict__ segs) {
  extern __shared__ double Eq[];
  const SegDesc sg = segs[blockIdx.y];
  const ProbDev& P = probs[sg.prob];
  const AxisDev& A = P.ax[sg.axis];
  const int t = blockIdx.x;
  if (t >= P.T) return;
  const int L = A.L, n0 = P.n0;
  const int hw = (L == 1) ? 0 : L / 2;
  const int nu = t / P.R, q = t % P.R;
  const double f = P.frac[nu * 3 + sg.axis];
  const double tq = P.tq[q];
  const double reach = 7.0 / tq;
  const double cn = (double)n0 * P.h;
  const int i0 = A.rlo - hw * n0;                 // endpoint index i of s_i = (i - f n0) h
  const int ni = A.nr + 2 * hw * n0 + 1;
  for (int j = threadIdx.x; j < ni; j += blockDim.x) {
    const double s = ((double)(i0 + j) - f * (double)n0) * P.h;
    // the cells kept below meet (-reach, reach): their endpoints lie within reach + h
    Eq[j] = (fabs(s) <= reach + 2.0 * P.h) ? erfc(tq * fabs(s)) : 0.0;
  }
  __syncthreads();
  const double sc = 0.88622692545275801365 / tq;   // sqrt(pi)/2 / t
  for (int rr = threadIdx.x; rr < A.nr; rr += blockDim.x) {
    const double r = (double)(A.rlo + rr);
    const int klo = (int)fmax((double)-hw, floor((r * P.h - reach) / cn - f) - 1.0);
    const int khi = (int)fmin((double)hw, ceil((r * P.h + reach + P.h) / cn - f) + 1.0);
    double acc = 0.0;
    for (int k = klo; k <= khi; ++k) {
      const double w = (L > 1 && (L % 2 == 0) && (k == -hw || k == hw)) ? 0.5 : 1.0;
      const int j = rr + (hw - k) * n0;           // cell [s_i, s_{i+1}], i = rlo + rr - k n0
      const double u = (r - ((double)k + f) * (double)n0) * P.h;
      const double a = tq * u, b = tq * (u + P.h);
      double v;
      if (a >= 0.0) v = Eq[j] - Eq[j + 1];
      else if (b <= 0.0) v = Eq[j + 1] - Eq[j];
      else v = erf(b) - erf(a);
      acc += w * (v * sc);
    }
    A.p[(size_t)t * A.nr + rr] = acc;
  }
}

__global__ void k_deftab(const ProbDev* __restrict__ probs, const DefTab* __restrict__ tabs) {
  const DefTab D = tabs[blockIdx.y];
  const ProbDev& P = probs[D.prob];
  const int per = P.ax[D.axis].per;
  const int cnt = P.R * D.N;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < cnt; it += gridDim.x * blockDim.x) {
    int q = it / D.N, i = it % D.N;
    double rho = (double)(i - D.pad);
    if (D.mode == 1) {
      // every cell's copy of the nucleus once (no window, no replication),
      // cells beyond the Gaussian's reach skipped, minus the replicated term
      const int n0 = P.n0;
      const double reach = 7.0 / P.tq[q] + 2.0 * P.h;
      const int klo = max(0, (int)floor(((rho + 0.5) * P.h - reach) / (n0 * P.h) - D.pos / n0) - 1);
      const int khi = min(D.L - 1, (int)ceil(((rho + 0.5) * P.h + reach) / (n0 * P.h) - D.pos / n0) + 1);
      double acc = 0.0;
      for (int k = klo; k <= khi; ++k) {
        const double dc = (rho + 0.5 - D.pos - (double)k * n0) * P.h;
        acc += gauss_cell(P.tq[q], dc - 0.5 * P.h, dc + 0.5 * P.h);
      }
      const int ir = i - D.pad;
      const int r = (ir < 0) ? ir : (ir >= D.L * n0 ? ir - (D.L - 1) * n0 : ir % n0);
      D.e[it] = acc - D.prep[(size_t)(D.nu * P.R + q) * D.nr + (r - D.rlo)];
      continue;
    }
    double dc = (rho + 0.5 - D.pos) * P.h;      // node centre - nucleus
    if (per) {
      double period = (double)D.N * P.h;
      dc = dc - period * floor(dc / period + 0.5);
    }
    D.e[it] = gauss_cell(P.tq[q], dc - 0.5 * P.h, dc + 0.5 * P.h);
  }
}

// ---------------------------------------------------------------- K2 ----
__device__ inline double gval(const AxisDev& A, int mode, int n0, int mu, int cell, int rho) {
  if (mode == RING) {
    int j = posmod(rho - cell * n0, A.N);
    return A.g[mu * A.W + j];
  }
  if (mode == WALL && (rho < -A.pad || rho >= A.N - A.pad)) return 0.0;
  int j = rho - cell * n0 - A.jlo;
  if (j < 0 || j >= A.W) return 0.0;
  return A.g[mu * A.W + j];
}

// One CTA per task: folded pair products Z[r][mu nu] and the S1 / A1 forms.
__global__ void k_gram_fold(const ProbDev* __restrict__ probs, const GramTask* __restrict__ tasks) {
  const GramTask T = tasks[blockIdx.x];
  const ProbDev& P = probs[T.prob];
  const AxisDev& A = P.ax[T.axis];
  const int m0 = P.m0, n0 = P.n0, np = m0 * m0;
  const bool direct = (T.ptab >= 0);      // defect tables: no replication
  const int tot = T.nfold * np;
  for (int it = threadIdx.x; it < tot; it += blockDim.x) {
    int rr = it / np, pr = it % np, mu = pr / m0, nu = pr % m0;
    int r = T.foldlo + rr;
    double acc = 0.0;
    if (direct) {
      if (r >= T.rho0 && r < T.rho1)
        acc = gval(A, T.mode, n0, mu, T.a, r) * gval(A, T.mode, n0, nu, T.b, r);
    } else if (T.mode == RING) {
      // only the cells c whose node r + c n0 meets the support of g_mu(cell a):
      // c n0 in [a n0 + smin - r, a n0 + smin - r + slen) modulo the ring
      const int lo = T.a * n0 + A.smin - r;
      const int c0 = floordiv(lo + n0 - 1, n0), c1 = floordiv(lo + A.slen - 1, n0);
      if (A.slen >= A.N || c1 - c0 + 1 >= A.L) {
        for (int c = 0; c < A.L; ++c) {
          int rho = r + c * n0;
          acc += gval(A, RING, n0, mu, T.a, rho) * gval(A, RING, n0, nu, T.b, rho);
        }
      } else {
        for (int c = c0; c <= c1; ++c) {
          int rho = r + posmod(c, A.L) * n0;
          acc += gval(A, RING, n0, mu, T.a, rho) * gval(A, RING, n0, nu, T.b, rho);
        }
      }
    } else if (T.mode == VIRT || (r >= 0 && r < n0)) {
      // all nodes rho = r (mod n0) in the window (WALL: interior cells 0..L-1)
      int c0 = floordiv(T.rho0 - r + n0 - 1, n0), c1 = floordiv(T.rho1 - 1 - r, n0);
      if (T.mode == WALL) { c0 = max(c0, 0); c1 = min(c1, A.L - 1); }
      for (int c = c0; c <= c1; ++c) {
        int rho = r + c * n0;
        acc += gval(A, T.mode, n0, mu, T.a, rho) * gval(A, T.mode, n0, nu, T.b, rho);
      }
    } else {
      // WALL padding node: replicated from the end cell (clamped cell index)
      int rho = (r < 0) ? r : r + (A.L - 1) * n0;
      if (rho >= T.rho0 && rho < T.rho1)
        acc = gval(A, WALL, n0, mu, T.a, rho) * gval(A, WALL, n0, nu, T.b, rho);
    }
    T.Zs[it] = acc;
  }
  if (direct) return;   // defect forms carry no mass / stiffness part
  // RING: only the nodes of the support of g_mu(cell a) (the others add zeros)
  const bool ring_sup = (T.mode == RING && A.slen < A.N);
  const int nrho = ring_sup ? A.slen : T.rho1 - T.rho0;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    int mu = pr / m0, nu = pr % m0;
    double s = 0.0, a = 0.0;
    for (int t = 0; t < nrho; ++t) {
      const int rho = ring_sup ? posmod(T.a * n0 + A.smin + t, A.N) : T.rho0 + t;
      double ga = gval(A, T.mode, n0, mu, T.a, rho);
      if (ga == 0.0) continue;
      double b0 = gval(A, T.mode, n0, nu, T.b, rho);
      double bm = gval(A, T.mode, n0, nu, T.b, rho - 1);
      double bp = gval(A, T.mode, n0, nu, T.b, rho + 1);
      s += ga * (4.0 * b0 + bm + bp);
      a += ga * (2.0 * b0 - bm - bp);
    }
    T.X[0 * np + pr] = s * (P.h / 6.0);
    T.X[1 * np + pr] = a / P.h;
  }
}

// One CTA per task: X_t[mu nu] = sum_r P_t[r] Z[r][mu nu].
__global__ void k_gram_pot(const ProbDev* __restrict__ probs, const GramTask* __restrict__ tasks,
                           const DefTab* __restrict__ dtabs) {
  const GramTask T = tasks[blockIdx.x];
  if (T.split) return;   // mixed form: contracted by k_split_gemm
  const ProbDev& P = probs[T.prob];
  const AxisDev& A = P.ax[T.axis];
  const int np = P.m0 * P.m0;
  const bool direct = (T.ptab >= 0);
  const int nt = direct ? P.R : P.T;
  const double* tab = direct ? dtabs[T.ptab].e : A.p;
  const int ld = direct ? dtabs[T.ptab].N : A.nr;
  const int off = direct ? (T.foldlo + dtabs[T.ptab].pad) : (T.foldlo - A.rlo);
  double* out = T.X + (direct ? 0 : 2 * np);
  for (int it = threadIdx.x; it < nt * np; it += blockDim.x) {
    int t = it / np, pr = it % np;
    const double* pt = tab + (size_t)t * ld + off;
    double acc = 0.0;
    for (int rr = 0; rr < T.nfold; ++rr) acc += pt[rr] * T.Zs[(size_t)rr * np + pr];
    out[(size_t)t * np + pr] = acc;
  }
}

// ---------------------------------------------------------------- K3 ----
// H/S block from three per-axis factor sets (Lemma 3.4):
//   H = 1/2 (A0 S1 S2 + S0 A1 S2 + S0 S1 A2) - sum_t w_t M0_t M1_t M2_t,  S = S0 S1 S2
// (products elementwise in mu nu), w_t = Z_nu c_q for t = nu*R + q.  Optional
// subtraction of a Toeplitz generator (boundary blocks E = block - T_{k-m}),
// optional defect term (-dZ c_q Y0_q Y1_q Y2_q).


__global__ void k_combine(const ProbDev* __restrict__ probs, const CombineTask* __restrict__ tasks) {
  const CombineTask C = tasks[blockIdx.x];
  const ProbDev& P = probs[C.prob];
  const int m0 = P.m0, np = m0 * m0;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    double h = 0.0, s = 0.0, v = 0.0;
    if (C.X0) {   // lattice part (absent for a defect-only block)
      double s0 = C.X0[pr], s1 = C.X1[pr], s2 = C.X2[pr];
      double a0 = C.X0[np + pr], a1 = C.X1[np + pr], a2 = C.X2[np + pr];
      h = 0.5 * (a0 * s1 * s2 + s0 * a1 * s2 + s0 * s1 * a2);
      for (int t = 0; t < P.T; ++t) {
        double w = P.Z[t / P.R] * P.cq[t % P.R];
        v += w * C.X0[(2 + t) * np + pr] * C.X1[(2 + t) * np + pr] * C.X2[(2 + t) * np + pr];
      }
      s = s0 * s1 * s2;
    }
    if (C.D0) {
      double dv = 0.0;
      for (int q = 0; q < P.R; ++q)
        dv += P.cq[q] * C.D0[q * np + pr] * C.D1[q * np + pr] * C.D2[q * np + pr];
      v += C.dZ * dv;
    }
    h -= v;
    if (C.subH) {
      int ps = C.subT ? ((pr % m0) * m0 + pr / m0) : pr;
      h -= C.subH[ps];
      s -= C.subS[ps];
    }
    if (C.outH) C.outH[pr] = h;
    if (C.outS) C.outS[pr] = s;
    if (C.outHT) {
      const int tr = (pr % m0) * m0 + pr / m0;
      C.outHT[tr] = h;
      C.outST[tr] = s;
    }
  }
}

// ------------------------------------------------------------ defects ----
// Field of the chain's defects on the axis-0 nodes (reading R-DEF).
__global__ void k_defect_field(const ProbDev* __restrict__ probs, const DefField* __restrict__ tasks) {
  const DefField T = tasks[blockIdx.y];
  const ProbDev& P = probs[T.prob];
  const int np = P.m0 * P.m0, R = P.R;
  const int tot = T.N * np;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    const int rho = it / np, pr = it % np;
    double acc = 0.0;
    for (int d = 0; d < T.ndef; ++d) {
      const DefRef& Rf = T.refs[d];
      double s = 0.0;
      for (int q = 0; q < R; ++q)
        s += P.cq[q] * Rf.D1[q * np + pr] * Rf.D2[q * np + pr] * Rf.e[(size_t)q * T.N + rho];
      acc += Rf.dz * s;
    }
    T.F[it] = acc;
  }
}

// One CTA per defect block.
__global__ void k_defect_blocks(const ProbDev* __restrict__ probs, const DefBlock* __restrict__ tasks) {
  const DefBlock T = tasks[blockIdx.x];
  const ProbDev& P = probs[T.prob];
  const AxisDev& A = P.ax[0];
  const int m0 = P.m0, np = m0 * m0, n0 = P.n0;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    const int mu = pr / m0, nu = pr % m0;
    double acc = 0.0;
    for (int rho = T.rho0; rho < T.rho1; ++rho) {
      double ga = gval(A, T.mode, n0, mu, T.a, rho);
      if (ga == 0.0) continue;
      double gb = gval(A, T.mode, n0, nu, T.b, rho);
      int row = (T.mode == RING) ? posmod(rho, A.N) : rho + T.pad;
      acc += ga * gb * T.F[(size_t)row * np + pr];
    }
    T.outH[pr] = -acc;
    T.outS[pr] = 0.0;
  }
}

void launch_defects(const ProbDev* probs, const DefField* fields, int nf, const DefBlock* blocks, int nb,
                    cudaStream_t st) {
  if (nf) k_defect_field<<<dim3(64, nf), 256, 0, st>>>(probs, fields);
  if (nb) k_defect_blocks<<<nb, 128, 0, st>>>(probs, blocks);
}

// ---------------------------------------------------------------- K4 ----


__global__ void k_axis_dft(const ProbDev* __restrict__ probs, const DftTask* __restrict__ tasks) {
  extern __shared__ cplx tw[];   // exp(-2 pi i t / L), t < L
  const DftTask D = tasks[blockIdx.y];
  const ProbDev& P = probs[D.prob];
  for (int t = threadIdx.x; t < D.L; t += blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)D.L, &s, &c);
    tw[t] = cmk(c, s);
  }
  __syncthreads();
  // the factors are real: Xh[L - j] = conj(Xh[j]), so only j <= L / 2 is summed
  const int per = P.nF * P.m0 * P.m0;
  const int tot = (D.L / 2 + 1) * per;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < tot; it += gridDim.x * blockDim.x) {
    int j = it / per, e = it % per;
    double re = 0.0, im = 0.0;
    for (int o = 0; o < D.noff; ++o) {
      cplx w = tw[(int)(((long long)j * D.offs[o]) % D.L)];
      double x = D.X[(size_t)o * per + e];
      re += w.x * x;
      im += w.y * x;
    }
    D.Xh[it] = cmk(re, im);
    if (j > 0 && 2 * j != D.L) D.Xh[(size_t)(D.L - j) * per + e] = cmk(re, -im);
  }
}

// ------------------------------------------------------------ launchers ----
// maxT, maxni: the largest term count and endpoint count of the segments
void launch_vec1d(const ProbDev* probs, const SegDesc* gsegs, int ngseg, const SegDesc* psegs,
                  int npseg, const DefTab* dtabs, int ndtab, int maxT, int maxni, cudaStream_t st) {
  if (ngseg) k_gref<<<dim3(8, ngseg), 256, 0, st>>>(probs, gsegs);
  if (npseg) {
    const size_t sm = (size_t)maxni * sizeof(double);
    if (sm <= 160 * 1024) {
      FOCK_SMEM_OPTIN(k_ptab_nodes);
      k_ptab_nodes<<<dim3(maxT, npseg), 256, sm, st>>>(probs, psegs);
    } else {
      k_ptab<<<dim3(16, npseg), 256, 0, st>>>(probs, psegs);
    }
  }
  if (ndtab) k_deftab<<<dim3(8, ndtab), 256, 0, st>>>(probs, dtabs);
}

void launch_gram(const ProbDev* probs, const GramTask* tasks, int ntask, const DefTab* dtabs,
                 cudaStream_t st) {
  if (!ntask) return;
  k_gram_fold<<<ntask, 256, 0, st>>>(probs, tasks);
  k_gram_pot<<<ntask, 256, 0, st>>>(probs, tasks, dtabs);
}

void launch_combine(const ProbDev* probs, const CombineTask* tasks, int n, cudaStream_t st) {
  if (n) k_combine<<<n, 256, 0, st>>>(probs, tasks);
}

void launch_axis_dft(const ProbDev* probs, const DftTask* tasks, int n, int maxL, cudaStream_t st) {
  if (!n) return;
  size_t sm = (size_t)maxL * sizeof(cplx);
  FOCK_SMEM_OPTIN(k_axis_dft);
  k_axis_dft<<<dim3(32, n), 256, sm, st>>>(probs, tasks);
}

}  // namespace fock
