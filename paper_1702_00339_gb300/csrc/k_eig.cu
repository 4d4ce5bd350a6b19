// Stage (b) and the Fourier side of stage (c).
//
//  k_fblocks   one CTA per Fourier index j: forms the m0 x m0 Hermitian pair
//              (Hbar_j, Sbar_j) and, on request, stores it and/or solves the
//              generalized eigenproblem Hbar u = l Sbar u in FP64.
//     source FACTORS (periodic lattice, Thm. 3.3 with the CP rank of the
//       potential, Remark 3.5): Hbar_j = 1/2 sum_p (prod_{l!=p} Shat_l) Ahat_p
//       - sum_t w_t prod_l Mhat_{l,t}, Sbar_j = prod_l Shat_l, elementwise in
//       (mu, nu), each factor picked at the axis component j_l;
//     source TOEPLITZ (box chain, Remark 3.2): the size-M block circulant
//       that embeds the symmetric block Toeplitz matrix with generators
//       T_d = block (k+d, k), |d| <= D: Chat_j = T_0 + sum_d (w^{jd} T_d +
//       w^{-jd} T_d^T), w = exp(-2 pi i / M) (Eq. A.3 convention).
//     eigensolver: Cholesky Sbar = L L^H and C = L^-1 Hbar L^-H when the
//       factor certifies that Sbar has no eigenvalue at or below tau (the
//       dependency cut; lambda_min >= 1 / ||L^-1||_F^2 > tau), else the
//       Jacobi eigendecomposition Sbar = Q diag(s) Q^H,
//       X = Q_K diag(s_K)^-1/2 over the kept directions K = {s > tau} (tau the
//       problem's dependency cut: every direction when none is numerically
//       singular, so C = X^H Hbar X has the pencil's eigenvalues exactly) --
//       then Householder reduction of C to a real tridiagonal and
//       Sturm-sequence bisection per eigenvalue, FP32 first then FP64 with
//       division-free counts (ascending, so the block spectrum comes out
//       sorted); the removed directions report +inf.  The lowest eigenvalue
//       of an embedding block (preconditioner shift only) stops at 1e-9
//       relative.  One warp per block for m0 <= 8.
//  k_sigma      shift of the preconditioner: min_j lambda_min(Chat_j) - delta.
//  k_precond    K_j = (Chat_H,j - sigma Chat_S,j)^-1 per Fourier index.
//  k_sort_*     ascending sort of (eigenvalue, Fourier index) pairs.
#include <float.h>
#include <algorithm>

#include "common.cuh"

namespace fock {

enum FSource { FROM_FACTORS = 0, FROM_TOEPLITZ = 1 };

// ---- dense Hermitian helpers (shared memory, whole CTA) ----

// In-place lower Cholesky of a Hermitian positive definite m x m (row-major).
__device__ bool cta_cholesky(cplx* a, int m) {
  __shared__ int bad;
  __shared__ double s_inv;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      double d = a[k * m + k].x;
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      const double r = rsqrt_nr(d);       // 1 / sqrt(d) (Newton-Raphson from an FP32 seed)
      a[k * m + k] = cmk(d * r, 0.0);
      s_inv = r;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) a[i * m + k] = cscale(a[i * m + k], inv);
    __syncthreads();
    int nt = m - k - 1;
    for (int it = threadIdx.x; it < nt * nt; it += blockDim.x) {
      int i = k + 1 + it / nt, j = k + 1 + it % nt;
      if (j <= i) a[i * m + j] = csub(a[i * m + j], cmulc(a[i * m + k], a[j * m + k]));
    }
    __syncthreads();
  }
  return bad == 0;
}

// Cyclic Jacobi eigendecomposition of a Hermitian n x n matrix a (row-major,
// stride ld >= n + (n & 1)), whole CTA.  Each step rotates n/2 disjoint
// index pairs (round-robin ordering, an odd n gets a zero pad index).  For a
// pair (p, q) with a_pq = r e^{i phi} the unitary U = diag(1, e^{-i phi}) J,
// J the real rotation that annihilates the real pair (a_pp, r, a_qq), gives
// a <- U^H a U and v <- v U.  On return the diagonal of a holds the
// eigenvalues (real parts) and the columns of v the eigenvectors.  A pair is
// skipped once |a_pq| <= 1e-15 ||a||_F; at most 30 sweeps.
__device__ void cta_jacobi_herm(cplx* a, cplx* v, int n, int ld) {
  __shared__ double rc[MAXM0 / 2 + 1], rs[MAXM0 / 2 + 1];
  __shared__ cplx rph[MAXM0 / 2 + 1];
  __shared__ int rp[MAXM0 / 2 + 1], rq[MAXM0 / 2 + 1];
  __shared__ int nrot;
  __shared__ double red[32], s_thr2;
  const int ne = n + (n & 1);
  double part = 0.0;
  for (int it = threadIdx.x; it < n * n; it += blockDim.x) part += cabs2(a[(it / n) * ld + (it % n)]);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    s_thr2 = 1e-30 * t;   // (1e-15 ||a||_F)^2
  }
  for (int it = threadIdx.x; it < ne * ne; it += blockDim.x) {
    int i = it / ne, j = it % ne;
    v[i * ld + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
    if (i == n || j == n) a[i * ld + j] = cmk(0.0, 0.0);
  }
  __syncthreads();
  const double thr2 = s_thr2;
  const int np2 = ne / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    if (threadIdx.x == 0) nrot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < ne - 1; ++rnd) {
      for (int pi = threadIdx.x; pi < np2; pi += blockDim.x) {
        int x = (pi == 0) ? 0 : ((pi - 1 + rnd) % (ne - 1)) + 1;
        int y = ((ne - 2 - pi + rnd) % (ne - 1)) + 1;
        int p = min(x, y), q = max(x, y);
        cplx apq = a[p * ld + q];
        const double r2 = cabs2(apq), app = a[p * ld + p].x, aqq = a[q * ld + q].x;
        double c = 1.0, s = 0.0;
        cplx ph = cmk(1.0, 0.0);
        if (r2 > thr2 && r2 > 1e-34 * fabs(app * aqq)) {   // |a_pq| > thr and > 1e-17 sqrt|a_pp a_qq|
          // reciprocals and square roots by Newton-Raphson from FP32 seeds
          const double rr = rsqrt_nr(r2);                    // 1 / |a_pq|
          ph = cscale(apq, rr);
          const double th = (aqq - app) * (0.5 * rr);
          const double y = fma(th, th, 1.0);
          double t = rcp_nr(fabs(th) + y * rsqrt_nr(y));     // 1 / (|th| + sqrt(th^2 + 1))
          if (th < 0.0) t = -t;
          c = rsqrt_nr(fma(t, t, 1.0));
          s = t * c;
          atomicAdd(&nrot, 1);
        }
        rp[pi] = p; rq[pi] = q; rc[pi] = c; rs[pi] = s; rph[pi] = ph;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < np2 * ne; it += blockDim.x) {   // rows: U^H a
        int pi = it / ne, jj = it % ne;
        double s = rs[pi];
        if (s == 0.0) continue;
        int p = rp[pi], q = rq[pi];
        double c = rc[pi];
        cplx ap = a[p * ld + jj], aq = cmul(rph[pi], a[q * ld + jj]);
        a[p * ld + jj] = csub(cscale(ap, c), cscale(aq, s));
        a[q * ld + jj] = cadd(cscale(ap, s), cscale(aq, c));
      }
      __syncthreads();
      for (int it = threadIdx.x; it < np2 * ne; it += blockDim.x) {   // columns: a U, v U
        int pi = it / ne, ii = it % ne;
        double s = rs[pi];
        if (s == 0.0) continue;
        int p = rp[pi], q = rq[pi];
        double c = rc[pi];
        cplx phc = cconj(rph[pi]);
        cplx ap = a[ii * ld + p], aq = cmul(phc, a[ii * ld + q]);
        a[ii * ld + p] = csub(cscale(ap, c), cscale(aq, s));
        a[ii * ld + q] = cadd(cscale(ap, s), cscale(aq, c));
        cplx vp = v[ii * ld + p], vq = cmul(phc, v[ii * ld + q]);
        v[ii * ld + p] = csub(cscale(vp, c), cscale(vq, s));
        v[ii * ld + q] = cadd(cscale(vp, s), cscale(vq, c));
      }
      __syncthreads();
    }
    int done = (nrot == 0);
    __syncthreads();
    if (done) break;
  }
}

// Eigendecomposition a = Q diag(w) Q^H of a Hermitian n x n matrix (row-major,
// stride ld, n <= MAXM0), whole CTA (blockDim a multiple of 32), in about a
// quarter of the FP64 instructions of the cyclic Jacobi method above:
//  1. Householder reduction to tridiagonal form.  Step k maps x = a[k+1:, k]
//     to (alpha, 0, ..., 0) with the reflector H_k = I - beta u u^H,
//     u = (1, v_1, ...), alpha = -e^{i theta} ||x||, e^{i theta} = x_1 / |x_1|,
//     beta = 1 + |x_1| / ||x||, v_i = x_i / (x_1 - alpha); the trailing block
//     becomes H_k A H_k through p = beta A u, w = p - (beta / 2)(u^H p) u,
//     A <- A - u w^H - w u^H.  The v_i stay below the subdiagonal of column k.
//  2. The Hermitian tridiagonal T (real diagonal d, complex subdiagonal
//     alpha_k) equals D T' D^H with T' real symmetric (subdiagonal |alpha_k|)
//     and D = diag(phi), phi_0 = 1, phi_{k+1} = phi_k alpha_k / |alpha_k|.
//  3. T' = Z diag(w) Z^T by the implicit QL iteration with Wilkinson's shift
//     (Bowdler, Martin, Reinsch and Wilkinson, Numer. Math. 11 (1968)), its
//     plane rotations accumulated into Z (the real parts of v); warp 0, each
//     lane carrying its own copy of the tridiagonal and one row of Z.  An
//     off-diagonal is negligible at eps ||T'||_inf (absolute accuracy, the
//     reduction's own backward error).
//  4. Q = H_0 ... H_{n-3} D Z, applied to v in place.
// On return the diagonal of a holds the eigenvalues (real parts, unordered)
// and the columns of v the orthonormal eigenvectors.  Returns false, a and v
// then undefined, if some eigenvalue took more than 60 QL iterations.
__device__ bool cta_herm_eig(cplx* a, cplx* v, int n, int ld) {
  __shared__ double hb[MAXM0], hd[MAXM0], he[MAXM0];
  __shared__ cplx hphi[MAXM0], hpw[MAXM0];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // ---- 1. tridiagonal reduction ----
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    if (warp == 0) {
      const cplx xi = (lane < m) ? a[(k + 1 + lane) * ld + k] : cmk(0.0, 0.0);
      double tail = (lane >= 1) ? cabs2(xi) : 0.0;
      for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
      const cplx x1 = cmk(__shfl_sync(0xffffffffu, xi.x, 0), __shfl_sync(0xffffffffu, xi.y, 0));
      double beta = 0.0;
      if (tail > 0.0) {
        const double ax1 = sqrt(cabs2(x1));
        const double sig = sqrt(fma(ax1, ax1, tail));
        const cplx ph = (ax1 > 0.0) ? cscale(x1, 1.0 / ax1) : cmk(1.0, 0.0);
        beta = 1.0 + ax1 / sig;
        const cplx inv_u1 = cscale(cconj(ph), 1.0 / (ax1 + sig));   // 1 / (x_1 - alpha)
        if (lane >= 1 && lane < m) a[(k + 1 + lane) * ld + k] = cmul(xi, inv_u1);
        if (lane == 0) a[(k + 1) * ld + k] = cscale(ph, -sig);        // alpha
      }
      if (lane == 0) hb[k] = beta;
    }
    __syncthreads();
    const double beta = hb[k];
    if (beta == 0.0) continue;                 // uniform: already reduced
    // p = beta A u over the trailing block (4 threads per row)
    const int tot = m * 4, totr = (tot + 31) & ~31;
    for (int it = threadIdx.x; it < totr; it += blockDim.x) {
      const int r = it >> 2, part = it & 3;
      cplx acc = cmk(0.0, 0.0);
      if (it < tot) {
        const cplx* row = a + (size_t)(k + 1 + r) * ld + (k + 1);
        for (int c = part; c < m; c += 4) {
          const cplx uc = (c == 0) ? cmk(1.0, 0.0) : a[(k + 1 + c) * ld + k];
          acc = cfma(row[c], uc, acc);
        }
      }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (it < tot && part == 0) hpw[r] = cscale(acc, beta);
    }
    __syncthreads();
    // w = p - (beta / 2)(u^H p) u   (u^H p real up to rounding)
    if (warp == 0) {
      const cplx ui = (lane == 0) ? cmk(1.0, 0.0) : ((lane < m) ? a[(k + 1 + lane) * ld + k] : cmk(0.0, 0.0));
      const cplx pi = (lane < m) ? hpw[lane] : cmk(0.0, 0.0);
      double up = ui.x * pi.x + ui.y * pi.y;   // Re(conj(u_i) p_i)
      for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(0xffffffffu, up, o);
      const double K = 0.5 * beta * up;
      __syncwarp();
      if (lane < m) hpw[lane] = csub(pi, cscale(ui, K));
    }
    __syncthreads();
    // A <- A - u w^H - w u^H on the trailing block
    for (int it = threadIdx.x; it < m * m; it += blockDim.x) {
      const int i = it / m, j = it % m;
      const cplx ui = (i == 0) ? cmk(1.0, 0.0) : a[(k + 1 + i) * ld + k];
      const cplx uj = (j == 0) ? cmk(1.0, 0.0) : a[(k + 1 + j) * ld + k];
      cplx* aij = a + (size_t)(k + 1 + i) * ld + (k + 1 + j);
      *aij = crank2(*aij, ui, hpw[j], hpw[i], uj);
    }
    __syncthreads();
  }
  // ---- 2. real tridiagonal T' and the phases D ----
  if (threadIdx.x == 0) {
    cplx phi = cmk(1.0, 0.0);
    for (int k = 0; k < n; ++k) {
      hd[k] = a[k * ld + k].x;
      hphi[k] = phi;
      if (k + 1 < n) {
        const cplx al = a[(k + 1) * ld + k];
        const double aa = sqrt(cabs2(al));
        he[k] = aa;
        if (aa > 0.0) phi = cmul(phi, cscale(al, 1.0 / aa));
      } else {
        he[k] = 0.0;
      }
    }
    s_ok = 1;
  }
  for (int it = threadIdx.x; it < n * n; it += blockDim.x) {   // Z = I
    const int i = it / n, j = it % n;
    v[i * ld + j] = cmk(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // ---- 3. implicit QL on warp 0 ----
  if (warp == 0) {
    double d[MAXM0], e[MAXM0];
    double tn = 0.0;
    for (int i = 0; i < n; ++i) {
      d[i] = hd[i];
      e[i] = he[i];
      tn = fmax(tn, fabs(d[i]) + e[i] + (i > 0 ? e[i - 1] : 0.0));
    }
    const double small = 2.220446049250313e-16 * tn;   // eps ||T'||_inf
    bool ok = true;
    for (int l = 0; l < n && ok; ++l) {
      for (int iter = 0;; ++iter) {
        int m = l;
        while (m + 1 < n && fabs(e[m]) > small) ++m;
        if (m == l) break;                               // d[l] is an eigenvalue
        if (iter == 60) { ok = false; break; }
        // shift: the eigenvalue of the leading 2 x 2 of block l..m nearer d[l]
        double g = (d[l + 1] - d[l]) * rcp_nr(2.0 * e[l]);
        const double q1 = fma(g, g, 1.0);
        const double r1 = q1 * rsqrt_nr(q1);
        g = d[m] - d[l] + e[l] * rcp_nr(g + copysign(r1, g));
        double s = 1.0, c = 1.0, p = 0.0;
        bool split = false;
        for (int i = m - 1; i >= l; --i) {
          const double f = s * e[i], b = c * e[i];
          const double q2 = fma(f, f, g * g);
          if (q2 == 0.0) {                               // the chase stopped: restart
            d[i + 1] -= p;
            e[m] = 0.0;
            split = true;
            break;
          }
          const double ir = rsqrt_nr(q2);
          e[i + 1] = q2 * ir;
          s = f * ir;
          c = g * ir;
          g = d[i + 1] - p;
          const double r = fma(d[i] - g, s, 2.0 * c * b);
          p = s * r;
          d[i + 1] = g + p;
          g = fma(c, r, -b);
          if (lane < n) {                                // rotate columns i, i + 1 of Z
            const double zi = v[lane * ld + i].x, zj = v[lane * ld + i + 1].x;
            v[lane * ld + i + 1].x = fma(s, zi, c * zj);
            v[lane * ld + i].x = fma(c, zi, -s * zj);
          }
        }
        if (split) continue;
        d[l] -= p;
        e[l] = g;
        e[m] = 0.0;
      }
    }
    if (!ok && lane == 0) s_ok = 0;
    if (lane < n) hd[lane] = d[lane];
  }
  __syncthreads();
  if (!s_ok) return false;
  // ---- 4. Q = H_0 ... H_{n-3} D Z ----
  for (int it = threadIdx.x; it < n * n; it += blockDim.x) {
    const int i = it / n, j = it % n;
    v[i * ld + j] = cscale(hphi[i], v[i * ld + j].x);
  }
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const double beta = hb[k];
    if (beta == 0.0) continue;
    const int m = n - k - 1;
    // t_j = u^H V[k+1:, j]  (4 threads per column)
    const int tot = n * 4, totr = (tot + 31) & ~31;
    for (int it = threadIdx.x; it < totr; it += blockDim.x) {
      const int j = it >> 2, part = it & 3;
      cplx acc = cmk(0.0, 0.0);
      if (it < tot)
        for (int i = part; i < m; i += 4) {
          const cplx ui = (i == 0) ? cmk(1.0, 0.0) : a[(k + 1 + i) * ld + k];
          acc = cfmac(v[(k + 1 + i) * ld + j], ui, acc);         // conj(u_i) V_ij
        }
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (it < tot && part == 0) hpw[j] = cscale(acc, beta);
    }
    __syncthreads();
    for (int it = threadIdx.x; it < m * n; it += blockDim.x) {
      const int i = it / n, j = it % n;
      const cplx ui = (i == 0) ? cmk(1.0, 0.0) : a[(k + 1 + i) * ld + k];
      v[(k + 1 + i) * ld + j] = cfma(cmk(-ui.x, -ui.y), hpw[j], v[(k + 1 + i) * ld + j]);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i * ld + i] = cmk(hd[i], 0.0);
  __syncthreads();
  return true;
}

// Reduction of a Hermitian pencil block (h, s), both m x m with stride m, to
// a standard Hermitian matrix: eigendecomposition s = Q diag(w) Q^H
// (cta_herm_eig; in a, q: scratch of ld x ld, ld = m + (m & 1)), kept set
// K = {w_i > tau} (tau absolute: the dependency cut) in ascending index,
// X = Q_K diag(w_K)^-1/2, and h <- X^H h X (r x r, stride r, exactly
// Hermitian).  With every direction kept, X^H s X = I and the eigenvalues of
// h are the pencil's.  Returns r = |K|.  sv and keep are shared arrays of
// MAXM0 entries.
// a may be s itself (even m: the same layout); the copy is then skipped and,
// should QL run out of iterations, -1 is returned (s is overwritten) so that the
// caller forms s again and calls back with jacobi = true.
__device__ int cta_lowdin_reduce(cplx* h, const cplx* s, cplx* a, cplx* q, int m, double tau,
                                 double* sv, int* keep, bool jacobi) {
  __shared__ int s_r;
  const int ld = m + (m & 1);
  const bool inplace = ((const void*)a == (const void*)s);
  if (!inplace) {
    for (int it = threadIdx.x; it < m * m; it += blockDim.x) a[(it / m) * ld + (it % m)] = s[it];
    __syncthreads();
  }
  if (jacobi || !cta_herm_eig(a, q, m, ld)) {   // QL out of iterations: the Jacobi method
    if (!jacobi && inplace) return -1;
    if (!inplace) {
      for (int it = threadIdx.x; it < m * m; it += blockDim.x) a[(it / m) * ld + (it % m)] = s[it];
      __syncthreads();
    }
    cta_jacobi_herm(a, q, m, ld);
  }
  if (threadIdx.x == 0) {
    int r = 0;
    for (int i = 0; i < m; ++i)
      if (a[i * ld + i].x > tau && a[i * ld + i].x > 0.0) { keep[r] = i; sv[r] = a[i * ld + i].x; ++r; }
    s_r = r;
  }
  __syncthreads();
  const int r = s_r;
  cplx* X = a;   // m x r
  for (int it = threadIdx.x; it < m * r; it += blockDim.x) {
    int mu = it / r, c = it % r;
    X[it] = cscale(q[mu * ld + keep[c]], 1.0 / sqrt(sv[c]));
  }
  __syncthreads();
  cplx* Y = q;   // m x r, Y = h X
  for (int it = threadIdx.x; it < m * r; it += blockDim.x) {
    int mu = it / r, c = it % r;
    cplx acc = cmk(0.0, 0.0);
    for (int nu = 0; nu < m; ++nu) acc = cfma(h[mu * m + nu], X[nu * r + c], acc);
    Y[it] = acc;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {   // h = X^H Y
    int ia = it / r, ib = it % r;
    cplx acc = cmk(0.0, 0.0);
    for (int mu = 0; mu < m; ++mu) acc = cfmac(Y[mu * r + ib], X[mu * r + ia], acc);
    h[it] = acc;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < r * r; it += blockDim.x) {
    int ia = it / r, ib = it % r;
    if (ia < ib) {
      cplx hm = cscale(cadd(h[it], cconj(h[ib * r + ia])), 0.5);
      h[it] = hm;
      h[ib * r + ia] = cconj(hm);
    } else if (ia == ib) {
      h[it].y = 0.0;
    }
  }
  __syncthreads();
  return r;
}

// Reduction of a Hermitian pencil block (h, s), m x m with stride m, by
// Cholesky: s = L L^H, h <- L^-1 h L^-H (exactly Hermitian), when the
// factorisation certifies that s has no eigenvalue at or below tau
// (lambda_min(s) = 1 / ||L^-1||_2^2 >= 1 / ||L^-1||_F^2 > tau): then no
// direction is numerically singular and the reduction is the pencil's own.
// Returns false with h unchanged otherwise (the caller takes the Jacobi
// route).  a, q: scratch of m x m.  About m^3 complex multiply-adds against
// ~100 m^3 for the Jacobi eigendecomposition.
__device__ bool cta_cholesky_reduce(cplx* h, const cplx* s, cplx* a, cplx* q, int m, double tau) {
  __shared__ double red[32];
  __shared__ int s_ok;
  for (int it = threadIdx.x; it < m * m; it += blockDim.x) a[it] = s[it];
  __syncthreads();
  if (!cta_cholesky(a, m)) return false;                 // uniform: a shared flag
  // q = L^-1 (lower triangular), one thread per column
  for (int c = threadIdx.x; c < m; c += blockDim.x)
    for (int i = 0; i < m; ++i) {
      if (i < c) { q[i * m + c] = cmk(0.0, 0.0); continue; }
      cplx t = cmk(i == c ? 1.0 : 0.0, 0.0);
      for (int k = c; k < i; ++k) t = csub(t, cmul(a[i * m + k], q[k * m + c]));
      q[i * m + c] = cscale(t, rcp_nr(a[i * m + i].x));
    }
  __syncthreads();
  double part = 0.0;
  for (int it = threadIdx.x; it < m * m; it += blockDim.x) part += cabs2(q[it]);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    s_ok = (t > 0.0 && t * tau < 1.0);                     // 1 / ||L^-1||_F^2 > tau
  }
  __syncthreads();
  if (!s_ok) return false;
  for (int it = threadIdx.x; it < m * m; it += blockDim.x) {   // a = L^-1 h
    const int i = it / m, j = it % m;
    cplx t = cmk(0.0, 0.0);
    for (int k = 0; k <= i; ++k) t = cfma(q[i * m + k], h[k * m + j], t);
    a[it] = t;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < m * m; it += blockDim.x) {   // h = a L^-H (lower triangle)
    const int i = it / m, j = it % m;
    if (j > i) continue;
    cplx t = cmk(0.0, 0.0);
    for (int k = 0; k <= j; ++k) t = cfmac(a[i * m + k], q[j * m + k], t);
    h[it] = t;
  }
  __syncthreads();
  for (int it = threadIdx.x; it < m * m; it += blockDim.x) {   // exactly Hermitian
    const int i = it / m, j = it % m;
    if (j > i) h[it] = cconj(h[j * m + i]);
    else if (j == i) h[it].y = 0.0;
  }
  __syncthreads();
  return true;
}

// Householder reduction of Hermitian c (full storage, destroyed) to a real
// symmetric tridiagonal (d, e) with e_k = |c'_{k+1,k}| (a diagonal unitary
// scaling removes the phases).
__device__ void cta_tridiag(cplx* c, int m, double* d, double* e, cplx* v, cplx* p) {
  __shared__ double red[32];
  __shared__ double s_tau, s_K, s_norm;
  for (int k = 0; k < m - 2; ++k) {
    // ||x||^2, x = c[k+1:, k]
    double part = 0.0;
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) part += cabs2(c[i * m + k]);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += red[w];
      // square roots and reciprocals by Newton-Raphson from FP32 seeds
      const double xn = (s > 0.0) ? s * rsqrt_nr(s) : 0.0;
      const cplx x0 = c[(k + 1) * m + k];
      const double a2 = cabs2(x0);
      const double ra = (a2 > 0.0) ? rsqrt_nr(a2) : 0.0;
      const double ax0 = a2 * ra;
      cplx ph = (a2 > 0.0) ? cscale(x0, ra) : cmk(1.0, 0.0);
      cplx alpha = cscale(ph, -xn);
      d[k] = c[k * m + k].x;
      e[k] = xn;
      double vn2 = 2.0 * (s + xn * ax0);
      s_tau = (vn2 > 0.0) ? 2.0 * rcp_nr(vn2) : 0.0;
      s_norm = xn;
      v[k + 1] = csub(x0, alpha);
    }
    __syncthreads();
    for (int i = k + 2 + threadIdx.x; i < m; i += blockDim.x) v[i] = c[i * m + k];
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) {
        cplx s = cmk(0.0, 0.0);
        for (int j = k + 1; j < m; ++j) s = cfma(c[i * m + j], v[j], s);
        p[i] = cscale(s, tau);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double K = 0.0;   // (tau/2) v^H p, real for Hermitian c
        for (int i = k + 1; i < m; ++i) K += v[i].x * p[i].x + v[i].y * p[i].y;
        s_K = 0.5 * tau * K;
      }
      __syncthreads();
      const double K = s_K;
      for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) p[i] = csub(p[i], cscale(v[i], K));
      __syncthreads();
      const int nt = m - k - 1;
      for (int it = threadIdx.x; it < nt * nt; it += blockDim.x) {
        int i = k + 1 + it / nt, j = k + 1 + it % nt;
        // c -= v w^H + w v^H   (w stored in p)
        c[i * m + j] = crank2(c[i * m + j], v[i], p[j], p[i], v[j]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (m >= 2) {
      d[m - 2] = c[(m - 2) * m + (m - 2)].x;
      d[m - 1] = c[(m - 1) * m + (m - 1)].x;
      e[m - 2] = sqrt(cabs2(c[(m - 1) * m + (m - 2)]));
    } else {
      d[0] = c[0].x;
    }
  }
  __syncthreads();
}

__device__ inline cplx twiddle(long long num, int M) {   // exp(-2 pi i num / M)
  double s, c;
  sincospi(-2.0 * (double)(num % M) / (double)M, &s, &c);
  return cmk(c, s);
}

// Sbar_j of a block formed again, with the arithmetic of the formation in
// k_fblocks (used where the block's eigendecomposition works in Sbar's own
// storage and a route that overwrote it fell through).  tw: ldj^2 entries of
// scratch for the Toeplitz twiddles.
__device__ void reform_S(const FBlockTask& F, const ProbDev& P, int j, int m0, cplx* S, cplx* tw, int ldj) {
  const int np = m0 * m0;
  if (F.source == FROM_FACTORS) {
    const int j3 = j % F.L[2], j2 = (j / F.L[2]) % F.L[1], j1 = j / (F.L[1] * F.L[2]);
    const int nfe = P.nF * np;
    const cplx* x0 = F.Xh[0] + (size_t)j1 * nfe;
    const cplx* x1 = F.Xh[1] + (size_t)j2 * nfe;
    const cplx* x2 = F.Xh[2] + (size_t)j3 * nfe;
    const int nup = m0 * (m0 + 1) / 2;
    for (int u = threadIdx.x; u < nup; u += blockDim.x) {
      int mu = 0, rem = u;
      while (rem >= m0 - mu) { rem -= m0 - mu; ++mu; }
      const int nu = mu + rem, pr = mu * m0 + nu, tr = nu * m0 + mu;
      cplx s = cmul(x0[pr], cmul(x1[pr], x2[pr]));
      if (mu == nu) s.y = 0.0;
      S[pr] = s;
      S[tr] = cconj(s);
    }
    __syncthreads();
  } else {
    const bool tab = (F.D <= ldj * ldj);
    if (tab) {
      for (int dd2 = 1 + threadIdx.x; dd2 <= F.D; dd2 += blockDim.x) tw[dd2 - 1] = twiddle((long long)j * dd2, F.M);
      __syncthreads();
    }
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      const int mu = pr / m0, nu = pr % m0, tr = nu * m0 + mu;
      cplx s = cmk(F.TS[pr], 0.0);
      for (int dd2 = 1; dd2 <= F.D; ++dd2) {
        const cplx w = tab ? tw[dd2 - 1] : twiddle((long long)j * dd2, F.M);
        const double* ts = F.TS + (size_t)dd2 * np;
        s = cadd(s, cmk(w.x * (ts[pr] + ts[tr]), w.y * (ts[pr] - ts[tr])));
      }
      S[pr] = s;
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      const int mu = pr / m0, nu = pr % m0;
      if (mu < nu) {
        const cplx sm2 = cscale(cadd(S[pr], cconj(S[nu * m0 + mu])), 0.5);
        S[pr] = sm2; S[nu * m0 + mu] = cconj(sm2);
      } else if (mu == nu) {
        S[pr].y = 0.0;
      }
    }
    __syncthreads();
  }
}

__global__ void k_fblocks(const ProbDev* __restrict__ probs, const FBlockTask* __restrict__ tasks, int x0) {
  extern __shared__ cplx sm[];
  const FBlockTask F = tasks[blockIdx.y];
  const int jl = x0 + blockIdx.x; // local output index (a launch may cover a range of them)
  if (jl >= F.nj) return;
  const int j = F.j0 + jl;        // Fourier index
  // Real generators: the block at -j (componentwise mod L) is the complex
  // conjugate of the block at j, with the same spectrum.  When both indices
  // are in this task's range and no blocks are stored, the lower index
  // solves the pair and writes both; the higher one does nothing.
  int jm = -1;
  if (F.source == FROM_FACTORS && F.want == 1 && !F.outH) {
    const int j3 = j % F.L[2], j2 = (j / F.L[2]) % F.L[1], j1 = j / (F.L[1] * F.L[2]);
    const int m1 = (F.L[0] - j1) % F.L[0], m2 = (F.L[1] - j2) % F.L[1], m3 = (F.L[2] - j3) % F.L[2];
    jm = (m1 * F.L[1] + m2) * F.L[2] + m3;
    if (jm == j || jm < F.j0 || jm >= F.j0 + F.nj) jm = -1;
    else if (jm < j) return;
  }
  const ProbDev& P = probs[F.prob];
  const int m0 = P.m0, np = m0 * m0;
  const int ldj = m0 + (m0 & 1);
  // even m0: the overlap's eigendecomposition works in Sbar's own storage (the
  // same m0 x m0 layout), so a block needs three m0^2 arrays and 32 x 32 blocks
  // fit four CTAs per SM; odd m0 keeps a padded work array of its own
  const bool alias = !(m0 & 1);
  cplx* H = sm;
  cplx* S = sm + np;
  cplx* Aj = alias ? S : S + np;                       // eigendecomposition work, ldj x ldj
  cplx* Qj = alias ? S + np : Aj + ldj * ldj;          // its eigenvectors, ldj x ldj
  cplx* v = Qj + ldj * ldj;
  cplx* pv = v + MAXM0;
  double* dd = (double*)(pv + MAXM0);
  double* ee = dd + MAXM0;
  double* e2 = ee + MAXM0;                 // e^2, and FP32 copies of d and e^2
  float* df = (float*)(e2 + MAXM0);
  float* e2f = df + MAXM0;
  // eigenvectors (F.vecs): a copy of the reduced matrix and its Jacobi eigenvectors
  cplx* Vc = (cplx*)(((uintptr_t)(e2f + MAXM0) + 15) & ~(uintptr_t)15);
  cplx* Wv = Vc + ldj * ldj;

  if (F.source == FROM_FACTORS) {
    const int j3 = j % F.L[2], j2 = (j / F.L[2]) % F.L[1], j1 = j / (F.L[1] * F.L[2]);
    const int nfe = P.nF * np;
    const cplx* x0 = F.Xh[0] + (size_t)j1 * nfe;
    const cplx* x1 = F.Xh[1] + (size_t)j2 * nfe;
    const cplx* x2 = F.Xh[2] + (size_t)j3 * nfe;
    // H and S are Hermitian (each axis factor is, and so is a Hadamard product
    // of Hermitian matrices): the upper triangle, enumerated compactly so that
    // whole warps share the work, is formed and mirrored; the diagonal is real
    const int nup = m0 * (m0 + 1) / 2;
    for (int u = threadIdx.x; u < nup; u += blockDim.x) {
      int mu = 0, rem = u;
      while (rem >= m0 - mu) { rem -= m0 - mu; ++mu; }
      const int nu = mu + rem, pr = mu * m0 + nu, tr = nu * m0 + mu;
      cplx s0 = x0[pr], s1 = x1[pr], s2 = x2[pr];
      cplx a0 = x0[np + pr], a1 = x1[np + pr], a2 = x2[np + pr];
      cplx s12 = cmul(s1, s2);
      cplx hk = cadd(cmul(a0, s12), cmul(s0, cadd(cmul(a1, s2), cmul(s1, a2))));
      hk = cscale(hk, 0.5);
      cplx vv = cmk(0.0, 0.0);
      for (int t = 0; t < P.T; ++t) {
        double w = P.Z[t / P.R] * P.cq[t % P.R];
        cplx pr3 = cmul(cmul(x0[(2 + t) * np + pr], x1[(2 + t) * np + pr]), x2[(2 + t) * np + pr]);
        vv.x = fma(pr3.x, w, vv.x);
        vv.y = fma(pr3.y, w, vv.y);
      }
      cplx h = csub(hk, vv), s = cmul(s0, s12);
      if (mu == nu) { h.y = 0.0; s.y = 0.0; }
      H[pr] = h; S[pr] = s;
      H[tr] = cconj(h); S[tr] = cconj(s);
    }
  } else {
    // twiddles exp(-2 pi i j d / M), d = 1..D, once per block (in the
    // eigenvector scratch, free until the reduction) when they fit
    cplx* tw = Qj;
    const bool tab = (F.D <= ldj * ldj);
    if (tab) {
      for (int dd2 = 1 + threadIdx.x; dd2 <= F.D; dd2 += blockDim.x) tw[dd2 - 1] = twiddle((long long)j * dd2, F.M);
      __syncthreads();
    }
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      int mu = pr / m0, nu = pr % m0, tr = nu * m0 + mu;
      cplx h = cmk(F.TH[pr], 0.0), s = cmk(F.TS[pr], 0.0);
      for (int dd2 = 1; dd2 <= F.D; ++dd2) {
        cplx w = tab ? tw[dd2 - 1] : twiddle((long long)j * dd2, F.M);
        const double* th = F.TH + (size_t)dd2 * np;
        const double* ts = F.TS + (size_t)dd2 * np;
        // w T_d[mu][nu] + conj(w) T_d[nu][mu]
        h = cadd(h, cmk(w.x * (th[pr] + th[tr]), w.y * (th[pr] - th[tr])));
        s = cadd(s, cmk(w.x * (ts[pr] + ts[tr]), w.y * (ts[pr] - ts[tr])));
      }
      H[pr] = h;
      S[pr] = s;
    }
  }
  __syncthreads();
  // exact Hermitian symmetrisation of the formed pair (removes rounding
  // asymmetry; the factor route forms Hermitian blocks directly)
  if (F.source != FROM_FACTORS) {
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      int mu = pr / m0, nu = pr % m0;
      if (mu < nu) {
        cplx h1 = H[pr], h2 = H[nu * m0 + mu], s1 = S[pr], s2 = S[nu * m0 + mu];
        cplx hm = cscale(cadd(h1, cconj(h2)), 0.5), sm2 = cscale(cadd(s1, cconj(s2)), 0.5);
        H[pr] = hm; H[nu * m0 + mu] = cconj(hm);
        S[pr] = sm2; S[nu * m0 + mu] = cconj(sm2);
      } else if (mu == nu) {
        H[pr].y = 0.0; S[pr].y = 0.0;
      }
    }
    __syncthreads();
  }
  if (F.outH)
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      F.outH[(size_t)jl * np + pr] = H[pr];
      F.outS[(size_t)jl * np + pr] = S[pr];
    }
  if (F.want == 0) return;
  __syncthreads();
  // reduction on the directions of Sbar above the dependency cut (only
  // numerically singular Bloch combinations are removed)
  __shared__ int keep[MAXM0];
  __shared__ double sv[MAXM0];
  __shared__ double s_tau;
  if (F.source == FROM_FACTORS) {
    if (threadIdx.x == 0) s_tau = *F.tau;
  } else {
    // B = |T_S[0]| + sum_{d >= 1} (|T_S[d]| + |T_S[d]|^T) of the embedded
    // generators, tau = null_tau(||B||_F)
    double part = 0.0;
    for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
      const int tr = (pr % m0) * m0 + pr / m0;
      double b = fabs(F.TS[pr]);
      for (int dd2 = 1; dd2 <= F.D; ++dd2) b += fabs(F.TS[(size_t)dd2 * np + pr]) + fabs(F.TS[(size_t)dd2 * np + tr]);
      part += b * b;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    __shared__ double red_b[32];
    if ((threadIdx.x & 31) == 0) red_b[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red_b[w];
      s_tau = null_tau(sqrt(t), (double)F.M * m0);   // the embedding's order
    }
  }
  __syncthreads();
  // Cholesky when it certifies that nothing is numerically singular, else the
  // eigendecomposition of Sbar_j with the cut
  const bool chol = cta_cholesky_reduce(H, S, Aj, Qj, m0, s_tau);
  if (!chol && alias) reform_S(F, P, j, m0, S, Qj, ldj);   // the attempt factored Sbar in place
  int r = chol ? m0 : cta_lowdin_reduce(H, S, Aj, Qj, m0, s_tau, sv, keep, false);
  if (r < 0) {                                             // QL ran out on Sbar in place
    reform_S(F, P, j, m0, S, Qj, ldj);
    r = cta_lowdin_reduce(H, S, Aj, Qj, m0, s_tau, sv, keep, true);
  }
  if (!chol && F.neig && threadIdx.x == 0) atomicAdd(F.neig, 1);
  const int ldr = r + (r & 1);
  if (F.vecs) {   // the reduced matrix, kept for its eigenvectors
    for (int it = threadIdx.x; it < r * r; it += blockDim.x) Vc[(it / r) * ldr + it % r] = H[it];
    __syncthreads();
  }
  if (r > 0) cta_tridiag(H, r, dd, ee, v, pv);
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double e2i = (i + 1 < r) ? ee[i] * ee[i] : 0.0;
    e2[i] = e2i;
    df[i] = (float)dd[i];
    e2f[i] = (float)e2i;
  }
  __syncthreads();
  if (F.want == 1) {
    for (int i = threadIdx.x; i < m0; i += blockDim.x) {
      const double lam = (i < r) ? tridiag_eig_fast(df, e2f, dd, e2, r, i, 0.0) : INFINITY;
      F.ev[(size_t)jl * m0 + i] = lam;
      if (F.blk) F.blk[(size_t)jl * m0 + i] = j;
      if (jm >= 0) {   // the conjugate block's spectrum
        F.ev[(size_t)(jm - F.j0) * m0 + i] = lam;
        if (F.blk) F.blk[(size_t)(jm - F.j0) * m0 + i] = jm;
      }
    }
  } else if (threadIdx.x == 0) {
    // the lowest eigenvalue of an embedding block only sets the preconditioner
    // shift (lowered by 2e-5 relative afterwards): 1e-9 relative suffices
    F.ev[jl] = (r > 0) ? tridiag_eig_fast(df, e2f, dd, e2, r, 0, 1e-9) : INFINITY;
  }
  if (F.vecs && F.want == 1) {
    // eigenvectors of the reduced matrix by Jacobi (orthonormal also inside
    // degenerate clusters), ordered by eigenvalue, mapped back by the
    // reduction's transform: y = L^-H w (Cholesky route) or X w (X = Q_K
    // diag(s_K)^-1/2), so y^H Sbar_j y = 1; the conjugate block gets conj(y)
    __shared__ int ord[MAXM0];
    __syncthreads();
    if (r > 0) cta_jacobi_herm(Vc, Wv, r, ldr);
    if (threadIdx.x == 0) {
      for (int i = 0; i < r; ++i) ord[i] = i;
      for (int i = 1; i < r; ++i) {
        const int o = ord[i];
        const double e = Vc[o * ldr + o].x;
        int q = i - 1;
        while (q >= 0 && Vc[ord[q] * ldr + ord[q]].x > e) { ord[q + 1] = ord[q]; --q; }
        ord[q + 1] = o;
      }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < np; it += blockDim.x) {
      const int i = it / m0, mu = it % m0;
      cplx y = cmk(0.0, 0.0);
      if (i < r) {
        const int c = ord[i];
        if (chol) {
          for (int nu = mu; nu < m0; ++nu) y = cadd(y, cmul(cconj(Qj[nu * m0 + mu]), Wv[nu * ldr + c]));
        } else {
          for (int nu = 0; nu < r; ++nu) y = cadd(y, cmul(Aj[mu * r + nu], Wv[nu * ldr + c]));
        }
      }
      F.vecs[(size_t)jl * np + it] = y;
      if (jm >= 0) F.vecs[(size_t)(jm - F.j0) * np + it] = cconj(y);
    }
  }
}

// Lattice eigenvectors from Fourier-block eigenvectors (Prop. A.1, the
// columns of the inverse DFT over the lattice index, U = (F^* (x) I) Ubar):
// U[c][(k, mu)] = f_j[k] y[mu] with f_j[k] = exp(+2 pi i j.k / L) / sqrt(|L|),
// for each requested pair c (Fourier index jbar[c], block-local vector
// vec[c] in ys).  One thread per entry; twiddles by sincospi of the exact
// integer phase j.k mod L.
__global__ void k_bloch_vectors(int L1, int L2, int L3, int m0, int nsel, const int* __restrict__ jbar,
                                const cplx* __restrict__ ys, const int* __restrict__ slot, cplx* __restrict__ U) {
  const long long nb = (long long)L1 * L2 * L3 * m0, tot = nb * nsel;
  const double inv = rsqrt((double)L1 * L2 * L3);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < tot; it += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(it / nb);
    const long long a = it % nb;
    const int mu = (int)(a % m0);
    const long long kb = a / m0;
    const int k3 = (int)(kb % L3), k2 = (int)((kb / L3) % L2), k1 = (int)(kb / ((long long)L2 * L3));
    const int j = jbar[c];
    const int j3 = j % L3, j2 = (j / L3) % L2, j1 = j / (L2 * L3);
    // phase 2 pi (j1 k1 / L1 + j2 k2 / L2 + j3 k3 / L3), each term reduced exactly
    const double ph = 2.0 * ((double)((long long)j1 * k1 % L1) / L1 + (double)((long long)j2 * k2 % L2) / L2 +
                             (double)((long long)j3 * k3 % L3) / L3);
    double sn, cs;
    sincospi(ph, &sn, &cs);
    const cplx y = ys[(size_t)slot[c] * m0 + mu];
    U[it] = cscale(cmul(cmk(cs, sn), y), inv);
  }
}

void launch_bloch_vectors(int L1, int L2, int L3, int m0, int nsel, const int* jbar, const cplx* ys, const int* slot,
                          cplx* U, cudaStream_t st) {
  if (nsel > 0) k_bloch_vectors<<<1024, 256, 0, st>>>(L1, L2, L3, m0, nsel, jbar, ys, slot, U);
}

// One CTA per periodic problem: its dependency cut (NullTask).
__global__ void k_null_tau(const NullTask* __restrict__ tasks) {
  const NullTask T = tasks[blockIdx.x];
  const int np = T.m0 * T.m0;
  const size_t os = (size_t)T.nF * np;   // offset stride of a factor tensor
  double part = 0.0;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    double b = 1.0;
    for (int a = 0; a < 3; ++a) {
      double acc = 0.0;
      for (int o = 0; o < T.noff[a]; ++o) acc += fabs(T.X[a][(size_t)o * os + pr]);
      b *= acc;
    }
    part += b * b;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    *T.tau = null_tau(sqrt(t), (double)T.nb);
  }
}

void launch_null_tau(const NullTask* tasks, int ntask, cudaStream_t st) {
  if (ntask) k_null_tau<<<ntask, 256, 0, st>>>(tasks);
}

// ---- preconditioner ----


__global__ void k_sigma(const PrecTask* __restrict__ tasks) {
  const PrecTask T = tasks[blockIdx.x];
  __shared__ double red[256];
  double mn = DBL_MAX;
  for (int j = threadIdx.x; j < T.M; j += blockDim.x) mn = fmin(mn, T.emin[j]);
  red[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *T.sigma = red[0] - T.rel_shift * (1.0 + fabs(red[0]));
}

__global__ void k_precond(const ProbDev* __restrict__ probs, const PrecTask* __restrict__ tasks) {
  extern __shared__ cplx sm[];
  const PrecTask T = tasks[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= T.M) return;
  const int m0 = probs[T.prob].m0, np = m0 * m0;
  const double sg = *T.sigma;
  cplx* A = sm;
  cplx* Li = sm + np;
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    cplx h = T.CH[(size_t)j * np + pr], s = T.CS[(size_t)j * np + pr];
    A[pr] = csub(h, cscale(s, sg));
  }
  __syncthreads();
  cta_cholesky(A, m0);
  // Li = L^-1 (lower), thread per column
  for (int c = threadIdx.x; c < m0; c += blockDim.x) {
    for (int i = 0; i < m0; ++i) {
      cplx s = cmk(i == c ? 1.0 : 0.0, 0.0);
      for (int q = c; q < i; ++q) s = csub(s, cmul(A[i * m0 + q], Li[q * m0 + c]));
      Li[i * m0 + c] = (i < c) ? cmk(0.0, 0.0) : cscale(s, 1.0 / A[i * m0 + i].x);
    }
  }
  __syncthreads();
  // K = L^-H L^-1 : K[a][b] = sum_i conj(Li[i][a]) Li[i][b]
  for (int pr = threadIdx.x; pr < np; pr += blockDim.x) {
    int a = pr / m0, b = pr % m0;
    cplx s = cmk(0.0, 0.0);
    for (int i = max(a, b); i < m0; ++i) s = cadd(s, cmulc(Li[i * m0 + b], Li[i * m0 + a]));
    T.K[(size_t)j * np + pr] = s;
  }
}

// ---- sorting of (value, index) pairs ----
// Order: ascending value, ties by ascending index.  Pads carry +inf and an
// index above every real one, so they sort after the removed directions'
// +inf entries and the result is deterministic.

__device__ inline bool pair_gt(double va, int ia, double vb, int ib) {
  return va > vb || (va == vb && ia > ib);
}

__global__ void k_sort_small(const SortTask* __restrict__ tasks) {
  extern __shared__ double ssv[];
  const SortTask T = tasks[blockIdx.x];
  int n2 = 1;
  while (n2 < T.n) n2 <<= 1;
  double* sv = ssv;
  int* si = (int*)(ssv + n2);
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    sv[i] = (i < T.n) ? T.v[i] : INFINITY;
    si[i] = (i < T.n) ? (T.idx ? T.idx[i] : i) : 0x7fffffff;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        int ij = i ^ jj;
        if (ij > i) {
          bool up = ((i & k) == 0);
          if (pair_gt(sv[i], si[i], sv[ij], si[ij]) == up) {
            double tv = sv[i]; sv[i] = sv[ij]; sv[ij] = tv;
            int ti = si[i]; si[i] = si[ij]; si[ij] = ti;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < T.n; i += blockDim.x) {
    T.v[i] = sv[i];
    if (T.idx) T.idx[i] = si[i];
  }
}

// one compare-exchange pass of a global bitonic network (n2 a power of 2;
// v/idx padded to n2 with +inf)
__global__ void k_bitonic_pass(double* v, int* idx, int n2, int k, int jj) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    int ij = i ^ jj;
    if (ij > i) {
      bool up = ((i & k) == 0);
      if (pair_gt(v[i], idx[i], v[ij], idx[ij]) == up) {
        double tv = v[i]; v[i] = v[ij]; v[ij] = tv;
        int ti = idx[i]; idx[i] = idx[ij]; idx[ij] = ti;
      }
    }
  }
}

__global__ void k_pad_copy(const double* v, const int* idx, int n, double* pv, int* pidx, int n2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += gridDim.x * blockDim.x) {
    pv[i] = (i < n) ? v[i] : INFINITY;
    pidx[i] = (i < n) ? (idx ? idx[i] : i) : 0x7fffffff;
  }
}

__global__ void k_unpad_copy(const double* pv, const int* pidx, int n, double* v, int* idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[i] = pv[i];
    if (idx) idx[i] = pidx[i];
  }
}

// ---- launchers ----
// m0: the launch's largest block order; any_odd: some block of the launch has
// odd m0 (its layout keeps a padded work array of its own)
size_t fblocks_smem(int m0, bool vectors, bool any_odd) {
  const int ldj = m0 + (m0 & 1);
  const size_t mats = (!any_odd && !(m0 & 1)) ? (size_t)2 * m0 * m0 + (size_t)ldj * ldj
                                              : (size_t)2 * m0 * m0 + (size_t)2 * ldj * ldj;
  return (mats + 2 * MAXM0) * sizeof(cplx) + 3 * MAXM0 * sizeof(double) + 2 * MAXM0 * sizeof(float) +
         (vectors ? 16 + 2 * ldj * ldj * sizeof(cplx) : 0);
}

// x0, nx: the launch covers local indices x0 .. x0 + nx - 1 of every task
// (nx < 0: up to maxnj), so that a large solve can be issued in pieces
void launch_fblocks(const ProbDev* probs, const FBlockTask* tasks, int ntask, int maxnj, int maxm0,
                    cudaStream_t st, bool vectors, int x0, int nx, bool any_odd) {
  const int gx = (nx < 0) ? maxnj - x0 : std::min(nx, maxnj - x0);
  if (!ntask || gx <= 0) return;
  size_t sm = fblocks_smem(maxm0, vectors, any_odd);
  FOCK_SMEM_OPTIN(k_fblocks);
  {   // the largest shared-memory carveout: four 32 x 32 blocks (~54 KB each) per SM
    static std::once_flag carve;
    std::call_once(carve, [] { cudaFuncSetAttribute(k_fblocks, cudaFuncAttributePreferredSharedMemoryCarveout, 100); });
  }
  // the rotation and update phases of an m0 x m0 block have about m0^2 / 2
  // parallel items: one warp for m0 <= 8 (more independent blocks resident
  // per SM keep the FP64 pipe busy), up to four warps for m0 = 32
  const int threads = (maxm0 <= 8) ? 32 : (maxm0 <= 16) ? 64 : 128;
  k_fblocks<<<dim3(gx, ntask), threads, sm, st>>>(probs, tasks, x0);
}

void launch_precond(const ProbDev* probs, const PrecTask* tasks, int ntask, int maxM, int maxm0,
                    cudaStream_t st) {
  if (!ntask) return;
  k_sigma<<<ntask, 256, 0, st>>>(tasks);
  size_t sm = (size_t)2 * maxm0 * maxm0 * sizeof(cplx);
  FOCK_SMEM_OPTIN(k_precond);
  k_precond<<<dim3(maxM, ntask), 128, sm, st>>>(probs, tasks);
}

void launch_sort_small(const SortTask* tasks, int ntask, int maxn, cudaStream_t st) {
  if (!ntask) return;
  int n2 = 1;
  while (n2 < maxn) n2 <<= 1;
  size_t sm = (size_t)n2 * (sizeof(double) + sizeof(int));
  FOCK_SMEM_OPTIN(k_sort_small);
  k_sort_small<<<ntask, 512, sm, st>>>(tasks);
}

// sort n pairs in place with scratch (pv, pidx of length n2 = next pow2)
void launch_sort_global(double* v, int* idx, int n, double* pv, int* pidx, cudaStream_t st) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  int grid = (n2 + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_pad_copy<<<grid, 256, 0, st>>>(v, idx, n, pv, pidx, n2);
  for (int k = 2; k <= n2; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) k_bitonic_pass<<<grid, 256, 0, st>>>(pv, pidx, n2, k, jj);
  k_unpad_copy<<<grid, 256, 0, st>>>(pv, pidx, n, v, idx);
}

}  // namespace fock
