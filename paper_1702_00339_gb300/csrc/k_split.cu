// FP64 matrix products on the fifth-generation tensor cores by exact
// split products (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication", Numer. Algorithms 59 (2012)), used by the mixed
// form for the quadrature contractions of stage (a) (Lemma 2.1 display,
// Eqs. 2.16-2.17: X_t[mu nu] = sum_r P_t[r] Z[r][mu nu]).
//
// For a chunk of KC = 64 along the summation index, every row of A and every
// column of B is aligned to its largest binary exponent, and its 53-bit
// integer mantissas are cut into NDIG = 7 signed base-128 digits (|digit| <=
// 127, exact in BF16).  For each level g = j + l (2 <= g <= NDIG + 1) the
// products of digit planes j of A and l of B are summed by tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32) into one TMEM accumulator per level; the
// level sums are integers below 2^24, so FP32 accumulation is exact.  Each
// thread then combines its row's levels in 64-bit integers and adds the
// chunk, scaled by the two exponents, into FP64 accumulators.  Truncation:
// the digits keep 49 of the 53 mantissa bits and the levels above NDIG + 1
// are dropped, so each product carries a relative error below ~2^-46 of
// (row maximum x column maximum) per summand.
//
// One CTA of 128 threads per 128 x 64 output tile (M tiles of 128 rows of A,
// N tiles of 64 columns of B); operands staged by the threads into shared
// memory in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per
// core matrix); one thread issues the MMAs and commits them to an mbarrier;
// every wait is bounded (clock64), after which the kernel flags an error,
// frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace fock {

namespace {

constexpr int TM = 128, TN = 64, KC = 64, NDIG = 7;   // digit levels g = 2 .. NDIG + 1
constexpr int TMEM_COLS = 512;                                     // NLEV * TN = 448 used
constexpr uint32_t A_PLANE = TM * KC * 2, B_PLANE = TN * KC * 2;   // bytes per digit plane
constexpr size_t SPLIT_SMEM = (size_t)NDIG * (A_PLANE + B_PLANE) + 1024;
constexpr long long kWaitCycles = 4000000000ll;                    // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of an R x KC operand: core matrix (r/8, k/8),
// K-adjacent core matrices 128 B apart (LBO), 8-row groups KC/8 * 128 B apart (SBO)
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * (KC >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = (KC / 8) * 128;
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((lbo >> 4) & 0x3FFF) << 16 | ((sbo >> 4) & 0x3FFF) << 32 |
         (uint64_t)1 << 46;   // version 1, base offset 0, no swizzle
}

// instruction descriptor: D FP32, A and B BF16, both K-major, M = TM, N = TN
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

// biased exponent field of |x| (0 for zero and subnormals: they align as exponent 1)
__device__ __forceinline__ int exp_field(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return e == 0 ? 1 : e;
}

// the NDIG signed base-128 digits of x aligned to the exponent field E
__device__ __forceinline__ void digits(double x, int E, __nv_bfloat16* q) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  long long m = b & 0xFFFFFFFFFFFFFll;
  if (ex != 0) m |= 1ll << 52;
  const int sh = E - (ex == 0 ? 1 : ex);
  const long long a = (sh < 53) ? (m >> sh) : 0;
  const int sg = b < 0 ? -1 : 1;
#pragma unroll
  for (int j = 0; j < NDIG; ++j) q[j] = __int2bfloat16_rn(sg * (int)((a >> (46 - 7 * j)) & 127));
}

__device__ __forceinline__ double pow2(int e) {   // 2^e, 0 below the normal range
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase) {
  const long long t0 = clock64();
  uint32_t done = 0;
  while (!done) {
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
    if (!done && clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// Stage one operand chunk as digit planes: R rows of `rows` (<= TR), KC
// columns along k from k0; element (r, k) at P[r * sr + k * sk].  Rows that
// do not exist and k beyond K give zero digits.  Writes the row exponents.
template <int TR>
__device__ void stage(const double* __restrict__ P, long long sr, long long sk, int rows, int k0, int K,
                      unsigned char* planes, uint32_t plane_bytes, int* rexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (sk == 1) {
    // rows contiguous along k: one warp per row, lanes along k; the loads of
    // SU rows are issued before any of them is converted (their latency
    // overlaps instead of adding up row after row)
    constexpr int SU = 4;
    for (int r0 = warp; r0 < TR; r0 += 4 * SU) {
      double x0[SU], x1[SU];
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int r = r0 + 4 * u;
        x0[u] = 0.0; x1[u] = 0.0;
        if (r < rows) {
          if (k0 + lane < K) x0[u] = P[r * sr + (k0 + lane)];
          if (k0 + lane + 32 < K) x1[u] = P[r * sr + (k0 + lane + 32)];
        }
      }
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int r = r0 + 4 * u;
        if (r >= TR) break;
        const int E = __reduce_max_sync(0xffffffffu, max(exp_field(x0[u]), exp_field(x1[u])));
        if (lane == 0) rexp[r] = E;
        __nv_bfloat16 q[NDIG];
        digits(x0[u], E, q);
#pragma unroll
        for (int j = 0; j < NDIG; ++j) *(__nv_bfloat16*)(planes + j * plane_bytes + core_off(r, lane)) = q[j];
        digits(x1[u], E, q);
#pragma unroll
        for (int j = 0; j < NDIG; ++j) *(__nv_bfloat16*)(planes + j * plane_bytes + core_off(r, lane + 32)) = q[j];
      }
    }
  } else {
    // lanes along the rows (coalesced when rows are contiguous), loop along k
    // in groups of SK independent loads (the exponent pass and the digit pass
    // each keep SK loads in flight)
    constexpr int SK = 8;
    for (int r = threadIdx.x; r < TR; r += blockDim.x) {
      const bool live = (r < rows);
      int E = 1;
      for (int kb = 0; kb < KC; kb += SK) {
        double x[SK];
#pragma unroll
        for (int u = 0; u < SK; ++u)
          x[u] = (live && k0 + kb + u < K) ? P[r * sr + (long long)(k0 + kb + u) * sk] : 0.0;
#pragma unroll
        for (int u = 0; u < SK; ++u) E = max(E, exp_field(x[u]));
      }
      rexp[r] = E;
      for (int kb = 0; kb < KC; kb += SK) {
        double x[SK];
#pragma unroll
        for (int u = 0; u < SK; ++u)
          x[u] = (live && k0 + kb + u < K) ? P[r * sr + (long long)(k0 + kb + u) * sk] : 0.0;
#pragma unroll
        for (int u = 0; u < SK; ++u) {
          __nv_bfloat16 q[NDIG];
          digits(x[u], E, q);
#pragma unroll
          for (int j = 0; j < NDIG; ++j) *(__nv_bfloat16*)(planes + j * plane_bytes + core_off(r, kb + u)) = q[j];
        }
      }
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(128, 1) k_split_gemm(const SplitTask* __restrict__ tasks, int max_ks, int* err) {
  const SplitTask T = tasks[blockIdx.z / max_ks];
  const int ks = blockIdx.z % max_ks, nks = max(T.ksplit, 1);
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  if (ks >= nks || m0 >= T.M || n0 >= T.N) return;
  if (T.active && *T.active == 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Ap = (unsigned char*)(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
  unsigned char* Bp = Ap + NDIG * A_PLANE;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int rexpA[TM], rexpB[TN];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rowsA = min(TM, T.M - m0), colsB = min(TN, T.N - n0);
  const double* Ab = T.A + (long long)m0 * T.a_m;
  const double* Bb = T.B + (long long)n0 * T.b_n;
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;
  const int row = 32 * (warp & 3) + lane;     // this thread's TMEM lane = output row of the tile
  double acc[TN];
#pragma unroll
  for (int c = 0; c < TN; ++c) acc[c] = 0.0;
  // this CTA's chunks of the summation: [c_lo, c_hi) of ceil(K / KC)
  const int nchunk_all = (T.K + KC - 1) / KC, cps = (nchunk_all + nks - 1) / nks;
  const int c_lo = min(ks * cps, nchunk_all), c_hi = min(c_lo + cps, nchunk_all);
  const int nchunk = c_hi - c_lo;
  bool ok = true;
  for (int ch = 0; ch < nchunk && ok; ++ch) {
    const int k0 = (c_lo + ch) * KC;
    stage<TM>(Ab, T.a_m, T.a_k, rowsA, k0, T.K, Ap, A_PLANE, rexpA);
    stage<TN>(Bb, T.b_n, T.b_k, colsB, k0, T.K, Bp, B_PLANE, rexpB);
    asm volatile("fence.proxy.async.shared::cta;");   // generic-proxy writes -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(Ap), b0 = smem_u32(Bp);
      for (int g = 2; g <= NDIG + 1; ++g) {
        const uint32_t dcol = tbase + (uint32_t)((g - 2) * TN);
        uint32_t accum = 0;
        for (int j = 1; j <= NDIG; ++j) {
          const int l = g - j;
          if (l < 1 || l > NDIG) continue;
          for (int kk = 0; kk < KC / 16; ++kk) {
            const uint64_t da = smem_desc(a0 + (j - 1) * A_PLANE + kk * 256);
            const uint64_t db = smem_desc(b0 + (l - 1) * B_PLANE + kk * 256);
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                         :: "r"(dcol), "l"(da), "l"(db), "r"(kIdesc), "r"(accum));
            accum = 1;
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar)) : "memory");
    }
    if (!wait_phase(smem_u32(&mbar), (uint32_t)(ch & 1))) {
      atomicExch(&s_fail, 1);
    }
    __syncthreads();
    if (s_fail) { ok = false; break; }
    asm volatile("tcgen05.fence::after_thread_sync;");
    // combine the levels of this thread's row in 64-bit integers, add in FP64
    const double rs = pow2(rexpA[row] - 1050);
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
    for (int c0 = 0; c0 < TN; c0 += 8) {
      long long S[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) S[c] = 0;
#pragma unroll
      for (int g = 2; g <= NDIG + 1; ++g) {
        uint32_t v[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                       "=r"(v[7])
                     : "r"(lane_addr + (uint32_t)((g - 2) * TN + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int c = 0; c < 8; ++c)
          S[c] += (long long)__float2int_rn(__uint_as_float(v[c])) * (1ll << (7 * (NDIG + 1 - g)));
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c0 + c] = fma((double)S[c], rs * pow2(rexpB[c0 + c] - 1050), acc[c0 + c]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();   // the digit planes and TMEM are reused by the next chunk
  }
  if (!ok) {
    // an MMA group did not complete in time: wait (bounded) once more so no
    // write to TMEM is in flight when it is freed, flag the error
    if (tid == 0) {
      wait_phase(smem_u32(&mbar), (uint32_t)((nchunk - 1) & 1));
      atomicExch(err, 1);
    }
    __syncthreads();
  } else if (row < rowsA && T.work) {
    // a partial sum over this CTA's chunks, reduced by k_split_reduce
    double* Wr = T.work + ((long long)ks * T.M + m0 + row) * T.N + n0;
#pragma unroll
    for (int c = 0; c < TN; ++c)
      if (c < colsB) Wr[c] = acc[c];
  } else if (row < rowsA) {
    // value = S * 2^(EA + EB - 2100): the per-row and per-column factors
    // 2^(E - 1050) multiply to it
    double* Cr = T.C + (long long)(m0 + row) * T.c_m + (long long)n0 * T.c_n;
#pragma unroll
    for (int c = 0; c < TN; ++c)
      if (c < colsB) {
        double v = T.alpha * acc[c];
        if (T.beta != 0.0) v = fma(T.beta, Cr[(long long)c * T.c_n], v);
        Cr[(long long)c * T.c_n] = v;
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(TMEM_COLS));
}

// C = alpha sum_ks work[ks] + beta C for the tasks with partial sums, the
// K ranges added in a fixed order (results independent of scheduling); a
// symmetric C takes its upper triangle and mirrors it bitwise.
__global__ void k_split_reduce(const SplitTask* __restrict__ tasks) {
  const SplitTask T = tasks[blockIdx.y];
  if (!T.work) return;
  if (T.active && *T.active == 0) return;
  const long long mn = (long long)T.M * T.N;
  const int nks = max(T.ksplit, 1);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < mn; it += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(it / T.N), n = (int)(it % T.N);
    if (T.sym && m > n) continue;
    double s = 0.0;
    for (int ks = 0; ks < nks; ++ks) s += T.work[ks * mn + it];
    double* c = T.C + (long long)m * T.c_m + (long long)n * T.c_n;
    const double v = (T.beta != 0.0) ? fma(T.beta, *c, T.alpha * s) : T.alpha * s;
    *c = v;
    if (T.sym && m < n) T.C[(long long)n * T.c_m + (long long)m * T.c_n] = v;
  }
}

size_t split_gemm_smem() { return SPLIT_SMEM; }

void launch_split_gemm(const SplitTask* tasks, int ntask, int max_m, int max_n, int* err, cudaStream_t st,
                       int max_ks, bool reduce) {
  if (!ntask || max_m <= 0 || max_n <= 0) return;
  FOCK_SMEM_OPTIN(k_split_gemm);
  max_ks = max_ks < 1 ? 1 : max_ks;
  dim3 grid((max_n + TN - 1) / TN, (max_m + TM - 1) / TM, ntask * max_ks);
  k_split_gemm<<<grid, 128, SPLIT_SMEM, st>>>(tasks, max_ks, err);
  if (reduce) k_split_reduce<<<dim3(64, ntask), 256, 0, st>>>(tasks);
}

}  // namespace fock
