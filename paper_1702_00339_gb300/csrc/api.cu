// libfock host layer: problem validation, geometry and index maps, the
// device memory plan of a batch of problems, the stage drivers and the C ABI.
//
// A batch is planned twice with the same deterministic code: once to size
// the device slab, once with the real base address to fill the descriptors.
// Every array of the path lives in that slab; all arithmetic of the method
// runs in the kernels (k_assemble.cu, k_eig.cu, k_matvec.cu, k_lobpcg.cu).
#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fock.h"
#include "common.cuh"

namespace fock {















// launchers (defined in the .cu files)
void launch_vec1d(const ProbDev*, const SegDesc*, int, const SegDesc*, int, const DefTab*, int, int, int, cudaStream_t);
void launch_gram(const ProbDev*, const GramTask*, int, const DefTab*, cudaStream_t);
void launch_combine(const ProbDev*, const CombineTask*, int, cudaStream_t);
void launch_defects(const ProbDev*, const DefField*, int, const DefBlock*, int, cudaStream_t);
void launch_axis_dft(const ProbDev*, const DftTask*, int, int, cudaStream_t);
void launch_fblocks(const ProbDev*, const FBlockTask*, int, int, int, cudaStream_t, bool vectors = false,
                    int x0 = 0, int nx = -1, bool any_odd = true);
void launch_bloch_vectors(int, int, int, int, int, const int*, const cplx*, const int*, cplx*, cudaStream_t);
void launch_split_gemm(const SplitTask*, int, int, int, int*, cudaStream_t, int max_ks = 1, bool reduce = false);
void launch_null_tau(const NullTask*, int, cudaStream_t);
void launch_precond(const ProbDev*, const PrecTask*, int, int, int, cudaStream_t);
void launch_sort_small(const SortTask*, int, int, cudaStream_t);
void launch_sort_global(double*, int*, int, double*, int*, cudaStream_t);
void launch_twiddles(CircDev*, int, cudaStream_t);
void launch_fft(const FftTask*, int, int, int, int, int, cudaStream_t, bool);
void launch_fft_cc(const FftTask*, int, int, int, int, int, cudaStream_t, bool);
int fft_max_cc(int);
void launch_blockmul(const BmulTask*, int, int, int, cudaStream_t, bool);
void launch_eapply(const EApplyTask*, int, int, cudaStream_t);
int eapply_grid(long long items);
void launch_band_factor(const BandTask*, int, cudaStream_t);
void launch_band_solve(const BandTask*, int, int, int, int, cudaStream_t, bool);
int band_stage_doubles(int);
void launch_cell_canon(const CanonTask*, int, int, int, cudaStream_t);
void launch_gather(const GatherSeg*, int, uint32_t*, cudaStream_t);
void launch_cell_back(const double*, int, int, int, const double*, double*, int, cudaStream_t);
__global__ void k_init_x(const InitTask*);
void launch_gemm_tn(const GemmTask*, int, int, int, int, cudaStream_t);
__global__ void k_gemm_nn(const GemmTask*);
__global__ void k_resid(const ResidTask*, double);
__global__ void k_rr(const RRTask*, int, int);
__global__ void k_rr_cl(const RRTask*);
size_t rr_cl_smem(int, int);
__global__ void k_copy_cols(const CopyTask*);
__global__ void k_colnorm(const CopyTask*);
}  // namespace fock

using namespace fock;

struct fock_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // the structured problems' iteration runs on `hi` (greatest priority) while
  // the periodic problems' eigensolves run on `stream`; ev_fork / ev_join
  // order the two against `stream`
  cudaStream_t hi = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_chunk = nullptr;
  // while a plan's iteration runs on hi: the stream its periodic problems'
  // Fourier-block pieces go to (nullptr otherwise)
  cudaStream_t pstream = nullptr;
  // tuner results: FFT columns per CTA by (largest embedding M, largest column count)
  std::map<std::pair<int, int>, int> fft_tune;
  size_t budget = 0;
  char* arena = nullptr;
  size_t arena_cap = 0;
  uint32_t* hstage = nullptr;        // pinned host staging of gathered results
  size_t hstage_cap = 0;             // (words)
  cudaMemPool_t mempool = nullptr;   // serving workers: batches allocated stream-ordered from this pool
  std::string err;
  // kernel timers: events recorded around launches while enabled
  bool prof = false;
  struct Rec { const char* name; int nlaunch; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

namespace {
thread_local fock_ctx* g_prof = nullptr;   // context whose launches are being timed

cudaEvent_t prof_event(fock_ctx* c) {
  if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Brackets the launches issued in its scope with two events on the stream.
struct ProfScope {
  fock_ctx* c = nullptr;
  size_t idx = 0;
  ProfScope(const char* name, int nlaunch) {
    if (!g_prof || !g_prof->prof) return;
    c = g_prof;
    fock_ctx::Rec r{name, nlaunch, prof_event(c), prof_event(c)};
    cudaEventRecord(r.a, c->stream);
    idx = c->recs.size();
    c->recs.push_back(r);
  }
  ~ProfScope() {
    if (c) cudaEventRecord(c->recs[idx].b, c->stream);
  }
};
struct ProfBind {   // sets the context being timed for the duration of an API call
  fock_ctx* prev;
  explicit ProfBind(fock_ctx* c) : prev(g_prof) { g_prof = c; }
  ~ProfBind() { g_prof = prev; }
};
}  // namespace
#define PROF_CAT2(a, b) a##b
#define PROF_CAT(a, b) PROF_CAT2(a, b)
#define PROF(name, n) ProfScope PROF_CAT(prof_scope_, __LINE__)(name, n)

namespace {

const int kSmallSort = 4096;
const double kPrecShift = 2e-5;   // sigma = min_j lambda_min(Chat_j) - kPrecShift (1 + |.|)
// mixed form: the block iteration's dense products go to the tensor cores for
// chains of at least this many basis functions (the Gram sums are over them;
// shorter sums do not repay the digit splitting: measured 56 vs 50 ms per
// batch of 64 chains of 512 functions, 0.84 vs 1.66 s for one of 16384)
const int kSplitMinRows = 2048;
// Rayleigh-Ritz working matrices (3 ld^2 doubles) up to this many bytes live in
// shared memory
const size_t kRRSmemCap = 160 * 1024;
// Fourier blocks (CTAs, of which about half are conjugates that return at
// once) per piece launched beside a Rayleigh-Ritz launch: about three waves of
// the 32 x 32 block kernel on the SMs the iteration leaves free, ~10 ms
const int kPeriodicPieceCTAs = 3072;

int set_err(fock_ctx* c, int code, const std::string& m) {
  if (c) c->err = m;
  return code;
}

#define CUDA_TRY(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return set_err(ctx, FOCK_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---- host copy of one problem, with its quadrature table ----
struct HostProb {
  int L[3], per[3], N[3], n0;
  double b0, h, eps;
  int M0, m0, R, T, nF;
  std::vector<double> Z, frac, alpha, tq, cq;
  std::vector<int> ang, centre;
  int k_eig;
  int kind;            // 0 periodic (circulant eigensolve), 1 structured iteration
  int pchain = 0;      // structured path of a periodic chain (defects on a periodic axis 0)
  int mixed = 0;       // FOCK_MIXED or FOCK_MIXED_F32: dense products as tensor-core split products
  int f32 = 0;         // FOCK_MIXED_F32: FP32 preconditioner, FP32 matvecs until the residual is small
  int r2 = 0;          // box potential read as the plain lattice sum over the box's cells
  std::vector<fock_defect> defs;
};

// Guard vectors of the block iteration: k + g columns are iterated and the k
// lowest must converge; the guards move the convergence rate of the k-th
// eigenpair from lambda_{k+1} to lambda_{k+g+1} (clustered band edges).  Every
// guard also adds two slowly converging directions (its P and W columns) to the
// Rayleigh-Ritz basis: on 24 chains of 512 cells with k = 64, 8 guards instead
// of 16 cut the largest iteration count from 363 to 86 (FP64 form) and the
// time of each batch by 1.3-2.5x, with the same eigenvalues to 2e-15.
int lobpcg_guard(int k) { return std::max(4, k / 8); }

// Block size of the structured iteration: k + guards, or the whole space
// (N_b columns) when three blocks of it fit the Rayleigh-Ritz kernel -- then
// the first Rayleigh-Ritz step is exact and the solve ends there.
int lobpcg_block(int k, int Nb) {
  if (3 * Nb <= 255) return Nb;
  return k + lobpcg_guard(k);
}

int validate(const fock_problem& p, HostProb& H, std::string& why) {
  if (p.n0 <= 0 || !(p.b0 > 0.0)) { why = "n0 > 0 and b0 > 0 required"; return FOCK_EINVAL; }
  if (p.M0 < 1 || p.M0 > 8 || !p.Z || !p.frac) { why = "1 <= M0 <= 8 with Z and frac"; return FOCK_EINVAL; }
  if (p.m0 < 1 || p.m0 > MAXM0 || !p.exps || !p.ang || !p.centre) { why = "1 <= m0 <= 32 with exps/ang/centre"; return FOCK_EINVAL; }
  if (p.R < 3 || p.R > MAXR) { why = "3 <= R <= 64"; return FOCK_EINVAL; }
  if (p.ndef < 0 || (p.ndef > 0 && !p.defects)) { why = "ndef >= 0 with a defects array"; return FOCK_EINVAL; }
  if (p.precision != FOCK_FP64 && p.precision != FOCK_MIXED && p.precision != FOCK_MIXED_F32) {
    why = "precision FOCK_FP64, FOCK_MIXED or FOCK_MIXED_F32"; return FOCK_EINVAL;
  }
  H.mixed = (p.precision != FOCK_FP64) ? 1 : 0;
  H.f32 = (p.precision == FOCK_MIXED_F32) ? 1 : 0;
  H.n0 = p.n0; H.b0 = p.b0; H.h = p.b0 / p.n0;
  H.eps = (p.eps_support > 0.0) ? p.eps_support : 1e-14;
  int nlong = 0;
  bool dir_long = false;
  for (int a = 0; a < 3; ++a) {
    H.L[a] = p.L[a]; H.per[a] = p.periodic[a] ? 1 : 0; H.N[a] = p.N[a];
    if (p.L[a] < 1) { why = "L >= 1"; return FOCK_EINVAL; }
    if (H.per[a] && p.N[a] != p.L[a] * p.n0) { why = "periodic axis needs N = L*n0"; return FOCK_EINVAL; }
    if (!H.per[a] && p.N[a] < p.L[a] * p.n0) { why = "Dirichlet axis needs N >= L*n0"; return FOCK_EINVAL; }
    if (p.L[a] > 1) { ++nlong; if (!H.per[a]) dir_long = true; }
  }
  H.kind = (dir_long || p.ndef > 0) ? 1 : 0;
  if (H.kind == 1 && (nlong > 1 || p.L[0] == 1)) {
    why = "box problems and problems with defects must be chains along axis 0 (L1 >= 2, L2 = L3 = 1)";
    return FOCK_EINVAL;
  }
  H.pchain = (H.kind == 1 && H.per[0]) ? 1 : 0;
  if (p.ndef > 0) {
    if (p.periodic[1] || p.periodic[2]) { why = "defects need Dirichlet transverse axes"; return FOCK_EINVAL; }
    if (p.ndef > 64) { why = "at most 64 defects"; return FOCK_EINVAL; }
    H.defs.assign(p.defects, p.defects + p.ndef);
    for (const fock_defect& d : H.defs) {
      if (d.cell[0] < 0 || d.cell[0] >= p.L[0] || d.cell[1] != 0 || d.cell[2] != 0 ||
          d.nucleus < 0 || d.nucleus >= p.M0 || !std::isfinite(d.newZ)) {
        why = "defect cell / nucleus out of range or newZ not finite"; return FOCK_EINVAL;
      }
    }
  }
  H.M0 = p.M0; H.m0 = p.m0; H.R = p.R; H.T = p.M0 * p.R; H.nF = H.T + 2;
  H.Z.assign(p.Z, p.Z + p.M0);
  H.frac.assign(p.frac, p.frac + 3 * p.M0);
  H.alpha.assign(p.exps, p.exps + p.m0);
  H.ang.assign(p.ang, p.ang + p.m0);
  H.centre.assign(p.centre, p.centre + p.m0);
  for (int mu = 0; mu < p.m0; ++mu) {
    if (!(H.alpha[mu] > 0.0)) { why = "exponents must be positive"; return FOCK_EINVAL; }
    if (H.ang[mu] < 0 || H.ang[mu] > 3) { why = "ang in 0..3"; return FOCK_EINVAL; }
    if (H.centre[mu] < 0 || H.centre[mu] >= p.M0) { why = "centre out of range"; return FOCK_EINVAL; }
  }
  H.tq.resize(p.R);
  H.cq.resize(p.R);
  if (p.sinc_t && p.sinc_c) {
    for (int q = 0; q < p.R; ++q) {
      H.tq[q] = p.sinc_t[q]; H.cq[q] = p.sinc_c[q];
      if (!(H.tq[q] > 0.0)) { why = "sinc_t must be positive"; return FOCK_EINVAL; }
    }
  } else {
    double zmin, zmax;
    fock_default_range(&p, &zmin, &zmax);
    if (fock_sinc_table(p.R, zmin, zmax, H.tq.data(), H.cq.data(), nullptr) != FOCK_OK) {
      why = "default quadrature rule failed"; return FOCK_EINVAL;
    }
  }
  H.k_eig = (p.k_eig > 0) ? p.k_eig : 16;
  if (p.box_potential != 0 && p.box_potential != 1) { why = "box_potential 0 (replicated) or 1 (lattice sum)"; return FOCK_EINVAL; }
  if (p.box_potential == 1 && !(H.kind == 1 && !H.per[0])) {
    why = "box_potential 1 (the plain lattice sum) applies to box chains"; return FOCK_EINVAL;
  }
  H.r2 = p.box_potential;
  if (H.kind == 1) {
    int Nb = H.L[0] * H.m0;
    int kb = lobpcg_block(H.k_eig, Nb);
    // whole-space block: the first Rayleigh-Ritz step is exact, so the mixed
    // form has nothing to gain, and an FP32 Rayleigh-Ritz over [X | P | W]
    // (P, W inside span X) would only see noise: solved in FP64
    if (kb == Nb) H.f32 = 0;
    if (H.k_eig > Nb || 3 * kb > 255 || (kb < Nb && 3 * kb > Nb)) {
      why = "k_eig too large: k <= N_b and 3 (k + guard) <= min(N_b, 255) on chains with 3 N_b > 255"; return FOCK_EINVAL;
    }
  }
  return FOCK_OK;
}

// FNV-1a hash of the problem's parameters: the LOBPCG start of a problem is
// the same whatever batch it is solved in, and the same in every precision
// form (the forms then differ by their arithmetic alone).
uint64_t problem_seed(const HostProb& H) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  };
  mix(H.L, sizeof(H.L)); mix(H.per, sizeof(H.per)); mix(H.N, sizeof(H.N)); mix(&H.n0, sizeof(H.n0));
  mix(&H.r2, sizeof(H.r2));
  mix(&H.b0, sizeof(H.b0)); mix(&H.k_eig, sizeof(H.k_eig));
  mix(H.alpha.data(), H.alpha.size() * 8); mix(H.Z.data(), H.Z.size() * 8);
  mix(H.frac.data(), H.frac.size() * 8); mix(H.ang.data(), H.ang.size() * 4);
  mix(H.centre.data(), H.centre.size() * 4); mix(H.tq.data(), H.tq.size() * 8);
  for (const fock_defect& d : H.defs) { mix(d.cell, sizeof(d.cell)); mix(&d.nucleus, 4); mix(&d.newZ, 8); }
  return h;
}

inline int posmod_h(int a, int b) { int r = a % b; return r < 0 ? r + b : r; }

// smallest 2^a 3^b 5^c >= n
int smooth_at_least(int n) {
  for (int m = std::max(n, 1);; ++m) {
    int r = m;
    for (int f : {2, 3, 5}) while (r % f == 0) r /= f;
    if (r == 1) return m;
  }
}

std::vector<int> radix_factors(int M) {
  std::vector<int> f;
  int r = M;
  while (r % 4 == 0) { f.push_back(4); r /= 4; }
  for (int p : {2, 3, 5}) while (r % p == 0) { f.push_back(p); r /= p; }
  for (int p = 7; r > 1; p += 2) while (r % p == 0) { f.push_back(p); r /= p; }
  return f;
}

// ---- slab allocators used by the two planning passes ----
struct Slab {
  char* base = nullptr;  // null during the sizing pass
  size_t off = 0;
  std::vector<char>* stage = nullptr;   // upload slab: host staging copy
  template <class T> T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
  template <class T> T* put(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    size_t at = (off + 255) & ~(size_t)255;
    T* p = take<T>(v.size());
    if (stage) {
      if (stage->size() < off) stage->resize(off);
      std::memcpy(stage->data() + at, v.data(), v.size() * sizeof(T));
    }
    return p;
  }
};

// per-axis geometry of one problem (host side)
struct AxisPlan {
  int jmin, jmax;      // support of the reference-cell functions (virtual node index)
  int jlo, W, rlo, nr, pad;
  std::vector<int> offs;   // periodic: lattice offsets d with possibly non-zero forms
};

void axis_plan(const HostProb& H, int a, AxisPlan& A) {
  int N = H.N[a], L = H.L[a], n0 = H.n0;
  A.pad = H.per[a] ? 0 : (N - L * n0) / 2;
  int jmin = 1 << 30, jmax = -(1 << 30);
  for (int mu = 0; mu < H.m0; ++mu) {
    double cj = H.frac[H.centre[mu] * 3 + a] * n0 - 0.5;
    double r = std::sqrt(std::log(1.0 / H.eps) / H.alpha[mu]) / H.h;
    jmin = std::min(jmin, (int)std::floor(cj - r) - 1);
    jmax = std::max(jmax, (int)std::ceil(cj + r) + 1);
  }
  A.jmin = jmin; A.jmax = jmax;
  if (H.per[a]) {
    A.jlo = 0; A.W = N; A.rlo = 0; A.nr = n0;
    A.offs.clear();
    int span = jmax - jmin + 2;
    for (int d = 0; d < L; ++d) {
      int s = (d * n0) % N;
      int dist = std::min(s, N - s);
      if (span >= N || dist <= span) A.offs.push_back(d);
    }
  } else {
    A.jlo = jmin; A.W = jmax - jmin + 1;
    A.rlo = -A.pad; A.nr = N - (L - 1) * n0;
  }
}

// ---- one planned batch ----
struct Batch {
  int nprob = 0;
  std::vector<HostProb> hp;
  std::vector<AxisPlan> ap;          // [nprob*3]
  size_t bytes = 0;
  char* base = nullptr;
  bool own = false;                  // slab owned by the batch (fock_blocks)
  cudaStream_t pooled = nullptr;     // slab allocated from a memory pool on this stream
  // device descriptors
  ProbDev* d_probs = nullptr;
  std::vector<ProbDev> probs;
  // results gathered into one staging buffer: per problem the word offsets of
  // its eigenvalues, block indices and fail flag (-1: none)
  std::vector<GatherSeg> gseg;
  const GatherSeg* d_gseg = nullptr;
  uint32_t* d_ostage = nullptr;
  size_t ostage_words = 0;
  std::vector<long long> o_ev, o_blk, o_fail;
  std::vector<SegDesc> gsegs, psegs;
  SegDesc *d_gsegs = nullptr, *d_psegs = nullptr;
  std::vector<GramTask> gram; GramTask* d_gram = nullptr;
  // mixed form: the gram tasks' potential contractions as tensor-core split products
  std::vector<SplitTask> splits; SplitTask* d_splits = nullptr; int split_maxm = 0, split_maxn = 0;
  int* d_split_err = nullptr;
  long long o_split_err = -1;
  std::vector<CombineTask> combT, combE; CombineTask *d_combT = nullptr, *d_combE = nullptr;
  std::vector<DefTab> dtabs; DefTab* d_dtabs = nullptr;
  std::vector<DefField> dfields; DefField* d_dfields = nullptr;
  std::vector<DefBlock> dblocks; DefBlock* d_dblocks = nullptr;
  std::vector<DftTask> dft; DftTask* d_dft = nullptr; int maxLdft = 1;
  std::vector<FBlockTask> fbp, fbs; FBlockTask *d_fbp = nullptr, *d_fbs = nullptr;
  std::vector<NullTask> nulls; NullTask* d_nulls = nullptr;   // dependency cut of each periodic problem
  int maxnj_p = 0, maxnj_s = 0, maxm0 = 1;
  std::vector<PrecTask> prec; PrecTask* d_prec = nullptr; int maxM = 0;
  std::vector<CanonTask> canon; CanonTask* d_canon = nullptr; int maxcblk = 0;
  std::vector<FBlockTask> fbo; FBlockTask* d_fbo = nullptr;
  std::vector<SortTask> sorts; SortTask* d_sorts = nullptr; int maxsort = 0;
  std::vector<int> bigsort;          // problems whose eigenvalues need the global sort
  double* sort_pv = nullptr; int* sort_pi = nullptr;
  std::vector<CircDev> circs; CircDev* d_circs = nullptr;
  // per-problem outputs / structured operators
  struct PerProb {
    double* ev = nullptr; int* blk = nullptr; int nev = 0;
    // periodic factors
    double* X[3] = {nullptr, nullptr, nullptr};  // first task's X of each axis (periodic offsets contiguous)
    int ntask_axis[3] = {0, 0, 0};
    cplx* Xh[3] = {nullptr, nullptr, nullptr};
    // structured
    int Lc = 0, M = 0, D = 0, circ = -1;
    double *TH = nullptr, *TS = nullptr;
    int nE = 0;
    std::vector<int> Ek, Em;          // (row cell, column cell) of each boundary block
    // source of each E entry: 0 wall block (gram index Esrc), 1 periodic wrap
    // block (ring offset Esrc), 2 defect block
    std::vector<int> Ekind, Esrc;
    std::vector<double*> ringX;       // periodic chain: forms of each ring offset (or null)
    std::vector<double*> defD1, defD2; // per defect: transverse forms [R][m0^2]
    double *EH = nullptr, *ES = nullptr;
    int *Erows = nullptr, *Erowptr = nullptr, *Ecols = nullptr; int nErows = 0;
    cplx *CH = nullptr, *CS = nullptr, *K = nullptr;
    double *emin = nullptr, *sigma = nullptr;
    bool use_band = false;            // preconditioner: banded Cholesky (else circulant inverse)
    // cell canonical orthogonalisation: transformed operator used by the solver
    double *Xc = nullptr, *THc = nullptr, *TSc = nullptr, *EHc = nullptr, *ESc = nullptr;
    int* kept = nullptr;
    cplx *CHo = nullptr, *CSo = nullptr;   // Fourier blocks of the original operator (matvec API)
    double *band = nullptr, *sigma_band = nullptr;
    int *band_fail = nullptr;
    int* fail = nullptr;
  };
  std::vector<PerProb> pp;
  // LOBPCG state (structured problems)
  struct Lob {
    int n, k, kw, ld3;   // k: block size (wanted kw + guards)
    double *Y, *HY, *SY, *T1, *R, *GH, *GS, *work, *Cc, *Cx, *lam, *res;
    int *active, *fail;
  };
  std::vector<Lob> lob;              // index = structured problem order
  std::vector<int> sidx;             // problem index of each structured problem
  int kmax = 0;
  cplx *mvX = nullptr, *mvY1 = nullptr, *mvY2 = nullptr;   // FFT work (shared by all structured)
  std::vector<size_t> mv_off;        // per structured problem: offset (cplx) into mv buffers
  struct TL {
    void* d = nullptr; int n = 0; int ga = 1, gb = 1, tile = 16;
    // mixed form: the same products of mixed problems as tensor-core split tasks
    void* sd = nullptr; int sn = 0, sm = 1, snn = 1, sks = 1; bool sred = false;
  };
  // basis layout Y = [X | P | W] (k columns each)
  TL fwdXP, fwdW, fwdR, bmulHS2, bmulHS1, bmulK, invHXP, invSXP, invHW, invSW, invPW;
  TL eHXP, eHW;                      // boundary blocks (H and S in one task)
  TL rfwdXP, rinvHXP, rinvSXP, rbmulHS2, reHXP;   // image refresh at the FP32 -> FP64 switch
  TL bandF, bandS;
  int band_stage = 0;                // doubles of a band-solve shared-memory stage
  int band_ringrow = 0;              // largest (D + 1) m0 of the staged band solves
  int gemm_tiles = 0;                // TN tile sizes in use: bit 0 = 16, bit 1 = 20
  bool rr_small = false, rr_big = false;   // Rayleigh-Ritz launches needed (256 / 512 threads)
  int rr_small_ld = 0;               // largest ld of the shared-memory problems
  int rr_big_ld = 0;                 // largest ld of the others
  // the others on thread-block clusters (k_rr_cl) when the plan has no periodic
  // problems; beside periodic problems one CTA each (k_rr), whose narrow launch
  // leaves the other SMs to the periodic pieces (both give the same bits)
  bool rr_cluster = false;
  bool odd_m0 = true;                // some problem has odd m0 (Fourier-block layout, k_fblocks)
  int ptab_maxT = 0, ptab_maxni = 0; // potential tables: largest term count, endpoint count
  TL init, tnCx, nnW, pcG, pcM, pcZ, g1, g3, rr1, rr3, u1, u3, cp2k, resid, normP, normW;
  int fft_cc = 1, fft_chunks = 1;
  int fft_maxcols = 0;               // largest transform column count of a launch
  bool tuned = false;                // fft_cc chosen by the tuner (first execution)
  // the block iteration's body as two CUDA graphs, before and from the
  // Rayleigh-Ritz launch (captured on its second pass, replayed afterwards);
  // graph_failed: capture refused, launches stay eager
  cudaGraphExec_t iter_graph = nullptr, iter_graph_b = nullptr;
  bool graph_failed = false;
  int graph_nodes = 0;
  // periodic Fourier blocks issued in pieces: next local index, piece width
  int pchunk_next = 0, pchunk_w = 0;
  int eapply_gx = 16;
  int* d_ones = nullptr;
  int* d_active = nullptr;
  int* d_mode = nullptr;             // per structured problem: 1 while its matvecs run in FP32
  int* d_refresh = nullptr;          // per structured problem: 0 = refresh its [X | P] images now
  bool any_mixed = false;
  int* d_fail = nullptr;
  double* d_res = nullptr;
  double* d_lam = nullptr;
  // upload slab: parameters and descriptors, staged on the host, one copy
  size_t ubytes = 0;
  char* ubase = nullptr;
  std::vector<char> stage;
};

// Plan everything.  With S.base == nullptr only sizes are computed.
void plan(Batch& B, Slab& S, Slab& U) {
  const int np = B.nprob;
  B.probs.assign(np, ProbDev());
  B.pp.assign(np, Batch::PerProb());
  B.gsegs.clear(); B.psegs.clear(); B.gram.clear(); B.combT.clear(); B.combE.clear();
  B.dtabs.clear(); B.dfields.clear(); B.dblocks.clear();
  B.dft.clear(); B.fbp.clear(); B.fbs.clear(); B.nulls.clear(); B.prec.clear(); B.canon.clear(); B.fbo.clear(); B.maxcblk = 0; B.sorts.clear(); B.bigsort.clear();
  B.circs.clear(); B.lob.clear(); B.sidx.clear(); B.mv_off.clear();
  B.maxnj_p = B.maxnj_s = 0; B.maxm0 = 1; B.maxM = 0; B.maxsort = 0; B.kmax = 0; B.maxLdft = 1;
  B.odd_m0 = false;
  B.any_mixed = false;
  B.band_stage = 0;
  B.band_ringrow = 0;
  B.gemm_tiles = 0;
  B.rr_small = B.rr_big = false;
  B.rr_small_ld = B.rr_big_ld = 0;
  B.rr_cluster = false;
  B.ptab_maxT = 0; B.ptab_maxni = 0;
  size_t zs_total = 0;
  // ---- parameters, vectors, gram tasks ----
  for (int i = 0; i < np; ++i) {
    const HostProb& H = B.hp[i];
    ProbDev& P = B.probs[i];
    Batch::PerProb& Q = B.pp[i];
    P.m0 = H.m0; P.M0 = H.M0; P.R = H.R; P.T = H.T; P.nF = H.nF; P.n0 = H.n0;
    P.b0 = H.b0; P.h = H.h; P.eps = H.eps;
    B.maxm0 = std::max(B.maxm0, H.m0);
    B.odd_m0 = B.odd_m0 || (H.m0 & 1);
    std::vector<double> hpar;
    hpar.insert(hpar.end(), H.alpha.begin(), H.alpha.end());
    hpar.insert(hpar.end(), H.Z.begin(), H.Z.end());
    hpar.insert(hpar.end(), H.frac.begin(), H.frac.end());
    hpar.insert(hpar.end(), H.tq.begin(), H.tq.end());
    hpar.insert(hpar.end(), H.cq.begin(), H.cq.end());
    std::vector<int> hipar(H.ang.begin(), H.ang.end());
    hipar.insert(hipar.end(), H.centre.begin(), H.centre.end());
    const double* par = U.put(hpar);
    const int* ipar = U.put(hipar);
    P.alpha = par; P.Z = par + H.m0; P.frac = P.Z + H.M0; P.tq = P.frac + 3 * H.M0; P.cq = P.tq + H.R;
    P.ang = ipar; P.centre = ipar + H.m0;
    const int m2 = H.m0 * H.m0;
    for (int a = 0; a < 3; ++a) {
      AxisPlan& A = B.ap[i * 3 + a];
      AxisDev& D = P.ax[a];
      D.N = H.N[a]; D.L = H.L[a]; D.per = H.per[a]; D.pad = A.pad;
      D.jlo = A.jlo; D.W = A.W; D.rlo = A.rlo; D.nr = A.nr;
      D.smin = A.jmin; D.slen = A.jmax - A.jmin + 1;
      D.g = S.take<double>((size_t)H.m0 * A.W);
      D.p = S.take<double>((size_t)H.T * A.nr);
      B.gsegs.push_back({i, a, H.m0 * A.W});
      B.psegs.push_back({i, a, H.T * A.nr});
      B.ptab_maxT = std::max(B.ptab_maxT, H.T);
      B.ptab_maxni = std::max(B.ptab_maxni, A.nr + 2 * (H.L[a] == 1 ? 0 : H.L[a] / 2) * H.n0 + 1);
    }
    // gram tasks
    for (int a = 0; a < 3; ++a) {
      AxisPlan& A = B.ap[i * 3 + a];
      const int N = H.N[a], n0 = H.n0, L = H.L[a];
      double* xblock = nullptr;   // periodic axis: factors of all offsets contiguous
      if (H.per[a]) xblock = S.take<double>(A.offs.size() * (size_t)H.nF * m2);
      int nadded = 0;
      auto add = [&](int mode, int ca, int cb, int r0, int r1, int nfold, int foldlo) {
        GramTask t;
        t.prob = i; t.axis = a; t.mode = mode; t.a = ca; t.b = cb; t.rho0 = r0; t.rho1 = r1;
        t.ptab = -1; t.nfold = nfold; t.foldlo = foldlo; t.split = 0;
        t.X = xblock ? xblock + (size_t)(nadded++) * H.nF * m2 : S.take<double>((size_t)H.nF * m2);
        zs_total += (size_t)nfold * m2;
        t.Zs = nullptr;
        B.gram.push_back(t);
        return (int)B.gram.size() - 1;
      };
      if (H.per[a]) {
        Q.ntask_axis[a] = (int)A.offs.size();
        if (a == 0 && H.pchain) Q.ringX.assign(L, nullptr);
        for (size_t o = 0; o < A.offs.size(); ++o) {
          int ti = add(RING, A.offs[o], 0, 0, N, n0, 0);
          if (o == 0) Q.X[a] = B.gram[ti].X;
          if (a == 0 && H.pchain) Q.ringX[A.offs[o]] = B.gram[ti].X;
        }
        if (a == 0 && H.pchain) {
          // periodic chain on the structured path: generators A_d, d <= Dp, as
          // a Toeplitz band plus the wrap-around corner blocks; a chain too
          // short for the two to separate is its whole circulant as Toeplitz
          int Dp = 0;
          for (int d : A.offs) if (2 * d <= L) Dp = std::max(Dp, d);
          Q.Lc = L;
          Q.D = (L > 2 * Dp + 1) ? Dp : L - 1;
          Q.Ek.clear(); Q.Em.clear(); Q.Ekind.clear(); Q.Esrc.clear();
          if (Q.D < L - 1)
            for (int k = 0; k < L; ++k)
              for (int m = 0; m < L; ++m) {
                int dd = posmod_h(k - m, L);
                if (std::abs(k - m) > Q.D && Q.ringX[dd]) {
                  Q.Ek.push_back(k); Q.Em.push_back(m); Q.Ekind.push_back(1); Q.Esrc.push_back(dd);
                }
              }
        }
      } else if (L == 1) {
        int r0 = std::max(-A.pad, A.jlo - 1), r1 = std::min(N - A.pad, A.jlo + A.W + 1);
        int ti = add(WALL, 0, 0, r0, r1, A.nr, A.rlo);
        Q.X[a] = B.gram[ti].X;
        Q.ntask_axis[a] = 1;
      } else {
        // box chain axis (a == 0): Toeplitz generators d = 0..D, then boundary pairs
        int span = A.jmax - A.jmin + 2;
        int D = std::min(span / n0, L - 1);
        Q.Lc = L; Q.D = D;
        for (int d = 0; d <= D; ++d) {
          int lo = std::max(A.jlo, A.jlo + d * n0) - 1, hi = std::min(A.jlo + A.W, A.jlo + A.W + d * n0) + 1;
          int ti = add(VIRT, d, 0, lo, hi, n0, 0);
          if (d == 0) Q.X[a] = B.gram[ti].X;
        }
        Q.ntask_axis[a] = D + 1;
        std::vector<char> aff(L, 0);
        for (int k = 0; k < L; ++k)
          aff[k] = (k * n0 + A.jmin - 2 < 0) || (k * n0 + A.jmax + 2 > L * n0 - 1);
        Q.Ek.clear(); Q.Em.clear(); Q.Ekind.clear(); Q.Esrc.clear();
        for (int k = 0; k < L; ++k)
          for (int m = std::max(0, k - D); m <= std::min(L - 1, k + D); ++m)
            if (aff[k] && aff[m]) {
              if (k > m) {   // E(k, m) = E(m, k)^T: written by the combine task of (m, k)
                Q.Ek.push_back(k); Q.Em.push_back(m); Q.Ekind.push_back(3); Q.Esrc.push_back(-1);
                continue;
              }
              int lo = std::max(A.jlo + k * n0, A.jlo + m * n0) - 1;
              int hi = std::min(A.jlo + A.W + k * n0, A.jlo + A.W + m * n0) + 1;
              lo = std::max(lo, -A.pad); hi = std::min(hi, N - A.pad);
              int ti = add(WALL, k, m, lo, hi, A.nr, A.rlo);
              Q.Ek.push_back(k); Q.Em.push_back(m); Q.Ekind.push_back(0); Q.Esrc.push_back(ti);
            }
      }
    }
  }
  // ---- defects (reading R-DEF): tables, transverse forms, E entries ----
  for (int i = 0; i < np; ++i) {
    const HostProb& H = B.hp[i];
    Batch::PerProb& Q = B.pp[i];
    if (H.defs.empty() && !H.r2) continue;
    const int m2 = H.m0 * H.m0, n0 = H.n0, L = H.L[0];
    const AxisPlan& A0 = B.ap[i * 3 + 0];
    Q.defD1.clear(); Q.defD2.clear();
    std::vector<DefRef> refs;
    // the defects, then (box potential as the plain lattice sum, Sec. 2.3 case
    // (B)) one term per nucleus of the cell: its copies in every cell minus
    // its replicated potential, with the nucleus's charge
    std::vector<fock_defect> terms(H.defs);
    const size_t ndef_real = terms.size();
    if (H.r2)
      for (int nu = 0; nu < H.M0; ++nu) terms.push_back(fock_defect{{0, 0, 0}, nu, 0.0});   // newZ unused here
    for (size_t di = 0; di < terms.size(); ++di) {
      const fock_defect& d = terms[di];
      const bool lsum = di >= ndef_real;
      DefRef rf;
      DefTab t0;
      std::memset(&t0, 0, sizeof(t0));
      t0.prob = i; t0.axis = 0; t0.N = H.N[0]; t0.pad = A0.pad;
      t0.pos = ((double)d.cell[0] + H.frac[d.nucleus * 3 + 0]) * n0;
      t0.e = S.take<double>((size_t)H.R * H.N[0]);
      if (lsum) {
        t0.mode = 1; t0.L = L; t0.nu = d.nucleus; t0.nr = A0.nr; t0.rlo = A0.rlo;
        t0.prep = B.probs[i].ax[0].p;
      }
      B.dtabs.push_back(t0);
      rf.e = t0.e;
      rf.dz = lsum ? H.Z[d.nucleus] : d.newZ - H.Z[d.nucleus];
      for (int a = 1; a <= 2; ++a) {
        const AxisPlan& A = B.ap[i * 3 + a];
        DefTab ta;
        std::memset(&ta, 0, sizeof(ta));
        ta.prob = i; ta.axis = a; ta.N = H.N[a]; ta.pad = A.pad;
        ta.pos = H.frac[d.nucleus * 3 + a] * n0;
        ta.e = S.take<double>((size_t)H.R * H.N[a]);
        B.dtabs.push_back(ta);
        GramTask g;
        g.prob = i; g.axis = a; g.mode = WALL; g.a = 0; g.b = 0;
        g.rho0 = std::max(-A.pad, A.jlo - 1); g.rho1 = std::min(H.N[a] - A.pad, A.jlo + A.W + 1);
        g.ptab = (int)B.dtabs.size() - 1;
        g.nfold = g.rho1 - g.rho0; g.foldlo = g.rho0; g.split = 0;
        g.X = S.take<double>((size_t)H.R * m2);
        g.Zs = nullptr;
        zs_total += (size_t)g.nfold * m2;
        B.gram.push_back(g);
        (a == 1 ? rf.D1 : rf.D2) = g.X;
      }
      refs.push_back(rf);
    }
    DefField f;
    f.prob = i; f.N = H.N[0]; f.ndef = (int)refs.size(); f.refs = U.put(refs);
    f.F = S.take<double>((size_t)H.N[0] * m2);
    B.dfields.push_back(f);
    // a defect block on every pair of cells whose functions overlap
    const bool ring = H.pchain;
    const int span = A0.jmax - A0.jmin + 1;
    for (int k = 0; k < L; ++k)
      for (int m = 0; m < L; ++m) {
        bool pair = ring ? (Q.ringX[posmod_h(k - m, L)] != nullptr) : (std::abs(k - m) <= Q.D);
        if (!pair) continue;
        DefBlock b;
        b.prob = i; b.mode = ring ? RING : WALL; b.a = k; b.b = m; b.F = f.F;
        if (ring) {
          b.pad = 0;
          if (span >= H.N[0]) { b.rho0 = 0; b.rho1 = H.N[0]; }
          else { b.rho0 = k * n0 + A0.jmin; b.rho1 = k * n0 + A0.jmax + 1; }
        } else {
          b.pad = A0.pad;
          b.rho0 = std::max(std::max(A0.jlo + k * n0, A0.jlo + m * n0), -A0.pad);
          b.rho1 = std::min(std::min(A0.jlo + A0.W + k * n0, A0.jlo + A0.W + m * n0), H.N[0] - A0.pad);
        }
        b.outH = b.outS = nullptr;   // set once the E storage exists
        Q.Ek.push_back(k); Q.Em.push_back(m); Q.Ekind.push_back(2); Q.Esrc.push_back((int)B.dblocks.size());
        B.dblocks.push_back(b);
      }
  }
  // E entries grouped by block row (stable: the boundary/wrap block of a position precedes its defect block)
  for (int i = 0; i < np; ++i) {
    Batch::PerProb& Q = B.pp[i];
    const size_t n = Q.Ek.size();
    std::vector<size_t> ord(n);
    for (size_t e = 0; e < n; ++e) ord[e] = e;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
      return Q.Ek[x] != Q.Ek[y] ? Q.Ek[x] < Q.Ek[y] : Q.Em[x] < Q.Em[y];
    });
    std::vector<int> k2(n), m2v(n), kd(n), sr(n);
    for (size_t e = 0; e < n; ++e) { k2[e] = Q.Ek[ord[e]]; m2v[e] = Q.Em[ord[e]]; kd[e] = Q.Ekind[ord[e]]; sr[e] = Q.Esrc[ord[e]]; }
    Q.Ek = k2; Q.Em = m2v; Q.Ekind = kd; Q.Esrc = sr;
    Q.nE = (int)n;
  }
  // fold scratch (shared by all tasks of the batch)
  double* zs = S.take<double>(std::max<size_t>(zs_total, 1));
  {
    size_t o = 0;
    for (auto& t : B.gram) {
      t.Zs = zs + o;
      o += (size_t)t.nfold * B.probs[t.prob].m0 * B.probs[t.prob].m0;
    }
  }
  // mixed form: X_t[mu nu] = sum_r P_t[r] Z[r][mu nu] (T x nfold times nfold x m0^2) on the
  // tensor cores for the gram tasks of mixed problems
  B.splits.clear(); B.split_maxm = B.split_maxn = 0;
  for (auto& t : B.gram) {
    if (!B.hp[t.prob].mixed) continue;
    const ProbDev& P = B.probs[t.prob];
    const AxisDev& A = P.ax[t.axis];
    const bool direct = (t.ptab >= 0);
    const int np = P.m0 * P.m0;
    const double* tab = direct ? B.dtabs[t.ptab].e : A.p;
    const long long ld = direct ? B.dtabs[t.ptab].N : A.nr;
    const long long off = direct ? (t.foldlo + B.dtabs[t.ptab].pad) : (t.foldlo - A.rlo);
    SplitTask sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.M = direct ? P.R : P.T; sp.N = np; sp.K = t.nfold;
    sp.A = tab + off; sp.a_m = ld; sp.a_k = 1;
    sp.B = t.Zs; sp.b_k = np; sp.b_n = 1;
    sp.C = t.X + (direct ? 0 : 2 * np); sp.c_m = np; sp.c_n = 1;
    sp.alpha = 1.0; sp.beta = 0.0;
    B.splits.push_back(sp);
    B.split_maxm = std::max(B.split_maxm, sp.M);
    B.split_maxn = std::max(B.split_maxn, sp.N);
    t.split = 1;
  }
  if (!B.splits.empty()) B.d_split_err = S.take<int>(2);
  // ---- combine, DFT, Fourier blocks, structured operators ----
  for (int i = 0; i < np; ++i) {
    const HostProb& H = B.hp[i];
    Batch::PerProb& Q = B.pp[i];
    const int m2 = H.m0 * H.m0;
    const size_t xs = (size_t)H.nF * m2;
    if (H.kind == 0) {
      int ncell = H.L[0] * H.L[1] * H.L[2];
      for (int a = 0; a < 3; ++a) {
        AxisPlan& A = B.ap[i * 3 + a];
        Q.Xh[a] = S.take<cplx>((size_t)H.L[a] * xs);
        DftTask t;
        t.prob = i; t.L = H.L[a];
        std::vector<int> offs = H.per[a] ? A.offs : std::vector<int>{0};
        t.noff = (int)offs.size();
        t.offs = U.put(offs);
        t.X = Q.X[a]; t.Xh = Q.Xh[a];
        B.dft.push_back(t);
        B.maxLdft = std::max(B.maxLdft, t.L);
      }
      Q.nev = ncell * H.m0;
      Q.ev = S.take<double>(Q.nev);
      Q.blk = S.take<int>(Q.nev);
      Q.fail = S.take<int>(2);   // [0]: a block's Sbar not positive definite; [1]: blocks cut
      FBlockTask f;
      std::memset(&f, 0, sizeof(f));
      f.prob = i; f.source = 0; f.nj = ncell;
      for (int a = 0; a < 3; ++a) { f.L[a] = H.L[a]; f.Xh[a] = Q.Xh[a]; }
      f.want = 1; f.ev = Q.ev; f.blk = Q.blk; f.fail = Q.fail; f.neig = Q.fail + 1;
      NullTask nt;
      std::memset(&nt, 0, sizeof(nt));
      nt.m0 = H.m0; nt.nF = H.nF; nt.nb = ncell * H.m0;
      for (int a = 0; a < 3; ++a) {
        nt.X[a] = Q.X[a];
        nt.noff[a] = H.per[a] ? (int)B.ap[i * 3 + a].offs.size() : 1;
      }
      nt.tau = S.take<double>(1);
      f.tau = nt.tau;
      B.nulls.push_back(nt);
      B.fbp.push_back(f);
      B.maxnj_p = std::max(B.maxnj_p, ncell);
      if (Q.nev <= kSmallSort) {
        B.sorts.push_back({Q.nev, Q.ev, Q.blk});
        B.maxsort = std::max(B.maxsort, Q.nev);
      } else {
        B.bigsort.push_back(i);
      }
    } else {
      // Toeplitz generators and boundary blocks
      Q.TH = S.take<double>((size_t)(Q.D + 1) * m2);
      Q.TS = S.take<double>((size_t)(Q.D + 1) * m2);
      int g0 = -1;
      for (size_t t = 0; t < B.gram.size(); ++t)
        if (B.gram[t].prob == i && B.gram[t].axis == 0) { g0 = (int)t; break; }
      const double* X1 = Q.X[1];
      const double* X2 = Q.X[2];
      for (int d = 0; d <= Q.D; ++d) {
        CombineTask c;
        std::memset(&c, 0, sizeof(c));
        c.prob = i; c.X0 = H.pchain ? Q.ringX[d] : B.gram[g0 + d].X; c.X1 = X1; c.X2 = X2;
        c.outH = Q.TH + (size_t)d * m2; c.outS = Q.TS + (size_t)d * m2;
        B.combT.push_back(c);
      }
      Q.EH = S.take<double>((size_t)std::max(Q.nE, 1) * m2);
      Q.ES = S.take<double>((size_t)std::max(Q.nE, 1) * m2);
      Q.Xc = S.take<double>(m2);
      Q.kept = S.take<int>(1);
      Q.THc = S.take<double>((size_t)(Q.D + 1) * m2);
      Q.TSc = S.take<double>((size_t)(Q.D + 1) * m2);
      Q.EHc = S.take<double>((size_t)std::max(Q.nE, 1) * m2);
      Q.ESc = S.take<double>((size_t)std::max(Q.nE, 1) * m2);
      {
        CanonTask ct;
        ct.m0 = H.m0; ct.D = Q.D; ct.nE = Q.nE; ct.TH = Q.TH; ct.TS = Q.TS; ct.EH = Q.EH; ct.ES = Q.ES;
        ct.Xc = Q.Xc; ct.kept = Q.kept; ct.THc = Q.THc; ct.TSc = Q.TSc; ct.EHc = Q.EHc; ct.ESc = Q.ESc;
        ct.ring_full = (H.pchain && Q.D == Q.Lc - 1) ? 1 : 0;
        ct.nb = Q.Lc * H.m0;
        // transposed partner of each boundary block: itself on the diagonal;
        // else the entry at the mirrored position of the same kind and the
        // same rank among that position's entries (a position can hold a
        // wall block and a defect block)
        std::vector<int> part(std::max(Q.nE, 1), -1);
        {
          // entries are grouped by (row cell, column cell): index the groups
          std::vector<std::pair<long long, int>> key(Q.nE);
          for (int e = 0; e < Q.nE; ++e) key[e] = {(long long)Q.Ek[e] * (Q.Lc + 1) + Q.Em[e], e};
          std::sort(key.begin(), key.end());
          std::vector<int> rank(std::max(Q.nE, 1), 0);
          for (int a = 1; a < Q.nE; ++a)
            if (key[a].first == key[a - 1].first) rank[key[a].second] = rank[key[a - 1].second] + 1;
          for (int e = 0; e < Q.nE; ++e) {
            if (Q.Ek[e] == Q.Em[e]) { part[e] = e; continue; }
            const long long want = (long long)Q.Em[e] * (Q.Lc + 1) + Q.Ek[e];
            auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(want, -1));
            it += rank[e];
            // kinds must match (a wall block and its mirror entry, kind 3, count as one kind)
            auto base = [](int kd) { return kd == 3 ? 0 : kd; };
            if (it < key.end() && it->first == want && base(Q.Ekind[it->second]) == base(Q.Ekind[e]))
              part[e] = it->second;
          }
        }
        for (int e = 0; e < Q.nE; ++e)   // pairs must be mutual
          if (part[e] >= 0 && part[part[e]] != e) part[e] = -1;
        ct.Epart = U.put(part);
        B.canon.push_back(ct);
        B.maxcblk = std::max(B.maxcblk, 2 * (Q.D + 1) + 2 * Q.nE);
      }
      // mirror entries (kind 3) of the wall blocks, by position
      std::vector<std::pair<long long, int>> mirror;
      for (int e = 0; e < Q.nE; ++e)
        if (Q.Ekind[e] == 3) mirror.push_back({(long long)Q.Ek[e] * (Q.Lc + 1) + Q.Em[e], e});
      std::sort(mirror.begin(), mirror.end());
      for (int e = 0; e < Q.nE; ++e) {
        int k = Q.Ek[e], m = Q.Em[e], d = std::abs(k - m);
        if (Q.Ekind[e] == 3) continue;   // written transposed by the (m, k) wall block's combine task
        if (Q.Ekind[e] == 2) {   // defect block: written by k_defect_blocks
          B.dblocks[Q.Esrc[e]].outH = Q.EH + (size_t)e * m2;
          B.dblocks[Q.Esrc[e]].outS = Q.ES + (size_t)e * m2;
          continue;
        }
        CombineTask c;
        std::memset(&c, 0, sizeof(c));
        c.prob = i; c.X1 = X1; c.X2 = X2;
        if (Q.Ekind[e] == 0) {   // wall block: the block minus its Toeplitz generator
          c.X0 = B.gram[Q.Esrc[e]].X;
          c.subH = Q.TH + (size_t)d * m2; c.subS = Q.TS + (size_t)d * m2; c.subT = (k < m);
          if (k < m) {
            auto it = std::lower_bound(mirror.begin(), mirror.end(),
                                       std::make_pair((long long)m * (Q.Lc + 1) + k, -1));
            if (it != mirror.end() && it->first == (long long)m * (Q.Lc + 1) + k) {
              c.outHT = Q.EH + (size_t)it->second * m2;
              c.outST = Q.ES + (size_t)it->second * m2;
            }
          }
        } else {                 // wrap-around block of a periodic chain: A_{(k-m) mod L}
          c.X0 = Q.ringX[Q.Esrc[e]];
        }
        c.outH = Q.EH + (size_t)e * m2; c.outS = Q.ES + (size_t)e * m2;
        B.combE.push_back(c);
      }
      // CSR over block rows (the entries are already grouped by row k ascending)
      std::vector<int> rows, rowptr, cols;
      for (int e = 0; e < Q.nE; ++e) {
        if (rows.empty() || rows.back() != Q.Ek[e]) { rows.push_back(Q.Ek[e]); rowptr.push_back(e); }
        cols.push_back(Q.Em[e]);
      }
      rowptr.push_back(Q.nE);
      Q.nErows = (int)rows.size();
      Q.Erows = U.put(rows);
      Q.Erowptr = U.put(rowptr);
      Q.Ecols = U.put(cols);
      // circulant embedding
      Q.M = smooth_at_least(Q.Lc + Q.D);
      CircDev cd;
      std::memset(&cd, 0, sizeof(cd));
      cd.M = Q.M;
      std::vector<int> f = radix_factors(Q.M);
      cd.nfac = (int)f.size();
      for (int q = 0; q < cd.nfac; ++q) cd.fac[q] = f[q];
      cd.tw = S.take<cplx>(Q.M);
      Q.circ = (int)B.circs.size();
      B.circs.push_back(cd);
      B.maxM = std::max(B.maxM, Q.M);
      Q.CH = S.take<cplx>((size_t)Q.M * m2);
      Q.CS = S.take<cplx>((size_t)Q.M * m2);
      Q.CHo = S.take<cplx>((size_t)Q.M * m2);
      Q.CSo = S.take<cplx>((size_t)Q.M * m2);
      Q.K = S.take<cplx>((size_t)Q.M * m2);
      Q.emin = S.take<double>(Q.M);
      Q.sigma = S.take<double>(1);
      // banded Cholesky of H - sigma S when its one-CTA factorisation stays
      // within ~4 GFLOP (tens of ms); above that the circulant inverse
      Q.use_band = 2.0 * Q.Lc * (double)Q.D * Q.D * (double)H.m0 * H.m0 * H.m0 <= 4e9;
      if (Q.use_band) {
        Q.band = S.take<double>((size_t)Q.Lc * (Q.D + 1) * m2);
        Q.sigma_band = S.take<double>(1);
        Q.band_fail = S.take<int>(1);
      }
      Q.fail = S.take<int>(1);
      FBlockTask fb;
      std::memset(&fb, 0, sizeof(fb));
      fb.prob = i; fb.source = 1; fb.nj = Q.M; fb.M = Q.M; fb.D = Q.D; fb.TH = Q.THc; fb.TS = Q.TSc;
      fb.outH = Q.CH; fb.outS = Q.CS; fb.want = 2; fb.ev = Q.emin; fb.fail = Q.fail;
      B.fbs.push_back(fb);
      FBlockTask fo = fb;   // the original operator's blocks, for the matvec entry points
      fo.TH = Q.TH; fo.TS = Q.TS; fo.outH = Q.CHo; fo.outS = Q.CSo; fo.want = 0; fo.ev = nullptr;
      B.fbo.push_back(fo);
      B.maxnj_s = std::max(B.maxnj_s, Q.M);
      PrecTask pt;
      pt.prob = i; pt.M = Q.M; pt.emin = Q.emin; pt.sigma = Q.sigma; pt.CH = Q.CH; pt.CS = Q.CS; pt.K = Q.K;
      pt.rel_shift = kPrecShift;
      B.prec.push_back(pt);
      Q.nev = H.k_eig;
      Q.ev = S.take<double>(Q.nev);
      B.sidx.push_back(i);
      B.kmax = std::max(B.kmax, lobpcg_block(H.k_eig, Q.Lc * H.m0));
    }
  }
  // ---- LOBPCG state ----
  size_t mv_total = 0;
  for (size_t s = 0; s < B.sidx.size(); ++s) {
    int i = B.sidx[s];
    const HostProb& H = B.hp[i];
    Batch::PerProb& Q = B.pp[i];
    Batch::Lob l;
    l.n = Q.Lc * H.m0; l.kw = H.k_eig; l.k = lobpcg_block(H.k_eig, l.n);
    l.ld3 = 3 * l.k + 1;   // +1: Jacobi pads odd sizes
    size_t nk = (size_t)l.n * l.k;
    l.Y = S.take<double>(3 * nk); l.HY = S.take<double>(3 * nk); l.SY = S.take<double>(3 * nk);
    l.T1 = S.take<double>(2 * nk);
    l.R = S.take<double>(nk);
    l.GH = S.take<double>((size_t)l.ld3 * l.ld3); l.GS = S.take<double>((size_t)l.ld3 * l.ld3);
    l.work = S.take<double>((size_t)7 * l.ld3 * l.ld3);
    l.Cc = S.take<double>((size_t)l.ld3 * 2 * l.k);
    l.Cx = S.take<double>((size_t)l.k * l.k);
    B.lob.push_back(l);
    B.mv_off.push_back(mv_total);
    mv_total += (size_t)Q.M * H.m0 * 2 * l.k;   // matvecs of up to 2k columns
  }
  if (!B.sidx.empty()) {
    const int ns = (int)B.sidx.size();
    B.d_active = S.take<int>(ns);
    B.d_mode = S.take<int>(ns);
    B.d_refresh = S.take<int>(ns);
    B.d_fail = S.take<int>(ns);
    B.d_res = S.take<double>((size_t)ns * B.kmax);
    B.d_lam = S.take<double>((size_t)ns * B.kmax);
    for (int s = 0; s < ns; ++s) {
      B.lob[s].active = B.d_active + s;
      B.lob[s].fail = B.d_fail + s;
      B.lob[s].res = B.d_res + (size_t)s * B.kmax;
      B.lob[s].lam = B.d_lam + (size_t)s * B.kmax;
    }
    B.mvX = S.take<cplx>(mv_total);
    B.mvY1 = S.take<cplx>(mv_total);
    B.mvY2 = S.take<cplx>(mv_total);
  }
  if (!B.bigsort.empty()) {
    int mx = 0;
    for (int i : B.bigsort) mx = std::max(mx, B.pp[i].nev);
    int n2 = 1;
    while (n2 < mx) n2 <<= 1;
    B.sort_pv = S.take<double>(n2);
    B.sort_pi = S.take<int>(n2);
  }
  B.d_circs = U.put(B.circs);
  // ---- LOBPCG task lists (fixed addresses, built once) ----
  if (!B.sidx.empty()) {
    const int ns = (int)B.sidx.size();
    B.fft_cc = std::max(1, std::min(16, 98304 / (32 * std::max(B.maxM, 1))));
    int maxcols = 1;
    std::vector<FftTask> fXP, fW, fR, iHXP, iSXP, iHW, iSW, iPW;
    std::vector<BmulTask> bHS2, bHS1, bK;
    std::vector<EApplyTask> ehxp, ehw, rehxp;
    std::vector<FftTask> rfXP, riHXP, riSXP;
    std::vector<BmulTask> rbHS2;
    std::vector<InitTask> ini;
    std::vector<GemmTask> tcx, nw, pcg, pcm, pcz, gg1, gg3, uu1, uu3;
    std::vector<SplitTask> s_tcx, s_nw, s_gg1, s_gg3, s_uu1, s_uu3;
    std::vector<RRTask> r1, r3;
    std::vector<CopyTask> c2k, nP, nW;
    std::vector<ResidTask> rs;
    std::vector<BandTask> bnd;
    std::vector<int> ones(ns, 1);
    B.d_ones = U.put(ones);
    for (int s2 = 0; s2 < ns; ++s2) {
      const int i = B.sidx[s2];
      const HostProb& H = B.hp[i];
      Batch::PerProb& Q = B.pp[i];
      Batch::Lob& l = B.lob[s2];
      const int n = l.n, k = l.k, m0 = H.m0, ld3 = l.ld3;
      const size_t nk = (size_t)n * k;
      maxcols = std::max(maxcols, m0 * k);   // packed: two real columns per transform
      B.eapply_gx = std::max(B.eapply_gx, eapply_grid((long long)Q.nErows * m0 * 2 * k));
      cplx* X = B.mvX + B.mv_off[s2];
      cplx* Y1 = B.mvY1 + B.mv_off[s2];
      cplx* Y2 = B.mvY2 + B.mv_off[s2];
      const CircDev* cd = B.d_circs + Q.circ;
      // precision of the operator matvecs: the problem's current mode (mixed
      // form) or FP64; the circulant preconditioner of a mixed problem is FP32
      const int* opmode = H.f32 ? B.d_mode + s2 : nullptr;
      const int* pcmode = H.f32 ? B.d_ones + s2 : nullptr;
      if (H.f32) B.any_mixed = true;
      auto fwd = [&](const double* src, int ncol, const int* md) {
        FftTask t; std::memset(&t, 0, sizeof(t));
        t.prob = i; t.L = Q.Lc; t.m0 = m0; t.ncol = ncol; t.circ = cd; t.x = src; t.ldx = n; t.X = X;
        t.cc = B.fft_cc; t.mode = md; t.active = l.active;   // converged problems: no more matvecs
        return t;
      };
      auto inv = [&](cplx* from, double* dst, int ncol, const int* md) {
        FftTask t; std::memset(&t, 0, sizeof(t));
        t.prob = i; t.L = Q.Lc; t.m0 = m0; t.ncol = ncol; t.circ = cd; t.X = from; t.y = dst; t.ldy = n;
        t.beta = 0.0; t.cc = B.fft_cc; t.mode = md; t.active = l.active;
        return t;
      };
      double* Yx = l.Y;            // X: columns [0, k)
      double* Yw = l.Y + 2 * nk;   // W: columns [2k, 3k)
      fXP.push_back(fwd(Yx, 2 * k, opmode)); fW.push_back(fwd(Yw, k, opmode));
      iHXP.push_back(inv(Y1, l.HY, 2 * k, opmode)); iSXP.push_back(inv(Y2, l.SY, 2 * k, opmode));
      iHW.push_back(inv(Y1, l.HY + 2 * nk, k, opmode)); iSW.push_back(inv(Y2, l.SY + 2 * nk, k, opmode));
      bHS2.push_back({i, Q.M, m0, 2 * k, Q.CH, Q.CS, X, Y1, Y2, opmode, l.active});
      bHS1.push_back({i, Q.M, m0, k, Q.CH, Q.CS, X, Y1, Y2, opmode, l.active});
      if (Q.use_band) {
        BandTask bt;
        std::memset(&bt, 0, sizeof(bt));
        bt.m0 = m0; bt.L = Q.Lc; bt.D = Q.D; bt.k = k; bt.n = n;
        bt.TH = Q.THc; bt.TS = Q.TSc; bt.nE = Q.nE; bt.Ek = U.put(Q.Ek); bt.Em = U.put(Q.Em);
        bt.EH = Q.EHc; bt.ES = Q.ESc; bt.sigma0 = Q.sigma; bt.band = Q.band; bt.sigma_used = Q.sigma_band;
        bt.fail = Q.band_fail; bt.R = l.R; bt.W = Yw; bt.ld = n; bt.active = l.active;
        bt.fp32 = H.f32;
        bnd.push_back(bt);
        if (m0 % 2 == 0 && (Q.D + 1) * m0 * m0 <= band_stage_doubles(1 << 30)) {   // stageable
          B.band_stage = std::max(B.band_stage, (Q.D + 1) * m0 * m0);
          B.band_ringrow = std::max(B.band_ringrow, (Q.D + 1) * m0);
        }
      } else {
        fR.push_back(fwd(l.R, k, pcmode));
        iPW.push_back(inv(Y1, Yw, k, pcmode));
        bK.push_back({i, Q.M, m0, k, Q.K, nullptr, X, Y1, nullptr, pcmode, l.active});
      }
      auto ea = [&](const double* vals, const double* x, double* y, int ncol, const int* md) {
        EApplyTask t;
        std::memset(&t, 0, sizeof(t));
        t.prob = i; t.m0 = m0; t.ncol = ncol; t.nrows = Q.nErows; t.rows = Q.Erows; t.rowptr = Q.Erowptr;
        t.cols = Q.Ecols; t.vals = vals; t.x = x; t.ldx = n; t.y = y; t.ldy = n; t.mode = md; t.active = l.active;
        return t;
      };
      if (Q.nE) {
        // H and S boundary blocks applied to the same columns in one task
        auto hs = [](EApplyTask t, const double* v2, double* y2) { t.vals2 = v2; t.y2 = y2; return t; };
        ehxp.push_back(hs(ea(Q.EHc, Yx, l.HY, 2 * k, nullptr), Q.ESc, l.SY));
        ehw.push_back(hs(ea(Q.EHc, Yw, l.HY + 2 * nk, k, nullptr), Q.ESc, l.SY + 2 * nk));
      }
      // image refresh of [X | P] for the problems whose matvecs just switched to
      // FP64 (flag 0 = refresh, 2 = leave: matches neither precision variant)
      if (H.f32) {
        const int* rf = B.d_refresh + s2;
        rfXP.push_back(fwd(Yx, 2 * k, rf));
        riHXP.push_back(inv(Y1, l.HY, 2 * k, rf)); riSXP.push_back(inv(Y2, l.SY, 2 * k, rf));
        rbHS2.push_back({i, Q.M, m0, 2 * k, Q.CH, Q.CS, X, Y1, Y2, rf, l.active});
        if (Q.nE) {
          EApplyTask t2 = ea(Q.EHc, Yx, l.HY, 2 * k, rf);
          t2.vals2 = Q.ESc; t2.y2 = l.SY;
          rehxp.push_back(t2);
        }
      }
      ini.push_back({n, k, n, problem_seed(H), l.Y});   // start depends on the problem only
      auto gt = [&](int a, int b, const double* A, int lda, const double* Bm, int ldb, double* C, int ldc,
                    double alpha, double beta) {
        GemmTask g; g.active = l.active; g.n = n; g.a = a; g.b = b; g.A = A; g.lda = lda; g.B = Bm; g.ldb = ldb;
        g.C = C; g.ldc = ldc; g.alpha = alpha; g.beta = beta; g.sym = 0; g.split = 0;
        g.tile = (k % 20 == 0) ? 20 : 16;   // a property of the problem alone
        B.gemm_tiles |= (g.tile == 20) ? 2 : 1;
        return g;
      };
      // W made S-orthogonal to X before its images are formed:  C = (S X)^T W,
      // W -= X C (the images of the projected vectors are then fresh)
      tcx.push_back(gt(k, k, l.SY, n, Yw, n, l.Cx, k, 1.0, 0.0));
      nw.push_back(gt(k, k, l.Y, n, l.Cx, k, l.Y + 2 * nk, n, -1.0, 1.0));
      // P' made S-orthogonal to X' in the coefficients, before [X' | P'] = Y Cc is
      // formed: with z_X, z_P the two column blocks of Cc and G_S = Y^T S Y,
      // z_P -= z_X (z_X^T G_S z_P).  The images of [X' | P'] are computed fresh
      // afterwards, so they match P' however much the projection cancels (images
      // updated by linearity after a projection lose their relative accuracy in
      // the directions it cancels, and the Rayleigh-Ritz step amplifies that)
      {
        auto small = [&](GemmTask g, int rows) { g.n = rows; return g; };
        double* zX = l.Cc;
        double* zP = l.Cc + (size_t)ld3 * k;
        pcg.push_back(small(gt(3 * k, k, l.GS, ld3, zP, ld3, l.work, ld3, 1.0, 0.0), 3 * k));   // G_S z_P
        pcm.push_back(small(gt(k, k, zX, ld3, l.work, ld3, l.Cx, k, 1.0, 0.0), 3 * k));        // z_X^T (G_S z_P)
        pcz.push_back(small(gt(k, k, zX, ld3, l.Cx, k, zP, ld3, -1.0, 1.0), 3 * k));          // z_P -= z_X M
      }
      // Gram matrices Y^T H Y, Y^T S Y: symmetric, upper tiles only
      auto sym = [](GemmTask g) { g.sym = 1; return g; };
      gg1.push_back(sym(gt(k, k, l.Y, n, l.HY, n, l.GH, ld3, 1.0, 0.0)));
      gg1.push_back(sym(gt(k, k, l.Y, n, l.SY, n, l.GS, ld3, 1.0, 0.0)));
      gg3.push_back(sym(gt(3 * k, 3 * k, l.Y, n, l.HY, n, l.GH, ld3, 1.0, 0.0)));
      gg3.push_back(sym(gt(3 * k, 3 * k, l.Y, n, l.SY, n, l.GS, ld3, 1.0, 0.0)));
      const int big = (3 * (size_t)ld3 * ld3 * sizeof(double) > kRRSmemCap) ? 1 : 0;
      r1.push_back({l.active, k, k, ld3, l.GH, l.GS, l.work, l.lam, l.Cc, l.fail, opmode, big});
      r3.push_back({l.active, 3 * k, k, ld3, l.GH, l.GS, l.work, l.lam, l.Cc, l.fail, opmode, big});
      B.rr_small = B.rr_small || !big;
      B.rr_big = B.rr_big || big;
      if (!big) B.rr_small_ld = std::max(B.rr_small_ld, ld3);
      else B.rr_big_ld = std::max(B.rr_big_ld, ld3);
      // [X' | P'] = Y[:, :nb] Cc, then copied over [X | P]; images recomputed by a matvec
      uu1.push_back(gt(k, 2 * k, l.Y, n, l.Cc, ld3, l.T1, n, 1.0, 0.0));
      uu3.push_back(gt(3 * k, 2 * k, l.Y, n, l.Cc, ld3, l.T1, n, 1.0, 0.0));
      c2k.push_back({l.active, n, 2 * k, l.T1, n, l.Y, n});
      nP.push_back({l.active, n, k, nullptr, n, l.Y + nk, n});
      nW.push_back({l.active, n, k, nullptr, n, l.Y + 2 * nk, n});
      rs.push_back({l.active, n, k, n, l.Y, l.HY, l.SY, l.lam, l.R, l.res});
      if (H.mixed && n >= kSplitMinRows) {
        // mixed form: the block iteration's dense products on the tensor cores
        // (exact split products; the Gram sums over n split into K ranges)
        auto to_tn = [&](GemmTask& g, std::vector<SplitTask>& out) {
          SplitTask t;
          std::memset(&t, 0, sizeof(t));
          t.active = g.active; t.M = g.a; t.N = g.b; t.K = g.n;
          t.A = g.A; t.a_m = g.lda; t.a_k = 1; t.B = g.B; t.b_k = 1; t.b_n = g.ldb;
          t.C = g.C; t.c_m = 1; t.c_n = g.ldc; t.alpha = g.alpha; t.beta = g.beta;
          t.ksplit = std::min(32, std::max(1, ((t.K + 63) / 64 + 7) / 8));
          t.work = S.take<double>((size_t)t.ksplit * t.M * t.N);
          t.sym = g.sym;
          out.push_back(t);
          g.split = 1;
        };
        auto to_nn = [&](GemmTask& g, std::vector<SplitTask>& out) {
          SplitTask t;
          std::memset(&t, 0, sizeof(t));
          t.active = g.active; t.M = g.n; t.N = g.b; t.K = g.a;
          t.A = g.A; t.a_m = 1; t.a_k = g.lda; t.B = g.B; t.b_k = 1; t.b_n = g.ldb;
          t.C = g.C; t.c_m = 1; t.c_n = g.ldc; t.alpha = g.alpha; t.beta = g.beta;
          t.ksplit = 1; t.work = nullptr; t.sym = 0;
          out.push_back(t);
          g.split = 1;
        };
        to_tn(tcx.back(), s_tcx);
        to_nn(nw.back(), s_nw);
        to_tn(gg1[gg1.size() - 2], s_gg1); to_tn(gg1.back(), s_gg1);
        to_tn(gg3[gg3.size() - 2], s_gg3); to_tn(gg3.back(), s_gg3);
        to_nn(uu1.back(), s_uu1); to_nn(uu3.back(), s_uu3);
      }
    }
    B.fft_chunks = (maxcols + B.fft_cc - 1) / B.fft_cc;
    B.fft_maxcols = maxcols;
    auto TLp = [&](auto& v, Batch::TL& tl, int ga = 1, int gb = 1) {
      tl.d = (void*)U.put(v); tl.n = (int)v.size(); tl.ga = ga; tl.gb = gb;
    };
    const int kk = B.kmax;
    int maxld3 = 0;
    for (auto& l : B.lob) maxld3 = std::max(maxld3, l.ld3);
    TLp(fXP, B.fwdXP); TLp(fW, B.fwdW); TLp(fR, B.fwdR);
    TLp(iHXP, B.invHXP); TLp(iSXP, B.invSXP); TLp(iHW, B.invHW); TLp(iSW, B.invSW); TLp(iPW, B.invPW);
    TLp(bHS2, B.bmulHS2); TLp(bHS1, B.bmulHS1); TLp(bK, B.bmulK);
    TLp(ehxp, B.eHXP); TLp(ehw, B.eHW);
    TLp(rfXP, B.rfwdXP); TLp(riHXP, B.rinvHXP); TLp(riSXP, B.rinvSXP); TLp(rbHS2, B.rbmulHS2);
    TLp(rehxp, B.reHXP);
    TLp(ini, B.init);
    // TN products: ga, gb carry the largest output dimensions (tiles per launch)
    TLp(tcx, B.tnCx, kk, kk);
    TLp(nw, B.nnW);
    TLp(pcg, B.pcG); TLp(pcm, B.pcM, kk, kk); TLp(pcz, B.pcZ);
    TLp(gg1, B.g1, kk, kk);
    TLp(gg3, B.g3, 3 * kk, 3 * kk);
    B.tnCx.tile = B.pcM.tile = B.g1.tile = B.g3.tile = B.gemm_tiles;
    TLp(r1, B.rr1, maxld3); TLp(r3, B.rr3, maxld3);
    B.rr_cluster = B.fbp.empty();   // the periodic tasks are planned by now
    TLp(uu1, B.u1); TLp(uu3, B.u3);
    auto TLs = [&](std::vector<SplitTask>& v, Batch::TL& tl) {
      tl.sd = (void*)U.put(v); tl.sn = (int)v.size();
      tl.sm = tl.snn = tl.sks = 1; tl.sred = false;
      for (const SplitTask& t : v) {
        tl.sm = std::max(tl.sm, t.M); tl.snn = std::max(tl.snn, t.N); tl.sks = std::max(tl.sks, t.ksplit);
        tl.sred = tl.sred || t.work != nullptr;
      }
      while (tl.sn * tl.sks > 65535 && tl.sks > 1) tl.sks /= 2;   // grid z limit (tasks x K ranges)
    };
    TLs(s_tcx, B.tnCx); TLs(s_nw, B.nnW);
    TLs(s_gg1, B.g1); TLs(s_gg3, B.g3); TLs(s_uu1, B.u1); TLs(s_uu3, B.u3);
    TLp(c2k, B.cp2k);
    TLp(nP, B.normP);
    TLp(nW, B.normW);
    TLp(bnd, B.bandF);
    B.bandS = B.bandF;
    B.band_stage = band_stage_doubles(B.band_stage);
    TLp(rs, B.resid, kk);
  }
  // ---- descriptor arrays (uploaded in one copy with the parameters) ----
  B.d_probs = U.put(B.probs);
  B.d_gsegs = U.put(B.gsegs);
  B.d_psegs = U.put(B.psegs);
  B.d_gram = U.put(B.gram);
  B.d_splits = U.put(B.splits);
  B.d_combT = U.put(B.combT);
  B.d_combE = U.put(B.combE);
  B.d_dtabs = U.put(B.dtabs);
  B.d_dfields = U.put(B.dfields);
  B.d_dblocks = U.put(B.dblocks);
  B.d_dft = U.put(B.dft);
  B.d_fbp = U.put(B.fbp);
  B.d_fbs = U.put(B.fbs);
  B.d_nulls = U.put(B.nulls);
  B.d_prec = U.put(B.prec);
  B.d_canon = U.put(B.canon);
  B.d_fbo = U.put(B.fbo);
  B.d_sorts = U.put(B.sorts);
  // ---- result gather: eigenvalues, block indices and fail flags of every problem ----
  B.gseg.clear();
  B.o_ev.assign(np, -1); B.o_blk.assign(np, -1); B.o_fail.assign(np, -1);
  {
    size_t w = 0;
    auto seg = [&](const void* src, size_t words) {
      B.gseg.push_back({reinterpret_cast<const uint32_t*>(src), (unsigned int)words, (unsigned int)w});
      const long long off = (long long)w;
      w += (words + 1) & ~(size_t)1;   // 8-byte aligned starts
      return off;
    };
    for (int i = 0; i < np; ++i) {
      const Batch::PerProb& Q = B.pp[i];
      if (B.hp[i].kind == 0) {
        B.o_ev[i] = seg(Q.ev, 2 * (size_t)Q.nev);
        B.o_blk[i] = seg(Q.blk, (size_t)Q.nev);
        B.o_fail[i] = seg(Q.fail, 1);
      }
    }
    for (size_t s2 = 0; s2 < B.sidx.size(); ++s2) {
      const int i = B.sidx[s2];
      B.o_ev[i] = seg(B.lob[s2].lam, 2 * (size_t)B.pp[i].nev);
    }
    B.o_split_err = B.d_split_err ? seg(B.d_split_err, 1) : -1;
    B.ostage_words = w;
    B.d_ostage = S.take<uint32_t>(std::max<size_t>(w, 2));
    B.d_gseg = U.put(B.gseg);
  }
  B.bytes = S.off;
  B.ubytes = U.off;
}

}  // namespace

// ------------------------------------------------------------------ drivers
namespace {

int alloc_and_plan(fock_ctx* ctx, Batch& B, bool own) {
  Slab S0, U0;
  plan(B, S0, U0);
  size_t need = S0.off + 256, uneed = U0.off + 256;
  if (ctx->budget && need + uneed > ctx->budget)
    return set_err(ctx, FOCK_ENOMEM, "batch needs " + std::to_string(need + uneed) + " bytes, budget " +
                                         std::to_string(ctx->budget));
  char *mb = nullptr, *ub = nullptr;
  if (ctx->mempool) {
    CUDA_TRY(ctx, cudaMallocFromPoolAsync((void**)&mb, need, ctx->mempool, ctx->stream));
    CUDA_TRY(ctx, cudaMallocFromPoolAsync((void**)&ub, uneed, ctx->mempool, ctx->stream));
    B.pooled = ctx->stream;
  } else if (own) {
    CUDA_TRY(ctx, cudaMalloc(&mb, need));
    CUDA_TRY(ctx, cudaMalloc(&ub, uneed));
    B.own = true;
  } else {
    if (ctx->arena_cap < need + uneed) {
      if (ctx->arena) { cudaStreamSynchronize(ctx->stream); cudaFree(ctx->arena); ctx->arena = nullptr; ctx->arena_cap = 0; }
      size_t cap = (need + uneed) + (need + uneed) / 4;
      CUDA_TRY(ctx, cudaMalloc(&ctx->arena, cap));
      ctx->arena_cap = cap;
    }
    mb = ctx->arena;
    ub = ctx->arena + ((need + 255) & ~(size_t)255);
  }
  B.base = mb;
  B.ubase = ub;
  Slab S, U;
  S.base = mb;
  U.base = ub;
  B.stage.assign(U0.off + 16, 0);
  U.stage = &B.stage;
  plan(B, S, U);
  CUDA_TRY(ctx, cudaMemcpyAsync(ub, B.stage.data(), U.off, cudaMemcpyHostToDevice, ctx->stream));
  return FOCK_OK;
}

void free_batch(Batch& B) {
  if (B.iter_graph) cudaGraphExecDestroy(B.iter_graph);
  if (B.iter_graph_b) cudaGraphExecDestroy(B.iter_graph_b);
  B.iter_graph = B.iter_graph_b = nullptr;
  if (B.pooled) {
    cudaFreeAsync(B.base, B.pooled);
    cudaFreeAsync(B.ubase, B.pooled);
  } else if (B.own) {
    cudaFree(B.base);
    cudaFree(B.ubase);
  }
  B.base = B.ubase = nullptr;
}

int build_batch(fock_ctx* ctx, int nprob, const fock_problem* probs, Batch& B, bool own) {
  if (nprob <= 0 || !probs) return set_err(ctx, FOCK_EINVAL, "no problems");
  B.nprob = nprob;
  B.hp.assign(nprob, HostProb());
  B.ap.assign((size_t)nprob * 3, AxisPlan());
  for (int i = 0; i < nprob; ++i) {
    std::string why;
    int rc = validate(probs[i], B.hp[i], why);
    if (rc) return set_err(ctx, rc, "problem " + std::to_string(i) + ": " + why);
    for (int a = 0; a < 3; ++a) axis_plan(B.hp[i], a, B.ap[i * 3 + a]);
  }
  return alloc_and_plan(ctx, B, own);
}

void run_assemble(fock_ctx* ctx, Batch& B) {
  cudaStream_t st = ctx->stream;
  { PROF("k_vec1d", 2); launch_vec1d(B.d_probs, B.d_gsegs, (int)B.gsegs.size(), B.d_psegs, (int)B.psegs.size(),
                                     B.d_dtabs, (int)B.dtabs.size(), B.ptab_maxT, B.ptab_maxni, st); }
  { PROF("k_gram", 2); launch_gram(B.d_probs, B.d_gram, (int)B.gram.size(), B.d_dtabs, st); }
  if (!B.splits.empty()) {
    cudaMemsetAsync(B.d_split_err, 0, sizeof(int), st);
    PROF("k_split_gemm", 1);
    launch_split_gemm(B.d_splits, (int)B.splits.size(), B.split_maxm, B.split_maxn, B.d_split_err, st);
  }
  if (!B.combT.empty()) { PROF("k_combine", 2);
    launch_combine(B.d_probs, B.d_combT, (int)B.combT.size(), st);
    launch_combine(B.d_probs, B.d_combE, (int)B.combE.size(), st); }
  if (!B.dfields.empty()) { PROF("k_defects", 2);
    launch_defects(B.d_probs, B.d_dfields, (int)B.dfields.size(), B.d_dblocks, (int)B.dblocks.size(), st); }
}

void zero_fail_flags(Batch& B, int kind, cudaStream_t st) {
  // periodic problems: the flag and the count of blocks taking the eigendecomposition route
  for (int i = 0; i < B.nprob; ++i)
    if (B.hp[i].kind == kind && B.pp[i].fail)
      cudaMemsetAsync(B.pp[i].fail, 0, (kind == 0 ? 2 : 1) * sizeof(int), st);
}

// Periodic problems: per-axis DFTs and the dependency cuts (head), the
// Fourier-block eigensolves (in pieces of local indices when they share the
// GPU with a block iteration), then the sort of each spectrum (tail).
void run_periodic_head(fock_ctx* ctx, Batch& B, cudaStream_t st) {
  B.pchunk_next = 0;
  if (B.fbp.empty()) return;
  zero_fail_flags(B, 0, st);
  { PROF("k_axis_dft", 1); launch_axis_dft(B.d_probs, B.d_dft, (int)B.dft.size(), B.maxLdft, st); }
  { PROF("k_null_tau", 1); launch_null_tau(B.d_nulls, (int)B.nulls.size(), st); }
}
// the next nx local indices of every periodic task (nx < 0: all that remain)
void run_periodic_piece(fock_ctx* ctx, Batch& B, int nx, cudaStream_t st) {
  if (B.fbp.empty() || B.pchunk_next >= B.maxnj_p) return;
  const int w = (nx < 0) ? B.maxnj_p - B.pchunk_next : std::min(nx, B.maxnj_p - B.pchunk_next);
  { PROF("k_fblocks_eig", 1);
    launch_fblocks(B.d_probs, B.d_fbp, (int)B.fbp.size(), B.maxnj_p, B.maxm0, st, false, B.pchunk_next, w,
                   B.odd_m0); }
  B.pchunk_next += w;
}
void run_periodic_tail(fock_ctx* ctx, Batch& B, cudaStream_t st) {
  if (B.fbp.empty()) return;
  run_periodic_piece(ctx, B, -1, st);
  if (!B.sorts.empty()) { PROF("k_sort", 1); launch_sort_small(B.d_sorts, (int)B.sorts.size(), B.maxsort, st); }
  for (int i : B.bigsort) { PROF("k_sort_global", 1);
    launch_sort_global(B.pp[i].ev, B.pp[i].blk, B.pp[i].nev, B.sort_pv, B.sort_pi, st); }
}
void run_periodic(fock_ctx* ctx, Batch& B) {
  run_periodic_head(ctx, B, ctx->stream);
  run_periodic_tail(ctx, B, ctx->stream);
}

void run_struct_setup(fock_ctx* ctx, Batch& B) {
  cudaStream_t st = ctx->stream;
  if (B.fbs.empty()) return;
  zero_fail_flags(B, 1, st);
  { PROF("k_cell_canon", 2); launch_cell_canon(B.d_canon, (int)B.canon.size(), B.maxm0, B.maxcblk, st); }
  { PROF("k_twiddle", 1); launch_twiddles(B.d_circs, (int)B.circs.size(), st); }
  { PROF("k_fblocks_embed", 1);
    launch_fblocks(B.d_probs, B.d_fbs, (int)B.fbs.size(), B.maxnj_s, B.maxm0, st, false, 0, -1, B.odd_m0); }
  { PROF("k_precond", 2); launch_precond(B.d_probs, B.d_prec, (int)B.prec.size(), B.maxM, B.maxm0, st); }
  for (auto& Q : B.pp)
    if (Q.band_fail) cudaMemsetAsync(Q.band_fail, 0, sizeof(int), st);
  if (B.bandF.n) { PROF("k_band_factor", 1);
    launch_band_factor(reinterpret_cast<const BandTask*>(B.bandF.d), B.bandF.n, st); }
}

template <class T> const T* tl(const Batch::TL& t) { return reinterpret_cast<const T*>(t.d); }

void mv_fwd(Batch& B, const Batch::TL& t, cudaStream_t st) {
  PROF("k_fft", 1);
  launch_fft_cc(tl<FftTask>(t), t.n, (B.fft_maxcols + B.fft_cc - 1) / B.fft_cc, B.maxM, B.fft_cc, +1, st,
                B.any_mixed);
}
void mv_inv(Batch& B, const Batch::TL& t, cudaStream_t st) {
  PROF("k_fft", 1);
  launch_fft_cc(tl<FftTask>(t), t.n, (B.fft_maxcols + B.fft_cc - 1) / B.fft_cc, B.maxM, B.fft_cc, -1, st,
                B.any_mixed);
}

// Tuner of the embedded FFT's launch shape: columns per CTA trade shared memory
// per CTA (two M-point buffers per column) against CTAs per SM.  Timed once per
// (largest M, largest column count) on the plan's own forward transform of
// [X | P] (1, 2, 4, ... columns, three launches each after a warm-up, CUDA
// events on the plan's stream), cached in the context.  The width does not
// change any column's arithmetic, so results do not depend on the choice.
void tune_fft(fock_ctx* ctx, Batch& B, cudaStream_t st) {
  B.tuned = true;
  if (!B.fwdXP.n || B.fft_maxcols <= 0) return;
  const auto key = std::make_pair(B.maxM, B.fft_maxcols);
  const auto f = ctx->fft_tune.find(key);
  if (f != ctx->fft_tune.end()) { B.fft_cc = f->second; return; }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return;
  }
  const int top = std::min(16, fft_max_cc(B.maxM));
  float best = INFINITY;
  int bc = B.fft_cc;
  for (int cc = 1; cc <= top; cc *= 2) {
    const int ch = (B.fft_maxcols + cc - 1) / cc;
    launch_fft_cc(tl<FftTask>(B.fwdXP), B.fwdXP.n, ch, B.maxM, cc, +1, st, B.any_mixed);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) launch_fft_cc(tl<FftTask>(B.fwdXP), B.fwdXP.n, ch, B.maxM, cc, +1, st, B.any_mixed);
    cudaEventRecord(e1, st);
    float ms = INFINITY;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
      best = ms;
      bc = cc;
    }
  }
  cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B.fft_cc = bc;
  ctx->fft_tune[key] = bc;
}
void split_products(Batch& B, const Batch::TL& t, cudaStream_t st) {
  if (!t.sn) return;
  PROF("k_split_gemm", 1);
  launch_split_gemm((const SplitTask*)t.sd, t.sn, t.sm, t.snn, B.d_split_err, st, t.sks, t.sred);
}
void gemm_tn(Batch& B, const Batch::TL& t, cudaStream_t st) {
  { PROF("k_gemm_tn", 1);
    launch_gemm_tn(tl<GemmTask>(t), t.n, t.ga, t.gb, t.tile, st); }   // ga, gb: output dims; tile: tile-size bits
  split_products(B, t, st);
}
void gemm_nn(Batch& B, const Batch::TL& t, cudaStream_t st) {
  { PROF("k_gemm_nn", 1);
    if (t.n) k_gemm_nn<<<dim3(64, t.n), 256, 0, st>>>(tl<GemmTask>(t)); }
  split_products(B, t, st);
}
void rr(Batch& B, const Batch::TL& t, cudaStream_t st) {
  PROF("k_rr", 1);
  if (!t.n) return;
  FOCK_SMEM_OPTIN(k_rr);
  // problems whose working matrices fit shared memory: 256 threads; the
  // others (global memory, latency-bound): 512 threads, more warps in flight
  if (B.rr_small) {
    const int ld = B.rr_small_ld;
    const size_t sm = ((size_t)3 * ld * ld + (size_t)rr_stage_extra(ld)) * sizeof(double);
    k_rr<<<t.n, 256, sm, st>>>(tl<RRTask>(t), (int)sm, 0);
  }
  if (B.rr_big && !B.rr_cluster) {
    const size_t sm = (size_t)2 * kRRBlock * B.rr_big_ld * sizeof(double);
    k_rr<<<t.n, 512, sm, st>>>(tl<RRTask>(t), (int)sm, 1);
  }
  if (B.rr_big && B.rr_cluster) {
    // one cluster of kRRCluster CTAs per problem
    FOCK_SMEM_OPTIN(k_rr_cl);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(t.n * kRRCluster));
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = rr_cl_smem(B.rr_big_ld, B.kmax);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kRRCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_rr_cl, tl<RRTask>(t));
  }
}
// unit 2-norm columns before a matvec: the FFT packs two real columns per
// complex transform, and a column far smaller than its partner would get an
// image accurate only relative to the partner (Rayleigh-Ritz is invariant
// to column scaling)
void normalize(const Batch::TL& t, int maxcols, cudaStream_t st) {
  PROF("k_colnorm", 1);
  if (t.n) k_colnorm<<<dim3(maxcols, t.n), 256, 0, st>>>(tl<CopyTask>(t));
}
void copies(const Batch::TL& t, cudaStream_t st) {
  PROF("k_copy_cols", 1);
  if (t.n) k_copy_cols<<<dim3(32, t.n), 256, 0, st>>>(tl<CopyTask>(t));
}

// H and S images of the [X | P] columns (2k) or of the W columns (k) of every structured problem
void mv_HS(Batch& B, bool xp, cudaStream_t st) {
  mv_fwd(B, xp ? B.fwdXP : B.fwdW, st);
  const Batch::TL& bm = xp ? B.bmulHS2 : B.bmulHS1;
  { PROF("k_blockmul", 1); launch_blockmul(tl<BmulTask>(bm), bm.n, B.maxM, B.maxm0, st, B.any_mixed); }
  mv_inv(B, xp ? B.invHXP : B.invHW, st);
  mv_inv(B, xp ? B.invSXP : B.invSW, st);
  const Batch::TL& eh = xp ? B.eHXP : B.eHW;   // each task applies the H and the S blocks
  if (eh.n) { PROF("k_eapply", 1); launch_eapply(tl<EApplyTask>(eh), eh.n, B.eapply_gx, st); }
}

// [X | P] images in FP64 for the problems flagged in d_refresh only
void refresh_XP(Batch& B, cudaStream_t st) {
  mv_fwd(B, B.rfwdXP, st);
  { PROF("k_blockmul", 1); launch_blockmul(tl<BmulTask>(B.rbmulHS2), B.rbmulHS2.n, B.maxM, B.maxm0, st, false); }
  mv_inv(B, B.rinvHXP, st);
  mv_inv(B, B.rinvSXP, st);
  if (B.reHXP.n) { PROF("k_eapply", 1); launch_eapply(tl<EApplyTask>(B.reHXP), B.reHXP.n, B.eapply_gx, st); }
}

// One block-iteration step after the convergence test, in two parts.  A: W = K R
// (the shifted inverse of the embedding's Fourier blocks, or the banded factor)
// S-orthogonal to X, fresh images of W, the Gram matrices of [X | P | W].  B:
// Rayleigh-Ritz, P' S-orthogonal to X' in the coefficients, [X | P] <- Y Cc and
// their fresh images.  Launches only.
void lobpcg_body_a(Batch& B, cudaStream_t st) {
  if (B.bandS.n) { PROF("k_band_solve", 1); launch_band_solve(tl<BandTask>(B.bandS), B.bandS.n, B.kmax, B.band_stage, B.band_ringrow, st, B.any_mixed); }
  if (B.fwdR.n) {
    mv_fwd(B, B.fwdR, st);
    { PROF("k_blockmul", 1); launch_blockmul(tl<BmulTask>(B.bmulK), B.bmulK.n, B.maxM, B.maxm0, st, B.any_mixed); }
    mv_inv(B, B.invPW, st);
  }
  gemm_tn(B, B.tnCx, st);
  gemm_nn(B, B.nnW, st);
  normalize(B.normW, B.kmax, st);
  mv_HS(B, false, st);
  // Rayleigh-Ritz on [X | P | W]
  gemm_tn(B, B.g3, st);
}
void lobpcg_body_b(Batch& B, cudaStream_t st) {
  rr(B, B.rr3, st);
  // P' S-orthogonal to X' in the coefficients; [X | P] <- Y Cc, fresh images
  gemm_nn(B, B.pcG, st);
  gemm_tn(B, B.pcM, st);
  gemm_nn(B, B.pcZ, st);
  gemm_nn(B, B.u3, st);
  copies(B.cp2k, st);
  normalize(B.normP, B.kmax, st);
  mv_HS(B, true, st);
}

// on_left (optional): called after each convergence test with the problems
// (indices into B.sidx) that left the iteration in it, converged or broken down;
// no later launch touches their outputs, and the stream is idle at the call.
int run_lobpcg(fock_ctx* ctx, Batch& B, double tol, int maxit, std::vector<int>& iters,
               std::vector<double>& resid, std::vector<int>& conv,
               std::vector<std::vector<double>>* hist = nullptr,
               const std::function<void(const std::vector<int>&)>* on_left = nullptr) {
  cudaStream_t st = ctx->stream;
  const int ns = (int)B.sidx.size();
  iters.assign(ns, 0);
  resid.assign(ns, 0.0);
  conv.assign(ns, 0);
  if (hist) hist->assign(ns, std::vector<double>());
  if (!ns) return FOCK_OK;
  CUDA_TRY(ctx, cudaMemcpyAsync(B.d_active, B.d_ones, ns * sizeof(int), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(ctx, cudaMemsetAsync(B.d_fail, 0, ns * sizeof(int), st));
  // mixed form: matvecs in FP32 until the wanted residual falls below
  // kMixedSwitch, FP64 from then on (monotone), so that the converged pairs
  // come from FP64 images; no convergence decision during the FP32 phase
  // the FP32 phase also ends when its residual stops halving for two
  // iterations or after kMixedMaxIt iterations (an ill-conditioned pencil
  // cannot reach kMixedSwitch with FP32 images)
  const double kMixedSwitch = 1e-5;
  const int kMixedMaxIt = 10;
  std::vector<int> mode(ns, 0), f32_it(ns, 0), f32_stall(ns, 0);
  std::vector<double> f32_best(ns, INFINITY);
  for (int s2 = 0; s2 < ns; ++s2) mode[s2] = B.hp[B.sidx[s2]].f32;
  CUDA_TRY(ctx, cudaMemcpyAsync(B.d_mode, mode.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
  // X random, P = W = 0; Rayleigh-Ritz on X alone, then fresh images of [X | P]
  { PROF("k_init_x", 1); k_init_x<<<dim3(32, B.init.n), 256, 0, st>>>(tl<InitTask>(B.init)); }
  if (!B.tuned) tune_fft(ctx, B, st);
  mv_HS(B, true, st);
  gemm_tn(B, B.g1, st);
  rr(B, B.rr1, st);
  gemm_nn(B, B.u1, st);
  copies(B.cp2k, st);
  mv_HS(B, true, st);
  std::vector<double> hres((size_t)ns * B.kmax);
  std::vector<int> active(ns, 1);
  // a residual that stops improving below kFloorTol is at the rounding floor
  // of the pencil (it scales with the overlap's condition number); Rayleigh
  // quotients are then accurate to about the square of the residual over the
  // gap, so the problem is done, provided the current residual is still
  // within a factor 100 of that floor (a state that broke down after reaching
  // it keeps iterating, or ends unconverged).  1e-5 (tried) accepted a
  // defect chain whose slowly converging pair was still 4e-5 off.
  const double kFloorTol = 1e-6;
  const int kStagnation = 8;
  // a floor within 100 tol of the target is recognised after 3 iterations
  // without a halving of the residual (Rayleigh quotients are then exact to
  // ~(100 tol)^2 / gap)
  const double kNearFactor = 100.0;
  const int kStagnationNear = 3;
  std::vector<double> best(ns, INFINITY);
  std::vector<int> best_it(ns, 0);
  int it = 0;
  for (;; ++it) {
    { PROF("k_resid", 1); k_resid<<<dim3(B.kmax, B.resid.n), 256, 0, st>>>(tl<ResidTask>(B.resid), tol); }
    CUDA_TRY(ctx, cudaMemcpyAsync(hres.data(), B.d_res, hres.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    bool any = false, changed = false, switched = false;
    std::vector<int> just(ns, 0), left;
    for (int s2 = 0; s2 < ns; ++s2) {
      if (!active[s2]) continue;
      double mx = 0.0;
      bool bad = false;
      for (int c = 0; c < B.lob[s2].kw; ++c) {   // the wanted pairs decide convergence
        double r = hres[(size_t)s2 * B.kmax + c];
        if (!(r == r) || std::isinf(r)) bad = true; else mx = std::max(mx, r);
      }
      resid[s2] = bad ? INFINITY : mx;
      iters[s2] = it;
      if (hist) (*hist)[s2].push_back(resid[s2]);
      if (mode[s2] && !bad) {   // FP32 phase of the mixed form
        ++f32_it[s2];
        if (mx < 0.5 * f32_best[s2]) { f32_best[s2] = mx; f32_stall[s2] = 0; } else ++f32_stall[s2];
        if (mx <= kMixedSwitch || f32_stall[s2] >= 2 || f32_it[s2] >= kMixedMaxIt) {
          mode[s2] = 0; changed = true; switched = true; just[s2] = 1;
        }
        any = true;
        continue;
      }
      // the floor clock restarts only on a halving of the residual (fluctuations
      // at the floor within a factor 2 do not count as progress)
      if (!bad && mx < 0.5 * best[s2]) { best[s2] = mx; best_it[s2] = it; }
      if (bad) { active[s2] = 0; changed = true; }            // broken: stop, report no convergence
      else if (mx <= tol) { active[s2] = 0; conv[s2] = 1; changed = true; }
      else if (it == 0 && B.lob[s2].k == B.lob[s2].n) {
        // whole-space block: the start's Rayleigh-Ritz step over all n directions
        // is exact up to rounding, and [X | P | W] would add only noise directions
        active[s2] = 0; conv[s2] = 1; changed = true;
      }
      else if (mx <= 100.0 * best[s2] &&
               ((best[s2] <= kNearFactor * tol && it - best_it[s2] >= kStagnationNear) ||
                (best[s2] <= kFloorTol && it - best_it[s2] >= kStagnation))) {
        active[s2] = 0; conv[s2] = 1; changed = true;
      }
      else any = true;
      if (!active[s2]) left.push_back(s2);
    }
    if (on_left && *on_left && !left.empty()) (*on_left)(left);
    if (!any || it >= maxit) break;
    if (changed) {
      CUDA_TRY(ctx, cudaMemcpyAsync(B.d_active, active.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
      CUDA_TRY(ctx, cudaMemcpyAsync(B.d_mode, mode.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    if (switched) {   // FP64 images of [X | P] before mixing them with FP64 W images
      std::vector<int> rf(ns, 2);
      for (int s2 = 0; s2 < ns; ++s2) if (just[s2]) rf[s2] = 0;
      CUDA_TRY(ctx, cudaMemcpyAsync(B.d_refresh, rf.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
      refresh_XP(B, st);
      CUDA_TRY(ctx, cudaStreamSynchronize(st));   // rf is a host temporary
    }
    // the iteration's body: launches only (converged problems are skipped by
    // every kernel through their device-side flags), so from the second pass
    // on it is replayed as two CUDA graphs captured on that pass; with the
    // kernel timers on it stays eager
    if (!ctx->prof && it >= 1 && !B.iter_graph && !B.graph_failed) {
      B.graph_nodes = 0;
      auto capture = [&](void (*body)(Batch&, cudaStream_t), cudaGraphExec_t* out) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
        body(B, st);
        const cudaError_t ce = cudaStreamEndCapture(st, &g);
        bool ok = (ce == cudaSuccess && g && cudaGraphInstantiate(out, g, 0) == cudaSuccess);
        if (ok) {
          size_t nn = 0;
          if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess) B.graph_nodes += (int)nn;
        } else {
          *out = nullptr;
        }
        if (g) cudaGraphDestroy(g);
        return ok;
      };
      if (!capture(lobpcg_body_a, &B.iter_graph) || !capture(lobpcg_body_b, &B.iter_graph_b)) {
        if (B.iter_graph) cudaGraphExecDestroy(B.iter_graph);
        if (B.iter_graph_b) cudaGraphExecDestroy(B.iter_graph_b);
        B.iter_graph = B.iter_graph_b = nullptr;
        B.graph_failed = true;
        cudaGetLastError();
      }
    }
    const bool graphs = B.iter_graph && !ctx->prof;
    if (graphs) CUDA_TRY(ctx, cudaGraphLaunch(B.iter_graph, st));
    else lobpcg_body_a(B, st);
    // a piece of the periodic problems' Fourier-block eigensolves on their own
    // (lower-priority) stream, started when this stream reaches the
    // Rayleigh-Ritz launch, which occupies one SM per box chain: the piece fills
    // the other SMs meanwhile and is sized to end about when it does
    if (ctx->pstream && B.pchunk_next < B.maxnj_p) {
      CUDA_TRY(ctx, cudaEventRecord(ctx->ev_chunk, st));
      CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->pstream, ctx->ev_chunk, 0));
      run_periodic_piece(ctx, B, B.pchunk_w, ctx->pstream);
    }
    if (graphs) CUDA_TRY(ctx, cudaGraphLaunch(B.iter_graph_b, st));
    else lobpcg_body_b(B, st);
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return FOCK_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
struct fock_plan {
  fock_ctx* ctx = nullptr;
  Batch B;
  std::vector<int> iters, conv;
  std::vector<double> resid;
  std::vector<std::vector<double>> hist;   // per structured problem: residual of each iteration
  std::function<void(const std::vector<int>&)> on_left;   // see run_lobpcg (serving's early release)
};

namespace {

// After the shared assembly, the periodic problems (one pass of wide launches:
// a CTA per Fourier block) and the structured ones (a host-driven iteration of
// narrow launches: a CTA per problem in the Rayleigh-Ritz step, which leaves
// most SMs idle) run concurrently: the iteration on the context's
// greatest-priority stream, whose CTAs the hardware schedules first as SMs free
// up, the Fourier-block eigensolves on the context's stream, filling the rest.
// Both read only the assembled generators and write disjoint buffers.  With the
// kernel timers on, the two run one after the other on the context's stream,
// so that each timer measures its kernel alone.
int plan_execute(fock_plan& P, double tol, int maxit) {
  fock_ctx* ctx = P.ctx;
  Batch& B = P.B;
  run_assemble(ctx, B);
  const bool overlap = ctx->hi && !ctx->prof && !B.fbp.empty() && !B.fbs.empty();
  if (!overlap) {
    run_periodic(ctx, B);
    run_struct_setup(ctx, B);
    int rc = run_lobpcg(ctx, B, tol, maxit, P.iters, P.resid, P.conv, &P.hist, &P.on_left);
    if (rc) return rc;
  } else {
    cudaStream_t user = ctx->stream;
    CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, user));
    CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->hi, ctx->ev_fork, 0));
    run_periodic_head(ctx, B, user);
    // pieces of about kPeriodicPieceCTAs Fourier blocks ride along with the
    // iteration's Rayleigh-Ritz launches; the rest, and the sorts, follow it
    B.pchunk_w = std::max(1, kPeriodicPieceCTAs / std::max(1, (int)B.fbp.size()));
    ctx->pstream = user;
    ctx->stream = ctx->hi;
    run_struct_setup(ctx, B);
    int rc = run_lobpcg(ctx, B, tol, maxit, P.iters, P.resid, P.conv, &P.hist, &P.on_left);
    ctx->stream = user;
    ctx->pstream = nullptr;
    run_periodic_tail(ctx, B, user);
    // joined on every path: later work on the context's stream sees both
    cudaError_t e = cudaEventRecord(ctx->ev_join, ctx->hi);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ctx->ev_join, 0);
    if (rc) return rc;
    CUDA_TRY(ctx, e);
  }
  CUDA_TRY(ctx, cudaGetLastError());
  return FOCK_OK;
}

int plan_outputs(fock_plan& P, fock_output* outs, int on_device) {
  fock_ctx* ctx = P.ctx;
  Batch& B = P.B;
  const int nprob = B.nprob;
  std::vector<int> pfail(nprob, 0);
  int split_err = 0;
  for (int i = 0; i < nprob; ++i) {
    outs[i].n_evals = B.pp[i].nev;
    outs[i].iters = 0;
    outs[i].resid = 0.0;
    outs[i].status = FOCK_OK;
  }
  for (size_t s2 = 0; s2 < B.sidx.size() && s2 < P.iters.size(); ++s2) {
    const int i = B.sidx[s2];
    outs[i].iters = P.iters[s2];
    outs[i].resid = P.resid[s2];
    if (!P.conv[s2]) outs[i].status = FOCK_ENOCONV;
  }
  if (on_device) {   // device destinations: one device-to-device copy per array
    for (int i = 0; i < nprob; ++i) {
      const Batch::PerProb& Q = B.pp[i];
      const double* ev = (B.hp[i].kind == 0) ? Q.ev : nullptr;
      if (B.hp[i].kind == 0) {
        if (outs[i].block_of)
          CUDA_TRY(ctx, cudaMemcpyAsync(outs[i].block_of, Q.blk, Q.nev * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
        CUDA_TRY(ctx, cudaMemcpyAsync(&pfail[i], Q.fail, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      }
      if (ev && outs[i].evals)
        CUDA_TRY(ctx, cudaMemcpyAsync(outs[i].evals, ev, Q.nev * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    for (size_t s2 = 0; s2 < B.sidx.size(); ++s2) {
      const int i = B.sidx[s2];
      if (outs[i].evals)
        CUDA_TRY(ctx, cudaMemcpyAsync(outs[i].evals, B.lob[s2].lam, B.pp[i].nev * sizeof(double),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (B.d_split_err)
      CUDA_TRY(ctx, cudaMemcpyAsync(&split_err, B.d_split_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  } else {           // host destinations: gather on the device, one copy to pinned memory
    const size_t nw = B.ostage_words;
    if (ctx->hstage_cap < nw) {
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
      if (ctx->hstage) cudaFreeHost(ctx->hstage);
      ctx->hstage = nullptr; ctx->hstage_cap = 0;
      CUDA_TRY(ctx, cudaMallocHost(&ctx->hstage, (nw + nw / 4 + 2) * sizeof(uint32_t)));
      ctx->hstage_cap = nw + nw / 4 + 2;
    }
    launch_gather(B.d_gseg, (int)B.gseg.size(), B.d_ostage, ctx->stream);
    CUDA_TRY(ctx, cudaGetLastError());
    if (nw) CUDA_TRY(ctx, cudaMemcpyAsync(ctx->hstage, B.d_ostage, nw * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t* hs = ctx->hstage;
    for (int i = 0; i < nprob; ++i) {
      const size_t nev = (size_t)B.pp[i].nev;
      if (outs[i].evals && B.o_ev[i] >= 0) std::memcpy(outs[i].evals, hs + B.o_ev[i], nev * sizeof(double));
      if (outs[i].block_of && B.o_blk[i] >= 0) std::memcpy(outs[i].block_of, hs + B.o_blk[i], nev * sizeof(int));
      if (B.o_fail[i] >= 0) std::memcpy(&pfail[i], hs + B.o_fail[i], sizeof(int));
    }
    if (B.o_split_err >= 0) std::memcpy(&split_err, hs + B.o_split_err, sizeof(int));
  }
  int first = FOCK_OK;
  for (int i = 0; i < nprob; ++i) {
    if (split_err && B.hp[i].mixed) outs[i].status = FOCK_ETIMEOUT;   // its assembly did not complete
    if (pfail[i]) outs[i].status = FOCK_EINVAL;
    if (outs[i].status && !first) first = outs[i].status;
  }
  if (first == FOCK_EINVAL) set_err(ctx, first, "a Fourier-block mass matrix was not positive definite");
  if (first == FOCK_ENOCONV) set_err(ctx, first, "box eigensolver reached maxit");
  if (first == FOCK_ETIMEOUT) set_err(ctx, first, "a tensor-core completion wait of the mixed assembly ran out");
  return first;
}

}  // namespace

struct fock_blocks {
  fock_ctx* ctx;
  Batch B;
};

namespace fock {

int blocks_matvec_view(const fock_blocks* b, MatvecView* v) {
  if (!b || !v) return FOCK_EINVAL;
  const Batch& B = b->B;
  if (B.hp[0].kind != 1) return FOCK_EINVAL;
  const Batch::PerProb& Q = B.pp[0];
  v->Lc = Q.Lc; v->m0 = B.hp[0].m0; v->M = Q.M; v->nE = Q.nE; v->nErows = Q.nErows;
  v->circ = B.d_circs + Q.circ;
  v->CH = Q.CHo; v->CS = Q.CSo;
  v->Erows = Q.Erows; v->Erowptr = Q.Erowptr; v->Ecols = Q.Ecols;
  v->EH = Q.EH; v->ES = Q.ES;
  v->stream = b->ctx->stream;
  v->device = b->ctx->device;
  return FOCK_OK;
}

void set_ctx_error(fock_ctx* c, const char* msg) { if (c) c->err = msg; }
}  // namespace fock

// ------------------------------------------------------------------ serving hooks
// Used by the serving loop (serve.cu): size estimate of one request, private
// worker contexts that allocate from a shared pool, and one batched solve
// with host outputs.
namespace fock {

int detail_estimate(const fock_problem& p, size_t* bytes, int* n_evals, std::string& why) {
  Batch B;
  B.nprob = 1;
  B.hp.assign(1, HostProb());
  B.ap.assign(3, AxisPlan());
  int rc = validate(p, B.hp[0], why);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a) axis_plan(B.hp[0], a, B.ap[a]);
  Slab S0, U0;
  plan(B, S0, U0);
  *bytes = S0.off + U0.off + 512;
  *n_evals = B.pp[0].nev;
  return FOCK_OK;
}

// Host-only planning of one problem (no device): the sizing pass of plan().
int detail_layout(const fock_problem& p, Batch& B, std::string& why) {
  B.nprob = 1;
  B.hp.assign(1, HostProb());
  B.ap.assign(3, AxisPlan());
  int rc = validate(p, B.hp[0], why);
  if (rc) return rc;
  for (int a = 0; a < 3; ++a) axis_plan(B.hp[0], a, B.ap[a]);
  Slab S0, U0;
  plan(B, S0, U0);
  return FOCK_OK;
}

fock_ctx* detail_worker_ctx(int device, cudaMemPool_t pool, size_t budget) {
  if (cudaSetDevice(device) != cudaSuccess) return nullptr;
  fock_ctx* c = new fock_ctx();
  c->device = device;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return nullptr; }
  c->own_stream = true;
  c->mempool = pool;
  c->budget = budget;
  return c;
}

const char* detail_ctx_error(const fock_ctx* c) { return c->err.c_str(); }
cudaStream_t detail_ctx_stream(const fock_ctx* c) { return c->stream; }

// release (optional): called for each structured problem as soon as it leaves
// the block iteration, with its output (eigenvalues already in outs[i].evals on
// the host, n_evals, status, iters, resid); that problem's outs[i].evals is then
// set to null, so the batch's final outputs leave the caller's buffer alone (the
// caller may hand it back to its owner at once).  A mixed problem is released
// early only while the batch's tensor-core completion flag is clear; else its
// status (FOCK_ETIMEOUT) is decided with the batch's.
int detail_solve(fock_ctx* w, int n, const fock_problem* probs, fock_output* outs, double tol, int maxit,
                 const std::function<void(int, const fock_output&)>* release) {
  fock_plan P;
  P.ctx = w;
  if (release && *release) {
    P.on_left = [&P, outs, release](const std::vector<int>& left) {
      Batch& B = P.B;
      fock_ctx* c = P.ctx;
      int split_err = 0;
      std::vector<int> go;
      if (B.d_split_err &&
          cudaMemcpyAsync(&split_err, B.d_split_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return;
      for (int s2 : left) {
        const int i = B.sidx[s2];
        if (!outs[i].evals) continue;
        if (cudaMemcpyAsync(outs[i].evals, B.lob[s2].lam, B.pp[i].nev * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess)
          return;
        go.push_back(s2);
      }
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return;   // left to the batch's end
      for (int s2 : go) {
        const int i = B.sidx[s2];
        if (split_err && B.hp[i].mixed) continue;
        fock_output o = outs[i];
        o.n_evals = B.pp[i].nev;
        o.iters = P.iters[s2];
        o.resid = P.resid[s2];
        o.status = P.conv[s2] ? FOCK_OK : FOCK_ENOCONV;
        outs[i].evals = nullptr;
        (*release)(i, o);
      }
    };
  }
  int rc = build_batch(w, n, probs, P.B, false);
  if (rc == FOCK_OK) rc = plan_execute(P, tol, maxit);
  if (rc == FOCK_OK || rc == FOCK_ENOCONV) rc = plan_outputs(P, outs, 0);
  free_batch(P.B);
  cudaStreamSynchronize(w->stream);
  return rc;
}

}  // namespace fock

extern "C" {

int fock_create(fock_ctx** out, int device, size_t hbm_budget_bytes, void* stream) {
  if (!out) return FOCK_EINVAL;
  *out = nullptr;
  fock_ctx* c = new fock_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return FOCK_ECUDA; }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return FOCK_ECUDA; }
    c->own_stream = true;
  }
  {   // the structured iteration's stream (greatest priority); without it plans run serially
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->hi, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_chunk, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (c->hi) cudaStreamDestroy(c->hi);
      if (c->ev_fork) cudaEventDestroy(c->ev_fork);
      if (c->ev_join) cudaEventDestroy(c->ev_join);
      if (c->ev_chunk) cudaEventDestroy(c->ev_chunk);
      c->hi = nullptr; c->ev_fork = c->ev_join = c->ev_chunk = nullptr;
    }
  }
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    hbm_budget_bytes = (size_t)(0.9 * (double)fr);
  }
  c->budget = hbm_budget_bytes;
  *out = c;
  return FOCK_OK;
}

void fock_destroy(fock_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->arena) cudaFree(c->arena);
  if (c->hstage) cudaFreeHost(c->hstage);
  if (c->hi) { cudaStreamSynchronize(c->hi); cudaStreamDestroy(c->hi); }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_chunk) cudaEventDestroy(c->ev_chunk);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* fock_last_error(const fock_ctx* c) { return c ? c->err.c_str() : "null context"; }

int fock_problem_layout(const fock_problem* p, int* Nb, int* mcirc, int* D, int* nbound, int* Ek,
                        int* Em, int* Ekind, int cap) {
  if (!p) return FOCK_EINVAL;
  Batch B;
  std::string why;
  const int rc = fock::detail_layout(*p, B, why);
  if (rc != FOCK_OK) return rc;
  const HostProb& H = B.hp[0];
  const Batch::PerProb& Q = B.pp[0];
  const int ncell = H.L[0] * H.L[1] * H.L[2];
  if (Nb) *Nb = ncell * H.m0;
  if (mcirc) *mcirc = H.kind == 1 ? Q.M : ncell;
  if (D) *D = H.kind == 1 ? Q.D : 0;
  const int nE = H.kind == 1 ? Q.nE : 0;
  if (nbound) *nbound = nE;
  for (int e = 0; e < std::min(nE, cap); ++e) {
    if (Ek) Ek[e] = Q.Ek[e];
    if (Em) Em[e] = Q.Em[e];
    if (Ekind) Ekind[e] = Q.Ekind[e];
  }
  return FOCK_OK;
}

int fock_problem_check(const fock_problem* p, int* kind, int* n_evals, char* why, int why_cap) {
  if (why && why_cap > 0) why[0] = '\0';
  if (!p) return FOCK_EINVAL;
  HostProb H;
  std::string msg;
  const int rc = validate(*p, H, msg);
  if (rc != FOCK_OK) {
    if (why && why_cap > 0) {
      const size_t n = std::min(msg.size(), (size_t)(why_cap - 1));
      std::memcpy(why, msg.data(), n);
      why[n] = '\0';
    }
    return rc;
  }
  if (kind) *kind = H.kind;
  if (n_evals) *n_evals = (H.kind == 1) ? H.k_eig : H.L[0] * H.L[1] * H.L[2] * H.m0;
  return FOCK_OK;
}

int fock_synchronize(fock_ctx* c) {
  if (!c) return FOCK_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return FOCK_OK;
}

int fock_solve(fock_ctx* ctx, int nprob, const fock_problem* probs, fock_output* outs, int on_device) {
  if (!ctx || !outs) return FOCK_EINVAL;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ProfBind pb(ctx);
  fock_plan P;
  P.ctx = ctx;
  int rc = build_batch(ctx, nprob, probs, P.B, false);
  if (rc) return rc;
  rc = plan_execute(P, 1e-10, FOCK_DEFAULT_MAXIT);
  if (rc) return rc;
  return plan_outputs(P, outs, on_device);
}

int fock_plan_create(fock_ctx* ctx, int nprob, const fock_problem* probs, fock_plan** out) {
  if (!ctx || !out) return FOCK_EINVAL;
  *out = nullptr;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  fock_plan* P = new fock_plan();
  P->ctx = ctx;
  int rc = build_batch(ctx, nprob, probs, P->B, true);
  if (rc) { free_batch(P->B); delete P; return rc; }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) { free_batch(P->B); delete P; return set_err(ctx, FOCK_ECUDA, cudaGetErrorString(e)); }
  *out = P;
  return FOCK_OK;
}

int fock_plan_execute(fock_plan* P, double tol, int maxit) {
  if (!P) return FOCK_EINVAL;
  ProfBind pb(P->ctx);
  return plan_execute(*P, tol > 0 ? tol : 1e-10, maxit > 0 ? maxit : FOCK_DEFAULT_MAXIT);
}

int fock_plan_outputs(fock_plan* P, fock_output* outs, int on_device) {
  if (!P || !outs) return FOCK_EINVAL;
  return plan_outputs(*P, outs, on_device);
}

int fock_plan_info(const fock_plan* P, size_t* upload_bytes, size_t* device_bytes, size_t* n_evals) {
  if (!P) return FOCK_EINVAL;
  if (upload_bytes) *upload_bytes = P->B.ubytes;
  if (device_bytes) *device_bytes = P->B.bytes + P->B.ubytes;
  if (n_evals) {
    size_t n = 0;
    for (const auto& Q : P->B.pp) n += Q.nev;
    *n_evals = n;
  }
  return FOCK_OK;
}

int fock_plan_tuning(const fock_plan* P, int* fft_cc, int* graph_nodes) {
  if (!P) return FOCK_EINVAL;
  if (fft_cc) *fft_cc = P->B.tuned ? P->B.fft_cc : 0;
  if (graph_nodes) *graph_nodes = (P->B.iter_graph && P->B.iter_graph_b) ? P->B.graph_nodes : 0;
  return FOCK_OK;
}

int fock_plan_block_routes(const fock_plan* P, int i, int* n_eig) {
  if (!P || !n_eig || i < 0 || i >= P->B.nprob) return FOCK_EINVAL;
  *n_eig = 0;
  const Batch& B = P->B;
  if (B.hp[i].kind != 0 || !B.pp[i].fail) return FOCK_OK;
  fock_ctx* ctx = P->ctx;
  CUDA_TRY(ctx, cudaMemcpyAsync(n_eig, B.pp[i].fail + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return FOCK_OK;
}

int fock_plan_problem_sizes(const fock_plan* P, int i, int* Nb, int* mcirc, int* D, int* nbound) {
  if (!P || i < 0 || i >= P->B.nprob) return FOCK_EINVAL;
  const HostProb& H = P->B.hp[i];
  const Batch::PerProb& Q = P->B.pp[i];
  const int ncell = H.L[0] * H.L[1] * H.L[2];
  if (Nb) *Nb = ncell * H.m0;
  if (mcirc) *mcirc = H.kind == 1 ? Q.M : ncell;
  if (D) *D = H.kind == 1 ? Q.D : 0;
  if (nbound) *nbound = H.kind == 1 ? Q.nE : 0;
  return FOCK_OK;
}

int fock_plan_split_work(const fock_plan* P, double* tensor_flops, double* fp64_flops) {
  if (!P) return FOCK_EINVAL;
  double tf = 0.0, ff = 0.0;
  for (const SplitTask& t : P->B.splits) {
    const double tiles = (double)((t.M + 127) / 128) * ((t.N + 63) / 64), chunks = (double)((t.K + 63) / 64);
    tf += tiles * chunks * 28.0 * 4.0 * (128.0 * 64.0 * 16.0 * 2.0);
    ff += 2.0 * t.M * (double)t.N * t.K;
  }
  if (tensor_flops) *tensor_flops = tf;
  if (fp64_flops) *fp64_flops = ff;
  return FOCK_OK;
}

int fock_plan_history(const fock_plan* P, int i, double* res, int cap) {
  if (!P || i < 0 || i >= P->B.nprob) return FOCK_EINVAL;
  const auto& sid = P->B.sidx;
  for (size_t s2 = 0; s2 < sid.size() && s2 < P->hist.size(); ++s2)
    if (sid[s2] == i) {
      const std::vector<double>& h = P->hist[s2];
      for (int t = 0; t < std::min((int)h.size(), std::max(cap, 0)); ++t) if (res) res[t] = h[t];
      return (int)h.size();
    }
  return 0;
}

void fock_plan_free(fock_plan* P) {
  if (!P) return;
  cudaStreamSynchronize(P->ctx->stream);
  free_batch(P->B);
  delete P;
}

int fock_profile_enable(fock_ctx* c, int on) {
  if (!c) return FOCK_EINVAL;
  c->prof = on != 0;
  return FOCK_OK;
}

int fock_profile_reset(fock_ctx* c) {
  if (!c) return FOCK_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (auto& r : c->recs) { c->pool.push_back(r.a); c->pool.push_back(r.b); }
  c->recs.clear();
  return FOCK_OK;
}

int fock_profile_read(fock_ctx* c, int cap, char* names, int* launches, double* ms) {
  if (!c) return FOCK_EINVAL;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<std::string> nm;
  std::vector<int> cnt;
  std::vector<double> tot;
  for (auto& r : c->recs) {
    float t = 0.f;
    cudaEventElapsedTime(&t, r.a, r.b);
    size_t i = 0;
    while (i < nm.size() && nm[i] != r.name) ++i;
    if (i == nm.size()) { nm.push_back(r.name); cnt.push_back(0); tot.push_back(0.0); }
    cnt[i] += r.nlaunch;
    tot[i] += t;
  }
  int n = (int)std::min<size_t>(nm.size(), (size_t)std::max(cap, 0));
  for (int i = 0; i < n; ++i) {
    if (names) { std::memset(names + 32 * i, 0, 32); std::strncpy(names + 32 * i, nm[i].c_str(), 31); }
    if (launches) launches[i] = cnt[i];
    if (ms) ms[i] = tot[i];
  }
  return n;
}

int fock_assemble(fock_ctx* ctx, const fock_problem* p, fock_blocks** out) {
  if (!ctx || !p || !out) return FOCK_EINVAL;
  *out = nullptr;
  CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ProfBind pb(ctx);
  fock_blocks* b = new fock_blocks();
  b->ctx = ctx;
  int rc = build_batch(ctx, 1, p, b->B, true);
  if (rc) { free_batch(b->B); delete b; return rc; }
  run_assemble(ctx, b->B);
  run_struct_setup(ctx, b->B);
  if (!b->B.fbo.empty()) {   // Fourier blocks of the original operator for the matvec entry points
    PROF("k_fblocks_embed", 1);
    launch_fblocks(b->B.d_probs, b->B.d_fbo, (int)b->B.fbo.size(), b->B.maxnj_s, b->B.maxm0, ctx->stream);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) { free_batch(b->B); delete b; return set_err(ctx, FOCK_ECUDA, cudaGetErrorString(e)); }
  *out = b;
  return FOCK_OK;
}

void fock_blocks_free(fock_blocks* b) {
  if (!b) return;
  cudaStreamSynchronize(b->ctx->stream);
  free_batch(b->B);
  delete b;
}

int fock_blocks_info(const fock_blocks* b, int* Nb, int* ngen, int* nbound, int* mcirc) {
  if (!b) return FOCK_EINVAL;
  const HostProb& H = b->B.hp[0];
  const Batch::PerProb& Q = b->B.pp[0];
  int ncell = H.L[0] * H.L[1] * H.L[2];
  if (Nb) *Nb = ncell * H.m0;
  if (H.kind == 0) {
    if (ngen) *ngen = ncell;
    if (nbound) *nbound = 0;
    if (mcirc) *mcirc = ncell;
  } else {
    if (ngen) *ngen = 2 * Q.D + 1;
    if (nbound) *nbound = Q.nE;
    if (mcirc) *mcirc = Q.M;
  }
  return FOCK_OK;
}

int fock_blocks_copy_generators(const fock_blocks* b, double* Hout, double* Sout, double* EH, double* ES,
                                int* bound_rc) {
  if (!b) return FOCK_EINVAL;
  fock_ctx* ctx = b->ctx;
  const Batch& B = b->B;
  const HostProb& H = B.hp[0];
  const Batch::PerProb& Q = B.pp[0];
  const int m2 = H.m0 * H.m0;
  cudaStream_t st = ctx->stream;
  if (H.kind == 1) {
    std::vector<double> th((size_t)(Q.D + 1) * m2), ts((size_t)(Q.D + 1) * m2);
    CUDA_TRY(ctx, cudaMemcpyAsync(th.data(), Q.TH, th.size() * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaMemcpyAsync(ts.data(), Q.TS, ts.size() * 8, cudaMemcpyDeviceToHost, st));
    if (EH && Q.nE) CUDA_TRY(ctx, cudaMemcpyAsync(EH, Q.EH, (size_t)Q.nE * m2 * 8, cudaMemcpyDeviceToHost, st));
    if (ES && Q.nE) CUDA_TRY(ctx, cudaMemcpyAsync(ES, Q.ES, (size_t)Q.nE * m2 * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(ctx, cudaStreamSynchronize(st));
    for (int g = 0; g < 2 * Q.D + 1; ++g) {
      int d = g - Q.D, ad = std::abs(d);
      for (int mu = 0; mu < H.m0; ++mu)
        for (int nu = 0; nu < H.m0; ++nu) {
          int src = (d >= 0) ? (mu * H.m0 + nu) : (nu * H.m0 + mu);
          if (Hout) Hout[(size_t)g * m2 + mu * H.m0 + nu] = th[(size_t)ad * m2 + src];
          if (Sout) Sout[(size_t)g * m2 + mu * H.m0 + nu] = ts[(size_t)ad * m2 + src];
        }
    }
    if (bound_rc)
      for (int e = 0; e < Q.nE; ++e) { bound_rc[2 * e] = Q.Ek[e]; bound_rc[2 * e + 1] = Q.Em[e]; }
    return FOCK_OK;
  }
  // periodic: A_k = combine of the per-axis factors at offsets (k1, k2, k3)
  const int ncell = H.L[0] * H.L[1] * H.L[2];
  const size_t xs = (size_t)H.nF * m2;
  double *zero = nullptr, *gh = nullptr, *gs = nullptr;
  CombineTask* dt = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&zero, xs * 8));
  CUDA_TRY(ctx, cudaMalloc(&gh, (size_t)ncell * m2 * 8));
  CUDA_TRY(ctx, cudaMalloc(&gs, (size_t)ncell * m2 * 8));
  CUDA_TRY(ctx, cudaMalloc(&dt, (size_t)ncell * sizeof(CombineTask)));
  CUDA_TRY(ctx, cudaMemsetAsync(zero, 0, xs * 8, st));
  std::vector<const double*> fx[3];
  for (int a = 0; a < 3; ++a) {
    fx[a].assign(H.L[a], zero);
    const AxisPlan& A = B.ap[a];
    if (H.per[a]) {
      for (size_t o = 0; o < A.offs.size(); ++o) fx[a][A.offs[o]] = Q.X[a] + o * xs;
    } else {
      fx[a][0] = Q.X[a];
    }
  }
  std::vector<CombineTask> ct(ncell);
  for (int kb = 0; kb < ncell; ++kb) {
    int k3 = kb % H.L[2], k2 = (kb / H.L[2]) % H.L[1], k1 = kb / (H.L[1] * H.L[2]);
    CombineTask& c = ct[kb];
    std::memset(&c, 0, sizeof(c));
    c.prob = 0; c.X0 = fx[0][k1]; c.X1 = fx[1][k2]; c.X2 = fx[2][k3];
    c.outH = gh + (size_t)kb * m2; c.outS = gs + (size_t)kb * m2;
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(dt, ct.data(), ct.size() * sizeof(CombineTask), cudaMemcpyHostToDevice, st));
  launch_combine(B.d_probs, dt, ncell, st);
  if (Hout) CUDA_TRY(ctx, cudaMemcpyAsync(Hout, gh, (size_t)ncell * m2 * 8, cudaMemcpyDeviceToHost, st));
  if (Sout) CUDA_TRY(ctx, cudaMemcpyAsync(Sout, gs, (size_t)ncell * m2 * 8, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  cudaFree(zero); cudaFree(gh); cudaFree(gs); cudaFree(dt);
  return FOCK_OK;
}

namespace {
// Fourier indices [j0, j1) of an assembled periodic problem: eigenvalues
// sorted (ties by index) into evals / block_of, and optionally the block
// eigenvectors [j - j0][i][mu] (complex, interleaved) into vecs; host outputs.
int periodic_range(fock_ctx* ctx, Batch& B, int j0, int j1, double* evals, int* block_of, double* vecs) {
  const HostProb& H = B.hp[0];
  const int nj = j1 - j0, n = nj * H.m0;
  if (n == 0) return FOCK_OK;
  ProfBind pb(ctx);
  cudaStream_t st = ctx->stream;
  { PROF("k_axis_dft", 1); launch_axis_dft(B.d_probs, B.d_dft, (int)B.dft.size(), B.maxLdft, st); }
  { PROF("k_null_tau", 1); launch_null_tau(B.d_nulls, (int)B.nulls.size(), st); }
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  char* mem = nullptr;
  const size_t off_blk = ((size_t)n * 8 + 255) & ~(size_t)255;
  const size_t off_pv = off_blk + (((size_t)n * 4 + 255) & ~(size_t)255);
  const size_t off_pi = off_pv + (size_t)n2 * 8;
  const size_t off_t = (off_pi + (size_t)n2 * 4 + 255) & ~(size_t)255;
  const size_t off_v = (off_t + sizeof(FBlockTask) + 255) & ~(size_t)255;
  const size_t vbytes = vecs ? (size_t)n * H.m0 * sizeof(cplx) : 0;
  CUDA_TRY(ctx, cudaMalloc(&mem, off_v + vbytes));
  double* ev = (double*)mem;
  int* blk = (int*)(mem + off_blk);
  FBlockTask f = B.fbp[0];
  f.j0 = j0; f.nj = nj; f.outH = nullptr; f.outS = nullptr; f.want = 1; f.ev = ev; f.blk = blk; f.fail = nullptr;
  f.vecs = vecs ? (cplx*)(mem + off_v) : nullptr;
  int rc = FOCK_OK;
  cudaError_t e = cudaMemcpyAsync(mem + off_t, &f, sizeof(f), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    { PROF("k_fblocks_eig", 1);
      launch_fblocks(B.d_probs, (const FBlockTask*)(mem + off_t), 1, nj, H.m0, st, vecs != nullptr); }
    { PROF("k_sort_global", 1); launch_sort_global(ev, blk, n, (double*)(mem + off_pv), (int*)(mem + off_pi), st); }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(evals, ev, (size_t)n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && block_of) e = cudaMemcpyAsync(block_of, blk, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && vecs) e = cudaMemcpyAsync(vecs, mem + off_v, vbytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) rc = set_err(ctx, FOCK_ECUDA, cudaGetErrorString(e));
  cudaFree(mem);
  return rc;
}
}  // namespace

int fock_circulant_eig(fock_ctx* ctx, const fock_blocks* b, double* evals, int* block_of, double* evecs) {
  if (!ctx || !b || !evals) return FOCK_EINVAL;
  Batch& B = const_cast<Batch&>(b->B);
  if (B.hp[0].kind != 0) return set_err(ctx, FOCK_EINVAL, "not a periodic problem");
  const HostProb& H = B.hp[0];
  if (evecs) return periodic_range(ctx, B, 0, H.L[0] * H.L[1] * H.L[2], evals, block_of, evecs);
  ProfBind pb(ctx);
  run_periodic(ctx, B);
  const Batch::PerProb& Q = B.pp[0];
  int fail = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(evals, Q.ev, Q.nev * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (block_of) CUDA_TRY(ctx, cudaMemcpyAsync(block_of, Q.blk, Q.nev * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(&fail, Q.fail, 4, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (fail) return set_err(ctx, FOCK_EINVAL, "a Fourier-block mass matrix was not positive definite");
  return FOCK_OK;
}

int fock_circulant_eig_range(fock_ctx* ctx, const fock_blocks* b, int j0, int j1, double* evals,
                             int* block_of) {
  if (!ctx || !b || !evals) return FOCK_EINVAL;
  Batch& B = const_cast<Batch&>(b->B);
  if (B.hp[0].kind != 0) return set_err(ctx, FOCK_EINVAL, "not a periodic problem");
  const HostProb& H = B.hp[0];
  const int ncell = H.L[0] * H.L[1] * H.L[2];
  if (j0 < 0 || j1 < j0 || j1 > ncell) return set_err(ctx, FOCK_EINVAL, "need 0 <= j0 <= j1 <= |L|");
  return periodic_range(ctx, B, j0, j1, evals, block_of, nullptr);
}

int fock_bloch_vectors(fock_ctx* ctx, const fock_blocks* b, int nsel, const int* jbar, const int* rank,
                       double* U) {
  if (!ctx || !b || nsel < 0 || (nsel && (!jbar || !rank || !U))) return FOCK_EINVAL;
  Batch& B = const_cast<Batch&>(b->B);
  if (B.hp[0].kind != 0) return set_err(ctx, FOCK_EINVAL, "not a periodic problem");
  const HostProb& H = B.hp[0];
  const int ncell = H.L[0] * H.L[1] * H.L[2], m0 = H.m0;
  if (!nsel) return FOCK_OK;
  // distinct Fourier indices: one single-block task each
  std::vector<int> blocks_needed, slot(nsel);
  for (int c = 0; c < nsel; ++c) {
    if (jbar[c] < 0 || jbar[c] >= ncell || rank[c] < 0 || rank[c] >= m0)
      return set_err(ctx, FOCK_EINVAL, "bloch_vectors: Fourier index or rank out of range");
    auto it = std::find(blocks_needed.begin(), blocks_needed.end(), jbar[c]);
    const int q = (int)(it - blocks_needed.begin());
    if (it == blocks_needed.end()) blocks_needed.push_back(jbar[c]);
    slot[c] = q * m0 + rank[c];   // column of that block's eigenvector array
  }
  const int nd = (int)blocks_needed.size();
  ProfBind pb(ctx);
  cudaStream_t st = ctx->stream;
  { PROF("k_axis_dft", 1); launch_axis_dft(B.d_probs, B.d_dft, (int)B.dft.size(), B.maxLdft, st); }
  { PROF("k_null_tau", 1); launch_null_tau(B.d_nulls, (int)B.nulls.size(), st); }
  std::vector<FBlockTask> tasks(nd);
  const size_t nbv = (size_t)ncell * m0;
  const size_t off_ev = 0, off_y = ((size_t)nd * m0 * 8 + 255) & ~(size_t)255;
  const size_t off_t = (off_y + (size_t)nd * m0 * m0 * sizeof(cplx) + 255) & ~(size_t)255;
  const size_t off_i = (off_t + nd * sizeof(FBlockTask) + 255) & ~(size_t)255;
  const size_t off_u = (off_i + 2 * (size_t)nsel * sizeof(int) + 255) & ~(size_t)255;
  char* mem = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&mem, off_u + nbv * nsel * sizeof(cplx)));
  for (int q = 0; q < nd; ++q) {
    FBlockTask f = B.fbp[0];
    f.j0 = blocks_needed[q]; f.nj = 1; f.outH = nullptr; f.outS = nullptr; f.want = 1;
    f.ev = (double*)(mem + off_ev) + (size_t)q * m0; f.blk = nullptr; f.fail = nullptr;
    f.vecs = (cplx*)(mem + off_y) + (size_t)q * m0 * m0;
    tasks[q] = f;
  }
  std::vector<int> ibuf(2 * (size_t)nsel);
  for (int c = 0; c < nsel; ++c) { ibuf[c] = jbar[c]; ibuf[nsel + c] = slot[c]; }
  int rc = FOCK_OK;
  cudaError_t e = cudaMemcpyAsync(mem + off_t, tasks.data(), nd * sizeof(FBlockTask), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mem + off_i, ibuf.data(), ibuf.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    { PROF("k_fblocks_eig", 1); launch_fblocks(B.d_probs, (const FBlockTask*)(mem + off_t), nd, 1, m0, st, true); }
    { PROF("k_bloch_vectors", 1);
      launch_bloch_vectors(H.L[0], H.L[1], H.L[2], m0, nsel, (const int*)(mem + off_i), (const cplx*)(mem + off_y),
                           (const int*)(mem + off_i) + nsel, (cplx*)(mem + off_u), st); }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(U, mem + off_u, nbv * nsel * sizeof(cplx), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) rc = set_err(ctx, FOCK_ECUDA, cudaGetErrorString(e));
  cudaFree(mem);
  return rc;
}

int fock_split_dgemm(fock_ctx* ctx, int M, int N, int K, const double* A, long long a_m, long long a_k,
                     const double* B, long long b_k, long long b_n, double* C, long long c_m, long long c_n,
                     double alpha, double beta, int ksplit, int sym) {
  if (!ctx || M < 0 || N < 0 || K < 0 || (M && N && (!A || !B || !C)) || ksplit < 1 || ksplit > 1024 ||
      (sym && M != N))
    return FOCK_EINVAL;
  if (!M || !N) return FOCK_OK;
  cudaStream_t st = ctx->stream;
  SplitTask t;
  std::memset(&t, 0, sizeof(t));
  t.M = M; t.N = N; t.K = K; t.A = A; t.a_m = a_m; t.a_k = a_k; t.B = B; t.b_k = b_k; t.b_n = b_n;
  t.C = C; t.c_m = c_m; t.c_n = c_n; t.alpha = alpha; t.beta = beta;
  t.ksplit = ksplit; t.sym = sym ? 1 : 0;
  const bool red = ksplit > 1 || sym;
  char* mem = nullptr;
  const size_t wbytes = red ? (size_t)ksplit * M * N * sizeof(double) : 0;
  CUDA_TRY(ctx, cudaMalloc(&mem, 256 + sizeof(SplitTask) + 256 + wbytes));
  if (red) t.work = (double*)(mem + 512 + ((sizeof(SplitTask) + 255) & ~(size_t)255));
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(mem, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mem + 256, &t, sizeof(t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    { ProfBind pb(ctx); PROF("k_split_gemm", 1);
      launch_split_gemm((const SplitTask*)(mem + 256), 1, M, N, (int*)mem, st, ksplit, red); }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, mem, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(mem);
  if (e != cudaSuccess) return set_err(ctx, FOCK_ECUDA, cudaGetErrorString(e));
  if (herr) return set_err(ctx, FOCK_ETIMEOUT, "split_dgemm: a tensor-core commit did not complete in time");
  return FOCK_OK;
}

int fock_toeplitz_matvec(fock_ctx* ctx, const fock_blocks* b, int which, const double* x, double* y,
                         int nvec, int on_device) {
  if (!ctx || !b || !x || !y || nvec <= 0 || (which != FOCK_OP_H && which != FOCK_OP_S)) return FOCK_EINVAL;
  const Batch& B = b->B;
  const HostProb& H = B.hp[0];
  if (H.kind != 1) return set_err(ctx, FOCK_EINVAL, "matvec needs a box chain");
  const Batch::PerProb& Q = B.pp[0];
  cudaStream_t st = ctx->stream;
  const int n = Q.Lc * H.m0;
  const size_t nbytes = (size_t)n * nvec * 8;
  if (on_device && (const char*)x < (const char*)y + nbytes && (const char*)y < (const char*)x + nbytes)
    return set_err(ctx, FOCK_EINVAL, "matvec: device x and y must not overlap");
  double *dx = nullptr, *dy = nullptr;
  cplx *X = nullptr, *Y = nullptr;
  char* tasks = nullptr;
  if (on_device) { dx = const_cast<double*>(x); dy = y; }
  else {
    CUDA_TRY(ctx, cudaMalloc(&dx, nbytes));
    CUDA_TRY(ctx, cudaMalloc(&dy, nbytes));
    CUDA_TRY(ctx, cudaMemcpyAsync(dx, x, nbytes, cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(ctx, cudaMalloc(&X, (size_t)Q.M * H.m0 * nvec * sizeof(cplx)));
  CUDA_TRY(ctx, cudaMalloc(&Y, (size_t)Q.M * H.m0 * nvec * sizeof(cplx)));
  CUDA_TRY(ctx, cudaMalloc(&tasks, 4096));
  int cc = std::max(1, std::min(16, 98304 / (32 * Q.M)));
  FftTask tf; std::memset(&tf, 0, sizeof(tf));
  tf.prob = 0; tf.L = Q.Lc; tf.m0 = H.m0; tf.ncol = nvec; tf.circ = B.d_circs + Q.circ; tf.x = dx; tf.ldx = n;
  tf.X = X; tf.cc = cc;
  FftTask ti = tf; ti.x = nullptr; ti.X = Y; ti.y = dy; ti.ldy = n; ti.beta = 0.0;
  BmulTask bm = {0, Q.M, H.m0, nvec, which == FOCK_OP_H ? Q.CHo : Q.CSo, nullptr, X, Y, nullptr};
  EApplyTask ea;
  std::memset(&ea, 0, sizeof(ea));
  ea.prob = 0; ea.m0 = H.m0; ea.ncol = nvec; ea.nrows = Q.nErows; ea.rows = Q.Erows; ea.rowptr = Q.Erowptr;
  ea.cols = Q.Ecols; ea.vals = which == FOCK_OP_H ? Q.EH : Q.ES; ea.x = dx; ea.ldx = n; ea.y = dy; ea.ldy = n;
  char hbuf[4096];
  std::memcpy(hbuf, &tf, sizeof(tf));
  std::memcpy(hbuf + 512, &ti, sizeof(ti));
  std::memcpy(hbuf + 1024, &bm, sizeof(bm));
  std::memcpy(hbuf + 1536, &ea, sizeof(ea));
  CUDA_TRY(ctx, cudaMemcpyAsync(tasks, hbuf, 2048, cudaMemcpyHostToDevice, st));
  int chunks = (H.m0 * ((nvec + 1) / 2) + cc - 1) / cc;
  launch_fft((const FftTask*)tasks, 1, chunks, Q.M, cc, +1, st, false);
  launch_blockmul((const BmulTask*)(tasks + 1024), 1, Q.M, H.m0, st, false);
  launch_fft((const FftTask*)(tasks + 512), 1, chunks, Q.M, cc, -1, st, false);
  if (Q.nE) launch_eapply((const EApplyTask*)(tasks + 1536), 1, eapply_grid((long long)Q.nErows * H.m0 * nvec), st);
  if (!on_device) CUDA_TRY(ctx, cudaMemcpyAsync(y, dy, nbytes, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(ctx, cudaStreamSynchronize(st));
  CUDA_TRY(ctx, cudaGetLastError());
  if (!on_device) { cudaFree(dx); cudaFree(dy); }
  cudaFree(X); cudaFree(Y); cudaFree(tasks);
  return FOCK_OK;
}

int fock_box_eig(fock_ctx* ctx, const fock_blocks* b, int k, double tol, int maxit, double* evals,
                 double* evecs, int* iters) {
  if (!ctx || !b || !evals) return FOCK_EINVAL;
  Batch& B = const_cast<Batch&>(b->B);
  if (B.hp[0].kind != 1) return set_err(ctx, FOCK_EINVAL, "not a box problem");
  if (k <= 0 || k > B.lob[0].kw) return set_err(ctx, FOCK_EINVAL, "k exceeds the planned k_eig");
  ProfBind pb(ctx);
  std::vector<int> it, conv;
  std::vector<double> res;
  int rc = run_lobpcg(ctx, B, tol > 0 ? tol : 1e-10, maxit > 0 ? maxit : FOCK_DEFAULT_MAXIT, it, res, conv);
  if (rc) return rc;
  const Batch::Lob& l = B.lob[0];
  CUDA_TRY(ctx, cudaMemcpyAsync(evals, l.lam, (size_t)k * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (evecs) {   // back to the original basis: (I_L (x) Xc) V'
    const Batch::PerProb& Q = B.pp[0];
    launch_cell_back(Q.Xc, B.hp[0].m0, Q.Lc, k, l.Y, l.T1, l.n, ctx->stream);
    CUDA_TRY(ctx, cudaMemcpyAsync(evecs, l.T1, (size_t)l.n * k * 8, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (iters) *iters = it[0];
  if (!conv[0]) return set_err(ctx, FOCK_ENOCONV, "maxit reached");
  return FOCK_OK;
}

}  // extern "C"
