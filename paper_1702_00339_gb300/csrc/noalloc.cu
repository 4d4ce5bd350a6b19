// y = H x or S x for an assembled box chain without any device allocation.
//
// The allocating matvec entry point obtains its FFT work arrays with
// cudaMalloc on every call.  Some callers cannot do that: real-time loops
// that forbid allocator calls (and the device-wide synchronisation cudaFree
// implies) once they are running, and hosts whose own memory allocator owns
// the whole device, where a second allocator would compete for its memory.
// This variant keeps the forward transform, the per-frequency block products
// and the launch descriptors in one file-scope device array of fixed size
// (FOCK_NOALLOC_SCRATCH_BYTES), which every GPU that loads the library holds
// until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/fock.h"
#include "common.cuh"

namespace fock {
int blocks_matvec_view(const fock_blocks* b, MatvecView* v);
void set_ctx_error(fock_ctx* c, const char* msg);
void launch_fft(const FftTask*, int, int, int, int, int, cudaStream_t, bool);
void launch_blockmul(const BmulTask*, int, int, int, cudaStream_t, bool);
void launch_eapply(const EApplyTask*, int, int, cudaStream_t);
int eapply_grid(long long items);
}  // namespace fock

using namespace fock;

namespace {

constexpr size_t kDescBytes = 4096;   // launch descriptors at the start of the array
constexpr size_t kDescSlot = 256;     // one slot per descriptor, four slots used
static_assert(sizeof(FftTask) <= kDescSlot, "FftTask outgrew its descriptor slot");
static_assert(sizeof(BmulTask) <= kDescSlot, "BmulTask outgrew its descriptor slot");
static_assert(sizeof(EApplyTask) <= kDescSlot, "EApplyTask outgrew its descriptor slot");
static_assert(4 * kDescSlot <= kDescBytes, "descriptor slots exceed the descriptor area");

// The whole scratch of the entry point: descriptors, then the two complex
// work arrays (forward transform, block products).
static __device__ __align__(256) unsigned char g_noalloc_scratch[FOCK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the array for `dev` (looked up once per device, with the
// device current; the first call on a device must not be inside a stream
// capture).  The cached address belongs to the device's primary context and
// stays valid while that context lives, i.e. for the process unless the
// caller resets the device.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return FOCK_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return FOCK_ECUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FOCK_OK;
}

}  // namespace

extern "C" int fock_toeplitz_matvec_noalloc(fock_ctx* ctx, const fock_blocks* b, int which,
                                            const double* x, double* y, int nvec) {
  if (!ctx || !b || !x || !y || nvec <= 0 || (which != FOCK_OP_H && which != FOCK_OP_S))
    return FOCK_EINVAL;
  MatvecView v;
  if (blocks_matvec_view(b, &v) != FOCK_OK) {
    set_ctx_error(ctx, "matvec_noalloc: needs an assembled box chain");
    return FOCK_EINVAL;
  }
  const size_t work = (size_t)v.M * v.m0 * nvec;          // complex entries per work array
  if (kDescBytes + 2 * work * sizeof(cplx) > FOCK_NOALLOC_SCRATCH_BYTES) {
    set_ctx_error(ctx, "matvec_noalloc: M*m0*nvec exceeds the fixed scratch "
                       "(2*M*m0*nvec*16 + 4096 bytes must fit FOCK_NOALLOC_SCRATCH_BYTES)");
    return FOCK_EINVAL;
  }
  const int n = v.Lc * v.m0;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  const size_t bytes = (size_t)n * nvec * sizeof(double);
  if (xb < yb + bytes && yb < xb + bytes) {   // y is written before the boundary blocks read x
    set_ctx_error(ctx, "matvec_noalloc: x and y must not overlap");
    return FOCK_EINVAL;
  }
  // the caller's current device is restored on every return
  struct DeviceGuard {
    int prev = -1;
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
  } guard;
  if (cudaGetDevice(&guard.prev) != cudaSuccess) guard.prev = -1;
  if (cudaSetDevice(v.device) != cudaSuccess) return FOCK_ECUDA;
  void* base = nullptr;
  int rc = scratch_address(v.device, &base);
  if (rc) {
    set_ctx_error(ctx, "matvec_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return rc;
  }
  char* s = (char*)base;
  cplx* X = (cplx*)(s + kDescBytes);
  cplx* Y = X + work;
  const int cc = std::max(1, std::min(16, 98304 / (32 * v.M)));
  FftTask tf;
  std::memset(&tf, 0, sizeof(tf));
  tf.prob = 0; tf.L = v.Lc; tf.m0 = v.m0; tf.ncol = nvec; tf.circ = v.circ; tf.x = x; tf.ldx = n;
  tf.X = X; tf.cc = cc;
  FftTask ti = tf;
  ti.x = nullptr; ti.X = Y; ti.y = y; ti.ldy = n; ti.beta = 0.0;
  BmulTask bm = {0, v.M, v.m0, nvec, which == FOCK_OP_H ? v.CH : v.CS, nullptr, X, Y, nullptr};
  EApplyTask ea;
  std::memset(&ea, 0, sizeof(ea));
  ea.prob = 0; ea.m0 = v.m0; ea.ncol = nvec; ea.nrows = v.nErows; ea.rows = v.Erows; ea.rowptr = v.Erowptr;
  ea.cols = v.Ecols; ea.vals = which == FOCK_OP_H ? v.EH : v.ES; ea.x = x; ea.ldx = n; ea.y = y; ea.ldy = n;
  unsigned char desc[4 * kDescSlot];
  std::memcpy(desc, &tf, sizeof(tf));
  std::memcpy(desc + kDescSlot, &ti, sizeof(ti));
  std::memcpy(desc + 2 * kDescSlot, &bm, sizeof(bm));
  std::memcpy(desc + 3 * kDescSlot, &ea, sizeof(ea));
  if (cudaMemcpyAsync(s, desc, sizeof(desc), cudaMemcpyHostToDevice, v.stream) != cudaSuccess) {
    set_ctx_error(ctx, "matvec_noalloc: descriptor copy failed");
    return FOCK_ECUDA;
  }
  const int chunks = (v.m0 * ((nvec + 1) / 2) + cc - 1) / cc;
  launch_fft((const FftTask*)s, 1, chunks, v.M, cc, +1, v.stream, false);
  launch_blockmul((const BmulTask*)(s + 2 * kDescSlot), 1, v.M, v.m0, v.stream, false);
  launch_fft((const FftTask*)(s + kDescSlot), 1, chunks, v.M, cc, -1, v.stream, false);
  if (v.nE)
    launch_eapply((const EApplyTask*)(s + 3 * kDescSlot), 1, eapply_grid((long long)v.nErows * v.m0 * nvec), v.stream);
  cudaError_t e = cudaStreamSynchronize(v.stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_ctx_error(ctx, cudaGetErrorString(e));
    return FOCK_ECUDA;
  }
  return FOCK_OK;
}
