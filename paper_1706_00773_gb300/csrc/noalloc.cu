// noalloc.cu -- eig_secular_values_static: the eigenvalue stage of the update
// (deflation, root count at every pole, zero finder, merge) for callers that
// must not allocate device memory.
//
// Who needs it: a caller whose device memory is entirely owned by another
// manager (a framework's caching allocator, or a serving process that reserves
// HBM up front), and a latency-critical loop that cannot afford cudaMalloc /
// cudaFree (cudaFree synchronises the whole device).  Such a caller passes its
// own inputs and outputs; every temporary buffer of this entry point lives in
// one file-scope device array of fixed size, so nothing is allocated per call.
//
// Costs and rules of that choice:
//   - every GPU that loads this library holds kStaticBytes (6 MiB) of device
//     memory for the array until the process exits;
//   - problems larger than EIG_STATIC_MAX_N (or k > EIG_MAX_K) are rejected with
//     EIG_ETOOBIG;
//   - all calls share the one array, and it keeps the previous call's contents:
//     the status block and the work counter are cleared at the start of each
//     call, everything else is fully rewritten before it is read;
//   - calls whose work overlaps on the GPU (two streams, or two host threads)
//     race on the array and give wrong results: serialise them;
//   - the first call on a device does the set-up (looks up the array's device
//     address with cudaGetSymbolAddress, with that device current); make that
//     first call before any stream capture.  The address is kept together
//     with the device's current context: after cudaDeviceReset (which
//     reloads the module, so the array may move) the next call sees a new
//     context and does the set-up again instead of using a stale address.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "eig_internal.cuh"

using namespace eig;

namespace {

constexpr size_t kStaticBytes = size_t(6) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_eig_scratch[kStaticBytes];

std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// cuCtxGetCurrent from the driver, through the runtime (no link-time
// dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

constexpr size_t al(size_t v) { return (v + 255) / 256 * 256; }

// Byte size of the carve below for a padded rank K and leading dimension ld.
constexpr size_t scratch_bytes(size_t ld, size_t K) {
  return al(sizeof(DevStatus)) + al(4 * sizeof(int)) + al(8 * ld) /*lam_keep*/ +
         al(8 * ld * K) /*Us*/ + al(4 * ld) /*idx_keep*/ + al(4 * ld) /*idx_defl*/ +
         al(8 * ld) /*lam_defl*/ + al(4 * ld) /*pole_cnt*/ + al(4 * ld) /*origin*/ +
         al(8 * ld) /*tau*/ + al(4 * ld) /*iters*/ + al(4 * ld) /*flags*/ + al(8 * ld * K) /*alpha*/ +
         al(16 * ld) /*beta*/ + al(8 * ld) /*sidx*/ + al(8 * ld) /*mu_sec*/ +
         2 * al(8 * ld * K) /*U copy, run reflectors*/ + al(8 * ld) /*their scalars*/ + al(4 * ld) /*runs*/;
}
static_assert(scratch_bytes(EIG_STATIC_MAX_N, EIG_MAX_K) <= kStaticBytes,
              "static scratch too small for EIG_STATIC_MAX_N");

// Device address of the array on the current device (set up once per device).
int scratch_for_current_device(char** base, int* num_sms) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EIG_ECUDA;
  }
  // The device's context (cudaSetDevice initialises it when needed): the
  // cached address belongs to the context it was looked up in.
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return EIG_ECUDA;
  }
  CtxGetCurrentFn get_ctx = ctx_get_current();
  CUcontext ctx = nullptr;
  if (!get_ctx || get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return EIG_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_eig_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return EIG_ECUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return EIG_ECUDA;
    }
    g_scratch_dev[dev] = p;
    g_scratch_ctx[dev] = ctx;
    g_sms[dev] = sms;
  }
  *base = static_cast<char*>(g_scratch_dev[dev]);
  *num_sms = g_sms[dev];
  return EIG_OK;
}

#define CKS(x)                \
  do {                        \
    if ((x) != cudaSuccess) { \
      cudaGetLastError();     \
      return EIG_ECUDA;       \
    }                         \
  } while (0)

}  // namespace

extern "C" int eig_secular_values_static(int64_t n, int32_t k, const double* lambda,
                                         const double* U, const int8_t* sigma, double* mu,
                                         int32_t* iters, int32_t max_iter, void* stream) {
  if (n < 1 || k < 1 || !lambda || !U || !mu || max_iter < 0) return EIG_EINVAL;
  if (n > EIG_STATIC_MAX_N || k > EIG_MAX_K) return EIG_ETOOBIG;
  unsigned long long negmask = 0;
  int kplus = 0;
  if (!sigma_info(sigma, k, &negmask, &kplus)) return EIG_EINVAL;
  char* base = nullptr;
  int num_sms = 0;
  int rc = scratch_for_current_device(&base, &num_sms);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = padded_rank(k);
  const size_t ld = (size_t)((n + 31) / 32 * 32);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += al(bytes);
    return p;
  };
  DevStatus* st = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  int* counter = reinterpret_cast<int*>(take(4 * sizeof(int)));
  double* lam_keep = reinterpret_cast<double*>(take(8 * ld));
  double* Us = reinterpret_cast<double*>(take(8 * ld * K));
  int* idx_keep = reinterpret_cast<int*>(take(4 * ld));
  int* idx_defl = reinterpret_cast<int*>(take(4 * ld));
  double* lam_defl = reinterpret_cast<double*>(take(8 * ld));
  int* pole_cnt = reinterpret_cast<int*>(take(4 * ld));
  RootOut ro;
  ro.origin = reinterpret_cast<int*>(take(4 * ld));
  ro.tau = reinterpret_cast<double*>(take(8 * ld));
  ro.iters = reinterpret_cast<int*>(take(4 * ld));
  ro.flags = reinterpret_cast<int*>(take(4 * ld));
  ro.alpha = reinterpret_cast<double*>(take(8 * ld * K));
  ro.beta = reinterpret_cast<double*>(take(16 * ld));
  ro.sidx = reinterpret_cast<int*>(take(8 * ld));
  double* mu_sec = reinterpret_cast<double*>(take(8 * ld));
  double* Ur = reinterpret_cast<double*>(take(8 * ld * K));
  double* Vr = reinterpret_cast<double*>(take(8 * ld * K));
  double* taur = reinterpret_cast<double*>(take(8 * ld));
  int* runs = reinterpret_cast<int*>(take(4 * ld));
  if (off > kStaticBytes) return EIG_ETOOBIG;  // cannot happen (static_assert above)

  // The array keeps the last call's contents: clear what must start at zero.
  CKS(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
  CKS(cudaMemsetAsync(counter, 0, sizeof(int), s));
  // runs of equal lambda are rotated in a copy of U (the caller's U is input only)
  CKS(cudaMemcpyAsync(Ur, U, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, s));
  CKS(launch_runs_qr(n, k, lambda, Ur, Vr, taur, runs, st, s));
  CKS(launch_deflate(n, k, K, lambda, Ur, negmask, lam_keep, Us, (int)ld, idx_keep, idx_defl,
                     lam_defl, st, s));
  Sub sub;
  sub.n_dev = &st->n_keep;
  sub.ld = (int)ld;
  sub.K = K;
  sub.kplus = kplus + (K - k);
  sub.lam = lam_keep;
  sub.Us = Us;
  sub.idx = idx_keep;
  sub.st = st;
  sub.negmask = negmask;
  CKS(launch_counts(sub, nullptr, (int)ld, pole_cnt, s));
  CKS(launch_roots(sub, pole_cnt, max_iter ? max_iter : 128, counter, ro, st, num_sms, s));
  CKS(launch_assemble(sub, ro, n, idx_defl, lam_defl, st, mu_sec, mu, nullptr, s));
  if (iters) CKS(launch_scatter_iters(sub, n, ro.iters, lam_defl, mu_sec, iters, s));
  DevStatus host_st;
  CKS(cudaMemcpyAsync(&host_st, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  CKS(cudaStreamSynchronize(s));
  return status_of(host_st);
}
