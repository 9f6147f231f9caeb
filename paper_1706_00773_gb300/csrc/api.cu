// api.cu -- host side of the C ABI declared in include/eig_update.h: argument
// checks, workspace management, stage orchestration on one stream, tickets.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "eig_internal.cuh"

using namespace eig;

namespace {

constexpr int kDefaultMaxIter = 128;
constexpr int kCheckCols = 16;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Ticket {
  cudaEvent_t done = nullptr;
  DevStatus* host = nullptr;   // pinned copy of the device status at completion
  double* chk_host = nullptr;  // pinned copy of the check results (may be null)
  int64_t n = 0;
  int32_t k = 0;
  int32_t pre_status = EIG_OK;  // host-side failure before launch
  bool report = false;
};

// Sub-buffers of one update, carved from the handle's workspace.
struct Carve {
  double* U = nullptr;
  double* lam_keep = nullptr;
  double* Us = nullptr;
  int* idx_keep = nullptr;
  int* idx_defl = nullptr;
  double* lam_defl = nullptr;
  int* pole_cnt = nullptr;
  int* origin = nullptr;
  double* tau = nullptr;
  int* iters = nullptr;
  int* rflags = nullptr;
  double* alpha = nullptr;
  double* beta = nullptr;
  int* sidx = nullptr;
  double* mu_sec = nullptr;
  int* counter = nullptr;
  double* lam_old = nullptr;
  double* W = nullptr;
  double* X = nullptr;
  __nv_bfloat16* Qs = nullptr;   // mixed mode: slices of Q
  __nv_bfloat16* Ws = nullptr;   // mixed mode: slices of W
  int* erow = nullptr;
  int* fcol = nullptr;
  unsigned long long* rmax = nullptr;
  double* chk_tmp = nullptr;
  double* chk_out = nullptr;
  int* chk_cols = nullptr;
  DevStatus* st = nullptr;
  size_t bytes = 0;
};

Carve plan(char* base, int64_t n, int k, bool vectors, bool xbuf, bool report, bool mixed = false) {
  Carve c;
  const int K = padded_rank(k);
  const size_t ld = align_up((size_t)n, 32);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off = align_up(off + bytes, 256);
    return p;
  };
  c.st = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  c.counter = reinterpret_cast<int*>(take(sizeof(int) * 4));
  c.U = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * k));
  c.lam_keep = reinterpret_cast<double*>(take(sizeof(double) * ld));
  c.Us = reinterpret_cast<double*>(take(sizeof(double) * ld * K));
  c.idx_keep = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.idx_defl = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.lam_defl = reinterpret_cast<double*>(take(sizeof(double) * ld));
  c.pole_cnt = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.origin = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.tau = reinterpret_cast<double*>(take(sizeof(double) * ld));
  c.iters = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.rflags = reinterpret_cast<int*>(take(sizeof(int) * ld));
  c.alpha = reinterpret_cast<double*>(take(sizeof(double) * ld * K));
  c.beta = reinterpret_cast<double*>(take(sizeof(double) * ld * 2));
  c.sidx = reinterpret_cast<int*>(take(sizeof(int) * ld * 2));
  c.mu_sec = reinterpret_cast<double*>(take(sizeof(double) * ld));
  c.lam_old = reinterpret_cast<double*>(take(sizeof(double) * ld));
  if (report) {
    c.chk_tmp = reinterpret_cast<double*>(take(sizeof(double) * 3 * (size_t)n * kCheckCols));
    c.chk_out = reinterpret_cast<double*>(take(sizeof(double) * (kCheckCols + kCheckCols * kCheckCols)));
    c.chk_cols = reinterpret_cast<int*>(take(sizeof(int) * kCheckCols));
  }
  if (vectors && mixed) {
    const size_t planes = (size_t)tc_num_slices() * tc_slice_plane((int)n);
    c.Qs = reinterpret_cast<__nv_bfloat16*>(take(2 * planes));
    c.Ws = reinterpret_cast<__nv_bfloat16*>(take(2 * planes));
    c.erow = reinterpret_cast<int*>(take(sizeof(int) * ld));
    c.fcol = reinterpret_cast<int*>(take(sizeof(int) * ld));
    c.rmax = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * ld));
  } else if (vectors) {
    c.W = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * n));
  }
  if (vectors && xbuf) c.X = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * n));
  c.bytes = off;
  return c;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int status_of(const DevStatus& s) {
  if (s.flags & (ST_UNSORTED | ST_NONFINITE)) return EIG_EINVAL;
  if (s.flags & ST_TIMEOUT) return EIG_ETIMEOUT;
  if (s.flags & ST_NOTCONV) return EIG_ENOTCONV;
  return EIG_OK;
}

}  // namespace

struct eig_ctx {
  int device = 0;
  uint32_t mode = EIG_FP64;
  uint64_t budget = 0;
  int max_iter = kDefaultMaxIter;
  int num_sms = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  DevStatus* st_host = nullptr;  // pinned
  double* chk_host = nullptr;    // pinned
  cudaEvent_t ev[9] = {};
  cudaStream_t last_stream = nullptr;
  int last_launches = 0;
  bool last_pending = false;
  std::mutex mu;
  std::vector<Ticket> tickets;
};

namespace {

int ensure_ws(eig_ctx* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return EIG_OK;
  if (h->budget && bytes > h->budget) return EIG_ENOMEM;
  if (h->ws) {
    // Work already queued on other streams may still use the old buffer.
    cudaDeviceSynchronize();
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return EIG_ENOMEM;
  }
  h->ws = static_cast<char*>(p);
  h->ws_bytes = bytes;
  return EIG_OK;
}

bool sigma_info(const int8_t* sigma, int k, unsigned long long* negmask, int* kplus) {
  unsigned long long m = 0;
  int kp = 0;
  for (int c = 0; c < k; ++c) {
    const int v = sigma ? sigma[c] : 1;
    if (v == 1) {
      ++kp;
    } else if (v == -1) {
      m |= 1ull << c;
    } else {
      return false;
    }
  }
  *negmask = m;
  *kplus = kp;
  return true;
}

#define CK(x)                         \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) {          \
      cudaGetLastError();             \
      return EIG_ECUDA;               \
    }                                 \
  } while (0)

// Stages a2-a9 (+ the optional check) of one update, stream-ordered.  With
// ev != nullptr, events 0..8 are recorded at the stage boundaries.
int enqueue_update(eig_ctx* h, const eig_problem* P, const Carve& c, cudaStream_t s,
                   unsigned long long negmask, int kplus_k, cudaEvent_t* ev, int* launches) {
  int nl = 0;
#define MARK(i) \
  if (ev) CK(cudaEventRecord(ev[i], s))
  const int64_t n = P->n;
  const int k = P->k;
  const int K = padded_rank(k);
  const int ld = (int)align_up((size_t)n, 32);
  const bool vectors = (P->want & EIG_VECTORS) != 0;
  const bool report = (P->want & EIG_REPORT) != 0;
  const bool mixed = vectors && h->mode == EIG_MIXED;
  MARK(0);
  CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
  CK(launch_project_f64(n, k, P->Q, P->K, c.U, s));
  ++nl;
  CK(cudaMemcpyAsync(c.lam_old, P->lambda, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  MARK(1);
  CK(launch_deflate(n, k, K, P->lambda, c.U, negmask, c.lam_keep, c.Us, ld, c.idx_keep,
                    c.idx_defl, c.lam_defl, c.st, s));
  ++nl;
  MARK(2);
  Sub sub;
  sub.n_dev = &c.st->n_keep;
  sub.ld = ld;
  sub.K = K;
  sub.kplus = kplus_k + (K - k);
  sub.lam = c.lam_keep;
  sub.Us = c.Us;
  sub.idx = c.idx_keep;
  sub.st = c.st;
  sub.negmask = negmask;
  CK(launch_counts(sub, nullptr, ld, c.pole_cnt, s));
  ++nl;
  MARK(3);
  CK(cudaMemsetAsync(c.counter, 0, sizeof(int), s));
  RootOut ro{c.origin, c.tau, c.iters, c.rflags, c.alpha, c.beta, c.sidx};
  CK(launch_roots(sub, c.pole_cnt, h->max_iter, c.counter, ro, c.st, h->num_sms, s));
  ++nl;
  MARK(4);
  WSlices ws;
  if (mixed) {
    ws.Ws = c.Ws;
    ws.plane = tc_slice_plane((int)n);
    ws.lds = tc_slice_ld((int)n);
    ws.fcol = c.fcol;
    CK(cudaMemsetAsync(c.Ws, 0, 2 * (size_t)tc_num_slices() * ws.plane, s));
  } else if (vectors) {
    CK(cudaMemsetAsync(c.W, 0, sizeof(double) * (size_t)n * n, s));
  }
  // lam_old keeps the old eigenvalues, so the new ones go straight into lambda.
  CK(launch_assemble(sub, ro, n, c.idx_defl, c.lam_defl, c.st, c.mu_sec, P->lambda,
                     (vectors && !mixed) ? c.W : nullptr, s, ws));
  nl += 3;
  MARK(5);
  if (vectors) {
    double* Xdst = P->Q_out ? P->Q_out : c.X;
    if (mixed) {
      CK(launch_slice_q((int)n, P->Q, c.rmax, c.erow, c.Qs, c.st, s));
      MARK(6);
      CK(launch_gemm_tc((int)n, c.Qs, c.Ws, c.erow, c.fcol, Xdst, (int)n, c.st, &c.st->flags, s));
      nl += 3;
    } else {
      MARK(6);
      CK(launch_gemm_f64_guarded(n, n, n, P->Q, n, c.W, n, Xdst, n, c.st, s));
      ++nl;
    }
    MARK(7);
    if (report) {
      int cols[kCheckCols];
      const int nc = (int)(n < kCheckCols ? n : kCheckCols);
      for (int i = 0; i < nc; ++i) cols[i] = (int)((int64_t)i * (n - 1) / (nc > 1 ? nc - 1 : 1));
      CK(cudaMemcpyAsync(c.chk_cols, cols, sizeof(int) * nc, cudaMemcpyHostToDevice, s));
      CK(launch_check_pairs(n, k, P->Q, c.lam_old, P->K, negmask, Xdst, P->lambda, c.chk_cols, nc,
                            c.chk_tmp, c.chk_out, s));
      nl += 6;
    }
    if (!P->Q_out) {
      CK(launch_copy_guarded(P->Q, c.X, n * n, c.st, s));
      ++nl;
    }
  } else {
    MARK(6);
    MARK(7);
  }
  MARK(8);
#undef MARK
  if (launches) *launches = nl;
  return EIG_OK;
}

void fill_report(eig_report* rep, const eig_problem* P, const DevStatus& st, const double* chk,
                 int status) {
  std::memset(rep, 0, sizeof(*rep));
  rep->n = P->n;
  rep->k = P->k;
  rep->status = status;
  rep->n_deflated = st.n_defl;
  rep->iters_total = st.iters_total;
  rep->iters_max = st.iters_max;
  rep->n_notconv = st.n_notconv;
  rep->norm_A = st.lam_absmax + st.fro2;
  if (chk) {
    const int nc = (int)(P->n < kCheckCols ? P->n : kCheckCols);
    double r = 0.0, o = 0.0;
    for (int i = 0; i < nc; ++i) r = std::fmax(r, chk[i]);
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) {
        const double g = chk[nc + a + b * nc] - (a == b ? 1.0 : 0.0);
        o = std::fmax(o, std::fabs(g));
      }
    rep->n_checked = nc;
    rep->max_residual = r;
    rep->max_orth = o;
  }
}

int validate(const eig_problem* P, unsigned long long* negmask, int* kplus) {
  if (!P || P->n < 1 || P->k < 1 || P->k > EIG_MAX_K || !P->Q || !P->lambda || !P->K)
    return EIG_EINVAL;
  if (P->n > (int64_t)0x3fffffff) return EIG_EINVAL;
  if (P->Q_out && P->Q_out == P->Q) return EIG_EINVAL;
  if (!sigma_info(P->sigma, P->k, negmask, kplus)) return EIG_EINVAL;
  return EIG_OK;
}

}  // namespace

extern "C" {

const char* eig_version(void) { return "eigupdate-gb300 0.1 (sm_103a)"; }

int eig_update_init(const eig_init_params* params, eig_handle* out) {
  if (!out) return EIG_EINVAL;
  *out = nullptr;
  eig_init_params p{};
  if (params) p = *params;
  if (p.flags != 0 || (p.mode != EIG_FP64 && p.mode != EIG_MIXED) || p.max_iter < 0)
    return EIG_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p.device < 0 || p.device >= ndev) {
    cudaGetLastError();
    return EIG_ECUDA;
  }
  eig_ctx* h = new (std::nothrow) eig_ctx();
  if (!h) return EIG_ENOMEM;
  h->device = p.device;
  h->mode = p.mode;
  h->budget = p.hbm_budget;
  h->max_iter = p.max_iter ? p.max_iter : kDefaultMaxIter;
  DeviceGuard g(h->device);
  if (!g.ok || cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
      cudaMallocHost(&h->st_host, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&h->chk_host, sizeof(double) * (kCheckCols + kCheckCols * kCheckCols)) != cudaSuccess ||
      [&]() {
        for (auto& e : h->ev)
          if (cudaEventCreate(&e) != cudaSuccess) return true;
        return false;
      }()) {
    cudaGetLastError();
    eig_update_destroy(h);
    return EIG_ECUDA;
  }
  *out = h;
  return EIG_OK;
}

int eig_update_destroy(eig_handle h) {
  if (!h) return EIG_OK;
  {
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    for (Ticket& t : h->tickets) {
      if (t.done) cudaEventDestroy(t.done);
      if (t.host) cudaFreeHost(t.host);
      if (t.chk_host) cudaFreeHost(t.chk_host);
    }
    if (h->ws) cudaFree(h->ws);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->chk_host) cudaFreeHost(h->chk_host);
    for (auto& e : h->ev)
      if (e) cudaEventDestroy(e);
    cudaGetLastError();
  }
  delete h;
  return EIG_OK;
}

int eig_update_rank_k(eig_handle h, eig_problem* P, eig_report* rep, void* stream) {
  if (!h) return EIG_EINVAL;
  unsigned long long negmask = 0;
  int kplus = 0;
  int rc = validate(P, &negmask, &kplus);
  if (rc) return rc;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vectors = (P->want & EIG_VECTORS) != 0;
  const bool report = (P->want & EIG_REPORT) != 0 && vectors;
  eig_problem Pe = *P;
  if (!report) Pe.want &= ~EIG_REPORT;
  const bool mixed = h->mode == EIG_MIXED;
  const size_t need = plan(nullptr, P->n, P->k, vectors, P->Q_out == nullptr, report, mixed).bytes;
  rc = ensure_ws(h, need);
  if (rc) return rc;
  Carve c = plan(h->ws, P->n, P->k, vectors, P->Q_out == nullptr, report, mixed);
  rc = enqueue_update(h, &Pe, c, s, negmask, kplus, rep ? h->ev : nullptr, &h->last_launches);
  if (rc) return rc;
  h->last_stream = s;
  if (P->want & EIG_ASYNC) {
    CK(cudaMemcpyAsync(h->st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    h->last_pending = true;
    return EIG_OK;
  }
  CK(cudaMemcpyAsync(h->st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  if (report)
    CK(cudaMemcpyAsync(h->chk_host, c.chk_out, sizeof(double) * (kCheckCols + kCheckCols * kCheckCols),
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->last_pending = false;
  const int status = status_of(*h->st_host);
  if (rep) {
    fill_report(rep, P, *h->st_host, report ? h->chk_host : nullptr, status);
    auto span = [&](int a, int b) -> double {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
      }
      return ms;
    };
    rep->ms_total = span(0, 8);
    rep->ms_project = span(0, 1);
    rep->ms_deflate = span(1, 2);
    rep->ms_counts = span(2, 3);
    rep->ms_roots = span(3, 4);
    rep->ms_assemble = span(4, 5);
    rep->ms_slice = span(5, 6);
    rep->ms_gemm = span(6, 7);
    rep->launches = h->last_launches;
  }
  return status;
}

int eig_update_batch(eig_handle h, int32_t count, eig_problem* probs, uint64_t* tickets,
                     void* stream) {
  if (!h || count < 0 || (count > 0 && (!probs || !tickets))) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // One workspace large enough for every problem, so that no reallocation
  // happens while earlier problems are in flight.
  size_t need = 0;
  for (int i = 0; i < count; ++i) {
    const eig_problem* P = &probs[i];
    if (P->n < 1 || P->k < 1) continue;
    const bool vectors = (P->want & EIG_VECTORS) != 0;
    const bool report = (P->want & EIG_REPORT) != 0 && vectors;
    size_t b = plan(nullptr, P->n, P->k, vectors, P->Q_out == nullptr, report, h->mode == EIG_MIXED).bytes;
    if (b > need) need = b;
  }
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) {
    eig_problem Pe = probs[i];
    Ticket t;
    t.n = Pe.n;
    t.k = Pe.k;
    unsigned long long negmask = 0;
    int kplus = 0;
    t.pre_status = validate(&Pe, &negmask, &kplus);
    const bool vectors = (Pe.want & EIG_VECTORS) != 0;
    t.report = (Pe.want & EIG_REPORT) != 0 && vectors;
    if (!t.report) Pe.want &= ~EIG_REPORT;
    if (cudaMallocHost(&t.host, sizeof(DevStatus)) != cudaSuccess ||
        cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return EIG_ENOMEM;
    }
    std::memset(t.host, 0, sizeof(DevStatus));
    if (t.report && cudaMallocHost(&t.chk_host, sizeof(double) * (kCheckCols + kCheckCols * kCheckCols)) != cudaSuccess) {
      cudaGetLastError();
      return EIG_ENOMEM;
    }
    if (t.pre_status == EIG_OK) {
      Carve c = plan(h->ws, Pe.n, Pe.k, vectors, Pe.Q_out == nullptr, t.report, h->mode == EIG_MIXED);
      int nl = 0;
      t.pre_status = enqueue_update(h, &Pe, c, s, negmask, kplus, nullptr, &nl);
      if (t.pre_status == EIG_OK) {
        CK(cudaMemcpyAsync(t.host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
        if (t.report)
          CK(cudaMemcpyAsync(t.chk_host, c.chk_out, sizeof(double) * (kCheckCols + kCheckCols * kCheckCols),
                             cudaMemcpyDeviceToHost, s));
      }
    }
    CK(cudaEventRecord(t.done, s));
    std::lock_guard<std::mutex> lk(h->mu);
    h->tickets.push_back(t);
    tickets[i] = (uint64_t)h->tickets.size();  // 1-based
  }
  h->last_stream = s;
  return EIG_OK;
}

int eig_update_query(eig_handle h, int32_t what, const void* in, void* out, size_t out_bytes) {
  if (!h) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  switch (what) {
    case EIG_Q_STATUS:
    case EIG_Q_REPORT: {
      if (!in) return EIG_EINVAL;
      const uint64_t id = *static_cast<const uint64_t*>(in);
      Ticket t;
      {
        std::lock_guard<std::mutex> lk(h->mu);
        if (id < 1 || id > h->tickets.size()) return EIG_EINVAL;
        t = h->tickets[id - 1];
      }
      int status = t.pre_status;
      if (status == EIG_OK) {
        const cudaError_t q = cudaEventQuery(t.done);
        if (q == cudaErrorNotReady) {
          cudaGetLastError();
          status = EIG_EBUSY;
        } else if (q != cudaSuccess) {
          cudaGetLastError();
          status = EIG_ECUDA;
        } else {
          status = status_of(*t.host);
        }
      }
      if (what == EIG_Q_STATUS) {
        if (!out || out_bytes < sizeof(int32_t)) return EIG_EINVAL;
        *static_cast<int32_t*>(out) = status;
        return status;
      }
      if (!out || out_bytes < sizeof(eig_report)) return EIG_EINVAL;
      if (status == EIG_EBUSY) return EIG_EBUSY;
      eig_problem P{};
      P.n = t.n;
      P.k = t.k;
      fill_report(static_cast<eig_report*>(out), &P, *t.host, t.report ? t.chk_host : nullptr, status);
      return status;
    }
    case EIG_Q_LAST_STATUS: {
      if (!out || out_bytes < sizeof(int32_t)) return EIG_EINVAL;
      if (h->last_pending) {
        if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) {
          cudaGetLastError();
          return EIG_ECUDA;
        }
        h->last_pending = false;
      }
      const int status = status_of(*h->st_host);
      *static_cast<int32_t*>(out) = status;
      return status;
    }
    case EIG_Q_WORKSPACE: {
      const eig_problem* P = static_cast<const eig_problem*>(in);
      if (!P || !out || out_bytes < sizeof(uint64_t) || P->n < 1 || P->k < 1 || P->k > EIG_MAX_K)
        return EIG_EINVAL;
      const bool vectors = (P->want & EIG_VECTORS) != 0;
      *static_cast<uint64_t*>(out) = plan(nullptr, P->n, P->k, vectors, P->Q_out == nullptr,
                                          (P->want & EIG_REPORT) && vectors, h->mode == EIG_MIXED)
                                         .bytes;
      return EIG_OK;
    }
    case EIG_Q_COUNT: {
      const eig_count_args* a = static_cast<const eig_count_args*>(in);
      if (!a || a->n < 1 || a->k < 1 || a->k > EIG_MAX_K || a->npts < 0 || !a->lambda || !a->U ||
          (a->npts > 0 && (!a->x || !a->counts)))
        return EIG_EINVAL;
      unsigned long long negmask = 0;
      int kplus = 0;
      if (!sigma_info(a->sigma, a->k, &negmask, &kplus)) return EIG_EINVAL;
      if (a->npts == 0) return EIG_OK;
      const int K = padded_rank(a->k);
      const int ld = (int)align_up((size_t)a->n, 32);
      const size_t need = plan(nullptr, a->n, a->k, false, false, false).bytes;
      int rc = ensure_ws(h, need);
      if (rc) return rc;
      Carve c = plan(h->ws, a->n, a->k, false, false, false);
      cudaStream_t s = static_cast<cudaStream_t>(a->stream);
      CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
      CK(launch_prepare_undeflated(a->n, a->k, K, a->lambda, a->U, c.lam_keep, c.Us, ld,
                                   c.idx_keep, c.st, s));
      Sub sub;
      sub.n_dev = &c.st->n_keep;
      sub.ld = ld;
      sub.K = K;
      sub.kplus = kplus + (K - a->k);
      sub.lam = c.lam_keep;
      sub.Us = c.Us;
      sub.idx = c.idx_keep;
      sub.st = c.st;
      sub.negmask = negmask;
      CK(launch_counts(sub, a->x, a->npts, a->counts, s));
      CK(cudaStreamSynchronize(s));
      return EIG_OK;
    }
    default:
      return EIG_EINVAL;
  }
}

int eig_project(eig_handle h, int64_t n, int32_t k, const double* Q, const double* K, double* U,
                void* stream) {
  if (!h || n < 1 || k < 1 || !Q || !K || !U) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  CK(launch_project_f64(n, k, Q, K, U, static_cast<cudaStream_t>(stream)));
  return EIG_OK;
}

int eig_secular_values(eig_handle h, int64_t n, int32_t k, const double* lambda, const double* U,
                       const int8_t* sigma, double* mu, int32_t* iters, void* stream) {
  if (!h || n < 1 || k < 1 || k > EIG_MAX_K || !lambda || !U || !mu || n > (int64_t)0x3fffffff)
    return EIG_EINVAL;
  unsigned long long negmask = 0;
  int kplus = 0;
  if (!sigma_info(sigma, k, &negmask, &kplus)) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int K = padded_rank(k);
  const int ld = (int)align_up((size_t)n, 32);
  const size_t need = plan(nullptr, n, k, false, false, false).bytes;
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  Carve c = plan(h->ws, n, k, false, false, false);
  CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
  CK(launch_deflate(n, k, K, lambda, U, negmask, c.lam_keep, c.Us, ld, c.idx_keep, c.idx_defl,
                    c.lam_defl, c.st, s));
  Sub sub;
  sub.n_dev = &c.st->n_keep;
  sub.ld = ld;
  sub.K = K;
  sub.kplus = kplus + (K - k);
  sub.lam = c.lam_keep;
  sub.Us = c.Us;
  sub.idx = c.idx_keep;
  sub.st = c.st;
  sub.negmask = negmask;
  CK(launch_counts(sub, nullptr, ld, c.pole_cnt, s));
  CK(cudaMemsetAsync(c.counter, 0, sizeof(int), s));
  RootOut ro{c.origin, c.tau, c.iters, c.rflags, c.alpha, c.beta, c.sidx};
  CK(launch_roots(sub, c.pole_cnt, h->max_iter, c.counter, ro, c.st, h->num_sms, s));
  CK(launch_assemble(sub, ro, n, c.idx_defl, c.lam_defl, c.st, c.mu_sec, mu, nullptr, s));
  if (iters) CK(launch_scatter_iters(sub, n, c.iters, c.lam_defl, c.mu_sec, iters, s));
  CK(cudaMemcpyAsync(h->st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return status_of(*h->st_host);
}

int eig_make_rank2(int64_t n, int64_t j, const double* a, double* K, int8_t* sigma, void* stream) {
  if (n < 1 || j < 0 || j >= n || !a || !K || !sigma) return EIG_EINVAL;
  sigma[0] = 1;
  sigma[1] = -1;
  CK(launch_make_rank2(n, j, a, K, static_cast<cudaStream_t>(stream)));
  return EIG_OK;
}

}  // extern "C"
