// api.cu -- host side of the C ABI declared in include/eig_update.h: argument
// checks, workspace management, stage orchestration on one stream, tickets.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <new>
#include <vector>

#include "eig_internal.cuh"

using namespace eig;

namespace {

constexpr int kDefaultMaxIter = 128;
constexpr int kCheckCols = 16;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Completion resources of one eig_update_batch call, shared by its tickets
// and freed when the last of them is released.
struct BatchRes {
  cudaEvent_t done = nullptr;  // recorded after the call's last launch
  DevStatus* host = nullptr;   // pinned: one device status per problem of the call
  int live = 0;                // tickets of the call not released yet
};

// One problem of a batch.  Its id is (gen << 32) | (index + 1): a released
// slot is reused with gen + 1, so an id is never valid twice.
struct Ticket {
  int batch = -1;               // index into eig_ctx::batches
  int slot = 0;                 // status slot in the batch's pinned block
  int64_t n = 0;
  int32_t k = 0;
  int32_t pre_status = EIG_OK;  // host-side failure before launch
  uint32_t gen = 0;
  bool live = false;
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
  double* Vr = nullptr;  // runs of equal lam: reflectors, scalars, (g0, m) list
  double* taur = nullptr;
  int* runs = nullptr;
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
  c.Vr = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * k));
  c.taur = reinterpret_cast<double*>(take(sizeof(double) * ld));
  c.runs = reinterpret_cast<int*>(take(sizeof(int) * ld));
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
  bool last_counted = true;  // the last rank_k call's outcome is in the metrics
  // EIG_Q_METRICS counters (batch tickets are resolved when queried)
  int64_t m_calls = 0, m_updates = 0, m_pairs = 0, m_ok = 0, m_failed = 0, m_launches = 0, m_allocs = 0;
  int64_t m_unread = 0;  // EIG_ASYNC updates superseded before their status was read
  std::mutex mu;
  std::vector<Ticket> tickets;
  std::vector<int> free_tickets;
  std::vector<BatchRes> batches;
  std::vector<int> free_batches;
  // Class-concurrent schedule: one stream per rank class, fork/join events.
  static constexpr int kAux = 12;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t aux_fork = nullptr;
  cudaEvent_t aux_join[kAux] = {};
  bool aux_ready = false;
  // Side stream: the BF16 slicing of Q (mixed mode) overlaps the secular stages.
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
  bool side_ready = false;
  // Batch schedule tuner (EIG_TUNE): best schedule per batch signature,
  // optionally persisted in the file named by EIG_TUNE_CACHE.
  bool tune = false;
  std::map<std::string, Sched> tuned;
  std::string tune_file;
  int64_t m_tune_trials = 0, m_tune_hits = 0;
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
  ++h->m_allocs;
  return EIG_OK;
}

// Streams and events of the class-concurrent schedule (created on first use).
bool ensure_aux(eig_ctx* h) {
  if (h->aux_ready) return true;
  for (int i = 0; i < eig_ctx::kAux; ++i) {
    if (!h->aux[i] && cudaStreamCreateWithFlags(&h->aux[i], cudaStreamNonBlocking) != cudaSuccess) break;
    if (!h->aux_join[i] && cudaEventCreateWithFlags(&h->aux_join[i], cudaEventDisableTiming) != cudaSuccess) break;
    if (i == eig_ctx::kAux - 1) h->aux_ready = true;
  }
  if (h->aux_ready && !h->aux_fork && cudaEventCreateWithFlags(&h->aux_fork, cudaEventDisableTiming) != cudaSuccess)
    h->aux_ready = false;
  if (!h->aux_ready) cudaGetLastError();
  return h->aux_ready;
}

bool ensure_side(eig_ctx* h) {
  if (h->side_ready) return true;
  if ((h->side || cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) == cudaSuccess) &&
      (h->side_fork || cudaEventCreateWithFlags(&h->side_fork, cudaEventDisableTiming) == cudaSuccess) &&
      (h->side_join || cudaEventCreateWithFlags(&h->side_join, cudaEventDisableTiming) == cudaSuccess))
    h->side_ready = true;
  else
    cudaGetLastError();
  return h->side_ready;
}

// The tuner's cache file: one line per batch signature, "key streams order occ_div".
void load_tune_cache(eig_ctx* h) {
  const char* f = std::getenv("EIG_TUNE_CACHE");
  if (!f || !*f) return;
  h->tune_file = f;
  FILE* fp = std::fopen(f, "r");
  if (!fp) return;
  char key[512];
  int a = 0, b = 0, c = 0;
  while (std::fscanf(fp, "%511s %d %d %d", key, &a, &b, &c) == 4) {
    Sched sc;
    sc.streams = a < 1 ? 1 : (a > eig_ctx::kAux ? eig_ctx::kAux : a);
    sc.order = b ? 1 : 0;
    sc.occ_div = c < 1 ? 1 : (c > 4 ? 4 : c);
    h->tuned[key] = sc;
  }
  std::fclose(fp);
}

void save_tune_entry(eig_ctx* h, const std::string& key, const Sched& sc) {
  if (h->tune_file.empty()) return;
  FILE* fp = std::fopen(h->tune_file.c_str(), "a");
  if (!fp) return;
  std::fprintf(fp, "%s %d %d %d\n", key.c_str(), sc.streams, sc.order, sc.occ_div);
  std::fclose(fp);
}

// The CUDA call behind the calling thread's last EIG_ECUDA (eig_last_cuda_error).
thread_local int t_cuda_err = 0;
thread_local char t_cuda_call[192] = {0};

void note_cuda(cudaError_t e, const char* call, int line) {
  t_cuda_err = (int)e;
  std::snprintf(t_cuda_call, sizeof(t_cuda_call), "api.cu:%d %s", line, call);
}

#define CK(x)                             \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) {              \
      note_cuda(e_, #x, __LINE__);        \
      cudaGetLastError();                 \
      return EIG_ECUDA;                   \
    }                                     \
  } while (0)

// ---------------------------------------------------------------------------
// A table of updates and its workspace.  Every stage of every update of the
// table runs in one launch (one per padded rank K for the secular kernels):
// the device reads the ProbDesc table and per-stage prefix sums of the work.
// ---------------------------------------------------------------------------
struct TableItem {
  const eig_problem* P;
  unsigned long long negmask;
  int kplus;
  bool report;
};

struct Bump {
  char* base;
  size_t off = 0;
  explicit Bump(char* b) : base(b) {}
  char* take(size_t bytes, size_t align = 256) {
    off = align_up(off, align);
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

struct Table {
  // device pointers into the workspace
  ProbDesc* d_desc = nullptr;
  int* d_ids = nullptr;
  long long* d_colpre = nullptr;
  int* d_rbpre = nullptr;
  int* d_slpre = nullptr;
  int* d_gtpre = nullptr;
  long long* d_cppre = nullptr;
  void* d_maps = nullptr;
  DevStatus* d_st = nullptr;
  double* d_W = nullptr;
  size_t W_bytes = 0;
  __nv_bfloat16* d_Ws = nullptr;
  size_t Ws_bytes = 0;
  unsigned long long* d_rmax = nullptr;
  size_t rmax_bytes = 0;
  unsigned* d_wnz = nullptr;  // non-zero maps of W's leading slices (mixed mode)
  size_t wnz_bytes = 0;
  std::vector<ClassDesc> classes;
  std::vector<int> class_items;  // sum of n per class (grid bound)
  long long total_cols = 0, total_copy = 0;
  int64_t max_n = 0;
  int total_rb = 0, total_sl = 0, total_gt = 0;
  bool any_errors = false;  // some update wants the per-eigenpair report
  // report (single update only)
  double* chk_tmp = nullptr;
  double* chk_out = nullptr;
  int* chk_cols = nullptr;
  size_t table_bytes = 0;  // size of the packed host image
  size_t bytes = 0;        // workspace bytes
};

// Lays out (base == nullptr: sizes only) or builds the table.  host_img
// receives the packed image of the table region (copied to d_desc).
Table layout_table(eig_ctx* h, const std::vector<TableItem>& items, char* base, bool vectors, bool mixed,
                   std::vector<char>* host_img) {
  Table T;
  const int count = (int)items.size();
  Bump b(base);
  // --- table region (packed, copied from the host image in one transfer) ---
  const size_t t0 = b.off;
  T.d_desc = reinterpret_cast<ProbDesc*>(b.take(sizeof(ProbDesc) * count));
  T.d_ids = reinterpret_cast<int*>(b.take(sizeof(int) * count));
  T.d_colpre = reinterpret_cast<long long*>(b.take(sizeof(long long) * (count + 1)));
  T.d_rbpre = reinterpret_cast<int*>(b.take(sizeof(int) * (count + 1)));
  T.d_slpre = reinterpret_cast<int*>(b.take(sizeof(int) * (count + 1)));
  T.d_gtpre = reinterpret_cast<int*>(b.take(sizeof(int) * (count + 1)));
  T.d_cppre = reinterpret_cast<long long*>(b.take(sizeof(long long) * (count + 1)));
  T.d_maps = b.take(mixed && vectors ? (size_t)128 * 2 * count : 0, 128);
  T.table_bytes = b.off - t0;
  // --- class scratch (device-written) ---
  int cls_of[17];
  for (int i = 0; i < 17; ++i) cls_of[i] = -1;
  std::vector<int> order;  // table indices grouped by class
  for (int K : {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16}) {
    int c = -1;
    for (int i = 0; i < count; ++i) {
      if (padded_rank(items[i].P->k) != K) continue;
      if (c < 0) {
        c = (int)T.classes.size();
        cls_of[K] = c;
        ClassDesc cd{};
        cd.K = K;
        cd.ids = T.d_ids ? T.d_ids + order.size() : nullptr;
        T.classes.push_back(cd);
        T.class_items.push_back(0);
      }
      order.push_back(i);
      T.classes[c].count++;
      T.class_items[c] += (int)items[i].P->n;
    }
  }
  for (size_t ci = 0; ci < T.classes.size(); ++ci) {
    ClassDesc& cd = T.classes[ci];
    cd.perm = reinterpret_cast<int*>(b.take(sizeof(int) * (size_t)T.class_items[ci]));
    cd.pk = reinterpret_cast<int*>(b.take(sizeof(int) * (cd.count + 1)));
    cd.pd = reinterpret_cast<int*>(b.take(sizeof(int) * (cd.count + 1)));
    cd.counter = reinterpret_cast<int*>(b.take(sizeof(int) * 3));
  }
  // --- shared contiguous regions ---
  T.d_st = reinterpret_cast<DevStatus*>(b.take(sizeof(DevStatus) * count));
  size_t Wtot = 0, Wstot = 0, rtot = 0, ztot = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t n = items[i].P->n;
    Wtot += sizeof(double) * (size_t)n * n;
    Wstot += 2 * (size_t)tc_num_slices() * tc_slice_plane((int)n);
    rtot += sizeof(unsigned long long) * (size_t)n;
    ztot += sizeof(unsigned) * wnz_words((int)n);
  }
  if (vectors && !mixed) {
    T.d_W = reinterpret_cast<double*>(b.take(Wtot));
    T.W_bytes = Wtot;
  }
  if (vectors && mixed) {
    T.d_Ws = reinterpret_cast<__nv_bfloat16*>(b.take(Wstot));
    T.Ws_bytes = Wstot;
    T.d_rmax = reinterpret_cast<unsigned long long*>(b.take(rtot));
    T.rmax_bytes = rtot;
    T.d_wnz = reinterpret_cast<unsigned*>(b.take(ztot));
    T.wnz_bytes = ztot;
  }
  // --- per-update regions ---
  std::vector<ProbDesc> desc(count);
  std::vector<long long> colpre(count + 1, 0), cppre(count + 1, 0);
  std::vector<int> rbpre(count + 1, 0), slpre(count + 1, 0), gtpre(count + 1, 0);
  size_t woff = 0, wsoff = 0, roff = 0, woff2 = 0;
  for (int i = 0; i < count; ++i) {
    const eig_problem* P = items[i].P;
    const int64_t n = P->n;
    const int k = P->k;
    const int K = padded_rank(k);
    const size_t ld = align_up((size_t)n, 32);
    ProbDesc& d = desc[i];
    std::memset(&d, 0, sizeof(d));
    d.n = (int)n;
    d.k = k;
    d.K = K;
    d.ld = (int)ld;
    d.kplus = items[i].kplus + (K - k);
    d.negmask = items[i].negmask;
    d.Q = P->Q;
    d.lam = P->lambda;
    d.Km = P->K;
    d.st = T.d_st ? T.d_st + i : nullptr;
    d.U = reinterpret_cast<double*>(b.take(sizeof(double) * (size_t)n * k));
    d.lam_keep = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.Us = reinterpret_cast<double*>(b.take(sizeof(double) * ld * K));
    d.idx_keep = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.idx_defl = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.lam_defl = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.pole_cnt = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.origin = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.tau = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.iters = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.rflags = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.alpha = reinterpret_cast<double*>(b.take(sizeof(double) * ld * K));
    d.beta = reinterpret_cast<double*>(b.take(sizeof(double) * ld * 2));
    d.sidx = reinterpret_cast<int*>(b.take(sizeof(int) * ld * 2));
    d.mu_sec = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.lam_old = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.Vr = reinterpret_cast<double*>(b.take(sizeof(double) * (size_t)n * k));
    d.taur = reinterpret_cast<double*>(b.take(sizeof(double) * ld));
    d.runs = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
    d.errors = vectors ? P->errors : nullptr;
    // Products for the one-warp ranks only: with K >= 10 each warp multiplies
    // just its own rows (t = r u for a quarter of them), and the product loads
    // cost more than they save (measured k = 16: 83 -> 86 ms).
    d.Pp = warps_per_root(K) == 1 ? reinterpret_cast<double*>(b.take(sizeof(double) * ld * (size_t)(K * (K + 1) / 2)))
                                  : nullptr;
    if (d.errors) T.any_errors = true;
    if (n > T.max_n) T.max_n = n;
    if (mixed) {  // K split for the double-float projection
      d.Kh = reinterpret_cast<float*>(b.take(sizeof(float) * (size_t)n * k));
      d.Kl = reinterpret_cast<float*>(b.take(sizeof(float) * (size_t)n * k));
      d.Kexp = reinterpret_cast<int*>(b.take(sizeof(int) * 16));
    }
    if (mixed) {  // FP32 copies for the coarse phase of the zero finder
      d.lamf = reinterpret_cast<float2*>(b.take(sizeof(float2) * ld));
      d.Usf = reinterpret_cast<float*>(b.take(sizeof(float) * ld * K));
      d.Ulo = vectors ? reinterpret_cast<float*>(b.take(sizeof(float) * ld * K)) : nullptr;
    }
    if (vectors) {
      if (mixed) {
        d.Qs = reinterpret_cast<__nv_bfloat16*>(b.take(2 * (size_t)tc_num_slices() * tc_slice_plane((int)n)));
        d.Ws = T.d_Ws ? reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(T.d_Ws) + wsoff) : nullptr;
        wsoff += 2 * (size_t)tc_num_slices() * tc_slice_plane((int)n);
        d.erow = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
        d.fcol = reinterpret_cast<int*>(b.take(sizeof(int) * ld));
        d.rmax = T.d_rmax ? reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(T.d_rmax) + roff) : nullptr;
        roff += sizeof(unsigned long long) * (size_t)n;
        d.wnz = T.d_wnz ? reinterpret_cast<unsigned*>(reinterpret_cast<char*>(T.d_wnz) + woff2) : nullptr;
        woff2 += sizeof(unsigned) * wnz_words((int)n);
      } else {
        d.W = T.d_W ? reinterpret_cast<double*>(reinterpret_cast<char*>(T.d_W) + woff) : nullptr;
        woff += sizeof(double) * (size_t)n * n;
      }
      if (P->Q_out) {
        d.Xout = P->Q_out;
      } else {
        d.Xout = reinterpret_cast<double*>(b.take(sizeof(double) * (size_t)n * n));
        d.Qback = P->Q;
      }
    }
    if (items[i].report && count == 1) {
      T.chk_tmp = reinterpret_cast<double*>(b.take(sizeof(double) * 3 * (size_t)n * kCheckCols));
      T.chk_out = reinterpret_cast<double*>(b.take(sizeof(double) * (kCheckCols + kCheckCols * kCheckCols)));
      T.chk_cols = reinterpret_cast<int*>(b.take(sizeof(int) * kCheckCols));
    }
    colpre[i + 1] = colpre[i] + n;
    rbpre[i + 1] = rbpre[i] + (int)((n + 255) / 256);
    const int nt32 = (int)((n + 31) / 32);
    slpre[i + 1] = slpre[i] + nt32 * nt32;
    const int tile = mixed ? 128 : 64;
    const int ntg = (int)((n + tile - 1) / tile);
    gtpre[i + 1] = gtpre[i] + ntg * ntg;
    cppre[i + 1] = cppre[i] + ((vectors && !P->Q_out) ? n * n : 0);
  }
  T.total_cols = colpre[count];
  T.total_rb = rbpre[count];
  T.total_sl = slpre[count];
  T.total_gt = gtpre[count];
  T.total_copy = cppre[count];
  T.bytes = b.off;
  if (host_img && base) {
    host_img->assign(T.table_bytes, 0);
    char* img = host_img->data();
    auto put = [&](const void* dptr, const void* src, size_t bytes) {
      if (bytes) std::memcpy(img + (reinterpret_cast<const char*>(dptr) - reinterpret_cast<const char*>(T.d_desc)), src, bytes);
    };
    put(T.d_desc, desc.data(), sizeof(ProbDesc) * count);
    put(T.d_ids, order.data(), sizeof(int) * count);
    put(T.d_colpre, colpre.data(), sizeof(long long) * (count + 1));
    put(T.d_rbpre, rbpre.data(), sizeof(int) * (count + 1));
    put(T.d_slpre, slpre.data(), sizeof(int) * (count + 1));
    put(T.d_gtpre, gtpre.data(), sizeof(int) * (count + 1));
    put(T.d_cppre, cppre.data(), sizeof(long long) * (count + 1));
    if (mixed && vectors) {
      for (int i = 0; i < count; ++i) {
        char* mq = img + (reinterpret_cast<char*>(T.d_maps) - reinterpret_cast<char*>(T.d_desc)) + 256 * i;
        if (tc_encode_map(mq, desc[i].Qs, desc[i].n) != 0 || tc_encode_map(mq + 128, desc[i].Ws, desc[i].n) != 0)
          T.bytes = 0;  // signals failure
      }
    }
  }
  (void)h;
  (void)cls_of;
  return T;
}

// Stages a2-a11 (+ the optional check) of every update of the table,
// stream-ordered.  With ev != nullptr, events 0..8 mark the stage boundaries.
int enqueue_table(eig_ctx* h, const Table& T, int count, bool vectors, bool mixed, bool report,
                  cudaStream_t s, cudaEvent_t* ev, int* launches, const std::vector<char>& img,
                  const eig_problem* P0, unsigned long long negmask0, const Sched& sch = Sched()) {
  int nl = 0;
#define MARK(i) \
  if (ev) CK(cudaEventRecord(ev[i], s))
  MARK(0);
  CK(cudaMemcpyAsync(T.d_desc, img.data(), img.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(T.d_st, 0, sizeof(DevStatus) * count, s));
  CK(launch_project_grouped(T.d_desc, count, T.d_colpre, T.total_cols, s, mixed));
  CK(launch_runs_qr_grouped(T.d_desc, count, T.max_n, s));
  nl += mixed ? 3 : 2;
  MARK(1);
  CK(launch_deflate_grouped(T.d_desc, count, s));
  CK(launch_products_grouped(T.d_desc, count, T.d_colpre, T.total_cols, s));
  nl += 2;
  MARK(2);
  // Mixed mode: Q's BF16 digit slices depend on Q (and the rotation of runs
  // of equal lambda) only, so they are formed on the side stream while the
  // secular stages run (HBM-bound work next to FP64-bound work); the GEMM
  // waits for them.
  const bool side = vectors && mixed && sch.side && ensure_side(h);
  if (side) {
    CK(cudaEventRecord(h->side_fork, s));
    CK(cudaStreamWaitEvent(h->side, h->side_fork, 0));
    CK(launch_runs_rotate_q_grouped(T.d_desc, count, h->num_sms, h->side));
    CK(cudaMemsetAsync(T.d_rmax, 0, T.rmax_bytes, h->side));
    CK(launch_slice_q_grouped(T.d_desc, count, T.d_rbpre, T.total_rb, T.d_slpre, T.total_sl, h->side));
    nl += 4;
    CK(cudaEventRecord(h->side_join, h->side));
  }
  const int ncls = (int)T.classes.size();
  auto class_of = [&](int c) {
    ClassDesc cd = T.classes[c];
    if (!sch.order) cd.perm = nullptr;  // natural root order
    return cd;
  };
  if (sch.streams > 1 && ncls > 1 && h->aux_ready) {
    // Rank classes overlap: each runs its pole counts, zero finder and
    // assembly on its own stream (the classes touch disjoint updates), so the
    // tail of one class's persistent zero finder is filled by the others.
    if (vectors && mixed) CK(cudaMemsetAsync(T.d_Ws, 0, T.Ws_bytes, s));
    if (vectors && !mixed) CK(cudaMemsetAsync(T.d_W, 0, T.W_bytes, s));
    CK(cudaEventRecord(h->aux_fork, s));
    const int S = std::min(sch.streams, (int)eig_ctx::kAux);
    for (int c = 0; c < ncls; ++c) {
      cudaStream_t sc = h->aux[c % S];
      const ClassDesc cd = class_of(c);
      CK(cudaStreamWaitEvent(sc, h->aux_fork, 0));
      CK(launch_class_prefix(T.d_desc, cd, sc));
      CK(launch_counts_grouped(T.d_desc, cd, T.class_items[c], mixed, sc));
      CK(launch_order_roots_grouped(T.d_desc, cd, T.class_items[c], sc));
      CK(launch_roots_grouped(T.d_desc, cd, T.class_items[c], h->max_iter, h->num_sms, sc, sch.occ_div));
      CK(launch_assemble_grouped(T.d_desc, cd, T.class_items[c], T.class_items[c], vectors, mixed, sc));
      nl += (mixed ? 3 : 2) + (cd.perm ? 2 : 1) + 3;
      CK(cudaEventRecord(h->aux_join[c], sc));
    }
    for (int c = 0; c < ncls; ++c) CK(cudaStreamWaitEvent(s, h->aux_join[c], 0));
    MARK(3);
    MARK(4);
  } else {
    for (int c = 0; c < ncls; ++c) {
      CK(launch_class_prefix(T.d_desc, T.classes[c], s));
      CK(launch_counts_grouped(T.d_desc, T.classes[c], T.class_items[c], mixed, s));
      nl += mixed ? 3 : 2;
    }
    MARK(3);
    for (int c = 0; c < ncls; ++c) {
      const ClassDesc cd = class_of(c);
      CK(launch_order_roots_grouped(T.d_desc, cd, T.class_items[c], s));
      CK(launch_roots_grouped(T.d_desc, cd, T.class_items[c], h->max_iter, h->num_sms, s, sch.occ_div));
      nl += cd.perm ? 2 : 1;
    }
    MARK(4);
    if (vectors && mixed) CK(cudaMemsetAsync(T.d_Ws, 0, T.Ws_bytes, s));
    if (vectors && !mixed) CK(cudaMemsetAsync(T.d_W, 0, T.W_bytes, s));
    for (int c = 0; c < ncls; ++c) {
      CK(launch_assemble_grouped(T.d_desc, T.classes[c], T.class_items[c], T.class_items[c], vectors, mixed, s));
      nl += 3;
    }
  }
  if (vectors && T.any_errors) {
    CK(launch_errors_gap_grouped(T.d_desc, count, T.d_colpre, T.total_cols, s));
    ++nl;
  }
  MARK(5);
  if (vectors) {
    if (mixed) {
      if (side) {
        CK(cudaStreamWaitEvent(s, h->side_join, 0));
      } else {
        CK(launch_runs_rotate_q_grouped(T.d_desc, count, h->num_sms, s));
        CK(cudaMemsetAsync(T.d_rmax, 0, T.rmax_bytes, s));
        CK(launch_slice_q_grouped(T.d_desc, count, T.d_rbpre, T.total_rb, T.d_slpre, T.total_sl, s));
        nl += 4;
      }
      MARK(6);
      CK(launch_wnz_scan_grouped(T.d_desc, count, T.d_gtpre, T.total_gt, s));
      CK(launch_gemm_tc_grouped(T.d_desc, count, T.d_maps, T.d_gtpre, T.total_gt, s));
      nl += 2;
    } else {
      CK(launch_runs_apply_w_grouped(T.d_desc, count, h->num_sms, s));
      ++nl;
      MARK(6);
      CK(launch_gemm_f64_grouped(T.d_desc, count, T.d_gtpre, T.total_gt, s));
      ++nl;
    }
    MARK(7);
    if (report && count == 1) {
      const int64_t n = P0->n;
      int cols[kCheckCols];
      const int nc = (int)(n < kCheckCols ? n : kCheckCols);
      for (int i = 0; i < nc; ++i) cols[i] = (int)((int64_t)i * (n - 1) / (nc > 1 ? nc - 1 : 1));
      CK(cudaMemcpyAsync(T.chk_cols, cols, sizeof(int) * nc, cudaMemcpyHostToDevice, s));
      // The check needs the old lambda and this update's X (old Q is still intact).
      ProbDesc d0;
      std::memcpy(&d0, img.data(), sizeof(ProbDesc));
      CK(launch_check_pairs(n, P0->k, P0->Q, d0.lam_old, P0->K, negmask0, d0.Xout, P0->lambda,
                            T.chk_cols, nc, T.chk_tmp, T.chk_out, s));
      nl += 6;
    }
    if (T.total_copy > 0) {
      CK(launch_copyback_grouped(T.d_desc, count, T.d_cppre, T.total_copy, s));
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

// Batch signature for the tuner: mode, vectors, and per padded rank the
// number of updates and the size of their secular problems (log2 buckets).
std::string batch_signature(const std::vector<TableItem>& items, bool vectors, bool mixed) {
  int cnt[17] = {0};
  long long tot[17] = {0};
  for (const TableItem& it : items) {
    const int K = padded_rank(it.P->k);
    ++cnt[K];
    tot[K] += it.P->n;
  }
  auto lg = [](long long v) {
    int b = 0;
    while (v > 1) {
      v >>= 1;
      ++b;
    }
    return b;
  };
  std::string key = std::string(mixed ? "m" : "d") + (vectors ? "v" : "e");
  for (int K = 1; K <= 16; ++K)
    if (cnt[K]) key += "|" + std::to_string(K) + ":" + std::to_string(lg(cnt[K])) + ":" + std::to_string(lg(tot[K]));
  return key;
}

// Times the candidate schedules on a values-only copy of the table (each
// problem's lambda redirected to a workspace copy: the caller's data is not
// touched) and returns the fastest.  Every schedule gives identical results.
int tune_table(eig_ctx* h, const std::vector<TableItem>& items, bool mixed, cudaStream_t s, Sched* best) {
  const int count = (int)items.size();
  std::vector<eig_problem> tp(count);
  std::vector<TableItem> ti(count);
  size_t lam_bytes = 0;
  std::vector<size_t> lam_off(count);
  for (int i = 0; i < count; ++i) {
    tp[i] = *items[i].P;
    tp[i].want = EIG_VALUES;
    tp[i].Q_out = nullptr;
    tp[i].errors = nullptr;
    ti[i] = items[i];
    ti[i].P = &tp[i];
    ti[i].report = false;
    lam_off[i] = lam_bytes;
    lam_bytes += align_up(sizeof(double) * (size_t)tp[i].n, 256);
  }
  const size_t need = lam_bytes + layout_table(h, ti, nullptr, false, mixed, nullptr).bytes;
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) tp[i].lambda = reinterpret_cast<double*>(h->ws + lam_off[i]);
  std::vector<char> img;
  Table T = layout_table(h, ti, h->ws + lam_bytes, false, mixed, &img);
  if (T.bytes == 0) return EIG_ECUDA;
  const int S = std::min((int)T.classes.size(), (int)eig_ctx::kAux);
  std::vector<Sched> cand;
  std::vector<int> stream_opts{1};
  if (S > 1) stream_opts.push_back(S);
  for (int st : stream_opts)
    for (int od : {1, 2})
      for (int ord : {1, 0}) {
        Sched c;
        c.streams = st;
        c.order = ord;
        c.occ_div = od;
        cand.push_back(c);
      }
  float best_ms = -1.f;
  for (int t = -1; t < (int)cand.size(); ++t) {  // t = -1: warm-up
    const Sched& c = cand[t < 0 ? 0 : t];
    for (int i = 0; i < count; ++i)
      CK(cudaMemcpyAsync(tp[i].lambda, items[i].P->lambda, sizeof(double) * (size_t)tp[i].n,
                         cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(h->ev[0], s));
    int nl = 0;
    rc = enqueue_table(h, T, count, false, mixed, false, s, nullptr, &nl, img, nullptr, 0, c);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev[1], s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
    if (t < 0) continue;
    ++h->m_tune_trials;
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      *best = c;
    }
  }
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
  rep->iters32_total = st.iters32_total;
  rep->redo32_total = st.redo32_total;
  rep->gj32_total = st.gj32_total;
  rep->taylor_total = st.taylor_total;
  rep->n_runs = st.n_runs;
  rep->iters_max = st.iters_max;
  rep->n_notconv = st.n_notconv;
  rep->norm_A = st.lam_absmax + st.fro2;
  rep->max_pair_residual = st.err_max[0];
  rep->max_pair_rayleigh = st.err_max[1];
  rep->max_pair_orth = st.err_max[2];
  rep->tc_pair_tiles = st.tc_pair_tiles;
  rep->asm_fp64_cols = st.asm_fp64_cols;
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

int eig_last_cuda_error(char* msg, int32_t len) {
  if (msg && len > 0) {
    if (t_cuda_err == 0) {
      msg[0] = '\0';
    } else {
      std::snprintf(msg, (size_t)len, "%s: %s (%s)", cudaGetErrorName((cudaError_t)t_cuda_err),
                    cudaGetErrorString((cudaError_t)t_cuda_err), t_cuda_call);
    }
  }
  return t_cuda_err;
}

int eig_update_init(const eig_init_params* params, eig_handle* out) {
  if (!out) return EIG_EINVAL;
  *out = nullptr;
  eig_init_params p{};
  if (params) p = *params;
  if ((p.flags & ~EIG_TUNE) != 0 || (p.mode != EIG_FP64 && p.mode != EIG_MIXED) || p.max_iter < 0)
    return EIG_EINVAL;
  int ndev = 0;
  const cudaError_t de = cudaGetDeviceCount(&ndev);
  if (de != cudaSuccess || p.device < 0 || p.device >= ndev) {
    note_cuda(de != cudaSuccess ? de : cudaErrorInvalidDevice, "cudaGetDeviceCount", __LINE__);
    cudaGetLastError();
    return EIG_ECUDA;
  }
  eig_ctx* h = new (std::nothrow) eig_ctx();
  if (!h) return EIG_ENOMEM;
  h->device = p.device;
  h->mode = p.mode;
  h->budget = p.hbm_budget;
  h->max_iter = p.max_iter ? p.max_iter : kDefaultMaxIter;
  h->tune = (p.flags & EIG_TUNE) != 0;
  if (h->tune) load_tune_cache(h);
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
    for (BatchRes& b : h->batches) {
      if (b.done) cudaEventDestroy(b.done);
      if (b.host) cudaFreeHost(b.host);
    }
    if (h->ws) cudaFree(h->ws);
    for (auto& a : h->aux)
      if (a) cudaStreamDestroy(a);
    for (auto& e : h->aux_join)
      if (e) cudaEventDestroy(e);
    if (h->aux_fork) cudaEventDestroy(h->aux_fork);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->side_fork) cudaEventDestroy(h->side_fork);
    if (h->side_join) cudaEventDestroy(h->side_join);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->chk_host) cudaFreeHost(h->chk_host);
    for (auto& e : h->ev)
      if (e) cudaEventDestroy(e);
    cudaGetLastError();
  }
  delete h;
  return EIG_OK;
}

// Outcome of a synchronous (or synchronised) update in the handle's counters.
static void count_outcome(eig_ctx* h, int status) {
  std::lock_guard<std::mutex> lk(h->mu);
  if (status == EIG_OK) ++h->m_ok;
  else ++h->m_failed;
}

static int update_one(eig_ctx* h, eig_problem* P, unsigned long long negmask, int kplus, eig_report* rep,
                      void* stream);

int eig_update_rank_k(eig_handle h, eig_problem* P, eig_report* rep, void* stream) {
  if (!h) return EIG_EINVAL;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    ++h->m_calls;
    ++h->m_updates;
    if (P && P->n > 0) h->m_pairs += P->n;
  }
  unsigned long long negmask = 0;
  int kplus = 0;
  int rc = validate(P, &negmask, &kplus);
  if (rc) {
    count_outcome(h, rc);
    return rc;
  }
  rc = update_one(h, P, negmask, kplus, rep, stream);
  if (h->last_counted) return rc;
  if (!h->last_pending) {  // finished (or failed before its status copy)
    h->last_counted = true;
    count_outcome(h, rc);
  }
  return rc;
}

// The work of eig_update_rank_k after validation.
static int update_one(eig_ctx* h, eig_problem* P, unsigned long long negmask, int kplus, eig_report* rep,
                      void* stream) {
  int rc = EIG_OK;
  if (!h->last_counted) {  // an EIG_ASYNC update whose status nobody read
    std::lock_guard<std::mutex> lk(h->mu);
    ++h->m_unread;
  }
  h->last_counted = false;
  h->last_pending = false;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vectors = (P->want & EIG_VECTORS) != 0;
  const bool report = (P->want & EIG_REPORT) != 0 && vectors;
  const bool mixed = h->mode == EIG_MIXED;
  std::vector<TableItem> items{{P, negmask, kplus, report}};
  const size_t need = layout_table(h, items, nullptr, vectors, mixed, nullptr).bytes;
  rc = ensure_ws(h, need);
  if (rc) return rc;
  std::vector<char> img;
  Table T = layout_table(h, items, h->ws, vectors, mixed, &img);
  if (T.bytes == 0) return EIG_ECUDA;
  rc = enqueue_table(h, T, 1, vectors, mixed, report, s, rep ? h->ev : nullptr, &h->last_launches, img, P,
                     negmask);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->m_launches += h->last_launches;
  }
  h->last_stream = s;
  CK(cudaMemcpyAsync(h->st_host, T.d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  if (P->want & EIG_ASYNC) {
    h->last_pending = true;
    return EIG_OK;
  }
  if (report)
    CK(cudaMemcpyAsync(h->chk_host, T.chk_out, sizeof(double) * (kCheckCols + kCheckCols * kCheckCols),
                       cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->last_pending = false;
  const int status = status_of(*h->st_host);
  if (rep) {
    fill_report(rep, P, *h->st_host, report ? h->chk_host : nullptr, status);
    auto span = [&](int a0, int b0) -> double {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->ev[a0], h->ev[b0]) != cudaSuccess) {
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
  if (count == 0) return EIG_OK;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool mixed = h->mode == EIG_MIXED;
  // Valid problems with and without vectors form two tables (one launch
  // sequence each); invalid ones get their status without any launch.
  std::vector<TableItem> tab[2];
  std::vector<int> slot[2];
  std::vector<int> pre(count, EIG_OK);
  for (int i = 0; i < count; ++i) {
    unsigned long long negmask = 0;
    int kplus = 0;
    pre[i] = validate(&probs[i], &negmask, &kplus);
    if (pre[i] != EIG_OK) continue;
    const int v = (probs[i].want & EIG_VECTORS) ? 1 : 0;
    tab[v].push_back({&probs[i], negmask, kplus, false});
    slot[v].push_back(i);
  }
  // Schedule of each table: the tuned one for its signature (EIG_TUNE; timed
  // now if the signature is new), else the default sequential schedule.
  Sched sch[2];
  if (h->tune && (tab[0].size() + tab[1].size()) > 1 && ensure_aux(h)) {
    for (int v = 0; v < 2; ++v) {
      if (tab[v].empty()) continue;
      const std::string key = batch_signature(tab[v], v == 1, mixed);
      auto it = h->tuned.find(key);
      if (it != h->tuned.end()) {
        sch[v] = it->second;
        ++h->m_tune_hits;
        continue;
      }
      Sched best;
      const int trc = tune_table(h, tab[v], mixed, s, &best);
      if (trc) return trc;
      h->tuned[key] = best;
      save_tune_entry(h, key, best);
      sch[v] = best;
    }
  }
  size_t need = 0;
  for (int v = 0; v < 2; ++v)
    if (!tab[v].empty()) need = std::max(need, layout_table(h, tab[v], nullptr, v == 1, mixed, nullptr).bytes);
  {
    std::lock_guard<std::mutex> lk(h->mu);
    ++h->m_calls;
  }
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  // One pinned status block and one event for the whole call.
  BatchRes B;
  if (cudaMallocHost(&B.host, sizeof(DevStatus) * (size_t)count) != cudaSuccess ||
      cudaEventCreateWithFlags(&B.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (B.host) cudaFreeHost(B.host);
    return EIG_ENOMEM;
  }
  std::memset(B.host, 0, sizeof(DevStatus) * (size_t)count);
  auto fail = [&](int code) {
    cudaStreamSynchronize(s);  // copies into B.host may be queued
    cudaGetLastError();
    cudaEventDestroy(B.done);
    cudaFreeHost(B.host);
    return code;
  };
  for (int v = 0; v < 2; ++v) {
    if (tab[v].empty()) continue;
    std::vector<char> img;
    Table T = layout_table(h, tab[v], h->ws, v == 1, mixed, &img);
    if (T.bytes == 0) return fail(EIG_ECUDA);
    int nl = 0;
    rc = enqueue_table(h, T, (int)tab[v].size(), v == 1, mixed, false, s, nullptr, &nl, img, nullptr, 0, sch[v]);
    if (rc) return fail(rc);
    {
      std::lock_guard<std::mutex> lk(h->mu);
      h->m_launches += nl;
    }
    for (size_t j = 0; j < tab[v].size(); ++j)
      if (cudaMemcpyAsync(B.host + slot[v][j], T.d_st + j, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
        return fail(EIG_ECUDA);
    // The next table reuses the workspace: keep the tables stream-ordered.
  }
  if (cudaEventRecord(B.done, s) != cudaSuccess) return fail(EIG_ECUDA);
  std::lock_guard<std::mutex> lk(h->mu);
  int bi;
  if (!h->free_batches.empty()) {
    bi = h->free_batches.back();
    h->free_batches.pop_back();
  } else {
    bi = (int)h->batches.size();
    h->batches.emplace_back();
  }
  B.live = count;
  h->batches[bi] = B;
  for (int i = 0; i < count; ++i) {
    int ti;
    if (!h->free_tickets.empty()) {
      ti = h->free_tickets.back();
      h->free_tickets.pop_back();
    } else {
      ti = (int)h->tickets.size();
      h->tickets.emplace_back();
    }
    Ticket& t = h->tickets[ti];
    t.batch = bi;
    t.slot = i;
    t.n = probs[i].n;
    t.k = probs[i].k;
    t.pre_status = pre[i];
    t.live = true;
    tickets[i] = ((uint64_t)t.gen << 32) | (uint64_t)(ti + 1);
    ++h->m_updates;
    h->m_pairs += probs[i].n > 0 ? probs[i].n : 0;
  }
  h->last_stream = s;
  return EIG_OK;
}

// The live ticket an id names, or null (call with h->mu held).
static Ticket* find_ticket(eig_ctx* h, uint64_t id) {
  const uint64_t idx = (id & 0xffffffffull);
  if (idx < 1 || idx > h->tickets.size()) return nullptr;
  Ticket& t = h->tickets[idx - 1];
  if (!t.live || t.gen != (uint32_t)(id >> 32)) return nullptr;
  return &t;
}

// Final status of a ticket (EIG_EBUSY while its batch runs).  Call with h->mu held.
static int ticket_status(eig_ctx* h, const Ticket& t, DevStatus* st_out) {
  if (t.pre_status != EIG_OK) return t.pre_status;
  const BatchRes& b = h->batches[t.batch];
  const cudaError_t q = cudaEventQuery(b.done);
  if (q == cudaErrorNotReady) {
    cudaGetLastError();
    return EIG_EBUSY;
  }
  if (q != cudaSuccess) {
    cudaGetLastError();
    return EIG_ECUDA;
  }
  if (st_out) *st_out = b.host[t.slot];
  return status_of(b.host[t.slot]);
}

int eig_update_release(eig_handle h, uint64_t ticket) {
  if (!h) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  std::lock_guard<std::mutex> lk(h->mu);
  Ticket* t = find_ticket(h, ticket);
  if (!t) return EIG_EINVAL;
  const int status = ticket_status(h, *t, nullptr);
  if (status == EIG_EBUSY) return EIG_EBUSY;
  if (status == EIG_OK) ++h->m_ok;
  else ++h->m_failed;
  t->live = false;
  ++t->gen;
  h->free_tickets.push_back((int)((ticket & 0xffffffffull) - 1));
  BatchRes& b = h->batches[t->batch];
  if (--b.live == 0) {
    cudaEventDestroy(b.done);
    cudaFreeHost(b.host);
    b = BatchRes{};
    h->free_batches.push_back(t->batch);
  }
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
      DevStatus dst{};
      int status;
      {
        std::lock_guard<std::mutex> lk(h->mu);
        const Ticket* tp = find_ticket(h, id);
        if (!tp) return EIG_EINVAL;
        t = *tp;
        status = ticket_status(h, t, &dst);
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
      fill_report(static_cast<eig_report*>(out), &P, dst, nullptr, status);
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
      if (!h->last_counted) {
        h->last_counted = true;
        count_outcome(h, status);
      }
      *static_cast<int32_t*>(out) = status;
      return status;
    }
    case EIG_Q_METRICS: {
      if (!out || out_bytes < sizeof(eig_metrics)) return EIG_EINVAL;
      eig_metrics m{};
      std::lock_guard<std::mutex> lk(h->mu);
      m.calls = h->m_calls;
      m.updates = h->m_updates;
      m.eigenpairs = h->m_pairs;
      m.updates_ok = h->m_ok;
      m.updates_failed = h->m_failed;
      m.launches = h->m_launches;
      m.workspace_allocs = h->m_allocs;
      m.workspace_bytes = h->ws_bytes;
      m.tune_trials = h->m_tune_trials;
      m.tune_hits = h->m_tune_hits;
      for (const Ticket& t : h->tickets) {  // live batch tickets: resolved now, without waiting
        if (!t.live) continue;
        const int status = ticket_status(h, t, nullptr);
        if (status == EIG_EBUSY) ++m.updates_pending;
        else if (status == EIG_OK) ++m.updates_ok;
        else ++m.updates_failed;
      }
      m.updates_pending += h->m_unread + (h->last_counted ? 0 : 1);
      *static_cast<eig_metrics*>(out) = m;
      return EIG_OK;
    }
    case EIG_Q_WORKSPACE: {
      const eig_problem* P = static_cast<const eig_problem*>(in);
      if (!P || !out || out_bytes < sizeof(uint64_t) || P->n < 1 || P->k < 1 || P->k > EIG_MAX_K)
        return EIG_EINVAL;
      const bool vectors = (P->want & EIG_VECTORS) != 0;
      std::vector<TableItem> one{{P, 0, P->k, (P->want & EIG_REPORT) && vectors}};
      *static_cast<uint64_t*>(out) =
          layout_table(h, one, nullptr, vectors, h->mode == EIG_MIXED, nullptr).bytes;
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
  // runs of equal lambda are rotated in a copy of U (the caller's U is input only)
  CK(cudaMemcpyAsync(c.U, U, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, s));
  CK(launch_runs_qr(n, k, lambda, c.U, c.Vr, c.taur, c.runs, c.st, s));
  CK(launch_deflate(n, k, K, lambda, c.U, negmask, c.lam_keep, c.Us, ld, c.idx_keep, c.idx_defl,
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

int eig_pole_counts(eig_handle h, int64_t n, int32_t k, const double* lambda, const double* U,
                    const int8_t* sigma, int32_t* counts, int32_t* counts32, int32_t* idx_keep, int64_t* n_keep,
                    void* stream) {
  if (!h || n < 1 || k < 1 || k > EIG_MAX_K || !lambda || !U || !counts || !n_keep ||
      n > (int64_t)0x3fffffff)
    return EIG_EINVAL;
  unsigned long long negmask = 0;
  int kplus = 0;
  if (!sigma_info(sigma, k, &negmask, &kplus)) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool mixed = h->mode == EIG_MIXED;
  // The update's own launch sequence (a table of one, values only), stopped
  // after the pole counts: the caller's U stands in for U = Q^T K.
  eig_problem P{};
  P.n = n;
  P.k = k;
  P.lambda = const_cast<double*>(lambda);
  P.sigma = sigma;
  std::vector<TableItem> items{{&P, negmask, kplus, false}};
  const size_t need = layout_table(h, items, nullptr, false, mixed, nullptr).bytes;
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  std::vector<char> img;
  Table T = layout_table(h, items, h->ws, false, mixed, &img);
  if (T.bytes == 0 || T.classes.size() != 1) return EIG_ECUDA;
  ProbDesc d0;
  std::memcpy(&d0, img.data(), sizeof(ProbDesc));
  CK(cudaMemcpyAsync(T.d_desc, img.data(), img.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(T.d_st, 0, sizeof(DevStatus), s));
  CK(cudaMemcpyAsync(d0.U, U, sizeof(double) * (size_t)n * k, cudaMemcpyDeviceToDevice, s));
  CK(launch_runs_qr_grouped(T.d_desc, 1, n, s));
  CK(launch_deflate_grouped(T.d_desc, 1, s));
  CK(launch_class_prefix(T.d_desc, T.classes[0], s));
  if (mixed) {
    CK(launch_counts_grouped(T.d_desc, T.classes[0], T.class_items[0], true, s, 1));
    if (counts32) CK(cudaMemcpyAsync(counts32, d0.pole_cnt, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    CK(launch_counts_grouped(T.d_desc, T.classes[0], T.class_items[0], true, s, 2));
  } else {
    CK(launch_counts_grouped(T.d_desc, T.classes[0], T.class_items[0], false, s));
    if (counts32) CK(cudaMemsetAsync(counts32, 0xff, sizeof(int) * (size_t)n, s));
  }
  CK(cudaMemcpyAsync(h->st_host, T.d_st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int status = status_of(*h->st_host);
  const int64_t nk = h->st_host->n_keep;
  *n_keep = status == EIG_EINVAL ? 0 : nk;
  if (status == EIG_EINVAL) return status;
  if (nk > 0) {
    CK(cudaMemcpyAsync(counts, d0.pole_cnt, sizeof(int) * (size_t)nk, cudaMemcpyDeviceToDevice, s));
    if (idx_keep) CK(cudaMemcpyAsync(idx_keep, d0.idx_keep, sizeof(int) * (size_t)nk, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  return status;
}

int eig_perturbation(eig_handle h, int64_t n, int32_t k, const double* Q, const double* lambda,
                     const double* K, const int8_t* sigma, double* mu, double* X, void* stream) {
  if (!h || n < 1 || k < 1 || k > EIG_MAX_K || !Q || !lambda || !K || !mu || !X ||
      n > (int64_t)0x3fffffff || X == Q)
    return EIG_EINVAL;
  unsigned long long negmask = 0;
  int kplus = 0;
  if (!sigma_info(sigma, k, &negmask, &kplus)) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool mixed = (h->mode == EIG_MIXED);
  // workspace: status, U, W (or W^T), and in mixed mode the slices of Q and W^T
  auto layout = [&](char* base, DevStatus** st, double** U, double** W, __nv_bfloat16** Qs,
                    __nv_bfloat16** Ws, unsigned long long** rmax, int** erow, int** fcol) {
    Bump b(base);
    *st = reinterpret_cast<DevStatus*>(b.take(sizeof(DevStatus)));
    *U = reinterpret_cast<double*>(b.take(sizeof(double) * (size_t)n * k));
    *W = reinterpret_cast<double*>(b.take(sizeof(double) * (size_t)n * n));
    if (mixed) {
      const size_t planes = 2 * (size_t)tc_num_slices() * tc_slice_plane((int)n);
      *Qs = reinterpret_cast<__nv_bfloat16*>(b.take(planes));
      *Ws = reinterpret_cast<__nv_bfloat16*>(b.take(planes));
      *rmax = reinterpret_cast<unsigned long long*>(b.take(sizeof(unsigned long long) * (size_t)n));
      *erow = reinterpret_cast<int*>(b.take(sizeof(int) * (size_t)n));
      *fcol = reinterpret_cast<int*>(b.take(sizeof(int) * (size_t)n));
    }
    return b.off;
  };
  DevStatus* st = nullptr;
  double *U = nullptr, *W = nullptr;
  __nv_bfloat16 *Qs = nullptr, *Ws = nullptr;
  unsigned long long* rmax = nullptr;
  int *erow = nullptr, *fcol = nullptr;
  const size_t need = layout(nullptr, &st, &U, &W, &Qs, &Ws, &rmax, &erow, &fcol);
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  layout(h->ws, &st, &U, &W, &Qs, &Ws, &rmax, &erow, &fcol);
  CK(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
  CK(launch_project_f64(n, k, Q, K, U, s));
  CK(launch_perturb_w(n, k, lambda, U, negmask, mixed, W, s));
  CK(launch_perturb_mu(n, k, lambda, U, negmask, mu, s));  // after W: mu may alias lambda
  if (mixed) {
    CK(launch_slice_q((int)n, W, rmax, fcol, Ws, nullptr, s));  // rows of W^T = columns of W
    CK(launch_slice_q((int)n, Q, rmax, erow, Qs, nullptr, s));
    CK(launch_gemm_tc((int)n, Qs, Ws, erow, fcol, X, (int)n, nullptr, &st->flags, s));
  } else {
    CK(launch_gemm_f64(n, n, n, Q, n, W, n, X, n, s));
  }
  CK(cudaMemcpyAsync(h->st_host, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return status_of(*h->st_host);
}

int eig_update_select(eig_handle h, int64_t n, int32_t k, const double* Q, const double* lambda,
                      const double* K, const int8_t* sigma, double vl, double vu, int64_t max_m,
                      double* mu, double* X, int64_t* m_out, void* stream) {
  if (!h || n < 1 || k < 1 || k > EIG_MAX_K || !Q || !lambda || !K || !mu || !m_out || max_m < 0 ||
      n > (int64_t)0x3fffffff || !(vl < vu))
    return EIG_EINVAL;
  unsigned long long negmask = 0;
  int kplus = 0;
  if (!sigma_info(sigma, k, &negmask, &kplus)) return EIG_EINVAL;
  DeviceGuard g(h->device);
  if (!g.ok) return EIG_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int Kp = padded_rank(k);
  const int ld = (int)align_up((size_t)n, 32);
  const size_t cap = (size_t)(max_m < n ? max_m : n);
  // workspace: the secular carve (values only) + window ints + W_sel
  const bool mixed = (h->mode == EIG_MIXED);
  const size_t base = align_up(plan(nullptr, n, k, false, false, false).bytes, 256);
  // FP32 copies for the mixed-mode zero finder, then W_sel
  const size_t f32_bytes = mixed ? align_up(sizeof(float2) * ld, 256) + align_up(sizeof(float) * ld * Kp, 256) : 0;
  const size_t wsel_bytes = X ? align_up(sizeof(double) * (size_t)n * (cap > 0 ? cap : 1), 256) : 0;
  // mixed mode: X_sel = Q W_sel as split-BF16 products on the tensor cores
  // (slices of Q and of W_sel's columns, row and column exponents)
  const bool tc = mixed && X;
  const size_t capc = cap > 0 ? cap : 1;
  const size_t qs_bytes = tc ? align_up(2 * (size_t)tc_num_slices() * tc_slice_plane((int)n), 256) : 0;
  const size_t ws_bytes = tc ? align_up(2 * (size_t)tc_num_slices() * (size_t)tc_slice_ld((int)n) * capc, 256) : 0;
  const size_t aux_bytes = tc ? align_up(8 * (size_t)n, 256) + align_up(4 * (size_t)n, 256) + align_up(4 * capc, 256) : 0;
  const size_t pp_bytes = align_up(sizeof(double) * (size_t)ld * (size_t)(Kp * (Kp + 1) / 2), 256);
  // mixed mode: K split for the double-float projection (as the full update's)
  const size_t ksplit_bytes = mixed ? 2 * align_up(sizeof(float) * (size_t)n * k, 256) + 256 : 0;
  const size_t need = base + 256 + f32_bytes + wsel_bytes + qs_bytes + ws_bytes + aux_bytes + pp_bytes + ksplit_bytes;
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  Carve c = plan(h->ws, n, k, false, false, false);
  int* win = reinterpret_cast<int*>(h->ws + base);               // 8 ints + 2 count slots
  double* pts = reinterpret_cast<double*>(h->ws + base + 128);    // vl, vu
  float2* lamf = mixed ? reinterpret_cast<float2*>(h->ws + base + 256) : nullptr;
  float* Usf = mixed ? reinterpret_cast<float*>(h->ws + base + 256 + align_up(sizeof(float2) * ld, 256)) : nullptr;
  double* Wsel = X ? reinterpret_cast<double*>(h->ws + base + 256 + f32_bytes) : nullptr;
  char* tcb = h->ws + base + 256 + f32_bytes + wsel_bytes;
  __nv_bfloat16* Qs = tc ? reinterpret_cast<__nv_bfloat16*>(tcb) : nullptr;
  __nv_bfloat16* Ws = tc ? reinterpret_cast<__nv_bfloat16*>(tcb + qs_bytes) : nullptr;
  unsigned long long* rmax = tc ? reinterpret_cast<unsigned long long*>(tcb + qs_bytes + ws_bytes) : nullptr;
  int* erow = tc ? reinterpret_cast<int*>(tcb + qs_bytes + ws_bytes + align_up(8 * (size_t)n, 256)) : nullptr;
  int* fcol = tc ? reinterpret_cast<int*>(tcb + qs_bytes + ws_bytes + align_up(8 * (size_t)n, 256) +
                                          align_up(4 * (size_t)n, 256))
                 : nullptr;
  // products of the kept rows, as the update's zero finder takes them
  double* Pp = reinterpret_cast<double*>(tcb + qs_bytes + ws_bytes + aux_bytes);
  char* ksb = tcb + qs_bytes + ws_bytes + aux_bytes + pp_bytes;
  float* Kh = mixed ? reinterpret_cast<float*>(ksb) : nullptr;
  float* Kl = mixed ? reinterpret_cast<float*>(ksb + align_up(sizeof(float) * (size_t)n * k, 256)) : nullptr;
  int* Kexp = mixed ? reinterpret_cast<int*>(ksb + 2 * align_up(sizeof(float) * (size_t)n * k, 256)) : nullptr;
  const double xv[2] = {vl, vu};
  CK(cudaMemsetAsync(c.st, 0, sizeof(DevStatus), s));
  CK(cudaMemcpyAsync(pts, xv, sizeof(xv), cudaMemcpyHostToDevice, s));
  // the full update's projection in either mode, so that the roots agree bit for bit
  if (mixed)
    CK(launch_project_mixed(n, k, Q, K, c.U, Kh, Kl, Kexp, s));
  else
    CK(launch_project_f64(n, k, Q, K, c.U, s));
  CK(launch_runs_qr(n, k, lambda, c.U, c.Vr, c.taur, c.runs, c.st, s));
  CK(launch_deflate(n, k, Kp, lambda, c.U, negmask, c.lam_keep, c.Us, ld, c.idx_keep, c.idx_defl,
                    c.lam_defl, c.st, s, lamf, Usf));
  Sub sub;
  sub.n_dev = &c.st->n_keep;
  sub.ld = ld;
  sub.K = Kp;
  sub.kplus = kplus + (Kp - k);
  sub.lam = c.lam_keep;
  sub.Us = c.Us;
  sub.idx = c.idx_keep;
  sub.st = c.st;
  sub.negmask = negmask;
  sub.lamf = lamf;
  sub.Usf = Usf;
  if (warps_per_root(Kp) == 1) {  // as the update: products for the one-warp ranks
    CK(launch_products(c.Us, Kp, ld, c.st, Pp, s));
    sub.Pp = Pp;
  }
  CK(launch_counts(sub, pts, 2, win + 8, s));
  CK(launch_select_window(sub, c.st, c.lam_defl, vl, vu, win + 8, win, s));
  int hw[8];
  CK(cudaMemcpyAsync(hw, win, sizeof(hw), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->st_host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h->st_host->flags & (ST_UNSORTED | ST_NONFINITE)) return EIG_EINVAL;
  const int nk = hw[6];
  int r0 = hw[0], r1 = hw[1];
  r0 = r0 < 0 ? 0 : (r0 > nk ? nk : r0);
  r1 = r1 < r0 ? r0 : (r1 > nk ? nk : r1);
  const int qa = hw[2], qb = hw[3], dlo = hw[4], dsel = hw[5];
  const int64_t m = (int64_t)(r1 - r0) + dsel;
  *m_out = m;
  if (m > max_m) return EIG_ETOOBIG;
  if (m == 0) return EIG_OK;
  if (r1 > r0) {
    // true pole counts around the interval, placeholders elsewhere
    const int p0 = qa > 0 ? qa - 1 : 0;
    const int p1 = qb < nk ? qb + 1 : nk;
    CK(launch_select_fill(nk, p0, p1, c.pole_cnt, s));
    CK(launch_counts(sub, nullptr, ld, c.pole_cnt, s, p0, p1));
    CK(cudaMemcpyAsync(c.counter, &r0, sizeof(int), cudaMemcpyHostToDevice, s));
    RootOut ro{c.origin, c.tau, c.iters, c.rflags, c.alpha, c.beta, c.sidx};
    CK(launch_roots(sub, c.pole_cnt, h->max_iter, c.counter, ro, c.st, h->num_sms, s, r1 - r0, r1));
  }
  if (Wsel) CK(cudaMemsetAsync(Wsel, 0, sizeof(double) * (size_t)n * (size_t)m, s));
  RootOut ro{c.origin, c.tau, c.iters, c.rflags, c.alpha, c.beta, c.sidx};
  CK(launch_assemble_select(sub, ro, n, c.idx_defl, c.lam_defl, dlo, dsel, r0, r1, c.mu_sec, mu, Wsel, s));
  if (X) {
    CK(launch_runs_apply_w(n, k, c.Vr, c.taur, c.runs, c.st, Wsel, n, m, h->num_sms, s));  // W_sel <- B W_sel
    if (tc) {
      CK(launch_slice_q((int)n, Q, rmax, erow, Qs, c.st, s));
      CK(launch_slice_cols((int)n, (int)m, Wsel, fcol, Ws, s));
      CK(launch_gemm_tc((int)n, Qs, Ws, erow, fcol, X, (int)n, c.st, &c.st->flags, s, (int)m));
    } else {
      CK(launch_gemm_f64(n, m, n, Q, n, Wsel, n, X, n, s));
    }
  }
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

// ===========================================================================
// Serving: resident decompositions, chained requests, continuous batching.
// ===========================================================================
struct SrvRequest {
  int resident = 0;
  int k = 0;
  std::vector<double> K;  // host copy, n x k column-major
  std::vector<int8_t> sigma;
  unsigned long long negmask = 0;
  int kplus = 0;
  int status = EIG_EBUSY;
  int batch_size = 0;
  double submit_ms = 0, launch_ms = -1, done_ms = -1;
};

struct SrvResident {
  int64_t n = 0;
  double* Q = nullptr;
  double* lambda = nullptr;
  bool busy = false;
};

struct SrvSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* kstage = nullptr;  // pinned staging for the batch's K payloads
  size_t kstage_bytes = 0;
  DevStatus* st_host = nullptr;  // pinned, max_batch entries
  bool busy = false;
  std::vector<uint64_t> reqs;
  std::vector<eig_problem> probs;
};

struct eig_srv {
  eig_ctx* h = nullptr;
  int max_batch = 64;
  bool mixed = false;
  std::vector<SrvSlot> slots;
  std::vector<SrvResident> residents;
  std::deque<uint64_t> pending;
  std::vector<SrvRequest> reqs;
  int inflight = 0;
  std::chrono::steady_clock::time_point t0;
  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

size_t srv_request_bytes(eig_srv* S, const SrvRequest& r) {
  const SrvResident& res = S->residents[r.resident];
  eig_problem P{};
  P.n = res.n;
  P.k = r.k;
  P.want = EIG_VALUES | EIG_VECTORS;
  std::vector<TableItem> one{{&P, 0, r.k, false}};
  return layout_table(S->h, one, nullptr, true, S->mixed, nullptr).bytes + 4096 +
         align_up(sizeof(double) * (size_t)res.n * r.k, 256);
}

// Reap every finished batch; returns requests completed.
int srv_reap(eig_srv* S) {
  int done = 0;
  for (SrvSlot& sl : S->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) {
      cudaGetLastError();
      continue;
    }
    const double t = S->now_ms();
    for (size_t j = 0; j < sl.reqs.size(); ++j) {
      SrvRequest& r = S->reqs[sl.reqs[j] - 1];
      r.status = (q == cudaSuccess) ? status_of(sl.st_host[j]) : EIG_ECUDA;
      r.done_ms = t;
      S->residents[r.resident].busy = false;
      ++done;
    }
    if (q != cudaSuccess) cudaGetLastError();
    S->inflight -= (int)sl.reqs.size();
    sl.reqs.clear();
    sl.busy = false;
  }
  return done;
}

// Admit pending requests into a batch on a free slot and launch it.
int srv_launch(eig_srv* S, SrvSlot& sl) {
  std::vector<uint64_t> pick;
  std::vector<char> taken(S->residents.size(), 0);
  size_t bytes = 0, kbytes = 0;
  for (auto it = S->pending.begin(); it != S->pending.end() && (int)pick.size() < S->max_batch;) {
    SrvRequest& r = S->reqs[*it - 1];
    if (S->residents[r.resident].busy || taken[r.resident]) {
      ++it;
      continue;
    }
    const size_t need = srv_request_bytes(S, r);
    if (need > sl.ws_bytes) {  // can never fit this slot: reject
      r.status = EIG_ENOMEM;
      r.done_ms = S->now_ms();
      it = S->pending.erase(it);
      continue;
    }
    if (bytes + need > sl.ws_bytes) break;  // admission by free workspace
    bytes += need;
    kbytes += align_up(sizeof(double) * (size_t)S->residents[r.resident].n * r.k, 256);
    taken[r.resident] = 1;
    pick.push_back(*it);
    it = S->pending.erase(it);
  }
  if (pick.empty()) return 0;
  if (kbytes > sl.kstage_bytes) {
    if (sl.kstage) cudaFreeHost(sl.kstage);
    sl.kstage = nullptr;
    sl.kstage_bytes = 0;
    if (cudaMallocHost(&sl.kstage, kbytes) != cudaSuccess) {
      cudaGetLastError();
      for (uint64_t t : pick) S->pending.push_front(t);
      return EIG_ENOMEM;
    }
    sl.kstage_bytes = kbytes;
  }
  // K payloads: pinned staging -> the head of the slot workspace.
  sl.probs.assign(pick.size(), eig_problem{});
  std::vector<TableItem> items;
  size_t koff = 0;
  for (size_t j = 0; j < pick.size(); ++j) {
    SrvRequest& r = S->reqs[pick[j] - 1];
    SrvResident& res = S->residents[r.resident];
    const size_t kb = sizeof(double) * (size_t)res.n * r.k;
    std::memcpy(reinterpret_cast<char*>(sl.kstage) + koff, r.K.data(), kb);
    eig_problem& P = sl.probs[j];
    P.n = res.n;
    P.k = r.k;
    P.Q = res.Q;
    P.lambda = res.lambda;
    P.K = reinterpret_cast<const double*>(sl.ws + koff);
    P.sigma = r.sigma.empty() ? nullptr : r.sigma.data();
    P.Q_out = nullptr;
    P.want = EIG_VALUES | EIG_VECTORS;
    items.push_back({&P, r.negmask, r.kplus, false});
    koff += align_up(kb, 256);
  }
  CK(cudaMemcpyAsync(sl.ws, sl.kstage, koff, cudaMemcpyHostToDevice, sl.stream));
  std::vector<char> img;
  Table T = layout_table(S->h, items, sl.ws + koff, true, S->mixed, &img);
  if (T.bytes == 0) return EIG_ECUDA;
  int nl = 0;
  Sched sch;
  sch.side = false;  // the slots share the handle: keep each batch on its slot's stream
  int rc = enqueue_table(S->h, T, (int)items.size(), true, S->mixed, false, sl.stream, nullptr, &nl, img,
                         nullptr, 0, sch);
  if (rc) return rc;
  CK(cudaMemcpyAsync(sl.st_host, T.d_st, sizeof(DevStatus) * items.size(), cudaMemcpyDeviceToHost,
                     sl.stream));
  CK(cudaEventRecord(sl.done, sl.stream));
  const double t = S->now_ms();
  for (uint64_t tk : pick) {
    SrvRequest& r = S->reqs[tk - 1];
    r.launch_ms = t;
    r.batch_size = (int)pick.size();
    S->residents[r.resident].busy = true;
  }
  sl.reqs = pick;
  sl.busy = true;
  S->inflight += (int)pick.size();
  return (int)pick.size();
}

}  // namespace

extern "C" {

int eig_server_create(const eig_server_params* params, eig_server* out) {
  if (!out) return EIG_EINVAL;
  *out = nullptr;
  eig_server_params p{};
  if (params) p = *params;
  const int slots = p.slots > 0 ? p.slots : 2;
  const int max_batch = p.max_batch > 0 ? p.max_batch : 64;
  const uint64_t budget = p.hbm_budget ? p.hbm_budget : (uint64_t)8 << 30;
  if (slots > 16 || max_batch > 4096) return EIG_EINVAL;
  eig_init_params ip{};
  ip.device = p.device;
  ip.mode = p.mode;
  eig_handle h = nullptr;
  int rc = eig_update_init(&ip, &h);
  if (rc) return rc;
  eig_srv* S = new (std::nothrow) eig_srv();
  if (!S) {
    eig_update_destroy(h);
    return EIG_ENOMEM;
  }
  S->h = h;
  S->max_batch = max_batch;
  S->mixed = p.mode == EIG_MIXED;
  S->t0 = std::chrono::steady_clock::now();
  S->slots.resize(slots);
  DeviceGuard g(h->device);
  for (SrvSlot& sl : S->slots) {
    sl.ws_bytes = align_up(budget / slots, 256);
    void* w = nullptr;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&w, sl.ws_bytes) != cudaSuccess ||
        cudaMallocHost(&sl.st_host, sizeof(DevStatus) * max_batch) != cudaSuccess) {
      cudaGetLastError();
      if (w) sl.ws = static_cast<char*>(w);
      eig_server_destroy(S);
      return EIG_ENOMEM;
    }
    sl.ws = static_cast<char*>(w);
  }
  *out = S;
  return EIG_OK;
}

int eig_server_destroy(eig_server S) {
  if (!S) return EIG_OK;
  {
    DeviceGuard g(S->h->device);
    for (SrvSlot& sl : S->slots) {
      if (sl.stream) cudaStreamSynchronize(sl.stream);
      if (sl.ws) cudaFree(sl.ws);
      if (sl.kstage) cudaFreeHost(sl.kstage);
      if (sl.st_host) cudaFreeHost(sl.st_host);
      if (sl.done) cudaEventDestroy(sl.done);
      if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    cudaGetLastError();
  }
  eig_update_destroy(S->h);
  delete S;
  return EIG_OK;
}

int eig_server_add_resident(eig_server S, int64_t n, double* Q, double* lambda, int32_t* id) {
  if (!S || n < 1 || n > (int64_t)0x3fffffff || !Q || !lambda || !id) return EIG_EINVAL;
  SrvResident r;
  r.n = n;
  r.Q = Q;
  r.lambda = lambda;
  S->residents.push_back(r);
  *id = (int32_t)S->residents.size() - 1;
  return EIG_OK;
}

int eig_server_submit(eig_server S, int32_t id, int32_t k, const double* K, const int8_t* sigma,
                      uint64_t* ticket) {
  if (!S || id < 0 || id >= (int32_t)S->residents.size() || k < 1 || k > EIG_MAX_K || !K || !ticket)
    return EIG_EINVAL;
  SrvRequest r;
  if (!sigma_info(sigma, k, &r.negmask, &r.kplus)) return EIG_EINVAL;
  r.resident = id;
  r.k = k;
  const int64_t n = S->residents[id].n;
  r.K.assign(K, K + (size_t)n * k);
  if (sigma) r.sigma.assign(sigma, sigma + k);
  r.submit_ms = S->now_ms();
  S->reqs.push_back(std::move(r));
  *ticket = (uint64_t)S->reqs.size();
  S->pending.push_back(*ticket);
  return EIG_OK;
}

int eig_server_poll(eig_server S, int32_t wait_us) {
  if (!S) return EIG_EINVAL;
  DeviceGuard g(S->h->device);
  if (!g.ok) return EIG_ECUDA;
  int done = srv_reap(S);
  bool launched = false;
  for (SrvSlot& sl : S->slots) {
    if (sl.busy || S->pending.empty()) continue;
    const int rc = srv_launch(S, sl);
    if (rc < 0) return rc;
    launched = launched || rc > 0;
  }
  if (!launched && done == 0 && S->inflight > 0 && wait_us > 0) {
    const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(wait_us);
    while (std::chrono::steady_clock::now() < until) {
      done = srv_reap(S);
      if (done > 0) break;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
  return done;
}

int eig_server_query(eig_server S, uint64_t ticket, eig_request_info* out) {
  if (!S || !out || ticket < 1 || ticket > S->reqs.size()) return EIG_EINVAL;
  const SrvRequest& r = S->reqs[ticket - 1];
  out->status = r.status;
  out->resident = r.resident;
  out->k = r.k;
  out->batch_size = r.batch_size;
  out->submit_ms = r.submit_ms;
  out->launch_ms = r.launch_ms;
  out->done_ms = r.done_ms;
  return r.status;
}

int eig_server_pending(eig_server S) {
  if (!S) return EIG_EINVAL;
  return (int)S->pending.size() + S->inflight;
}

}  // extern "C"
