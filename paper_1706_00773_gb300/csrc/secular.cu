// secular.cu -- dispatch of the secular stage on the padded rank K, and the
// launchers of its rank-independent kernels.  The kernels themselves are in
// secular_impl.cuh; each rank's entry points are compiled in their own
// translation unit (secular_perk.cu).
#include "secular_impl.cuh"
#include "secular_entries.cuh"

namespace eig {

cudaError_t launch_counts(const Sub& sub, const double* x, int npts, int* counts, cudaStream_t s,
                          int pt0, int pt_end) {
  if (!x && pt0 < 0) return cudaErrorInvalidValue;
  if (!x && pt_end <= pt0) return cudaSuccess;  // empty window
  switch (sub.K) {
#define C_(K_) case K_: return sec_counts<K_>(sub, x, npts, counts, s, pt0, pt_end);
    C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(10) C_(12) C_(14) C_(16)
#undef C_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_roots(const Sub& sub, const int* pole_cnt, int max_iter, int* counter,
                         const RootOut& out, DevStatus* st, int num_sms, cudaStream_t s,
                         int m_count, int m_end) {
  if (m_count < 0) m_count = sub.ld;
  switch (sub.K) {
#define R_(K_) case K_: return sec_roots<K_>(sub, pole_cnt, max_iter, counter, out, st, num_sms, s, m_count, m_end);
    R_(1) R_(2) R_(3) R_(4) R_(5) R_(6) R_(7) R_(8) R_(10) R_(12) R_(14) R_(16)
#undef R_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_select_window(const Sub& sub, const DevStatus* st, const double* lam_defl, double vl,
                                 double vu, const int* c2, int* out, cudaStream_t s) {
  select_window_kernel<<<1, 32, 0, s>>>(sub, st, lam_defl, vl, vu, c2, out);
  return cudaGetLastError();
}

cudaError_t launch_select_fill(int nk, int p0, int p1, int* pole_cnt, cudaStream_t s) {
  if (nk <= 0) return cudaSuccess;
  const int blocks = (nk + 255) / 256 < 4096 ? (nk + 255) / 256 : 4096;
  select_fill_kernel<<<blocks, 256, 0, s>>>(nk, p0, p1, pole_cnt);
  return cudaGetLastError();
}

cudaError_t launch_assemble_select(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                                   const double* lam_defl, int dlo, int dsel, int r0, int r1, double* mu_sec,
                                   double* mu_out, double* W, cudaStream_t s) {
  switch (sub.K) {
#define S_(K_) case K_: return sec_assemble_select<K_>(sub, roots, n, idx_defl, lam_defl, dlo, dsel, r0, r1, mu_sec, mu_out, W, s);
    S_(1) S_(2) S_(3) S_(4) S_(5) S_(6) S_(7) S_(8) S_(10) S_(12) S_(14) S_(16)
#undef S_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_assemble(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                            const double* lam_defl, const DevStatus* st, double* mu_sec,
                            double* lam_out, double* W, cudaStream_t s, const WSlices& ws) {
  switch (sub.K) {
#define A_(K_) case K_: return sec_assemble<K_>(sub, roots, n, idx_defl, lam_defl, st, mu_sec, lam_out, W, s, ws);
    A_(1) A_(2) A_(3) A_(4) A_(5) A_(6) A_(7) A_(8) A_(10) A_(12) A_(14) A_(16)
#undef A_
    default: return cudaErrorInvalidValue;
  }
}


cudaError_t launch_class_prefix(const ProbDesc* P, const ClassDesc& c, cudaStream_t s) {
  class_prefix_kernel<<<1, 32, 0, s>>>(P, c);
  return cudaGetLastError();
}

cudaError_t launch_counts_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, bool mixed,
                                  cudaStream_t s, int passes) {
  switch (c.K) {
#define C_(K_) case K_: return sec_counts_grouped<K_>(P, c, max_items, mixed, passes, s);
    C_(1) C_(2) C_(3) C_(4) C_(5) C_(6) C_(7) C_(8) C_(10) C_(12) C_(14) C_(16)
#undef C_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_order_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, cudaStream_t s) {
  if (!c.perm || max_items <= 0) return cudaSuccess;
  int blocks = (max_items + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  order_roots_grouped_kernel<<<blocks, 256, 0, s>>>(P, c);
  return cudaGetLastError();
}

cudaError_t launch_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_iter,
                                 int num_sms, cudaStream_t s, int occ_div) {
  switch (c.K) {
#define R_(K_) case K_: return sec_roots_grouped<K_>(P, c, max_items, max_iter, num_sms, s, occ_div);
    R_(1) R_(2) R_(3) R_(4) R_(5) R_(6) R_(7) R_(8) R_(10) R_(12) R_(14) R_(16)
#undef R_
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_assemble_grouped(const ProbDesc* P, const ClassDesc& c, int max_items,
                                    int max_defl, bool vectors, bool mixed, cudaStream_t s) {
  switch (c.K) {
#define A_(K_) case K_: return sec_assemble_grouped<K_>(P, c, max_items, max_defl, vectors, mixed, s);
    A_(1) A_(2) A_(3) A_(4) A_(5) A_(6) A_(7) A_(8) A_(10) A_(12) A_(14) A_(16)
#undef A_
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace eig
