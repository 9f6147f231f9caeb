// secular_entries.cuh -- per-rank entry points of the secular kernels.  Each
// is instantiated for one padded rank K in its own translation unit
// (secular_perk.cu compiled with -DEIG_SECULAR_K=K); secular.cu dispatches on K.
#pragma once

#include "eig_internal.cuh"

namespace eig {

template <int K>
cudaError_t sec_counts(const Sub& sub, const double* x, int npts, int* counts, cudaStream_t s, int pt0,
                       int pt_end);
template <int K>
cudaError_t sec_roots(const Sub& sub, const int* pole_cnt, int max_iter, int* counter, const RootOut& out,
                      DevStatus* st, int num_sms, cudaStream_t s, int m_count, int m_end);
template <int K>
cudaError_t sec_assemble(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                         const double* lam_defl, const DevStatus* st, double* mu_sec, double* lam_out, double* W,
                         cudaStream_t s, const WSlices& ws);
template <int K>
cudaError_t sec_assemble_select(const Sub& sub, const RootOut& roots, int64_t n, const int* idx_defl,
                                const double* lam_defl, int dlo, int dsel, int r0, int r1, double* mu_sec,
                                double* mu_out, double* W, cudaStream_t s);
template <int K>
cudaError_t sec_counts_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, bool mixed, int passes,
                               cudaStream_t s);
template <int K>
cudaError_t sec_roots_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_iter, int num_sms,
                              cudaStream_t s, int occ_div);
template <int K>
cudaError_t sec_assemble_grouped(const ProbDesc* P, const ClassDesc& c, int max_items, int max_defl,
                                 bool vectors, bool mixed, cudaStream_t s);

}  // namespace eig
