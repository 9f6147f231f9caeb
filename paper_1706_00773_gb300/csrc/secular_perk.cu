// secular_perk.cu -- the secular kernels of one padded rank.  The build
// compiles this file once per K in {1..8, 10, 12, 14, 16} with
// -DEIG_SECULAR_K=K; secular.cu dispatches to the entry points defined here.
#ifndef EIG_SECULAR_K
#error "compile with -DEIG_SECULAR_K=<padded rank>"
#endif
#include "secular_impl.cuh"
#include "secular_entries.cuh"

namespace eig {

template cudaError_t sec_counts<EIG_SECULAR_K>(const Sub&, const double*, int, int*, cudaStream_t, int, int);
template cudaError_t sec_roots<EIG_SECULAR_K>(const Sub&, const int*, int, int*, const RootOut&, DevStatus*, int,
                                              cudaStream_t, int, int);
template cudaError_t sec_assemble<EIG_SECULAR_K>(const Sub&, const RootOut&, int64_t, const int*, const double*,
                                                 const DevStatus*, double*, double*, double*, cudaStream_t,
                                                 const WSlices&);
template cudaError_t sec_assemble_select<EIG_SECULAR_K>(const Sub&, const RootOut&, int64_t, const int*,
                                                        const double*, int, int, int, int, double*, double*,
                                                        double*, cudaStream_t);
template cudaError_t sec_counts_grouped<EIG_SECULAR_K>(const ProbDesc*, const ClassDesc&, int, bool, int,
                                                       cudaStream_t);
template cudaError_t sec_roots_grouped<EIG_SECULAR_K>(const ProbDesc*, const ClassDesc&, int, int, int,
                                                      cudaStream_t, int);
template cudaError_t sec_assemble_grouped<EIG_SECULAR_K>(const ProbDesc*, const ClassDesc&, int, int, bool, bool,
                                                         cudaStream_t);

}  // namespace eig
