// occri_pairs_f64_g5.cu -- pair-transform kernels for double, grid edges 60.
#include "occri_pairs.cuh"
#include "occri_pairs_decl.h"

namespace occri {
namespace pairs {
template cudaError_t run_wave<double, 60>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 60>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 60>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 60>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
}  // namespace pairs
}  // namespace occri
