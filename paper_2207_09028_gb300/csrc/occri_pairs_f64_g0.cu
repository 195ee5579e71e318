// occri_pairs_f64_g0.cu -- pair-transform kernels for double, grid edges 8 9 10 12 15 16 18 20 24 25 27.
#include "occri_pairs.cuh"
#include "occri_pairs_decl.h"

namespace occri {
namespace pairs {
template cudaError_t run_wave<double, 8>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 8>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 8>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 9>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 9>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 9>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 10>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 10>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 10>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 12>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 12>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 12>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 15>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 15>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 15>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 16>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 16>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 16>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 18>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 18>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 18>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 20>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 20>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 20>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 24>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 24>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 24>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 25>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 25>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 25>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_wave<double, 27>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<double, 27>(const PairParams&, const cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_qtables<double, 27>(const PairParams&, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 8>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 9>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 10>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 12>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 15>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 16>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 18>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 20>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 24>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 25>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<double, 27>(const PairParams&, const cplx_t<double>*, const cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, cplx_t<double>*, double*, cudaStream_t);
}  // namespace pairs
}  // namespace occri
