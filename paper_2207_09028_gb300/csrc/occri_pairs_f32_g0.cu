// occri_pairs_f32_g0.cu -- pair-transform kernels for float, grid edges 8 9 10 12 15 16 18 20 24 25 27.
#include "occri_pairs.cuh"
#include "occri_pairs_decl.h"

namespace occri {
namespace pairs {
template cudaError_t run_wave<float, 8>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 8>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 8>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 9>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 9>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 9>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 10>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 10>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 10>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 12>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 12>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 12>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 15>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 15>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 15>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 16>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 16>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 16>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 18>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 18>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 18>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 20>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 20>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 20>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 24>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 24>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 24>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 25>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 25>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 25>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 27>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 27>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 27>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 8>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 9>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 10>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 12>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 15>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 16>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 18>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 20>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 24>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 25>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 27>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
}  // namespace pairs
}  // namespace occri
