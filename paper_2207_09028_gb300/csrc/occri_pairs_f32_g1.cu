// occri_pairs_f32_g1.cu -- pair-transform kernels for float, grid edges 30 32 36.
#include "occri_pairs.cuh"
#include "occri_pairs_decl.h"

namespace occri {
namespace pairs {
template cudaError_t run_wave<float, 30>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 30>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 30>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 32>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 32>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 32>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_wave<float, 36>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cudaStream_t, cudaEvent_t*, cudaEvent_t);
template cudaError_t run_domega_wave<float, 36>(const PairParams&, const cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_qtables<float, 36>(const PairParams&, float*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 30>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 32>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
template cudaError_t run_vjp_wave<float, 36>(const PairParams&, const cplx_t<float>*, const cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, cplx_t<float>*, double*, cudaStream_t);
}  // namespace pairs
}  // namespace occri
