// occri_pairs_decl.h -- per-edge entry points of the pair-transform kernels.
// Definitions live in occri_pairs.cuh and are instantiated, a few grid edges
// per translation unit, in occri_pairs_<precision>_<group>.cu.
#pragma once

#include "occri_internal.h"

namespace occri {
namespace pairs {

template <typename T, int N>
cudaError_t run_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S, cplx_t<T>* Y,
                     cudaStream_t st, cudaEvent_t* ev, cudaEvent_t ev_y);
template <typename T, int N>
cudaError_t run_domega_wave(const PairParams& p, const cplx_t<T>* psi, cplx_t<T>* S,
                            double* dacc, cudaStream_t st);
template <typename T, int N>
cudaError_t run_qtables(const PairParams& p, T* vq, cudaStream_t st);
template <typename T, int N>
cudaError_t run_vjp_wave(const PairParams& p, const cplx_t<T>* psi, const cplx_t<T>* gam,
                         cplx_t<T>* S0, cplx_t<T>* S1, cplx_t<T>* G, double* dacc,
                         cudaStream_t st);

}  // namespace pairs
}  // namespace occri
