// occri_pairs_dispatch.cu -- runtime grid edge -> compiled pair-transform kernels.
#include "occri_pairs_decl.h"

namespace occri {

template <typename T>
cudaError_t launch_pair_wave(const Plan& p, int k, int kp0, int nkp, int diag, cudaStream_t s,
                             void* scratch, void* Yacc, cudaEvent_t* ev, cudaEvent_t ev_y) {
  PairParams pp = p.pair_params();
  pp.k = k;
  pp.kp0 = kp0;
  pp.nkp = nkp;
  pp.diag = diag;
  const cplx_t<T>* psi = (const cplx_t<T>*)p.psi;
  cplx_t<T>* S = (cplx_t<T>*)scratch;
  cplx_t<T>* Y = (cplx_t<T>*)Yacc;
  switch (p.N[0]) {
#define OCCRI_PAIR_CASE(NN) \
  case NN:                  \
    return pairs::run_wave<T, NN>(pp, psi, S, Y, s, ev, ev_y);
    OCCRI_FOR_EACH_N(OCCRI_PAIR_CASE)
#undef OCCRI_PAIR_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_domega_wave(const Plan& p, int k, int kp0, int nkp, int diag,
                               cudaStream_t s) {
  PairParams pp = p.pair_params();
  pp.k = k;
  pp.kp0 = kp0;
  pp.nkp = nkp;
  pp.diag = diag;
  const cplx_t<T>* psi = (const cplx_t<T>*)p.psi;
  cplx_t<T>* S = (cplx_t<T>*)p.scratch;
  switch (p.N[0]) {
#define OCCRI_DOMEGA_CASE(NN) \
  case NN:                    \
    return pairs::run_domega_wave<T, NN>(pp, psi, S, p.dacc, s);
    OCCRI_FOR_EACH_N(OCCRI_DOMEGA_CASE)
#undef OCCRI_DOMEGA_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_qtables(const Plan& p, cudaStream_t s) {
  const PairParams pp = p.pair_params();
  switch (p.N[0]) {
#define OCCRI_QTAB_CASE(NN) \
  case NN:                  \
    return pairs::run_qtables<T, NN>(pp, (T*)p.vq, s);
    OCCRI_FOR_EACH_N(OCCRI_QTAB_CASE)
#undef OCCRI_QTAB_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_vjp_wave(const Plan& p, int k, int kp0, int nkp, int diag, double* dacc,
                            cudaStream_t s) {
  PairParams pp = p.pair_params();
  pp.k = k;
  pp.kp0 = kp0;
  pp.nkp = nkp;
  pp.diag = diag;
  const cplx_t<T>* psi = (const cplx_t<T>*)p.psi;
  const cplx_t<T>* gam = (const cplx_t<T>*)p.gam;
  cplx_t<T>* S0 = (cplx_t<T>*)p.scratch;
  cplx_t<T>* S1 = (cplx_t<T>*)p.scratch2;
  cplx_t<T>* G = (cplx_t<T>*)p.gpsi;
  switch (p.N[0]) {
#define OCCRI_VJP_CASE(NN) \
  case NN:                 \
    return pairs::run_vjp_wave<T, NN>(pp, psi, gam, S0, S1, G, dacc, s);
    OCCRI_FOR_EACH_N(OCCRI_VJP_CASE)
#undef OCCRI_VJP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_vjp_wave<float>(const Plan&, int, int, int, int, double*,
                                            cudaStream_t);
template cudaError_t launch_vjp_wave<double>(const Plan&, int, int, int, int, double*,
                                             cudaStream_t);
template cudaError_t launch_pair_wave<float>(const Plan&, int, int, int, int, cudaStream_t, void*,
                                             void*, cudaEvent_t*, cudaEvent_t);
template cudaError_t launch_pair_wave<double>(const Plan&, int, int, int, int, cudaStream_t, void*,
                                              void*, cudaEvent_t*, cudaEvent_t);
template cudaError_t launch_qtables<float>(const Plan&, cudaStream_t);
template cudaError_t launch_qtables<double>(const Plan&, cudaStream_t);
template cudaError_t launch_domega_wave<float>(const Plan&, int, int, int, int, cudaStream_t);
template cudaError_t launch_domega_wave<double>(const Plan&, int, int, int, int, cudaStream_t);

}  // namespace occri
