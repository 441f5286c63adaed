// Hessian row tables and folds (internal; see k_hessian.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dq {

cudaError_t hess_rows(const double *params, const int32_t *occ, int V, const int32_t *shift_v, const double *shift,
                      int J, int batch, const double *data, int nfeat, const double *rw, int nobs, double *prow,
                      double *drow, double *wrow, int nsm, cudaStream_t s, int64_t *launches);
cudaError_t hess_combine(const double *G, const int32_t *vrow0, const int32_t *nshift, const double *coef, int j0,
                         int nv, int v0, int batch, int V, double *Ht, cudaStream_t s, int64_t *launches);
cudaError_t hess_fold(const double *Ht, const int32_t *optr, const int32_t *oidx, int P, int V, double *H,
                      cudaStream_t s, int64_t *launches);

// Gradients of expectations by shift rules (density circuits):
// g[v0 + vl] = sum_s coef[j_s] sum_r sum_o w[r][o] E[((j_s - j0) * batch + r) * nobs + o]
// over the shift rows j_s of local occurrence vl (w = NULL: ones).
cudaError_t shift_combine(const double *E, const double *w, const int32_t *vrow0, const int32_t *nshift,
                          const double *coef, int j0, int nv, int v0, int batch, int nobs, double *g, cudaStream_t s,
                          int64_t *launches);
// grad[p] = sum over occurrences v of p of g[v].
cudaError_t shift_fold(const double *g, const int32_t *optr, const int32_t *oidx, int P, double *grad, cudaStream_t s,
                       int64_t *launches);

}  // namespace dq
