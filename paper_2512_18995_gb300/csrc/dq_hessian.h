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

}  // namespace dq
