// Right-hand sides of the Laguerre-harmonic chain (Section 4.1, Eq.
// laguerre_h).  Harmonic m of the time-domain wave field solves
//
//   div(V grad Q_m) - (h^2 / (4 rho^2)) Q_m
//       = -delta(x - x_0) f_m + (h^2 / rho^2) a_m sum_{k<m} (m - k) w_k Q_k,
//
//   a_m = sqrt(m! / (m + alpha)!),   w_k = sqrt((k + alpha)! / k!),
//
// i.e. the operator of ax_solve with kappa = V, q = h^2 / (4 rho^2) and
// physical right-hand side f = f_m src - c2 a_m S_m, c2 = h^2 / rho^2,
// S_m = sum_{k<m} (m - k) w_k Q_k.  The sum is carried by two running fields
// instead of being re-summed over all previous harmonics:
//
//   T_{m+1} = T_m + w_m Q_m        (T_m = sum_{k<m} w_k Q_k)
//   S_{m+1} = S_m + T_{m+1}        (S_{m+1} - S_m = sum_{k<=m} w_k Q_k),
//
// so each harmonic costs one pass over five fields (read Q, T, S, c2, src;
// write T, S, f) whatever m is.  The weights are host scalars.
#include <algorithm>
#include <cmath>

#include "ax_common.cuh"

namespace ax {
namespace {

// Q may be null (then w_m is 0 and Q is not read: harmonic 0 has no solved
// field to add).
__global__ void laguerre_step_kernel(const double *Q, double *__restrict__ T, double *__restrict__ S,
                                     const double *__restrict__ c2, const double *__restrict__ src, double w_m,
                                     double a_next, double f_next, double *__restrict__ f_out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const double t = Q ? fma(w_m, Q[e], T[e]) : T[e];
    const double s = S[e] + t;
    T[e] = t;
    S[e] = s;
    f_out[e] = fma(f_next, src[e], -c2[e] * a_next * s);
  }
}

}  // namespace
}  // namespace ax

extern "C" int ax_laguerre_step(ax_operator *op, const double *Q, double *T, double *S, const double *c2,
                                const double *src, double w_m, double a_next, double f_next, double *f_out,
                                void *stream) {
  if (!op || !T || !S || !c2 || !src || !f_out) return AX_ERR_INVALID_ARG;
  if (!std::isfinite(w_m) || !std::isfinite(a_next) || !std::isfinite(f_next)) return AX_ERR_INVALID_ARG;
  if (!Q && w_m != 0.0) return AX_ERR_INVALID_ARG;
  if (Q && (Q == T || Q == S || Q == f_out)) return AX_ERR_INVALID_ARG;  // T, S, f_out are written
  const size_t n = (size_t)op->nr * op->nz;
  const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
  ax::note_launch();
  ax::laguerre_step_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(Q, T, S, c2, src, w_m, a_next, f_next, f_out,
                                                                      n);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}
