// Diagnostics of the state on the moving mesh: the kinetic energy of Sec. 7.2
// and the integrals that the scheme conserves (mass, momentum) plus the area.
#include <cuda_runtime.h>

#include <cstdint>

#include "gb_internal.h"

namespace gb {

// Integrals of the nodal interpolants (int f = J sum_i wq_i f_i on each affine element):
// mass, kinetic energy rho |u|^2 / 2 = c^2 (q2^2 + q3^2) / (2 q1), momentum and area.
// One thread per element (grid-stride), block partials in a fixed order, then one
// block sums the partials: the result does not depend on scheduling.
constexpr int kDiagBlocks = 1184, kDiagThreads = 256;

__device__ __forceinline__ void block_sum5(double (&acc)[5], double *part) {
  __shared__ double red[kDiagThreads / 32][5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    part[threadIdx.x] = v;
  }
}

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) diagnostics_kernel(const T *q, bool pert, int64_t stride, int Np,
                                                                  const MeshRec *mesh, const double *xn, double px,
                                                                  double py, const double *wq, double c, int64_t K,
                                                                  double *part) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < K; e += (int64_t)gridDim.x * blockDim.x) {
    const MeshRec rec = mesh[e];
    double x[3], y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      x[k] = xn[2 * rec.v[k]] + rec.shift[2 * k] * px;
      y[k] = xn[2 * rec.v[k] + 1] + rec.shift[2 * k + 1] * py;
    }
    const double J = 0.25 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
    const T *qe = q + e * stride;
    double m = 0.0, ke = 0.0, mu = 0.0, mv = 0.0, w = 0.0;
    for (int n = 0; n < Np; ++n) {
      const double q1 = (double)qe[n] + (pert ? 1.0 : 0.0);
      const double q2 = (double)qe[Np + n], q3 = (double)qe[2 * Np + n];
      const double wn = wq[n];
      m += wn * q1;
      ke += wn * 0.5 * c * c * (q2 * q2 + q3 * q3) / q1;
      mu += wn * c * q2;
      mv += wn * c * q3;
      w += wn;
    }
    acc[0] += J * m; acc[1] += J * ke; acc[2] += J * mu; acc[3] += J * mv; acc[4] += J * w;
  }
  block_sum5(acc, part + 5 * blockIdx.x);
}

__global__ void __launch_bounds__(kDiagThreads) diagnostics_reduce_kernel(const double *part, int nblocks, double *out) {
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] += part[5 * b + k];
  block_sum5(acc, out);
}

int diagnostics_scratch_doubles() { return 5 * kDiagBlocks; }

int launch_diagnostics(int N, const void *q, bool is_float, bool perturbation, int64_t stride, const MeshRec *mesh,
                       const double *xn, double px, double py, const double *wq, double c, int64_t K, double *part,
                       double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int Np = (N + 1) * (N + 2) / 2;
  int64_t blocks = (K + kDiagThreads - 1) / kDiagThreads;
  if (blocks > kDiagBlocks) blocks = kDiagBlocks;
  if (blocks < 1) blocks = 1;
  if (is_float)
    diagnostics_kernel<float><<<(unsigned)blocks, kDiagThreads, 0, st>>>((const float *)q, perturbation, stride, Np, mesh,
                                                                           xn, px, py, wq, c, K, part);
  else
    diagnostics_kernel<double><<<(unsigned)blocks, kDiagThreads, 0, st>>>((const double *)q, perturbation, stride, Np,
                                                                            mesh, xn, px, py, wq, c, K, part);
  diagnostics_reduce_kernel<<<1, kDiagThreads, 0, st>>>(part, (int)blocks, out);
  return (int)cudaGetLastError();
}

}  // namespace gb
