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

// ctl (recording mode, else NULL): ctl[0] steps since recording was enabled, ctl[1]
// records written; only every `every`-th step is integrated.
__device__ __forceinline__ bool diag_skip(const int64_t *ctl, int every) {
  return ctl != nullptr && (ctl[0] + 1) % every != 0;
}

template <typename T>
__global__ void __launch_bounds__(kDiagThreads) diagnostics_kernel(const T *q, bool pert, int64_t stride, int Np,
                                                                  const MeshRec *mesh, const double *xn, double px,
                                                                  double py, const double *wq, double c, int64_t K,
                                                                  double *part, const int64_t *ctl, int every) {
  if (diag_skip(ctl, every)) return;   // uniform over the grid
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

// Recording mode: one record (t, mass, E_K, momentum x, y, area) into slot
// ctl[1] mod cap of the ring hist, then the counters advance.
__global__ void __launch_bounds__(kDiagThreads) diagnostics_record_kernel(const double *part, int nblocks,
                                                                         const double *clock, int64_t *ctl, int every,
                                                                         double *hist, int64_t cap) {
  const bool skip = diag_skip(ctl, every);
  __shared__ double tot[5];
  if (!skip) {
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
      for (int k = 0; k < 5; ++k) acc[k] += part[5 * b + k];
    block_sum5(acc, tot);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!skip) {
      double *r = hist + 6 * (ctl[1] % cap);
      r[0] = clock[0];
      r[1] = tot[0];
      r[2] = tot[1] / tot[4];
      r[3] = tot[2];
      r[4] = tot[3];
      r[5] = tot[4];
      ctl[1] += 1;
    }
    ctl[0] += 1;
  }
}

static_assert(kDiagBlocks >= kRecMaxCtas, "the partials buffer also serves the fused record");
int diagnostics_scratch_doubles() { return 5 * kDiagBlocks; }

static int64_t diag_blocks(int64_t K) {
  int64_t blocks = (K + kDiagThreads - 1) / kDiagThreads;
  if (blocks > kDiagBlocks) blocks = kDiagBlocks;
  return blocks < 1 ? 1 : blocks;
}

static void launch_partials(int N, const void *q, bool is_float, bool perturbation, int64_t stride, const MeshRec *mesh,
                            const double *xn, double px, double py, const double *wq, double c, int64_t K, double *part,
                            const int64_t *ctl, int every, cudaStream_t st) {
  const int Np = (N + 1) * (N + 2) / 2;
  const unsigned blocks = (unsigned)diag_blocks(K);
  if (is_float)
    diagnostics_kernel<float><<<blocks, kDiagThreads, 0, st>>>((const float *)q, perturbation, stride, Np, mesh, xn, px,
                                                                 py, wq, c, K, part, ctl, every);
  else
    diagnostics_kernel<double><<<blocks, kDiagThreads, 0, st>>>((const double *)q, perturbation, stride, Np, mesh, xn,
                                                                  px, py, wq, c, K, part, ctl, every);
}

int launch_diagnostics(int N, const void *q, bool is_float, bool perturbation, int64_t stride, const MeshRec *mesh,
                       const double *xn, double px, double py, const double *wq, double c, int64_t K, double *part,
                       double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  launch_partials(N, q, is_float, perturbation, stride, mesh, xn, px, py, wq, c, K, part, nullptr, 1, st);
  diagnostics_reduce_kernel<<<1, kDiagThreads, 0, st>>>(part, (int)diag_blocks(K), out);
  return (int)cudaGetLastError();
}

int launch_diagnostics_record(int N, const void *q, bool is_float, bool perturbation, int64_t stride,
                              const MeshRec *mesh, const double *xn, double px, double py, const double *wq, double c,
                              int64_t K, double *part, const double *clock, int64_t *ctl, int every, double *hist,
                              int64_t cap, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  launch_partials(N, q, is_float, perturbation, stride, mesh, xn, px, py, wq, c, K, part, ctl, every, st);
  diagnostics_record_kernel<<<1, kDiagThreads, 0, st>>>(part, (int)diag_blocks(K), clock, ctl, every, hist, cap);
  return (int)cudaGetLastError();
}

}  // namespace gb
