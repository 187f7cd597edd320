// Device helpers shared by the 3D stage kernels (gb_kernels3d.cu: the one-thread-per-node
// kernels; gb_kernels3d_tc.cu: the tensor-core kernel): the 10-moment flux matrix product,
// the stage motion factors and the per-element geometry at a stage (Sec. 5, GCL).
#ifndef GB_KERNELS3D_DEV_CUH
#define GB_KERNELS3D_DEV_CUH

#include <cuda_runtime.h>

#include <cstdint>

#include "gb3d_internal.h"

namespace gb {

// geometry block per element (in T): G^-1 (9, row-major r_x r_y r_z s_x ... t_z),
// vertex grid velocities (4 x 3, vertex-major), per face nx ny nz Fscale (16), padding
constexpr int GEO3 = 40, GEO3_V = 9, GEO3_F = 21;

template <typename T> __device__ __forceinline__ T fma3(T a, T b, T c);
template <> __device__ __forceinline__ double fma3<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <> __device__ __forceinline__ float fma3<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ bool bad3(double v) { return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000; }
__device__ __forceinline__ bool bad3(float v) { return (__float_as_int(v) & 0x7f800000) == 0x7f800000; }

// y = At_n w for the 10-moment Hermite system (Sec. 2 structure, 3D)
template <typename T>
__device__ __forceinline__ void apply_An(T nx, T ny, T nz, const T (&w)[10], T (&y)[10]) {
  const T s2 = (T)1.41421356237309504880;
  y[0] = nx * w[1] + ny * w[2] + nz * w[3];
  y[1] = nx * fma3(s2, w[7], w[0]) + ny * w[4] + nz * w[5];
  y[2] = nx * w[4] + ny * fma3(s2, w[8], w[0]) + nz * w[6];
  y[3] = nx * w[5] + ny * w[6] + nz * fma3(s2, w[9], w[0]);
  y[4] = nx * w[2] + ny * w[1];
  y[5] = nx * w[3] + nz * w[1];
  y[6] = ny * w[3] + nz * w[2];
  y[7] = s2 * nx * w[1];
  y[8] = s2 * ny * w[2];
  y[9] = s2 * nz * w[3];
}

// stage motion factors from the device clock: v = g1 S1 + g2 S2, x_i = x_n + x1 S1 + x2 S2
// (S1, S2: the per-vertex velocity shapes of the motion, 3 components each)
struct Motion3 { double g1, g2, x1, x2; };

__device__ __forceinline__ Motion3 stage_motion3(const Stage3Args &a, int stage) {
  Motion3 m{0.0, 0.0, 0.0, 0.0};
  if (!a.moving) return m;
  const double w = a.omega;
  if (stage < 0) {
    m.g1 = cos(w * a.rhs_time);
    m.g2 = sin(w * a.rhs_time);
    return m;
  }
  const double t = a.clock[0], dt = a.dt;
  const double cst[4] = {0.0, 0.5, 0.5, 1.0};
  const double ti = t + cst[stage] * dt;
  m.g1 = cos(w * ti);
  m.g2 = sin(w * ti);
  if (stage > 0) {
    const double tp = t + cst[stage - 1] * dt, ap = cst[stage == 3 ? 3 : 1];   // a_{i,i-1} = 1/2, 1/2, 1
    m.x1 = dt * ap * cos(w * tp);
    m.x2 = dt * ap * sin(w * tp);
  }
  return m;
}

// Geometry of element `elem` at the stage (one thread): G^-1, the vertex grid velocities, the
// outward normals and Fscale of the four faces into gout (GEO3 values).  Vertex positions and
// their differences in FP64, the small motion increments x1 S1 + x2 S2 in T, everything after
// the edge vectors in T (FP64 in GB_FP64).
template <typename T>
__device__ __forceinline__ void element_geometry3(const Stage3Args &a, int64_t elem, double x1, double x2, double g1,
                                                  double g2, T *gout) {
  const MeshRec3 rec = a.mesh[elem];
  // stage positions x_n + shift + x1 S1 + x2 S2: the vertex positions and their differences
  // in FP64, the motion increments (small against the edges) in T
  const T x1t = (T)x1, x2t = (T)x2, g1t = (T)g1, g2t = (T)g2;
  double P0[3];
  T S0[3];   // x1 S1 + x2 S2 of vertex 0
  T dv[4][3], vv[4][3];   // dv[k] = P_k - P_0 (dv[0] = 0); vv[k] the grid velocity of vertex k
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t v = rec.v[k];
    const double2 *sh = reinterpret_cast<const double2 *>(a.shape) + 3 * v;
    const double2 s01 = sh[0], s23 = sh[1], s45 = sh[2];
    const T S1[3] = {(T)s01.x, (T)s01.y, (T)s23.x}, S2[3] = {(T)s23.y, (T)s45.x, (T)s45.y};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double Pk = a.xn[3 * v + d] + rec.shift[3 * k + d] * a.period[d];
      const T inc = fma3(x1t, S1[d], x2t * S2[d]);
      vv[k][d] = fma3(g1t, S1[d], g2t * S2[d]);
      if (k == 0) {
        P0[d] = Pk;
        S0[d] = inc;
        dv[0][d] = (T)0;
      } else {
        dv[k][d] = (T)(Pk - P0[d]) + (inc - S0[d]);
      }
    }
  }
  T G[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int q = 0; q < 3; ++q) G[d][q] = (T)0.5 * dv[q + 1][d];
  const T C00 = G[1][1] * G[2][2] - G[1][2] * G[2][1];
  const T C01 = G[1][2] * G[2][0] - G[1][0] * G[2][2];
  const T C02 = G[1][0] * G[2][1] - G[1][1] * G[2][0];
  const T J = G[0][0] * C00 + G[0][1] * C01 + G[0][2] * C02;
  if (!(J > (T)0)) atomicOr(a.status, GB_STATUS_MESH);
  const T iJ = (T)1 / J;
  // G^-1 = adj(G) / J; row a of G^-1 is the gradient of reference coordinate a
  T *g = gout;
  g[0] = C00 * iJ; g[3] = C01 * iJ; g[6] = C02 * iJ;
  g[1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) * iJ;
  g[4] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) * iJ;
  g[7] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) * iJ;
  g[2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) * iJ;
  g[5] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) * iJ;
  g[8] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) * iJ;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) g[GEO3_V + 3 * k + d] = vv[k][d];
  // faces (local vertex triples) and the orientation of (P_b - P_a) x (P_c - P_a)
  // relative to the outward normal; compile-time so that dv stays in registers
  constexpr int fvt[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
  constexpr float fsign[4] = {-1.0f, 1.0f, 1.0f, -1.0f};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int va = fvt[f][0], vb = fvt[f][1], vc = fvt[f][2];
    const T ux = dv[vb][0] - dv[va][0], uy = dv[vb][1] - dv[va][1], uz = dv[vb][2] - dv[va][2];
    const T wx = dv[vc][0] - dv[va][0], wy = dv[vc][1] - dv[va][1], wz = dv[vc][2] - dv[va][2];
    const T nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    const T len = sqrt(nx * nx + ny * ny + nz * nz);
    const T sg = (T)fsign[f] / len;
    g[GEO3_F + 4 * f] = nx * sg;
    g[GEO3_F + 1 + 4 * f] = ny * sg;
    g[GEO3_F + 2 + 4 * f] = nz * sg;
    g[GEO3_F + 3 + 4 * f] = (T)0.25 * len * iJ;   // face area / (2 J)
  }
}

}  // namespace gb

#endif
