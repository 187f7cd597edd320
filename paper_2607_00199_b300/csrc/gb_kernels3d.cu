// CUDA kernels of the 3D (tetrahedral, 10-field) ALE-DG Galerkin-Boltzmann solver.
//
// One fused kernel per SARK stage (Sec. 4) computes, for a tile of E elements per CTA:
//   geometry  : stage vertex positions y_i = y_n + xfac1 S1(X) + xfac2 S2(X) and
//               velocities v_y = gfac1 S1(X) + gfac2 S2(X) of the travelling-wave motion
//               (Sec. 5) in FP64, then the edge vectors (FP64 differences) and from them
//               G = dx/d(r,s,t), J, G^-1, the four outward normals and Fscale = face
//               area / (2 J) in the field precision (FP64 in GB_FP64) (GCL);
//   volume    : Dr, Ds, Dt of the 10 fields, chain rule, (A + v_G) . grad q;
//   surface   : neighbour traces through the face-node permutation table, the upwind
//               fluxes c/2 (|At_n| - At_n) dq (|At_n| = alpha At_n^2 + beta At_n^4,
//               applied as repeated products with the sparse At_n) and max(v_G.n, 0) dq,
//               scaled by Fscale and lifted with LIFT;
//   cubature  : q1..q4 at the degree-3N points, Ntilde there, projected onto fields 5..10;
//   update    : the SARK stage / final combination (fields 1..4 RK4, 5..10 exponential).
// One thread per (element, node) for the volume, lift and update phases; the surface
// and cubature phases loop over (element, face node) and (element, point) items.
// T = double (GB_FP64) or float (GB_MIXED: FP32 perturbations of the rest state, FP64
// geometry, motion and SARK coefficients).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "gb3d_internal.h"
#include "gb_kernels3d_dev.cuh"

namespace gb {

template <int N>
struct Dim3 {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NFN = 4 * Nfp;
  static constexpr int qc = (3 * N + 2) / 2;
  static constexpr int Nc = qc * qc * qc;
  static constexpr int NQ = 10 * Np;
};

// elements per CTA: (T, N)
template <typename T, int N> struct Tile3 { static constexpr int E = sizeof(T) == 8 ? (N <= 2 ? 16 : (N == 3 ? 8 : 4)) : (N <= 2 ? 32 : (N == 3 ? 12 : 8)); };

// operator block (in T): Dr, Ds, Dt, LIFT and the barycentric table, then I and P, then
// (in int) the neighbour node table and the face masks.  The first part always lives in
// shared memory; I and P too in FP32 up to N = 3 (IP_SMEM), otherwise they are read
// through the L1 cache.
template <typename T, int N>
struct Op3 {
  typedef Dim3<N> D;
  static constexpr bool IP_SMEM = sizeof(T) == 4 && N <= 3;
  static constexpr int DrT = 0;                           // [m][n] = Dr[n][m]
  static constexpr int DsT = DrT + D::Np * D::Np;
  static constexpr int DtT = DsT + D::Np * D::Np;
  static constexpr int LiftT = DtT + D::Np * D::Np;       // [j][n] = LIFT[n][j]
  static constexpr int Bary = LiftT + D::NFN * D::Np;     // [n][4]
  static constexpr int IT = Bary + 4 * D::Np;             // [m][c] = I[c][m]; row-major I[c][m] when IP_SMEM
  static constexpr int PT = IT + D::Np * D::Nc;           // [c][n] = P[n][c]
  static constexpr int Size = PT + D::Nc * D::Np;
  static constexpr int SmemSize = IP_SMEM ? Size : IT;    // staged in shared memory
  static constexpr int TabInts = 4 * 4 * 6 * D::Nfp + 4 * D::Nfp;   // neighbour node table, fmask
  // shared-memory path: cubature points per work item (the last item of an element may hold
  // fewer; N = 3: 12 elements x 21 items of <= 6 of the 125 points fill a 256-thread CTA in one
  // round), nodes per projection item, vector widths
  static constexpr int CPI = N == 3 ? 6 : (N == 2 ? 4 : 2);
  // projection items (element, NG nodes, FG fields); N = 3: 12 x 10 x 2 = 240 items of 2 x 3
  // outputs in one round, instead of 360 items of 4 x 1 (104 threads ran a second one)
  static constexpr int NG = N == 3 ? 2 : (D::Np % 4 == 0 ? 4 : (D::Np % 2 == 0 ? 2 : 1));
  static constexpr int FG = N == 3 ? 3 : 1;
  static_assert(D::Np % NG == 0 && 6 % FG == 0, "projection items must split the nodes and fields evenly");
};


// asynchronous global -> shared copies (cp.async): 16 bytes (both addresses 16-byte aligned)
// or 4 bytes
__device__ __forceinline__ void cp_async16_3(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4_3(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// the own fields of tile t (nel elements, contiguous) into shared memory, asynchronously
template <typename T>
__device__ __forceinline__ void prefetch_tile3(const T *qin, int64_t elem0, int nel, int NQ, T *dst, bool al16) {
  const char *src = reinterpret_cast<const char *>(qin + elem0 * NQ);
  char *d = reinterpret_cast<char *>(dst);
  const int bytes = nel * NQ * (int)sizeof(T);
  const int b16 = al16 ? (bytes & ~15) : 0;
  for (int i = 16 * (int)threadIdx.x; i < b16; i += 16 * (int)blockDim.x) cp_async16_3(d + i, src + i);
  for (int i = b16 + 4 * (int)threadIdx.x; i < bytes; i += 4 * (int)blockDim.x) cp_async4_3(d + i, src + i);
  asm volatile("cp.async.commit_group;" ::: "memory");
}


template <typename T, int N, int STAGE>
__global__ void __launch_bounds__(((Tile3<T, N>::E * Dim3<N>::Np + 31) / 32) * 32)
stage3_kernel(const Stage3Args a) {
  typedef Dim3<N> D;
  typedef Op3<T, N> L;
  constexpr int E = Tile3<T, N>::E;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN, Nc = D::Nc, NQ = D::NQ;
  constexpr bool PERTURB = sizeof(T) == 4;
  const T ISQ2 = (T)0.70710678118654752440;

  extern __shared__ __align__(16) unsigned char smem3[];
  T *sops = reinterpret_cast<T *>(smem3);
  int *stab = reinterpret_cast<int *>(sops + L::SmemSize);   // nbr_node [f][f2][p][k], then fmask [f][k]
  T *sq = reinterpret_cast<T *>(stab + ((L::TabInts + 3) & ~3));
  T *sflux = sq + E * NQ;          // [E][10][NFN]
  T *snt = sflux + E * 10 * NFN;   // [E][6][Nc]
  T *sgeo = snt + E * 6 * Nc;      // [E][GEO3]
  // FP32 up to N = 3: a second own-field buffer, filled for the next tile while this one computes
  constexpr bool DB = sizeof(T) == 4 && N <= 3;
  static_assert(!DB || (L::SmemSize + ((L::TabInts + 3) & ~3) + E * (NQ + 10 * NFN + 6 * Nc + GEO3)) % 4 == 0,
                "the second own-field buffer must start on a 16-byte boundary");
  T *const sqA = sq, *const sqB = sgeo + E * GEO3;
  // FP32 at N = 3, with spare threads after the node threads: those threads form the next tile's
  // geometry during this tile's last phase, into a second geometry buffer
  constexpr int NODE_THREADS = E * Np, THREADS = ((E * Np + 31) / 32) * 32;
  constexpr bool PG = DB && THREADS - NODE_THREADS >= E;
  T *const sgA = sgeo, *const sgB = sqB + E * NQ;
  __shared__ double s_motion[4];

  const int tid = threadIdx.x, nthr = blockDim.x;
  const T *gops = reinterpret_cast<const T *>(a.ops);
  for (int i = tid; i < L::SmemSize; i += nthr) sops[i] = gops[i];
  for (int i = tid; i < L::TabInts; i += nthr) stab[i] = a.tab[i];
  if (tid == 0) {
    const Motion3 m = stage_motion3(a, STAGE);
    s_motion[0] = m.g1; s_motion[1] = m.g2; s_motion[2] = m.x1; s_motion[3] = m.x2;
    if (STAGE == 3 && blockIdx.x == 0) {
      // final vertex update factors dt sum_j b_j (cos, sin)(omega t_j)
      double f1 = 0.0, f2 = 0.0;
      if (a.moving) {
        const double t = a.clock[0], dt = a.dt, w = a.omega;
        f1 = dt * (cos(w * t) / 6.0 + cos(w * (t + 0.5 * dt)) * (2.0 / 3.0) + cos(w * (t + dt)) / 6.0);
        f2 = dt * (sin(w * t) / 6.0 + sin(w * (t + 0.5 * dt)) * (2.0 / 3.0) + sin(w * (t + dt)) / 6.0);
      }
      const_cast<double *>(a.clock)[1] = f1;
      const_cast<double *>(a.clock)[2] = f2;
    }
  }
  __syncthreads();
  const double g1 = s_motion[0], g2 = s_motion[1], x1 = s_motion[2], x2 = s_motion[3];
  const int *snbr = stab;
  const int *sfmask = stab + 4 * 4 * 6 * Nfp;
  const T *gIT = (L::IP_SMEM ? sops : gops) + L::IT;
  const T *gPT = (L::IP_SMEM ? sops : gops) + L::PT;

  // this stage's SARK coefficients of the two field classes, converted once per thread
  T kE[2], kA0[2], kA1[2], kB0[2], kB1[2];
#pragma unroll
  for (int cl = 0; cl < 2; ++cl) {
    kE[cl] = (T)a.co.E[cl][STAGE < 0 ? 0 : (STAGE < 3 ? STAGE + 1 : 4)];
    kA0[cl] = (T)(STAGE == 0 ? a.co.A[cl][4] : STAGE == 1 ? a.co.A[cl][8] : STAGE == 2 ? a.co.A[cl][12] : 0.0);
    kA1[cl] = (T)(STAGE == 1 ? a.co.A[cl][9] : STAGE == 2 ? a.co.A[cl][14] : 0.0);
    kB0[cl] = (T)(STAGE == 1 ? a.co.B[cl][0] : STAGE == 2 ? a.co.B[cl][2] : STAGE == 3 ? a.co.B[cl][3] : 0.0);
    kB1[cl] = (T)a.co.B[cl][1];
  }
  const T *qin = reinterpret_cast<const T *>(a.qin);
  const int e_loc = tid / Np, n_loc = tid - (tid / Np) * Np;
  const bool node_thread = e_loc < E;
  const T c = (T)a.c;

  const int64_t ntiles = (a.K + E - 1) / E;
  const bool al16 = (reinterpret_cast<uintptr_t>(qin) & 15) == 0;
  if (DB && (int64_t)blockIdx.x < ntiles) {
    const int64_t e0 = (int64_t)blockIdx.x * E;
    prefetch_tile3<T>(qin, e0, (int)((a.K - e0) < E ? (a.K - e0) : E), NQ, sqA, al16);
  }
  if (PG && (int64_t)blockIdx.x < ntiles) {   // the first tile's geometry
    const int64_t e0 = (int64_t)blockIdx.x * E;
    const int n0 = (int)((a.K - e0) < E ? (a.K - e0) : E);
    for (int e = tid; e < n0; e += nthr) element_geometry3<T>(a, e0 + e, x1, x2, g1, g2, sgA + e * GEO3);
  }
  int cur = 0, gcur = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t elem0 = tile * E;
    const int nel = (int)((a.K - elem0) < E ? (a.K - elem0) : E);
    T *sq = (DB && cur) ? sqB : sqA;
    T *sg = (PG && gcur) ? sgB : sgA;
    if constexpr (DB) {
      // this tile's fields have arrived and every thread has left the previous tile; the other
      // buffer (the previous tile's) takes the next tile's
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
      const int64_t nt = tile + gridDim.x;
      if (nt < ntiles) {
        const int64_t e1 = nt * E;
        prefetch_tile3<T>(qin, e1, (int)((a.K - e1) < E ? (a.K - e1) : E), NQ, cur ? sqA : sqB, al16);
      }
      cur ^= 1;
    } else {
      const T *src = qin + elem0 * NQ;
      const int cnt = nel * NQ;
      for (int i = tid; i < cnt; i += nthr) sq[i] = src[i];
    }
    // ---- geometry, one thread per element (with PG already formed during the previous tile and
    //      made visible, with this tile's fields, by the barrier above) ----
    if constexpr (!PG) {
      for (int e = tid; e < nel; e += nthr) element_geometry3<T>(a, elem0 + e, x1, x2, g1, g2, sg + e * GEO3);
      __syncthreads();
    }

    // ---- volume term, one thread per node ----
    T rhs[10];
    if (node_thread && e_loc < nel) {
      const T *q = sq + e_loc * NQ;
      T qr[10], qs[10], qt[10];
#pragma unroll
      for (int f = 0; f < 10; ++f) { qr[f] = 0; qs[f] = 0; qt[f] = 0; }
#pragma unroll 4
      for (int m = 0; m < Np; ++m) {
        const T dr = sops[L::DrT + m * Np + n_loc], ds = sops[L::DsT + m * Np + n_loc], dt = sops[L::DtT + m * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 10; ++f) {
          const T v = q[f * Np + m];
          qr[f] = fma3(dr, v, qr[f]);
          qs[f] = fma3(ds, v, qs[f]);
          qt[f] = fma3(dt, v, qt[f]);
        }
      }
      const T *g = sg + e_loc * GEO3;
      const T *bl = sops + L::Bary + 4 * n_loc;
      const T *gv = g + GEO3_V;
      const T vgx = bl[0] * gv[0] + bl[1] * gv[3] + bl[2] * gv[6] + bl[3] * gv[9];
      const T vgy = bl[0] * gv[1] + bl[1] * gv[4] + bl[2] * gv[7] + bl[3] * gv[10];
      const T vgz = bl[0] * gv[2] + bl[1] * gv[5] + bl[2] * gv[8] + bl[3] * gv[11];
      T qx[10], qy[10], qz[10];
#pragma unroll
      for (int f = 0; f < 10; ++f) {
        qx[f] = fma3(g[0], qr[f], fma3(g[3], qs[f], g[6] * qt[f]));
        qy[f] = fma3(g[1], qr[f], fma3(g[4], qs[f], g[7] * qt[f]));
        qz[f] = fma3(g[2], qr[f], fma3(g[5], qs[f], g[8] * qt[f]));
      }
      // -c (At_x q_x + At_y q_y + At_z q_z) + v_G . grad q
      T ax[10], ay[10], az[10];
      apply_An<T>((T)1, (T)0, (T)0, qx, ax);
      apply_An<T>((T)0, (T)1, (T)0, qy, ay);
      apply_An<T>((T)0, (T)0, (T)1, qz, az);
#pragma unroll
      for (int f = 0; f < 10; ++f)
        rhs[f] = fma3(vgx, qx[f], fma3(vgy, qy[f], fma3(vgz, qz[f], -c * (ax[f] + ay[f] + az[f]))));
    }

    // ---- surface fluxes at the face nodes ----
    const T al = (T)((9.0 - 1.7320508075688772935) / 6.0), be = (T)((1.7320508075688772935 - 3.0) / 6.0);
    for (int item = tid; item < E * NFN; item += nthr) {
      const int e = item / NFN, j = item - NFN * (item / NFN);
      if (e >= nel) continue;
      const int f = j / Nfp, k = j - Nfp * (j / Nfp);
      const int vol = sfmask[f * Nfp + k];
      const int nb = a.mesh[elem0 + e].nbr[f];
      const int64_t e2 = nb >> 5;
      const int p = (nb >> 2) & 7, f2 = nb & 3;
      const int vol2 = snbr[((f * 4 + f2) * 6 + p) * Nfp + k];
      const T *qp = qin + e2 * NQ + vol2;
      const T *qm = sq + e * NQ + vol;
      T w[10];
#pragma unroll
      for (int fld = 0; fld < 10; ++fld) w[fld] = qp[fld * Np] - qm[fld * Np];
      const T *g = sg + e * GEO3;
      const T nx = g[GEO3_F + 4 * f], ny = g[GEO3_F + 1 + 4 * f], nz = g[GEO3_F + 2 + 4 * f], fs = g[GEO3_F + 3 + 4 * f];
      const T *bl = sops + L::Bary + 4 * vol;
      const T *gv = g + GEO3_V;
      T vn = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) vn = fma3(bl[k], fma3(gv[3 * k], nx, fma3(gv[3 * k + 1], ny, gv[3 * k + 2] * nz)), vn);
      const T ale = vn > (T)0 ? vn : (T)0;
      T y1[10], y2[10], y3[10], y4[10];
      apply_An<T>(nx, ny, nz, w, y1);
      apply_An<T>(nx, ny, nz, y1, y2);
      apply_An<T>(nx, ny, nz, y2, y3);
      apply_An<T>(nx, ny, nz, y3, y4);
      const T h = (T)0.5 * c;
      T *fl = sflux + e * 10 * NFN + j;
#pragma unroll
      for (int fld = 0; fld < 10; ++fld)
        fl[fld * NFN] = fs * fma3(ale, w[fld], h * (fma3(al, y2[fld], be * y4[fld]) - y1[fld]));
    }
    // ---- cubature: q1..q4 at the points, Ntilde there ----
    const T itau = (T)a.inv_tau;
    if constexpr (L::IP_SMEM) {
      // item = (element, group of CPI points): q1..q4 of the element in registers, one row of
      // I per point, so every operator load feeds four FMAs
      constexpr int CPI = L::CPI, NPG = (Nc + CPI - 1) / CPI;
      for (int item = tid; item < E * NPG; item += nthr) {
        const int e = item / NPG, c0 = (item - NPG * (item / NPG)) * CPI;
        const int npt = Nc - c0 < CPI ? Nc - c0 : CPI;   // points of this item
        if (e >= nel) continue;
        const T *q = sq + e * NQ;
        T qr4[4][Np];
#pragma unroll
        for (int f = 0; f < 4; ++f)
#pragma unroll
          for (int m = 0; m < Np; ++m) qr4[f][m] = q[f * Np + m];
#pragma unroll 1
        for (int k = 0; k < npt; ++k) {
          const int cpt = c0 + k;
          const T *irow = sops + L::IT + cpt * Np;
          T im[Np];
          if constexpr (Np % 4 == 0) {   // 16-byte rows: conflict-free vector loads
#pragma unroll
            for (int m = 0; m < Np; m += 4) {
              const float4 v = *reinterpret_cast<const float4 *>(irow + m);
              im[m] = v.x; im[m + 1] = v.y; im[m + 2] = v.z; im[m + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int m = 0; m < Np; ++m) im[m] = irow[m];
          }
          T q1 = 0, q2 = 0, q3 = 0, q4 = 0;
#pragma unroll
          for (int m = 0; m < Np; ++m) {
            q1 = fma3(im[m], qr4[0][m], q1);
            q2 = fma3(im[m], qr4[1][m], q2);
            q3 = fma3(im[m], qr4[2][m], q3);
            q4 = fma3(im[m], qr4[3][m], q4);
          }
          q1 += (T)1;
          const T r1 = itau / q1, rs = r1 * ISQ2;
          T *nt = snt + e * 6 * Nc + cpt;
          nt[0] = q2 * q3 * r1;
          nt[Nc] = q2 * q4 * r1;
          nt[2 * Nc] = q3 * q4 * r1;
          nt[3 * Nc] = q2 * q2 * rs;
          nt[4 * Nc] = q3 * q3 * rs;
          nt[5 * Nc] = q4 * q4 * rs;
        }
      }
    } else
    for (int item = tid; item < E * Nc; item += nthr) {
      const int e = item / Nc, cpt = item - Nc * (item / Nc);
      if (e >= nel) continue;
      const T *q = sq + e * NQ;
      T q1 = 0, q2 = 0, q3 = 0, q4 = 0;
#pragma unroll 4
      for (int m = 0; m < Np; ++m) {
        const T im = __ldg(gIT + m * Nc + cpt);
        q1 = fma3(im, q[m], q1);
        q2 = fma3(im, q[Np + m], q2);
        q3 = fma3(im, q[2 * Np + m], q3);
        q4 = fma3(im, q[3 * Np + m], q4);
      }
      if (PERTURB) q1 += (T)1;
      const T r1 = itau / q1, rs = r1 * ISQ2;
      T *nt = snt + e * 6 * Nc + cpt;
      nt[0] = q2 * q3 * r1;
      nt[Nc] = q2 * q4 * r1;
      nt[2 * Nc] = q3 * q4 * r1;
      nt[3 * Nc] = q2 * q2 * rs;
      nt[4 * Nc] = q3 * q3 * rs;
      nt[5 * Nc] = q4 * q4 * rs;
    }
    __syncthreads();

    // ---- projection P Ntilde (shared-memory path): item = (element, group of NG nodes,
    //      group of FG fields), written over the element's field tile (no longer needed) ----
    T *sproj = sq;   // [E][6][Np]
    if constexpr (L::IP_SMEM) {
      constexpr int NG = L::NG, NGR = Np / NG, FG = L::FG, NFG = 6 / FG;
      for (int item = tid; item < E * NGR * NFG; item += nthr) {
        const int fg = item % NFG, rest = item / NFG, gq = rest % NGR, e = rest / NGR;
        if (e >= nel) continue;
        const T *nt = snt + e * 6 * Nc + fg * FG * Nc;
        const T *pc = sops + L::PT + gq * NG;
        T acc[FG][NG];
#pragma unroll
        for (int ff = 0; ff < FG; ++ff)
#pragma unroll
          for (int i = 0; i < NG; ++i) acc[ff][i] = 0;
#pragma unroll 5
        for (int cpt = 0; cpt < Nc; ++cpt) {
          T pv[NG];
          if constexpr (NG == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(pc + cpt * Np);
            pv[0] = v.x; pv[1] = v.y; pv[2] = v.z; pv[3] = v.w;
          } else if constexpr (NG == 2) {
            const float2 v = *reinterpret_cast<const float2 *>(pc + cpt * Np);
            pv[0] = v.x; pv[1] = v.y;
          } else {
#pragma unroll
            for (int i = 0; i < NG; ++i) pv[i] = pc[cpt * Np + i];
          }
#pragma unroll
          for (int ff = 0; ff < FG; ++ff) {
            const T nv = nt[ff * Nc + cpt];
#pragma unroll
            for (int i = 0; i < NG; ++i) acc[ff][i] = fma3(pv[i], nv, acc[ff][i]);
          }
        }
#pragma unroll
        for (int ff = 0; ff < FG; ++ff) {
          T *o = sproj + e * 6 * Np + (fg * FG + ff) * Np + gq * NG;
#pragma unroll
          for (int i = 0; i < NG; ++i) o[i] = acc[ff][i];
        }
      }
      __syncthreads();
    }

    // ---- lift, projection, SARK update (node threads); the next tile's geometry (spare threads) ----
    if (PG && tid >= NODE_THREADS) {
      const int64_t nt = tile + gridDim.x;
      if (nt < ntiles) {
        const int64_t e1 = nt * E;
        const int n1 = (int)((a.K - e1) < E ? (a.K - e1) : E);
        for (int e = tid - NODE_THREADS; e < n1; e += nthr - NODE_THREADS)
          element_geometry3<T>(a, e1 + e, x1, x2, g1, g2, (gcur ? sgA : sgB) + e * GEO3);
      }
    }
    if (node_thread && e_loc < nel) {
      const T *fl = sflux + e_loc * 10 * NFN;
#pragma unroll 4
      for (int j = 0; j < NFN; ++j) {
        const T lj = sops[L::LiftT + j * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 10; ++f) rhs[f] = fma3(lj, fl[f * NFN + j], rhs[f]);
      }
      if constexpr (L::IP_SMEM) {
#pragma unroll
        for (int f = 0; f < 6; ++f) rhs[4 + f] += sproj[e_loc * 6 * Np + f * Np + n_loc];
      } else {
        const T *nt = snt + e_loc * 6 * Nc;
#pragma unroll 5
        for (int cpt = 0; cpt < Nc; ++cpt) {
          const T pc = __ldg(gPT + cpt * Np + n_loc);
#pragma unroll
          for (int f = 0; f < 6; ++f) rhs[4 + f] = fma3(pc, nt[f * Nc + cpt], rhs[4 + f]);
        }
      }
      const int64_t base = (elem0 + e_loc) * NQ + n_loc;
      const T dt = (T)a.dt;
      if (STAGE < 0) {
        T *F = reinterpret_cast<T *>(a.Fout);
#pragma unroll
        for (int f = 0; f < 10; ++f) F[base + f * Np] = rhs[f];
      } else {
        const T *qn = reinterpret_cast<const T *>(a.qn);
        T *qout = reinterpret_cast<T *>(a.qout);
        T *F0 = reinterpret_cast<T *>(a.F0);
        T *acc = reinterpret_cast<T *>(a.acc);
        bool bad = false;
        // every load of the node's ten fields is issued before any store (q_{n+1} overwrites
        // q_n in place at the last stage, so the compiler may not reorder them itself): one
        // memory round trip instead of one per field
        T xv[10], x0[10], x1[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) {
          const int64_t idx = base + f * Np;
          xv[f] = STAGE == 0 ? (L::IP_SMEM ? qin[idx] : sq[e_loc * NQ + f * Np + n_loc]) : qn[idx];   // stage 0: qin is q_n
          x0[f] = (STAGE == 1 || STAGE == 2) ? F0[idx] : (T)0;
          x1[f] = STAGE >= 2 ? acc[idx] : (T)0;
        }
#pragma unroll
        for (int f = 0; f < 10; ++f) {
          const int cl = f < 4 ? 0 : 1;
          const int64_t idx = base + f * Np;
          const T r = rhs[f], qv = xv[f];
          if (STAGE == 0) {
            F0[idx] = r;
            qout[idx] = kE[cl] * qv + dt * (kA0[cl] * r);
          } else if (STAGE == 1) {
            qout[idx] = kE[cl] * qv + dt * (kA0[cl] * x0[f] + kA1[cl] * r);
            acc[idx] = kB0[cl] * x0[f] + kB1[cl] * r;
          } else if (STAGE == 2) {
            qout[idx] = kE[cl] * qv + dt * (kA0[cl] * x0[f] + kA1[cl] * r);
            acc[idx] = x1[f] + kB0[cl] * r;
          } else {
            const T out = kE[cl] * qv + dt * (x1[f] + kB0[cl] * r);
            qout[idx] = out;
            bad |= bad3(out);
          }
        }
        if (STAGE == 3 && bad) atomicOr(a.status, GB_STATUS_NAN);
      }
    }
    // with the double buffers the next tile's first barrier (before any of its shared-memory
    // writes and before the next prefetch) also separates it from this tile's reads
    if constexpr (!DB) __syncthreads();
    gcur ^= 1;
  }
}

// ---------------------------------------------------------------------------
template <typename T, int N>
static size_t stage3_smem() {
  typedef Dim3<N> D;
  typedef Op3<T, N> L;
  constexpr int E = Tile3<T, N>::E;
  // second own-field buffer, second geometry buffer (stage3_kernel)
  constexpr bool DB = sizeof(T) == 4 && N <= 3;
  constexpr bool PG = DB && ((E * D::Np + 31) / 32) * 32 - E * D::Np >= E;
  return sizeof(T) * (size_t)L::SmemSize + sizeof(int) * (size_t)((L::TabInts + 3) & ~3) +
         sizeof(T) * (size_t)E * (D::NQ + 10 * D::NFN + 6 * D::Nc + GEO3 + (DB ? D::NQ : 0) + (PG ? GEO3 : 0));
}

template <typename T, int N, int STAGE>
static int launch3_one(const Stage3Args &a, cudaStream_t st, int num_sms) {
  constexpr int E = Tile3<T, N>::E;
  const int threads = ((E * Dim3<N>::Np + 31) / 32) * 32;
  const size_t smem = stage3_smem<T, N>();
  // the shared-memory opt-in and the occupancy are per-device facts, cached per device ordinal
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return (int)derr;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  static bool attr_set[64] = {};
  if (!attr_set[dev]) {
    cudaError_t err = cudaFuncSetAttribute(stage3_kernel<T, N, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    attr_set[dev] = true;
  }
  static int per_sm_d[64] = {};
  int &per_sm = per_sm_d[dev];
  if (per_sm == 0) {
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage3_kernel<T, N, STAGE>, threads, smem);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t ntiles = (a.K + E - 1) / E;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  stage3_kernel<T, N, STAGE><<<(unsigned)grid, threads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename T, int N>
static int launch3_n(const Stage3Args &a, cudaStream_t st, int num_sms) {
  switch (a.stage) {
    case -1: return launch3_one<T, N, -1>(a, st, num_sms);
    case 0: return launch3_one<T, N, 0>(a, st, num_sms);
    case 1: return launch3_one<T, N, 1>(a, st, num_sms);
    case 2: return launch3_one<T, N, 2>(a, st, num_sms);
    case 3: return launch3_one<T, N, 3>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_stage3(int N, bool fp64, const Stage3Args &a, void *stream, int num_sms) {
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64) {
    switch (N) {
      case 1: return launch3_n<double, 1>(a, st, num_sms);
      case 2: return launch3_n<double, 2>(a, st, num_sms);
      case 3: return launch3_n<double, 3>(a, st, num_sms);
      case 4: return launch3_n<double, 4>(a, st, num_sms);
    }
  } else {
    switch (N) {
      case 1: return launch3_n<float, 1>(a, st, num_sms);
      case 2: return launch3_n<float, 2>(a, st, num_sms);
      case 3: return launch3_n<float, 3>(a, st, num_sms);
      case 4: return launch3_n<float, 4>(a, st, num_sms);
    }
  }
  return (int)cudaErrorInvalidValue;
}

// ---- vertex update, motion shapes, node coordinates, precision conversion ----------

// x_{n+1} = x_n + fin1 S1(X) + fin2 S2(X); t_{n+1} = t_n + dt
__global__ void vertex_update3_kernel(double *xn, const double *shape, int64_t nv, double *clock, double dt) {
  const double f1 = clock[1], f2 = clock[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int d = 0; d < 3; ++d) xn[3 * i + d] += f1 * shape[6 * i + d] + f2 * shape[6 * i + 3 + d];
  if (blockIdx.x == 0 && threadIdx.x == 0) clock[0] += dt;
}

int launch_vertex_update3(double *xn, const double *shape, int64_t nv, double *clock, double dt, void *stream) {
  int64_t blocks = (nv + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  vertex_update3_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(xn, shape, nv, clock, dt);
  return (int)cudaGetLastError();
}

// Velocity shapes at the Lagrangian positions, v(X, t) = S1(X) cos(omega t) + S2(X) sin(omega t),
// stored per vertex as S1x S1y S1z S2x S2y S2z.
// Travelling wave (y only): v_y = -omega A(X) e^{-r^2/r0sq} cos(k X - omega t).
__global__ void shape3_kernel(const double *X, double *shape, int64_t nv, Wave3 m) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
    const double r2 = (y - m.yc) * (y - m.yc) + (z - m.zc) * (z - m.zc);
    const double amp = -m.omega * (m.A0 + m.A1 * x / m.Lx) * exp(-r2 / m.r0sq);
    const double kx = 2.0 * 3.14159265358979323846 / m.wavelength * x;
    double *o = shape + 6 * i;
    o[0] = 0.0; o[1] = amp * cos(kx); o[2] = 0.0;
    o[3] = 0.0; o[4] = amp * sin(kx); o[5] = 0.0;
  }
}

// Taylor-Green deformation (Sec. 7.2): x_d = X_d + A sin(omega t) S(X_a) S(X_b) over the other
// two coordinates a, b, S(s) = sin(2 pi (s + L/2) / L), omega = 2 pi / T: S1 = A omega (...), S2 = 0.
__global__ void shape3_tgv_kernel(const double *X, double *shape, int64_t nv, double A, double omega, double L) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    double S[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) S[d] = sin(2.0 * 3.14159265358979323846 * (X[3 * i + d] + 0.5 * L) / L);
    const double amp = A * omega;
    double *o = shape + 6 * i;
    o[0] = amp * S[1] * S[2]; o[1] = amp * S[0] * S[2]; o[2] = amp * S[0] * S[1];
    o[3] = 0.0; o[4] = 0.0; o[5] = 0.0;
  }
}

static unsigned vertex_blocks(int64_t nv) {
  int64_t blocks = (nv + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

int launch_shape3(const double *X, double *shape, int64_t nv, const Wave3 &m, void *stream) {
  shape3_kernel<<<vertex_blocks(nv), 256, 0, (cudaStream_t)stream>>>(X, shape, nv, m);
  return (int)cudaGetLastError();
}

int launch_shape3_tgv(const double *X, double *shape, int64_t nv, double A, double omega, double L, void *stream) {
  shape3_tgv_kernel<<<vertex_blocks(nv), 256, 0, (cudaStream_t)stream>>>(X, shape, nv, A, omega, L);
  return (int)cudaGetLastError();
}

// ---- diagnostics: integrals of the nodal interpolants over the moving tetrahedra ----------
// int f = J sum_i wq_i f_i per element (wq = 1^T Mhat, J = det G, G = dx/d(r,s,t)), for
// f = rho, rho |u|^2 / 2 = c^2 (q2^2 + q3^2 + q4^2) / (2 q1), rho u, rho v, rho w and 1.
// One thread per element (grid-stride), block partials in a fixed order, one block sums
// them: the result does not depend on scheduling.
constexpr int kDiag3Threads = 256;

__device__ __forceinline__ void block_sum6(double (&acc)[6], double *part) {
  __shared__ double red[kDiag3Threads / 32][6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    part[threadIdx.x] = v;
  }
}

// ctl (recording mode, else NULL): ctl[0] steps since recording began, ctl[1] records
// written; only every `every`-th step is integrated (uniform over the grid).
template <typename T>
__global__ void __launch_bounds__(kDiag3Threads) diagnostics3_kernel(const T *q, bool pert, int Np, const MeshRec3 *mesh,
                                                                    const double *xn, double px, double py, double pz,
                                                                    const double *wq, double c, int64_t K, double *part,
                                                                    const int64_t *ctl, int every) {
  if (ctl != nullptr && (ctl[0] + 1) % every != 0) return;
  const double per[3] = {px, py, pz};
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < K; e += (int64_t)gridDim.x * blockDim.x) {
    const MeshRec3 rec = mesh[e];
    double P[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int d = 0; d < 3; ++d) P[k][d] = xn[3 * (int64_t)rec.v[k] + d] + rec.shift[3 * k + d] * per[d];
    double G[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int j = 0; j < 3; ++j) G[d][j] = 0.5 * (P[j + 1][d] - P[0][d]);
    const double J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                     G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const T *qe = q + e * 10 * Np;
    double m = 0.0, ke = 0.0, mu = 0.0, mv = 0.0, mw = 0.0, w = 0.0;
    for (int n = 0; n < Np; ++n) {
      const double q1 = (double)qe[n] + (pert ? 1.0 : 0.0);
      const double q2 = (double)qe[Np + n], q3 = (double)qe[2 * Np + n], q4 = (double)qe[3 * Np + n];
      const double wn = wq[n];
      m += wn * q1;
      ke += wn * 0.5 * c * c * (q2 * q2 + q3 * q3 + q4 * q4) / q1;
      mu += wn * c * q2;
      mv += wn * c * q3;
      mw += wn * c * q4;
      w += wn;
    }
    acc[0] += J * m; acc[1] += J * ke; acc[2] += J * mu; acc[3] += J * mv; acc[4] += J * mw; acc[5] += J * w;
  }
  block_sum6(acc, part + 6 * blockIdx.x);
}

// out = (int rho, int rho |u|^2 / 2, int rho u, int rho v, int rho w, |Omega|)
__global__ void __launch_bounds__(kDiag3Threads) diagnostics3_reduce_kernel(const double *part, int nblocks, double *out) {
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += part[6 * b + k];
  block_sum6(acc, out);
}

// recording mode: one record (t, mass, E_K, int rho u, int rho v, |Omega|) into slot
// ctl[1] mod cap of the ring, then the counters advance
__global__ void __launch_bounds__(kDiag3Threads) diagnostics3_record_kernel(const double *part, int nblocks,
                                                                           const double *clock, int64_t *ctl, int every,
                                                                           double *hist, int64_t cap) {
  const bool skip = (ctl[0] + 1) % every != 0;
  __shared__ double tot[6];
  if (!skip) {
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] += part[6 * b + k];
    block_sum6(acc, tot);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!skip) {
      double *r = hist + 6 * (ctl[1] % cap);
      r[0] = clock[0];
      r[1] = tot[0];
      r[2] = tot[1] / tot[5];
      r[3] = tot[2];
      r[4] = tot[3];
      r[5] = tot[5];
      ctl[1] += 1;
    }
    ctl[0] += 1;
  }
}

int diagnostics3_blocks(int64_t K) {
  int64_t blocks = (K + kDiag3Threads - 1) / kDiag3Threads;
  if (blocks > kDiag3MaxBlocks) blocks = kDiag3MaxBlocks;
  return blocks < 1 ? 1 : (int)blocks;
}

static void diag3_partials(const Diag3Args &d, const int64_t *ctl, int every, cudaStream_t st) {
  const unsigned blocks = (unsigned)diagnostics3_blocks(d.K);
  if (d.is_float)
    diagnostics3_kernel<float><<<blocks, kDiag3Threads, 0, st>>>((const float *)d.q, true, d.Np, d.mesh, d.xn,
                                                                   d.period[0], d.period[1], d.period[2], d.wq, d.c, d.K,
                                                                   d.part, ctl, every);
  else
    diagnostics3_kernel<double><<<blocks, kDiag3Threads, 0, st>>>((const double *)d.q, false, d.Np, d.mesh, d.xn,
                                                                    d.period[0], d.period[1], d.period[2], d.wq, d.c,
                                                                    d.K, d.part, ctl, every);
}

int launch_diagnostics3(const Diag3Args &d, double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  diag3_partials(d, nullptr, 1, st);
  diagnostics3_reduce_kernel<<<1, kDiag3Threads, 0, st>>>(d.part, diagnostics3_blocks(d.K), out);
  return (int)cudaGetLastError();
}

int launch_diagnostics3_record(const Diag3Args &d, const double *clock, int64_t *ctl, int every, double *hist,
                               int64_t cap, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  diag3_partials(d, ctl, every, st);
  diagnostics3_record_kernel<<<1, kDiag3Threads, 0, st>>>(d.part, diagnostics3_blocks(d.K), clock, ctl, every, hist,
                                                          cap);
  return (int)cudaGetLastError();
}

// physical node coordinates: x = sum_v l_v(node) (X_v + shift_v)
__global__ void nodes3_kernel(const double *bary, int Np, const double *xn, const MeshRec3 *mesh, double px, double py,
                              double pz, int64_t K, double *out) {
  const double per[3] = {px, py, pz};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * Np; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / Np;
    const int n = (int)(i - e * Np);
    const MeshRec3 rec = mesh[e];
    double x[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
      for (int d = 0; d < 3; ++d) x[d] += bary[4 * n + k] * (xn[3 * (int64_t)rec.v[k] + d] + rec.shift[3 * k + d] * per[d]);
    for (int d = 0; d < 3; ++d) out[3 * i + d] = x[d];
  }
}

int launch_nodes3(const double *bary, int Np, const double *xn, const MeshRec3 *mesh, const double period[3], int64_t K,
                  double *out, void *stream) {
  nodes3_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(bary, Np, xn, mesh, period[0], period[1], period[2], K, out);
  return (int)cudaGetLastError();
}

// canonical FP64 <-> FP32 perturbation (field 1 minus the rest density 1)
__global__ void cast3_kernel(double *d, float *f, int64_t K, int Np, bool to_float) {
  const int NQ = 10 * Np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * NQ; i += (int64_t)gridDim.x * blockDim.x) {
    const int fn = (int)(i % NQ);
    const double rest = fn < Np ? 1.0 : 0.0;
    if (to_float) f[i] = (float)(d[i] - rest);
    else d[i] = (double)f[i] + rest;
  }
}

int launch_cast3(double *d, float *f, int64_t K, int Np, bool to_float, void *stream) {
  cast3_kernel<<<2048, 256, 0, (cudaStream_t)stream>>>(d, f, K, Np, to_float);
  return (int)cudaGetLastError();
}

// ---- operator block ----
template <typename T, int N>
static void fill3(const RefOps3 &R, std::vector<T> &h) {
  typedef Dim3<N> D;
  typedef Op3<T, N> L;
  const int Np = D::Np, NFN = D::NFN, Nc = D::Nc;
  h.assign(L::Size, (T)0);
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) {
      h[L::DrT + m * Np + n] = (T)R.Dr[n * Np + m];
      h[L::DsT + m * Np + n] = (T)R.Ds[n * Np + m];
      h[L::DtT + m * Np + n] = (T)R.Dt[n * Np + m];
    }
  for (int n = 0; n < Np; ++n)
    for (int j = 0; j < NFN; ++j) h[L::LiftT + j * Np + n] = (T)R.LIFT[n * NFN + j];
  for (int n = 0; n < Np; ++n)
    for (int v = 0; v < 4; ++v) h[L::Bary + 4 * n + v] = (T)R.bary[n * 4 + v];
  for (int q = 0; q < Nc; ++q)
    for (int m = 0; m < Np; ++m) h[L::IT + (L::IP_SMEM ? q * Np + m : m * Nc + q)] = (T)R.I[q * Np + m];
  for (int n = 0; n < Np; ++n)
    for (int q = 0; q < Nc; ++q) h[L::PT + q * Np + n] = (T)R.P[n * Nc + q];
}

template <typename T>
static int upload_vec(const std::vector<T> &h, void **dev, void *stream) {
  cudaError_t err = cudaMalloc(dev, h.size() * sizeof(T));
  if (err != cudaSuccess) return (int)err;
  err = cudaMemcpyAsync(*dev, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    cudaFree(*dev);
    *dev = nullptr;
  }
  return (int)err;
}

int upload_ops3(int N, bool fp64, const RefOps3 &R, void **dev_ops, int **dev_tab, double **dev_bary, size_t *bytes,
                void *stream) {
  size_t total = 0;
  int rc = 0;
  if (fp64) {
    std::vector<double> h;
    switch (N) {
      case 1: fill3<double, 1>(R, h); break;
      case 2: fill3<double, 2>(R, h); break;
      case 3: fill3<double, 3>(R, h); break;
      case 4: fill3<double, 4>(R, h); break;
      default: return (int)cudaErrorInvalidValue;
    }
    rc = upload_vec(h, dev_ops, stream);
    total += h.size() * sizeof(double);
  } else {
    std::vector<float> h;
    switch (N) {
      case 1: fill3<float, 1>(R, h); break;
      case 2: fill3<float, 2>(R, h); break;
      case 3: fill3<float, 3>(R, h); break;
      case 4: fill3<float, 4>(R, h); break;
      default: return (int)cudaErrorInvalidValue;
    }
    rc = upload_vec(h, dev_ops, stream);
    total += h.size() * sizeof(float);
  }
  if (rc) return rc;
  std::vector<int> tab(R.nbr_node);
  tab.insert(tab.end(), R.fmask.begin(), R.fmask.end());
  rc = upload_vec(tab, (void **)dev_tab, stream);
  if (rc) return rc;
  total += tab.size() * sizeof(int);
  rc = upload_vec(R.bary, (void **)dev_bary, stream);
  total += R.bary.size() * sizeof(double);
  *bytes = total;
  return rc;
}

}  // namespace gb
