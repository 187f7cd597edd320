// CUDA kernels of the ALE-DG Galerkin-Boltzmann solver (sm_103a).
//
// One fused kernel per SARK stage (Sec. 4) covers the whole right-hand side
// of Secs. 2-5 for a tile of E elements per CTA:
//   geometry  : stage vertex positions x_i = x_n + xfac S(X) and velocities
//               v_i = gfac S(X) (Sec. 5), geometric factors, normals and
//               Fscale from the three vertices in FP64 (GCL, Sec. 5);
//   volume    : Dr, Ds of the 6 fields, chain rule, (A + v_G) . grad q;
//   surface   : neighbour traces, the upwind fluxes of Sec. 3 (Atilde_n and
//               |Atilde_n| = alpha Atilde_n^2 + beta Atilde_n^4, the ALE flux
//               max(v_G.n, 0)), scaled by Fscale, lifted with LIFT;
//   cubature  : q1..q3 interpolated to the degree-3N rule, Ntilde there,
//               projected back onto fields 4..6 (Sec. 3);
//   update    : the SARK stage / final combination of Sec. 4.
// The kernel is persistent: the grid covers the SMs and each CTA loops over
// element tiles, with the reference operators staged once in shared memory.
// T is the field/arithmetic type; the library instantiates it for double
// (GB_FP64).  GB_MIXED uses the tensor-core kernel of gb_kernels_tc.cu.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "gb_internal.h"

namespace gb {

// ---------------------------------------------------------------------------
// compile-time sizes
// ---------------------------------------------------------------------------
template <int N>
struct Dim {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int NFN = 3 * (N + 1);
  static constexpr int qc = (3 * N + 2) / 2;
  static constexpr int Nc = qc * qc;
  static constexpr int NQ = 6 * Np;
};

// elements per CTA, per order and type
template <typename T, int N> struct Tile;
template <> struct Tile<double, 1> { static constexpr int E = 32; };
template <> struct Tile<double, 2> { static constexpr int E = 32; };
template <> struct Tile<double, 3> { static constexpr int E = 16; };
template <> struct Tile<double, 4> { static constexpr int E = 16; };
template <> struct Tile<double, 5> { static constexpr int E = 12; };
template <> struct Tile<double, 6> { static constexpr int E = 8; };

// layout of the operator block (in T), all stored so that consecutive
// threads read consecutive entries
template <int N>
struct OpLayout {
  typedef Dim<N> D;
  static constexpr int DrT = 0;                          // [m][n] = Dr[n][m]
  static constexpr int DsT = DrT + D::Np * D::Np;
  static constexpr int LiftT = DsT + D::Np * D::Np;      // [j][n] = LIFT[n][j]
  static constexpr int IT = LiftT + D::NFN * D::Np;      // [m][c] = I[c][m]
  static constexpr int PT = IT + D::Np * D::Nc;          // [c][n] = P[n][c]
  static constexpr int Bary = PT + D::Nc * D::Np;        // [n][3] barycentric coordinates of the nodes
  static constexpr int Size = Bary + 3 * D::Np;
};

__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__host__ __device__ constexpr int row_start(int N, int j) { return j * (N + 1) - j * (j - 1) / 2; }

// volume node of face node k on face f (counter-clockwise along the face)
template <int N>
__device__ __forceinline__ int fmask(int f, int k) {
  return f == 0 ? k : (f == 1 ? row_start(N, k) + (N - k) : row_start(N, N - k));
}

// per-element geometry block in shared memory (in T)
//   0..3  rx sx ry sy
//   4..9  vertex velocities vx0 vy0 vx1 vy1 vx2 vy2
//   10 + 20 f + (0..12): h|At_n| entries M00 M03 M04 M05 M33 M34 M35 M44 M45 M55 N11 N12 N22
//   10 + 20 f + 13..16 : h nx, h ny, h sqrt2 nx, h sqrt2 ny   (h = c Fscale / 2)
//   10 + 20 f + 17..19 : nx, ny, Fscale
//   70                  : J at x_{n+1} (stage 3 with fused diagnostics)
constexpr int GEO = 72;

__device__ __forceinline__ bool bad_double(double v) {
  return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool bad_value(double v) { return bad_double(v); }
__device__ __forceinline__ bool bad_value(float v) {
  return (__float_as_int(v) & 0x7f800000) == 0x7f800000;
}

// motion scalars of the stage, from the device clock
struct StageMotion { double gfac, xfac; };

__device__ __forceinline__ StageMotion stage_motion(const StageArgs &a) {
  StageMotion m{0.0, 0.0};
  if (a.motion_A == 0.0) return m;
  const double w = a.motion_w, Aw = a.motion_A * a.motion_w;
  if (a.stage < 0) {
    m.gfac = Aw * cos(w * a.rhs_time);
    return m;
  }
  const double t = a.clock[0], dt = a.dt;
  // RK4 nodes c = (0, 1/2, 1/2, 1); the stage position uses a_{i,i-1} = (1/2, 1/2, 1)
  const double cst[4] = {0.0, 0.5, 0.5, 1.0};
  const double aprev[4] = {0.0, 0.5, 0.5, 1.0};
  m.gfac = Aw * cos(w * (t + cst[a.stage] * dt));
  if (a.stage > 0) m.xfac = dt * aprev[a.stage] * Aw * cos(w * (t + cst[a.stage - 1] * dt));
  return m;
}

// ---------------------------------------------------------------------------
// the fused stage kernel
// ---------------------------------------------------------------------------
// Exterior state of a boundary face node (reading; the paper states neither condition):
// nb = -1 wall moving with the grid velocity (vgx, vgy) -- the particle velocities reflected
// about it, in moments the affine map below with (wx, wy) = v_G / c; nb = -2 far field --
// the free-stream equilibrium.  qm points at the node's field 1 value (stride Np); in the
// perturbation representation q1 is 1 + qm[0] and the map is applied to the full state.
template <typename T, int Np, bool PERTURB>
__device__ __forceinline__ void boundary_state(int nb, const T *qm, T vgx, T vgy, T inv_c, const double *far, T (&qe)[6]) {
  if (nb == -1) {
    const T wx = vgx * inv_c, wy = vgy * inv_c;
    const T q1 = qm[0] + (PERTURB ? (T)1 : (T)0), q2 = qm[Np], q3 = qm[2 * Np];
    const T s2 = (T)2.8284271247461900976;   // 2 sqrt2
    qe[0] = qm[0];
    qe[1] = (T)2 * wx * q1 - q2;
    qe[2] = (T)2 * wy * q1 - q3;
    qe[3] = qm[3 * Np] + (T)4 * wx * wy * q1 - (T)2 * wx * q3 - (T)2 * wy * q2;
    qe[4] = qm[4 * Np] + s2 * (wx * wx * q1 - wx * q2);
    qe[5] = qm[5 * Np] + s2 * (wy * wy * q1 - wy * q3);
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f) qe[f] = (T)far[f];
  }
}

template <typename T, int N, int STAGE, bool BC = false, bool REC = false>
__global__ void __launch_bounds__(((Tile<T, N>::E * Dim<N>::Np + 31) / 32) * 32)
stage_kernel(const StageArgs a) {
  typedef Dim<N> D;
  typedef OpLayout<N> L;
  constexpr int E = Tile<T, N>::E;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN, Nc = D::Nc, NQ = D::NQ;
  constexpr bool PERTURB = sizeof(T) == 4;
  const T SQ2 = (T)1.4142135623730950488;
  const T ISQ2 = (T)0.70710678118654752440;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sops = reinterpret_cast<T *>(smem_raw);
  T *sq = sops + L::Size;              // [E][6][Np]
  T *sflux = sq + E * NQ;              // [E][6][NFN]
  T *snt = sflux + E * 6 * NFN;        // [E][3][Nc]
  T *sgeo = snt + E * 3 * Nc;          // [E][GEO]
  __shared__ double s_motion[3];
  // REC: whether this step is recorded, read before any CTA can advance the counter
  const bool record = REC && ((a.rec_ctl[0] + 1) % a.rec_every == 0);
  const double t_now = a.clock[0];
  double dacc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};

  const int tid = threadIdx.x;
  const int nthr = blockDim.x;

  // operators: once per CTA
  const T *gops = reinterpret_cast<const T *>(a.ops);
  for (int i = tid; i < L::Size; i += nthr) sops[i] = gops[i];
  if (tid == 0) {
    StageMotion m = stage_motion(a);
    s_motion[0] = m.gfac;
    s_motion[1] = m.xfac;
    // factor of the final vertex update x_{n+1} = x_n + dt sum_j b_j v_j (RK4 b)
    double fin = 0.0;
    if (STAGE == 3 && a.motion_A != 0.0) {
      const double t = t_now, dt = a.dt, w = a.motion_w, Aw = a.motion_A * a.motion_w;
      fin = dt * Aw * (cos(w * t) / 6.0 + cos(w * (t + 0.5 * dt)) * (2.0 / 3.0) + cos(w * (t + dt)) / 6.0);
    }
    s_motion[2] = fin;
  }
  __syncthreads();
  if (STAGE == 3 && blockIdx.x == 0 && tid == 0) const_cast<double *>(a.clock)[1] = s_motion[2];
  const double gfac = s_motion[0], xfac = s_motion[1], fin = s_motion[2];

  const T *qin = reinterpret_cast<const T *>(a.qin);
  const int e_loc = tid / Np, n_loc = tid - (tid / Np) * Np;
  const bool node_thread = e_loc < E;

  const int64_t ntiles = (a.K + E - 1) / E;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t elem0 = tile * E;
    const int nel = (int)((a.K - elem0) < E ? (a.K - elem0) : E);

    // ---- load the tile's fields (contiguous) ----
    {
      const T *src = qin + elem0 * NQ;
      const int cnt = nel * NQ;
      for (int i = tid; i < cnt; i += nthr) sq[i] = src[i];
    }
    // ---- geometry: one thread per (element, face), FP64 ----
    for (int item = tid; item < 3 * E; item += nthr) {
      const int e = item / 3, f = item - 3 * (item / 3);
      if (e >= nel) continue;
      const MeshRec rec = a.mesh[elem0 + e];
      double px[3], py[3], sx_[3], sy_[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 xv = reinterpret_cast<const double2 *>(a.xn)[rec.v[k]];
        const double2 sv = reinterpret_cast<const double2 *>(a.shape)[rec.v[k]];
        sx_[k] = sv.x;
        sy_[k] = sv.y;
        px[k] = xv.x + rec.shift[2 * k] * a.period[0] + xfac * sv.x;
        py[k] = xv.y + rec.shift[2 * k + 1] * a.period[1] + xfac * sv.y;
      }
      const double xr = 0.5 * (px[1] - px[0]), xs = 0.5 * (px[2] - px[0]);
      const double yr = 0.5 * (py[1] - py[0]), ys = 0.5 * (py[2] - py[0]);
      const double J = xr * ys - xs * yr;
      if (!(J > 0.0)) atomicOr(a.status, GB_STATUS_MESH);
      const double iJ = 1.0 / J;
      T *g = sgeo + e * GEO;
      if (f == 0) {
        g[0] = (T)(ys * iJ);
        g[1] = (T)(-yr * iJ);
        g[2] = (T)(-xs * iJ);
        g[3] = (T)(xr * iJ);
        if (REC && record) {   // J at x_{n+1}, where the recorded integrals are taken
          double xn1[3], yn1[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            xn1[k] = px[k] + (fin - xfac) * sx_[k];
            yn1[k] = py[k] + (fin - xfac) * sy_[k];
          }
          g[70] = (T)(0.25 * ((xn1[1] - xn1[0]) * (yn1[2] - yn1[0]) - (xn1[2] - xn1[0]) * (yn1[1] - yn1[0])));
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g[4 + 2 * k] = (T)(gfac * sx_[k]);
          g[5 + 2 * k] = (T)(gfac * sy_[k]);
        }
      }
      const int f1 = f == 2 ? 0 : f + 1;
      const double dx = px[f1] - px[f], dy = py[f1] - py[f];
      const double len = sqrt(dx * dx + dy * dy);
      const double nx = dy / len, ny = -dx / len;
      const double fs = 0.5 * len * iJ;
      const double h = 0.5 * a.c * fs;
      // |At_n| = alpha At_n^2 + beta At_n^4 on the blocks {1,4,5,6} and {2,3}
      const double al = (9.0 - 1.7320508075688772935) / 6.0, be = (1.7320508075688772935 - 3.0) / 6.0;
      const double nn = nx * nx + ny * ny, s2 = 1.4142135623730950488;
      const double e00 = nn, e01 = 2.0 * nx * ny, e02 = s2 * nx * nx, e03 = s2 * ny * ny;
      const double e11 = nn, e12 = s2 * nx * ny, e13 = e12;
      const double e22 = 2.0 * nx * nx, e23 = 0.0, e33 = 2.0 * ny * ny;
      const double m[4][4] = {{e00, e01, e02, e03}, {e01, e11, e12, e13}, {e02, e12, e22, e23}, {e03, e13, e23, e33}};
      double m4[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) m4[i][j] = m[i][0] * m[0][j] + m[i][1] * m[1][j] + m[i][2] * m[2][j] + m[i][3] * m[3][j];
      const double o11 = 3.0 * nx * nx + ny * ny, o12 = 2.0 * nx * ny, o22 = nx * nx + 3.0 * ny * ny;
      const double p11 = o11 * o11 + o12 * o12, p12 = o11 * o12 + o12 * o22, p22 = o12 * o12 + o22 * o22;
      T *gf = g + 10 + 20 * f;
      const int ii[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
      const int jj[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
#pragma unroll
      for (int k = 0; k < 10; ++k) gf[k] = (T)(h * (al * m[ii[k]][jj[k]] + be * m4[ii[k]][jj[k]]));
      gf[10] = (T)(h * (al * o11 + be * p11));
      gf[11] = (T)(h * (al * o12 + be * p12));
      gf[12] = (T)(h * (al * o22 + be * p22));
      gf[13] = (T)(h * nx);
      gf[14] = (T)(h * ny);
      gf[15] = (T)(h * s2 * nx);
      gf[16] = (T)(h * s2 * ny);
      gf[17] = (T)nx;
      gf[18] = (T)ny;
      gf[19] = (T)fs;
    }
    __syncthreads();

    // ---- volume term ----
    T rhs[6];
    if (node_thread && e_loc < nel) {
      const T *q = sq + e_loc * NQ;
      T qr[6], qs[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) { qr[f] = 0; qs[f] = 0; }
#pragma unroll 5
      for (int m = 0; m < Np; ++m) {
        const T dr = sops[L::DrT + m * Np + n_loc], ds = sops[L::DsT + m * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const T v = q[f * Np + m];
          qr[f] = fmaT(dr, v, qr[f]);
          qs[f] = fmaT(ds, v, qs[f]);
        }
      }
      const T *g = sgeo + e_loc * GEO;
      const T rx = g[0], sx = g[1], ry = g[2], sy = g[3];
      const T l0 = sops[L::Bary + 3 * n_loc], l1 = sops[L::Bary + 3 * n_loc + 1], l2 = sops[L::Bary + 3 * n_loc + 2];
      const T vgx = l0 * g[4] + l1 * g[6] + l2 * g[8];
      const T vgy = l0 * g[5] + l1 * g[7] + l2 * g[9];
      T qx[6], qy[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        qx[f] = fmaT(rx, qr[f], sx * qs[f]);
        qy[f] = fmaT(ry, qr[f], sy * qs[f]);
      }
      const T c = (T)a.c;
      rhs[0] = -c * (qx[1] + qy[2]);
      rhs[1] = -c * (qx[0] + SQ2 * qx[4] + qy[3]);
      rhs[2] = -c * (qx[3] + qy[0] + SQ2 * qy[5]);
      rhs[3] = -c * (qx[2] + qy[1]);
      rhs[4] = -c * (SQ2 * qx[1]);
      rhs[5] = -c * (SQ2 * qy[2]);
#pragma unroll
      for (int f = 0; f < 6; ++f) rhs[f] = fmaT(vgx, qx[f], fmaT(vgy, qy[f], rhs[f]));
    }

    // ---- surface fluxes at the face nodes ----
    for (int item = tid; item < E * NFN; item += nthr) {
      const int e = item / NFN, j = item - NFN * (item / NFN);
      if (e >= nel) continue;
      const int f = j / Nfp, k = j - Nfp * (j / Nfp);
      const int vol = fmask<N>(f, k);
      const MeshRec &rec = a.mesh[elem0 + e];
      const int nb = rec.nbr[f];
      const T *qm = sq + e * NQ + vol;
      const T *g = sgeo + e * GEO;
      const T *gf = g + 10 + 20 * f;
      const T l0 = sops[L::Bary + 3 * vol], l1 = sops[L::Bary + 3 * vol + 1], l2 = sops[L::Bary + 3 * vol + 2];
      const T vgx = l0 * g[4] + l1 * g[6] + l2 * g[8];
      const T vgy = l0 * g[5] + l1 * g[7] + l2 * g[9];
      T w[6];
      if (BC && nb < 0) {
        T qe[6];
        boundary_state<T, Np, PERTURB>(nb, qm, vgx, vgy, (T)(1.0 / a.c), a.far, qe);
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) w[fld] = qe[fld] - qm[fld * Np];
      } else {
        const int64_t e2 = nb >> 2;
        const int f2 = nb & 3;
        const int vol2 = fmask<N>(f2, Nfp - 1 - k);
        const T *qp = qin + e2 * NQ + vol2;
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) w[fld] = qp[fld * Np] - qm[fld * Np];
      }
      const T vn = vgx * gf[17] + vgy * gf[18];
      const T ale = vn > (T)0 ? vn * gf[19] : (T)0;
      const T M00 = gf[0], M03 = gf[1], M04 = gf[2], M05 = gf[3], M33 = gf[4], M34 = gf[5], M35 = gf[6];
      const T M44 = gf[7], M45 = gf[8], M55 = gf[9], N11 = gf[10], N12 = gf[11], N22 = gf[12];
      const T hnx = gf[13], hny = gf[14], hsx = gf[15], hsy = gf[16];
      T o[6];
      o[0] = M00 * w[0] + M03 * w[3] + M04 * w[4] + M05 * w[5] - hnx * w[1] - hny * w[2];
      o[3] = M03 * w[0] + M33 * w[3] + M34 * w[4] + M35 * w[5] - hnx * w[2] - hny * w[1];
      o[4] = M04 * w[0] + M34 * w[3] + M44 * w[4] + M45 * w[5] - hsx * w[1];
      o[5] = M05 * w[0] + M35 * w[3] + M45 * w[4] + M55 * w[5] - hsy * w[2];
      o[1] = N11 * w[1] + N12 * w[2] - hnx * w[0] - hsx * w[4] - hny * w[3];
      o[2] = N12 * w[1] + N22 * w[2] - hny * w[0] - hsy * w[5] - hnx * w[3];
      T *fl = sflux + e * 6 * NFN + j;
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) fl[fld * NFN] = fmaT(ale, w[fld], o[fld]);
    }
    // ---- cubature: q1..q3 at the points, Ntilde there ----
    const T itau = (T)a.inv_tau;
    for (int item = tid; item < E * Nc; item += nthr) {
      const int e = item / Nc, cpt = item - Nc * (item / Nc);
      if (e >= nel) continue;
      const T *q = sq + e * NQ;
      T q1 = 0, q2 = 0, q3 = 0;
#pragma unroll 5
      for (int m = 0; m < Np; ++m) {
        const T im = sops[L::IT + m * Nc + cpt];
        q1 = fmaT(im, q[m], q1);
        q2 = fmaT(im, q[Np + m], q2);
        q3 = fmaT(im, q[2 * Np + m], q3);
      }
      if (PERTURB) q1 += (T)1;
      const T r1 = itau / q1;
      const T rs = r1 * ISQ2;
      T *nt = snt + e * 3 * Nc + cpt;
      nt[0] = q2 * q3 * r1;
      nt[Nc] = q2 * q2 * rs;
      nt[2 * Nc] = q3 * q3 * rs;
    }
    __syncthreads();

    // ---- lift, projection, SARK update ----
    if (node_thread && e_loc < nel) {
      const T *fl = sflux + e_loc * 6 * NFN;
#pragma unroll 3
      for (int j = 0; j < NFN; ++j) {
        const T lj = sops[L::LiftT + j * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 6; ++f) rhs[f] = fmaT(lj, fl[f * NFN + j], rhs[f]);
      }
      const T *nt = snt + e_loc * 3 * Nc;
#pragma unroll 7
      for (int cpt = 0; cpt < Nc; ++cpt) {
        const T pc = sops[L::PT + cpt * Np + n_loc];
        rhs[3] = fmaT(pc, nt[cpt], rhs[3]);
        rhs[4] = fmaT(pc, nt[Nc + cpt], rhs[4]);
        rhs[5] = fmaT(pc, nt[2 * Nc + cpt], rhs[5]);
      }
      const int64_t base = (elem0 + e_loc) * NQ + n_loc;
      const T dt = (T)a.dt;
      if (STAGE < 0) {
        T *F = reinterpret_cast<T *>(a.Fout);
#pragma unroll
        for (int f = 0; f < 6; ++f) F[base + f * Np] = rhs[f];
      } else {
        const T *qn = reinterpret_cast<const T *>(a.qn);
        T *qout = reinterpret_cast<T *>(a.qout);
        T *F0 = reinterpret_cast<T *>(a.F0);
        T *acc = reinterpret_cast<T *>(a.acc);
        bool bad = false;
        T qrec[3] = {0, 0, 0};
        // every load of the node's six fields is issued before any store (q_{n+1} overwrites
        // q_n in place at the last stage, so the compiler may not reorder them itself)
        T xv[6], x0[6], x1[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int64_t idx = base + f * Np;
          xv[f] = STAGE == 0 ? sq[e_loc * NQ + f * Np + n_loc] : qn[idx];
          x0[f] = (STAGE == 1 || STAGE == 2) ? F0[idx] : (T)0;
          x1[f] = STAGE >= 2 ? acc[idx] : (T)0;
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          const int cl = f < 3 ? 0 : 1;
          const int64_t idx = base + f * Np;
          const T r = rhs[f];
          if (STAGE == 0) {
            const T qv = xv[f];
            F0[idx] = r;
            qout[idx] = (T)a.co.E[cl][1] * qv + dt * ((T)a.co.A[cl][4] * r);
          } else if (STAGE == 1) {
            const T qv = xv[f], f0 = x0[f];
            qout[idx] = (T)a.co.E[cl][2] * qv + dt * ((T)a.co.A[cl][8] * f0 + (T)a.co.A[cl][9] * r);
            acc[idx] = (T)a.co.B[cl][0] * f0 + (T)a.co.B[cl][1] * r;
          } else if (STAGE == 2) {
            const T qv = xv[f], f0 = x0[f], ac = x1[f];
            qout[idx] = (T)a.co.E[cl][3] * qv + dt * ((T)a.co.A[cl][12] * f0 + (T)a.co.A[cl][14] * r);
            acc[idx] = ac + (T)a.co.B[cl][2] * r;
          } else {
            const T qv = xv[f], ac = x1[f];
            const T out = (T)a.co.E[cl][4] * qv + dt * (ac + (T)a.co.B[cl][3] * r);
            qout[idx] = out;
            bad |= bad_value(out);
            if (REC && f < 3) qrec[f] = out;
          }
        }
        if (STAGE == 3 && bad) atomicOr(a.status, GB_STATUS_NAN);
        if (REC && record) {   // fused diagnostics: this node's share of the integrals of q_{n+1} on x_{n+1}
          const double jw = (double)sgeo[e_loc * GEO + 70] * a.rec_wq[n_loc], cc = a.c;
          const double q1 = (double)qrec[0] + (PERTURB ? 1.0 : 0.0), q2 = (double)qrec[1], q3 = (double)qrec[2];
          dacc[0] += jw * q1;
          dacc[1] += jw * 0.5 * cc * cc * (q2 * q2 + q3 * q3) / q1;
          dacc[2] += jw * cc * q2;
          dacc[3] += jw * cc * q3;
          dacc[4] += jw;
        }
      }
    }
    __syncthreads();
  }
  if constexpr (REC) fused_record(a, record, dacc, t_now + a.dt);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T, int N>
static size_t stage_smem() {
  typedef Dim<N> D;
  constexpr int E = Tile<T, N>::E;
  return sizeof(T) * (size_t)(OpLayout<N>::Size + E * (D::NQ + 6 * D::NFN + 3 * D::Nc + GEO));
}

template <typename T, int N, int STAGE, bool BC, bool REC = false>
static int launch_one(const StageArgs &a, cudaStream_t st, int num_sms) {
  constexpr int E = Tile<T, N>::E;
  const int threads = ((E * Dim<N>::Np + 31) / 32) * 32;
  const size_t smem = stage_smem<T, N>();
  // the shared-memory opt-in and the occupancy are per-device facts, cached per device ordinal
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return (int)derr;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  static bool attr_set[64] = {};
  if (!attr_set[dev]) {
    cudaError_t err = cudaFuncSetAttribute(stage_kernel<T, N, STAGE, BC, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    attr_set[dev] = true;
  }
  static int per_sm_d[64] = {};
  int &per_sm = per_sm_d[dev];
  if (per_sm == 0) {
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel<T, N, STAGE, BC, REC>, threads, smem);
    if (err != cudaSuccess) return (int)err;
  }
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (a.K + E - 1) / E;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (REC && grid > kRecMaxCtas) grid = kRecMaxCtas;
  if (grid < 1) grid = 1;
  stage_kernel<T, N, STAGE, BC, REC><<<(unsigned)grid, threads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <typename T, int N, bool BC>
static int launch_stage_nb(const StageArgs &a, cudaStream_t st, int num_sms) {
  switch (a.stage) {
    case -1: return launch_one<T, N, -1, BC>(a, st, num_sms);
    case 0: return launch_one<T, N, 0, BC>(a, st, num_sms);
    case 1: return launch_one<T, N, 1, BC>(a, st, num_sms);
    case 2: return launch_one<T, N, 2, BC>(a, st, num_sms);
    case 3:
      return a.rec_every > 0 ? launch_one<T, N, 3, BC, true>(a, st, num_sms) : launch_one<T, N, 3, BC>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

// meshes with boundary faces use the BC variant (orders 1..4)
template <typename T, int N>
static int launch_stage_n(const StageArgs &a, cudaStream_t st, int num_sms) {
  if (a.bc) {
    if constexpr (N <= 4) return launch_stage_nb<T, N, true>(a, st, num_sms);
    return (int)cudaErrorInvalidValue;
  }
  return launch_stage_nb<T, N, false>(a, st, num_sms);
}

template <typename T>
static int launch_stage_t(int N, const StageArgs &a, void *stream, int num_sms) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (N) {
    case 1: return launch_stage_n<T, 1>(a, st, num_sms);
    case 2: return launch_stage_n<T, 2>(a, st, num_sms);
    case 3: return launch_stage_n<T, 3>(a, st, num_sms);
    case 4: return launch_stage_n<T, 4>(a, st, num_sms);
    case 5: return launch_stage_n<T, 5>(a, st, num_sms);
    case 6: return launch_stage_n<T, 6>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_stage_fp64(int N, const StageArgs &a, void *stream, int num_sms) {
  return launch_stage_t<double>(N, a, stream, num_sms);
}

// final vertex update of the step, x_{n+1} = x_n + fin S(X), and t_n += dt
__global__ void vertex_update_kernel(double *xn, const double *shape, double *clock, double dt, int64_t nv) {
  const double fin = clock[1];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    xn[2 * v] += fin * shape[2 * v];
    xn[2 * v + 1] += fin * shape[2 * v + 1];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) clock[0] += dt;
}

int launch_vertex_update(const StageArgs &a, int64_t n_vert, void *stream) {
  int64_t blocks = (n_vert + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  vertex_update_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      const_cast<double *>(a.xn), a.shape, const_cast<double *>(a.clock), a.dt, n_vert);
  return (int)cudaGetLastError();
}

// vertex velocity shape S(X) of the prescribed motion (Sec. 7.1 form)
__global__ void shape_kernel(const double *X, double *shape, int64_t nv, int kind, double Lx, double Ly) {
  const double two_pi = 6.283185307179586476925;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (kind == GB_MOTION_SINXY) s = sin(two_pi * X[2 * v] / Lx) * sin(two_pi * X[2 * v + 1] / Ly);
    shape[2 * v] = kind == GB_MOTION_PLUNGE ? 0.0 : s;
    shape[2 * v + 1] = kind == GB_MOTION_PLUNGE ? 1.0 : s;
  }
}

int launch_shape(const double *X, double *shape, int64_t n_vert, int kind, double Lx, double Ly, void *stream) {
  int64_t blocks = (n_vert + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  shape_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(X, shape, n_vert, kind, Lx, Ly);
  return (int)cudaGetLastError();
}

// physical node coordinates from the current vertices (P1 map)
template <int N>
__global__ void nodes_kernel(const double *bary, const double *xn, const MeshRec *mesh, double px, double py,
                             int64_t K, double *out) {
  constexpr int Np = Dim<N>::Np;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K * Np; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / Np;
    const int n = (int)(i - e * Np);
    const MeshRec rec = mesh[e];
    double x = 0.0, y = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double l = bary[3 * n + k];
      x += l * (xn[2 * rec.v[k]] + rec.shift[2 * k] * px);
      y += l * (xn[2 * rec.v[k] + 1] + rec.shift[2 * k + 1] * py);
    }
    out[2 * i] = x;
    out[2 * i + 1] = y;
  }
}

int launch_nodes(int N, const double *ops, const double *xn, const MeshRec *mesh, double px, double py, int64_t K,
                 double *out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = 1024, thr = 256;
  switch (N) {
#define GB_NODES_CASE(n) \
  case n: nodes_kernel<n><<<blocks, thr, 0, st>>>(ops + OpLayout<n>::Bary, xn, mesh, px, py, K, out); break;
    GB_NODES_CASE(1) GB_NODES_CASE(2) GB_NODES_CASE(3) GB_NODES_CASE(4) GB_NODES_CASE(5) GB_NODES_CASE(6)
#undef GB_NODES_CASE
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

// operator block (FP64) in the layout of OpLayout
template <int N>
static void fill_ops(const RefOps &R, std::vector<double> &h) {
  typedef Dim<N> D;
  typedef OpLayout<N> L;
  h.assign(L::Size, 0.0);
  for (int n = 0; n < D::Np; ++n)
    for (int m = 0; m < D::Np; ++m) {
      h[L::DrT + m * D::Np + n] = R.Dr[n * D::Np + m];
      h[L::DsT + m * D::Np + n] = R.Ds[n * D::Np + m];
    }
  for (int n = 0; n < D::Np; ++n)
    for (int j = 0; j < D::NFN; ++j) h[L::LiftT + j * D::Np + n] = R.LIFT[n * D::NFN + j];
  for (int c = 0; c < D::Nc; ++c)
    for (int m = 0; m < D::Np; ++m) {
      h[L::IT + m * D::Nc + c] = R.I[c * D::Np + m];
      h[L::PT + c * D::Np + m] = R.P[m * D::Nc + c];
    }
  for (int n = 0; n < D::Np; ++n) {
    h[L::Bary + 3 * n] = -0.5 * (R.r[n] + R.s[n]);
    h[L::Bary + 3 * n + 1] = 0.5 * (1.0 + R.r[n]);
    h[L::Bary + 3 * n + 2] = 0.5 * (1.0 + R.s[n]);
  }
}

int upload_ops(int N, const RefOps &R, double **dev_ops, void *stream) {
  std::vector<double> h;
  switch (N) {
    case 1: fill_ops<1>(R, h); break;
    case 2: fill_ops<2>(R, h); break;
    case 3: fill_ops<3>(R, h); break;
    case 4: fill_ops<4>(R, h); break;
    case 5: fill_ops<5>(R, h); break;
    case 6: fill_ops<6>(R, h); break;
    default: return (int)cudaErrorInvalidValue;
  }
  void *d = nullptr;
  cudaError_t err = cudaMalloc(&d, h.size() * sizeof(double));
  if (err != cudaSuccess) return (int)err;
  err = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    cudaFree(d);
    return (int)err;
  }
  *dev_ops = reinterpret_cast<double *>(d);
  return 0;
}

}  // namespace gb
