// Perfectly matched layer of the 2D solver (the airfoil case's outer boundary).
//
// Reading (the paper names a PML with auxiliary fields but prints no equations): complex
// stretching of one direction e (radial for the O-grid's outer ring), planar approximation,
// frequency shift alpha.  With L = R_e + R_t the advective operator split into its part
// along e and the rest, and Phi the auxiliary fields of the layer's elements,
//     dq/dt   = L(q) + Ntilde(q) - sigma Phi
//     dPhi/dt = R_e(q) - (alpha + sigma) Phi,
// R_e = (A_e + v_e) d_e q in the volume (A_e = -c Atilde_e, d_e = e . grad) plus the LIFT of
// the face terms 1/2 (n.e)(A_e + v_e) dq + (n.e)^2 1/2 (c |Atilde_n| + |v_n|) dq
// (the central part of the upwind flux along e exactly, its dissipation shared by (n.e)^2).
//
// The stage kernels are unchanged: after stage i, one launch over the layer's elements
// forms R_e(q_i) and Phi_i's contribution, which the SARK combinations take linearly:
//     dF_i = -sigma Phi_i,  q_{i+1} += dt cq dF_i,  (F_0 or the accumulator) += cs dF_i,
// with (cq, cs) the coefficients of F_i in stage i's combination for the field's class, and
// advances Phi by the RK4 stages (Phi_{i+1} = Phi_n + dt a_{i+1,i} G_i, G_i = R_e - (alpha +
// sigma) Phi_i; Phi_{n+1} = Phi_n + dt sum_j b_j G_j).  Phi_i is read before it is replaced,
// by the same thread.
#include <cuda_runtime.h>

#include <cstdint>

#include "gb_internal.h"

namespace gb {

namespace {

template <int N>
struct PmlDim {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int NFN = 3 * (N + 1);
  static constexpr int E = 8;   // elements per CTA
  // operator block (T): Dr^T [m][n], Ds^T [m][n], LIFT^T [j][n], barycentric coordinates [n][3]
  static constexpr int DrT = 0, DsT = Np * Np, LiftT = 2 * Np * Np, Bary = LiftT + NFN * Np;
  static constexpr int OpSize = Bary + 3 * Np;
};

__host__ __device__ constexpr int pml_row_start(int N, int j) { return j * (N + 1) - j * (j - 1) / 2; }

// volume node of face node k on face f (counter-clockwise along the face)
template <int N>
__device__ __forceinline__ int pml_fmask(int f, int k) {
  return f == 0 ? k : (f == 1 ? pml_row_start(N, k) + (N - k) : pml_row_start(N, N - k));
}

// y = Atilde_n w for the 2D moment system (Atilde_x, Atilde_y of Sec. 2)
template <typename T>
__device__ __forceinline__ void pml_apply_An(T nx, T ny, const T (&w)[6], T (&y)[6]) {
  const T s2 = (T)1.4142135623730950488;
  y[0] = nx * w[1] + ny * w[2];
  y[1] = nx * (w[0] + s2 * w[4]) + ny * w[3];
  y[2] = nx * w[3] + ny * (w[0] + s2 * w[5]);
  y[3] = nx * w[2] + ny * w[1];
  y[4] = s2 * nx * w[1];
  y[5] = s2 * ny * w[2];
}

template <typename T, int N, int STAGE>
__global__ void __launch_bounds__(((PmlDim<N>::E * PmlDim<N>::Np + 31) / 32) * 32)
pml_stage_kernel(const StageArgs a, const PmlArgs p) {
  typedef PmlDim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN, E = D::E;
  constexpr bool PERTURB = sizeof(T) == 4;
  __shared__ T sops[D::OpSize];
  __shared__ T sq[E][6 * Np];
  __shared__ T strc[E][6 * NFN];   // neighbour traces q+, then the face terms along e
  __shared__ T sgeo[E][20];        // rx sx ry sy, vertex velocities (6), per face nx ny Fscale (9), J
  __shared__ MeshRec srec[E];
  __shared__ int32_t selem[E];
  __shared__ double s_motion[2];

  const int tid = threadIdx.x, nthr = blockDim.x;
  const T *gops = reinterpret_cast<const T *>(p.ops);
  for (int i = tid; i < D::OpSize; i += nthr) sops[i] = gops[i];
  if (tid == nthr - 1) {
    // the stage's motion factors, as the stage kernels form them: v_i = gfac S(X),
    // x_i = x_n + xfac S(X) (RK4 nodes and a_{i,i-1})
    double gfac = 0.0, xfac = 0.0;
    if (a.motion_A != 0.0) {
      const double w = a.motion_w, Aw = a.motion_A * a.motion_w, t = a.clock[0], dt = a.dt;
      const double cst[4] = {0.0, 0.5, 0.5, 1.0};
      // the phases in FP64; their cosines in T (these factors scale FP32 terms in GB_MIXED)
      const double p0 = w * (t + cst[STAGE] * dt), p1 = STAGE > 0 ? w * (t + cst[STAGE - 1] * dt) : 0.0;
      gfac = Aw * (double)cos((T)p0);
      if (STAGE > 0) xfac = dt * cst[STAGE == 3 ? 3 : 1] * Aw * (double)cos((T)p1);
    }
    s_motion[0] = gfac;
    s_motion[1] = xfac;
  }
  const T *qin = reinterpret_cast<const T *>(a.qin);
  const T c = (T)a.c, half = (T)0.5;
  const T al = (T)((9.0 - 1.7320508075688772935) / 6.0), be = (T)((1.7320508075688772935 - 3.0) / 6.0);
  const int e_loc = tid / Np, n_loc = tid - Np * (tid / Np);
  T *phin = reinterpret_cast<T *>(p.phin), *phis = reinterpret_cast<T *>(p.phis);
  T *phia = reinterpret_cast<T *>(p.phiacc);
  T *qo = reinterpret_cast<T *>(a.qout);
  T *sto = reinterpret_cast<T *>(STAGE == 0 ? a.F0 : a.acc);

  for (int64_t l0 = (int64_t)blockIdx.x * E; l0 < p.n_layer; l0 += (int64_t)gridDim.x * E) {
    const int nel = (int)((p.n_layer - l0) < E ? (p.n_layer - l0) : E);
    // phase 0: this tile's element indices; every node's own layer data straight into
    // registers (independent of everything else, so their latency overlaps the rest)
    if (tid < nel) selem[tid] = p.elem[l0 + tid];
    const bool node = e_loc < nel;
    T ph[6], pn[6], pa[6], sig = 0, ex = 0, ey = 0;   // Phi_i, Phi_n, the RK4 sum
    if (node) {
      const T *pe = reinterpret_cast<const T *>(p.node) + ((l0 + e_loc) * 3) * Np;
      sig = pe[n_loc]; ex = pe[Np + n_loc]; ey = pe[2 * Np + n_loc];
      const int64_t base = (l0 + e_loc) * 6 * Np + n_loc;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        ph[f] = STAGE == 0 ? phin[base + f * Np] : phis[base + f * Np];
        pn[f] = STAGE == 0 ? ph[f] : phin[base + f * Np];
        pa[f] = STAGE == 0 ? (T)0 : phia[base + f * Np];
      }
    }
    __syncthreads();
    // phase 1: own fields and mesh records; the node's q_{i+1} and stored F values
    T qv[6], sv[6];
    const int64_t qbase = node ? (int64_t)selem[e_loc] * p.stride + n_loc : 0;
    if (node) {
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        qv[f] = qo[qbase + f * Np];
        sv[f] = STAGE < 3 ? sto[qbase + f * Np] : (T)0;
      }
    }
    for (int i = tid; i < nel * 6 * Np; i += nthr) {
      const int el = i / (6 * Np), j = i - 6 * Np * (i / (6 * Np));
      sq[el][j] = qin[(int64_t)selem[el] * p.stride + j];
    }
    if (tid < nel) srec[tid] = a.mesh[selem[tid]];
    __syncthreads();
    // phase 2: neighbour traces (all face nodes) and, for one thread per element, the
    // stage geometry (FP64 vertex positions, T afterwards)
    for (int item = tid; item < nel * NFN; item += nthr) {
      const int el = item / NFN, j = item - NFN * (item / NFN);
      const int f = j / Nfp, k = j - Nfp * (j / Nfp);
      const int nb = srec[el].nbr[f];
      if (nb >= 0) {
        const T *qp = qin + (int64_t)(nb >> 2) * p.stride + pml_fmask<N>(nb & 3, Nfp - 1 - k);
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) strc[el][fld * NFN + j] = qp[fld * Np];
      }
    }
    const double gfac = s_motion[0], xfac = s_motion[1];
    for (int el = tid; el < nel; el += nthr) {
      const MeshRec &rec = srec[el];
      // vertex positions and their differences in FP64, the stage increments xfac S in T
      double bx[3], by[3];
      T vx[3], vy[3], ix[3], iy[3];
      const T xft = (T)xfac, gft = (T)gfac;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 xv = reinterpret_cast<const double2 *>(a.xn)[rec.v[k]];
        const double2 sv = reinterpret_cast<const double2 *>(a.shape)[rec.v[k]];
        bx[k] = xv.x + rec.shift[2 * k] * a.period[0];
        by[k] = xv.y + rec.shift[2 * k + 1] * a.period[1];
        const T sx = (T)sv.x, sy = (T)sv.y;
        ix[k] = xft * sx; iy[k] = xft * sy;
        vx[k] = gft * sx; vy[k] = gft * sy;
      }
      T ex[3], ey[3];   // edge f from vertex f to f + 1
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const int f1 = (f + 1) % 3;
        ex[f] = (T)(bx[f1] - bx[f]) + (ix[f1] - ix[f]);
        ey[f] = (T)(by[f1] - by[f]) + (iy[f1] - iy[f]);
      }
      const T xr = (T)0.5 * ex[0], yr = (T)0.5 * ey[0];
      const T xs = (T)-0.5 * ex[2], ys = (T)-0.5 * ey[2];
      const T J = xr * ys - xs * yr, iJ = (T)1 / J;
      T *g = sgeo[el];
      g[0] = ys * iJ; g[1] = -yr * iJ; g[2] = -xs * iJ; g[3] = xr * iJ;
#pragma unroll
      for (int k = 0; k < 3; ++k) { g[4 + 2 * k] = vx[k]; g[5 + 2 * k] = vy[k]; }
      // face f runs from vertex f to f + 1; outward normal of a counter-clockwise triangle
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const T dx = ex[f], dy = ey[f];
        const T len = sqrt(dx * dx + dy * dy);
        g[10 + 3 * f] = dy / len;
        g[11 + 3 * f] = -dx / len;
        g[12 + 3 * f] = (T)0.5 * len * iJ;   // sJ / J with sJ = len / 2
      }
      g[19] = J;
    }
    __syncthreads();
    // phase 3: face terms along e at every face node, over the traces in place
    for (int item = tid; item < nel * NFN; item += nthr) {
      const int el = item / NFN, j = item - NFN * (item / NFN);
      const int f = j / Nfp, k = j - Nfp * (j / Nfp);
      const int vol = pml_fmask<N>(f, k);
      const int nb = srec[el].nbr[f];
      const T *qm = sq[el] + vol;
      const T *g = sgeo[el];
      const T *bl = sops + D::Bary + 3 * vol;
      const T vgx = bl[0] * g[4] + bl[1] * g[6] + bl[2] * g[8];
      const T vgy = bl[0] * g[5] + bl[1] * g[7] + bl[2] * g[9];
      T w[6];
      if (nb < 0) {
        T qe[6];
        if (nb == -1) {
          const T wx = vgx / c, wy = vgy / c;
          const T q1 = qm[0] + (PERTURB ? (T)1 : (T)0), q2 = qm[Np], q3 = qm[2 * Np];
          const T s2 = (T)2.8284271247461900976;   // the bounce-back wall ghost state
          qe[0] = qm[0];
          qe[1] = (T)2 * wx * q1 - q2;
          qe[2] = (T)2 * wy * q1 - q3;
          qe[3] = qm[3 * Np] + (T)4 * wx * wy * q1 - (T)2 * wx * q3 - (T)2 * wy * q2;
          qe[4] = qm[4 * Np] + s2 * (wx * wx * q1 - wx * q2);
          qe[5] = qm[5 * Np] + s2 * (wy * wy * q1 - wy * q3);
        } else {
#pragma unroll
          for (int fld = 0; fld < 6; ++fld) qe[fld] = (T)a.far[fld];
        }
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) w[fld] = qe[fld] - qm[fld * Np];
      } else {
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) w[fld] = strc[el][fld * NFN + j] - qm[fld * Np];
      }
      const T nx = g[10 + 3 * f], ny = g[11 + 3 * f], fs = g[12 + 3 * f];
      const T *pe = reinterpret_cast<const T *>(p.node) + ((l0 + el) * 3) * Np;
      const T fex = pe[Np + vol], fey = pe[2 * Np + vol];
      const T ne = nx * fex + ny * fey, vn = vgx * nx + vgy * ny, ve = vgx * fex + vgy * fey;
      T y1[6], y2[6], y3[6], y4[6], ye[6];
      pml_apply_An<T>(nx, ny, w, y1);
      pml_apply_An<T>(nx, ny, y1, y2);
      pml_apply_An<T>(nx, ny, y2, y3);
      pml_apply_An<T>(nx, ny, y3, y4);
      pml_apply_An<T>(fex, fey, w, ye);
      const T avn = vn < (T)0 ? -vn : vn;
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) {
        const T cen = half * ne * (ve * w[fld] - c * ye[fld]);
        const T dis = half * (c * (al * y2[fld] + be * y4[fld]) + avn * w[fld]);
        strc[el][fld * NFN + j] = fs * (cen + ne * ne * dis);
      }
    }
    __syncthreads();
    // phase 4: volume terms along e, LIFT of the face terms, the layer's updates (one thread per node)
    if (node) {
      const T *q = sq[e_loc];
      T qr[6], qs[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) { qr[f] = 0; qs[f] = 0; }
      for (int m = 0; m < Np; ++m) {
        const T dr = sops[D::DrT + m * Np + n_loc], ds = sops[D::DsT + m * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          qr[f] += dr * q[f * Np + m];
          qs[f] += ds * q[f * Np + m];
        }
      }
      const T *g = sgeo[e_loc];
      const T *bl = sops + D::Bary + 3 * n_loc;
      const T vgx = bl[0] * g[4] + bl[1] * g[6] + bl[2] * g[8];
      const T vgy = bl[0] * g[5] + bl[1] * g[7] + bl[2] * g[9];
      const T ve = vgx * ex + vgy * ey;
      T de[6], ye[6], R[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const T qx = g[0] * qr[f] + g[1] * qs[f], qy = g[2] * qr[f] + g[3] * qs[f];
        de[f] = ex * qx + ey * qy;
      }
      pml_apply_An<T>(ex, ey, de, ye);
#pragma unroll
      for (int f = 0; f < 6; ++f) R[f] = ve * de[f] - c * ye[f];
      for (int m = 0; m < NFN; ++m) {
        const T lm = sops[D::LiftT + m * Np + n_loc];
#pragma unroll
        for (int f = 0; f < 6; ++f) R[f] += lm * strc[e_loc][f * NFN + m];
      }
      // dF = -sigma Phi_i into the stage combinations; Phi by RK4
      const int64_t base = (l0 + e_loc) * 6 * Np + n_loc;
      const T dt = (T)a.dt, decay = (T)p.alpha + sig;
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        const int cl = f < 3 ? 0 : 1;
        const T dF = -sig * ph[f];
        const T G = R[f] - decay * ph[f];
        const int64_t iq = qbase + f * Np, i = base + f * Np;
        qo[iq] = qv[f] + dt * (T)p.cq[cl] * dF;
        if (STAGE < 3) sto[iq] = sv[f] + (T)p.cs[cl] * dF;
        if (STAGE == 0) {
          phis[i] = pn[f] + dt * (T)0.5 * G;
          phia[i] = G / (T)6;
        } else if (STAGE == 1) {
          phis[i] = pn[f] + dt * (T)0.5 * G;
          phia[i] = pa[f] + G / (T)3;
        } else if (STAGE == 2) {
          phis[i] = pn[f] + dt * G;
          phia[i] = pa[f] + G / (T)3;
        } else {
          phin[i] = pn[f] + dt * (pa[f] + G / (T)6);
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int N, int STAGE>
int pml_launch_one(const StageArgs &a, const PmlArgs &p, cudaStream_t st, int num_sms) {
  typedef PmlDim<N> D;
  const int threads = ((D::E * D::Np + 31) / 32) * 32;
  int64_t blocks = (p.n_layer + D::E - 1) / D::E;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  pml_stage_kernel<T, N, STAGE><<<(unsigned)blocks, threads, 0, st>>>(a, p);
  return (int)cudaGetLastError();
}

template <typename T, int N>
int pml_launch_n(const StageArgs &a, const PmlArgs &p, cudaStream_t st, int num_sms) {
  switch (a.stage) {
    case 0: return pml_launch_one<T, N, 0>(a, p, st, num_sms);
    case 1: return pml_launch_one<T, N, 1>(a, p, st, num_sms);
    case 2: return pml_launch_one<T, N, 2>(a, p, st, num_sms);
    case 3: return pml_launch_one<T, N, 3>(a, p, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

template <typename T>
int pml_launch_t(int N, const StageArgs &a, const PmlArgs &p, cudaStream_t st, int num_sms) {
  switch (N) {
    case 1: return pml_launch_n<T, 1>(a, p, st, num_sms);
    case 2: return pml_launch_n<T, 2>(a, p, st, num_sms);
    case 3: return pml_launch_n<T, 3>(a, p, st, num_sms);
    case 4: return pml_launch_n<T, 4>(a, p, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace

int launch_pml_stage(int N, bool fp64, const StageArgs &a, const PmlArgs &p, void *stream, int num_sms) {
  if (p.n_layer <= 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  return fp64 ? pml_launch_t<double>(N, a, p, st, num_sms) : pml_launch_t<float>(N, a, p, st, num_sms);
}

int pml_ops_size(int N) {
  switch (N) {
    case 1: return PmlDim<1>::OpSize;
    case 2: return PmlDim<2>::OpSize;
    case 3: return PmlDim<3>::OpSize;
    case 4: return PmlDim<4>::OpSize;
  }
  return 0;
}

}  // namespace gb
