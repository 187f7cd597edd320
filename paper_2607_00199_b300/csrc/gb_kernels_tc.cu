// GB_MIXED stage kernel on the tensor cores.
//
// Same right-hand side and SARK combination as the FP64 stage kernel (Secs.
// 2-5), with the four dense contractions of the semi-discrete form (Dr/Ds on
// the 6 fields, LIFT on the face fluxes, the cubature interpolation I and the
// projection P) issued as mma.sync.m16n8k8 TF32 products with FP32
// accumulation.  Each operand is split into a TF32 head and a TF32 tail
// (x = hi + lo) and every product is formed as hi*hi + hi*lo + lo*hi, which
// keeps the contractions at FP32 accuracy (the dropped lo*lo term is ~2^-22
// relative).
//
// A warp owns a tile of 16 elements (the M dimension of every product):
//   rows = elements, columns = nodes / face nodes / cubature points.
// The reference operators are constant B operands, pre-split and stored in
// per-lane fragment order (one 16-byte load per fragment), read through the L1
// cache with the evict-last priority: a copy in every CTA's shared memory measured
// 3% slower (it cost 20 KB per CTA and a staging pass at every launch).
// The cubature chain reuses the accumulator fragment of I q directly as the A
// fragment of P Ntilde: the 8 columns of a chunk are taken in the order
// (0,2,4,6,1,3,5,7), which is folded into the P table.
//
// Data: fields are FP32 perturbations from the rest state (q1 = 1, others 0)
// in an element-major layout with a padded element stride S (S >= 6 Np,
// S = 4 mod 8: conflict-free fragment loads from the staged tile), elements
// numbered along a Morton curve.  Per tile: the own fields and all neighbour
// traces are staged in shared memory with cp.async, the geometry is formed
// while the copies are in flight (FP64 stage positions and edge differences,
// FP32 afterwards), and the SARK combination runs as a coalesced pass over
// the tile.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "gb_internal.h"

namespace gb {


template <int N>
struct TcDim {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int NFN = 3 * (N + 1);
  static constexpr int Nc = ((3 * N + 2) / 2) * ((3 * N + 2) / 2);
  static constexpr int KS = (Np + 7) / 8;       // k-steps over nodes
  static constexpr int KF = (NFN + 7) / 8;      // k-steps over face nodes
  static constexpr int NT = (Np + 7) / 8;       // n-tiles over output nodes
  static constexpr int CH = (Nc + 7) / 8;       // cubature chunks of 8 points
  static constexpr int S = tc_round_s(6 * Np);  // element stride of the field layout
  static constexpr int FJ = 8 * KF;             // face-node slots per field
  static constexpr int ST = tc_round_s(6 * FJ); // element stride of the trace / flux buffer
  static constexpr int OUTS = S > ST ? S : ST;  // row capacity of the trace buffer, reused for the rhs tile
  // B-fragment sets (32 lanes x float4 each)
  static constexpr int B_DR = 0;
  static constexpr int B_DS = B_DR + KS * NT;
  static constexpr int B_LIFT = B_DS + KS * NT;
  static constexpr int B_I = B_LIFT + KF * NT;
  static constexpr int B_P = B_I + CH * KS;
  static constexpr int NSETS = B_P + CH * NT;
  static constexpr int GEOS = 17;               // per element: rx sx ry sy iJ vx[3] vy[3] ex[3] ey[3]
  static constexpr int W = 4;                   // most warps per CTA (the launch picks 1, 2 or 4)
  static constexpr int WARP_FLOATS = 16 * S + 16 * OUTS + 16 * GEOS + 4;
};


__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// two splits with one packed subtraction
__device__ __forceinline__ void split_tf32x2(float2 x, unsigned &h0, unsigned &l0, unsigned &h1, unsigned &l1) {
  h0 = to_tf32(x.x);
  h1 = to_tf32(x.y);
  const float2 r = __fadd2_rn(x, make_float2(-__uint_as_float(h0), -__uint_as_float(h1)));
  l0 = to_tf32(r.x);
  l1 = to_tf32(r.y);
}

// not volatile: the compiler may interleave products into independent accumulators
__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += (ahi + alo)(bhi + blo), dropping alo * blo; b = (blo0, blo1, bhi0, bhi1)
__device__ __forceinline__ void mma3(float (&c)[4], const unsigned (&ahi)[4], const unsigned (&alo)[4], const float4 b) {
  mma_tf32(c, alo, __float_as_uint(b.z), __float_as_uint(b.w));
  mma_tf32(c, ahi, __float_as_uint(b.x), __float_as_uint(b.y));
  mma_tf32(c, ahi, __float_as_uint(b.z), __float_as_uint(b.w));
}

// operator tables: read-only and reused by every tile, so loaded with the L1 evict-last
// priority (measured 2% per step over plain read-only loads, which the streaming state
// reads evicted)
__device__ __forceinline__ float4 ldg_keep(const float4 *p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// packed FP32x2 arithmetic (two lanes of independent values per instruction)
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float a, float2 x, float2 y) { return __ffma2_rn(bc2(a), x, y); }
__device__ __forceinline__ float2 mul2(float a, float2 x) { return __fmul2_rn(bc2(a), x); }

__device__ __forceinline__ void tc_cp_async16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void tc_cp_async4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void tc_cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void tc_l2_prefetch(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A fragment of rows (element) x columns [col0, col0 + 8) from a row-major smem tile
// with row stride `stride`; columns >= ncol are zero.
template <int STRIDE>
__device__ __forceinline__ void load_a(const float *tile, int col0, int ncol, int g, int t, unsigned (&hi)[4], unsigned (&lo)[4]) {
  const int c0 = col0 + t, c1 = col0 + t + 4;
  const float x0 = c0 < ncol ? tile[g * STRIDE + c0] : 0.0f;
  const float x1 = c0 < ncol ? tile[(g + 8) * STRIDE + c0] : 0.0f;
  const float x2 = c1 < ncol ? tile[g * STRIDE + c1] : 0.0f;
  const float x3 = c1 < ncol ? tile[(g + 8) * STRIDE + c1] : 0.0f;
  split_tf32x2(make_float2(x0, x1), hi[0], lo[0], hi[1], lo[1]);
  split_tf32x2(make_float2(x2, x3), hi[2], lo[2], hi[3], lo[3]);
}

// Exterior state of a boundary face node, FP32 perturbation form (reading; see the FP64
// kernel): nb = -1 wall moving with the grid velocity (vgx, vgy), the particle velocities
// reflected about it (affine map of the moments with (wx, wy) = v_G / c, applied to the full
// state q1 = 1 + qm[0]); nb = -2 far field, the free-stream equilibrium minus the rest state.
template <int Np>
__device__ __forceinline__ void tc_boundary_state(int nb, const float *qm, float vgx, float vgy, float inv_c,
                                                  const float *farf, float (&qe)[6]) {
  if (nb == -1) {
    const float wx = vgx * inv_c, wy = vgy * inv_c;
    const float q1 = 1.0f + qm[0], q2 = qm[Np], q3 = qm[2 * Np];
    const float s2 = 2.8284271247461901f;   // 2 sqrt2
    qe[0] = qm[0];
    qe[1] = 2.0f * wx * q1 - q2;
    qe[2] = 2.0f * wy * q1 - q3;
    qe[3] = qm[3 * Np] + 4.0f * wx * wy * q1 - 2.0f * wx * q3 - 2.0f * wy * q2;
    qe[4] = qm[4 * Np] + s2 * (wx * wx * q1 - wx * q2);
    qe[5] = qm[5 * Np] + s2 * (wy * wy * q1 - wy * q3);
  } else {
#pragma unroll
    for (int f = 0; f < 6; ++f) qe[f] = farf[f];
  }
}

// One 16-element tile of one request: staging, geometry, volume, surface, cubature and the SARK
// combination.  BC: the mesh has boundary faces (neighbour codes -1 wall, -2 far field).  gfac / xfac are the stage's motion factors of the request; next_tile (or -1) is the
// tile this warp takes next in the same request (prefetched towards L2).
template <int N, int STAGE, bool BC, bool REC = false>
__device__ __forceinline__ void tc_tile(const StageArgs &a, int64_t tile, int64_t next_tile, double gfac, double xfac,
                                        const float4 *__restrict__ btab, float *own, float *trc, float *geo,
                                        const float (&bl)[TcDim<N>::NT][2][3], int lane, bool record = false,
                                        double fin = 0.0, double *dacc = nullptr) {
  typedef TcDim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN, KS = D::KS, KF = D::KF, NT = D::NT, CH = D::CH;
  constexpr int S = D::S, ST = D::ST, FJ = D::FJ, GEOS = D::GEOS;
  const float SQ2 = 1.41421356237309505f, ISQ2 = 0.70710678118654752f;
  const int g = lane >> 2, t = lane & 3;
  const float *qin = reinterpret_cast<const float *>(a.qin);
  const float c = (float)a.c, mc = -(float)a.c, mcs = -(float)a.c * SQ2;
  const float itau = (float)a.inv_tau;
  {
    const int64_t e0 = tile * 16;
    const int nel = (int)((a.K - e0) < 16 ? (a.K - e0) : 16);
    __syncwarp();
    // ---- stage the tile's fields (contiguous) ----
    {
      const float *src = qin + e0 * S;
      for (int i = lane; i < 4 * S; i += 32) tc_cp_async16(own + 4 * i, src + 4 * i);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // ---- neighbour traces: item = (element, face), 48 per tile ----
    for (int item = lane; item < 48; item += 32) {
      const int el = item % 16, f = item / 16;
      if (el < nel) {
        const int nb = a.mesh[e0 + el].nbr[f];
        if (BC && nb < 0) continue;   // exterior state formed in the flux phase
        const int f2 = nb & 3;
        const float *qp = qin + (int64_t)(nb >> 2) * S;
#pragma unroll
        for (int k = 0; k < Nfp; ++k) {
          const int vol2 = tc_fmask<N>(f2, Nfp - 1 - k);
#pragma unroll
          for (int fld = 0; fld < 6; ++fld) tc_cp_async4(trc + el * ST + fld * FJ + f * Nfp + k, qp + fld * Np + vol2);
        }
      }
    }
    if (lane == 0) {
      const unsigned bytes = 16 * S * sizeof(float);
      if (STAGE >= 1) {
        tc_l2_prefetch(reinterpret_cast<const float *>(a.qn) + e0 * S, bytes);
        if (STAGE <= 2) tc_l2_prefetch(reinterpret_cast<const float *>(a.F0) + e0 * S, bytes);
        if (STAGE >= 2) tc_l2_prefetch(reinterpret_cast<const float *>(a.acc) + e0 * S, bytes);
      }
      if (next_tile >= 0) {
        tc_l2_prefetch(qin + next_tile * 16 * S, bytes);
        const int64_t m0 = next_tile * 16;
        const int64_t mcount = (a.K - m0) < 16 ? (a.K - m0) : 16;   // records that exist
        tc_l2_prefetch(a.mesh + m0, (unsigned)(mcount * sizeof(MeshRec)));
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // ---- geometry of the tile's elements (lanes 0..15), while the copies fly ----
    double Jn1 = 0.0;   // REC: J of element `lane` at x_{n+1}
    if (lane < 16) {
      float *gm = geo + lane * GEOS;
      float ex[3] = {1.f, 0.f, -1.f}, ey[3] = {0.f, 1.f, -1.f}, vx[3] = {0.f, 0.f, 0.f}, vy[3] = {0.f, 0.f, 0.f};
      if (lane < nel) {
        const MeshRec rec = a.mesh[e0 + lane];
        // vertex positions x_n + shift and their differences in FP64; the stage's small motion
        // increments xfac S(X) in FP32
        double bx[3], by[3], pxn[3], pyn[3];
        float ix[3], iy[3];
        const float xff = (float)xfac, gff = (float)gfac;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double2 xv = reinterpret_cast<const double2 *>(a.xn)[rec.v[k]];
          const double2 sv = reinterpret_cast<const double2 *>(a.shape)[rec.v[k]];
          bx[k] = xv.x + rec.shift[2 * k] * a.period[0];
          by[k] = xv.y + rec.shift[2 * k + 1] * a.period[1];
          if (REC && record) {   // x_{n+1}, where the recorded integrals are taken
            pxn[k] = fma(fin, sv.x, bx[k]);
            pyn[k] = fma(fin, sv.y, by[k]);
          }
          const float sx = (float)sv.x, sy = (float)sv.y;
          ix[k] = xff * sx;
          iy[k] = xff * sy;
          vx[k] = gff * sx;
          vy[k] = gff * sy;
        }
        if (REC && record) Jn1 = 0.25 * ((pxn[1] - pxn[0]) * (pyn[2] - pyn[0]) - (pxn[2] - pxn[0]) * (pyn[1] - pyn[0]));
        ex[0] = (float)(bx[1] - bx[0]) + (ix[1] - ix[0]); ey[0] = (float)(by[1] - by[0]) + (iy[1] - iy[0]);
        ex[1] = (float)(bx[2] - bx[1]) + (ix[2] - ix[1]); ey[1] = (float)(by[2] - by[1]) + (iy[2] - iy[1]);
        ex[2] = (float)(bx[0] - bx[2]) + (ix[0] - ix[2]); ey[2] = (float)(by[0] - by[2]) + (iy[0] - iy[2]);
      }
      const float xr = 0.5f * ex[0], yr = 0.5f * ey[0], xs = -0.5f * ex[2], ys = -0.5f * ey[2];
      const float J = xr * ys - xs * yr;
      if (lane < nel && !(J > 0.0f)) atomicOr(a.status, GB_STATUS_MESH);
      const float iJ = 1.0f / J;
      gm[0] = ys * iJ; gm[1] = -yr * iJ; gm[2] = -xs * iJ; gm[3] = xr * iJ; gm[4] = iJ;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        gm[5 + k] = vx[k];
        gm[8 + k] = vy[k];
        gm[11 + k] = ex[k];
        gm[14 + k] = ey[k];
      }
    }
    // the own fields (first group) are needed now; the traces only for the surface term
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp();

    // accumulators: rhs[field][n-tile][fragment]
    float acc[6][NT][4];
#pragma unroll
    for (int f = 3; f < 6; ++f)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[f][nt][j] = 0.0f;
    // ---- collision term: I q at the cubature points, Ntilde there, P back (fields 4..6) ----
    {
      unsigned qh[3][KS][4], ql[3][KS][4];
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) load_a<S>(own, f * Np + ks * 8, f * Np + Np, g, t, qh[f][ks], ql[f][ks]);
#pragma unroll 1
      for (int ch = 0; ch < CH; ++ch) {
        float qc[3][4];
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
          for (int j = 0; j < 4; ++j) qc[f][j] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
          const float4 b = ldg_keep(btab + (D::B_I + ch * KS + ks) * 32 + lane);
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(qc[f], ql[f][ks], __float_as_uint(b.z), __float_as_uint(b.w));
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(qc[f], qh[f][ks], __float_as_uint(b.x), __float_as_uint(b.y));
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(qc[f], qh[f][ks], __float_as_uint(b.z), __float_as_uint(b.w));
        }
        // Ntilde at the 4 (element, point) positions; the accumulator order (c0, c2, c1, c3)
        // is the A-fragment order of the permuted chunk
        unsigned nh[3][4], nl[3][4];
        // fragment slots (j, j + 1) take accumulator entries (jp, jp + 2), jp = j / 2
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
          const int jp = j >> 1;
          const float2 q1 = __fadd2_rn(bc2(1.0f), make_float2(qc[0][jp], qc[0][jp + 2]));
          const float2 q2 = make_float2(qc[1][jp], qc[1][jp + 2]), q3 = make_float2(qc[2][jp], qc[2][jp + 2]);
          const float2 r1 = mul2(itau, make_float2(__frcp_rn(q1.x), __frcp_rn(q1.y)));
          const float2 rs = mul2(ISQ2, r1);
          split_tf32x2(__fmul2_rn(__fmul2_rn(q2, q3), r1), nh[0][j], nl[0][j], nh[0][j + 1], nl[0][j + 1]);
          split_tf32x2(__fmul2_rn(__fmul2_rn(q2, q2), rs), nh[1][j], nl[1][j], nh[1][j + 1], nl[1][j + 1]);
          split_tf32x2(__fmul2_rn(__fmul2_rn(q3, q3), rs), nh[2][j], nl[2][j], nh[2][j + 1], nl[2][j + 1]);
        }
        float4 bp[NT];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) bp[nt] = ldg_keep(btab + (D::B_P + ch * NT + nt) * 32 + lane);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(acc[3 + f][nt], nl[f], __float_as_uint(bp[nt].z), __float_as_uint(bp[nt].w));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(acc[3 + f][nt], nh[f], __float_as_uint(bp[nt].x), __float_as_uint(bp[nt].y));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int f = 0; f < 3; ++f) mma_tf32(acc[3 + f][nt], nh[f], __float_as_uint(bp[nt].z), __float_as_uint(bp[nt].w));
      }
    }

#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[f][nt][j] = 0.0f;

    // per-row geometry of this lane's two elements (rows g and g + 8)
    float rxr[2], sxr[2], ryr[2], syr[2], vgxp[2][NT][2], vgyp[2][NT][2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float *gm = geo + (g + 8 * h) * GEOS;
      rxr[h] = gm[0]; sxr[h] = gm[1]; ryr[h] = gm[2]; syr[h] = gm[3];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int col = 0; col < 2; ++col) {
          vgxp[h][nt][col] = bl[nt][col][0] * gm[5] + bl[nt][col][1] * gm[6] + bl[nt][col][2] * gm[7];
          vgyp[h][nt][col] = bl[nt][col][0] * gm[8] + bl[nt][col][1] * gm[9] + bl[nt][col][2] * gm[10];
        }
    }

    // ---- volume: (A + v_G) . grad q ----
#pragma unroll 1
    for (int f = 0; f < 6; ++f) {
      float dr[NT][4], ds[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) { dr[nt][j] = 0.0f; ds[nt][j] = 0.0f; }
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        unsigned ahi[4], alo[4];
        load_a<S>(own, f * Np + ks * 8, f * Np + Np, g, t, ahi, alo);
        float4 br[NT], bs[NT];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          br[nt] = ldg_keep(btab + (D::B_DR + ks * NT + nt) * 32 + lane);
          bs[nt] = ldg_keep(btab + (D::B_DS + ks * NT + nt) * 32 + lane);
        }
        // split terms outermost: consecutive products go to independent accumulators
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_tf32(dr[nt], alo, __float_as_uint(br[nt].z), __float_as_uint(br[nt].w));
          mma_tf32(ds[nt], alo, __float_as_uint(bs[nt].z), __float_as_uint(bs[nt].w));
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_tf32(dr[nt], ahi, __float_as_uint(br[nt].x), __float_as_uint(br[nt].y));
          mma_tf32(ds[nt], ahi, __float_as_uint(bs[nt].x), __float_as_uint(bs[nt].y));
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_tf32(dr[nt], ahi, __float_as_uint(br[nt].z), __float_as_uint(br[nt].w));
          mma_tf32(ds[nt], ahi, __float_as_uint(bs[nt].z), __float_as_uint(bs[nt].w));
        }
      }
      // pointwise: chain rule, v_G . grad q_f and the Atilde couplings (Sec. 2), on the
      // two columns of a fragment row at once
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j0 = 2 * h;
          const float2 d_r = make_float2(dr[nt][j0], dr[nt][j0 + 1]), d_s = make_float2(ds[nt][j0], ds[nt][j0 + 1]);
          const float2 qx = fma2(sxr[h], d_s, mul2(rxr[h], d_r));
          const float2 qy = fma2(syr[h], d_s, mul2(ryr[h], d_r));
          const float2 ale = __ffma2_rn(make_float2(vgyp[h][nt][0], vgyp[h][nt][1]), qy,
                                        __fmul2_rn(make_float2(vgxp[h][nt][0], vgxp[h][nt][1]), qx));
          auto A = [&](int ff) { return make_float2(acc[ff][nt][j0], acc[ff][nt][j0 + 1]); };
          auto P = [&](int ff, float2 v) { acc[ff][nt][j0] = v.x; acc[ff][nt][j0 + 1] = v.y; };
          switch (f) {
            case 0: P(0, __fadd2_rn(A(0), ale)); P(1, fma2(mc, qx, A(1))); P(2, fma2(mc, qy, A(2))); break;
            case 1: P(1, __fadd2_rn(A(1), ale)); P(0, fma2(mc, qx, A(0))); P(3, fma2(mc, qy, A(3)));
                    P(4, fma2(mcs, qx, A(4))); break;
            case 2: P(2, __fadd2_rn(A(2), ale)); P(0, fma2(mc, qy, A(0))); P(3, fma2(mc, qx, A(3)));
                    P(5, fma2(mcs, qy, A(5))); break;
            case 3: P(3, __fadd2_rn(A(3), ale)); P(2, fma2(mc, qx, A(2))); P(1, fma2(mc, qy, A(1))); break;
            case 4: P(4, __fadd2_rn(A(4), ale)); P(1, fma2(mcs, qx, A(1))); break;
            default: P(5, __fadd2_rn(A(5), ale)); P(2, fma2(mcs, qy, A(2))); break;
          }
        }
    }

    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    // ---- surface fluxes: item = (element, face), flux overwrites the trace in place ----
    for (int item = lane; item < 48; item += 32) {
      const int el = item % 16, f = item / 16;
      if (el >= nel) continue;
      const int nbf = BC ? a.mesh[e0 + el].nbr[f] : 0;
      const float *gm = geo + el * GEOS;
      const float dx = gm[11 + f], dy = gm[14 + f];
      const float len = sqrtf(dx * dx + dy * dy);
      const float il = 1.0f / len;
      const float nx = dy * il, ny = -dx * il;
      const float fs = 0.5f * len * gm[4];
      const float h = 0.5f * c * fs;
      const float al = (9.0f - 1.7320508075688772f) / 6.0f, be = (1.7320508075688772f - 3.0f) / 6.0f;
      const float nn = nx * nx + ny * ny;
      const float m00 = nn, m01 = 2.0f * nx * ny, m02 = SQ2 * nx * nx, m03 = SQ2 * ny * ny;
      const float m12 = SQ2 * nx * ny, m22 = 2.0f * nx * nx, m33 = 2.0f * ny * ny;
      const float q00 = m00 * m00 + m01 * m01 + m02 * m02 + m03 * m03;
      const float q01 = m00 * m01 + m01 * m00 + m02 * m12 + m03 * m12;
      const float q02 = m00 * m02 + m01 * m12 + m02 * m22;
      const float q03 = m00 * m03 + m01 * m12 + m03 * m33;
      const float q11 = m01 * m01 + m00 * m00 + m12 * m12 + m12 * m12;
      const float q12 = m01 * m02 + m00 * m12 + m12 * m22;
      const float q13 = m01 * m03 + m00 * m12 + m12 * m33;
      const float q22 = m02 * m02 + m12 * m12 + m22 * m22;
      const float q23 = m02 * m03 + m12 * m12;
      const float q33 = m03 * m03 + m12 * m12 + m33 * m33;
      const float M00 = h * (al * m00 + be * q00), M03 = h * (al * m01 + be * q01), M04 = h * (al * m02 + be * q02);
      const float M05 = h * (al * m03 + be * q03), M33 = h * (al * m00 + be * q11), M34 = h * (al * m12 + be * q12);
      const float M35 = h * (al * m12 + be * q13), M44 = h * (al * m22 + be * q22), M45 = h * (be * q23);
      const float M55 = h * (al * m33 + be * q33);
      const float o11 = 3.0f * nx * nx + ny * ny, o12 = 2.0f * nx * ny, o22 = nx * nx + 3.0f * ny * ny;
      const float N11 = h * (al * o11 + be * (o11 * o11 + o12 * o12));
      const float N12 = h * (al * o12 + be * (o11 * o12 + o12 * o22));
      const float N22 = h * (al * o22 + be * (o12 * o12 + o22 * o22));
      const float nhx = -h * nx, nhy = -h * ny, nsx = -h * SQ2 * nx, nsy = -h * SQ2 * ny;
      const float vx0 = gm[5], vx1 = gm[6], vx2 = gm[7], vy0 = gm[8], vy1 = gm[9], vy2 = gm[10];
      const float *bary = reinterpret_cast<const float *>(a.ops) + D::NSETS * 128;
      // face nodes in pairs (k, k + 1); an odd last node is paired with itself
#pragma unroll
      for (int k = 0; k < Nfp; k += 2) {
        const int k1 = k + 1 < Nfp ? k + 1 : k;
        const int vol0 = tc_fmask<N>(f, k), vol1 = tc_fmask<N>(f, k1);
        float *tr0 = trc + el * ST + f * Nfp + k, *tr1 = trc + el * ST + f * Nfp + k1;
        const float *qm0 = own + el * S + vol0, *qm1 = own + el * S + vol1;
        const float *b = bary + 4 * vol0, *c1 = bary + 4 * vol1;
        const float gx0 = __ldg(b) * vx0 + __ldg(b + 1) * vx1 + __ldg(b + 2) * vx2;
        const float gy0 = __ldg(b) * vy0 + __ldg(b + 1) * vy1 + __ldg(b + 2) * vy2;
        const float gx1 = __ldg(c1) * vx0 + __ldg(c1 + 1) * vx1 + __ldg(c1 + 2) * vx2;
        const float gy1 = __ldg(c1) * vy0 + __ldg(c1 + 1) * vy1 + __ldg(c1 + 2) * vy2;
        float2 w[6];
        if (BC && nbf < 0) {
          float qe0[6], qe1[6];
          tc_boundary_state<Np>(nbf, qm0, gx0, gy0, 1.0f / c, a.farf, qe0);
          tc_boundary_state<Np>(nbf, qm1, gx1, gy1, 1.0f / c, a.farf, qe1);
#pragma unroll
          for (int fld = 0; fld < 6; ++fld) w[fld] = make_float2(qe0[fld] - qm0[fld * Np], qe1[fld] - qm1[fld * Np]);
        } else {
#pragma unroll
          for (int fld = 0; fld < 6; ++fld)
            w[fld] = make_float2(tr0[fld * FJ] - qm0[fld * Np], tr1[fld * FJ] - qm1[fld * Np]);
        }
        float2 ale;
        {
          const float vn0 = gx0 * nx + gy0 * ny, vn1 = gx1 * nx + gy1 * ny;
          ale = make_float2(vn0 > 0.0f ? vn0 * fs : 0.0f, vn1 > 0.0f ? vn1 * fs : 0.0f);
        }
        float2 o[6];
        o[0] = __ffma2_rn(ale, w[0], fma2(M00, w[0], fma2(M03, w[3], fma2(M04, w[4], fma2(M05, w[5], fma2(nhx, w[1], mul2(nhy, w[2])))))));
        o[3] = __ffma2_rn(ale, w[3], fma2(M03, w[0], fma2(M33, w[3], fma2(M34, w[4], fma2(M35, w[5], fma2(nhx, w[2], mul2(nhy, w[1])))))));
        o[4] = __ffma2_rn(ale, w[4], fma2(M04, w[0], fma2(M34, w[3], fma2(M44, w[4], fma2(M45, w[5], mul2(nsx, w[1]))))));
        o[5] = __ffma2_rn(ale, w[5], fma2(M05, w[0], fma2(M35, w[3], fma2(M45, w[4], fma2(M55, w[5], mul2(nsy, w[2]))))));
        o[1] = __ffma2_rn(ale, w[1], fma2(N11, w[1], fma2(N12, w[2], fma2(nhx, w[0], fma2(nsx, w[4], mul2(nhy, w[3]))))));
        o[2] = __ffma2_rn(ale, w[2], fma2(N12, w[1], fma2(N22, w[2], fma2(nhy, w[0], fma2(nsy, w[5], mul2(nhx, w[3]))))));
#pragma unroll
        for (int fld = 0; fld < 6; ++fld) {
          tr0[fld * FJ] = o[fld].x;
          if (k1 != k) tr1[fld * FJ] = o[fld].y;
        }
      }
    }
    __syncwarp();

    // ---- LIFT of the fluxes: fields in two groups of three, split terms outermost ----
#pragma unroll
    for (int fg = 0; fg < 6; fg += 3) {
#pragma unroll
      for (int kf = 0; kf < KF; ++kf) {
        unsigned ahi[3][4], alo[3][4];
#pragma unroll
        for (int ff = 0; ff < 3; ++ff) load_a<ST>(trc, (fg + ff) * FJ + kf * 8, (fg + ff) * FJ + NFN, g, t, ahi[ff], alo[ff]);
        float4 bq[NT];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) bq[nt] = ldg_keep(btab + (D::B_LIFT + kf * NT + nt) * 32 + lane);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int ff = 0; ff < 3; ++ff) mma_tf32(acc[fg + ff][nt], alo[ff], __float_as_uint(bq[nt].z), __float_as_uint(bq[nt].w));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int ff = 0; ff < 3; ++ff) mma_tf32(acc[fg + ff][nt], ahi[ff], __float_as_uint(bq[nt].x), __float_as_uint(bq[nt].y));
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int ff = 0; ff < 3; ++ff) mma_tf32(acc[fg + ff][nt], ahi[ff], __float_as_uint(bq[nt].z), __float_as_uint(bq[nt].w));
      }
    }

    // ---- rhs tile to shared memory (over the fluxes), then the SARK pass ----
    __syncwarp();
    float *out = trc;   // [16][S]
#pragma unroll
    for (int f = 0; f < 6; ++f)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int row = g + 8 * (j >> 1), n = nt * 8 + 2 * t + (j & 1);
          if (n < Np) out[row * S + f * Np + n] = acc[f][nt][j];
        }
    __syncwarp();
    {
      const float dt = (float)a.dt;
      // lane slots w = lane + 32 sl of each element's 6 Np values; class 0 for fields 1..3;
      // the coefficients arrive in FP32 (set_mixed_coefs)
      constexpr int NSL = (6 * Np + 31) / 32;
      float E1[NSL], A0[NSL], A1[NSL], Bc[NSL], B1[NSL];
#pragma unroll
      for (int sl = 0; sl < NSL; ++sl) {
        const int cl = (lane + 32 * sl) < 3 * Np ? 0 : 1;
        E1[sl] = a.kco[cl][0];
        A0[sl] = a.kco[cl][1];
        A1[sl] = a.kco[cl][2];
        Bc[sl] = a.kco[cl][3];
        B1[sl] = a.kco[cl][4];
      }
      bool bad = false;
      float *Fo = reinterpret_cast<float *>(a.Fout);
      float *qo = reinterpret_cast<float *>(a.qout);
      float *F0 = reinterpret_cast<float *>(a.F0);
      float *ac = reinterpret_cast<float *>(a.acc);
      const float *qn = reinterpret_cast<const float *>(a.qn);
      // Batches of RB rows: every load of a batch is issued before any store of it
      // (outputs may alias inputs: q_{n+1} overwrites q_n in place), so a batch costs
      // one memory round trip instead of one per row.  The loads are read-once streams
      // (ld.global.cs, evict first), which keeps the operator tables in L1.
      constexpr int RB = 8;
#pragma unroll 1
      for (int r0 = 0; r0 < 16; r0 += RB) {
        float rv[RB][NSL], x0[RB][NSL], x1[RB][NSL], x2[RB][NSL];
#pragma unroll
        for (int rr = 0; rr < RB; ++rr)
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl) {
            const int r = r0 + rr, w = lane + 32 * sl;
            const bool ok = r < nel && w < 6 * Np;
            const int64_t gi = (e0 + r) * S + w;
            rv[rr][sl] = ok ? out[r * S + w] : 0.0f;
            x0[rr][sl] = x1[rr][sl] = x2[rr][sl] = 0.0f;
            if (ok) {
              if (STAGE == 0) x0[rr][sl] = own[r * S + w];
              if (STAGE >= 1) x0[rr][sl] = __ldcs(qn + gi);
              if (STAGE == 1 || STAGE == 2) x1[rr][sl] = __ldcs(F0 + gi);
              if (STAGE >= 2) x2[rr][sl] = __ldcs(ac + gi);
            }
          }
        // rows in pairs (rr, rr + 1): one packed instruction for both
#pragma unroll
        for (int rr = 0; rr < RB; rr += 2)
#pragma unroll
          for (int sl = 0; sl < NSL; ++sl) {
            const int r = r0 + rr, w = lane + 32 * sl;
            if (!(w < 6 * Np) || r >= nel) continue;
            const bool ok1 = r + 1 < nel;
            const int64_t gi = (e0 + r) * S + w, gi1 = gi + S;
            const float2 r_ = make_float2(rv[rr][sl], rv[rr + 1][sl]), qv = make_float2(x0[rr][sl], x0[rr + 1][sl]);
            const float2 f0 = make_float2(x1[rr][sl], x1[rr + 1][sl]), av = make_float2(x2[rr][sl], x2[rr + 1][sl]);
            float2 o = make_float2(0.0f, 0.0f), o2 = make_float2(0.0f, 0.0f);
            if (STAGE < 0) {
              o = r_;
            } else if (STAGE == 0) {
              o2 = r_;
              o = fma2(dt, mul2(A0[sl], r_), mul2(E1[sl], qv));
            } else if (STAGE == 1) {
              o = fma2(dt, fma2(A1[sl], r_, mul2(A0[sl], f0)), mul2(E1[sl], qv));
              o2 = fma2(B1[sl], r_, mul2(Bc[sl], f0));
            } else if (STAGE == 2) {
              o = fma2(dt, fma2(A1[sl], r_, mul2(A0[sl], f0)), mul2(E1[sl], qv));
              o2 = fma2(Bc[sl], r_, av);
            } else {
              o = fma2(dt, fma2(Bc[sl], r_, av), mul2(E1[sl], qv));
              bad |= (__float_as_int(o.x) & 0x7f800000) == 0x7f800000;
              bad |= ok1 && (__float_as_int(o.y) & 0x7f800000) == 0x7f800000;
              if (REC && record && w < 3 * Np) {   // q_{n+1} of fields 1..3 over the (already read) rhs
                out[r * S + w] = o.x;
                if (ok1) out[(r + 1) * S + w] = o.y;
              }
            }
            float *dst = STAGE < 0 ? Fo : qo;
            dst[gi] = o.x;
            if (ok1) dst[gi1] = o.y;
            if (STAGE == 0) {
              F0[gi] = o2.x;
              if (ok1) F0[gi1] = o2.y;
            } else if (STAGE == 1 || STAGE == 2) {
              ac[gi] = o2.x;
              if (ok1) ac[gi1] = o2.y;
            }
          }
      }
      if (STAGE == 3 && bad) atomicOr(a.status, GB_STATUS_NAN);
    }
    // ---- fused diagnostics (REC, record steps): integrals of q_{n+1} over the tile on x_{n+1}:
    //      J w_n q1, J w_n c^2 (q2^2 + q3^2) / (2 q1), J w_n c q2, J w_n c q3, J w_n ----
    if (REC && record) {
      __syncwarp();
      const double cc = a.c;
      constexpr int NIT = (16 * Np + 31) / 32;
#pragma unroll 1
      for (int it = 0; it < NIT; ++it) {
        const int item = lane + 32 * it, r = item / Np, n = item - Np * (item / Np);
        const double J = __shfl_sync(0xffffffffu, Jn1, r & 15);
        if (item < 16 * Np && r < nel) {
          const double q1 = 1.0 + (double)out[r * S + n], q2 = (double)out[r * S + Np + n];
          const double q3 = (double)out[r * S + 2 * Np + n], jw = J * a.rec_wq[n];
          dacc[0] += jw * q1;
          dacc[1] += jw * 0.5 * cc * cc * (q2 * q2 + q3 * q3) / q1;
          dacc[2] += jw * cc * q2;
          dacc[3] += jw * cc * q3;
          dacc[4] += jw;
        }
      }
    }
  }
}

template <int N>
__device__ __forceinline__ void tc_load_bary(const void *ops, int lane, float (&bl)[TcDim<N>::NT][2][3]) {
  typedef TcDim<N> D;
  const int t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < D::NT; ++nt)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = nt * 8 + 2 * t + j;
      const float *bary = reinterpret_cast<const float *>(ops) + D::NSETS * 128 + 4 * (n < D::Np ? n : 0);
      bl[nt][j][0] = bary[0];
      bl[nt][j][1] = bary[1];
      bl[nt][j][2] = bary[2];
    }
}

template <int N, int STAGE, bool BC, bool REC = false>
__global__ void __launch_bounds__(32 * TcDim<N>::W, (N <= 4 ? 3 : 1)) tc_stage_kernel(const StageArgs a) {
  typedef TcDim<N> D;
  const int W = blockDim.x >> 5;                // warps per CTA: a launch parameter (1, 2 or 4)
  extern __shared__ float4 tc_smem4[];
  const float4 *btab = reinterpret_cast<const float4 *>(a.ops);     // [NSETS][32], read through L1
  float *wbase = reinterpret_cast<float *>(tc_smem4);
  __shared__ double s_motion[3];
  // REC: whether this step is recorded, read before any CTA can advance the counter
  const bool record = REC && ((a.rec_ctl[0] + 1) % a.rec_every == 0);
  const double t_now = a.clock[0];
  if (threadIdx.x == 0) {
    double gf, xf, fin;
    tc_stage_motion<STAGE>(a, gf, xf, fin);
    s_motion[0] = gf;
    s_motion[1] = xf;
    s_motion[2] = fin;
  }
  __syncthreads();
  if (STAGE == 3 && blockIdx.x == 0 && threadIdx.x == 0) const_cast<double *>(a.clock)[1] = s_motion[2];
  const double gfac = s_motion[0], xfac = s_motion[1], fin = s_motion[2];
  double dacc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *own = wbase + warp * D::WARP_FLOATS;   // [16][S]   fields of the tile
  float *trc = own + 16 * D::S;                 // [16][ST] traces -> fluxes, then [16][S] rhs (16 OUTS floats)
  float *geo = trc + 16 * D::OUTS;              // [16][GEOS]
  float bl[D::NT][2][3];                        // barycentric coordinates of this lane's output nodes
  tc_load_bary<N>(a.ops, lane, bl);
  const int64_t ntile = (a.K + 15) >> 4;
  const int64_t tstride = (int64_t)gridDim.x * W;
  for (int64_t tile = (int64_t)blockIdx.x * W + warp; tile < ntile; tile += tstride)
    tc_tile<N, STAGE, BC, REC>(a, tile, tile + tstride < ntile ? tile + tstride : -1, gfac, xfac, btab, own, trc, geo, bl,
                               lane, record, fin, dacc);
  if constexpr (REC) fused_record(a, record, dacc, t_now + a.dt);
}

// Many requests of the same order in one launch: tile T of the launch is tile
// T - tile_start[r] of request r (tile_start is the exclusive prefix of the
// requests' tile counts).  Each warp derives its request's motion factors.
template <int N, int STAGE>
__global__ void __launch_bounds__(32 * TcDim<N>::W, (N <= 4 ? 3 : 1)) tc_group_kernel(const GroupArgs gd) {
  typedef TcDim<N> D;
  const int W = blockDim.x >> 5;                // warps per CTA: a launch parameter (1, 2 or 4)
  extern __shared__ float4 tc_smem4[];
  const float4 *btab = reinterpret_cast<const float4 *>(gd.ops);
  float *wbase = reinterpret_cast<float *>(tc_smem4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *own = wbase + warp * D::WARP_FLOATS;
  float *trc = own + 16 * D::S;
  float *geo = trc + 16 * D::OUTS;
  float bl[D::NT][2][3];
  tc_load_bary<N>(gd.ops, lane, bl);
  const int64_t tstride = (int64_t)gridDim.x * W;
  for (int64_t T = (int64_t)blockIdx.x * W + warp; T < gd.total_tiles; T += tstride) {
    int lo = 0, hi = gd.n - 1;              // last r with tile_start[r] <= T
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (gd.tile_start[mid] <= T) lo = mid; else hi = mid - 1;
    }
    const StageArgs &a = gd.args[lo];
    const int64_t tile = T - gd.tile_start[lo];
    const int64_t ntile = gd.tile_start[lo + 1] - gd.tile_start[lo];
    double gf = 0.0, xf = 0.0;
    if (lane == 0) {
      double fin;
      tc_stage_motion<STAGE>(a, gf, xf, fin);
      if (STAGE == 3 && tile == 0) const_cast<double *>(a.clock)[1] = fin;
    }
    gf = __shfl_sync(0xffffffffu, gf, 0);
    xf = __shfl_sync(0xffffffffu, xf, 0);
    tc_tile<N, STAGE, false>(a, tile, tile + tstride < ntile ? tile + tstride : -1, gf, xf, btab, own, trc, geo, bl, lane);
  }
}

// ---------------------------------------------------------------------------
constexpr int kTcMaxDevices = 64;

template <int N>
static size_t tc_smem(int W = TcDim<N>::W) {
  typedef TcDim<N> D;
  return sizeof(float) * (size_t)W * D::WARP_FLOATS;
}

// The stage's SARK coefficients for the mixed kernel, in FP32, per field class:
// E_{i+1} (E at the final stage), the two atilde of the stage combination, and the two
// btilde weights of the running accumulator (Sec. 4); stage -1 (rhs only) uses none.
void set_mixed_coefs(StageArgs &a) {
  for (int cl = 0; cl < 2; ++cl) {
    const int s = a.stage;
    const double *E = a.co.E[cl], *A = a.co.A[cl], *B = a.co.B[cl];
    a.kco[cl][0] = (float)(s < 0 ? E[0] : (s < 3 ? E[s + 1] : E[4]));
    a.kco[cl][1] = (float)(s == 0 ? A[4] : s == 1 ? A[8] : s == 2 ? A[12] : 0.0);
    a.kco[cl][2] = (float)(s == 1 ? A[9] : s == 2 ? A[14] : 0.0);
    a.kco[cl][3] = (float)(s == 1 ? B[0] : s == 2 ? B[2] : s == 3 ? B[3] : 0.0);
    a.kco[cl][4] = (float)B[1];
  }
  for (int f = 0; f < 6; ++f) a.farf[f] = (float)a.far[f];
}

template <int N, int STAGE, bool BC, bool REC = false>
static int tc_launch_one(const StageArgs &a_in, cudaStream_t st, int num_sms) {
  StageArgs a = a_in;
  set_mixed_coefs(a);
  typedef TcDim<N> D;
  const int W = (a.warps_per_cta == 1 || a.warps_per_cta == 2) ? a.warps_per_cta : D::W;
  const size_t smem = tc_smem<N>(W);
  const int threads = 32 * W;
  // the shared-memory opt-in and the occupancy are per-device facts: cached per device ordinal
  // (the first launch on a device queries them; none happen during a graph capture after it)
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return (int)derr;
  if (dev < 0 || dev >= kTcMaxDevices) return (int)cudaErrorInvalidDevice;
  static bool attr_set[kTcMaxDevices] = {};
  if (!attr_set[dev]) {
    cudaError_t err = cudaFuncSetAttribute(tc_stage_kernel<N, STAGE, BC, REC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<N>());
    if (err != cudaSuccess) return (int)err;
    attr_set[dev] = true;
  }
  static int per_sm_w[kTcMaxDevices][5] = {};
  int &per_sm = per_sm_w[dev][W];
  if (per_sm == 0) {
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_stage_kernel<N, STAGE, BC, REC>, threads, smem);
    if (err != cudaSuccess) return (int)err;
    if (per_sm < 1) per_sm = 1;
  }
  int64_t grid = (int64_t)num_sms * per_sm;
  const int64_t need = ((a.K + 15) / 16 + W - 1) / W;
  if (grid > need) grid = need;
  if (REC && grid > kRecMaxCtas) grid = kRecMaxCtas;
  if (grid < 1) grid = 1;
  tc_stage_kernel<N, STAGE, BC, REC><<<(unsigned)grid, threads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <int N, bool BC>
static int tc_launch_nb(const StageArgs &a, cudaStream_t st, int num_sms) {
  switch (a.stage) {
    case -1: return tc_launch_one<N, -1, BC>(a, st, num_sms);
    case 0: return tc_launch_one<N, 0, BC>(a, st, num_sms);
    case 1: return tc_launch_one<N, 1, BC>(a, st, num_sms);
    case 2: return tc_launch_one<N, 2, BC>(a, st, num_sms);
    case 3:
      return a.rec_every > 0 ? tc_launch_one<N, 3, BC, true>(a, st, num_sms) : tc_launch_one<N, 3, BC>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

// meshes with boundary faces use the BC variant (orders 1..4)
template <int N>
static int tc_launch_n(const StageArgs &a, cudaStream_t st, int num_sms) {
  if (a.bc) {
    if constexpr (N <= 4) return tc_launch_nb<N, true>(a, st, num_sms);
    return (int)cudaErrorInvalidValue;
  }
  return tc_launch_nb<N, false>(a, st, num_sms);
}

int launch_stage_mixed(int N, const StageArgs &a, void *stream, int num_sms) {
  // shape kShapeUm: the tcgen05 kernel, except where it does not apply (boundary faces, the
  // last stage with fused diagnostics), where the 4-warp shape of this kernel runs
  if (a.warps_per_cta == kShapeUm && a.ops_um && !a.bc && !(a.stage == 3 && a.rec_every > 0) && um_supported(N))
    return launch_stage_um(N, a, stream, num_sms);
  cudaStream_t st = (cudaStream_t)stream;
  switch (N) {
    case 1: return tc_launch_n<1>(a, st, num_sms);
    case 2: return tc_launch_n<2>(a, st, num_sms);
    case 3: return tc_launch_n<3>(a, st, num_sms);
    case 4: return tc_launch_n<4>(a, st, num_sms);
    case 5: return tc_launch_n<5>(a, st, num_sms);
    case 6: return tc_launch_n<6>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

template <int N, int STAGE>
static int tc_group_launch_one(const GroupArgs &g, cudaStream_t st, int num_sms) {
  typedef TcDim<N> D;
  const int W = (g.warps == 1 || g.warps == 2) ? g.warps : D::W;
  const size_t smem = tc_smem<N>(W);
  const int threads = 32 * W;
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return (int)derr;
  if (dev < 0 || dev >= kTcMaxDevices) return (int)cudaErrorInvalidDevice;
  static bool attr_set[kTcMaxDevices] = {};   // per device ordinal, like the single-solver launcher
  if (!attr_set[dev]) {
    cudaError_t err = cudaFuncSetAttribute(tc_group_kernel<N, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<N>());
    if (err != cudaSuccess) return (int)err;
    attr_set[dev] = true;
  }
  static int per_sm_d[kTcMaxDevices][5] = {};
  int &per_sm = per_sm_d[dev][W];
  if (per_sm == 0) {
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_group_kernel<N, STAGE>, threads, smem);
    if (err != cudaSuccess) return (int)err;
  }
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  const int64_t need = (g.total_tiles + W - 1) / W;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  tc_group_kernel<N, STAGE><<<(unsigned)grid, threads, smem, st>>>(g);
  return (int)cudaGetLastError();
}

template <int N>
static int tc_group_launch_n(int stage, const GroupArgs &g, cudaStream_t st, int num_sms) {
  switch (stage) {
    case 0: return tc_group_launch_one<N, 0>(g, st, num_sms);
    case 1: return tc_group_launch_one<N, 1>(g, st, num_sms);
    case 2: return tc_group_launch_one<N, 2>(g, st, num_sms);
    case 3: return tc_group_launch_one<N, 3>(g, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_group_mixed(int N, int stage, const GroupArgs &g, void *stream, int num_sms) {
  cudaStream_t st = (cudaStream_t)stream;
  switch (N) {
    case 1: return tc_group_launch_n<1>(stage, g, st, num_sms);
    case 2: return tc_group_launch_n<2>(stage, g, st, num_sms);
    case 3: return tc_group_launch_n<3>(stage, g, st, num_sms);
    case 4: return tc_group_launch_n<4>(stage, g, st, num_sms);
    case 5: return tc_group_launch_n<5>(stage, g, st, num_sms);
    case 6: return tc_group_launch_n<6>(stage, g, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

// final vertex update of every request of a group: x_{n+1} = x_n + fin S(X), t += dt
__global__ void group_vertex_update_kernel(const GroupArgs g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.total_vertices;
       i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (g.vtx_start[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const StageArgs &a = g.args[lo];
    const int64_t v = i - g.vtx_start[lo];
    double *xn = const_cast<double *>(a.xn);
    const double fin = a.clock[1];
    xn[2 * v] += fin * a.shape[2 * v];
    xn[2 * v + 1] += fin * a.shape[2 * v + 1];
    if (v == 0) const_cast<double *>(a.clock)[0] += a.dt;
  }
}

int launch_group_vertex_update(const GroupArgs &g, void *stream) {
  int64_t blocks = (g.total_vertices + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  group_vertex_update_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(g);
  return (int)cudaGetLastError();
}

int mixed_stride(int N) {
  switch (N) {
    case 1: return TcDim<1>::S;
    case 2: return TcDim<2>::S;
    case 3: return TcDim<3>::S;
    case 4: return TcDim<4>::S;
    case 5: return TcDim<5>::S;
    case 6: return TcDim<6>::S;
  }
  return 0;
}

// ---- operator tables: B fragments (hi, lo) per lane, then the node barycentric table ----
static inline float tf32_round_host(float x) {
  // round to nearest, ties away from zero, at 10 explicit mantissa bits (cvt.rna.tf32.f32)
  uint32_t u;
  memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x1000u;
    u &= 0xffffe000u;
  }
  float r;
  memcpy(&r, &u, 4);
  return r;
}

template <int N>
static void fill_tc(const RefOps &Rf, std::vector<float> &h) {
  typedef TcDim<N> D;
  const int Np = D::Np, NFN = D::NFN, Nc = D::Nc;
  h.assign((size_t)D::NSETS * 128 + 4 * 32, 0.0f);
  auto put = [&](int set, auto Bfun) {   // Bfun(k, n) -> value of the K x N operand
    for (int lane = 0; lane < 32; ++lane) {
      const int gq = lane >> 2, tq = lane & 3;
      const float v0 = (float)Bfun(tq, gq), v1 = (float)Bfun(tq + 4, gq);
      const float h0 = tf32_round_host(v0), h1 = tf32_round_host(v1);
      float *o = &h[((size_t)set * 32 + lane) * 4];
      o[0] = tf32_round_host(v0 - h0);
      o[1] = tf32_round_host(v1 - h1);
      o[2] = h0;
      o[3] = h1;
    }
  };
  for (int ks = 0; ks < D::KS; ++ks)
    for (int nt = 0; nt < D::NT; ++nt) {
      put(D::B_DR + ks * D::NT + nt, [&](int k, int n) {
        const int m = ks * 8 + k, o = nt * 8 + n;
        return (m < Np && o < Np) ? Rf.Dr[o * Np + m] : 0.0;
      });
      put(D::B_DS + ks * D::NT + nt, [&](int k, int n) {
        const int m = ks * 8 + k, o = nt * 8 + n;
        return (m < Np && o < Np) ? Rf.Ds[o * Np + m] : 0.0;
      });
    }
  for (int kf = 0; kf < D::KF; ++kf)
    for (int nt = 0; nt < D::NT; ++nt)
      put(D::B_LIFT + kf * D::NT + nt, [&](int k, int n) {
        const int j = kf * 8 + k, o = nt * 8 + n;
        return (j < NFN && o < Np) ? Rf.LIFT[o * NFN + j] : 0.0;
      });
  for (int ch = 0; ch < D::CH; ++ch)
    for (int ks = 0; ks < D::KS; ++ks)
      put(D::B_I + ch * D::KS + ks, [&](int k, int n) {
        const int m = ks * 8 + k, cp = ch * 8 + n;
        return (m < Np && cp < Nc) ? Rf.I[cp * Np + m] : 0.0;
      });
  for (int ch = 0; ch < D::CH; ++ch)
    for (int nt = 0; nt < D::NT; ++nt)
      put(D::B_P + ch * D::NT + nt, [&](int k, int n) {
        // chunk columns taken in the order (0,2,4,6,1,3,5,7): k < 4 -> point 2k, k >= 4 -> 2(k-4)+1
        const int cp = ch * 8 + (k < 4 ? 2 * k : 2 * (k - 4) + 1), o = nt * 8 + n;
        return (cp < Nc && o < Np) ? Rf.P[o * Nc + cp] : 0.0;
      });
  // fragment float4 = (lo0, lo1, hi0, hi1): mma3 uses .x/.y as the tail and .z/.w as the head
  float *bary = &h[(size_t)D::NSETS * 128];
  for (int n = 0; n < Np && n < 32; ++n) {
    bary[4 * n] = (float)(-0.5 * (Rf.r[n] + Rf.s[n]));
    bary[4 * n + 1] = (float)(0.5 * (1.0 + Rf.r[n]));
    bary[4 * n + 2] = (float)(0.5 * (1.0 + Rf.s[n]));
  }
}

int upload_ops_mixed(int N, const RefOps &Rf, float **dev_ops, void *stream) {
  std::vector<float> h;
  switch (N) {
    case 1: fill_tc<1>(Rf, h); break;
    case 2: fill_tc<2>(Rf, h); break;
    case 3: fill_tc<3>(Rf, h); break;
    case 4: fill_tc<4>(Rf, h); break;
    case 5: fill_tc<5>(Rf, h); break;
    case 6: fill_tc<6>(Rf, h); break;
    default: return (int)cudaErrorInvalidValue;
  }
  void *d = nullptr;
  cudaError_t err = cudaMalloc(&d, h.size() * sizeof(float));
  if (err != cudaSuccess) return (int)err;
  err = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    cudaFree(d);
    return (int)err;
  }
  *dev_ops = reinterpret_cast<float *>(d);
  return 0;
}

// ---------------------------------------------------------------------------
// canonical <-> internal (element-major, stride S, Morton order) relayout.
// perm[i] = canonical index of internal element i.  rest is added to field 1
// on the way out and subtracted on the way in (0 for arrays that are not states).
template <typename Tc, bool TO_INTERNAL>
__global__ void relayout_kernel(Tc *canon, float *inner, const int32_t *perm, int64_t K, int Np, int S, double rest) {
  const int NQ = 6 * Np;
  const int64_t total = K * NQ;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / NQ;
    const int fn = (int)(i - e * NQ);
    const int64_t ci = (int64_t)perm[e] * NQ + fn;
    const int64_t ii = e * S + fn;
    const double r = fn < Np ? rest : 0.0;
    if (TO_INTERNAL) inner[ii] = (float)((double)canon[ci] - r);
    else canon[ci] = (Tc)((double)inner[ii] + r);
  }
}

int launch_relayout(const void *canon_src, void *canon_dst, bool canon_is_double, bool to_internal, float *inner,
                    const int32_t *perm, int64_t K, int Np, int S, double rest, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = 2048, thr = 256;
  if (to_internal) {
    if (canon_is_double)
      relayout_kernel<double, true><<<blocks, thr, 0, st>>>(const_cast<double *>((const double *)canon_src), inner, perm, K, Np, S, rest);
    else
      relayout_kernel<float, true><<<blocks, thr, 0, st>>>(const_cast<float *>((const float *)canon_src), inner, perm, K, Np, S, rest);
  } else {
    if (canon_is_double)
      relayout_kernel<double, false><<<blocks, thr, 0, st>>>((double *)canon_dst, inner, perm, K, Np, S, rest);
    else
      relayout_kernel<float, false><<<blocks, thr, 0, st>>>((float *)canon_dst, inner, perm, K, Np, S, rest);
  }
  return (int)cudaGetLastError();
}

}  // namespace gb
