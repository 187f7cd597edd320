// GB_MIXED 3D stage kernel on the tensor cores (tetrahedra, 10 moment fields, N <= 3).
//
// Same right-hand side and SARK combination as the one-thread-per-node kernels of
// gb_kernels3d.cu (Secs. 2-5 in 3D), with the four dense contractions of the
// semi-discrete form issued as mma.sync.m16n8k8 TF32 products with FP32 accumulation:
//   volume      D_a q_f for a = r, s, t and the 10 fields  (K = Np, N = Np per direction)
//   lift        LIFT flux_f for the 10 fields               (K = 4 Nfp, N = Np)
//   cubature    I q_f at the degree-3N points, fields 1..4   (K = Np, N = Nc, chunks of 8)
//   projection  P Ntilde_f onto fields 5..10                (K = Nc, N = Np)
// Every operand is split into a TF32 head and tail (x = hi + lo) and every product is
// formed as hi*hi + hi*lo + lo*hi (relative error ~2^-21; the dropped lo*lo is 2^-22).
// Each operand's head is x rounded to 10 mantissa bits by two integer operations and its
// tail is the exact FP32 remainder, whose low bits the tensor core ignores.
//
// Work layout: one warp owns a tile of 16 consecutive elements, the M dimension of every
// product (rows = elements, columns = nodes, face nodes or cubature points).  A CTA of W
// warps holds the B-fragment table in shared memory (FP32, split into head and tail on
// use: read through L1 it missed, since the warps' shared tiles leave L1 too small for
// it); its warps work without waiting on one another (one CTA barrier, after the table is
// loaded).  Per tile:
//   1. the tile's fields are copied into shared memory by cp.async (rows padded to a
//      stride S = 4 mod 8, so that A-fragment loads are free of bank conflicts) while
//      lanes 0..15 form one element's geometry each (FP64 vertex positions and
//      differences, FP32 afterwards; the same routine as the FP32 kernel);
//   2. the neighbour traces of the first face-node k-step are requested (cp.async into
//      this lane's slots), to arrive during the cubature;
//   3. cubature chain, chunk by chunk: the accumulator fragment of I q is reused directly
//      as the A fragment of P Ntilde (the chunk's 8 points taken in the order
//      0,2,4,6,1,3,5,7, folded into the P table); the result seeds the accumulators of
//      fields 5..10;
//   4. surface: each lane forms the upwind flux exactly at the four (element, face node)
//      slots of the A fragment it feeds to the lift product, from the traces in its slots
//      (the next k-step's traces arrive in a second slot set meanwhile);
//   5. the accumulators of n-tiles 1.. are parked in shared memory (fragment order);
//   6. per n-tile: volume (the three derivative fragments of each field, then the chain
//      rule, the grid velocity term v_G . grad q_f = sum_a vt_a D_a q_f with
//      vt_a = (G^-1 v_G)_a, and the Atilde couplings, all in the thread that holds the
//      node), then the SARK combination straight from the accumulators (node pairs).
// The rhs accumulators of all 10 fields (10 x ceil(Np/8) fragments) stay in registers
// through steps 3 and 4; step 6 holds one n-tile's at a time.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <vector>

#include "gb3d_internal.h"
#include "gb_kernels3d_dev.cuh"

namespace gb {

template <int N>
struct Tc3Dim {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NFN = 4 * Nfp;
  static constexpr int QC = (3 * N + 2) / 2;
  static constexpr int Nc = QC * QC * QC;
  static constexpr int NQ = 10 * Np;
  static constexpr int KS = (Np + 7) / 8;   // k-steps over nodes
  static constexpr int NT = KS;             // n-tiles over output nodes
  static constexpr int KF = (NFN + 7) / 8;  // k-steps over face nodes
  static constexpr int CH = (Nc + 7) / 8;   // cubature chunks of 8 points
  static constexpr int S = NQ + (12 - NQ % 8) % 8;   // element stride of the shared tile, S = 4 mod 8
  // B-fragment sets (32 lanes x float2 (b0, b1) each, FP32; split into head and tail on use)
  static constexpr int B_VOL = 0;                     // [a][ks][nt]: D_a^T
  static constexpr int B_LIFT = B_VOL + 3 * KS * NT;  // [kf][nt]: LIFT^T
  static constexpr int B_I = B_LIFT + KF * NT;        // [ch][ks]: I^T
  static constexpr int B_P = B_I + CH * KS;           // [ch][nt]: P^T, chunk columns permuted
  static constexpr int NSETS = B_P + CH * NT;
  // after the sets (offsets in 4-byte words): barycentric node coordinates [Np][4] (float),
  // face-node volume indices [4][Nfp] (int), neighbour node table [4][4][6][Nfp] (int)
  static constexpr int TAB_SETS = NSETS * 64;        // floats of the sets, copied into shared memory
  static constexpr int TAB_BARY = TAB_SETS;
  static constexpr int TAB_FMASK = TAB_BARY + 4 * Np;
  static constexpr int TAB_NBR = TAB_FMASK + 4 * Nfp;
  static constexpr int TAB_WORDS = TAB_NBR + 96 * Nfp;
  // per-element geometry in shared memory (floats): [0, 9) G^-1 (row a = grad of reference
  // coordinate a); [12, 28) per face nx ny nz Fscale; [28, 44) per face v_k . n (4 vertices);
  // [44, 48) neighbour codes (int bits); [48, 60) (G^-1 v_k)_a as [a][k].  Every group read
  // by a 16-byte load starts on a multiple of 4 floats; stride 60: the 16-byte loads of two
  // elements in a quarter warp fall in different banks.
  static constexpr int GEO = 60, G_FACE = 12, G_VN = 28, G_NBR = 44, G_VTIL = 48;
  static_assert(G_FACE % 4 == 0 && G_VN % 4 == 0 && G_VTIL + 12 <= GEO && GEO % 4 == 0, "geometry layout");
  static constexpr int FLS = 41;            // per lane and k-step: 4 x 10 traces, then fluxes (odd stride)
  // per warp, reused: two sets of trace / flux slots (surface phase: the next k-step's
  // neighbour traces arrive while this one's fluxes are formed), then the parked
  // accumulators of n-tiles 1..NT-1 (volume phase)
  static constexpr int SCR = 64 * FLS > 10 * (NT - 1) * 128 ? 64 * FLS : 10 * (NT - 1) * 128;
  static constexpr int WARP_FLOATS = 16 * S + 16 * GEO + ((SCR + 3) & ~3);
  static_assert(Np % 2 == 0, "node pairs of the SARK pass need an even Np");
  static_assert(NQ % 4 == 0, "element rows must be whole 16-byte chunks");
  static_assert(WARP_FLOATS % 4 == 0 && TAB_SETS % 4 == 0, "warp regions must start on 16-byte boundaries");
  static constexpr int MAX_WARPS = 8;       // warps per CTA
};

__device__ __forceinline__ void t3_cp16(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void t3_cp4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void t3_l2_prefetch(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// head = x rounded to 10 mantissa bits (ties away from zero), tail = x - head (exact)
__device__ __forceinline__ void t3_split(float x, unsigned &hi, unsigned &lo) {
  hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void t3_mma(float (&c)[4], const unsigned (&a)[4], float b0, float b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}

// c += (ahi + alo)(bhi + blo) without alo*blo; b = (blo0, blo1, bhi0, bhi1)
__device__ __forceinline__ void t3_mma3(float (&c)[4], const unsigned (&ah)[4], const unsigned (&al)[4], const float4 b) {
  t3_mma(c, al, b.z, b.w);
  t3_mma(c, ah, b.x, b.y);
  t3_mma(c, ah, b.z, b.w);
}

// shared-memory loads that stay where they are written: the volume phase is unrolled over
// the ten fields, and loads the compiler hoisted out of later fields' products would hold
// their registers over the whole phase (with the 10 x ceil(Np/8) accumulators live)
__device__ __forceinline__ float t3_lds(const float *p) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ float2 t3_lds2(const float *p) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

// A fragment (rows g, g + 8; columns col0 + t, col0 + t + 4) of a shared tile with row
// stride STRIDE; columns >= ncol read as zero
template <int STRIDE>
__device__ __forceinline__ void t3_lda(const float *tile, int col0, int ncol, int g, int t, unsigned (&hi)[4],
                                       unsigned (&lo)[4]) {
  const int c0 = col0 + t, c1 = c0 + 4;
  t3_split(c0 < ncol ? t3_lds(tile + g * STRIDE + c0) : 0.0f, hi[0], lo[0]);
  t3_split(c0 < ncol ? t3_lds(tile + (g + 8) * STRIDE + c0) : 0.0f, hi[1], lo[1]);
  t3_split(c1 < ncol ? t3_lds(tile + g * STRIDE + c1) : 0.0f, hi[2], lo[2]);
  t3_split(c1 < ncol ? t3_lds(tile + (g + 8) * STRIDE + c1) : 0.0f, hi[3], lo[3]);
}

// small read-only tables (node coordinates, face-node and neighbour-node indices), loaded
// where they are used: the tile loop would otherwise keep loop-invariant loads of them in
// registers across the whole tile
__device__ __forceinline__ float4 t3_ldg4(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ int t3_ldgi(const int *p) {
  int v;
  asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

// streaming state loads of the SARK pass, issued where they are written (five fields' worth
// at a time) rather than hoisted over the volume products
__device__ __forceinline__ float2 t3_ldcs2(const float *p) {
  float2 v;
  asm volatile("ld.global.cs.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// B fragment `set` of this lane from the shared operator table, split: (lo0, lo1, hi0, hi1).
// The address is formed next to the load by an opaque add: otherwise the tile loop keeps the
// addresses of all fragment sets, which do not change from tile to tile, in registers.
__device__ __forceinline__ float4 t3_ldb(const float *tabs, int set, int lane) {
  const unsigned base = (unsigned)__cvta_generic_to_shared(tabs) + 8u * (unsigned)lane;
  unsigned addr;
  asm volatile("add.u32 %0, %1, %2;" : "=r"(addr) : "r"(base), "r"(256u * (unsigned)set));
  float2 b;
  asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(b.x), "=f"(b.y) : "r"(addr));
  unsigned h0, l0, h1, l1;
  t3_split(b.x, h0, l0);
  t3_split(b.y, h1, l1);
  return make_float4(__uint_as_float(l0), __uint_as_float(l1), __uint_as_float(h0), __uint_as_float(h1));
}

__device__ __forceinline__ float2 t3_f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 t3_fma2(float a, float2 x, float2 y) { return __ffma2_rn(make_float2(a, a), x, y); }

// Upwind flux (Sec. 3, 3D) at face node j of tile row `row`: c/2 (|At_n| - At_n)(q+ - q-)
// + max(v_G . n, 0)(q+ - q-), times Fscale; |At_n| = al At_n^2 + be At_n^4 on the
// spectrum {0, +-1, +-sqrt3} of the unit-normal flux matrix.
// The neighbour traces q+ of this lane's four A-fragment slots (rows g, g + 8; face nodes
// 8 kf + t, 8 kf + t + 4) into its slot set, 10 fields each, by 4-byte cp.async (one group)
template <int N>
__device__ __forceinline__ void t3_fetch_traces(const float *qin, const float *geo, const int *tabi, int nel, int kf,
                                                int g, int t, float *slots) {
  typedef Tc3Dim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN, NQ = D::NQ, GEO = D::GEO;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int row = g + 8 * (s & 1), j = 8 * kf + t + 4 * (s >> 1);
    if (row < nel && j < NFN) {
      const int f = j / Nfp, k = j - (j / Nfp) * Nfp;
      const int nb = __float_as_int(geo[row * GEO + D::G_NBR + f]);
      const int64_t e2 = (int64_t)(nb >> 5);
      const int p = (nb >> 2) & 7, f2 = nb & 3;
      const int vol2 = t3_ldgi(tabi + D::TAB_NBR + ((f * 4 + f2) * 6 + p) * Nfp + k);
      const float *qp = qin + e2 * NQ + vol2;
#pragma unroll
      for (int fld = 0; fld < 10; ++fld) t3_cp4(slots + s * 10 + fld, qp + fld * Np);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void t3_flux(const float *own, const float *geo, const int *tabi, const float4 *bary4,
                                        int row, int j, float hc, const float *qplus, float (&out)[10]) {
  typedef Tc3Dim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, S = D::S, GEO = D::GEO;
  const float *gm = geo + row * GEO;
  const int f = j / Nfp, k = j - (j / Nfp) * Nfp;
  const int vol = t3_ldgi(tabi + D::TAB_FMASK + f * Nfp + k);
  const float *qm = own + row * S + vol;
  float w[10];
#pragma unroll
  for (int fld = 0; fld < 10; ++fld) w[fld] = qplus[fld] - qm[fld * Np];
  const float4 nf = *reinterpret_cast<const float4 *>(gm + D::G_FACE + 4 * f);   // nx ny nz Fscale
  const float4 vk = *reinterpret_cast<const float4 *>(gm + D::G_VN + 4 * f);
  const float4 bb = t3_ldg4(bary4 + vol);
  const float vn = bb.x * vk.x + bb.y * vk.y + bb.z * vk.z + bb.w * vk.w;
  const float ale = vn > 0.0f ? vn : 0.0f;
  const float ha = hc * (float)((9.0 - 1.7320508075688772935) / 6.0);
  const float hb = hc * (float)((1.7320508075688772935 - 3.0) / 6.0);
  float y[10], z[10], r[10];
  apply_An<float>(nf.x, nf.y, nf.z, w, y);
#pragma unroll
  for (int fld = 0; fld < 10; ++fld) r[fld] = __fmaf_rn(ale, w[fld], -hc * y[fld]);
  apply_An<float>(nf.x, nf.y, nf.z, y, z);
#pragma unroll
  for (int fld = 0; fld < 10; ++fld) r[fld] = __fmaf_rn(ha, z[fld], r[fld]);
  apply_An<float>(nf.x, nf.y, nf.z, z, y);
  apply_An<float>(nf.x, nf.y, nf.z, y, z);
#pragma unroll
  for (int fld = 0; fld < 10; ++fld) out[fld] = nf.w * __fmaf_rn(hb, z[fld], r[fld]);
}

template <int N, int STAGE>
__global__ void __launch_bounds__(32 * Tc3Dim<N>::MAX_WARPS) tc3_stage_kernel(const Stage3Args a) {
  typedef Tc3Dim<N> D;
  constexpr int Np = D::Np, NFN = D::NFN, NQ = D::NQ, KS = D::KS, NT = D::NT, KF = D::KF, CH = D::CH;
  constexpr int S = D::S, GEO = D::GEO;
  const float SQ2 = 1.41421356237309505f, ISQ2 = 0.70710678118654752f;
  extern __shared__ __align__(16) float t3_smem[];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int nwarps = blockDim.x >> 5;
  const int64_t ntiles = (a.K + 15) / 16;
  float *tabs = t3_smem;                       // the B-fragment sets
  float *own = t3_smem + D::TAB_SETS + warp * D::WARP_FLOATS;
  float *geo = own + 16 * S;
  float *park = geo + 16 * GEO;                // parked accumulators, [f][nt - 1][j][lane]
  float *fls = park + lane * D::FLS;           // this lane's trace / flux slots, set 0 (set 1: + 32 FLS)
  const float4 *bary4 = reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.ops_tc) + D::TAB_BARY);
  const int *tabi = reinterpret_cast<const int *>(a.ops_tc);
  const float *qin = reinterpret_cast<const float *>(a.qin);
  // the operator table into shared memory, once per CTA
  {
    const float4 *src = reinterpret_cast<const float4 *>(a.ops_tc);
    float4 *dst = reinterpret_cast<float4 *>(tabs);
    for (int i = threadIdx.x; i < D::TAB_SETS / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  // stage motion factors (FP64), once per CTA
  __shared__ double s_motion[4];
  if (threadIdx.x == 0) {
    const Motion3 m = stage_motion3(a, STAGE);
    s_motion[0] = m.g1;
    s_motion[1] = m.g2;
    s_motion[2] = m.x1;
    s_motion[3] = m.x2;
    if (STAGE == 3 && blockIdx.x == 0) {
      // final vertex update factors dt sum_j b_j (cos, sin)(omega t_j)
      double f1 = 0.0, f2 = 0.0;
      if (a.moving) {
        const double t0 = a.clock[0], dt = a.dt, w = a.omega;
        f1 = dt * (cos(w * t0) / 6.0 + cos(w * (t0 + 0.5 * dt)) * (2.0 / 3.0) + cos(w * (t0 + dt)) / 6.0);
        f2 = dt * (sin(w * t0) / 6.0 + sin(w * (t0 + 0.5 * dt)) * (2.0 / 3.0) + sin(w * (t0 + dt)) / 6.0);
      }
      a.clock[1] = f1;
      a.clock[2] = f2;
    }
  }
  bool bad = false;
  __syncthreads();

  // one tile per warp (a loop over tiles here kept the loop-invariant table addresses and
  // loads of every phase live across the whole tile, past the 255 registers)
  const int64_t tile = (int64_t)blockIdx.x * nwarps + warp;
  if (tile < ntiles) {
  const int64_t e0 = tile * 16;
  const int nel = (int)((a.K - e0) < 16 ? (a.K - e0) : 16);

  // ---- 1. the tile's fields (contiguous rows of NQ floats) into the padded shared tile ----
  {
    const float *src = qin + e0 * NQ;
    if ((reinterpret_cast<uintptr_t>(qin) & 15) == 0) {
      constexpr int C = NQ / 4;
      for (int i = lane; i < nel * C; i += 32) {
        const int e = i / C, c4 = i - (i / C) * C;
        t3_cp16(own + e * S + 4 * c4, src + (int64_t)e * NQ + 4 * c4);
      }
    } else {
      for (int i = lane; i < nel * NQ; i += 32) {
        const int e = i / NQ, c1 = i - (i / NQ) * NQ;
        t3_cp4(own + e * S + c1, src + (int64_t)e * NQ + c1);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // geometry, one element per lane 0..15, while the copies fly
  if (lane < 16) {
    float *gm = geo + lane * GEO;
    if (lane < nel) {
      float gt[GEO3];
      element_geometry3<float>(a, e0 + lane, s_motion[2], s_motion[3], s_motion[0], s_motion[1], gt);
      const int4 nb = *reinterpret_cast<const int4 *>(a.mesh[e0 + lane].nbr);
#pragma unroll
      for (int i = 0; i < 9; ++i) gm[i] = gt[i];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float nx = gt[GEO3_F + 4 * f], ny = gt[GEO3_F + 1 + 4 * f], nz = gt[GEO3_F + 2 + 4 * f];
        gm[D::G_FACE + 4 * f] = nx;
        gm[D::G_FACE + 1 + 4 * f] = ny;
        gm[D::G_FACE + 2 + 4 * f] = nz;
        gm[D::G_FACE + 3 + 4 * f] = gt[GEO3_F + 3 + 4 * f];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          gm[D::G_VN + 4 * f + k] = gt[GEO3_V + 3 * k] * nx + gt[GEO3_V + 3 * k + 1] * ny + gt[GEO3_V + 3 * k + 2] * nz;
      }
      gm[D::G_NBR] = __int_as_float(nb.x);
      gm[D::G_NBR + 1] = __int_as_float(nb.y);
      gm[D::G_NBR + 2] = __int_as_float(nb.z);
      gm[D::G_NBR + 3] = __int_as_float(nb.w);
#pragma unroll
      for (int ra = 0; ra < 3; ++ra)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          gm[D::G_VTIL + 4 * ra + k] = gt[3 * ra] * gt[GEO3_V + 3 * k] + gt[3 * ra + 1] * gt[GEO3_V + 3 * k + 1] +
                                       gt[3 * ra + 2] * gt[GEO3_V + 3 * k + 2];
    } else {
      for (int i = 0; i < GEO; ++i) gm[i] = 0.0f;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  // ---- 2. the neighbour traces of the first face-node k-step, in flight during the cubature ----
  t3_fetch_traces<N>(qin, geo, tabi, nel, 0, g, t, fls);

  // accumulators of the right-hand side: acc[field][n-tile][fragment]
  float acc[10][NT][4];
#pragma unroll
  for (int f = 0; f < 10; ++f)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[f][nt][j] = 0.0f;

  // ---- 3. collision term: I q at the cubature points, Ntilde there, P back (fields 5..10) ----
  {
    const float itau = (float)a.inv_tau;
#pragma unroll 2
    for (int ch = 0; ch < CH; ++ch) {
      float qc[4][4];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int j = 0; j < 4; ++j) qc[f][j] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const float4 b = t3_ldb(tabs, D::B_I + ch * KS + ks, lane);
        unsigned ah[4][4], al[4][4];
#pragma unroll
        for (int f = 0; f < 4; ++f) t3_lda<S>(own, f * Np + ks * 8, f * Np + Np, g, t, ah[f], al[f]);
#pragma unroll
        for (int f = 0; f < 4; ++f) t3_mma(qc[f], al[f], b.z, b.w);
#pragma unroll
        for (int f = 0; f < 4; ++f) t3_mma(qc[f], ah[f], b.x, b.y);
#pragma unroll
        for (int f = 0; f < 4; ++f) t3_mma(qc[f], ah[f], b.z, b.w);
      }
      // Ntilde in A-fragment slot order: slot s takes accumulator entry (0, 2, 1, 3)[s]
      float nv[6][4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int j = s == 0 ? 0 : (s == 1 ? 2 : (s == 2 ? 1 : 3));
        const float q1 = 1.0f + qc[0][j], q2 = qc[1][j], q3 = qc[2][j], q4 = qc[3][j];
        const float r1 = itau * __frcp_rn(q1), rs = r1 * ISQ2;
        nv[0][s] = q2 * q3 * r1;
        nv[1][s] = q2 * q4 * r1;
        nv[2][s] = q3 * q4 * r1;
        nv[3][s] = q2 * q2 * rs;
        nv[4][s] = q3 * q3 * rs;
        nv[5][s] = q4 * q4 * rs;
      }
      float4 bp[NT];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) bp[nt] = t3_ldb(tabs, D::B_P + ch * NT + nt, lane);
#pragma unroll
      for (int k6 = 0; k6 < 6; ++k6) {
        unsigned nh[4], nl[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) t3_split(nv[k6][s], nh[s], nl[s]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) t3_mma3(acc[4 + k6][nt], nh, nl, bp[nt]);
      }
    }
  }

  if (STAGE >= 1 && lane == 0) {   // the SARK pass's inputs of this tile, towards L2
    const unsigned bytes = (unsigned)(nel * NQ * sizeof(float));
    t3_l2_prefetch(reinterpret_cast<const float *>(a.qn) + e0 * NQ, bytes);
    if (STAGE <= 2) t3_l2_prefetch(reinterpret_cast<const float *>(a.F0) + e0 * NQ, bytes);
    if (STAGE >= 2) t3_l2_prefetch(reinterpret_cast<const float *>(a.acc) + e0 * NQ, bytes);
  }

  // ---- 4. surface: fluxes at this lane's A-fragment slots, lifted k-step by k-step ----
  {
    const float hc = 0.5f * (float)a.c;
#pragma unroll 1
    for (int kf = 0; kf < KF; ++kf) {
      float *cur_slots = fls + (kf & 1) * 32 * D::FLS;
      if (kf + 1 < KF) {   // the next k-step's traces into the other slot set
        t3_fetch_traces<N>(qin, geo, tabi, nel, kf + 1, g, t, fls + ((kf + 1) & 1) * 32 * D::FLS);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      }
      // one item at a time (the accumulators leave no room for four items' temporaries in
      // registers): its traces are read from its slots and its fluxes written over them
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        const int row = g + 8 * (s & 1), j = 8 * kf + t + 4 * (s >> 1);
        float *slot = cur_slots + s * 10;
        float fl[10];
        if (row < nel && j < NFN) {
          t3_flux<N>(own, geo, tabi, bary4, row, j, hc, slot, fl);
        } else {
#pragma unroll
          for (int fld = 0; fld < 10; ++fld) fl[fld] = 0.0f;
        }
#pragma unroll
        for (int fld = 0; fld < 10; ++fld) slot[fld] = fl[fld];
      }
      float4 bl[NT];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) bl[nt] = t3_ldb(tabs, D::B_LIFT + kf * NT + nt, lane);
#pragma unroll
      for (int f = 0; f < 10; ++f) {
        unsigned ah[4], al[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) t3_split(cur_slots[s * 10 + f], ah[s], al[s]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) t3_mma3(acc[f][nt], ah, al, bl[nt]);
      }
    }
  }

  // ---- 5. park the accumulators of n-tiles 1.. in this lane's slots (fragment order; the
  //      flux slots are free now), so that the volume phase holds one n-tile at a time ----
  __syncwarp();
#pragma unroll
  for (int f = 0; f < 10; ++f)
#pragma unroll
    for (int nt = 1; nt < NT; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) park[((f * (NT - 1) + nt - 1) * 4 + j) * 32 + lane] = acc[f][nt][j];

  // ---- 6. per n-tile: volume (v_G . grad q_f and -c Atilde . grad q, Sec. 2), then the SARK
  //      stage / final combination (fields 1..4 RK4, 5..10 exponential) on its node pairs ----
  const float mc = -(float)a.c, mcs = -(float)a.c * SQ2;
  float gi[2][9];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int i = 0; i < 9; ++i) gi[h][i] = geo[(g + 8 * h) * GEO + i];
  // SARK coefficients of this stage for the two field classes
  float kE[2], kA0[2], kA1[2], kB0[2], kB1[2];
#pragma unroll
  for (int cl = 0; cl < 2; ++cl) {
    kE[cl] = (float)a.co.E[cl][STAGE < 0 ? 0 : (STAGE < 3 ? STAGE + 1 : 4)];
    kA0[cl] = (float)(STAGE == 0 ? a.co.A[cl][4] : STAGE == 1 ? a.co.A[cl][8] : STAGE == 2 ? a.co.A[cl][12] : 0.0);
    kA1[cl] = (float)(STAGE == 1 ? a.co.A[cl][9] : STAGE == 2 ? a.co.A[cl][14] : 0.0);
    kB0[cl] = (float)(STAGE == 1 ? a.co.B[cl][0] : STAGE == 2 ? a.co.B[cl][2] : STAGE == 3 ? a.co.B[cl][3] : 0.0);
    kB1[cl] = (float)a.co.B[cl][1];
  }
  const float dtf = (float)a.dt;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    float cur[10][4];
#pragma unroll
    for (int f = 0; f < 10; ++f)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        cur[f][j] = nt == 0 ? acc[f][0][j] : t3_lds(park + ((f * (NT - 1) + nt - 1) * 4 + j) * 32 + lane);
    // the grid velocity in reference coordinates, vt_a = (G^-1 v_G)_a, at this thread's node
    // pairs: sum over the vertices of the barycentric weights times (G^-1 v_k)_a
    float2 vtr[2][3];
    {
      const int n0 = nt * 8 + 2 * t;
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 b0 = n0 < Np ? t3_ldg4(bary4 + n0) : z4, b1 = n0 + 1 < Np ? t3_ldg4(bary4 + n0 + 1) : z4;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int ra = 0; ra < 3; ++ra) {
          const float4 v = *reinterpret_cast<const float4 *>(geo + (g + 8 * h) * GEO + D::G_VTIL + 4 * ra);
          vtr[h][ra] = make_float2(b0.x * v.x + b0.y * v.y + b0.z * v.z + b0.w * v.w,
                                   b1.x * v.x + b1.y * v.y + b1.z * v.z + b1.w * v.w);
        }
    }
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      float d[3][4];
#pragma unroll
      for (int ra = 0; ra < 3; ++ra)
#pragma unroll
        for (int j = 0; j < 4; ++j) d[ra][j] = 0.0f;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        unsigned ah[4], al[4];
        t3_lda<S>(own, f * Np + ks * 8, f * Np + Np, g, t, ah, al);
        float4 b[3];
#pragma unroll
        for (int ra = 0; ra < 3; ++ra) b[ra] = t3_ldb(tabs, D::B_VOL + (ra * KS + ks) * NT + nt, lane);
#pragma unroll
        for (int ra = 0; ra < 3; ++ra) t3_mma(d[ra], al, b[ra].z, b[ra].w);
#pragma unroll
        for (int ra = 0; ra < 3; ++ra) t3_mma(d[ra], ah, b[ra].x, b[ra].y);
#pragma unroll
        for (int ra = 0; ra < 3; ++ra) t3_mma(d[ra], ah, b[ra].z, b[ra].w);
      }
      // pointwise on the node pair (2t, 2t + 1) of rows g and g + 8
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j0 = 2 * h;
        const float2 dr = t3_f2(d[0][j0], d[0][j0 + 1]), ds = t3_f2(d[1][j0], d[1][j0 + 1]),
                     dq = t3_f2(d[2][j0], d[2][j0 + 1]);
        const float2 wr = vtr[h][0], ws = vtr[h][1], wt = vtr[h][2];
        const float2 ale = __ffma2_rn(wt, dq, __ffma2_rn(ws, ds, __fmul2_rn(wr, dr)));
        const float *G = gi[h];
        // physical derivative d/dx_dd of field f at the pair
        auto PD = [&](int dd) { return t3_fma2(G[6 + dd], dq, t3_fma2(G[3 + dd], ds, __fmul2_rn(make_float2(G[dd], G[dd]), dr))); };
        auto A = [&](int ff) { return t3_f2(cur[ff][j0], cur[ff][j0 + 1]); };
        auto P = [&](int ff, float2 v) { cur[ff][j0] = v.x; cur[ff][j0 + 1] = v.y; };
        P(f, __fadd2_rn(A(f), ale));
        switch (f) {
          case 0: { const float2 qx = PD(0), qy = PD(1), qz = PD(2);
                    P(1, t3_fma2(mc, qx, A(1))); P(2, t3_fma2(mc, qy, A(2))); P(3, t3_fma2(mc, qz, A(3))); break; }
          case 1: { const float2 qx = PD(0), qy = PD(1), qz = PD(2);
                    P(0, t3_fma2(mc, qx, A(0))); P(4, t3_fma2(mc, qy, A(4))); P(5, t3_fma2(mc, qz, A(5)));
                    P(7, t3_fma2(mcs, qx, A(7))); break; }
          case 2: { const float2 qx = PD(0), qy = PD(1), qz = PD(2);
                    P(0, t3_fma2(mc, qy, A(0))); P(4, t3_fma2(mc, qx, A(4))); P(6, t3_fma2(mc, qz, A(6)));
                    P(8, t3_fma2(mcs, qy, A(8))); break; }
          case 3: { const float2 qx = PD(0), qy = PD(1), qz = PD(2);
                    P(0, t3_fma2(mc, qz, A(0))); P(5, t3_fma2(mc, qx, A(5))); P(6, t3_fma2(mc, qy, A(6)));
                    P(9, t3_fma2(mcs, qz, A(9))); break; }
          case 4: { const float2 qx = PD(0), qy = PD(1);
                    P(1, t3_fma2(mc, qy, A(1))); P(2, t3_fma2(mc, qx, A(2))); break; }
          case 5: { const float2 qx = PD(0), qz = PD(2);
                    P(1, t3_fma2(mc, qz, A(1))); P(3, t3_fma2(mc, qx, A(3))); break; }
          case 6: { const float2 qy = PD(1), qz = PD(2);
                    P(2, t3_fma2(mc, qz, A(2))); P(3, t3_fma2(mc, qy, A(3))); break; }
          case 7: P(1, t3_fma2(mcs, PD(0), A(1))); break;
          case 8: P(2, t3_fma2(mcs, PD(1), A(2))); break;
          default: P(3, t3_fma2(mcs, PD(2), A(3))); break;
        }
      }
    }
    // SARK on this n-tile's node pairs, five fields at a time: every load before any store
    // (q_{n+1} overwrites q_n in place at the last stage)
#pragma unroll
    for (int f0 = 0; f0 < 10; f0 += 5) {
      float2 xv[5][2], x0[5][2], xa[5][2];
#pragma unroll
      for (int ff = 0; ff < 5; ++ff)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int f = f0 + ff, row = g + 8 * h, n0 = nt * 8 + 2 * t;
          xv[ff][h] = x0[ff][h] = xa[ff][h] = make_float2(0.f, 0.f);
          if (STAGE >= 0 && row < nel && n0 < Np) {
            const int64_t idx = (e0 + row) * NQ + f * Np + n0;
            xv[ff][h] = STAGE == 0 ? t3_lds2(own + row * S + f * Np + n0)
                                   : t3_ldcs2(reinterpret_cast<const float *>(a.qn) + idx);
            if (STAGE == 1 || STAGE == 2)
              x0[ff][h] = t3_ldcs2(reinterpret_cast<const float *>(a.F0) + idx);
            if (STAGE >= 2) xa[ff][h] = t3_ldcs2(reinterpret_cast<const float *>(a.acc) + idx);
          }
        }
#pragma unroll
      for (int ff = 0; ff < 5; ++ff)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int f = f0 + ff, cl = f < 4 ? 0 : 1, row = g + 8 * h, n0 = nt * 8 + 2 * t;
          if (!(row < nel && n0 < Np)) continue;
          const int64_t idx = (e0 + row) * NQ + f * Np + n0;
          const float2 r = t3_f2(cur[f][2 * h], cur[f][2 * h + 1]);
          if (STAGE < 0) {
            *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.Fout) + idx) = r;
            continue;
          }
          const float2 dt2 = make_float2(dtf, dtf), qv = xv[ff][h], p0 = x0[ff][h], pa = xa[ff][h];
          float2 o;
          if (STAGE == 0) {
            *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.F0) + idx) = r;
            o = t3_fma2(kE[cl], qv, __fmul2_rn(dt2, __fmul2_rn(make_float2(kA0[cl], kA0[cl]), r)));
          } else if (STAGE == 1 || STAGE == 2) {
            const float2 sa = t3_fma2(kA0[cl], p0, __fmul2_rn(make_float2(kA1[cl], kA1[cl]), r));
            o = t3_fma2(kE[cl], qv, __fmul2_rn(dt2, sa));
            *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.acc) + idx) =
                STAGE == 1 ? t3_fma2(kB0[cl], p0, __fmul2_rn(make_float2(kB1[cl], kB1[cl]), r)) : t3_fma2(kB0[cl], r, pa);
          } else {
            o = t3_fma2(kE[cl], qv, __fmul2_rn(dt2, t3_fma2(kB0[cl], r, pa)));
            bad |= bad3(o.x) || bad3(o.y);
          }
          *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.qout) + idx) = o;
        }
    }
  }
  }   // tile
  if (STAGE == 3 && bad) atomicOr(a.status, GB_STATUS_NAN);
}

// ---------------------------------------------------------------------------
// launch: CTAs of W warps, one 16-element tile per warp, the operator table in each CTA's
// shared memory

bool stage3_tc_supported(int N) { return N >= 1 && N <= 3; }

template <int N>
static size_t tc3_smem(int W) {
  return sizeof(float) * ((size_t)Tc3Dim<N>::TAB_SETS + (size_t)W * Tc3Dim<N>::WARP_FLOATS);
}

int stage3_tc_max_warps(int N) {
  auto fit = [](size_t per_warp, size_t table, int cap) {
    int w = cap;
    while (w > 1 && table + (size_t)w * per_warp > (size_t)227 * 1024) --w;
    return w;
  };
  switch (N) {
    case 1: return fit(sizeof(float) * Tc3Dim<1>::WARP_FLOATS, sizeof(float) * Tc3Dim<1>::TAB_SETS, Tc3Dim<1>::MAX_WARPS);
    case 2: return fit(sizeof(float) * Tc3Dim<2>::WARP_FLOATS, sizeof(float) * Tc3Dim<2>::TAB_SETS, Tc3Dim<2>::MAX_WARPS);
    case 3: return fit(sizeof(float) * Tc3Dim<3>::WARP_FLOATS, sizeof(float) * Tc3Dim<3>::TAB_SETS, Tc3Dim<3>::MAX_WARPS);
  }
  return 0;
}

template <int N, int STAGE>
static int launch_tc3_one(const Stage3Args &a, cudaStream_t st, int W, int num_sms) {
  const size_t smem = tc3_smem<N>(W);
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return (int)err;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  // per device: the shared-memory opt-in (the largest so far)
  static std::atomic<int> opted[64];
  if ((int)smem > opted[dev].load(std::memory_order_relaxed)) {
    err = cudaFuncSetAttribute(tc3_stage_kernel<N, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    int prev = opted[dev].load(std::memory_order_relaxed);
    while ((int)smem > prev && !opted[dev].compare_exchange_weak(prev, (int)smem)) {
    }
  }
  (void)num_sms;
  const int64_t ntiles = (a.K + 15) / 16;
  const int64_t grid = (ntiles + W - 1) / W;
  if (grid < 1) return 0;
  tc3_stage_kernel<N, STAGE><<<(unsigned)grid, 32 * W, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <int N>
static int launch_tc3_n(const Stage3Args &a, cudaStream_t st, int W, int num_sms) {
  switch (a.stage) {
    case -1: return launch_tc3_one<N, -1>(a, st, W, num_sms);
    case 0: return launch_tc3_one<N, 0>(a, st, W, num_sms);
    case 1: return launch_tc3_one<N, 1>(a, st, W, num_sms);
    case 2: return launch_tc3_one<N, 2>(a, st, W, num_sms);
    case 3: return launch_tc3_one<N, 3>(a, st, W, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_stage3_tc(int N, const Stage3Args &a, void *stream, int warps_per_cta, int num_sms) {
  if (warps_per_cta < 1 || warps_per_cta > stage3_tc_max_warps(N)) return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  switch (N) {
    case 1: return launch_tc3_n<1>(a, st, warps_per_cta, num_sms);
    case 2: return launch_tc3_n<2>(a, st, warps_per_cta, num_sms);
    case 3: return launch_tc3_n<3>(a, st, warps_per_cta, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

// ---- operator table: B fragments per lane (FP32), then the node tables ----

template <int N>
static void fill_tc3(const RefOps3 &R, std::vector<float> &h) {
  typedef Tc3Dim<N> D;
  const int Np = D::Np, NFN = D::NFN, Nc = D::Nc, Nfp = D::Nfp;
  h.assign((size_t)D::TAB_WORDS, 0.0f);
  // fragment of the K x N operand B(k, n): lane (g, t) holds B(t, g) and B(t + 4, g), in FP32
  // (the kernel splits each value into its TF32 head and tail)
  auto put = [&](int set, auto B) {
    for (int lane = 0; lane < 32; ++lane) {
      const int gq = lane >> 2, tq = lane & 3;
      float *o = &h[((size_t)set * 32 + lane) * 2];
      o[0] = (float)B(tq, gq);
      o[1] = (float)B(tq + 4, gq);
    }
  };
  const std::vector<double> *Dop[3] = {&R.Dr, &R.Ds, &R.Dt};
  for (int ra = 0; ra < 3; ++ra)
    for (int ks = 0; ks < D::KS; ++ks)
      for (int nt = 0; nt < D::NT; ++nt)
        put(D::B_VOL + (ra * D::KS + ks) * D::NT + nt, [&](int k, int n) {
          const int m = ks * 8 + k, o = nt * 8 + n;
          return (m < Np && o < Np) ? (*Dop[ra])[o * Np + m] : 0.0;
        });
  for (int kf = 0; kf < D::KF; ++kf)
    for (int nt = 0; nt < D::NT; ++nt)
      put(D::B_LIFT + kf * D::NT + nt, [&](int k, int n) {
        const int j = kf * 8 + k, o = nt * 8 + n;
        return (j < NFN && o < Np) ? R.LIFT[o * NFN + j] : 0.0;
      });
  for (int ch = 0; ch < D::CH; ++ch)
    for (int ks = 0; ks < D::KS; ++ks)
      put(D::B_I + ch * D::KS + ks, [&](int k, int n) {
        const int m = ks * 8 + k, cp = ch * 8 + n;
        return (m < Np && cp < Nc) ? R.I[cp * Np + m] : 0.0;
      });
  for (int ch = 0; ch < D::CH; ++ch)
    for (int nt = 0; nt < D::NT; ++nt)
      put(D::B_P + ch * D::NT + nt, [&](int k, int n) {
        // k < 4 is the chunk's point 2k, k >= 4 its point 2(k - 4) + 1 (accumulator reuse)
        const int cp = ch * 8 + (k < 4 ? 2 * k : 2 * (k - 4) + 1), o = nt * 8 + n;
        return (cp < Nc && o < Np) ? R.P[o * Nc + cp] : 0.0;
      });
  for (int n = 0; n < Np; ++n)
    for (int v = 0; v < 4; ++v) h[D::TAB_BARY + 4 * n + v] = (float)R.bary[n * 4 + v];
  int *hi = reinterpret_cast<int *>(h.data());
  for (int i = 0; i < 4 * Nfp; ++i) hi[D::TAB_FMASK + i] = R.fmask[i];
  for (int i = 0; i < 96 * Nfp; ++i) hi[D::TAB_NBR + i] = R.nbr_node[i];
}

int upload_ops3_tc(int N, const RefOps3 &R, void **dev, size_t *bytes, void *stream) {
  if ((int)R.fmask.size() != 4 * R.Nfp || (int)R.nbr_node.size() != 96 * R.Nfp) return (int)cudaErrorInvalidValue;
  std::vector<float> h;
  switch (N) {
    case 1: fill_tc3<1>(R, h); break;
    case 2: fill_tc3<2>(R, h); break;
    case 3: fill_tc3<3>(R, h); break;
    default: return (int)cudaErrorInvalidValue;
  }
  cudaError_t err = cudaMalloc(dev, h.size() * sizeof(float));
  if (err != cudaSuccess) return (int)err;
  err = cudaMemcpyAsync(*dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
  if (err != cudaSuccess) {
    cudaFree(*dev);
    *dev = nullptr;
    return (int)err;
  }
  *bytes = h.size() * sizeof(float);
  return 0;
}

}  // namespace gb
