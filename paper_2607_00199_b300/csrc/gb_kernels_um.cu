// GB_MIXED stage kernel on the fifth-generation tensor cores (tcgen05) with the
// accumulators in tensor memory (TMEM).
//
// Same right-hand side and SARK combination as the other stage kernels (Secs. 2-5):
// F = volume + surface + P Ntilde(I q) at the stage geometry, then the stage or final
// SARK combination.  The work is laid out by element tiles:
//
//   a CTA (one per SM, persistent) owns tiles of 128 consecutive (Morton-ordered)
//   elements in turn; element e of a tile is TMEM lane e, and two compute threads
//   (t and t + 128) share its pointwise work; four helper warps form the next tile's
//   geometry and halo, issue the interpolation and projection products and the bulk copies.
//
// The four dense contractions of the semi-discrete form (Sec. 3) are M = 128 (elements)
// tcgen05.mma products of kind::tf32, each accumulator fed by one lane, accumulating in
// FP32 in TMEM:
//   V_f  = Q_f [Dr | Ds]^T      (f = 1..6; A = the field's nodal values)
//   C_f  = Q_f I^T              (f = 1..3; the values at the cubature points)
//   R_f += Ntilde_f P^T         (f = 4..6; the projected collision term)
//   R_f += Flux_f LIFT^T        (f = 1..6; the lifted face fluxes)
// Each operand is split into a TF32 head rounded to nearest and its FP32 tail (x = hi + lo),
// and every product is formed as hi*hi + hi*lo + lo*hi; the tail is truncated to TF32 by
// the tensor core, so a product carries ~2^-21 relative error (the operator tables are split
// on the host the same way, from FP64).  The tails of the field tile sit in shared memory in
// the K-major core-matrix layout (one of the three products reads them there); every other
// A operand (the field heads, Ntilde, the fluxes) is written by its element's threads
// straight into its TMEM lane with tcgen05.st.
//
// The pointwise work runs per element with the element's values in registers: the
// geometric factors from the FP64 stage vertices (Sec. 5: FP64 positions and edge
// differences, FP32 afterwards, as in the other mixed kernel), the chain rule with the
// Atilde couplings and the v_G . grad q advection (Sec. 2), Ntilde at the cubature points,
// the upwind face fluxes F_S and F_ALE (Sec. 3) with the neighbour traces read from the
// staged tile (neighbours inside the tile), from the halo the helpers staged (the tile's
// out-of-tile faces) or, past the halo's capacity, from global memory, and the SARK
// combination of the element's row.
//
// Data movement per tile is bulk copies with completion on mbarriers: the tile's own fields
// q_i arrive while the previous tile finishes (prefetched once its fluxes are formed), F_0 and
// the accumulator are loaded at the start of the tile, q_n once the volume and interpolation
// products have read the tail tile; the SARK outputs are written into those staged rows and
// leave as bulk stores.  Four MMA batches per tile (volume, then interpolation, projection,
// lift), each committed to an mbarrier.  Every wait is bounded: on expiry the kernel sets
// GB_STATUS_TIMEOUT, waits (bounded) for what it issued, frees its TMEM and returns.
//
// Field layout: the element-major FP32 perturbation layout of the GB_MIXED path (element
// stride S = 4 mod 8 floats, fields of Np values), unchanged.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "gb_internal.h"

namespace gb {

template <int N>
struct UmDim {
  static constexpr int Np = (N + 1) * (N + 2) / 2;
  static constexpr int Nfp = N + 1;
  static constexpr int NFN = 3 * (N + 1);
  static constexpr int Nc = ((3 * N + 2) / 2) * ((3 * N + 2) / 2);
  static constexpr int S = tc_round_s(6 * Np);   // element stride of the field layout (floats)
  static constexpr int S4 = S / 4;               // 16-byte chunks per element row
  static constexpr int NPP = (Np + 3) & ~3;      // field column stride of the tail tile in shared memory
  static constexpr int KV = (Np + 7) & ~7;       // K of the Dr/Ds and I products; field stride of the TMEM heads
  static constexpr int CA = (6 * NPP + (KV - NPP) + 3) & ~3;   // tail-tile columns (the last field's K overrun included)
  static constexpr int NV = (2 * KV + 15) & ~15; // N of the volume product: Dr rows at 0, Ds rows at KV
  static constexpr int NCM = (Nc + 15) & ~15;    // N of the interpolation product
  static constexpr int KC = (Nc + 7) & ~7;       // K of the projection product
  static constexpr int NR = 16;                  // N of the projection and lift products (Np <= 15)
  static constexpr int KL = (NFN + 7) & ~7;      // K of the lift product
  static constexpr int NVC = NV + NCM;           // rows of the [Dr | Ds | I] table; TMEM columns of fields 1..3
  // operator tables (floats), each as its TF32 head then its tail, core-matrix K-major layout:
  // entry (n, k) of an R x K table at (k / 4) (4 R) + 4 n + k % 4.  BV: the rows of Dr (at 0),
  // Ds (at KV) and I (at NV), NVC x KV; the volume products read its first NV rows, the
  // interpolation products the NCM rows from NV
  static constexpr int BV = 0;
  static constexpr int BP = BV + 2 * NVC * KV;
  static constexpr int BL = BP + 2 * NR * KC;
  static constexpr int BBAR = BL + 2 * NR * KL;  // per node ((1 + r) / 2, (1 + s) / 2)
  static constexpr int BTOT = BBAR + 2 * 16;
  // dynamic shared memory (floats): q_n then q_{i+1} [128 x S], own fields [128 x S], F_0 and
  // the accumulator [128 x SAW each: rows of S, or the field-tail tile of 128 x CA in the one
  // that the stage leaves free], tables, geometry [128 x GW], halo of the out-of-tile
  // neighbour traces [HMAX x HW]
  static constexpr int SAW = CA > S ? CA : S;
  static constexpr int SM_A = 0;
  static constexpr int SM_RAW = SM_A + 128 * S;
  static constexpr int SM_X1 = SM_RAW + 128 * S;
  static constexpr int SM_X2 = SM_X1 + 128 * SAW;
  static constexpr int SM_B = SM_X2 + 128 * SAW;
  static constexpr int SM_G = SM_B + BTOT;         // per element geometry of a tile [128][GW]
  static constexpr int GW = 20;                    // rx sx ry sy 1/J, edges x3 y3, vertex velocities x3 y3, neighbours 3
  static constexpr int HMAX = 48;                  // halo entries: out-of-tile faces of a tile
  static constexpr int HW = 6 * Nfp;               // floats per halo entry (face node k, field fld at 6 k + fld)
  static constexpr int SM_H = SM_G + 128 * GW;
  static constexpr int SM_END = SM_H + HMAX * HW;
  // TMEM columns (512 allocated), per field f (see um_tv and the functions after it):
  //   [0, 96)        field heads (KV columns per field); later Ntilde tails and flux tails
  //   from T_V0      fields 1..3: [Vr | Vs | C] (NVC columns), then fields 4..6: [Vr | Vs] (NV);
  //                  R_f takes the Vr columns of field f once they are read, the Ntilde heads
  //                  replace C in place, and at N >= 3 the flux heads take the Vs columns
  //   from T_END     free: Ntilde tails where they fit (N <= 3), flux heads at N <= 2
  static constexpr uint32_t T_QH = 0, T_V0 = 96;
  static constexpr uint32_t T_END = T_V0 + 3 * NVC + 3 * NV;
  static constexpr int NCH = KC / 8, HALF = (NCH + 1) / 2;        // cubature chunks; those of thread half 0
  static constexpr bool SLOTS_FREE = (512 - (int)T_END) / 8 >= 3 * NCH;
  static constexpr int NQL = 6 * KV / 8;                          // 8-column slots over the field heads
  static_assert(N >= 1 && N <= 4, "the tcgen05 kernel covers orders 1..4");
  static_assert(6 * KV <= 96 && 6 * KL <= 96 && T_END <= 512 && KC <= NCM && NVC <= 256, "TMEM map");
  static_assert(NV == 32 ? (Np > 8 && KL <= KV) : T_END + 6 * KL <= 512, "flux heads");
  static_assert(SLOTS_FREE || (NV == 32 && 3 * HALF <= 6 + NQL / 2 && 3 * (NCH - HALF) <= 6 + (NQL - NQL / 2)),
                "Ntilde tail slots");
};

// TMEM column of the volume products of field f (Vr at +0, Vs at +KV; C at +NV for f < 3)
template <int N>
__host__ __device__ constexpr uint32_t um_tv(int f) {
  typedef UmDim<N> D;
  return f < 3 ? D::T_V0 + f * D::NVC : D::T_V0 + 3 * D::NVC + (f - 3) * D::NV;
}
template <int N>
__host__ __device__ constexpr uint32_t um_tc(int f) { return um_tv<N>(f) + UmDim<N>::NV; }   // f < 3
template <int N>
__host__ __device__ constexpr uint32_t um_tr(int f) { return um_tv<N>(f); }                  // R_f, 16 columns
template <int N>
__host__ __device__ constexpr uint32_t um_tfl(int f) { return UmDim<N>::T_QH + f * UmDim<N>::KL; }
template <int N>
__host__ __device__ constexpr uint32_t um_tfh(int f) {
  typedef UmDim<N> D;
  return D::NV == 32 ? um_tv<N>(f) + D::KV : D::T_END + f * D::KL;
}

// 8-column TMEM slot of the Ntilde tails of field f, cubature chunk ks.  Where there is room
// past the products they go there.  Otherwise chunk ks, formed by thread half h = (ks >= HALF),
// goes first to the Vs columns of nodes [8h, 8h + 8) of a field (read by the same half
// itself), then to a half of the field-head columns (free once the first MMA batch is
// complete).  So no thread overwrites columns that the other thread of its element may still
// have to read.
template <int N>
__host__ __device__ constexpr uint32_t um_nslot(int f, int ks) {
  typedef UmDim<N> D;
  if (D::SLOTS_FREE) return D::T_END + 8 * (f * D::NCH + ks);
  const int h = ks >= D::HALF ? 1 : 0;
  const int i = f * (h ? D::NCH - D::HALF : D::HALF) + (ks - (h ? D::HALF : 0));
  if (i < 6) return um_tv<N>(i) + D::KV + 8 * h;
  return D::T_QH + 8 * ((h ? D::NQL / 2 : 0) + (i - 6));
}

// ---- PTX wrappers -----------------------------------------------------------------
__device__ __forceinline__ uint32_t um_sa(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, K-major without swizzle: a core matrix is 8 rows x 16
// bytes stored as 128 contiguous bytes; lbo = byte distance between core matrices adjacent
// in K, sbo = between core matrices adjacent in M (or N); bit 46 = descriptor version
__device__ __forceinline__ uint64_t um_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major, M = 128
__host__ __device__ constexpr uint32_t um_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void um_mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void um_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
               :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
// the same, issued by the calling thread only where `issue` is set: a whole warp runs the
// issue code (its descriptors stay warp-uniform) and one lane executes the instruction
__device__ __forceinline__ void um_mma_ss_p(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc, uint32_t issue) {
  asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 q, %5, 0;\n\t"
               "@q tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(issue) : "memory");
}
__device__ __forceinline__ void um_mma_ts_p(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc, uint32_t issue) {
  asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.ne.b32 q, %5, 0;\n\t"
               "@q tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}"
               :: "r"(d), "r"(a), "l"(b), "r"(idesc), "r"(acc), "r"(issue) : "memory");
}
__device__ __forceinline__ void um_commit_p(uint64_t *mbar, uint32_t issue) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t"
               "@q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
               :: "r"(um_sa(mbar)), "r"(issue) : "memory");
}
__device__ __forceinline__ void um_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(um_sa(mbar)) : "memory");
}
__device__ __forceinline__ void um_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void um_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void um_fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void um_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void um_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ bool um_try_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(um_sa(mbar)), "r"(parity) : "memory");
  return ok != 0;
}
// bounded wait (about a second at the SM clock); false if it ran out
__device__ __forceinline__ bool um_wait(uint64_t *mbar, uint32_t parity) {
  if (um_try_wait(mbar, parity)) return true;
  const long long t0 = clock64();
  while (!um_try_wait(mbar, parity))
    if (clock64() - t0 > (1ll << 31)) return false;
  return true;
}
__device__ __forceinline__ void um_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(um_sa(mbar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(um_sa(dst)), "l"(src), "r"(bytes), "r"(um_sa(mbar)) : "memory");
}

// tcgen05.ld / st of 8 or 16 consecutive 32-bit columns of this thread's lane
#define UM_R8(v, o) "=r"(v[o + 0]), "=r"(v[o + 1]), "=r"(v[o + 2]), "=r"(v[o + 3]), "=r"(v[o + 4]), "=r"(v[o + 5]), \
                    "=r"(v[o + 6]), "=r"(v[o + 7])
#define UM_W8(v, o) "r"(v[o + 0]), "r"(v[o + 1]), "r"(v[o + 2]), "r"(v[o + 3]), "r"(v[o + 4]), "r"(v[o + 5]), \
                    "r"(v[o + 6]), "r"(v[o + 7])
__device__ __forceinline__ void um_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];" : UM_R8(v, 0) : "r"(taddr));
}
__device__ __forceinline__ void um_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : UM_R8(v, 0), UM_R8(v, 8) : "r"(taddr));
}
__device__ __forceinline__ void um_st8(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" :: "r"(taddr), UM_W8(v, 0) : "memory");
}
__device__ __forceinline__ void um_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               :: "r"(taddr), UM_W8(v, 0), UM_W8(v, 8) : "memory");
}

// ties the loaded registers to the preceding tcgen05.wait::ld, so that no use of them is
// scheduled before the wait
__device__ __forceinline__ void um_regs8(uint32_t *v) {
  asm volatile("" : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]));
}

// x rounded to TF32 (10 explicit mantissa bits, to nearest, ties away from zero: the
// rounding of cvt.rna.tf32.f32) with two integer operations; x is finite here
__device__ __forceinline__ float um_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// volume index of node k of face f for a face index known only at run time
template <int N>
__device__ __forceinline__ int um_fmask_rt(int f, int k) {
  const int j = N - k;
  const int rs_k = k * (N + 1) - k * (k - 1) / 2, rs_j = j * (N + 1) - j * (j - 1) / 2;
  return f == 0 ? k : (f == 1 ? rs_k + (N - k) : rs_j);
}

// ---- the kernel --------------------------------------------------------------------
// packed FP32x2 arithmetic (two nodes or points per instruction)
__device__ __forceinline__ float2 um_f2(uint32_t x, uint32_t y) { return make_float2(__uint_as_float(x), __uint_as_float(y)); }
__device__ __forceinline__ float2 um_b2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 um_fma2(float a, float2 x, float2 y) { return __ffma2_rn(um_b2(a), x, y); }
__device__ __forceinline__ float2 um_mul2(float a, float2 x) { return __fmul2_rn(um_b2(a), x); }
__device__ __forceinline__ float um_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void um_arrive(uint64_t *mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(um_sa(mbar)) : "memory");
}

// per-element geometry of a stage (Sec. 5): the chain-rule factors, 1/J, the three edge
// vectors and the vertex grid velocities (v_0 and the differences v_1 - v_0, v_2 - v_0), from
// which the grid velocity at a node is interpolated where it is used, with the node's
// barycentrics ((1 + r) / 2, (1 + s) / 2) from the shared tables
template <int N>
struct UmGeo {
  float rx, sx, ry, sy, iJ;
  float ex[3], ey[3];
  float vx0, vy0, dvx1, dvy1, dvx2, dvy2;
  const float *bar;
};

// tails (smem tile) and heads (TMEM) of fields [3H, 3H + 3) of the element's row
template <int N, int H>
__device__ __forceinline__ void um_convert(const float *row, float *sA, uint32_t tl, int el, bool live) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, NPP = D::NPP, KV = D::KV, CA = D::CA;
  constexpr int F0 = 3 * H, W0 = F0 * Np, W1 = (F0 + 3) * Np;    // row floats [W0, W1)
  constexpr int J0 = W0 / 4, J1 = (W1 + 3) / 4;                   // float4 chunks covering them
  float q[4 * (J1 - J0)];
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    const float4 v = live ? reinterpret_cast<const float4 *>(row)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    q[4 * (j - J0) + 0] = v.x;
    q[4 * (j - J0) + 1] = v.y;
    q[4 * (j - J0) + 2] = v.z;
    q[4 * (j - J0) + 3] = v.w;
  }
  auto val = [&](int f, int n) -> float { return n < Np ? q[f * Np + n - 4 * J0] : 0.0f; };
  // tail k-groups of the three fields (the K overrun past the last field goes with H = 1)
  constexpr int G0 = F0 * NPP / 4, G1 = H ? CA / 4 : (F0 + 3) * NPP / 4;
#pragma unroll
  for (int g = G0; g < G1; ++g) {
    float lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int col = 4 * g + i, f = col / NPP, n = col % NPP;
      const float x = f < 6 ? val(f, n) : 0.0f;
      lv[i] = x - um_tf32(x);
    }
    reinterpret_cast<float4 *>(sA)[g * 128 + el] = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
#pragma unroll
  for (int f = F0; f < F0 + 3; ++f)
#pragma unroll
    for (int j = 0; j < KV; j += 8) {
      uint32_t hv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) hv[i] = __float_as_uint(um_tf32(val(f, j + i)));
      um_st8(tl + D::T_QH + f * KV + j, hv);
    }
}

// volume terms (A + v_G) . grad q (Sec. 2, Sec. 3) at nodes [8H, 8H + 8) of the element, into R
template <int N, int H>
__device__ __forceinline__ void um_volume(uint32_t tl, const UmGeo<N> &G, float mc, float mcs) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, KV = D::KV;
  constexpr int n0 = 8 * H;
  if constexpr (n0 < Np) {
    constexpr int P0 = n0 / 2;   // first node pair
    // the grid velocity at the node pairs of this half (P1 interpolation of the vertex values)
    float2 vgx[4], vgy[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (n0 + 2 * p >= Np) break;
      const float4 b4 = reinterpret_cast<const float4 *>(G.bar)[P0 + p];
      const float2 an = make_float2(b4.x, b4.z), bn = make_float2(b4.y, b4.w);
      vgx[p] = __ffma2_rn(bn, um_b2(G.dvx2), __ffma2_rn(an, um_b2(G.dvx1), um_b2(G.vx0)));
      vgy[p] = __ffma2_rn(bn, um_b2(G.dvy2), __ffma2_rn(an, um_b2(G.dvy1), um_b2(G.vy0)));
    }
    float2 rhs[6][4];
#pragma unroll
    for (int f = 0; f < 6; ++f)
#pragma unroll
      for (int p = 0; p < 4; ++p) rhs[f][p] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int f0 = 0; f0 < 6; f0 += 3) {
      uint32_t vr[3][8], vs[3][8];
#pragma unroll
      for (int ff = 0; ff < 3; ++ff) {
        um_ld8(tl + um_tv<N>(f0 + ff) + n0, vr[ff]);
        um_ld8(tl + um_tv<N>(f0 + ff) + KV + n0, vs[ff]);
      }
      um_wait_ld();
#pragma unroll
      for (int ff = 0; ff < 3; ++ff) {
        um_regs8(vr[ff]);
        um_regs8(vs[ff]);
      }
#pragma unroll
      for (int ff = 0; ff < 3; ++ff) {
        const int f = f0 + ff;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (n0 + 2 * p >= Np) break;
          const float2 d_r = um_f2(vr[ff][2 * p], vr[ff][2 * p + 1]), d_s = um_f2(vs[ff][2 * p], vs[ff][2 * p + 1]);
          const float2 qx = um_fma2(G.sx, d_s, um_mul2(G.rx, d_r));
          const float2 qy = um_fma2(G.sy, d_s, um_mul2(G.ry, d_r));
          const float2 ale = __ffma2_rn(vgy[p], qy, __fmul2_rn(vgx[p], qx));
          switch (f) {
            case 0: rhs[0][p] = __fadd2_rn(rhs[0][p], ale); rhs[1][p] = um_fma2(mc, qx, rhs[1][p]);
                    rhs[2][p] = um_fma2(mc, qy, rhs[2][p]); break;
            case 1: rhs[1][p] = __fadd2_rn(rhs[1][p], ale); rhs[0][p] = um_fma2(mc, qx, rhs[0][p]);
                    rhs[3][p] = um_fma2(mc, qy, rhs[3][p]); rhs[4][p] = um_fma2(mcs, qx, rhs[4][p]); break;
            case 2: rhs[2][p] = __fadd2_rn(rhs[2][p], ale); rhs[0][p] = um_fma2(mc, qy, rhs[0][p]);
                    rhs[3][p] = um_fma2(mc, qx, rhs[3][p]); rhs[5][p] = um_fma2(mcs, qy, rhs[5][p]); break;
            case 3: rhs[3][p] = __fadd2_rn(rhs[3][p], ale); rhs[2][p] = um_fma2(mc, qx, rhs[2][p]);
                    rhs[1][p] = um_fma2(mc, qy, rhs[1][p]); break;
            case 4: rhs[4][p] = __fadd2_rn(rhs[4][p], ale); rhs[1][p] = um_fma2(mcs, qx, rhs[1][p]); break;
            default: rhs[5][p] = __fadd2_rn(rhs[5][p], ale); rhs[2][p] = um_fma2(mcs, qy, rhs[2][p]); break;
          }
        }
      }
    }
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      uint32_t v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[i] = n0 + i < Np ? __float_as_uint((i & 1) ? rhs[f][i >> 1].y : rhs[f][i >> 1].x) : 0u;
      um_st8(tl + um_tr<N>(f) + n0, v);
    }
  }
}

// Ntilde (Sec. 2) at the cubature points of chunks [C0, C1) (8 points each), loaded in one
// batch: heads in place, tails to the slots
template <int N, int H>
__device__ __forceinline__ void um_cubature(uint32_t tl, float itau) {
  typedef UmDim<N> D;
  constexpr int NCH = D::KC / 8, HALF = (NCH + 1) / 2;
  constexpr int C0 = H ? HALF : 0, C1 = H ? NCH : HALF, NC = C1 - C0;
  const float ISQ2 = 0.70710678118654752f;
  if constexpr (NC > 0) {
    uint32_t cq[3][NC][8];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int ch = 0; ch < NC; ++ch) um_ld8(tl + um_tc<N>(f) + 8 * (C0 + ch), cq[f][ch]);
    um_wait_ld();
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int ch = 0; ch < NC; ++ch) um_regs8(cq[f][ch]);
#pragma unroll
    for (int ch = 0; ch < NC; ++ch) {
      uint32_t hv[3][8], lv[3][8];
#pragma unroll
      for (int i = 0; i < 8; i += 2) {
        const float2 q1 = __fadd2_rn(um_b2(1.0f), um_f2(cq[0][ch][i], cq[0][ch][i + 1]));
        const float2 q2 = um_f2(cq[1][ch][i], cq[1][ch][i + 1]), q3 = um_f2(cq[2][ch][i], cq[2][ch][i + 1]);
        const float2 r1 = um_mul2(itau, make_float2(um_rcp(q1.x), um_rcp(q1.y)));
        const float2 rs = um_mul2(ISQ2, r1);
        const float2 nv[3] = {__fmul2_rn(__fmul2_rn(q2, q3), r1), __fmul2_rn(__fmul2_rn(q2, q2), rs),
                              __fmul2_rn(__fmul2_rn(q3, q3), rs)};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const float2 t = make_float2(um_tf32(nv[f].x), um_tf32(nv[f].y));
          const float2 l = __fadd2_rn(nv[f], make_float2(-t.x, -t.y));
          hv[f][i] = __float_as_uint(t.x); hv[f][i + 1] = __float_as_uint(t.y);
          lv[f][i] = __float_as_uint(l.x); lv[f][i + 1] = __float_as_uint(l.y);
        }
      }
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        um_st8(tl + um_tc<N>(f) + 8 * (C0 + ch), hv[f]);
        um_st8(tl + um_nslot<N>(f, C0 + ch), lv[f]);
      }
    }
  }
}

// upwind F_S and F_ALE (Sec. 3) at face nodes j = f Nfp + k in [8H, 8H + 8) of the element:
// fl[fld][j - 8H].  qm is the element's own staged row; the trace across face f comes from
// src[f]: the neighbour's staged row or its global row (hal[f] = false: node vol2 of field
// fld at fld Np + vol2) or a halo entry (hal[f] = true: face node k of field fld at 6 k + fld)
template <int N, int H>
__device__ __forceinline__ void um_flux(const UmGeo<N> &G, const float *qm, const float *const (&src)[3],
                                        const bool (&hal)[3], const int (&f2)[3], float c, float (&fl)[6][8]) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, NFN = D::NFN;
  const float SQ2 = 1.41421356237309505f;
#pragma unroll
  for (int fld = 0; fld < 6; ++fld)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) fl[fld][jj] = 0.0f;
  // the neighbour traces of all of this half's face nodes first (one round trip)
  float nv[8][6];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      const int j = f * Nfp + k;
      if (j < 8 * H || j >= 8 * H + 8) continue;
      const int off = hal[f] ? 6 * k : um_fmask_rt<N>(f2[f], Nfp - 1 - k), st = hal[f] ? 1 : Np;
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) nv[j - 8 * H][fld] = src[f][off + fld * st];
    }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    // faces that have a node in this half
    if (!((f + 1) * Nfp > 8 * H && f * Nfp < 8 * H + 8 && f * Nfp < NFN)) continue;
    const float dx = G.ex[f], dy = G.ey[f];
    const float len = sqrtf(dx * dx + dy * dy);
    const float il = 1.0f / len;
    const float nx = dy * il, ny = -dx * il;
    const float fs = 0.5f * len * G.iJ;
    const float h = 0.5f * c * fs;
    const float al = (9.0f - 1.7320508075688772f) / 6.0f, be = (1.7320508075688772f - 3.0f) / 6.0f;
    // |At_n| on the {1,4,5,6} block and the {2,3} block, closed form alpha At_n^2 + beta At_n^4
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
    // the face's nodes in this half, two at a time in packed FP32x2 arithmetic (the face
    // constants are shared; a node left over at the end goes in the .x lane alone)
    const int kA = 8 * H - f * Nfp > 0 ? 8 * H - f * Nfp : 0;
    const int kB = 8 * H + 8 - f * Nfp < Nfp ? 8 * H + 8 - f * Nfp : Nfp;
#pragma unroll
    for (int k = kA; k < kB; k += 2) {
      const bool two = k + 1 < kB;
      const int jA = f * Nfp + k - 8 * H, jB = two ? jA + 1 : jA;
      const int volA = tc_fmask<N>(f, k), volB = two ? tc_fmask<N>(f, k + 1) : volA;
      float2 w[6];
#pragma unroll
      for (int fld = 0; fld < 6; ++fld)
        w[fld] = make_float2(nv[jA][fld] - qm[fld * Np + volA], nv[jB][fld] - qm[fld * Np + volB]);
      const float2 abA = reinterpret_cast<const float2 *>(G.bar)[volA], abB = reinterpret_cast<const float2 *>(G.bar)[volB];
      const float2 ra = make_float2(abA.x, abB.x), sb = make_float2(abA.y, abB.y);
      const float2 gx = __ffma2_rn(sb, um_b2(G.dvx2), __ffma2_rn(ra, um_b2(G.dvx1), um_b2(G.vx0)));
      const float2 gy = __ffma2_rn(sb, um_b2(G.dvy2), __ffma2_rn(ra, um_b2(G.dvy1), um_b2(G.vy0)));
      const float2 vn = __ffma2_rn(um_b2(ny), gy, __fmul2_rn(um_b2(nx), gx));
      const float2 ale = make_float2(vn.x > 0.0f ? vn.x * fs : 0.0f, vn.y > 0.0f ? vn.y * fs : 0.0f);
      auto acc = [](float2 s, float c, float2 x) { return __ffma2_rn(um_b2(c), x, s); };
      float2 o[6];
      o[0] = acc(acc(acc(acc(acc(acc(__fmul2_rn(ale, w[0]), M00, w[0]), M03, w[3]), M04, w[4]), M05, w[5]), nhx, w[1]), nhy, w[2]);
      o[3] = acc(acc(acc(acc(acc(acc(__fmul2_rn(ale, w[3]), M03, w[0]), M33, w[3]), M34, w[4]), M35, w[5]), nhx, w[2]), nhy, w[1]);
      o[4] = acc(acc(acc(acc(acc(__fmul2_rn(ale, w[4]), M04, w[0]), M34, w[3]), M44, w[4]), M45, w[5]), nsx, w[1]);
      o[5] = acc(acc(acc(acc(acc(__fmul2_rn(ale, w[5]), M05, w[0]), M35, w[3]), M45, w[4]), M55, w[5]), nsy, w[2]);
      o[1] = acc(acc(acc(acc(acc(__fmul2_rn(ale, w[1]), N11, w[1]), N12, w[2]), nhx, w[0]), nsx, w[4]), nhy, w[3]);
      o[2] = acc(acc(acc(acc(acc(__fmul2_rn(ale, w[2]), N12, w[1]), N22, w[2]), nhy, w[0]), nsy, w[5]), nhx, w[3]);
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) {
        fl[fld][jA] = o[fld].x;
        if (two) fl[fld][jB] = o[fld].y;
      }
    }
  }
}

template <int N, int H>
__device__ __forceinline__ void um_flux_store(uint32_t tl, const float (&fl)[6][8]) {
  typedef UmDim<N> D;
  constexpr int KL = D::KL;
  if constexpr (8 * H < KL) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      uint32_t hv[8], lv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float x = fl[f][i], t = um_tf32(x);
        hv[i] = __float_as_uint(t);
        lv[i] = __float_as_uint(x - t);
      }
      um_st8(tl + um_tfh<N>(f) + 8 * H, hv);
      um_st8(tl + um_tfl<N>(f) + 8 * H, lv);
    }
  }
}

// SARK combination (Sec. 4) of row chunks [J0, J1) of the element, in the staged rows
template <int N, int STAGE, int H>
__device__ __forceinline__ void um_sark(uint32_t tl, float4 *rowq, float4 *row1, float4 *row2, const float (&k0)[5],
                                        const float (&k1)[5], float dt, bool &bad) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, S4 = D::S4, HALF = (S4 + 1) / 2;
  constexpr int J0 = H ? HALF : 0, J1 = H ? S4 : HALF;
  constexpr int FA = (4 * J0) / Np, FB = ((4 * J1 - 1) / Np < 5 ? (4 * J1 - 1) / Np : 5);   // fields touched
  uint32_t rr[FB - FA + 1][16];
#pragma unroll
  for (int f = FA; f <= FB; ++f) um_ld16(tl + um_tr<N>(f), rr[f - FA]);
  um_wait_ld();
#pragma unroll
  for (int f = FA; f <= FB; ++f) {
    um_regs8(rr[f - FA]);
    um_regs8(rr[f - FA] + 8);
  }
#pragma unroll
  for (int j = J0; j < J1; ++j) {
    float r_[4], qv[4] = {0.f, 0.f, 0.f, 0.f}, f0[4] = {0.f, 0.f, 0.f, 0.f}, av[4] = {0.f, 0.f, 0.f, 0.f}, o[4], o2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int w = 4 * j + i;
      r_[i] = w < 6 * Np ? __uint_as_float(rr[w / Np - FA][w % Np]) : 0.0f;
    }
    if (STAGE >= 0) {
      const float4 x = rowq[j];
      qv[0] = x.x; qv[1] = x.y; qv[2] = x.z; qv[3] = x.w;
    }
    if (STAGE == 1 || STAGE == 2) {
      const float4 x = row1[j];
      f0[0] = x.x; f0[1] = x.y; f0[2] = x.z; f0[3] = x.w;
    }
    if (STAGE >= 2) {
      const float4 x = row2[j];
      av[0] = x.x; av[1] = x.y; av[2] = x.z; av[3] = x.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int w = 4 * j + i;
      const float *k = w < 3 * Np ? k0 : k1;   // E, A_a, A_b, B_a, B_b of the field class
      o2[i] = 0.0f;
      if (STAGE < 0) {
        o[i] = r_[i];
      } else if (STAGE == 0) {
        o2[i] = r_[i];
        o[i] = dt * (k[1] * r_[i]) + k[0] * qv[i];
      } else if (STAGE == 1) {
        o[i] = dt * (k[2] * r_[i] + k[1] * f0[i]) + k[0] * qv[i];
        o2[i] = k[4] * r_[i] + k[3] * f0[i];
      } else if (STAGE == 2) {
        o[i] = dt * (k[2] * r_[i] + k[1] * f0[i]) + k[0] * qv[i];
        o2[i] = k[3] * r_[i] + av[i];
      } else {
        o[i] = dt * (k[3] * r_[i] + av[i]) + k[0] * qv[i];
        if (w < 6 * Np) bad |= (__float_as_int(o[i]) & 0x7f800000) == 0x7f800000;
      }
    }
    rowq[j] = make_float4(o[0], o[1], o[2], o[3]);
    if (STAGE == 0 || STAGE == 1) row1[j] = make_float4(o2[0], o2[1], o2[2], o2[3]);
    if (STAGE == 2) row2[j] = make_float4(o2[0], o2[1], o2[2], o2[3]);
  }
}

// motion factors of the stage (Sec. 5, RK4 nodes c = (0, 1/2, 1/2, 1) and weights): grid velocity
// v_i = gf S(X), stage position x_i = x_n + xf S(X), final vertex factor x_{n+1} = x_n + fin S(X).
// Called by a whole warp: lanes 0..2 evaluate cos(w (t_n + k dt / 2)) (one FP64 cosine each,
// in parallel), lane 0 combines them.
__device__ __forceinline__ void um_stage_motion_warp(const StageArgs &a, int stage, int lane, double &gf, double &xf,
                                                     double &fin) {
  gf = 0.0; xf = 0.0; fin = 0.0;
  if (a.motion_A == 0.0) return;
  const double w = a.motion_w, Aw = a.motion_A * a.motion_w, dt = a.dt;
  double ck = 0.0;
  if (lane < 3) ck = stage < 0 ? cos(w * a.rhs_time) : cos(w * (a.clock[0] + 0.5 * lane * dt));
  const double c0 = __shfl_sync(0xffffffffu, ck, 0), c1 = __shfl_sync(0xffffffffu, ck, 1),
               c2 = __shfl_sync(0xffffffffu, ck, 2);
  if (stage < 0) {
    gf = Aw * c0;
    return;
  }
  const double cs[3] = {c0, c1, c2};   // at t_n, t_n + dt / 2, t_n + dt
  const int node[4] = {0, 1, 1, 2};    // c_i = node[i] / 2
  gf = Aw * cs[node[stage]];
  if (stage > 0) xf = dt * (stage == 3 ? 1.0 : 0.5) * Aw * cs[node[stage - 1]];
  if (stage == 3) fin = dt * Aw * (c0 / 6.0 + c1 * (2.0 / 3.0) + c2 / 6.0);
}

// Shared-memory buffers of a tile (element-major rows of stride S unless noted):
//   sA    the head tile of the own fields (core-matrix layout) for the first MMA batch;
//         afterwards q_n, then q_{i+1} (or F in the rhs-only mode), stored back by a bulk copy
//   sRaw  the own fields q_i (neighbour traces and q^- of the flux); the next tile's q_i is
//         prefetched into it once this tile's fluxes are formed
//   sX1   F_0 (read at stages 1-2; written at stage 0; the accumulator written at stage 1)
//   sX2   the btilde accumulator (read at stages 2-3, written at stage 2)
//   sG    the geometry of the tile's elements, formed by the helper warps one tile ahead
//   sH    the halo of the tile's out-of-tile neighbour traces, staged one tile ahead
// Warps 0-7 compute (two threads per element: thread t handles element t % 128 and half
// t / 128 of each phase's nodes, points, face nodes or row chunks); lane 0 of compute warp
// w < 6 also issues the first products (volume, and for w < 3 the interpolation in the same
// instruction) and the lift products of field w, at the two points where the compute warps
// would otherwise wait for them.  Warps 8-11 are helpers: thread 256 + i forms the geometry of
// element i of the next tile while the current one is computed, the helpers stage the traces
// across the next tile's out-of-tile faces (a halo of up to HMAX faces; a Morton tile of 128
// triangles has about 32), and lane 0 of helper warp 8 + f (f < 3) issues the projection
// products of field f; warp 8 also issues the bulk copies.  Every accumulator has one issuing
// thread, so its sums run in a fixed order.  Hand-offs are mbarriers, one phase per tile
// each: the copies and MMA commits complete the "data" barriers, the compute threads arrive
// on the "operands ready" ones.
constexpr int kUmThreads = 384;
constexpr int kUmIssuers = 4;       // helper warps committing the projection batch
constexpr int kUmFieldIssuers = 6;  // compute warps committing the first and the lift batches

// K / 8 k-steps of the three split products hi*hi + hi*lo + lo*hi of one field into
// accumulator d, issued by the lane with `issue` set.  A heads in TMEM at a_hi; A tails in TMEM
// at a_lo_t, or (lo_in_smem) in shared memory at descriptor a_lo_s; B heads and tails at
// descriptors bh, bl, advancing by b_step per k-step.  The first product overwrites d when
// `overwrite` is set.
__device__ __forceinline__ void um_mma_field(uint32_t d, uint32_t a_hi, uint32_t a_lo_t, uint64_t a_lo_s, bool lo_in_smem,
                                             uint64_t bh, uint64_t bl, uint64_t b_step, uint32_t id, int ksteps,
                                             bool overwrite, uint32_t issue) {
  for (int ks = 0; ks < ksteps; ++ks) {
    const uint64_t b0 = bh + ks * b_step, b1 = bl + ks * b_step;
    um_mma_ts_p(d, a_hi + 8 * ks, b0, id, (overwrite && ks == 0) ? 0u : 1u, issue);
    um_mma_ts_p(d, a_hi + 8 * ks, b1, id, 1u, issue);
    if (lo_in_smem) um_mma_ss_p(d, a_lo_s + ks * (uint64_t)((2 * 2048) >> 4), b0, id, 1u, issue);
    else um_mma_ts_p(d, a_lo_t + 8 * ks, b0, id, 1u, issue);
  }
}

// inputs of an element's geometry: its mesh record and the current positions and motion
// shapes of its vertices (loaded ahead of their use)
struct UmGeoIn {
  MeshRec rec;
  double2 xv[3], sv[3];   // as loaded: nothing waits for the loads until the geometry is formed
};
__device__ __forceinline__ MeshRec um_rec(const StageArgs &a, int64_t e) { return a.mesh[e]; }
__device__ __forceinline__ void um_vertices(const StageArgs &a, UmGeoIn &in) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    in.xv[k] = reinterpret_cast<const double2 *>(a.xn)[in.rec.v[k]];
    in.sv[k] = reinterpret_cast<const double2 *>(a.shape)[in.rec.v[k]];
  }
}

// the element's geometry at the stage (Sec. 5) into its row of the geometry buffer; a face
// whose neighbour lies outside the tile [t0e, t0e + nel) gets a halo slot from the shared
// counter while slots last (code -(slot + 1) in the row, the neighbour code in hsrc[slot]);
// the other faces keep the neighbour code (element << 2 | face)
template <int N>
__device__ __forceinline__ void um_geometry(const StageArgs &a, const UmGeoIn &in, bool live, int64_t t0e, int nel,
                                            float xff, float gff, float *g, int *hcount, int *hsrc) {
  const MeshRec &rec = in.rec;
  double bx[3], by[3];
  float ix[3], iy[3], vx[3], vy[3], ex[3], ey[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    bx[k] = in.xv[k].x + rec.shift[2 * k] * a.period[0];
    by[k] = in.xv[k].y + rec.shift[2 * k + 1] * a.period[1];
    const float sxk = (float)in.sv[k].x, syk = (float)in.sv[k].y;
    ix[k] = xff * sxk;
    iy[k] = xff * syk;
    vx[k] = gff * sxk;
    vy[k] = gff * syk;
  }
  // FP64 vertex positions and edge differences, the small stage increments in FP32
  ex[0] = (float)(bx[1] - bx[0]) + (ix[1] - ix[0]); ey[0] = (float)(by[1] - by[0]) + (iy[1] - iy[0]);
  ex[1] = (float)(bx[2] - bx[1]) + (ix[2] - ix[1]); ey[1] = (float)(by[2] - by[1]) + (iy[2] - iy[1]);
  ex[2] = (float)(bx[0] - bx[2]) + (ix[0] - ix[2]); ey[2] = (float)(by[0] - by[2]) + (iy[0] - iy[2]);
  const float xr = 0.5f * ex[0], yr = 0.5f * ey[0], xs = -0.5f * ex[2], ys = -0.5f * ey[2];
  const float J = xr * ys - xs * yr;
  if (live && !(J > 0.0f)) atomicOr(a.status, GB_STATUS_MESH);
  const float iJ = 1.0f / J;
  int code[3];
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const int nb = rec.nbr[f];
    const int64_t nbe = nb >> 2;
    code[f] = nb;
    if (live && !(nbe >= t0e && nbe < t0e + nel)) {
      const int sl = atomicAdd(hcount, 1);
      if (sl < UmDim<N>::HMAX) {
        hsrc[sl] = nb;
        code[f] = -(sl + 1);
      }
    }
  }
  float4 *g4 = reinterpret_cast<float4 *>(g);
  g4[0] = make_float4(ys * iJ, -yr * iJ, -xs * iJ, xr * iJ);
  g4[1] = make_float4(iJ, ex[0], ex[1], ex[2]);
  g4[2] = make_float4(ey[0], ey[1], ey[2], vx[0]);
  g4[3] = make_float4(vx[1], vx[2], vy[0], vy[1]);
  g4[4] = make_float4(vy[2], __int_as_float(code[0]), __int_as_float(code[1]), __int_as_float(code[2]));
}

// the halo: the traces across the out-of-tile faces listed in hsrc[0, cnt), entry s holding
// the neighbour's values at this side's face nodes k (field fld at 6 k + fld); helper thread
// hi takes entries hi, hi + 128, ...
template <int N>
__device__ __forceinline__ void um_halo(const float *qin, const int *hsrc, int cnt, int hi, float *halo) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, Nfp = D::Nfp, S = D::S, HW = D::HW;
  for (int sl = hi; sl < cnt; sl += 128) {
    const int nb = hsrc[sl];
    const float *qp = qin + (int64_t)(nb >> 2) * S;
    const int f2 = nb & 3;
    float v[HW];
#pragma unroll
    for (int k = 0; k < Nfp; ++k) {
      const int vol2 = um_fmask_rt<N>(f2, Nfp - 1 - k);
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) v[6 * k + fld] = qp[fld * Np + vol2];
    }
#pragma unroll
    for (int i = 0; i < HW; ++i) halo[sl * HW + i] = v[i];
  }
}

// one kernel for every stage (the stage is a run-time argument), so that the launches of a
// step share their code
template <int N>
__global__ void __launch_bounds__(kUmThreads, 1) um_stage_kernel(const StageArgs a) {
  const int STAGE = a.stage;
  typedef UmDim<N> D;
  constexpr int S = D::S, NPP = D::NPP, KV = D::KV, GW = D::GW;
  constexpr int NV = D::NV, KC = D::KC, KL = D::KL;
  const float SQ2 = 1.41421356237309505f;
  extern __shared__ __align__(1024) float um_smem[];
  float *sA = um_smem + D::SM_A;
  float *sRaw = um_smem + D::SM_RAW;
  float *sX1 = um_smem + D::SM_X1;
  float *sX2 = um_smem + D::SM_X2;
  float *sB = um_smem + D::SM_B;
  float *sG = um_smem + D::SM_G;
  float *sH = um_smem + D::SM_H;
  __shared__ int s_hcount, s_hsrc[D::HMAX];   // halo entries of the next tile and their neighbours
  // data: q_i, F_0/accumulator, q_n loaded; shared tile free (the previous stores have read
  // it); volume, interpolation, projection, lift products done (one commit per issuer);
  // geometry and halo of the tile formed (128 helper threads each)
  __shared__ __align__(8) uint64_t mb_ld, mb_x, mb_qn, mb_free, mb_v, mb_c, mb_p, mb_l, mb_geo, mb_halo;
  // operands ready (256 compute threads): heads and tails; geometry read; R and Ntilde;
  // fluxes; output rows
  __shared__ __align__(8) uint64_t mb_opA, mb_gread, mb_opN, mb_opF, mb_out;
  __shared__ uint32_t s_tmem;
  __shared__ double s_motion[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float *qin = reinterpret_cast<const float *>(a.qin);
  const int64_t ntile = (a.K + 127) >> 7;
  auto tile_rows = [&](int64_t t_) { return (int)((a.K - t_ * 128) < 128 ? (a.K - t_ * 128) : 128); };

  __shared__ __align__(8) uint64_t mb_tab;   // operator tables staged
  if (tid == 0) {
    uint64_t *one[4] = {&mb_ld, &mb_x, &mb_qn, &mb_free};
    for (int i = 0; i < 4; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(um_sa(one[i])) : "memory");
    uint64_t *iss[4] = {&mb_v, &mb_c, &mb_p, &mb_l};
    for (int i = 0; i < 4; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                   :: "r"(um_sa(iss[i])), "r"((i == 0 || i == 3) ? kUmFieldIssuers : kUmIssuers) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(um_sa(&mb_geo)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" :: "r"(um_sa(&mb_halo)) : "memory");
    s_hcount = 0;
    uint64_t *many[5] = {&mb_opA, &mb_gread, &mb_opN, &mb_opF, &mb_out};
    for (int i = 0; i < 5; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 256;" :: "r"(um_sa(many[i])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(um_sa(&mb_tab)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // the operator tables and the first tile's own fields, in flight during the set-up
    um_bulk_load(sB, a.ops_um, (uint32_t)(D::BTOT * sizeof(float)), &mb_tab);
    um_arrive(&mb_free);   // the shared tile of the first tile is free
    if ((int64_t)blockIdx.x < ntile)
      um_bulk_load(sRaw, qin + (int64_t)blockIdx.x * 128 * S, (uint32_t)(tile_rows(blockIdx.x) * S * sizeof(float)), &mb_ld);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(um_sa(&s_tmem)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  um_fence_async_smem();
  um_fence_before();
  __syncthreads();
  um_fence_after();
  const uint32_t tm = s_tmem;
  bool failed = !__all_sync(0xffffffffu, um_wait(&mb_tab, 0));
  const uint32_t one = lane == 0 ? 1u : 0u;   // the lane that executes its warp's MMAs and commits
  // the field-tail tile: in the F_0 / accumulator buffer that the stage does not use (stages
  // 0, 1: the accumulator's; stages 2, 3 and the rhs: F_0's, loaded at stage 2 only once the
  // first products have read the tails)
  float *sT = (STAGE == 0 || STAGE == 1) ? sX2 : sX1;
  const uint32_t sB_a = um_sa(sB);
  // descriptors at the operands' bases; an operand at byte offset o has descriptor base + o / 16
  const uint64_t dA = um_desc(um_sa(sT), 2048, 128);
  const uint64_t dBV = um_desc(sB_a + 4 * D::BV, D::NVC * 16, 128);
  const uint64_t dBP = um_desc(sB_a + 4 * D::BP, 256, 128), dBL = um_desc(sB_a + 4 * D::BL, 256, 128);
  constexpr uint32_t idV = um_idesc(NV), idC = um_idesc(D::NCM), idR = um_idesc(16);

  if (warp >= 8) {
    // ================= helpers: geometry one tile ahead, MMA issue, bulk copies =================
    const int hi = tid - 256, iw = warp - 8;   // element of the next tile, issuer index
    const bool copier = tid == 256;
    unsigned armed = (copier && (int64_t)blockIdx.x < ntile) ? 1u : 0u;   // phases in flight from this thread
    uint32_t ld_par = 0;  // parity of the armed phase of mb_ld
    // the first tile's geometry inputs: the mesh records first, before anything waits
    const bool first = (int64_t)blockIdx.x < ntile;
    const int64_t t0 = blockIdx.x, r0 = a.K - t0 * 128;
    UmGeoIn in0;
    if (first) in0.rec = um_rec(a, t0 * 128 + (hi < r0 ? hi : 0));
    // the stage's motion factors (FP64 cosines: three lanes of warp 11 in parallel) after the
    // set-up barrier, so that the compute warps and the first bulk copies do not wait for them
    if (warp == 11) {
      double gf, xf, fin;
      um_stage_motion_warp(a, STAGE, lane, gf, xf, fin);
      if (lane == 0) {
        s_motion[0] = gf;
        s_motion[1] = xf;
        if (STAGE == 3 && blockIdx.x == 0) const_cast<double *>(a.clock)[1] = fin;
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const float gff = (float)s_motion[0], xff = (float)s_motion[1];
    // the first tile's geometry and halo
    if (first) {
      um_vertices(a, in0);
      um_geometry<N>(a, in0, hi < r0, t0 * 128, tile_rows(t0), xff, gff, sG + hi * GW, &s_hcount, s_hsrc);
      um_arrive(&mb_geo);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      um_halo<N>(qin, s_hsrc, s_hcount < D::HMAX ? s_hcount : D::HMAX, hi, sH);
      um_arrive(&mb_halo);
    }
    // A failed (timed-out) wait does not leave the loop at once: the helpers meet at named
    // barriers, so the rest of the iteration is skipped and they leave together at its end.
    uint32_t par = 0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x, par ^= 1u) {
      const int64_t e0 = tile * 128;
      const uint32_t tile_bytes = (uint32_t)(tile_rows(tile) * S * sizeof(float));
      const bool more = tile + gridDim.x < ntile;
      // the next tile's geometry inputs: its mesh record now, its vertex data after the
      // interpolation batch is issued, the arithmetic once the projection batch is issued
      const int64_t tn = tile + gridDim.x, rn = a.K - tn * 128;
      UmGeoIn gin;
      if (more) gin.rec = um_rec(a, tn * 128 + (hi < rn ? hi : 0));
      if (copier) {
        // the previous tile's stores have read the shared tile and the staged rows (the first
        // tile's is free from the set-up)
        if (tile != (int64_t)blockIdx.x) {
          // the output rows leave in the first bulk group, F_0 or the accumulator in a second
          if (STAGE >= 0 && STAGE <= 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          else asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          um_arrive(&mb_free);
        }
        if (STAGE >= 1) {
          // F_0 at stage 1, the accumulator at stages 2 and 3 (F_0 at stage 2 comes with q_n)
          if (tile != (int64_t)blockIdx.x) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(um_sa(&mb_x)), "r"(tile_bytes) : "memory");
          if (STAGE == 1)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(um_sa(sX1)), "l"(reinterpret_cast<const float *>(a.F0) + e0 * S), "r"(tile_bytes),
                            "r"(um_sa(&mb_x)) : "memory");
          if (STAGE >= 2)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(um_sa(sX2)), "l"(reinterpret_cast<const float *>(a.acc) + e0 * S), "r"(tile_bytes),
                            "r"(um_sa(&mb_x)) : "memory");
          armed |= 2u;
        }
      }
      // ---- interpolation products of field iw < 3, once the volume products are complete (they
      //      go first: the compute threads need them first) ----
      if (!failed) {
        if (!__all_sync(0xffffffffu, um_wait(&mb_v, par))) {
          failed = true;
        } else {
          um_fence_after();
          if (iw < 3)
            um_mma_field(tm + um_tc<N>(iw), tm + D::T_QH + iw * KV, 0u, dA + (uint64_t)(((iw * NPP / 4) * 2048) >> 4), true,
                         dBV + (uint64_t)NV, dBV + (uint64_t)NV + (uint64_t)((D::NVC * KV) >> 2), (uint64_t)(2 * D::NVC),
                         idC, KV / 8, true, one);
          um_commit_p(&mb_c, one);
          if (one) armed |= 16u;
        }
      }
      // ---- q_n into the shared tile once the volume and interpolation products have read it ----
      if (copier && STAGE >= 0 && !failed) {
        if (!um_wait(&mb_c, par)) {
          failed = true;
        } else {
          // (at stage 0 the SARK pass writes F_0 into sX1 once q_n is in: the previous F_0 store
          // has read it by then)
          asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          if (STAGE == 2) {   // q_n and F_0, the latter over the tails that the products have read
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(um_sa(&mb_qn)), "r"(2 * tile_bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(um_sa(sA)), "l"(reinterpret_cast<const float *>(a.qn) + e0 * S), "r"(tile_bytes),
                            "r"(um_sa(&mb_qn)) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(um_sa(sX1)), "l"(reinterpret_cast<const float *>(a.F0) + e0 * S), "r"(tile_bytes),
                            "r"(um_sa(&mb_qn)) : "memory");
          } else {
            um_bulk_load(sA, reinterpret_cast<const float *>(a.qn) + e0 * S, tile_bytes, &mb_qn);
          }
          armed |= 4u;
        }
      }
      if (more) um_vertices(a, gin);
      // ---- projection products: R_{4..6} += Ntilde P^T, field iw ----
      if (!failed) {
        if (!__all_sync(0xffffffffu, um_wait(&mb_opN, par))) {
          failed = true;
        } else {
          um_fence_after();
          if (iw < 3) {
            // the tails sit in 8-column slots that are not contiguous across k-steps
            const uint32_t d = tm + um_tr<N>(3 + iw);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ++ks) {
              const uint64_t b0 = dBP + (uint64_t)((4 * 2 * ks * 16 * 4) >> 4);
              const uint64_t b1 = dBP + (uint64_t)((4 * (16 * KC + 2 * ks * 16 * 4)) >> 4);
              const uint32_t ah = tm + um_tc<N>(iw) + 8 * ks;
              um_mma_ts_p(d, tm + um_nslot<N>(iw, ks), b0, idR, 1u, one);
              um_mma_ts_p(d, ah, b0, idR, 1u, one);
              um_mma_ts_p(d, ah, b1, idR, 1u, one);
            }
          }
          um_commit_p(&mb_p, one);
          if (one) armed |= 32u;
        }
      }
      // ---- the next tile's geometry and halo slots, once the compute threads have read this
      //      tile's geometry ----
      if (more) {
        if (!failed && !um_wait(&mb_gread, par)) failed = true;
        asm volatile("bar.sync 1, 128;" ::: "memory");   // this tile's halo entries are all staged
        if (hi == 0) s_hcount = 0;
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (!failed) {
          um_geometry<N>(a, gin, hi < rn, tn * 128, tile_rows(tn), xff, gff, sG + hi * GW, &s_hcount, s_hsrc);
          um_arrive(&mb_geo);
        }
      }
      // ---- the next tile's own fields, once this tile's fluxes have read the current ones ----
      if (copier && more && !failed) {
        if (!um_wait(&mb_opF, par)) {
          failed = true;
        } else {
          um_fence_async_smem();
          um_bulk_load(sRaw, qin + tn * 128 * S, (uint32_t)(tile_rows(tn) * S * sizeof(float)), &mb_ld);
          ld_par = par ^ 1u;
        }
      }
      // ---- the next tile's halo, once this tile's fluxes have read the current one ----
      if (more) {
        if (!failed && !um_wait(&mb_opF, par)) failed = true;
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the next tile's slots are all assigned
        if (!failed) {
          um_halo<N>(qin, s_hsrc, s_hcount < D::HMAX ? s_hcount : D::HMAX, hi, sH);
          um_arrive(&mb_halo);
        }
      }
      // ---- stores of the output rows ----
      if (copier && !failed) {
        if (!um_wait(&mb_out, par)) {
          failed = true;
        } else {
          auto store = [&](void *dst, const float *src) {
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                         :: "l"(reinterpret_cast<float *>(dst) + e0 * S), "r"(um_sa(src)), "r"(tile_bytes) : "memory");
          };
          store(STAGE < 0 ? a.Fout : a.qout, sA);
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          if (STAGE == 0) store(a.F0, sX1);
          if (STAGE == 1) store(a.acc, sX1);
          if (STAGE == 2) store(a.acc, sX2);
          if (STAGE >= 0 && STAGE <= 2) asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      // all helpers leave together if any of them saw a wait run out
      {
        uint32_t any;
        asm volatile("{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.or.pred po, 1, 128, pi;\n\t"
                     "selp.u32 %0, 1, 0, po;\n\t}" : "=r"(any) : "r"((uint32_t)failed) : "memory");
        if (any) {
          failed = true;
          break;
        }
      }
      armed = (copier && more) ? 1u : 0u;   // the other phases of this tile are complete
    }
    if (failed) {
      // wait (bounded) for everything this thread started in the current phase
      uint64_t *bars[7] = {&mb_ld, &mb_x, &mb_qn, &mb_v, &mb_c, &mb_p, &mb_l};   // bulk copies and MMA commits
      for (int i = 0; i < 7; ++i)
        if (armed & (1u << i)) um_wait(bars[i], i == 0 ? ld_par : par);
      atomicOr(a.status, GB_STATUS_TIMEOUT);
    }
    if (copier) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  } else {
    // ================= compute: warps 0-7 =================
    const int el = tid & 127, h = tid >> 7;
    const uint32_t tl = tm + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's 32 lanes
    const float c = (float)a.c, mc = -(float)a.c, mcs = -(float)a.c * SQ2, itau = (float)a.inv_tau;
    const float *bar = sB + D::BBAR;
    const float dt = (float)a.dt;
    const float k0[5] = {a.kco[0][0], a.kco[0][1], a.kco[0][2], a.kco[0][3], a.kco[0][4]};
    const float k1[5] = {a.kco[1][0], a.kco[1][1], a.kco[1][2], a.kco[1][3], a.kco[1][4]};
    bool bad = false;
    uint32_t par = 0;
    uint32_t carmed = 0;   // this lane's MMA commits in flight: 1 volume, 2 lift
    for (int64_t tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x, par ^= 1u) {
      const int64_t e0 = tile * 128;
      const int nel = tile_rows(tile);
      const bool live = el < nel;
      // the own fields in; at stage 2 the tails go over F_0, which the previous tile's SARK pass
      // has read once all its threads have arrived
      if (!__all_sync(0xffffffffu, um_wait(&mb_ld, par) &&
                                       (STAGE != 2 || tile == (int64_t)blockIdx.x || um_wait(&mb_out, par ^ 1u)))) {
        failed = true;
        break;
      }
      // ---- heads and tails of the own fields ----
      const float *row = sRaw + el * S;
      if (h == 0) um_convert<N, 0>(row, sT, tl, el, live);
      else um_convert<N, 1>(row, sT, tl, el, live);
      um_wait_st();
      um_fence_async_smem();
      um_fence_before();
      um_arrive(&mb_opA);
      // ---- volume products of field `warp` (warps 0-5), once every element's operands are in ----
      if (warp < kUmFieldIssuers) {
        if (!__all_sync(0xffffffffu, um_wait(&mb_opA, par))) { failed = true; break; }
        um_fence_after();
        um_mma_field(tm + um_tv<N>(warp), tm + D::T_QH + warp * KV, 0u, dA + (uint64_t)(((warp * NPP / 4) * 2048) >> 4),
                     true, dBV, dBV + (uint64_t)((D::NVC * KV) >> 2), (uint64_t)(2 * D::NVC), idV, KV / 8, true, one);
        um_commit_p(&mb_v, one);
        carmed = one;
      }
      // ---- the tile's geometry, formed by the helpers ----
      if (!__all_sync(0xffffffffu, um_wait(&mb_geo, par))) { failed = true; break; }
      UmGeo<N> G;
      int code[3];
      {
        const float4 *g4 = reinterpret_cast<const float4 *>(sG + el * GW);
        const float4 w0 = g4[0], w1 = g4[1], w2 = g4[2], w3 = g4[3], w4 = g4[4];
        G.rx = w0.x; G.sx = w0.y; G.ry = w0.z; G.sy = w0.w;
        G.iJ = w1.x; G.ex[0] = w1.y; G.ex[1] = w1.z; G.ex[2] = w1.w;
        G.ey[0] = w2.x; G.ey[1] = w2.y; G.ey[2] = w2.z;
        const float vx[3] = {w2.w, w3.x, w3.y}, vy[3] = {w3.z, w3.w, w4.x};
        code[0] = __float_as_int(w4.y); code[1] = __float_as_int(w4.z); code[2] = __float_as_int(w4.w);
        um_arrive(&mb_gread);
        G.vx0 = vx[0]; G.dvx1 = vx[1] - vx[0]; G.dvx2 = vx[2] - vx[0];
        G.vy0 = vy[0]; G.dvy1 = vy[1] - vy[0]; G.dvy2 = vy[2] - vy[0];
        G.bar = bar;
      }
      // ---- volume terms, into R ----
      if (!__all_sync(0xffffffffu, um_wait(&mb_v, par))) { failed = true; break; }
      um_fence_after();
      carmed &= ~1u;
      if (h == 0) um_volume<N, 0>(tl, G, mc, mcs);
      else um_volume<N, 1>(tl, G, mc, mcs);
      // ---- collision term at the cubature points (its tails go to columns that this thread
      //      has read itself, or that no thread reads any more) ----
      if (!__all_sync(0xffffffffu, um_wait(&mb_c, par))) { failed = true; break; }
      um_fence_after();
      if (h == 0) um_cubature<N, 0>(tl, itau);
      else um_cubature<N, 1>(tl, itau);
      um_wait_st();
      um_fence_before();
      um_arrive(&mb_opN);
      // ---- face fluxes while the projection runs: neighbour traces from the staged tile, the
      //      halo, or (past the halo's capacity) global memory ----
      if (!__all_sync(0xffffffffu, um_wait(&mb_halo, par))) { failed = true; break; }
      float fl[6][8];
      {
        const float *src[3];
        bool hal[3];
        int f2[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          hal[f] = code[f] < 0;
          const int64_t nbe = code[f] >> 2;
          f2[f] = code[f] & 3;
          src[f] = hal[f] ? sH + (-code[f] - 1) * D::HW
                          : ((nbe >= e0 && nbe < e0 + nel) ? sRaw + (nbe - e0) * S : qin + nbe * S);
        }
        if (h == 0) um_flux<N, 0>(G, row, src, hal, f2, c, fl);
        else um_flux<N, 1>(G, row, src, hal, f2, c, fl);
        if (!live) {
#pragma unroll
          for (int f = 0; f < 6; ++f)
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) fl[f][jj] = 0.0f;
        }
      }
      if (!__all_sync(0xffffffffu, um_wait(&mb_p, par))) { failed = true; break; }
      um_fence_after();
      if (h == 0) um_flux_store<N, 0>(tl, fl);
      else um_flux_store<N, 1>(tl, fl);
      um_wait_st();
      um_fence_before();
      um_arrive(&mb_opF);
      // ---- lift products of field `warp` (warps 0-5), once every element's fluxes are in ----
      if (warp < kUmFieldIssuers) {
        if (!__all_sync(0xffffffffu, um_wait(&mb_opF, par))) { failed = true; break; }
        um_fence_after();
        um_mma_field(tm + um_tr<N>(warp), tm + um_tfh<N>(warp), tm + um_tfl<N>(warp), 0u, false, dBL,
                     dBL + (uint64_t)((4 * 16 * KL) >> 4), (uint64_t)((4 * 2 * 16 * 4) >> 4), idR, KL / 8, false, one);
        um_commit_p(&mb_l, one);
        carmed = 2u * one;
      }
      // ---- SARK combination once the lift and the staged rows are in ----
      if (!__all_sync(0xffffffffu, um_wait(&mb_l, par))) { failed = true; break; }
      carmed = 0u;
      if (STAGE >= 0 && !__all_sync(0xffffffffu, um_wait(&mb_qn, par))) { failed = true; break; }
      // (the rhs rows go into sA: the previous tile's stores have read it)
      if (STAGE < 0 && !__all_sync(0xffffffffu, um_wait(&mb_free, par))) { failed = true; break; }
      if (STAGE >= 1 && !__all_sync(0xffffffffu, um_wait(&mb_x, par))) { failed = true; break; }
      um_fence_after();
      {
        float4 *rowq = reinterpret_cast<float4 *>(sA + el * S);
        float4 *row1 = reinterpret_cast<float4 *>(sX1 + el * S);
        float4 *row2 = reinterpret_cast<float4 *>(sX2 + el * S);
        bool bd = false;
#define UM_SARK(ST)                                                                          \
  if (h == 0) um_sark<N, ST, 0>(tl, rowq, row1, row2, k0, k1, dt, bd);                       \
  else um_sark<N, ST, 1>(tl, rowq, row1, row2, k0, k1, dt, bd);
        switch (STAGE) {
          case -1: UM_SARK(-1) break;
          case 0: UM_SARK(0) break;
          case 1: UM_SARK(1) break;
          case 2: UM_SARK(2) break;
          default: UM_SARK(3) break;
        }
#undef UM_SARK
        bad |= live && bd;
      }
      um_fence_async_smem();
      um_fence_before();
      um_arrive(&mb_out);
    }
    if (STAGE == 3 && bad) atomicOr(a.status, GB_STATUS_NAN);
    if (failed) {
      // wait (bounded) for the products this lane issued in the current tile
      if (carmed & 1u) um_wait(&mb_v, par);
      if (carmed & 2u) um_wait(&mb_l, par);
      atomicOr(a.status, GB_STATUS_TIMEOUT);
    }
  }
  if (tid == 0) {   // the set-up copies have landed (at once, unless a wait ran out)
    um_wait(&mb_tab, 0);
    if ((int64_t)blockIdx.x < ntile && failed) um_wait(&mb_ld, 0);
  }
  um_fence_before();
  __syncthreads();
  um_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tm) : "memory");
}

// ---- host side -------------------------------------------------------------------------
namespace {

constexpr int kUmMaxDevices = 64;

template <int N>
int um_launch_one(const StageArgs &a_in, cudaStream_t st, int num_sms) {
  typedef UmDim<N> D;
  StageArgs a = a_in;
  set_mixed_coefs(a);
  // at least 116 KB, so that no two CTAs share an SM: each holds all 512 TMEM columns
  const size_t smem = sizeof(float) * (size_t)D::SM_END > (size_t)116 * 1024 ? sizeof(float) * (size_t)D::SM_END
                                                                                : (size_t)116 * 1024;
  // the shared-memory opt-in is a per-device attribute: set once per device
  static bool attr_set[kUmMaxDevices] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return (int)err;
  if (dev < 0 || dev >= kUmMaxDevices) return (int)cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    err = cudaFuncSetAttribute(um_stage_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    attr_set[dev] = true;
  }
  const int64_t ntile = (a.K + 127) / 128;
  int64_t grid = num_sms < ntile ? num_sms : ntile;
  if (grid < 1) grid = 1;
  um_stage_kernel<N><<<(unsigned)grid, kUmThreads, smem, st>>>(a);
  return (int)cudaGetLastError();
}

template <int N>
int um_launch_n(const StageArgs &a, cudaStream_t st, int num_sms) {
  if (a.stage < -1 || a.stage > 3) return (int)cudaErrorInvalidValue;
  return um_launch_one<N>(a, st, num_sms);
}

float um_tf32_host(double v) {
  // round to nearest, ties away from zero, at 10 explicit mantissa bits (as cvt.rna.tf32.f32)
  float x = (float)v;
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
void um_fill(const RefOps &Rf, std::vector<float> &h) {
  typedef UmDim<N> D;
  constexpr int Np = D::Np, Nc = D::Nc, NFN = D::NFN;
  h.assign(D::BTOT, 0.0f);
  auto put = [&](int base, int rows, int kcols, auto fn) {   // fn(n, k): entry of the rows x kcols operand
    for (int n = 0; n < rows; ++n)
      for (int k = 0; k < kcols; ++k) {
        const double v = fn(n, k);
        const float hi = um_tf32_host(v), lo = um_tf32_host(v - (double)hi);
        const int off = (k / 4) * (rows * 4) + n * 4 + (k % 4);
        h[base + off] = hi;
        h[base + rows * kcols + off] = lo;
      }
  };
  put(D::BV, D::NVC, D::KV, [&](int n, int k) -> double {   // rows: Dr, Ds, I
    if (k >= Np) return 0.0;
    if (n < Np) return Rf.Dr[n * Np + k];
    if (n >= D::KV && n - D::KV < Np) return Rf.Ds[(n - D::KV) * Np + k];
    if (n >= D::NV && n - D::NV < Nc) return Rf.I[(n - D::NV) * Np + k];
    return 0.0;
  });
  put(D::BP, D::NR, D::KC, [&](int o, int k) -> double { return (o < Np && k < Nc) ? Rf.P[o * Nc + k] : 0.0; });
  put(D::BL, D::NR, D::KL, [&](int o, int k) -> double { return (o < Np && k < NFN) ? Rf.LIFT[o * NFN + k] : 0.0; });
  for (int n = 0; n < Np; ++n) {
    h[D::BBAR + 2 * n] = (float)(0.5 * (1.0 + Rf.r[n]));
    h[D::BBAR + 2 * n + 1] = (float)(0.5 * (1.0 + Rf.s[n]));
  }
}

}  // namespace

bool um_supported(int N) { return N >= 1 && N <= 4; }

int launch_stage_um(int N, const StageArgs &a, void *stream, int num_sms) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!a.ops_um || a.bc || (a.stage == 3 && a.rec_every > 0)) return (int)cudaErrorInvalidValue;
  switch (N) {
    case 1: return um_launch_n<1>(a, st, num_sms);
    case 2: return um_launch_n<2>(a, st, num_sms);
    case 3: return um_launch_n<3>(a, st, num_sms);
    case 4: return um_launch_n<4>(a, st, num_sms);
  }
  return (int)cudaErrorInvalidValue;
}

int upload_ops_um(int N, const RefOps &Rf, float **dev_ops, void *stream) {
  std::vector<float> h;
  switch (N) {
    case 1: um_fill<1>(Rf, h); break;
    case 2: um_fill<2>(Rf, h); break;
    case 3: um_fill<3>(Rf, h); break;
    case 4: um_fill<4>(Rf, h); break;
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

}  // namespace gb
