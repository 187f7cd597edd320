// Internal declarations of the 3D (tetrahedral, 10-field) solver: shared by its host
// side (gb3d.cpp) and its kernels (gb_kernels3d.cu).
#ifndef GB3D_INTERNAL_H
#define GB3D_INTERNAL_H

#include <stdint.h>

#include "gb_internal.h"

namespace gb {

// Per-element record, 48 bytes: vertex ids; per face the neighbour packed as
// (element << 5 | permutation code << 2 | face) (permutation codes of kPerm3); the
// periodic shift of each vertex as signed multiples of the periods (x, y, z per vertex).
struct __attribute__((aligned(16))) MeshRec3 {
  int32_t v[4];
  int32_t nbr[4];
  int8_t shift[12];
  int8_t pad[4];
};
static_assert(sizeof(MeshRec3) == 48, "MeshRec3 must be 48 bytes");

// travelling-wave lateral motion of the deforming channel (y displacement only)
struct Wave3 {
  double A0, A1, Lx, wavelength, omega, r0sq, yc, zc;
};

struct Stage3Args {
  const void *qin, *qn;
  void *qout, *F0, *acc, *Fout;
  const double *xn;      // n_vert x 3 current vertex positions
  const double *shape;   // n_vert x 6: velocity shapes S1 (xyz), S2 (xyz)
  const MeshRec3 *mesh;
  const void *ops;       // operator block (T), layout in gb_kernels3d.cu
  const void *ops_tc;    // GB_MIXED, N <= 3: the tensor-core kernel's table (gb_kernels3d_tc.cu), else NULL
  const int *tab;        // neighbour face-node table [4][4][6][Nfp], then fmask [4][Nfp]
  double *clock;         // t_n, then the final vertex-update factors f1, f2
  int *status;
  int64_t K;
  double period[3];
  double c, inv_tau, dt;
  int moving;            // 0: static mesh
  double omega;
  int stage;             // -1: rhs only, 0..3 SARK stage
  double rhs_time;
  SarkCoef co;
};

// inputs of the diagnostics reductions: the canonical state (FP64, or FP32 perturbations
// of the rest state), current vertices, 1^T Mhat, and scratch for 6 doubles per block
struct Diag3Args {
  const void *q;
  bool is_float;
  int Np;
  const MeshRec3 *mesh;
  const double *xn;
  double period[3];
  const double *wq;
  double c;
  int64_t K;
  double *part;
};
constexpr int kDiag3MaxBlocks = 1184;

int launch_stage3(int N, bool fp64, const Stage3Args &a, void *stream, int num_sms);
// the GB_MIXED tensor-core stage kernel (16-element warp tiles, CTAs of
// 1..stage3_tc_max_warps(N) warps)
bool stage3_tc_supported(int N);
int stage3_tc_max_warps(int N);
int launch_stage3_tc(int N, const Stage3Args &a, void *stream, int warps_per_cta, int num_sms);
int upload_ops3_tc(int N, const RefOps3 &R, void **dev, size_t *bytes, void *stream);
int diagnostics3_blocks(int64_t K);
int launch_diagnostics3(const Diag3Args &d, double *out, void *stream);
int launch_diagnostics3_record(const Diag3Args &d, const double *clock, int64_t *ctl, int every, double *hist,
                               int64_t cap, void *stream);
int launch_vertex_update3(double *xn, const double *shape, int64_t nv, double *clock, double dt, void *stream);
int launch_shape3(const double *X, double *shape, int64_t nv, const Wave3 &m, void *stream);
int launch_shape3_tgv(const double *X, double *shape, int64_t nv, double A, double omega, double L, void *stream);
int launch_nodes3(const double *bary, int Np, const double *xn, const MeshRec3 *mesh, const double period[3], int64_t K,
                  double *out, void *stream);
int launch_cast3(double *d, float *f, int64_t K, int Np, bool to_float, void *stream);
int upload_ops3(int N, bool fp64, const RefOps3 &R, void **dev_ops, int **dev_tab, double **dev_bary, size_t *bytes,
                void *stream);

}  // namespace gb

#endif
