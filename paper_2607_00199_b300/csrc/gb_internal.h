// Internal declarations shared by the host API (gb_api.cpp), the reference
// builder (gb_reference.cpp) and the CUDA kernels (gb_kernels.cu).
#ifndef GB_INTERNAL_H
#define GB_INTERNAL_H

#include <stdint.h>

#include <vector>

#include "gb.h"

#define GB_MAX_N 6

// device status bits (OR-ed by the kernels, read by gb_sync / gb_fields)
#define GB_STATUS_NAN  1
#define GB_STATUS_MESH 2
#define GB_STATUS_TIMEOUT 4   // a bounded wait on the tensor cores or a bulk copy ran out

namespace gb {

// Reference operators of order N, FP64, row-major (see gb_reference.cpp).
struct RefOps {
  int N = 0, Np = 0, Nfp = 0, Nc = 0;
  std::vector<double> r, s;      // Np
  std::vector<double> Dr, Ds;    // Np x Np
  std::vector<double> LIFT;      // Np x 3Nfp
  std::vector<double> I, P;      // Nc x Np, Np x Nc
  std::vector<double> cr, cs, cw;
  std::vector<int> fmask;        // 3 x Nfp, counter-clockwise along each face
  std::vector<double> wq;        // Np: 1^T Mhat, integral of each nodal basis function
};

bool build_reference(int N, RefOps &R);

// Reference operators of the tetrahedron (3D, 10 fields), FP64, row-major.
#define GB3_MAX_N 4
struct RefOps3 {
  int N = 0, Np = 0, Nfp = 0, Nc = 0;
  std::vector<double> r, s, t;        // Np
  std::vector<double> Dr, Ds, Dt;     // Np x Np
  std::vector<double> LIFT;           // Np x 4 Nfp (parameter measure: every face has area 2)
  std::vector<double> I, P;           // Nc x Np, Np x Nc
  std::vector<double> cr, cs, ct, cw; // Nc
  std::vector<double> wq;             // Np: 1^T Mhat
  std::vector<double> bary;           // Np x 4
  std::vector<int> fmask;             // 4 x Nfp, increasing volume index
  std::vector<int> nbr_node;          // [f][f2][perm][k]: neighbour volume node of my face node k
};
// the six permutations of a face's three vertices, in a fixed order: code p maps my
// face vertex i to the neighbour's face vertex kPerm3[p][i]
static const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
bool build_reference3d(int N, RefOps3 &R);
void sark_coefficients(double gamma, double E[5], double A[16], double B[4]);

// Per-element mesh record, 32 bytes: vertex ids, face neighbours packed as
// (neighbour element << 2 | neighbour face) or, for a boundary face, -1 (wall) or -2
// (far field), and periodic shifts of the three vertices as signed multiples of the
// periods (x then y per vertex).
struct __attribute__((aligned(16))) MeshRec {
  int32_t v[3];
  int32_t nbr[3];
  int8_t shift[6];
  int8_t pad[2];
};
static_assert(sizeof(MeshRec) == 32, "MeshRec must be 32 bytes");

// SARK coefficients for the two field classes (0: fields 1-3, gamma = 0;
// 1: fields 4-6, gamma = -dt/tau), plus the RK4 vertex tableau factors.
struct SarkCoef {
  double E[2][5];
  double A[2][16];
  double B[2][4];
};

// Everything a stage kernel needs, passed by value.
struct StageArgs {
  const void *qin;      // q_i: self values and neighbour traces
  const void *qn;       // q_n
  void *qout;           // q_{i+1}, or q_{n+1} at the last stage (may alias qn)
  void *F0;             // F_0 (written at stage 0, read at stages 1-2)
  void *acc;            // running btilde combination
  void *Fout;           // right-hand side output (rhs-only mode)
  const double *xn;     // current vertex positions, n_vert x 2
  const double *shape;  // vertex velocity shape S(X), n_vert x 2
  const MeshRec *mesh;
  const double *ops;    // device copy of the operators (layout in gb_kernels.cu)
  const float *ops_um;  // GB_MIXED, N <= 4: operator tables of the tcgen05 kernel (layout in gb_kernels_um.cu)
  const double *clock;  // device time t_n
  int *status;
  int64_t K;
  double period[2];
  double c, inv_tau;
  double dt;
  // grid velocity of stage i at a vertex: gfac[i] * S(X); stage position
  // x_i = x_n + xfac[i] * S(X).  Derived per block from the clock.
  double motion_A, motion_w;   // A and 2 pi / T (A = 0: static)
  int stage;                   // -1: rhs only, 0..3: SARK stage
  int warps_per_cta;           // GB_MIXED launch shape (1, 2 or 4; 0 = 4), chosen by the tuner
  double rhs_time;             // rhs-only mode: evaluate the grid velocity at this time
  SarkCoef co;
  // GB_MIXED: this stage's SARK coefficients in FP32 per field class (E, A_a, A_b, B_a, B_b,
  // see set_mixed_coefs), so that the kernel converts nothing from FP64
  float kco[2][5];
  // boundary faces (nbr < 0: -1 wall, -2 far field) present; far-field state q_inf in the
  // field representation of the kernel (FP64 full state, or FP32 perturbation)
  int bc;
  double far[6];
  float farf[6];
  // diagnostics fused into the last stage (rec_every > 0): on every rec_every-th step the
  // stage-3 kernel integrates mass, E_K, momentum and area of q_{n+1} on x_{n+1} (weights
  // rec_wq = 1^T Mhat), leaves per-CTA partials in rec_part and the last CTA to finish writes
  // the record (t, mass, E_K, momentum x, y, area) into the ring rec_hist of rec_cap records;
  // rec_ctl = (steps since enabled, records written), rec_done a CTA counter (zero between launches)
  int rec_every;
  int64_t rec_cap;
  const double *rec_wq;
  double *rec_part;
  unsigned *rec_done;
  int64_t *rec_ctl;
  double *rec_hist;
};

// Perfectly matched layer (gb_pml.cu): the layer's elements and auxiliary fields, in the
// representation of the stage kernels (T = double for GB_FP64, float for GB_MIXED)
struct PmlArgs {
  const void *ops;              // Dr^T, Ds^T, LIFT^T, node barycentrics (T; layout in gb_pml.cu)
  const int32_t *elem;          // n_layer element indices in the kernels' numbering
  const void *node;             // n_layer x 3 x Np (T): sigma, e_x, e_y at every node
  void *phin, *phis, *phiacc;   // n_layer x 6 x Np (T): Phi_n, the stage value, the RK4 sum
  int64_t n_layer;
  int64_t stride;               // element stride of the field arrays
  double alpha;                 // frequency shift
  double cq[2], cs[2];          // per field class: the coefficient of F_i in q_{i+1} (times dt)
                                // and in the stored F_0 / accumulator, for this stage
};
int launch_pml_stage(int N, bool fp64, const StageArgs &a, const PmlArgs &p, void *stream, int num_sms);
int pml_ops_size(int N);

// element stride (floats) of the GB_MIXED field layout: the smallest s >= x with s = 4 mod 8
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int tc_round_s(int x) { return ((x - 4 + 7) / 8) * 8 + 4; }   // smallest s >= x, s = 4 mod 8

#ifdef __CUDACC__
// volume index of node k (counter-clockwise) of face f of the reference triangle of order N
template <int N>
__device__ __forceinline__ int tc_fmask(int f, int k) {
  constexpr int NN = N;
  auto rs = [](int j) { return j * (NN + 1) - j * (j - 1) / 2; };
  return f == 0 ? k : (f == 1 ? rs(k) + (NN - k) : rs(NN - k));
}

// motion factors of a stage for one request: v_i = gfac S(X), x_i = x_n + xfac S(X),
// and the factor of the final vertex update x_{n+1} = x_n + fin S(X) (RK4 nodes and weights)
template <int STAGE>
__device__ __forceinline__ void tc_stage_motion(const StageArgs &a, double &gf, double &xf, double &fin) {
  gf = 0.0; xf = 0.0; fin = 0.0;
  if (a.motion_A == 0.0) return;
  const double w = a.motion_w, Aw = a.motion_A * a.motion_w;
  if (STAGE < 0) {
    gf = Aw * cos(w * a.rhs_time);
    return;
  }
  const double tt = a.clock[0], dt = a.dt;
  const double cst[4] = {0.0, 0.5, 0.5, 1.0};
  gf = Aw * cos(w * (tt + cst[STAGE] * dt));
  if (STAGE > 0) xf = dt * cst[STAGE == 3 ? 3 : 1] * Aw * cos(w * (tt + cst[STAGE - 1] * dt));
  if (STAGE == 3) fin = dt * Aw * (cos(w * tt) / 6.0 + cos(w * (tt + 0.5 * dt)) * (2.0 / 3.0) + cos(w * (tt + dt)) / 6.0);
}

#endif

// most CTAs of a launch with the fused record (the size of its partials buffer)
constexpr int kRecMaxCtas = 1184;

// Fused diagnostics: every CTA of a stage-3 launch calls this once at its end with its
// threads' partial sums (mass, kinetic energy, momentum x, y, area); the last CTA to finish
// sums the per-CTA partials in CTA order (so the result does not depend on scheduling),
// writes the record and advances the step counter.  Requires blockDim.x <= 1024 and a
// multiple of 32; all threads of the CTA must call it.
#ifdef __CUDACC__
__device__ __forceinline__ void fused_record(const StageArgs &a, bool record, double (&acc)[5], double t_next) {
  __shared__ double red[32][5];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (record) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      double v = acc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (record)
      for (int k = 0; k < 5; ++k) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += red[w][k];
        a.rec_part[5 * blockIdx.x + k] = v;
      }
    __threadfence();
    last = atomicAdd(a.rec_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    if (record) {
      double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (unsigned b = 0; b < gridDim.x; ++b)
        for (int k = 0; k < 5; ++k) tot[k] += ((volatile double *)a.rec_part)[5 * b + k];
      double *r = a.rec_hist + 6 * (a.rec_ctl[1] % a.rec_cap);
      r[0] = t_next;
      r[1] = tot[0];
      r[2] = tot[1] / tot[4];
      r[3] = tot[2];
      r[4] = tot[3];
      r[5] = tot[4];
      a.rec_ctl[1] += 1;
    }
    a.rec_ctl[0] += 1;
    *a.rec_done = 0u;
  }
}
#endif

// Several requests (solvers) of one order stepped by one launch per stage:
// args[r] are their stage arguments, tile_start the exclusive prefix of their
// 16-element tile counts (n + 1 entries), vtx_start the prefix of their vertex
// counts (n + 1 entries); all three arrays live in device memory.
struct GroupArgs {
  const StageArgs *args;
  const int64_t *tile_start;
  const int64_t *vtx_start;
  int n;
  int64_t total_tiles;
  int64_t total_vertices;
  const void *ops;
  int warps;   // warps per CTA of the group kernel (1, 2 or 4), chosen by the group tuner
};

// Launchers (gb_kernels.cu).  Return a cudaError_t value as int.
int launch_stage_fp64(int N, const StageArgs &a, void *stream, int num_sms);
int launch_stage_mixed(int N, const StageArgs &a, void *stream, int num_sms);
int launch_vertex_update(const StageArgs &a, int64_t n_vert, void *stream);
int launch_shape(const double *X, double *shape, int64_t n_vert, int kind, double Lx, double Ly, void *stream);
int launch_nodes(int N, const double *ops, const double *xn, const MeshRec *mesh, double px, double py,
                 int64_t K, double *out, void *stream);
int launch_relayout(const void *canon_src, void *canon_dst, bool canon_is_double, bool to_internal, float *inner,
                    const int32_t *perm, int64_t K, int Np, int S, double rest, void *stream);
int mixed_stride(int N);   // element stride (floats) of the GB_MIXED field layout
void set_mixed_coefs(StageArgs &a);   // fill a.kco from a.co and a.stage (host)
// integrals over the mesh at the current vertices: out[0] = int rho, out[1] = int rho |u|^2 / 2,
// out[2] = int rho u, out[3] = int rho v, out[4] = area; fields of element e at
// q[e * stride + f * Np + n] (+ 1 on field 1 when perturbation), FP64 or FP32
// part: diagnostics_scratch_doubles() doubles of block partials; out: 5 doubles (device)
int launch_diagnostics(int N, const void *q, bool is_float, bool perturbation, int64_t stride, const MeshRec *mesh,
                       const double *xn, double px, double py, const double *wq, double c, int64_t K, double *part,
                       double *out, void *stream);
int diagnostics_scratch_doubles();
// the same integrals recorded on the device every `every` steps (ctl: int64 step and
// record counters; hist: cap records of 6 doubles t, mass, E_K, momentum x, y, area)
int launch_diagnostics_record(int N, const void *q, bool is_float, bool perturbation, int64_t stride,
                              const MeshRec *mesh, const double *xn, double px, double py, const double *wq, double c,
                              int64_t K, double *part, const double *clock, int64_t *ctl, int every, double *hist,
                              int64_t cap, void *stream);
int launch_group_mixed(int N, int stage, const GroupArgs &g, void *stream, int num_sms);
// GB_MIXED on the tcgen05 tensor cores (gb_kernels_um.cu): 128-element CTA tiles, orders 1..4,
// meshes without boundary faces, no fused diagnostics; selected by warps_per_cta == kShapeUm
constexpr int kShapeUm = 8;
bool um_supported(int N);
int launch_stage_um(int N, const StageArgs &a, void *stream, int num_sms);
int upload_ops_um(int N, const RefOps &R, float **dev_ops, void *stream);
int launch_group_vertex_update(const GroupArgs &g, void *stream);
// the solver's rhs-only launch arguments, its device buffers' layout, stream and device ordinal
int rhs_launch_view(gb_solver *s, double t, StageArgs *a, const int32_t **perm, int *N, int64_t *K, int *Np,
                    int *precision, void **stream, int *num_sms, int *device);
int set_solver_error(gb_solver *s, int code, const char *msg);
int upload_ops(int N, const RefOps &R, double **dev_ops, void *stream);
int upload_ops_mixed(int N, const RefOps &R, float **dev_ops, void *stream);

}  // namespace gb

#endif
