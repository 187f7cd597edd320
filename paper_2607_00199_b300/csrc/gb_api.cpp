// C ABI of libgb (declared in include/gb.h): solver lifetime, mesh validation
// and connectivity, state transfer, and the SARK step driver (Sec. 4) that
// enqueues the fused stage kernels of gb_kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "gb.h"
#include "gb_internal.h"
#include "gb3d.h"

#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>

using gb::MeshRec;

struct gb_solver {
  gb::Solver3 *s3 = nullptr;   // set for dim = 3 solvers: every call routes to gb3d.cpp
  int N = 0, Np = 0, Nfp = 0, Nc = 0, precision = GB_FP64;
  int64_t K = 0, nv = 0;
  double c = 0, tau = 0, period[2] = {0, 0};
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  int device = 0;              // CUDA device ordinal current at gb_create: all of the solver's memory lives there
  std::string err;
  gb::RefOps ref;
  gb_motion motion{GB_MOTION_STATIC, 0, 1, 1, 1};
  double coef_dt = -1.0;
  // one SARK step captured as a CUDA graph (gb_step); rebuilt when dt, the motion or the stream change
  cudaGraphExec_t step_graph = nullptr;
  double graph_dt = -1.0;
  bool graph_warm = false;     // one uncaptured step ran with the current settings
  bool use_graph = true;
  int warps = 0;               // GB_MIXED warps per CTA chosen by tune_launch (0 = not tuned yet)
  gb::SarkCoef co{};
  size_t elem_bytes = 8;
  // device memory
  double *d_ops = nullptr;     // FP64 operator block (canonical kernel, node coordinates)
  float *d_ops_mixed = nullptr;  // FP32 operator block of the GB_MIXED kernel
  float *d_ops_um = nullptr;     // GB_MIXED, N <= 4, no boundary faces: tables of the tcgen05 kernel
  MeshRec *d_mesh = nullptr;     // canonical element order
  MeshRec *d_mesh_int = nullptr; // GB_MIXED: Morton element order, neighbours renumbered
  int32_t *d_perm = nullptr;     // GB_MIXED: canonical index of internal element i
  double *d_X = nullptr, *d_xn = nullptr, *d_shape = nullptr, *d_clock = nullptr;
  int *d_status = nullptr;
  void *d_qn = nullptr, *d_b1 = nullptr, *d_b2 = nullptr, *d_F0 = nullptr, *d_acc = nullptr;
  double *d_tmp = nullptr;     // FP64 staging (GB_MIXED transfers, node coordinates)
  double *d_diag = nullptr;    // 1^T Mhat (Np), 5 result slots, block partials
  // recorded diagnostics: every diag_every steps into a ring of diag_cap records
  int diag_every = 0;
  int64_t diag_cap = 0;
  double *d_hist = nullptr;
  int64_t *d_hctl = nullptr;   // steps since enabled, records written
  unsigned *d_done = nullptr;  // CTA counter of the fused record (zero between launches)
  size_t tmp_bytes = 0;
  int64_t device_bytes = 0;
  int has_bc = 0;              // the mesh has wall / far-field faces (gb_create_bounded)
  double far[6] = {0, 0, 0, 0, 0, 0};   // far-field state in the kernels' representation
  // perfectly matched layer (gb_set_pml): layer elements in ascending canonical order
  int64_t n_layer = 0;
  double pml_alpha = 0.0;
  void *d_pml_ops = nullptr, *d_pml_node = nullptr, *d_phi = nullptr;   // d_phi: Phi_n, stage, RK4 sum
  int32_t *d_pml_elem = nullptr;
  size_t pml_bytes = 0;
};

static std::string g_create_error;

static int fail(gb_solver *s, int code, const std::string &msg) {
  if (s) s->err = msg; else g_create_error = msg;
  return code;
}

static int cuda_fail(gb_solver *s, cudaError_t e, const char *where) {
  return fail(s, GB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static int dev_alloc(gb_solver *s, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(s, GB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  s->device_bytes += (int64_t)bytes;
  return GB_OK;
}

static void free_all(gb_solver *s) {
  void *ptrs[] = {s->d_ops, s->d_ops_mixed, s->d_ops_um, s->d_mesh, s->d_mesh_int, s->d_perm, s->d_X, s->d_xn, s->d_shape,
                  s->d_clock, s->d_status, s->d_qn, s->d_b1, s->d_b2, s->d_F0, s->d_acc, s->d_tmp, s->d_diag,
                  s->d_hist, s->d_hctl, s->d_done, s->d_pml_ops, s->d_pml_node, s->d_phi, s->d_pml_elem};
  for (void *p : ptrs)
    if (p) cudaFree(p);
}

static void dev_free(gb_solver *s, void **p, size_t bytes) {
  if (*p) {
    cudaFree(*p);
    s->device_bytes -= (int64_t)bytes;
    *p = nullptr;
  }
}

// integration weights and scratch of the diagnostics (allocated on first use)
static int ensure_diag(gb_solver *s) {
  if (s->d_diag) return GB_OK;
  int rc = dev_alloc(s, (void **)&s->d_diag, sizeof(double) * (s->Np + 5 + gb::diagnostics_scratch_doubles()));
  if (!rc) rc = dev_alloc(s, (void **)&s->d_done, sizeof(unsigned));
  if (rc) return rc;
  cudaError_t ze = cudaMemsetAsync(s->d_done, 0, sizeof(unsigned), s->stream);
  if (ze != cudaSuccess) return cuda_fail(s, ze, "diagnostics counter");
  cudaError_t ce = cudaMemcpyAsync(s->d_diag, s->ref.wq.data(), sizeof(double) * s->Np, cudaMemcpyHostToDevice, s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail(s, ce, "diagnostics weights");
}

// after a step: the recorded diagnostics, when enabled
static int record_diagnostics(gb_solver *s, void *stream) {
  if (s->diag_every <= 0) return GB_OK;
  const bool mixed = s->precision == GB_MIXED;
  const int64_t stride = mixed ? gb::mixed_stride(s->N) : 6 * s->Np;
  int lr = gb::launch_diagnostics_record(s->N, s->d_qn, mixed, mixed, stride, mixed ? s->d_mesh_int : s->d_mesh, s->d_xn,
                                         s->period[0], s->period[1], s->d_diag, s->c, s->K, s->d_diag + s->Np + 5,
                                         s->d_clock, s->d_hctl, s->diag_every, s->d_hist, s->diag_cap, stream);
  return lr ? cuda_fail(s, (cudaError_t)lr, "diagnostics record launch") : GB_OK;
}

static int ensure_tmp(gb_solver *s, size_t bytes) {
  if (s->tmp_bytes >= bytes) return GB_OK;
  if (s->d_tmp) {
    cudaFree(s->d_tmp);
    s->device_bytes -= (int64_t)s->tmp_bytes;
    s->d_tmp = nullptr;
    s->tmp_bytes = 0;
  }
  int rc = dev_alloc(s, (void **)&s->d_tmp, bytes);
  if (rc == GB_OK) s->tmp_bytes = bytes;
  return rc;
}

static gb::StageArgs base_args(gb_solver *s) {
  gb::StageArgs a;
  memset(&a, 0, sizeof(a));
  a.xn = s->d_xn;
  a.shape = s->d_shape;
  const bool mixed = s->precision == GB_MIXED;
  a.mesh = mixed ? s->d_mesh_int : s->d_mesh;
  a.ops = mixed ? reinterpret_cast<const double *>(s->d_ops_mixed) : s->d_ops;
  a.ops_um = mixed ? s->d_ops_um : nullptr;
  a.clock = s->d_clock;
  a.status = s->d_status;
  a.K = s->K;
  a.period[0] = s->period[0];
  a.period[1] = s->period[1];
  a.c = s->c;
  a.inv_tau = 1.0 / s->tau;
  const bool moving = s->motion.kind == GB_MOTION_SINXY || s->motion.kind == GB_MOTION_PLUNGE;
  a.motion_A = moving ? s->motion.A : 0.0;
  a.motion_w = moving ? 2.0 * M_PI / s->motion.T : 0.0;
  a.bc = s->has_bc;
  memcpy(a.far, s->far, sizeof(a.far));
  a.co = s->co;
  a.warps_per_cta = s->warps;
  return a;
}

static int launch_stage(gb_solver *s, const gb::StageArgs &a) {
  int rc = s->precision == GB_FP64 ? gb::launch_stage_fp64(s->N, a, s->stream, s->num_sms)
                                   : gb::launch_stage_mixed(s->N, a, s->stream, s->num_sms);
  if (rc != 0) return cuda_fail(s, (cudaError_t)rc, "stage kernel launch");
  return GB_OK;
}

// the layer's terms of SARK stage a.stage (after the stage kernel, before the next one)
static int launch_pml(gb_solver *s, const gb::StageArgs &a) {
  if (s->n_layer <= 0) return GB_OK;
  const bool fp64 = s->precision == GB_FP64;
  const size_t eb = fp64 ? sizeof(double) : sizeof(float);
  const size_t phi_elems = (size_t)s->n_layer * 6 * s->Np;
  gb::PmlArgs p;
  memset(&p, 0, sizeof(p));
  p.ops = s->d_pml_ops;
  p.elem = s->d_pml_elem;
  p.node = s->d_pml_node;
  p.phin = s->d_phi;
  p.phis = (char *)s->d_phi + eb * phi_elems;
  p.phiacc = (char *)s->d_phi + 2 * eb * phi_elems;
  p.n_layer = s->n_layer;
  p.stride = fp64 ? 6 * s->Np : gb::mixed_stride(s->N);
  p.alpha = s->pml_alpha;
  // coefficients of F_i in stage i's combinations (as the stage kernels form them)
  for (int cl = 0; cl < 2; ++cl) {
    const double *A = s->co.A[cl], *B = s->co.B[cl];
    switch (a.stage) {
      case 0: p.cq[cl] = A[4]; p.cs[cl] = 1.0; break;
      case 1: p.cq[cl] = A[9]; p.cs[cl] = B[1]; break;
      case 2: p.cq[cl] = A[14]; p.cs[cl] = B[2]; break;
      default: p.cq[cl] = B[3]; p.cs[cl] = 0.0; break;
    }
  }
  int rc = gb::launch_pml_stage(s->N, fp64, a, p, s->stream, s->num_sms);
  return rc ? cuda_fail(s, (cudaError_t)rc, "layer kernel launch") : GB_OK;
}

struct gb_group {
  int capacity = 0, num_sms = 1, device = 0;
  int warps[GB_MAX_N + 1] = {};   // group-kernel warps per CTA last used for each order (0: none yet)
  bool fixed[GB_MAX_N + 1] = {};  // set by gb_group_set_launch_config: no tuning for that order
  cudaStream_t stream = nullptr;
  gb::StageArgs *d_args = nullptr, *h_args = nullptr;   // [4][capacity]
  int64_t *d_prefix = nullptr, *h_prefix = nullptr;     // tile prefix (n+1), then vertex prefix (n+1)
  cudaEvent_t uploaded = nullptr;
  std::string err;
};

// SARK coefficients of both field classes for step size dt (cached per solver)
static void set_coefficients(gb_solver *s, double dt) {
  if (dt == s->coef_dt) return;
  double E[5], A[16], B[4];
  gb::sark_coefficients(0.0, E, A, B);
  memcpy(s->co.E[0], E, sizeof(E)); memcpy(s->co.A[0], A, sizeof(A)); memcpy(s->co.B[0], B, sizeof(B));
  gb::sark_coefficients(-dt / s->tau, E, A, B);
  memcpy(s->co.E[1], E, sizeof(E)); memcpy(s->co.A[1], A, sizeof(A)); memcpy(s->co.B[1], B, sizeof(B));
  s->coef_dt = dt;
}

// Launch-shape tuner (GB_MIXED): warps per CTA, 1, 2 or 4.  Fewer warps per CTA
// spread the 16-element tiles of a small mesh over more SMs; more warps share one
// copy of the operator tables.  The tuner times the rhs-only stage
// kernel (which writes only the scratch buffer b2 and leaves the state alone) on
// the solver's own data for each shape and keeps the fastest; a candidate after
// the first must win by 3%.  Choices are cached per (device, N, size class of K) for the process.
static std::mutex g_tune_mu;
typedef std::tuple<int, int, int64_t> TuneKey;   // (device, N, size class)
static std::map<TuneKey, int> g_tuned;           // -> solver launch shape
static std::map<TuneKey, int> g_group_tuned;     // (device, N, tile-count class) -> group warps per CTA

// size class of a mesh or a group: the bit length of (count - 1), i.e. counts in (2^(c-1), 2^c]
static int64_t k_class(int64_t count) {
  int64_t c = 0;
  for (int64_t x = count - 1; x > 0; x >>= 1) ++c;
  return c;
}

static int tune_launch(gb_solver *s) {
  if (s->precision != GB_MIXED || s->warps != 0) return GB_OK;
  const TuneKey key(s->device, s->N, k_class(s->K));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      s->warps = it->second;
      return GB_OK;
    }
  }
  gb::StageArgs a = base_args(s);
  a.stage = -1;
  a.qin = s->d_qn;
  a.qn = s->d_qn;
  a.Fout = s->d_b2;
  a.rhs_time = 0.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  // candidates: the tcgen05 kernel's 128-element CTA tiles where it applies, then the
  // mma.sync kernel's 16-element warp tiles with 4, 2 or 1 warps per CTA; a later candidate
  // must beat the best so far by 3%
  int cand[4], ncand = 0;
  if (s->d_ops_um) cand[ncand++] = gb::kShapeUm;
  cand[ncand++] = 4;
  cand[ncand++] = 2;
  cand[ncand++] = 1;
  int best = cand[0];
  float best_ms = 1e30f;
  for (int i = 0; i < ncand && ce == cudaSuccess; ++i) {
    a.warps_per_cta = cand[i];
    int rc = gb::launch_stage_mixed(s->N, a, s->stream, s->num_sms);   // warm-up
    if (rc) { ce = (cudaError_t)rc; break; }
    ce = cudaEventRecord(e0, s->stream);
    for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {
      rc = gb::launch_stage_mixed(s->N, a, s->stream, s->num_sms);
      if (rc) ce = (cudaError_t)rc;
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s->stream);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess && ms < 0.97f * best_ms) {
      best_ms = ms;
      best = cand[i];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "launch tuning");
  s->warps = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best;
  return GB_OK;
}

static void drop_graph(gb_solver *s) {
  if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
  s->step_graph = nullptr;
  s->graph_dt = -1.0;
  s->graph_warm = false;
}

// Morton (Z-order) numbering of the element centroids: internal element i is
// canonical element perm[i].  Keeps face neighbours close in memory.
static std::vector<int32_t> morton_order(const std::vector<double> &cx, const std::vector<double> &cy) {
  const size_t K = cx.size();
  double x0 = cx[0], x1 = cx[0], y0 = cy[0], y1 = cy[0];
  for (size_t i = 0; i < K; ++i) {
    x0 = std::min(x0, cx[i]); x1 = std::max(x1, cx[i]);
    y0 = std::min(y0, cy[i]); y1 = std::max(y1, cy[i]);
  }
  const double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
  auto spread = [](uint32_t v) {
    v &= 0xffff;
    v = (v | (v << 8)) & 0x00ff00ff;
    v = (v | (v << 4)) & 0x0f0f0f0f;
    v = (v | (v << 2)) & 0x33333333;
    v = (v | (v << 1)) & 0x55555555;
    return v;
  };
  std::vector<std::pair<uint32_t, int32_t>> key(K);
  for (size_t i = 0; i < K; ++i) {
    uint32_t ix = (uint32_t)((cx[i] - x0) * sx), iy = (uint32_t)((cy[i] - y0) * sy);
    key[i] = {spread(ix) | (spread(iy) << 1), (int32_t)i};
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> perm(K);
  for (size_t i = 0; i < K; ++i) perm[i] = key[i].second;
  return perm;
}

static int create2d(const gb_mesh *mesh, const int8_t *face_bc, const double *far_state, int N, double Ma, double Re,
                    int precision, void *cuda_stream, gb_solver **out);

extern "C" {

int gb_create_bounded(const gb_mesh *mesh, const int8_t *face_bc, const double *far_state, int N, double Ma,
                      double Re, int precision, void *cuda_stream, gb_solver **out) {
  if (!out) return fail(nullptr, GB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !face_bc || !far_state) return fail(nullptr, GB_EINVAL, "mesh, face_bc or far_state is NULL");
  if (mesh->dim != 2) return fail(nullptr, GB_EINVAL, "gb_create_bounded: dim must be 2");
  if (N < 1 || N > 4) return fail(nullptr, GB_EINVAL, "gb_create_bounded: N must be in 1..4");
  if (!(far_state[0] > 0.0) || !std::isfinite(far_state[0]) || !std::isfinite(far_state[1]) || !std::isfinite(far_state[2]))
    return fail(nullptr, GB_EINVAL, "far_state must be finite with rho > 0");
  return create2d(mesh, face_bc, far_state, N, Ma, Re, precision, cuda_stream, out);
}

int gb_create(const gb_mesh *mesh, int N, double Ma, double Re, int precision, void *cuda_stream, gb_solver **out) {
  if (!out) return fail(nullptr, GB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !mesh->X || !mesh->EToV) return fail(nullptr, GB_EINVAL, "mesh, X or EToV is NULL");
  if (mesh->dim != 2 && mesh->dim != 3) return fail(nullptr, GB_EINVAL, "dim must be 2 or 3");
  if (mesh->n_vert <= 0 || mesh->n_elem <= 0) return fail(nullptr, GB_EINVAL, "empty mesh");
  if (mesh->n_elem >= (int64_t(1) << 29)) return fail(nullptr, GB_EINVAL, "n_elem must be < 2^29");
  if (mesh->n_vert >= (int64_t(1) << 31)) return fail(nullptr, GB_EINVAL, "n_vert must be < 2^31");
  if (N < 1 || N > GB_MAX_N) return fail(nullptr, GB_EINVAL, "N must be in 1..6");
  if (!(Ma > 0.0) || !(Re > 0.0) || !std::isfinite(Ma) || !std::isfinite(Re))
    return fail(nullptr, GB_EINVAL, "Ma and Re must be positive and finite");
  if (precision != GB_FP64 && precision != GB_MIXED) return fail(nullptr, GB_EINVAL, "precision must be GB_FP64 or GB_MIXED");
  if (mesh->dim == 3) {
    gb::Solver3 *s3 = nullptr;
    std::string err;
    int rc = gb::s3_create(mesh, N, Ma, Re, precision, cuda_stream, &s3, err);
    if (rc != GB_OK) return fail(nullptr, rc, err);
    gb_solver *s = new gb_solver();
    s->s3 = s3;
    s->N = N;
    s->precision = precision;
    s->K = mesh->n_elem;
    s->nv = mesh->n_vert;
    *out = s;
    return GB_OK;
  }
  return create2d(mesh, nullptr, nullptr, N, Ma, Re, precision, cuda_stream, out);
}

}  // extern "C"

static int create2d(const gb_mesh *mesh, const int8_t *face_bc, const double *far_state, int N, double Ma, double Re,
                    int precision, void *cuda_stream, gb_solver **out) {
  if (!mesh->X || !mesh->EToV) return fail(nullptr, GB_EINVAL, "mesh, X or EToV is NULL");
  if (mesh->n_vert <= 0 || mesh->n_elem <= 0) return fail(nullptr, GB_EINVAL, "empty mesh");
  if (mesh->n_elem >= (int64_t(1) << 29)) return fail(nullptr, GB_EINVAL, "n_elem must be < 2^29");
  if (!(Ma > 0.0) || !(Re > 0.0) || !std::isfinite(Ma) || !std::isfinite(Re))
    return fail(nullptr, GB_EINVAL, "Ma and Re must be positive and finite");
  if (precision != GB_FP64 && precision != GB_MIXED) return fail(nullptr, GB_EINVAL, "precision must be GB_FP64 or GB_MIXED");
  const int64_t K = mesh->n_elem, nv = mesh->n_vert;
  for (int64_t i = 0; i < 3 * K; ++i)
    if (mesh->EToV[i] < 0 || mesh->EToV[i] >= nv) return fail(nullptr, GB_EINVAL, "EToV entry out of range");

  // periods and integer shift codes
  std::vector<double> sh(6 * K, 0.0);
  if (mesh->elem_shift) memcpy(sh.data(), mesh->elem_shift, sizeof(double) * 6 * K);
  double period[2] = {0.0, 0.0};
  for (int64_t i = 0; i < 6 * K; ++i) {
    double v = fabs(sh[i]);
    int d = (int)(i & 1);
    if (!std::isfinite(sh[i])) return fail(nullptr, GB_EINVAL, "non-finite elem_shift");
    if (v > 0.0 && (period[d] == 0.0 || v < period[d])) period[d] = v;
  }
  std::vector<MeshRec> rec(K);
  for (int64_t e = 0; e < K; ++e) {
    MeshRec &r = rec[e];
    memset(&r, 0, sizeof(r));
    for (int k = 0; k < 3; ++k) r.v[k] = mesh->EToV[3 * e + k];
    for (int k = 0; k < 6; ++k) {
      double p = period[k & 1];
      double v = sh[6 * e + k];
      long m = p > 0.0 ? lround(v / p) : 0;
      if (labs(m) > 7 || fabs(v - m * p) > 1e-12 * (1.0 + fabs(v)))
        return fail(nullptr, GB_EINVAL, "elem_shift entries must be small integer multiples of one period per direction");
      r.shift[k] = (int8_t)m;
    }
  }
  auto vx = [&](int64_t e, int k, int d) { return mesh->X[2 * (int64_t)rec[e].v[k] + d] + rec[e].shift[2 * k + d] * period[d]; };
  // positive orientation (Sec. 3: all elements positively oriented)
  for (int64_t e = 0; e < K; ++e) {
    double J = (vx(e, 1, 0) - vx(e, 0, 0)) * (vx(e, 2, 1) - vx(e, 0, 1)) - (vx(e, 2, 0) - vx(e, 0, 0)) * (vx(e, 1, 1) - vx(e, 0, 1));
    if (!(J > 0.0)) {
      char buf[128];
      snprintf(buf, sizeof(buf), "element %lld is not positively oriented (J <= 0)", (long long)e);
      return fail(nullptr, GB_EMESH, buf);
    }
  }
  // face connectivity: face f of element e runs from local vertex f to f+1;
  // every unordered vertex pair must occur on exactly two faces
  std::unordered_map<uint64_t, int64_t> first;   // key -> 3 e + f of the first face, -1 once paired
  first.reserve((size_t)(3 * K));
  int has_bc = 0;
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 3; ++f) {
      if (face_bc && face_bc[3 * e + f] != GB_BC_INTERIOR) {
        const int b = face_bc[3 * e + f];
        if (b != GB_BC_WALL && b != GB_BC_FARFIELD) return fail(nullptr, GB_EINVAL, "face_bc entries must be 0, 1 or 2");
        rec[e].nbr[f] = -b;
        has_bc = 1;
        continue;
      }
      uint64_t a = (uint32_t)rec[e].v[f], b = (uint32_t)rec[e].v[(f + 1) % 3];
      if (a == b) return fail(nullptr, GB_EMESH, "degenerate face (repeated vertex id)");
      uint64_t key = a < b ? (a << 32 | b) : (b << 32 | a);
      auto it = first.find(key);
      if (it == first.end()) {
        first.emplace(key, e * 3 + f);
        continue;
      }
      if (it->second < 0) return fail(nullptr, GB_EMESH, "a face is shared by more than two elements");
      const int64_t e2 = it->second / 3;
      const int f2 = (int)(it->second % 3);
      it->second = -1;
      // opposite traversal and a single translation between the two copies of the edge
      if (rec[e2].v[f2] != rec[e].v[(f + 1) % 3] || rec[e2].v[(f2 + 1) % 3] != rec[e].v[f])
        return fail(nullptr, GB_EMESH, "neighbouring elements are not consistently oriented");
      for (int d = 0; d < 2; ++d) {
        double ta = vx(e, f, d) - vx(e2, (f2 + 1) % 3, d);
        double tb = vx(e, (f + 1) % 3, d) - vx(e2, f2, d);
        if (fabs(ta - tb) > 1e-9 * (1.0 + fabs(period[d]))) return fail(nullptr, GB_EMESH, "periodic face copies do not match");
      }
      rec[e].nbr[f] = (int32_t)((e2 << 2) | f2);
      rec[e2].nbr[f2] = (int32_t)((e << 2) | f);
    }
  for (const auto &kv : first)
    if (kv.second >= 0)
      return fail(nullptr, GB_EMESH, face_bc ? "an interior face has no neighbour (tag boundary faces in face_bc)"
                                             : "the mesh is not closed: a face has no neighbour (only periodic meshes are "
                                               "supported by gb_create; see gb_create_bounded)");

  gb_solver *s = new gb_solver();
  s->N = N;
  s->Np = (N + 1) * (N + 2) / 2;
  s->Nfp = N + 1;
  s->K = K;
  s->nv = nv;
  s->precision = precision;
  s->c = 1.0 / Ma;
  s->tau = Ma * Ma / Re;
  s->period[0] = period[0];
  s->period[1] = period[1];
  s->stream = (cudaStream_t)cuda_stream;
  s->elem_bytes = precision == GB_FP64 ? sizeof(double) : sizeof(float);
  s->has_bc = has_bc;
  if (far_state) {
    // free-stream equilibrium (Sec. 2 maps; second moments at equilibrium), minus the rest
    // state in the perturbation representation of GB_MIXED
    const double rho = far_state[0], u2 = rho * far_state[1] / s->c, u3 = rho * far_state[2] / s->c;
    const double q[6] = {rho, u2, u3, u2 * u3 / rho, u2 * u2 / (M_SQRT2 * rho), u3 * u3 / (M_SQRT2 * rho)};
    for (int k = 0; k < 6; ++k) s->far[k] = q[k] - ((precision == GB_MIXED && k == 0) ? 1.0 : 0.0);
  }
  if (!gb::build_reference(N, s->ref)) {
    delete s;
    return fail(nullptr, GB_EINVAL, "reference operator construction failed");
  }
  s->Nc = s->ref.Nc;

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (ce != cudaSuccess) {
    delete s;
    return fail(nullptr, GB_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
  }
  s->device = dev;
  int rc = gb::upload_ops(N, s->ref, &s->d_ops, s->stream);
  if (rc == 0 && precision == GB_MIXED) rc = gb::upload_ops_mixed(N, s->ref, &s->d_ops_mixed, s->stream);
  if (rc == 0 && precision == GB_MIXED && gb::um_supported(N) && !has_bc)
    rc = gb::upload_ops_um(N, s->ref, &s->d_ops_um, s->stream);
  if (rc != 0) {
    std::string m = std::string("operator upload: ") + cudaGetErrorString((cudaError_t)rc);
    free_all(s);
    delete s;
    return fail(nullptr, GB_ECUDA, m);
  }
  // GB_MIXED: element-major layout with the padded stride S, tiles of 16 elements, Morton order
  const int64_t Kpad = precision == GB_MIXED ? ((K + 15) / 16) * 16 : K;
  const int64_t per_elem = precision == GB_MIXED ? gb::mixed_stride(N) : 6 * s->Np;
  std::vector<int32_t> perm;
  std::vector<MeshRec> rec_int;
  if (precision == GB_MIXED) {
    std::vector<double> cx(K), cy(K);
    for (int64_t e = 0; e < K; ++e) {
      cx[e] = (vx(e, 0, 0) + vx(e, 1, 0) + vx(e, 2, 0)) / 3.0;
      cy[e] = (vx(e, 0, 1) + vx(e, 1, 1) + vx(e, 2, 1)) / 3.0;
    }
    perm = morton_order(cx, cy);
    std::vector<int32_t> inv(K);
    for (int64_t i = 0; i < K; ++i) inv[perm[i]] = (int32_t)i;
    rec_int.resize(K);
    for (int64_t i = 0; i < K; ++i) {
      rec_int[i] = rec[perm[i]];
      for (int f = 0; f < 3; ++f) {
        const int32_t nb = rec_int[i].nbr[f];
        if (nb >= 0) rec_int[i].nbr[f] = (inv[nb >> 2] << 2) | (nb & 3);
      }
    }
  }
  const size_t fbytes = (size_t)Kpad * per_elem * s->elem_bytes;
  void **fields[] = {&s->d_qn, &s->d_b1, &s->d_b2, &s->d_F0, &s->d_acc};
  int arc = GB_OK;
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_mesh, sizeof(MeshRec) * K);
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_X, sizeof(double) * 2 * nv);
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_xn, sizeof(double) * 2 * nv);
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_shape, sizeof(double) * 2 * nv);
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_clock, sizeof(double) * 2);
  arc = arc ? arc : dev_alloc(s, (void **)&s->d_status, sizeof(int));
  for (void **p : fields) arc = arc ? arc : dev_alloc(s, p, fbytes);
  if (precision == GB_MIXED) {
    arc = arc ? arc : dev_alloc(s, (void **)&s->d_mesh_int, sizeof(MeshRec) * K);
    arc = arc ? arc : dev_alloc(s, (void **)&s->d_perm, sizeof(int32_t) * K);
  }
  if (arc != GB_OK) {
    g_create_error = s->err;
    free_all(s);
    delete s;
    return arc;
  }
  double clock0[2] = {0.0, 0.0};
  int zero = 0;
  ce = cudaMemcpyAsync(s->d_mesh, rec.data(), sizeof(MeshRec) * K, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess && precision == GB_MIXED)
    ce = cudaMemcpyAsync(s->d_mesh_int, rec_int.data(), sizeof(MeshRec) * K, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess && precision == GB_MIXED)
    ce = cudaMemcpyAsync(s->d_perm, perm.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_X, mesh->X, sizeof(double) * 2 * nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_xn, mesh->X, sizeof(double) * 2 * nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->d_shape, 0, sizeof(double) * 2 * nv, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_clock, clock0, sizeof(clock0), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
  for (void **p : fields)
    if (ce == cudaSuccess) ce = cudaMemsetAsync(*p, 0, fbytes, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) {
    cuda_fail(s, ce, "gb_create upload");
    g_create_error = s->err;
    free_all(s);
    delete s;
    return GB_ECUDA;
  }
  *out = s;
  return GB_OK;
}

static void free_pml(gb_solver *s) {
  const size_t eb = s->precision == GB_FP64 ? sizeof(double) : sizeof(float);
  dev_free(s, &s->d_phi, s->pml_bytes);
  dev_free(s, &s->d_pml_node, eb * 3 * s->Np * (size_t)s->n_layer);
  dev_free(s, (void **)&s->d_pml_elem, sizeof(int32_t) * (size_t)s->n_layer);
  dev_free(s, &s->d_pml_ops, eb * (size_t)gb::pml_ops_size(s->N));
  s->n_layer = 0;
  s->pml_bytes = 0;
}

template <typename T>
static std::vector<unsigned char> as_bytes(const std::vector<double> &v) {
  std::vector<unsigned char> out(v.size() * sizeof(T));
  T *o = reinterpret_cast<T *>(out.data());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return out;
}

extern "C" {

int gb_set_motion(gb_solver *s, const gb_motion *m) {
  if (!s || !m) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) {
    if (m->kind == GB_MOTION_STATIC) return gb::s3_set_static(s->s3);
    if (m->kind == GB_MOTION_TGV3D) return gb::s3_set_tgv_motion(s->s3, m->A, m->T, m->Lx);
    return fail(s, GB_EINVAL, "dim = 3 solvers take GB_MOTION_STATIC, GB_MOTION_TGV3D or gb_set_wave_motion");
  }
  if (m->kind == GB_MOTION_TGV3D) return fail(s, GB_EINVAL, "GB_MOTION_TGV3D applies to dim = 3 solvers");
  if (m->kind != GB_MOTION_STATIC && m->kind != GB_MOTION_SINXY && m->kind != GB_MOTION_PLUNGE)
    return fail(s, GB_EINVAL, "unknown motion kind");
  if (m->kind == GB_MOTION_PLUNGE && (!(m->T > 0.0) || !std::isfinite(m->A) || !std::isfinite(m->T)))
    return fail(s, GB_EINVAL, "GB_MOTION_PLUNGE needs T > 0 and finite A");
  if (m->kind == GB_MOTION_SINXY) {
    if (!(m->T > 0.0) || !(m->Lx != 0.0) || !(m->Ly != 0.0) || !std::isfinite(m->A) || !std::isfinite(m->T))
      return fail(s, GB_EINVAL, "GB_MOTION_SINXY needs T > 0, Lx != 0, Ly != 0 and finite A");
  }
  s->motion = *m;
  drop_graph(s);
  int rc = gb::launch_shape(s->d_X, s->d_shape, s->nv, m->kind, m->Lx, m->Ly, s->stream);
  if (rc != 0) return cuda_fail(s, (cudaError_t)rc, "shape kernel");
  return GB_OK;
}

int gb_set_fields(gb_solver *s, const double *q_host, double t) {
  if (!s || !q_host) return fail(s, GB_EINVAL, "NULL argument");
  if (!std::isfinite(t)) return fail(s, GB_EINVAL, "t must be finite");
  if (s->s3) return gb::s3_set_fields(s->s3, q_host, t);
  const size_t n = (size_t)s->K * 6 * s->Np;
  cudaError_t ce;
  if (s->precision == GB_FP64) {
    ce = cudaMemcpyAsync(s->d_qn, q_host, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  } else {
    int rc = ensure_tmp(s, n * sizeof(double));
    if (rc) return rc;
    ce = cudaMemcpyAsync(s->d_tmp, q_host, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess) {
      int lr = gb::launch_relayout(s->d_tmp, nullptr, true, true, (float *)s->d_qn, s->d_perm, s->K, s->Np,
                                   gb::mixed_stride(s->N), 1.0, s->stream);
      if (lr) ce = (cudaError_t)lr;
    }
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_clock, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess && s->d_phi) ce = cudaMemsetAsync(s->d_phi, 0, s->pml_bytes, s->stream);   // Phi = 0
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_fields");
  return GB_OK;
}

int gb_sync(gb_solver *s) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_sync(s->s3);
  int status = 0, zero = 0;
  cudaError_t ce = cudaMemcpyAsync(&status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_sync");
  if (status & GB_STATUS_MESH) return fail(s, GB_EMESH, "an element reached J <= 0 during a stage");
  if (status & GB_STATUS_NAN) return fail(s, GB_ENAN, "a NaN or Inf appeared in the fields");
  return GB_OK;
}

int gb_fields(gb_solver *s, double *q_host_out, double *t_out) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_fields(s->s3, q_host_out, t_out);
  int st = gb_sync(s);
  const size_t n = (size_t)s->K * 6 * s->Np;
  cudaError_t ce = cudaSuccess;
  if (q_host_out) {
    if (s->precision == GB_FP64) {
      ce = cudaMemcpyAsync(q_host_out, s->d_qn, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    } else {
      int rc = ensure_tmp(s, n * sizeof(double));
      if (rc) return rc;
      int lr = gb::launch_relayout(nullptr, s->d_tmp, true, false, (float *)s->d_qn, s->d_perm, s->K, s->Np,
                                   gb::mixed_stride(s->N), 1.0, s->stream);
      ce = lr ? (cudaError_t)lr : cudaMemcpyAsync(q_host_out, s->d_tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
  }
  double clk[2] = {0, 0};
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(clk, s->d_clock, sizeof(clk), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_fields");
  if (t_out) *t_out = clk[0];
  return st;
}

int gb_set_vertices(gb_solver *s, const double *x_host) {
  if (!s || !x_host) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return gb::s3_set_vertices(s->s3, x_host);
  cudaError_t ce = cudaMemcpyAsync(s->d_xn, x_host, sizeof(double) * 2 * s->nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_vertices");
  return GB_OK;
}

int gb_vertices(gb_solver *s, double *x_host_out) {
  if (!s || !x_host_out) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return gb::s3_vertices(s->s3, x_host_out);
  cudaError_t ce = cudaMemcpyAsync(x_host_out, s->d_xn, sizeof(double) * 2 * s->nv, cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_vertices");
  return GB_OK;
}

int gb_nodes(gb_solver *s, double *xy_out) {
  if (!s || !xy_out) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return gb::s3_nodes(s->s3, xy_out);
  const size_t n = (size_t)s->K * s->Np * 2;
  int rc = ensure_tmp(s, n * sizeof(double));
  if (rc) return rc;
  int lr = gb::launch_nodes(s->N, s->d_ops, s->d_xn, s->d_mesh, s->period[0], s->period[1], s->K, s->d_tmp, s->stream);
  cudaError_t ce = lr ? (cudaError_t)lr : cudaMemcpyAsync(xy_out, s->d_tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_nodes");
  return GB_OK;
}

int gb_rhs(gb_solver *s, double t, const void *q_dev, void *F_dev) {
  if (!s || !q_dev || !F_dev) return fail(s, GB_EINVAL, "NULL argument");
  if (!std::isfinite(t)) return fail(s, GB_EINVAL, "t must be finite");
  if (s->s3) return gb::s3_rhs(s->s3, t, q_dev, F_dev);
  gb::StageArgs a = base_args(s);
  a.stage = -1;
  a.rhs_time = t;
  if (s->precision == GB_FP64) {
    a.qin = q_dev;
    a.qn = q_dev;
    a.Fout = F_dev;
    return launch_stage(s, a);
  }
  // GB_MIXED: canonical FP32 perturbations -> internal layout in the stage buffers b1, b2
  int lr = gb::launch_relayout(q_dev, nullptr, false, true, (float *)s->d_b1, s->d_perm, s->K, s->Np,
                               gb::mixed_stride(s->N), 0.0, s->stream);
  if (lr) return cuda_fail(s, (cudaError_t)lr, "gb_rhs relayout");
  a.qin = s->d_b1;
  a.qn = s->d_b1;
  a.Fout = s->d_b2;
  int rc = launch_stage(s, a);
  if (rc) return rc;
  lr = gb::launch_relayout(nullptr, F_dev, false, false, (float *)s->d_b2, s->d_perm, s->K, s->Np,
                           gb::mixed_stride(s->N), 0.0, s->stream);
  if (lr) return cuda_fail(s, (cudaError_t)lr, "gb_rhs relayout");
  return GB_OK;
}

static int step_impl(gb_solver *s, double dt, int64_t nsteps, double *kernel_ms);

int gb_step(gb_solver *s, double dt, int64_t nsteps) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_step(s->s3, dt, nsteps);
  if (nsteps > 0) {
    int trc = tune_launch(s);
    if (trc) return trc;
  }
  // the legacy default stream cannot be captured; tiny runs are not worth a capture
  if (!s->use_graph || !s->stream || nsteps < 2 || !(dt > 0.0) || !std::isfinite(dt)) return step_impl(s, dt, nsteps, nullptr);
  if (s->step_graph && s->graph_dt != dt) drop_graph(s);
  if (!s->graph_warm || s->graph_dt != dt) {
    // first step with these settings runs directly (kernel attributes, coefficients)
    int rc = step_impl(s, dt, 1, nullptr);
    if (rc) return rc;
    s->graph_warm = true;
    s->graph_dt = dt;
    --nsteps;
  }
  if (!s->step_graph) {
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_step capture");
    int rc = step_impl(s, dt, 1, nullptr);
    ce = cudaStreamEndCapture(s->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&s->step_graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      s->step_graph = nullptr;
      return cuda_fail(s, ce, "gb_step graph");
    }
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    cudaError_t ce = cudaGraphLaunch(s->step_graph, s->stream);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_step graph launch");
  }
  return GB_OK;
}

int gb_step_timed(gb_solver *s, double dt, int64_t nsteps, double *kernel_ms) {
  if (!kernel_ms) return fail(s, GB_EINVAL, "kernel_ms is NULL");
  if (s && s->s3) return gb::s3_step_timed(s->s3, dt, nsteps, kernel_ms);
  if (s && nsteps > 0) {
    int trc = tune_launch(s);
    if (trc) return trc;
  }
  int rc = step_impl(s, dt, nsteps, kernel_ms);
  return rc ? rc : gb_sync(s);
}

static int step_impl(gb_solver *s, double dt, int64_t nsteps, double *kernel_ms) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(s, GB_EINVAL, "dt must be positive and finite");
  if (nsteps < 0) return fail(s, GB_EINVAL, "nsteps must be >= 0");
  if (dt != s->coef_dt) {
    double E[5], A[16], B[4];
    gb::sark_coefficients(0.0, E, A, B);
    memcpy(s->co.E[0], E, sizeof(E)); memcpy(s->co.A[0], A, sizeof(A)); memcpy(s->co.B[0], B, sizeof(B));
    gb::sark_coefficients(-dt / s->tau, E, A, B);
    memcpy(s->co.E[1], E, sizeof(E)); memcpy(s->co.A[1], A, sizeof(A)); memcpy(s->co.B[1], B, sizeof(B));
    s->coef_dt = dt;
  }
  gb::StageArgs a = base_args(s);
  a.dt = dt;
  void *bufs_in[4] = {s->d_qn, s->d_b1, s->d_b2, s->d_b1};
  void *bufs_out[4] = {s->d_b1, s->d_b2, s->d_b1, s->d_qn};
  std::vector<cudaEvent_t> ev;
  if (kernel_ms) {
    ev.resize((size_t)nsteps * 10);
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        for (auto &x : ev)
          if (x) cudaEventDestroy(x);
        return fail(s, GB_ECUDA, "cudaEventCreate failed");
      }
  }
  int rc = GB_OK;
  for (int64_t k = 0; k < nsteps && rc == GB_OK; ++k) {
    for (int st = 0; st < 5 && rc == GB_OK; ++st) {
      if (kernel_ms) cudaEventRecord(ev[(size_t)k * 10 + 2 * st], s->stream);
      if (st < 4) {
        a.stage = st;
        a.qin = bufs_in[st];
        a.qn = s->d_qn;
        a.qout = bufs_out[st];
        a.F0 = s->d_F0;
        a.acc = s->d_acc;
        if (st == 3 && s->diag_every > 0 && s->n_layer == 0) {
          // diagnostics fused into the last stage: integrals of q_{n+1} on x_{n+1}, recorded by the
          // last CTA (partials in the diagnostics scratch, after the weights and result slots)
          a.rec_every = s->diag_every;
          a.rec_cap = s->diag_cap;
          a.rec_wq = s->d_diag;
          a.rec_part = s->d_diag + s->Np + 5;
          a.rec_done = s->d_done;
          a.rec_ctl = s->d_hctl;
          a.rec_hist = s->d_hist;
        }
        rc = launch_stage(s, a);
        a.rec_every = 0;
        if (rc == GB_OK) rc = launch_pml(s, a);
      } else {
        int lr = gb::launch_vertex_update(a, s->nv, s->stream);
        if (lr) rc = cuda_fail(s, (cudaError_t)lr, "vertex update launch");
        // with a layer the record follows its last correction: separate reduction launches
        if (rc == GB_OK && s->n_layer > 0) rc = record_diagnostics(s, s->stream);
      }
      if (kernel_ms) cudaEventRecord(ev[(size_t)k * 10 + 2 * st + 1], s->stream);
    }
  }
  if (kernel_ms) {
    cudaError_t ce = cudaStreamSynchronize(s->stream);
    for (int64_t k = 0; k < nsteps && ce == cudaSuccess && rc == GB_OK; ++k)
      for (int st = 0; st < 5; ++st) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev[(size_t)k * 10 + 2 * st], ev[(size_t)k * 10 + 2 * st + 1]) == cudaSuccess)
          kernel_ms[st] += ms;
      }
    for (auto &e : ev) cudaEventDestroy(e);
    if (ce != cudaSuccess && rc == GB_OK) rc = cuda_fail(s, ce, "gb_step_timed");
  }
  return rc;
}

// ---- groups: many GB_MIXED solvers of one order stepped by one launch per stage ----

int gb_group_create(int capacity, void *cuda_stream, gb_group **out) {
  if (!out || capacity < 1 || capacity > (1 << 20)) return fail(nullptr, GB_EINVAL, "gb_group_create: bad capacity or NULL out");
  *out = nullptr;
  gb_group *g = new gb_group();
  g->capacity = capacity;
  g->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  g->device = dev;
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t args_bytes = sizeof(gb::StageArgs) * 4 * (size_t)capacity;
  const size_t pre_bytes = sizeof(int64_t) * 2 * (size_t)(capacity + 1);
  if (ce == cudaSuccess) ce = cudaMalloc(&g->d_args, args_bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&g->d_prefix, pre_bytes);
  if (ce == cudaSuccess) ce = cudaMallocHost(&g->h_args, args_bytes);
  if (ce == cudaSuccess) ce = cudaMallocHost(&g->h_prefix, pre_bytes);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&g->uploaded, cudaEventDisableTiming);
  if (ce != cudaSuccess) {
    std::string m = std::string("gb_group_create: ") + cudaGetErrorString(ce);
    gb_group_destroy(g);
    return fail(nullptr, ce == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA, m);
  }
  *out = g;
  return GB_OK;
}

// Group launch-shape tuner: warps per CTA of the group kernel (4, 2 or 1) for the group's
// order and size class (tile count), timed on the group's own data with stage-0 launches, which
// only write the stage buffer b1 and F_0 of each member (both rewritten by the step's own stage
// 0); a later candidate must win by 3%.  Choices are cached per (device, N, tile-count class).
static int group_tune(gb_group *g, int N, gb::GroupArgs &ga) {
  if (g->fixed[N]) {
    ga.warps = g->warps[N];
    return GB_OK;
  }
  const TuneKey key(g->device, N, k_class(ga.total_tiles));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_group_tuned.find(key);
    if (it != g_group_tuned.end()) {
      ga.warps = g->warps[N] = it->second;
      return GB_OK;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  const int cand[3] = {4, 2, 1};
  int best = 4;
  float best_ms = 1e30f;
  ga.args = g->d_args;   // stage 0
  for (int i = 0; i < 3 && ce == cudaSuccess; ++i) {
    ga.warps = cand[i];
    int rc = gb::launch_group_mixed(N, 0, ga, g->stream, g->num_sms);   // warm-up
    if (rc) { ce = (cudaError_t)rc; break; }
    ce = cudaEventRecord(e0, g->stream);
    for (int r = 0; r < 2 && ce == cudaSuccess; ++r) {
      rc = gb::launch_group_mixed(N, 0, ga, g->stream, g->num_sms);
      if (rc) ce = (cudaError_t)rc;
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, g->stream);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess && ms < 0.97f * best_ms) {
      best_ms = ms;
      best = cand[i];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ce != cudaSuccess) {
    g->err = std::string("gb_group_step tuning: ") + cudaGetErrorString(ce);
    return GB_ECUDA;
  }
  ga.warps = g->warps[N] = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_group_tuned[key] = best;
  return GB_OK;
}

int gb_group_set_launch_config(gb_group *g, int N, int warps_per_cta) {
  if (!g || N < 1 || N > GB_MAX_N || (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4))
    return GB_EINVAL;
  g->warps[N] = warps_per_cta;
  g->fixed[N] = true;
  return GB_OK;
}

int gb_group_launch_config(gb_group *g, int N, int *warps_per_cta) {
  if (!g || !warps_per_cta || N < 1 || N > GB_MAX_N) return GB_EINVAL;
  *warps_per_cta = g->warps[N];
  return GB_OK;
}

int gb_group_step(gb_group *g, gb_solver *const *solvers, const double *dt, int n, int64_t nsteps) {
  if (!g) return fail(nullptr, GB_EINVAL, "gb_group_step: NULL group");
  auto gfail = [&](int code, const std::string &m) { g->err = m; return code; };
  if (!solvers || !dt || n < 1 || n > g->capacity) return gfail(GB_EINVAL, "gb_group_step: bad arguments or n > capacity");
  if (nsteps < 0) return gfail(GB_EINVAL, "gb_group_step: nsteps < 0");
  const int N = solvers[0] ? solvers[0]->N : 0;
  for (int r = 0; r < n; ++r) {
    gb_solver *s = solvers[r];
    if (!s) return gfail(GB_EINVAL, "gb_group_step: NULL solver");
    if (s->s3) return gfail(GB_EINVAL, "gb_group_step: dim = 3 solvers cannot be grouped");
    if (s->has_bc) return gfail(GB_EINVAL, "gb_group_step: solvers with boundary faces cannot be grouped");
    if (s->n_layer > 0) return gfail(GB_EINVAL, "gb_group_step: solvers with a perfectly matched layer cannot be grouped");
    if (s->precision != GB_MIXED) return gfail(GB_EINVAL, "gb_group_step: only GB_MIXED solvers can be grouped");
    if (s->N != N) return gfail(GB_EINVAL, "gb_group_step: all solvers of a group must have the same N");
    if (s->stream != g->stream) return gfail(GB_EINVAL, "gb_group_step: solvers must use the group's stream");
    if (!(dt[r] > 0.0) || !std::isfinite(dt[r])) return gfail(GB_EINVAL, "gb_group_step: dt must be positive and finite");
  }
  // the pinned staging buffers may still be read by the previous upload
  cudaError_t ce = cudaEventSynchronize(g->uploaded);
  if (ce != cudaSuccess) return gfail(GB_ECUDA, std::string("gb_group_step: ") + cudaGetErrorString(ce));
  int64_t *tstart = g->h_prefix, *vstart = g->h_prefix + (n + 1);
  tstart[0] = 0;
  vstart[0] = 0;
  for (int r = 0; r < n; ++r) {
    gb_solver *s = solvers[r];
    set_coefficients(s, dt[r]);
    gb::StageArgs a = base_args(s);
    a.dt = dt[r];
    void *bufs_in[4] = {s->d_qn, s->d_b1, s->d_b2, s->d_b1};
    void *bufs_out[4] = {s->d_b1, s->d_b2, s->d_b1, s->d_qn};
    for (int st = 0; st < 4; ++st) {
      a.stage = st;
      a.qin = bufs_in[st];
      a.qn = s->d_qn;
      a.qout = bufs_out[st];
      a.F0 = s->d_F0;
      a.acc = s->d_acc;
      gb::set_mixed_coefs(a);
      g->h_args[(size_t)st * g->capacity + r] = a;
    }
    tstart[r + 1] = tstart[r] + (s->K + 15) / 16;
    vstart[r + 1] = vstart[r] + s->nv;
  }
  ce = cudaMemcpyAsync(g->d_args, g->h_args, sizeof(gb::StageArgs) * 4 * (size_t)g->capacity, cudaMemcpyHostToDevice, g->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(g->d_prefix, g->h_prefix, sizeof(int64_t) * 2 * (size_t)(n + 1), cudaMemcpyHostToDevice, g->stream);
  if (ce == cudaSuccess) ce = cudaEventRecord(g->uploaded, g->stream);
  if (ce != cudaSuccess) return gfail(GB_ECUDA, std::string("gb_group_step upload: ") + cudaGetErrorString(ce));
  gb::GroupArgs ga;
  ga.tile_start = g->d_prefix;
  ga.vtx_start = g->d_prefix + (n + 1);
  ga.n = n;
  ga.total_tiles = tstart[n];
  ga.total_vertices = vstart[n];
  ga.ops = solvers[0]->d_ops_mixed;
  ga.warps = 4;
  if (nsteps > 0) {
    int rc = group_tune(g, N, ga);
    if (rc) return rc;
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    for (int st = 0; st < 4; ++st) {
      ga.args = g->d_args + (size_t)st * g->capacity;
      int rc = gb::launch_group_mixed(N, st, ga, g->stream, g->num_sms);
      if (rc) return gfail(GB_ECUDA, std::string("gb_group_step launch: ") + cudaGetErrorString((cudaError_t)rc));
    }
    ga.args = g->d_args + 3 * (size_t)g->capacity;
    int rc = gb::launch_group_vertex_update(ga, g->stream);
    if (rc) return gfail(GB_ECUDA, std::string("gb_group_step launch: ") + cudaGetErrorString((cudaError_t)rc));
    for (int r = 0; r < n; ++r)
      if (record_diagnostics(solvers[r], g->stream)) return gfail(GB_ECUDA, "gb_group_step: " + solvers[r]->err);
  }
  return GB_OK;
}

int gb_group_destroy(gb_group *g) {
  if (!g) return GB_OK;
  if (g->uploaded) cudaEventSynchronize(g->uploaded);
  if (g->stream) cudaStreamSynchronize(g->stream); else cudaDeviceSynchronize();
  if (g->d_args) cudaFree(g->d_args);
  if (g->d_prefix) cudaFree(g->d_prefix);
  if (g->h_args) cudaFreeHost(g->h_args);
  if (g->h_prefix) cudaFreeHost(g->h_prefix);
  if (g->uploaded) cudaEventDestroy(g->uploaded);
  delete g;
  return GB_OK;
}

const char *gb_group_last_error(gb_group *g) { return g ? g->err.c_str() : g_create_error.c_str(); }

int gb_set_diagnostics(gb_solver *s, int every, int64_t capacity) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (every < 0 || (every > 0 && (capacity < 1 || capacity > ((int64_t)1 << 32))))
    return fail(s, GB_EINVAL, "every must be >= 0 and capacity in 1 .. 2^32");
  if (s->s3) return gb::s3_set_diagnostics(s->s3, every, capacity);
  cudaError_t ce = s->stream ? cudaStreamSynchronize(s->stream) : cudaDeviceSynchronize();
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_diagnostics");
  drop_graph(s);
  dev_free(s, (void **)&s->d_hist, sizeof(double) * 6 * (size_t)s->diag_cap);
  dev_free(s, (void **)&s->d_hctl, 2 * sizeof(int64_t));
  s->diag_every = 0;
  s->diag_cap = 0;
  if (every == 0) return GB_OK;
  int rc = ensure_diag(s);
  if (!rc) rc = dev_alloc(s, (void **)&s->d_hist, sizeof(double) * 6 * (size_t)capacity);
  if (!rc) rc = dev_alloc(s, (void **)&s->d_hctl, 2 * sizeof(int64_t));
  if (rc) {
    dev_free(s, (void **)&s->d_hist, sizeof(double) * 6 * (size_t)capacity);
    return rc;
  }
  ce = cudaMemsetAsync(s->d_hctl, 0, 2 * sizeof(int64_t), s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_diagnostics");
  s->diag_every = every;
  s->diag_cap = capacity;
  return GB_OK;
}

int gb_diagnostics_history(gb_solver *s, double *out, int64_t max, int64_t *count, int64_t *total) {
  if (!s || !count || (max > 0 && !out) || max < 0) return fail(s, GB_EINVAL, "NULL argument or max < 0");
  *count = 0;
  if (total) *total = 0;
  const double *hist = s->d_hist;
  const int64_t *hctl = s->d_hctl;
  int every = s->diag_every;
  int64_t cap = s->diag_cap;
  if (s->s3) gb::s3_diag_ring(s->s3, &hist, &hctl, &every, &cap);
  if (every <= 0) return GB_OK;
  cudaStream_t st = s->s3 ? (cudaStream_t)gb::s3_stream(s->s3) : s->stream;
  int64_t ctl[2] = {0, 0};
  cudaError_t ce = cudaMemcpyAsync(ctl, hctl, sizeof(ctl), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_diagnostics_history");
  const int64_t kept = ctl[1] < cap ? ctl[1] : cap;
  const int64_t n = kept < max ? kept : max;
  // the n most recent records, oldest first: record j sits in slot j mod cap, so at
  // most two contiguous pieces of the ring
  if (n > 0) {
    const int64_t a = (ctl[1] - n) % cap;
    const int64_t first = n < cap - a ? n : cap - a;
    ce = cudaMemcpyAsync(out, hist + 6 * a, 6 * sizeof(double) * (size_t)first, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess && first < n)
      ce = cudaMemcpyAsync(out + 6 * first, hist, 6 * sizeof(double) * (size_t)(n - first), cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_diagnostics_history");
  }
  ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_diagnostics_history");
  *count = n;
  if (total) *total = ctl[1];
  return GB_OK;
}

int gb_diagnostics3d(gb_solver *s, double *out) {
  if (!s || !out) return fail(s, GB_EINVAL, "NULL argument");
  if (!s->s3) return fail(s, GB_EINVAL, "gb_diagnostics3d applies to dim = 3 solvers");
  return gb::s3_diagnostics(s->s3, out);
}

int gb_diagnostics(gb_solver *s, double *out) {
  if (!s || !out) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) {
    double r[6];
    int rc = gb::s3_diagnostics(s->s3, r);
    if (rc) return rc;
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
    out[3] = r[3];
    out[4] = r[5];
    return GB_OK;
  }
  {
    int rc = ensure_diag(s);
    if (rc) return rc;
  }
  const bool mixed = s->precision == GB_MIXED;
  const int64_t stride = mixed ? gb::mixed_stride(s->N) : 6 * s->Np;
  int lr = gb::launch_diagnostics(s->N, s->d_qn, mixed, mixed, stride, mixed ? s->d_mesh_int : s->d_mesh, s->d_xn,
                                  s->period[0], s->period[1], s->d_diag, s->c, s->K, s->d_diag + s->Np + 5,
                                  s->d_diag + s->Np, s->stream);
  if (lr) return cuda_fail(s, (cudaError_t)lr, "gb_diagnostics");
  double r[5];
  cudaError_t ce = cudaMemcpyAsync(r, s->d_diag + s->Np, sizeof(r), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_diagnostics");
  out[0] = r[0];
  out[1] = r[1] / r[4];
  out[2] = r[2];
  out[3] = r[3];
  out[4] = r[4];
  return GB_OK;
}

int gb_launch_config(gb_solver *s, int *warps_per_cta) {
  if (!s || !warps_per_cta) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return gb::s3_launch_config(s->s3, warps_per_cta);
  *warps_per_cta = s->precision == GB_MIXED ? (s->warps ? s->warps : 4) : 0;
  return GB_OK;
}

int gb_set_launch_config(gb_solver *s, int warps_per_cta) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_set_launch_config(s->s3, warps_per_cta);
  if (s->precision != GB_MIXED) return fail(s, GB_EINVAL, "launch shapes apply to GB_MIXED solvers");
  if (warps_per_cta == gb::kShapeUm && !s->d_ops_um)
    return fail(s, GB_EINVAL, "shape 8 (tcgen05, 128-element tiles) needs N <= 4 and a mesh without boundary faces");
  if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != gb::kShapeUm)
    return fail(s, GB_EINVAL, "the launch shape must be 1, 2 or 4 (warps per CTA) or 8 (tcgen05 tiles)");
  s->warps = warps_per_cta;
  drop_graph(s);
  return GB_OK;
}

int gb_set_graph(gb_solver *s, int enable) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_set_graph(s->s3, enable);
  s->use_graph = enable != 0;
  drop_graph(s);
  return GB_OK;
}

int gb_set_stream(gb_solver *s, void *cuda_stream) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_set_stream(s->s3, cuda_stream);
  cudaError_t ce = s->stream ? cudaStreamSynchronize(s->stream) : cudaDeviceSynchronize();
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_stream");
  drop_graph(s);
  s->stream = (cudaStream_t)cuda_stream;
  return GB_OK;
}

int gb_info(gb_solver *s, int *Np, int *Nfp, int *Nc, int64_t *n_elem, int64_t *n_vert, double *c, double *tau,
            int64_t *device_bytes) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return gb::s3_info(s->s3, Np, Nfp, Nc, n_elem, n_vert, c, tau, device_bytes);
  if (Np) *Np = s->Np;
  if (Nfp) *Nfp = s->Nfp;
  if (Nc) *Nc = s->Nc;
  if (n_elem) *n_elem = s->K;
  if (n_vert) *n_vert = s->nv;
  if (c) *c = s->c;
  if (tau) *tau = s->tau;
  if (device_bytes) *device_bytes = s->device_bytes;
  return GB_OK;
}

int gb_state_ptr(gb_solver *s, void **q_dev) {
  if (!s || !q_dev) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return gb::s3_state_ptr(s->s3, q_dev);
  *q_dev = s->d_qn;
  return GB_OK;
}

int gb_destroy(gb_solver *s) {
  if (!s) return GB_OK;
  if (s->s3) {
    gb::s3_destroy(s->s3);
    delete s;
    return GB_OK;
  }
  if (s->stream) cudaStreamSynchronize(s->stream); else cudaDeviceSynchronize();
  drop_graph(s);
  free_all(s);
  delete s;
  return GB_OK;
}

const char *gb_last_error(gb_solver *s) {
  if (s && s->s3 && s->err.empty()) return gb::s3_error(s->s3);
  return s ? s->err.c_str() : g_create_error.c_str();
}

int gb_set_pml(gb_solver *s, const gb_pml *p) {
  if (!s) return fail(s, GB_EINVAL, "NULL solver");
  if (s->s3) return fail(s, GB_EINVAL, "gb_set_pml applies to dim = 2 solvers");
  cudaError_t ce = s->stream ? cudaStreamSynchronize(s->stream) : cudaDeviceSynchronize();
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_pml");
  if (p) {
    const double vals[10] = {p->cx, p->cy, p->ex, p->ey, p->r0, p->d, p->sigma_max, p->power, p->alpha, 0.0};
    for (double v : vals)
      if (!std::isfinite(v)) return fail(s, GB_EINVAL, "gb_pml: non-finite parameter");
    if (p->kind != GB_PML_RADIAL && p->kind != GB_PML_SLAB && p->kind != GB_PML_UNIFORM)
      return fail(s, GB_EINVAL, "gb_pml: unknown kind");
    if (p->sigma_max < 0.0 || p->power < 0.0 || p->alpha < 0.0)
      return fail(s, GB_EINVAL, "gb_pml: sigma_max, power and alpha must be >= 0");
    if (p->kind != GB_PML_RADIAL && !(p->ex * p->ex + p->ey * p->ey > 0.0))
      return fail(s, GB_EINVAL, "gb_pml: the direction (ex, ey) must be non-zero");
    if (p->kind != GB_PML_UNIFORM && !(p->d > 0.0)) return fail(s, GB_EINVAL, "gb_pml: d must be > 0");
    if (s->N > 4) return fail(s, GB_EINVAL, "gb_pml: N must be <= 4");
  }
  drop_graph(s);
  free_pml(s);
  if (!p) return GB_OK;
  // sigma and the direction at every node, from the Lagrangian vertex positions
  const int Np = s->Np;
  std::vector<double> X((size_t)2 * s->nv);
  std::vector<MeshRec> mesh((size_t)s->K);
  std::vector<int32_t> perm;
  ce = cudaMemcpy(X.data(), s->d_X, sizeof(double) * X.size(), cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess) ce = cudaMemcpy(mesh.data(), s->d_mesh, sizeof(MeshRec) * mesh.size(), cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess && s->precision == GB_MIXED) {
    perm.resize((size_t)s->K);
    ce = cudaMemcpy(perm.data(), s->d_perm, sizeof(int32_t) * perm.size(), cudaMemcpyDeviceToHost);
  }
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_set_pml");
  double ux = p->ex, uy = p->ey;
  const double un = std::sqrt(ux * ux + uy * uy);
  if (un > 0.0) { ux /= un; uy /= un; }
  std::vector<double> node;                  // per layer element: sigma[Np], e_x[Np], e_y[Np]
  std::vector<int64_t> layer;                // canonical ids, ascending
  std::vector<double> sg(Np), exv(Np), eyv(Np);
  for (int64_t e = 0; e < s->K; ++e) {
    const MeshRec &rec = mesh[(size_t)e];
    bool any = false;
    for (int n = 0; n < Np; ++n) {
      const double l[3] = {-0.5 * (s->ref.r[n] + s->ref.s[n]), 0.5 * (1.0 + s->ref.r[n]), 0.5 * (1.0 + s->ref.s[n])};
      double x = 0.0, y = 0.0;
      for (int k = 0; k < 3; ++k) {
        x += l[k] * (X[2 * (size_t)rec.v[k]] + rec.shift[2 * k] * s->period[0]);
        y += l[k] * (X[2 * (size_t)rec.v[k] + 1] + rec.shift[2 * k + 1] * s->period[1]);
      }
      double r = 0.0, dx = ux, dy = uy;
      if (p->kind == GB_PML_RADIAL) {
        const double rx = x - p->cx, ry = y - p->cy;
        r = std::sqrt(rx * rx + ry * ry);
        dx = r > 0.0 ? rx / r : 0.0;
        dy = r > 0.0 ? ry / r : 0.0;
      } else if (p->kind == GB_PML_SLAB) {
        const double sp = (x - p->cx) * ux + (y - p->cy) * uy;
        r = std::fabs(sp);
        if (sp < 0.0) { dx = -ux; dy = -uy; }
      }
      double sigma = p->sigma_max;
      if (p->kind != GB_PML_UNIFORM) {
        const double depth = (r - p->r0) / p->d;
        sigma = depth > 0.0 ? p->sigma_max * std::pow(depth, p->power) : 0.0;
      }
      sg[n] = sigma; exv[n] = dx; eyv[n] = dy;
      any = any || sigma > 0.0;
    }
    if (!any) continue;
    layer.push_back(e);
    node.insert(node.end(), sg.begin(), sg.end());
    node.insert(node.end(), exv.begin(), exv.end());
    node.insert(node.end(), eyv.begin(), eyv.end());
  }
  s->pml_alpha = p->alpha;
  if (layer.empty()) return GB_OK;
  // element indices in the kernels' numbering
  std::vector<int32_t> elem(layer.size());
  if (s->precision == GB_MIXED) {
    std::vector<int32_t> inv((size_t)s->K);
    for (int64_t i = 0; i < s->K; ++i) inv[(size_t)perm[(size_t)i]] = (int32_t)i;
    for (size_t i = 0; i < layer.size(); ++i) elem[i] = inv[(size_t)layer[i]];
  } else {
    for (size_t i = 0; i < layer.size(); ++i) elem[i] = (int32_t)layer[i];
  }
  // operator block: Dr^T, Ds^T, LIFT^T, node barycentrics
  const int NFN = 3 * s->Nfp;
  std::vector<double> ops((size_t)gb::pml_ops_size(s->N));
  for (int m = 0; m < Np; ++m)
    for (int n = 0; n < Np; ++n) {
      ops[(size_t)m * Np + n] = s->ref.Dr[(size_t)n * Np + m];
      ops[(size_t)Np * Np + m * Np + n] = s->ref.Ds[(size_t)n * Np + m];
    }
  for (int j = 0; j < NFN; ++j)
    for (int n = 0; n < Np; ++n) ops[(size_t)2 * Np * Np + j * Np + n] = s->ref.LIFT[(size_t)n * NFN + j];
  for (int n = 0; n < Np; ++n) {
    const size_t b = (size_t)2 * Np * Np + (size_t)NFN * Np + 3 * n;
    ops[b] = -0.5 * (s->ref.r[n] + s->ref.s[n]);
    ops[b + 1] = 0.5 * (1.0 + s->ref.r[n]);
    ops[b + 2] = 0.5 * (1.0 + s->ref.s[n]);
  }
  const bool fp64 = s->precision == GB_FP64;
  const size_t eb = fp64 ? sizeof(double) : sizeof(float);
  std::vector<unsigned char> ops_b = fp64 ? as_bytes<double>(ops) : as_bytes<float>(ops);
  std::vector<unsigned char> node_b = fp64 ? as_bytes<double>(node) : as_bytes<float>(node);
  s->n_layer = (int64_t)layer.size();
  s->pml_bytes = 3 * eb * 6 * Np * layer.size();
  int rc = dev_alloc(s, &s->d_pml_ops, ops_b.size());
  if (!rc) rc = dev_alloc(s, (void **)&s->d_pml_elem, sizeof(int32_t) * elem.size());
  if (!rc) rc = dev_alloc(s, &s->d_pml_node, node_b.size());
  if (!rc) rc = dev_alloc(s, &s->d_phi, s->pml_bytes);
  if (rc) {
    free_pml(s);
    return rc;
  }
  ce = cudaMemcpy(s->d_pml_ops, ops_b.data(), ops_b.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(s->d_pml_elem, elem.data(), sizeof(int32_t) * elem.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(s->d_pml_node, node_b.data(), node_b.size(), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemset(s->d_phi, 0, s->pml_bytes);
  if (ce != cudaSuccess) {
    free_pml(s);
    return cuda_fail(s, ce, "gb_set_pml upload");
  }
  return GB_OK;
}

int gb_pml_fields(gb_solver *s, double *phi_out, int64_t *elem_out, int64_t *n_layer) {
  if (!s || !n_layer) return fail(s, GB_EINVAL, "NULL argument");
  if (s->s3) return fail(s, GB_EINVAL, "gb_pml_fields applies to dim = 2 solvers");
  *n_layer = s->n_layer;
  if (s->n_layer == 0 || (!phi_out && !elem_out)) return GB_OK;
  const size_t n = (size_t)s->n_layer * 6 * s->Np;
  cudaError_t ce = cudaStreamSynchronize(s->stream);
  if (ce == cudaSuccess && phi_out) {
    if (s->precision == GB_FP64) {
      ce = cudaMemcpy(phi_out, s->d_phi, n * sizeof(double), cudaMemcpyDeviceToHost);
    } else {
      std::vector<float> f(n);
      ce = cudaMemcpy(f.data(), s->d_phi, n * sizeof(float), cudaMemcpyDeviceToHost);
      for (size_t i = 0; i < n; ++i) phi_out[i] = (double)f[i];
    }
  }
  if (ce == cudaSuccess && elem_out) {
    std::vector<int32_t> e((size_t)s->n_layer), perm;
    ce = cudaMemcpy(e.data(), s->d_pml_elem, sizeof(int32_t) * e.size(), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess && s->precision == GB_MIXED) {
      perm.resize((size_t)s->K);
      ce = cudaMemcpy(perm.data(), s->d_perm, sizeof(int32_t) * perm.size(), cudaMemcpyDeviceToHost);
    }
    for (size_t i = 0; ce == cudaSuccess && i < e.size(); ++i)
      elem_out[i] = s->precision == GB_MIXED ? perm[(size_t)e[i]] : e[i];
  }
  if (ce != cudaSuccess) return cuda_fail(s, ce, "gb_pml_fields");
  return GB_OK;
}

int gb_set_wave_motion(gb_solver *s, const gb_wave_motion *m) {
  if (!s || !m) return fail(s, GB_EINVAL, "NULL argument");
  if (!s->s3) return fail(s, GB_EINVAL, "gb_set_wave_motion applies to dim = 3 solvers");
  return gb::s3_set_wave_motion(s->s3, m);
}

int gb_reference_operators(int N, double *r, double *s_, double *Dr, double *Ds, double *LIFT, double *Icub,
                           double *Pcub, double *cr, double *cs, double *cw, int *Nc_out) {
  gb::RefOps R;
  if (!gb::build_reference(N, R)) return GB_EINVAL;
  auto put = [](const std::vector<double> &v, double *o) {
    if (o) memcpy(o, v.data(), v.size() * sizeof(double));
  };
  put(R.r, r); put(R.s, s_); put(R.Dr, Dr); put(R.Ds, Ds); put(R.LIFT, LIFT);
  put(R.I, Icub); put(R.P, Pcub); put(R.cr, cr); put(R.cs, cs); put(R.cw, cw);
  if (Nc_out) *Nc_out = R.Nc;
  return GB_OK;
}

int gb_sark_coefficients(double gamma, double *E, double *A, double *B) {
  if (!E || !A || !B) return GB_EINVAL;
  if (!(gamma <= 0.0) || !std::isfinite(gamma)) return GB_EINVAL;
  gb::sark_coefficients(gamma, E, A, B);
  return GB_OK;
}

}  // extern "C"

namespace gb {

// View of a solver for the allocation-free right-hand side (gb_noalloc.cu): the
// stage arguments of an rhs-only launch at time t, the element permutation and
// the sizes.  Returns GB_EINVAL for a NULL solver.
int rhs_launch_view(gb_solver *s, double t, StageArgs *a, const int32_t **perm, int *N, int64_t *K, int *Np,
                    int *precision, void **stream, int *num_sms, int *device) {
  if (!s || s->s3) return GB_EINVAL;
  *a = base_args(s);
  a->stage = -1;
  a->rhs_time = t;
  *perm = s->d_perm;
  *N = s->N;
  *K = s->K;
  *Np = s->Np;
  *precision = s->precision;
  *stream = s->stream;
  *num_sms = s->num_sms;
  *device = s->device;
  return GB_OK;
}

int set_solver_error(gb_solver *s, int code, const char *msg) { return fail(s, code, msg); }

}  // namespace gb

