// Host side of the 3D (tetrahedral, 10-field) solver behind the C ABI of include/gb.h:
// mesh validation and face connectivity (with the face-node permutation of each shared
// face), operator upload, state transfer and the SARK step driver (Sec. 4) that
// enqueues the fused stage kernels of gb_kernels3d.cu.  The public entry points in
// gb_api.cpp route here when the solver was created with mesh->dim == 3.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "gb3d.h"
#include "gb3d_internal.h"

namespace gb {

struct Solver3 {
  int N = 0, Np = 0, Nfp = 0, Nc = 0, precision = GB_FP64;
  int64_t K = 0, nv = 0;
  double c = 0, tau = 0, period[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  int num_sms = 1;
  int device = 0;
  std::string err;
  RefOps3 ref;
  Wave3 wave{0, 0, 1, 1, 0, 1, 0, 0};
  int moving = 0;
  double omega = 0.0;          // angular frequency of the motion's time factors cos, sin(omega t)
  double coef_dt = -1.0;
  SarkCoef co{};
  cudaGraphExec_t graph = nullptr;
  double graph_dt = -1.0;
  bool graph_warm = false, use_graph = true;
  size_t elem_bytes = 8;
  void *d_ops = nullptr;
  void *d_ops_tc = nullptr;     // GB_MIXED, N <= 3: the tensor-core kernel's operator table
  int shape = 0;                // GB_MIXED launch shape (kShape3*); 0 = the default
  int *d_tab = nullptr;
  double *d_bary = nullptr;
  MeshRec3 *d_mesh = nullptr;
  double *d_X = nullptr, *d_xn = nullptr, *d_shape = nullptr, *d_clock = nullptr;
  int *d_status = nullptr;
  void *d_qn = nullptr, *d_b1 = nullptr, *d_b2 = nullptr, *d_F0 = nullptr, *d_acc = nullptr;
  double *d_tmp = nullptr;
  size_t tmp_bytes = 0;
  // diagnostics: 1^T Mhat (Np), 6 result slots, block partials; the record ring and its
  // counters (steps since recording began, records written)
  double *d_diag = nullptr, *d_hist = nullptr;
  int64_t *d_hctl = nullptr;
  int diag_every = 0;
  int64_t diag_cap = 0;
  int64_t device_bytes = 0;
};

static int fail3(Solver3 *s, std::string *err, int code, const std::string &msg) {
  if (s) s->err = msg;
  if (err) *err = msg;
  return code;
}

static int cuda_fail3(Solver3 *s, cudaError_t e, const char *where) {
  return fail3(s, nullptr, GB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static int alloc3(Solver3 *s, void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail3(s, nullptr, GB_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  s->device_bytes += (int64_t)bytes;
  return GB_OK;
}

static void free3(Solver3 *s) {
  void *ptrs[] = {s->d_ops, s->d_ops_tc, s->d_tab, s->d_bary, s->d_mesh, s->d_X, s->d_xn, s->d_shape, s->d_clock, s->d_status,
                  s->d_qn, s->d_b1, s->d_b2, s->d_F0, s->d_acc, s->d_tmp, s->d_diag, s->d_hist, s->d_hctl};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (s->graph) cudaGraphExecDestroy(s->graph);
}

static int ensure_tmp3(Solver3 *s, size_t bytes) {
  if (s->tmp_bytes >= bytes) return GB_OK;
  if (s->d_tmp) {
    cudaFree(s->d_tmp);
    s->device_bytes -= (int64_t)s->tmp_bytes;
    s->d_tmp = nullptr;
    s->tmp_bytes = 0;
  }
  int rc = alloc3(s, (void **)&s->d_tmp, bytes);
  if (rc == GB_OK) s->tmp_bytes = bytes;
  return rc;
}

static void drop_graph3(Solver3 *s) {
  if (s->graph) cudaGraphExecDestroy(s->graph);
  s->graph = nullptr;
  s->graph_dt = -1.0;
  s->graph_warm = false;
}

static const int kFace3[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

int s3_create(const gb_mesh *mesh, int N, double Ma, double Re, int precision, void *stream, Solver3 **out,
              std::string &err) {
  *out = nullptr;
  if (N < 1 || N > GB3_MAX_N) return fail3(nullptr, &err, GB_EINVAL, "N must be in 1..4 for dim = 3");
  const int64_t K = mesh->n_elem, nv = mesh->n_vert;
  if (K >= (int64_t(1) << 26)) return fail3(nullptr, &err, GB_EINVAL, "n_elem must be < 2^26 for dim = 3");
  for (int64_t i = 0; i < 4 * K; ++i)
    if (mesh->EToV[i] < 0 || mesh->EToV[i] >= nv) return fail3(nullptr, &err, GB_EINVAL, "EToV entry out of range");
  std::vector<double> sh(12 * K, 0.0);
  if (mesh->elem_shift) memcpy(sh.data(), mesh->elem_shift, sizeof(double) * 12 * K);
  double period[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < 12 * K; ++i) {
    if (!std::isfinite(sh[i])) return fail3(nullptr, &err, GB_EINVAL, "non-finite elem_shift");
    const double v = fabs(sh[i]);
    const int d = (int)(i % 3);
    if (v > 0.0 && (period[d] == 0.0 || v < period[d])) period[d] = v;
  }
  std::vector<MeshRec3> rec(K);
  for (int64_t e = 0; e < K; ++e) {
    MeshRec3 &r = rec[e];
    memset(&r, 0, sizeof(r));
    for (int k = 0; k < 4; ++k) r.v[k] = mesh->EToV[4 * e + k];
    for (int k = 0; k < 12; ++k) {
      const double p = period[k % 3], v = sh[12 * e + k];
      const long m = p > 0.0 ? lround(v / p) : 0;
      if (labs(m) > 7 || fabs(v - m * p) > 1e-12 * (1.0 + fabs(v)))
        return fail3(nullptr, &err, GB_EINVAL, "elem_shift entries must be small integer multiples of one period per direction");
      r.shift[k] = (int8_t)m;
    }
  }
  auto vx = [&](int64_t e, int k, int d) {
    return mesh->X[3 * (int64_t)rec[e].v[k] + d] + rec[e].shift[3 * k + d] * period[d];
  };
  for (int64_t e = 0; e < K; ++e) {
    double a[3][3];
    for (int q = 0; q < 3; ++q)
      for (int d = 0; d < 3; ++d) a[q][d] = vx(e, q + 1, d) - vx(e, 0, d);
    const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                       a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    if (!(det > 0.0)) {
      char buf[128];
      snprintf(buf, sizeof(buf), "element %lld is not positively oriented (J <= 0)", (long long)e);
      return fail3(nullptr, &err, GB_EMESH, buf);
    }
  }
  // faces by sorted vertex-id triples; each must be shared by exactly two elements, the two
  // copies related by one translation; the permutation code maps my face vertex i to the
  // neighbour's face vertex kPerm3[p][i]
  struct Key {
    uint32_t a, b, c;
    bool operator==(const Key &o) const { return a == o.a && b == o.b && c == o.c; }
  };
  struct KeyHash {
    size_t operator()(const Key &k) const { return ((size_t)k.a * 0x9E3779B97F4A7C15ull) ^ ((size_t)k.b * 0xBF58476D1CE4E5B9ull) ^ k.c; }
  };
  std::unordered_map<Key, int64_t, KeyHash> first;
  first.reserve((size_t)(4 * K));
  for (int64_t e = 0; e < K; ++e)
    for (int f = 0; f < 4; ++f) {
      uint32_t id[3];
      for (int i = 0; i < 3; ++i) id[i] = (uint32_t)rec[e].v[kFace3[f][i]];
      if (id[0] == id[1] || id[1] == id[2] || id[0] == id[2]) return fail3(nullptr, &err, GB_EMESH, "degenerate face (repeated vertex id)");
      uint32_t srt[3] = {id[0], id[1], id[2]};
      std::sort(srt, srt + 3);
      const Key key{srt[0], srt[1], srt[2]};
      auto it = first.find(key);
      if (it == first.end()) {
        first.emplace(key, e * 4 + f);
        continue;
      }
      if (it->second < 0) return fail3(nullptr, &err, GB_EMESH, "a face is shared by more than two elements");
      const int64_t e2 = it->second / 4;
      const int f2 = (int)(it->second % 4);
      it->second = -1;
      uint32_t id2[3];
      for (int i = 0; i < 3; ++i) id2[i] = (uint32_t)rec[e2].v[kFace3[f2][i]];
      int p12 = -1, p21 = -1;
      for (int p = 0; p < 6; ++p) {
        bool ok12 = true, ok21 = true;
        for (int i = 0; i < 3; ++i) {
          ok12 &= id[i] == id2[kPerm3[p][i]];
          ok21 &= id2[i] == id[kPerm3[p][i]];
        }
        if (ok12) p12 = p;
        if (ok21) p21 = p;
      }
      if (p12 < 0 || p21 < 0) return fail3(nullptr, &err, GB_EMESH, "inconsistent face vertex ids");
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) {
          const double t0 = vx(e, kFace3[f][0], d) - vx(e2, kFace3[f2][kPerm3[p12][0]], d);
          const double ti = vx(e, kFace3[f][i], d) - vx(e2, kFace3[f2][kPerm3[p12][i]], d);
          if (fabs(ti - t0) > 1e-9 * (1.0 + fabs(period[d]))) return fail3(nullptr, &err, GB_EMESH, "periodic face copies do not match");
        }
      rec[e].nbr[f] = (int32_t)((e2 << 5) | (p12 << 2) | f2);
      rec[e2].nbr[f2] = (int32_t)((e << 5) | (p21 << 2) | f);
    }
  for (const auto &kv : first)
    if (kv.second >= 0) return fail3(nullptr, &err, GB_EMESH, "the mesh is not closed: a face has no neighbour (only periodic meshes are supported)");

  Solver3 *s = new Solver3();
  s->N = N;
  s->K = K;
  s->nv = nv;
  s->precision = precision;
  s->c = 1.0 / Ma;
  s->tau = Ma * Ma / Re;
  for (int d = 0; d < 3; ++d) s->period[d] = period[d];
  s->stream = (cudaStream_t)stream;
  s->elem_bytes = precision == GB_FP64 ? sizeof(double) : sizeof(float);
  if (!build_reference3d(N, s->ref)) {
    delete s;
    return fail3(nullptr, &err, GB_EINVAL, "reference operator construction failed (dim = 3)");
  }
  s->Np = s->ref.Np;
  s->Nfp = s->ref.Nfp;
  s->Nc = s->ref.Nc;
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
  s->device = dev;
  if (ce != cudaSuccess) {
    delete s;
    return fail3(nullptr, &err, GB_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
  }
  size_t opbytes = 0;
  int rc = upload_ops3(N, precision == GB_FP64, s->ref, &s->d_ops, &s->d_tab, &s->d_bary, &opbytes, s->stream);
  if (rc) {
    std::string m = std::string("operator upload: ") + cudaGetErrorString((cudaError_t)rc);
    free3(s);
    delete s;
    return fail3(nullptr, &err, GB_ECUDA, m);
  }
  s->device_bytes += (int64_t)opbytes;
  if (precision == GB_MIXED && stage3_tc_supported(N)) {
    size_t tcbytes = 0;
    rc = upload_ops3_tc(N, s->ref, &s->d_ops_tc, &tcbytes, s->stream);
    if (rc) {
      std::string m = std::string("operator upload (tensor-core table): ") + cudaGetErrorString((cudaError_t)rc);
      free3(s);
      delete s;
      return fail3(nullptr, &err, GB_ECUDA, m);
    }
    s->device_bytes += (int64_t)tcbytes;
  }
  const size_t fbytes = (size_t)K * 10 * s->Np * s->elem_bytes;
  void **fields[] = {&s->d_qn, &s->d_b1, &s->d_b2, &s->d_F0, &s->d_acc};
  int arc = GB_OK;
  arc = arc ? arc : alloc3(s, (void **)&s->d_mesh, sizeof(MeshRec3) * K);
  arc = arc ? arc : alloc3(s, (void **)&s->d_X, sizeof(double) * 3 * nv);
  arc = arc ? arc : alloc3(s, (void **)&s->d_xn, sizeof(double) * 3 * nv);
  arc = arc ? arc : alloc3(s, (void **)&s->d_shape, sizeof(double) * 6 * nv);
  arc = arc ? arc : alloc3(s, (void **)&s->d_clock, sizeof(double) * 4);
  arc = arc ? arc : alloc3(s, (void **)&s->d_status, sizeof(int));
  for (void **p : fields) arc = arc ? arc : alloc3(s, p, fbytes);
  if (arc != GB_OK) {
    err = s->err;
    free3(s);
    delete s;
    return arc;
  }
  const double clock0[4] = {0, 0, 0, 0};
  const int zero = 0;
  ce = cudaMemcpyAsync(s->d_mesh, rec.data(), sizeof(MeshRec3) * K, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_X, mesh->X, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_xn, mesh->X, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->d_shape, 0, sizeof(double) * 6 * nv, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_clock, clock0, sizeof(clock0), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
  for (void **p : fields)
    if (ce == cudaSuccess) ce = cudaMemsetAsync(*p, 0, fbytes, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) {
    cuda_fail3(s, ce, "gb_create upload (dim = 3)");
    err = s->err;
    free3(s);
    delete s;
    return GB_ECUDA;
  }
  *out = s;
  return GB_OK;
}

void s3_destroy(Solver3 *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  free3(s);
  delete s;
}

const char *s3_error(Solver3 *s) { return s->err.c_str(); }

int s3_set_static(Solver3 *s) {
  s->moving = 0;
  s->omega = 0.0;
  drop_graph3(s);
  cudaError_t ce = cudaMemsetAsync(s->d_shape, 0, sizeof(double) * 6 * s->nv, s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "gb_set_motion (dim = 3)");
}

int s3_set_wave_motion(Solver3 *s, const gb_wave_motion *m) {
  const double vals[8] = {m->A0, m->A1, m->Lx, m->wavelength, m->omega, m->r0sq, m->yc, m->zc};
  for (double v : vals)
    if (!std::isfinite(v)) return fail3(s, nullptr, GB_EINVAL, "gb_wave_motion: non-finite parameter");
  if (!(m->Lx != 0.0) || !(m->wavelength != 0.0) || !(m->r0sq > 0.0))
    return fail3(s, nullptr, GB_EINVAL, "gb_wave_motion needs Lx != 0, wavelength != 0 and r0sq > 0");
  s->wave = Wave3{m->A0, m->A1, m->Lx, m->wavelength, m->omega, m->r0sq, m->yc, m->zc};
  s->moving = (m->A0 != 0.0 || m->A1 != 0.0) && m->omega != 0.0;
  s->omega = m->omega;
  drop_graph3(s);
  int rc = launch_shape3(s->d_X, s->d_shape, s->nv, s->wave, s->stream);
  return rc ? cuda_fail3(s, (cudaError_t)rc, "shape kernel (dim = 3)") : GB_OK;
}

int s3_set_tgv_motion(Solver3 *s, double A, double T, double L) {
  if (!std::isfinite(A) || !std::isfinite(T) || !std::isfinite(L) || !(T > 0.0) || !(L != 0.0))
    return fail3(s, nullptr, GB_EINVAL, "GB_MOTION_TGV3D needs finite A, T > 0 and L != 0");
  s->omega = 2.0 * 3.14159265358979323846 / T;
  s->moving = A != 0.0;
  drop_graph3(s);
  int rc = launch_shape3_tgv(s->d_X, s->d_shape, s->nv, A, s->omega, L, s->stream);
  return rc ? cuda_fail3(s, (cudaError_t)rc, "shape kernel (dim = 3)") : GB_OK;
}

int s3_set_fields(Solver3 *s, const double *q, double t) {
  const size_t n = (size_t)s->K * 10 * s->Np;
  cudaError_t ce;
  if (s->precision == GB_FP64) {
    ce = cudaMemcpyAsync(s->d_qn, q, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
  } else {
    int rc = ensure_tmp3(s, n * sizeof(double));
    if (rc) return rc;
    ce = cudaMemcpyAsync(s->d_tmp, q, n * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (ce == cudaSuccess) {
      int lr = launch_cast3(s->d_tmp, (float *)s->d_qn, s->K, s->Np, true, s->stream);
      if (lr) ce = (cudaError_t)lr;
    }
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_clock, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "gb_set_fields (dim = 3)");
}

int s3_sync(Solver3 *s) {
  int status = 0, zero = 0;
  cudaError_t ce = cudaMemcpyAsync(&status, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(s->d_status, &zero, sizeof(int), cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_sync (dim = 3)");
  if (status & GB_STATUS_MESH) return fail3(s, nullptr, GB_EMESH, "an element reached J <= 0 during a stage");
  if (status & GB_STATUS_NAN) return fail3(s, nullptr, GB_ENAN, "a NaN or Inf appeared in the fields");
  return GB_OK;
}

int s3_fields(Solver3 *s, double *q, double *t) {
  const int st = s3_sync(s);
  const size_t n = (size_t)s->K * 10 * s->Np;
  cudaError_t ce = cudaSuccess;
  if (q) {
    if (s->precision == GB_FP64) {
      ce = cudaMemcpyAsync(q, s->d_qn, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    } else {
      int rc = ensure_tmp3(s, n * sizeof(double));
      if (rc) return rc;
      int lr = launch_cast3(s->d_tmp, (float *)s->d_qn, s->K, s->Np, false, s->stream);
      ce = lr ? (cudaError_t)lr : cudaMemcpyAsync(q, s->d_tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    }
  }
  double clk[4] = {0, 0, 0, 0};
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(clk, s->d_clock, sizeof(clk), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_fields (dim = 3)");
  if (t) *t = clk[0];
  return st;
}

int s3_set_vertices(Solver3 *s, const double *x) {
  cudaError_t ce = cudaMemcpyAsync(s->d_xn, x, sizeof(double) * 3 * s->nv, cudaMemcpyHostToDevice, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "gb_set_vertices (dim = 3)");
}

int s3_vertices(Solver3 *s, double *x) {
  cudaError_t ce = cudaMemcpyAsync(x, s->d_xn, sizeof(double) * 3 * s->nv, cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "gb_vertices (dim = 3)");
}

int s3_nodes(Solver3 *s, double *xyz) {
  const size_t n = (size_t)s->K * s->Np * 3;
  int rc = ensure_tmp3(s, n * sizeof(double));
  if (rc) return rc;
  int lr = launch_nodes3(s->d_bary, s->Np, s->d_xn, s->d_mesh, s->period, s->K, s->d_tmp, s->stream);
  cudaError_t ce = lr ? (cudaError_t)lr : cudaMemcpyAsync(xyz, s->d_tmp, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "gb_nodes (dim = 3)");
}

static void set_coef3(Solver3 *s, double dt) {
  if (dt == s->coef_dt) return;
  double E[5], A[16], B[4];
  sark_coefficients(0.0, E, A, B);
  memcpy(s->co.E[0], E, sizeof(E)); memcpy(s->co.A[0], A, sizeof(A)); memcpy(s->co.B[0], B, sizeof(B));
  sark_coefficients(-dt / s->tau, E, A, B);
  memcpy(s->co.E[1], E, sizeof(E)); memcpy(s->co.A[1], A, sizeof(A)); memcpy(s->co.B[1], B, sizeof(B));
  s->coef_dt = dt;
}

static Diag3Args diag_args3(Solver3 *s) {
  Diag3Args d;
  d.q = s->d_qn;
  d.is_float = s->precision != GB_FP64;
  d.Np = s->Np;
  d.mesh = s->d_mesh;
  d.xn = s->d_xn;
  for (int k = 0; k < 3; ++k) d.period[k] = s->period[k];
  d.wq = s->d_diag;
  d.c = s->c;
  d.K = s->K;
  d.part = s->d_diag + s->Np + 6;
  return d;
}

static int ensure_diag3(Solver3 *s) {
  if (s->d_diag) return GB_OK;
  int rc = alloc3(s, (void **)&s->d_diag, sizeof(double) * (s->Np + 6 + 6 * (size_t)kDiag3MaxBlocks));
  if (rc) return rc;
  cudaError_t ce = cudaMemcpyAsync(s->d_diag, s->ref.wq.data(), sizeof(double) * s->Np, cudaMemcpyHostToDevice, s->stream);
  return ce == cudaSuccess ? GB_OK : cuda_fail3(s, ce, "diagnostics set-up (dim = 3)");
}

int s3_diagnostics(Solver3 *s, double *out) {
  int rc = ensure_diag3(s);
  if (rc) return rc;
  rc = launch_diagnostics3(diag_args3(s), s->d_diag + s->Np, s->stream);
  if (rc) return cuda_fail3(s, (cudaError_t)rc, "gb_diagnostics (dim = 3)");
  double r[6];
  cudaError_t ce = cudaMemcpyAsync(r, s->d_diag + s->Np, sizeof(r), cudaMemcpyDeviceToHost, s->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_diagnostics (dim = 3)");
  out[0] = r[0];
  out[1] = r[1] / r[5];
  out[2] = r[2];
  out[3] = r[3];
  out[4] = r[4];
  out[5] = r[5];
  return GB_OK;
}

static void free_ring3(Solver3 *s) {
  if (s->d_hist) {
    cudaFree(s->d_hist);
    s->device_bytes -= (int64_t)(sizeof(double) * 6 * (size_t)s->diag_cap);
    s->d_hist = nullptr;
  }
  if (s->d_hctl) {
    cudaFree(s->d_hctl);
    s->device_bytes -= (int64_t)(2 * sizeof(int64_t));
    s->d_hctl = nullptr;
  }
  s->diag_every = 0;
  s->diag_cap = 0;
}

int s3_set_diagnostics(Solver3 *s, int every, int64_t capacity) {
  cudaError_t ce = s->stream ? cudaStreamSynchronize(s->stream) : cudaDeviceSynchronize();
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_set_diagnostics (dim = 3)");
  drop_graph3(s);
  free_ring3(s);
  if (every == 0) return GB_OK;
  int rc = ensure_diag3(s);
  if (!rc) rc = alloc3(s, (void **)&s->d_hist, sizeof(double) * 6 * (size_t)capacity);
  if (!rc) {
    s->diag_cap = capacity;
    rc = alloc3(s, (void **)&s->d_hctl, 2 * sizeof(int64_t));
  }
  if (rc) {
    free_ring3(s);
    return rc;
  }
  ce = cudaMemsetAsync(s->d_hctl, 0, 2 * sizeof(int64_t), s->stream);
  if (ce != cudaSuccess) {
    free_ring3(s);
    return cuda_fail3(s, ce, "gb_set_diagnostics (dim = 3)");
  }
  s->diag_every = every;
  return GB_OK;
}

void *s3_stream(Solver3 *s) { return (void *)s->stream; }

int s3_diag_ring(Solver3 *s, const double **hist, const int64_t **ctl, int *every, int64_t *capacity) {
  *hist = s->d_hist;
  *ctl = s->d_hctl;
  *every = s->diag_every;
  *capacity = s->diag_cap;
  return GB_OK;
}

// the stage kernel of the solver's precision and launch shape: GB_FP64 and the FP32
// one-thread-per-node kernel (gb_kernels3d.cu), or the tensor-core kernel (gb_kernels3d_tc.cu)
static int launch3(Solver3 *s, const Stage3Args &a) {
  // (the tensor-core kernel stores the right-hand side as node pairs: an F_dev that is not
  // 8-byte aligned goes to the one-thread-per-node kernel)
  const bool fout_ok = a.stage >= 0 || (reinterpret_cast<uintptr_t>(a.Fout) & 7) == 0;
  if (s->precision == GB_MIXED && s->d_ops_tc && s->shape != kShape3Simt && fout_ok)
    return launch_stage3_tc(s->N, a, s->stream, s->shape ? s->shape : stage3_tc_max_warps(s->N), s->num_sms);
  return launch_stage3(s->N, s->precision == GB_FP64, a, s->stream, s->num_sms);
}

static Stage3Args base3(Solver3 *s) {
  Stage3Args a;
  memset(&a, 0, sizeof(a));
  a.xn = s->d_xn;
  a.shape = s->d_shape;
  a.mesh = s->d_mesh;
  a.ops = s->d_ops;
  a.ops_tc = s->d_ops_tc;
  a.tab = s->d_tab;
  a.clock = s->d_clock;
  a.status = s->d_status;
  a.K = s->K;
  for (int d = 0; d < 3; ++d) a.period[d] = s->period[d];
  a.c = s->c;
  a.inv_tau = 1.0 / s->tau;
  a.moving = s->moving;
  a.omega = s->omega;
  a.co = s->co;
  return a;
}

int s3_rhs(Solver3 *s, double t, const void *q_dev, void *F_dev) {
  Stage3Args a = base3(s);
  a.stage = -1;
  a.qin = q_dev;
  a.qn = q_dev;
  a.Fout = F_dev;
  a.rhs_time = t;
  int rc = launch3(s, a);
  return rc ? cuda_fail3(s, (cudaError_t)rc, "stage kernel launch (dim = 3)") : GB_OK;
}

// one SARK step: stages 0..3 (q_n -> b1 -> b2 -> b1 -> q_n) and the vertex update;
// events (optional) bracket every launch for tracing
static int step_once3(Solver3 *s, double dt, cudaEvent_t *ev) {
  Stage3Args a = base3(s);
  a.dt = dt;
  a.qn = s->d_qn;
  a.F0 = s->d_F0;
  a.acc = s->d_acc;
  const void *in[4] = {s->d_qn, s->d_b1, s->d_b2, s->d_b1};
  void *outp[4] = {s->d_b1, s->d_b2, s->d_b1, s->d_qn};
  for (int i = 0; i < 4; ++i) {
    a.stage = i;
    a.qin = in[i];
    a.qout = outp[i];
    if (ev) cudaEventRecord(ev[2 * i], s->stream);
    int rc = launch3(s, a);
    if (rc) return cuda_fail3(s, (cudaError_t)rc, "stage kernel launch (dim = 3)");
    if (ev) cudaEventRecord(ev[2 * i + 1], s->stream);
  }
  if (ev) cudaEventRecord(ev[8], s->stream);
  int rc = launch_vertex_update3(s->d_xn, s->d_shape, s->nv, s->d_clock, dt, s->stream);
  if (rc) return cuda_fail3(s, (cudaError_t)rc, "vertex update launch (dim = 3)");
  if (ev) cudaEventRecord(ev[9], s->stream);
  if (s->diag_every > 0) {
    // integrals of q_{n+1} on x_{n+1} at t_{n+1} (the clock has advanced), every diag_every-th step
    rc = launch_diagnostics3_record(diag_args3(s), s->d_clock, s->d_hctl, s->diag_every, s->d_hist, s->diag_cap,
                                    s->stream);
    if (rc) return cuda_fail3(s, (cudaError_t)rc, "diagnostics record launch (dim = 3)");
  }
  return GB_OK;
}

// GB_MIXED launch tuner (N <= 3), once per solver: time stages 0, 1 and 2 on the solver's own
// state (outputs into F_0 and the stage buffers, which hold nothing between steps; the state
// is not changed) for the tensor-core kernel with the most warps per CTA and for the
// one-thread-per-node kernel, and keep the faster (the second must win by 3%).  Not cached
// across solvers: the two kernels are close, and which wins depends on the mesh and motion,
// not only on N and K.
static int tune3(Solver3 *s) {
  if (s->precision != GB_MIXED || !s->d_ops_tc || s->shape != 0) return GB_OK;
  Stage3Args a = base3(s);
  a.dt = s->coef_dt;
  a.qn = s->d_qn;
  a.F0 = s->d_F0;
  a.acc = s->d_acc;
  const void *in[3] = {s->d_qn, s->d_b1, s->d_b2};
  void *outp[3] = {s->d_b1, s->d_b2, s->d_b1};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  const int cand[2] = {stage3_tc_max_warps(s->N), kShape3Simt};
  int best = cand[0];
  float best_ms = 1e30f;
  for (int i = 0; i < 2 && ce == cudaSuccess; ++i) {
    s->shape = cand[i];
    for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {   // warm-up, then timed
      if (rep == 1) ce = cudaEventRecord(e0, s->stream);
      for (int st = 0; st < 3 && ce == cudaSuccess; ++st) {
        a.stage = st;
        a.qin = in[st];
        a.qout = outp[st];
        const int rc = launch3(s, a);
        if (rc) ce = (cudaError_t)rc;
      }
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
  s->shape = 0;
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "launch tuning (dim = 3)");
  s->shape = best;
  return GB_OK;
}

int s3_step(Solver3 *s, double dt, int64_t nsteps) {
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail3(s, nullptr, GB_EINVAL, "dt must be positive and nsteps >= 0");
  set_coef3(s, dt);
  if (nsteps > 0) {
    const int trc = tune3(s);
    if (trc) return trc;
  }
  if (dt != s->graph_dt) drop_graph3(s);
  const bool can_graph = s->use_graph && s->stream != nullptr && nsteps >= 2;
  int64_t done = 0;
  if (can_graph && !s->graph) {
    if (!s->graph_warm) {
      int rc = step_once3(s, dt, nullptr);
      if (rc) return rc;
      s->graph_warm = true;
      ++done;
    }
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail3(s, ce, "graph capture (dim = 3)");
    int rc = step_once3(s, dt, nullptr);
    ce = cudaStreamEndCapture(s->stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&s->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail3(s, ce, "graph instantiate (dim = 3)");
    s->graph_dt = dt;
  }
  for (; done < nsteps; ++done) {
    if (s->graph) {
      cudaError_t ce = cudaGraphLaunch(s->graph, s->stream);
      if (ce != cudaSuccess) return cuda_fail3(s, ce, "graph launch (dim = 3)");
    } else {
      int rc = step_once3(s, dt, nullptr);
      if (rc) return rc;
      s->graph_warm = true;
    }
  }
  return GB_OK;
}

int s3_step_timed(Solver3 *s, double dt, int64_t nsteps, double *kernel_ms) {
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail3(s, nullptr, GB_EINVAL, "dt must be positive and nsteps >= 0");
  set_coef3(s, dt);
  if (nsteps > 0) {
    const int trc = tune3(s);
    if (trc) return trc;
  }
  cudaEvent_t ev[10];
  for (auto &e : ev) e = nullptr;
  cudaError_t ce = cudaSuccess;
  for (auto &e : ev)
    if (ce == cudaSuccess) ce = cudaEventCreate(&e);
  for (int64_t n = 0; n < nsteps && ce == cudaSuccess; ++n) {
    int rc = step_once3(s, dt, ev);
    if (rc) {
      for (auto &e : ev) if (e) cudaEventDestroy(e);
      return rc;
    }
    ce = cudaEventSynchronize(ev[9]);
    for (int k = 0; k < 5 && ce == cudaSuccess; ++k) {
      float ms = 0.0f;
      ce = cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
      kernel_ms[k] += ms;
    }
  }
  for (auto &e : ev) if (e) cudaEventDestroy(e);
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_step_timed (dim = 3)");
  return s3_sync(s);
}

int s3_info(Solver3 *s, int *Np, int *Nfp, int *Nc, int64_t *n_elem, int64_t *n_vert, double *c, double *tau,
            int64_t *device_bytes) {
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

int s3_state_ptr(Solver3 *s, void **q) {
  *q = s->d_qn;
  return GB_OK;
}

int s3_launch_config(Solver3 *s, int *shape) {
  if (s->precision != GB_MIXED) *shape = 0;
  else if (!s->d_ops_tc) *shape = kShape3Simt;
  else *shape = s->shape ? s->shape : stage3_tc_max_warps(s->N);
  return GB_OK;
}

int s3_set_launch_config(Solver3 *s, int shape) {
  if (s->precision != GB_MIXED) return fail3(s, nullptr, GB_EINVAL, "launch shapes apply to GB_MIXED solvers");
  if (shape != kShape3Simt) {
    if (!s->d_ops_tc) return fail3(s, nullptr, GB_EINVAL, "the tensor-core kernel needs N <= 3 (dim = 3); shape 16 is the one-thread-per-node kernel");
    if (shape < 1 || shape > stage3_tc_max_warps(s->N))
      return fail3(s, nullptr, GB_EINVAL, "the launch shape must be 1.." + std::to_string(stage3_tc_max_warps(s->N)) +
                                              " (tensor-core kernel, warps per CTA) or 16 (one thread per node) for dim = 3");
  }
  s->shape = shape;
  drop_graph3(s);
  return GB_OK;
}

int s3_set_graph(Solver3 *s, int enable) {
  s->use_graph = enable != 0;
  drop_graph3(s);
  return GB_OK;
}

int s3_set_stream(Solver3 *s, void *stream) {
  cudaError_t ce = cudaStreamSynchronize(s->stream);
  if (ce != cudaSuccess) return cuda_fail3(s, ce, "gb_set_stream (dim = 3)");
  s->stream = (cudaStream_t)stream;
  drop_graph3(s);
  return GB_OK;
}

}  // namespace gb

extern "C" int gb_reference_operators3d(int N, double *r, double *s, double *t, double *Dr, double *Ds, double *Dt,
                                        double *LIFT, double *Icub, double *Pcub, double *cr, double *cs, double *ct,
                                        double *cw, int *Nc_out) {
  gb::RefOps3 R;
  if (!gb::build_reference3d(N, R)) return GB_EINVAL;
  auto put = [](const std::vector<double> &v, double *out) {
    if (out) memcpy(out, v.data(), v.size() * sizeof(double));
  };
  put(R.r, r); put(R.s, s); put(R.t, t);
  put(R.Dr, Dr); put(R.Ds, Ds); put(R.Dt, Dt); put(R.LIFT, LIFT);
  put(R.I, Icub); put(R.P, Pcub);
  put(R.cr, cr); put(R.cs, cs); put(R.ct, ct); put(R.cw, cw);
  if (Nc_out) *Nc_out = R.Nc;
  return GB_OK;
}
