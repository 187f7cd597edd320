// Entry points of the 3D solver (gb3d.cpp) used by the C ABI in gb_api.cpp when a
// solver is created with mesh->dim == 3.  Same arguments and return codes as the
// public calls of include/gb.h of the same name.
#ifndef GB3D_H
#define GB3D_H

#include <stdint.h>

#include <string>

#include "gb.h"

namespace gb {

struct Solver3;

int s3_create(const gb_mesh *mesh, int N, double Ma, double Re, int precision, void *stream, Solver3 **out,
              std::string &err);
void s3_destroy(Solver3 *s);
const char *s3_error(Solver3 *s);
int s3_set_static(Solver3 *s);
int s3_set_wave_motion(Solver3 *s, const gb_wave_motion *m);
int s3_set_tgv_motion(Solver3 *s, double A, double T, double L);
int s3_diagnostics(Solver3 *s, double *out6);
int s3_set_diagnostics(Solver3 *s, int every, int64_t capacity);
// the record ring of gb_set_diagnostics (device pointers; NULL and every = 0 when off)
void *s3_stream(Solver3 *s);   // the solver's cudaStream_t (NULL = legacy default stream)
int s3_diag_ring(Solver3 *s, const double **hist, const int64_t **ctl, int *every, int64_t *capacity);
int s3_set_fields(Solver3 *s, const double *q, double t);
int s3_fields(Solver3 *s, double *q, double *t);
int s3_sync(Solver3 *s);
int s3_set_vertices(Solver3 *s, const double *x);
int s3_vertices(Solver3 *s, double *x);
int s3_nodes(Solver3 *s, double *xyz);
int s3_rhs(Solver3 *s, double t, const void *q_dev, void *F_dev);
int s3_step(Solver3 *s, double dt, int64_t nsteps);
int s3_step_timed(Solver3 *s, double dt, int64_t nsteps, double *kernel_ms);
int s3_info(Solver3 *s, int *Np, int *Nfp, int *Nc, int64_t *n_elem, int64_t *n_vert, double *c, double *tau,
            int64_t *device_bytes);
int s3_state_ptr(Solver3 *s, void **q);
int s3_set_graph(Solver3 *s, int enable);
// GB_MIXED launch shapes: 1..stage3_tc_max_warps(N) the tensor-core kernel with that many warps
// per CTA (N <= 3; the default, until the first step tunes it, is the most that fit), kShape3Simt the FP32
// one-thread-per-node kernel (every order)
constexpr int kShape3Simt = 16;
int s3_launch_config(Solver3 *s, int *shape);
int s3_set_launch_config(Solver3 *s, int shape);
int s3_set_stream(Solver3 *s, void *stream);

}  // namespace gb

#endif
