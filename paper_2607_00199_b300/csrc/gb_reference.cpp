// Host-side construction of the order-N reference operators and SARK coefficients.
//
// Everything here is set-up work done once per solver (or per dt) in long
// double and rounded to FP64 for upload:
//  * Warp & Blend nodes (Warburton 2006) on the reference triangle, the node set
//    of the paper's Sec. 3, with Warburton's optimised blend parameter alpha;
//  * the orthonormal Koornwinder-Dubiner modal basis and its Vandermonde
//    matrices, giving Dr = Vr V^-1, Ds = Vs V^-1 (D = M^-1 S of Sec. 3),
//    LIFT = V V^T E with E the 1D Gauss-Lobatto face mass (M^-1 M^f of Sec. 3);
//  * the degree-3N Stroud conical-product cubature (Gauss-Legendre x
//    Gauss-Jacobi(1,0), both by Golub-Welsch) with I = Vc V^-1 and
//    P = V V^T I^T W (the projection of Sec. 3);
//  * the SARK-4 coefficients of Sec. 4 written through phi-functions.
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "gb_internal.h"

namespace gb {

typedef long double ld;

static const ld kPi = 3.141592653589793238462643383279502884L;

// ---- small dense linear algebra ------------------------------------------

// Inverse of an n x n row-major matrix by Gauss-Jordan with partial pivoting.
static bool invert(std::vector<ld> a, int n, std::vector<ld> &inv) {
  inv.assign((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0L;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabsl(a[(size_t)r * n + col]) > fabsl(a[(size_t)piv * n + col])) piv = r;
    if (fabsl(a[(size_t)piv * n + col]) < 1e-300L) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    ld d = 1.0L / a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] *= d;
      inv[(size_t)col * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      ld f = a[(size_t)r * n + col];
      if (f == 0.0L) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  return true;
}

// C = A (m x k) * B (k x n), row-major.
static std::vector<ld> matmul(const std::vector<ld> &A, const std::vector<ld> &B, int m, int k, int n) {
  std::vector<ld> C((size_t)m * n, 0.0L);
  for (int i = 0; i < m; ++i)
    for (int p = 0; p < k; ++p) {
      ld a = A[(size_t)i * k + p];
      for (int j = 0; j < n; ++j) C[(size_t)i * n + j] += a * B[(size_t)p * n + j];
    }
  return C;
}

static std::vector<ld> transpose(const std::vector<ld> &A, int m, int n) {
  std::vector<ld> T((size_t)n * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) T[(size_t)j * m + i] = A[(size_t)i * n + j];
  return T;
}

// Eigen-decomposition of a symmetric n x n matrix by cyclic Jacobi rotations.
// On return a holds the eigenvalues on its diagonal, v the eigenvectors (columns).
static void jacobi_eigen(std::vector<ld> &a, int n, std::vector<ld> &v) {
  v.assign((size_t)n * n, 0.0L);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0L;
  for (int sweep = 0; sweep < 100; ++sweep) {
    ld off = 0.0L;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
    if (off < 1e-60L) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        ld apq = a[(size_t)p * n + q];
        if (fabsl(apq) < 1e-300L) continue;
        ld app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        ld theta = (aqq - app) / (2.0L * apq);
        ld t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
        ld c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
        for (int k = 0; k < n; ++k) {
          ld akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          ld apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          ld vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// ---- orthogonal polynomials -------------------------------------------------

// Three-term recurrence of the orthonormal Jacobi polynomials p_n for the weight
// (1-x)^a (1+x)^b:  x p_n = A_{n+1} p_{n+1} + B_n p_n + A_n p_{n-1}.
static ld jac_A(int n, ld a, ld b) {
  ld h = 2.0L * n + a + b;
  return 2.0L / h * sqrtl(n * (n + a + b) * (n + a) * (n + b) / ((h - 1.0L) * (h + 1.0L)));
}
static ld jac_B(int n, ld a, ld b) {
  if (n == 0) return (b - a) / (a + b + 2.0L);
  ld h = 2.0L * n + a + b;
  return (b * b - a * a) / (h * (h + 2.0L));
}
static ld jac_mass(ld a, ld b) {   // integral of the weight
  return powl(2.0L, a + b + 1.0L) * tgammal(a + 1.0L) * tgammal(b + 1.0L) / tgammal(a + b + 2.0L);
}

// Orthonormal Jacobi polynomial p_n^{(a,b)}(x).
static ld jacobi(ld x, ld a, ld b, int n) {
  ld p0 = 1.0L / sqrtl(jac_mass(a, b));
  if (n == 0) return p0;
  ld p1 = (x - jac_B(0, a, b)) * p0 / jac_A(1, a, b);
  for (int k = 1; k < n; ++k) {
    ld p2 = ((x - jac_B(k, a, b)) * p1 - jac_A(k, a, b) * p0) / jac_A(k + 1, a, b);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// d/dx p_n^{(a,b)} = sqrt(n (n+a+b+1)) p_{n-1}^{(a+1,b+1)} for the orthonormal family.
static ld jacobi_deriv(ld x, ld a, ld b, int n) {
  if (n == 0) return 0.0L;
  return sqrtl(n * (n + a + b + 1.0L)) * jacobi(x, a + 1.0L, b + 1.0L, n - 1);
}

// Gauss-Jacobi rule with n points (Golub-Welsch), nodes ascending.
static void gauss_jacobi(int n, ld a, ld b, std::vector<ld> &x, std::vector<ld> &w) {
  std::vector<ld> T((size_t)n * n, 0.0L), V;
  for (int i = 0; i < n; ++i) {
    T[(size_t)i * n + i] = jac_B(i, a, b);
    if (i + 1 < n) T[(size_t)i * n + i + 1] = T[(size_t)(i + 1) * n + i] = jac_A(i + 1, a, b);
  }
  jacobi_eigen(T, n, V);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (T[(size_t)order[j] * n + order[j]] < T[(size_t)order[i] * n + order[i]]) std::swap(order[i], order[j]);
  x.resize(n);
  w.resize(n);
  ld mu = jac_mass(a, b);
  for (int i = 0; i < n; ++i) {
    int k = order[i];
    x[i] = T[(size_t)k * n + k];
    w[i] = mu * V[k] * V[k];   // first component of the k-th eigenvector
  }
}

// N+1 Gauss-Lobatto points: +-1 and the Gauss-Jacobi(1,1) points of degree N-1.
static std::vector<ld> gauss_lobatto(int N) {
  std::vector<ld> x(N + 1);
  x[0] = -1.0L;
  x[N] = 1.0L;
  if (N > 1) {
    std::vector<ld> xi, wi;
    gauss_jacobi(N - 1, 1.0L, 1.0L, xi, wi);
    for (int i = 0; i < N - 1; ++i) x[i + 1] = xi[i];
  }
  return x;
}

// ---- Warp & Blend nodes -----------------------------------------------------

static ld alpha_opt(int N) {
  static const ld tab[15] = {0.0000L, 0.0000L, 1.4152L, 0.1001L, 0.2751L, 0.9800L, 1.0999L, 1.2832L,
                             1.3648L, 1.4773L, 1.4959L, 1.5743L, 1.5770L, 1.6223L, 1.6258L};
  return N <= 15 ? tab[N - 1] : 5.0L / 3.0L;
}

// 1D warp (GLL minus equidistant, interpolated on the equidistant points)
// divided by 1 - r^2; zero at the end points.  Barycentric Lagrange form.
static ld warp_over_blend(int N, ld r, const std::vector<ld> &gll) {
  if (fabsl(r) >= 1.0L - 1e-12L) return 0.0L;
  ld num = 0.0L, den = 0.0L;
  for (int i = 0; i <= N; ++i) {
    ld xi = -1.0L + 2.0L * i / N;
    ld wi = 1.0L;   // barycentric weight of equidistant point i
    for (int j = 0; j <= N; ++j)
      if (j != i) wi /= (xi - (-1.0L + 2.0L * j / N));
    if (fabsl(r - xi) < 1e-18L) return (gll[i] - xi) / (1.0L - r * r);
    ld t = wi / (r - xi);
    num += t * (gll[i] - xi);
    den += t;
  }
  return (num / den) / (1.0L - r * r);
}

static void warp_blend(int N, std::vector<ld> &r, std::vector<ld> &s) {
  const int Np = (N + 1) * (N + 2) / 2;
  r.resize(Np);
  s.resize(Np);
  std::vector<ld> gll = gauss_lobatto(N);
  ld alpha = alpha_opt(N);
  const ld sq3 = sqrtl(3.0L);
  int k = 0;
  for (int row = 0; row <= N; ++row)
    for (int m = 0; m <= N - row; ++m, ++k) {
      ld L1 = (ld)row / N, L3 = (ld)m / N, L2 = 1.0L - L1 - L3;
      // equilateral triangle, vertex of L1 on top
      ld x = L3 - L2, y = (2.0L * L1 - L2 - L3) / sq3;
      // edge L2-L3 (direction 0), L3-L1 (2 pi/3), L1-L2 (4 pi/3); blend 4 La Lb (1 + (alpha Lc)^2)
      ld Ls[3][3] = {{L2, L3, L1}, {L3, L1, L2}, {L1, L2, L3}};
      for (int e = 0; e < 3; ++e) {
        ld La = Ls[e][0], Lb = Ls[e][1], Lc = Ls[e][2];
        ld d = 4.0L * La * Lb * warp_over_blend(N, Lb - La, gll) * (1.0L + alpha * alpha * Lc * Lc);
        ld ang = 2.0L * kPi * e / 3.0L;
        x += cosl(ang) * d;
        y += sinl(ang) * d;
      }
      ld l1 = (sq3 * y + 1.0L) / 3.0L;
      ld l2 = (-3.0L * x - sq3 * y + 2.0L) / 6.0L;
      ld l3 = (3.0L * x - sq3 * y + 2.0L) / 6.0L;
      r[k] = l3 - l2 - l1;
      s[k] = l1 - l2 - l3;
    }
}

// ---- modal basis on the triangle ---------------------------------------------

struct Mode { int i, j; };
static std::vector<Mode> modes(int N) {
  std::vector<Mode> m;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j) m.push_back({i, j});
  return m;
}

// psi_ij(r,s) = sqrt2 p_i(a) p_j^{(2i+1,0)}(b) (1-b)^i and its (r,s) gradient.
static void mode_eval(ld r, ld s, int i, int j, ld *val, ld *dr, ld *ds) {
  ld a = (fabsl(1.0L - s) > 1e-16L) ? 2.0L * (1.0L + r) / (1.0L - s) - 1.0L : -1.0L;
  ld b = s;
  ld f = jacobi(a, 0, 0, i), df = jacobi_deriv(a, 0, 0, i);
  ld g = jacobi(b, 2.0L * i + 1.0L, 0, j), dg = jacobi_deriv(b, 2.0L * i + 1.0L, 0, j);
  ld sq2 = sqrtl(2.0L);
  ld omb_i = powl(1.0L - b, (ld)i);
  ld omb_im1 = i >= 1 ? powl(1.0L - b, (ld)(i - 1)) : 0.0L;
  if (val) *val = sq2 * f * g * omb_i;
  if (dr) *dr = 2.0L * sq2 * df * g * omb_im1;
  if (ds) *ds = sq2 * (df * g * (1.0L + a) * omb_im1 + f * dg * omb_i - i * f * g * omb_im1);
}

// ---- the reference element ------------------------------------------------------

bool build_reference(int N, RefOps &R) {
  if (N < 1 || N > GB_MAX_N) return false;
  const int Np = (N + 1) * (N + 2) / 2, Nfp = N + 1, NFN = 3 * Nfp;
  const int qc = (3 * N + 2) / 2;   // ceil((3N+1)/2): Stroud rule exact for degree 3N
  const int Nc = qc * qc;
  R.N = N; R.Np = Np; R.Nfp = Nfp; R.Nc = Nc;
  std::vector<ld> r, s;
  warp_blend(N, r, s);
  std::vector<Mode> md = modes(N);
  std::vector<ld> V((size_t)Np * Np), Vr((size_t)Np * Np), Vs((size_t)Np * Np);
  for (int k = 0; k < Np; ++k)
    for (int m = 0; m < Np; ++m)
      mode_eval(r[k], s[k], md[m].i, md[m].j, &V[(size_t)k * Np + m], &Vr[(size_t)k * Np + m], &Vs[(size_t)k * Np + m]);
  std::vector<ld> Vinv;
  if (!invert(V, Np, Vinv)) return false;
  std::vector<ld> Dr = matmul(Vr, Vinv, Np, Np, Np), Ds = matmul(Vs, Vinv, Np, Np, Np);
  std::vector<ld> Minv = matmul(V, transpose(V, Np, Np), Np, Np, Np);   // M^-1 = V V^T
  // face nodes, counter-clockwise along each face
  R.fmask.assign(NFN, 0);
  std::vector<int> rowstart(N + 1);
  for (int j = 0, acc = 0; j <= N; ++j) { rowstart[j] = acc; acc += N + 1 - j; }
  for (int k = 0; k <= N; ++k) {
    R.fmask[0 * Nfp + k] = k;                              // s = -1, left to right
    R.fmask[1 * Nfp + k] = rowstart[k] + (N - k);          // r + s = 0, bottom to top
    R.fmask[2 * Nfp + k] = rowstart[N - k];                // r = -1, top to bottom
  }
  // 1D face mass on the Gauss-Lobatto points: (V1 V1^T)^-1
  std::vector<ld> gll = gauss_lobatto(N), V1((size_t)Nfp * Nfp), M1;
  for (int k = 0; k < Nfp; ++k)
    for (int n = 0; n < Nfp; ++n) V1[(size_t)k * Nfp + n] = jacobi(gll[k], 0, 0, n);
  if (!invert(matmul(V1, transpose(V1, Nfp, Nfp), Nfp, Nfp, Nfp), Nfp, M1)) return false;
  std::vector<ld> E((size_t)Np * NFN, 0.0L);
  for (int f = 0; f < 3; ++f)
    for (int k = 0; k < Nfp; ++k)
      for (int l = 0; l < Nfp; ++l) E[(size_t)R.fmask[f * Nfp + k] * NFN + f * Nfp + l] = M1[(size_t)k * Nfp + l];
  std::vector<ld> LIFT = matmul(Minv, E, Np, Np, NFN);
  // Stroud conical-product cubature, b-major
  std::vector<ld> ga, wa, gb_, wb;
  gauss_jacobi(qc, 0.0L, 0.0L, ga, wa);
  gauss_jacobi(qc, 1.0L, 0.0L, gb_, wb);
  std::vector<ld> cr(Nc), cs(Nc), cw(Nc);
  for (int jb = 0; jb < qc; ++jb)
    for (int ia = 0; ia < qc; ++ia) {
      int k = jb * qc + ia;
      cr[k] = (1.0L + ga[ia]) * (1.0L - gb_[jb]) / 2.0L - 1.0L;
      cs[k] = gb_[jb];
      cw[k] = wa[ia] * wb[jb] / 2.0L;
    }
  std::vector<ld> Vc((size_t)Nc * Np);
  for (int k = 0; k < Nc; ++k)
    for (int m = 0; m < Np; ++m) mode_eval(cr[k], cs[k], md[m].i, md[m].j, &Vc[(size_t)k * Np + m], nullptr, nullptr);
  std::vector<ld> I = matmul(Vc, Vinv, Nc, Np, Np);
  std::vector<ld> ITW = transpose(I, Nc, Np);
  for (int i = 0; i < Np; ++i)
    for (int k = 0; k < Nc; ++k) ITW[(size_t)i * Nc + k] *= cw[k];
  std::vector<ld> P = matmul(Minv, ITW, Np, Np, Nc);
  // integral of each nodal basis function: 1^T Mhat, Mhat = (V V^T)^-1
  std::vector<ld> Mhat;
  if (!invert(Minv, Np, Mhat)) return false;
  std::vector<ld> wq(Np, 0.0L);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) wq[j] += Mhat[(size_t)i * Np + j];
  auto cp = [](const std::vector<ld> &a, std::vector<double> &b) {
    b.resize(a.size());
    for (size_t i = 0; i < a.size(); ++i) b[i] = (double)a[i];
  };
  cp(r, R.r); cp(s, R.s); cp(Dr, R.Dr); cp(Ds, R.Ds); cp(LIFT, R.LIFT);
  cp(I, R.I); cp(P, R.P); cp(cr, R.cr); cp(cs, R.cs); cp(cw, R.cw); cp(wq, R.wq);
  return true;
}


// ---- the reference tetrahedron (3D, 10 fields) -------------------------------------
//
// Reference tetrahedron v0 = (-1,-1,-1), v1 = (1,-1,-1), v2 = (-1,1,-1), v3 = (-1,-1,1);
// barycentric l0 = -(1+r+s+t)/2, l1 = (1+r)/2, l2 = (1+s)/2, l3 = (1+t)/2.  Faces
// (local vertex triples) 0 = (0,1,2), 1 = (0,1,3), 2 = (1,2,3), 3 = (0,2,3).  Node
// order: lattice (i, j, k) = N (l1, l2, l3) before warping, i fastest, k slowest.

static const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

static ld alpha_tet(int N) {
  static const ld tab[15] = {0.0L, 0.0L, 0.0L, 0.1002L, 1.1332L, 1.5608L, 1.3413L, 1.2577L,
                             1.1603L, 1.10153L, 0.6080L, 0.4523L, 0.8856L, 0.8717L, 0.9655L};
  return N <= 15 ? tab[N - 1] : 1.0L;
}

// Warp & Blend nodes on the tetrahedron (Warburton 2006): the equidistant nodes of the
// regular tetrahedron with edge 2 are moved by each face's warp (per face edge: the 1D
// warp along the edge direction, times 4 la lb (1 + (alpha lc)^2)), blended into the
// volume by lb lc ld (1 + (alpha la)^2) / ((lb + la/2)(lc + la/2)(ld + la/2)) with la the
// coordinate of the opposite vertex; edge nodes of a face take that face's warp.
// Output: barycentric coordinates lam[Np][4].
static void warp_blend_tet(int N, std::vector<std::array<ld, 4>> &lam) {
  const ld s3 = sqrtl(3.0L), s6 = sqrtl(6.0L);
  const ld V[4][3] = {{-1.0L, -1.0L / s3, -1.0L / s6}, {1.0L, -1.0L / s3, -1.0L / s6},
                      {0.0L, 2.0L / s3, -1.0L / s6}, {0.0L, 0.0L, 3.0L / s6}};
  const ld alpha = alpha_tet(N), tol = 1e-10L;
  std::vector<ld> gll = gauss_lobatto(N);
  lam.clear();
  for (int k = 0; k <= N; ++k)
    for (int j = 0; j <= N - k; ++j)
      for (int i = 0; i <= N - j - k; ++i) {
        ld L[4] = {1.0L - (ld)(i + j + k) / N, (ld)i / N, (ld)j / N, (ld)k / N};
        ld X[3] = {0, 0, 0}, sh[3] = {0, 0, 0};
        for (int v = 0; v < 4; ++v)
          for (int d = 0; d < 3; ++d) X[d] += L[v] * V[v][d];
        for (int f = 0; f < 4; ++f) {
          const int *fv = kFaceVerts[f];
          const int opp = 6 - fv[0] - fv[1] - fv[2];
          const ld La = L[opp];
          ld fw[3] = {0, 0, 0};
          for (int e = 0; e < 3; ++e) {
            const int a = fv[e], b = fv[(e + 1) % 3], c = fv[(e + 2) % 3];
            ld d[3], len = 0;
            for (int q = 0; q < 3; ++q) { d[q] = V[b][q] - V[a][q]; len += d[q] * d[q]; }
            len = sqrtl(len);
            const ld amt = 4.0L * L[a] * L[b] * warp_over_blend(N, L[b] - L[a], gll) * (1.0L + alpha * alpha * L[c] * L[c]);
            for (int q = 0; q < 3; ++q) fw[q] += amt * d[q] / len;
          }
          const ld Lb = L[fv[0]], Lc = L[fv[1]], Ld = L[fv[2]];
          ld blend = Lb * Lc * Ld;
          const ld den = (Lb + 0.5L * La) * (Lc + 0.5L * La) * (Ld + 0.5L * La);
          if (den > tol) blend = (1.0L + alpha * alpha * La * La) * blend / den;
          const int inside = (Lb > tol) + (Lc > tol) + (Ld > tol);
          if (La < tol && inside < 3) {
            for (int q = 0; q < 3; ++q) sh[q] = fw[q];
          } else {
            for (int q = 0; q < 3; ++q) sh[q] += blend * fw[q];
          }
        }
        for (int d = 0; d < 3; ++d) X[d] += sh[d];
        // barycentric coordinates of X in the regular tetrahedron: solve [V^T; 1] l = [X; 1]
        std::vector<ld> A(16), Ai;
        for (int v = 0; v < 4; ++v) {
          for (int d = 0; d < 3; ++d) A[(size_t)d * 4 + v] = V[v][d];
          A[12 + v] = 1.0L;
        }
        invert(A, 4, Ai);
        const ld rhs[4] = {X[0], X[1], X[2], 1.0L};
        std::array<ld, 4> l;
        for (int v = 0; v < 4; ++v) {
          l[v] = 0;
          for (int q = 0; q < 4; ++q) l[v] += Ai[(size_t)v * 4 + q] * rhs[q];
        }
        lam.push_back(l);
      }
}

// Homogeneous form of the orthonormal Jacobi polynomials: T_n(x, y) = y^n p_n(x / y),
// with its partial derivatives, from the three-term recurrence multiplied through by
// y^{n+1} (no division by y, so it is regular where the collapsed map is singular).
static void jacobi_homog(ld x, ld y, ld a, ld b, int n, ld *T, ld *Tx, ld *Ty) {
  ld t0 = 1.0L / sqrtl(jac_mass(a, b)), x0 = 0, y0 = 0;
  if (n == 0) { *T = t0; *Tx = 0; *Ty = 0; return; }
  const ld A1 = jac_A(1, a, b), B0 = jac_B(0, a, b);
  ld t1 = (x - B0 * y) * t0 / A1, x1 = t0 / A1, y1 = -B0 * t0 / A1;
  for (int k = 1; k < n; ++k) {
    const ld Ak = jac_A(k, a, b), Bk = jac_B(k, a, b), Ak1 = jac_A(k + 1, a, b);
    const ld t2 = ((x - Bk * y) * t1 - Ak * y * y * t0) / Ak1;
    const ld x2 = (t1 + (x - Bk * y) * x1 - Ak * y * y * x0) / Ak1;
    const ld y2 = (-Bk * t1 + (x - Bk * y) * y1 - 2.0L * Ak * y * t0 - Ak * y * y * y0) / Ak1;
    t0 = t1; x0 = x1; y0 = y1;
    t1 = t2; x1 = x2; y1 = y2;
  }
  *T = t1; *Tx = x1; *Ty = y1;
}

// Orthonormal tetrahedral mode psi_ijk = 2 sqrt2 p_i(a) p_j^{(2i+1,0)}(b) (1-b)^i
// p_k^{(2i+2j+2,0)}(c) (1-c)^{i+j} (collapsed a, b, c), written as
// 2 sqrt2 2^i T_i(2(1+r) - S, S) T_j(2(1+s) - (1-t), 1-t) p_k(t) with S = -s-t, so that
// value and gradient are polynomial evaluations everywhere on the element.
static void mode3_eval(ld r, ld s, ld t, int i, int j, int k, ld *val, ld *g) {
  const ld S = -s - t, w = 1.0L - t;
  ld A, Ax, Ay, B, Bx, By;
  jacobi_homog(2.0L * (1.0L + r) - S, S, 0, 0, i, &A, &Ax, &Ay);
  jacobi_homog(2.0L * (1.0L + s) - w, w, 2.0L * i + 1.0L, 0, j, &B, &Bx, &By);
  const ld ac = 2.0L * i + 2.0L * j + 2.0L;
  const ld C = jacobi(t, ac, 0, k), Ct = jacobi_deriv(t, ac, 0, k);
  const ld f = 2.0L * sqrtl(2.0L) * powl(2.0L, (ld)i);
  // dA/dr = 2 Ax; dA/ds = dA/dt = Ax - Ay (x = 2(1+r) + s + t, y = -s - t)
  // dB/ds = 2 Bx; dB/dt = Bx - By (x = 2(1+s) - 1 + t, y = 1 - t)
  if (val) *val = f * A * B * C;
  if (g) {
    g[0] = f * 2.0L * Ax * B * C;
    g[1] = f * ((Ax - Ay) * B * C + A * 2.0L * Bx * C);
    g[2] = f * ((Ax - Ay) * B * C + A * (Bx - By) * C + A * B * Ct);
  }
}

bool build_reference3d(int N, RefOps3 &R) {
  if (N < 1 || N > GB3_MAX_N) return false;
  const int Np = (N + 1) * (N + 2) * (N + 3) / 6, Nfp = (N + 1) * (N + 2) / 2, NFN = 4 * Nfp;
  const int qc = (3 * N + 2) / 2;   // ceil((3N+1)/2): conical rule exact for degree 3N
  const int Nc = qc * qc * qc;
  R.N = N; R.Np = Np; R.Nfp = Nfp; R.Nc = Nc;
  std::vector<std::array<ld, 4>> lam;
  warp_blend_tet(N, lam);
  std::vector<ld> r(Np), s(Np), t(Np);
  for (int n = 0; n < Np; ++n) {
    r[n] = 2.0L * lam[n][1] - 1.0L;
    s[n] = 2.0L * lam[n][2] - 1.0L;
    t[n] = 2.0L * lam[n][3] - 1.0L;
  }
  struct M3 { int i, j, k; };
  std::vector<M3> md;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k) md.push_back({i, j, k});
  std::vector<ld> V((size_t)Np * Np), Vd[3];
  for (auto &v : Vd) v.resize((size_t)Np * Np);
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m) {
      ld g[3];
      mode3_eval(r[n], s[n], t[n], md[m].i, md[m].j, md[m].k, &V[(size_t)n * Np + m], g);
      for (int d = 0; d < 3; ++d) Vd[d][(size_t)n * Np + m] = g[d];
    }
  std::vector<ld> Vinv;
  if (!invert(V, Np, Vinv)) return false;
  std::vector<ld> D[3];
  for (int d = 0; d < 3; ++d) D[d] = matmul(Vd[d], Vinv, Np, Np, Np);
  std::vector<ld> Minv = matmul(V, transpose(V, Np, Np), Np, Np, Np);
  // face nodes: nodes with zero coordinate of the opposite vertex, increasing index
  R.fmask.assign(NFN, 0);
  for (int f = 0; f < 4; ++f) {
    const int opp = 6 - kFaceVerts[f][0] - kFaceVerts[f][1] - kFaceVerts[f][2];
    int c = 0;
    for (int n = 0; n < Np; ++n)
      if (fabsl(lam[n][opp]) < 1e-10L) {
        if (c >= Nfp) return false;
        R.fmask[f * Nfp + c++] = n;
      }
    if (c != Nfp) return false;
  }
  // face mass in the parameter measure of each face (its own reference triangle):
  // (V2 V2^T)^-1 with the orthonormal triangle modes at the face nodes
  std::vector<Mode> md2 = modes(N);
  std::vector<ld> E((size_t)Np * NFN, 0.0L);
  for (int f = 0; f < 4; ++f) {
    std::vector<ld> V2((size_t)Nfp * Nfp), M2;
    for (int k = 0; k < Nfp; ++k) {
      const int n = R.fmask[f * Nfp + k];
      const ld r2 = 2.0L * lam[n][kFaceVerts[f][1]] - 1.0L, s2 = 2.0L * lam[n][kFaceVerts[f][2]] - 1.0L;
      for (int m = 0; m < Nfp; ++m) mode_eval(r2, s2, md2[m].i, md2[m].j, &V2[(size_t)k * Nfp + m], nullptr, nullptr);
    }
    if (!invert(matmul(V2, transpose(V2, Nfp, Nfp), Nfp, Nfp, Nfp), Nfp, M2)) return false;
    for (int k = 0; k < Nfp; ++k)
      for (int l = 0; l < Nfp; ++l) E[(size_t)R.fmask[f * Nfp + k] * NFN + f * Nfp + l] = M2[(size_t)k * Nfp + l];
  }
  std::vector<ld> LIFT = matmul(Minv, E, Np, Np, NFN);
  // conical-product cubature: Gauss-Legendre (a) x Gauss-Jacobi(1,0) (b) x Gauss-Jacobi(2,0) (c)
  std::vector<ld> ga, wa, gbv, wbv, gc, wc;
  gauss_jacobi(qc, 0.0L, 0.0L, ga, wa);
  gauss_jacobi(qc, 1.0L, 0.0L, gbv, wbv);
  gauss_jacobi(qc, 2.0L, 0.0L, gc, wc);
  std::vector<ld> cr(Nc), cs(Nc), ct(Nc), cw(Nc);
  for (int kc = 0; kc < qc; ++kc)
    for (int jb = 0; jb < qc; ++jb)
      for (int ia = 0; ia < qc; ++ia) {
        const int q = (kc * qc + jb) * qc + ia;
        ct[q] = gc[kc];
        cs[q] = (1.0L + gbv[jb]) * (1.0L - gc[kc]) / 2.0L - 1.0L;
        cr[q] = (1.0L + ga[ia]) * (1.0L - gbv[jb]) * (1.0L - gc[kc]) / 4.0L - 1.0L;
        cw[q] = wa[ia] * wbv[jb] * wc[kc] / 8.0L;
      }
  std::vector<ld> Vc((size_t)Nc * Np);
  for (int q = 0; q < Nc; ++q)
    for (int m = 0; m < Np; ++m) mode3_eval(cr[q], cs[q], ct[q], md[m].i, md[m].j, md[m].k, &Vc[(size_t)q * Np + m], nullptr);
  std::vector<ld> I = matmul(Vc, Vinv, Nc, Np, Np);
  std::vector<ld> ITW = transpose(I, Nc, Np);
  for (int i = 0; i < Np; ++i)
    for (int q = 0; q < Nc; ++q) ITW[(size_t)i * Nc + q] *= cw[q];
  std::vector<ld> P = matmul(Minv, ITW, Np, Np, Nc);
  std::vector<ld> Mhat;
  if (!invert(Minv, Np, Mhat)) return false;
  std::vector<ld> wq(Np, 0.0L);
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) wq[j] += Mhat[(size_t)i * Np + j];
  // neighbour face-node table: my face f (vertex ids in kFaceVerts order), neighbour face
  // f2, permutation code p (my face vertex i is the neighbour's face vertex kPerm3[p][i]):
  // the neighbour's volume node holding the same point as my face node k
  R.nbr_node.assign((size_t)4 * 4 * 6 * Nfp, -1);
  for (int f = 0; f < 4; ++f)
    for (int f2 = 0; f2 < 4; ++f2)
      for (int p = 0; p < 6; ++p)
        for (int k = 0; k < Nfp; ++k) {
          const int n = R.fmask[f * Nfp + k];
          ld nu[3];
          for (int i = 0; i < 3; ++i) nu[kPerm3[p][i]] = lam[n][kFaceVerts[f][i]];
          int best = -1;
          ld bd = 1e30L;
          for (int k2 = 0; k2 < Nfp; ++k2) {
            const int n2 = R.fmask[f2 * Nfp + k2];
            ld d = 0;
            for (int i = 0; i < 3; ++i) d += fabsl(lam[n2][kFaceVerts[f2][i]] - nu[i]);
            if (d < bd) { bd = d; best = n2; }
          }
          if (bd > 1e-10L) return false;
          R.nbr_node[((size_t)(f * 4 + f2) * 6 + p) * Nfp + k] = best;
        }
  auto cp = [](const std::vector<ld> &a, std::vector<double> &b) {
    b.resize(a.size());
    for (size_t i = 0; i < a.size(); ++i) b[i] = (double)a[i];
  };
  cp(r, R.r); cp(s, R.s); cp(t, R.t); cp(D[0], R.Dr); cp(D[1], R.Ds); cp(D[2], R.Dt); cp(LIFT, R.LIFT);
  cp(I, R.I); cp(P, R.P); cp(cr, R.cr); cp(cs, R.cs); cp(ct, R.ct); cp(cw, R.cw); cp(wq, R.wq);
  R.bary.resize((size_t)Np * 4);
  for (int n = 0; n < Np; ++n)
    for (int v = 0; v < 4; ++v) R.bary[(size_t)n * 4 + v] = (double)lam[n][v];
  return true;
}

// ---- SARK coefficients (Sec. 4) through phi-functions ---------------------------

// phi_k(z) = sum_m z^m / (m+k)!; series for |z| < 1, closed forms otherwise.
static ld phi(int k, ld z) {
  if (fabsl(z) < 1.0L) {
    ld term = 1.0L, sum = 0.0L;
    for (int i = 1; i <= k; ++i) term /= i;          // 1/k!
    for (int m = 0; m < 40; ++m) {
      sum += term;
      term *= z / (m + k + 1);
    }
    return sum;
  }
  ld e = expl(z);
  switch (k) {
    case 0: return e;
    case 1: return expm1l(z) / z;
    case 2: return (expm1l(z) - z) / (z * z);
    default: return (expm1l(z) - z - 0.5L * z * z) / (z * z * z);
  }
}

void sark_coefficients(double gamma, double E[5], double A[16], double B[4]) {
  ld g = gamma, h = 0.5L * g;
  ld p1h = phi(1, h), p2h = phi(2, h);
  ld p1 = phi(1, g), p2 = phi(2, g), p3 = phi(3, g);
  for (int i = 0; i < 16; ++i) A[i] = 0.0;
  A[1 * 4 + 0] = (double)(0.5L * p1h);
  A[2 * 4 + 0] = (double)(0.5L * p1h - p2h);
  A[2 * 4 + 1] = (double)p2h;
  A[3 * 4 + 0] = (double)(p1 - 2.0L * p2);
  A[3 * 4 + 1] = 0.0;
  A[3 * 4 + 2] = (double)(2.0L * p2);
  B[0] = (double)(p1 - 3.0L * p2 + 4.0L * p3);
  B[1] = B[2] = (double)(2.0L * p2 - 4.0L * p3);
  B[3] = (double)(4.0L * p3 - p2);
  E[0] = 1.0;
  E[1] = E[2] = (double)expl(h);
  E[3] = E[4] = (double)expl(g);
}

}  // namespace gb
