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
