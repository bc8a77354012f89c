// force.cu -- the fermion force of S = phi^dag A^{-1} phi, A = 4 m^2 - D_eo D_oe.
//
// With X = A^{-1} phi on the even sites and Y = D_oe X on the odd sites, the
// variation of S is dS = X^dag dD_eo Y - Y^dag dD_oe X.  For the link
// U = U_mu(x) with s = eta_mu(x) b_mu(x) this gives dS = Re Tr(K dU) with
//   K = 2 s Y(x+mu) X(x)^dag   (x even),   K = -2 s X(x+mu) Y(x)^dag   (x odd),
// the two terms of the general form s [Psi2(x+mu) Psi1(x)^dag - Psi1(x+mu)
// Psi2(x)^dag] (Psi1 = (X, -Y), Psi2 = (X, Y)) coinciding.  The kernel writes
// the gradient in the torch convention dS/dRe U + i dS/dIm U = K^dag, and
// optionally the Lie-algebra force f_a = Re Tr(i T_a U K), T_a = lambda_a / 2
// (derivative of S along U -> exp(i w T_a) U).  FP64 throughout.
#include "launch.h"

namespace stag {

// one thread per link (mu, lexicographic site); X, Y in the device SoA layout
__global__ void k_force(const Geom g, const double2 *__restrict__ X, const double2 *__restrict__ Y,
                        const void *links64, double2 *__restrict__ grad, double *__restrict__ lie) {
  const long long V = 2ll * g.Ve;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * V) return;
  const int mu = (int)(i / V);
  const long long lex = i % V;
  int x[4];
  {
    long long r = lex;
    x[0] = (int)(r % g.L0);
    r /= g.L0;
    x[1] = (int)(r % g.L1);
    r /= g.L1;
    x[2] = (int)(r % g.L2);
    x[3] = (int)(r / g.L2);
  }
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const int s = (int)(lex >> 1);
  const int Ls[4] = {g.L0, g.L1, g.L2, g.L3};
  int xf[4] = {x[0], x[1], x[2], x[3]};
  xf[mu] = (x[mu] + 1 == Ls[mu]) ? 0 : x[mu] + 1;
  const int sf = cb_of(g, xf[0], xf[1], xf[2], xf[3]);
  int eb = 0;
  for (int nu = 0; nu < mu; ++nu) eb += x[nu];
  double sg = (eb & 1) ? -1.0 : 1.0;
  if (mu == 3 && g.ap && x[3] == g.L3 - 1) sg = -sg;
  // K = c a b^dag with (a, b) = (Y(x+mu), X(x)), c = 2s on even x;
  //                      (X(x+mu), Y(x)), c = -2s on odd x
  const double2 *A = par == 0 ? Y : X;
  const double2 *B = par == 0 ? X : Y;
  const int sa = sf, sbb = s;
  const double c = par == 0 ? 2.0 * sg : -2.0 * sg;
  double2 av[3], bv[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    av[k] = A[(long long)k * g.Ve + sa];
    bv[k] = B[(long long)k * g.Ve + sbb];
  }
  // K_ab = c a_a conj(b_b)
  double2 K[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      K[3 * a + b] = make_double2(c * (av[a].x * bv[b].x + av[a].y * bv[b].y),
                                  c * (av[a].y * bv[b].x - av[a].x * bv[b].y));
  if (grad) {
    double2 *G = grad + i * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) G[3 * a + b] = make_double2(K[3 * b + a].x, -K[3 * b + a].y);  // K^dag
  }
  if (lie) {
    double u[18];
    load_link<P64, 0>(links64, g.Ve, par, mu, s, u);
    double2 M[9];  // M = U K
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double ur = u[2 * (3 * a + k)], ui = u[2 * (3 * a + k) + 1];
          re += ur * K[3 * k + b].x - ui * K[3 * k + b].y;
          im += ur * K[3 * k + b].y + ui * K[3 * k + b].x;
        }
        M[3 * a + b] = make_double2(re, im);
      }
    // f_a = Re Tr(i lambda_a M) / 2 = -Im Tr(lambda_a M) / 2
    const double r3 = 0.57735026918962576451;  // 1/sqrt(3)
    double *f = lie + i * 8;
    f[0] = -0.5 * (M[3].y + M[1].y);                        // lambda_1
    f[1] = -0.5 * (-M[3].x + M[1].x);                       // lambda_2: Im(-i M10 + i M01)
    f[2] = -0.5 * (M[0].y - M[4].y);                        // lambda_3
    f[3] = -0.5 * (M[6].y + M[2].y);                        // lambda_4
    f[4] = -0.5 * (-M[6].x + M[2].x);                       // lambda_5
    f[5] = -0.5 * (M[7].y + M[5].y);                        // lambda_6
    f[6] = -0.5 * (-M[7].x + M[5].x);                       // lambda_7
    f[7] = -0.5 * r3 * (M[0].y + M[4].y - 2.0 * M[8].y);    // lambda_8
  }
}

cudaError_t launch_force(Geom g, const double2 *X, const double2 *Y, const void *links64, double2 *grad,
                         double *lie, cudaStream_t st) {
  const long long n = 8ll * g.Ve;
  k_force<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, X, Y, links64, grad, lie);
  return cudaGetLastError();
}

}  // namespace stag
