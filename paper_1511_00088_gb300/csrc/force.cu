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
                        const void *links64, double2 *__restrict__ grad, double *__restrict__ lie,
                        double scale) {
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
  const double c = (par == 0 ? 2.0 * sg : -2.0 * sg) * scale;  // scale: the caller's chain-rule factor
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
                         double *lie, double scale, cudaStream_t st) {
  const long long n = 8ll * g.Ve;
  k_force<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, X, Y, links64, grad, lie, scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// the action S = phi^dag A^{-1} phi at an approximate solution x of A x = phi,
// in the stationary form S = 2 Re<phi, x> - Re<x, A x> (its error is second
// order in the residual phi - A x), summed in double-word arithmetic
// ---------------------------------------------------------------------------
// (hi, lo) += (bh, bl): Knuth's two-sum of the high parts (exact error term),
// the low parts and that error added, then renormalised (fast two-sum).
// Additions only, so no contraction into FMAs can change it.
__device__ __forceinline__ void dw_add(double &hi, double &lo, double bh, double bl) {
  const double s = hi + bh;
  const double bb = s - hi;
  const double e = (hi - (s - bb)) + (bh - bb);
  const double t = (lo + bl) + e;
  hi = s + t;
  lo = t - (hi - s);
}

__device__ __forceinline__ void dw_warp(double &hi, double &lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double h = __shfl_xor_sync(0xffffffffu, hi, o), l = __shfl_xor_sync(0xffffffffu, lo, o);
    dw_add(hi, lo, h, l);
  }
}

// fixed-order (hi, lo) sum over the block's threads -> thread 0
template <int BT>
__device__ __forceinline__ void dw_block(double &hi, double &lo) {
  __shared__ double sh[BT / 32], sl[BT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  dw_warp(hi, lo);
  if (lane == 0) {
    sh[warp] = hi;
    sl[warp] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < BT / 32; ++w) dw_add(hi, lo, sh[w], sl[w]);
  }
}

constexpr int ACT_BT = 256;

// per block: the double-word sum over its sites of 2 Re(phi . x) - Re(x . Ax)
// (device SoA layout, one system) -> part[2 block], part[2 block + 1]
__global__ void __launch_bounds__(ACT_BT) k_action_part(VecArg phi, VecArg x, VecArg ax, int Ve, double *part) {
  const int s = blockIdx.x * ACT_BT + threadIdx.x;
  double hi = 0.0, lo = 0.0;
  if (s < Ve) {
    double f[6], xv[6], av[6];
    load_vec<P64>(phi, 0, s, Ve, f);
    load_vec<P64>(x, 0, s, Ve, xv);
    load_vec<P64>(ax, 0, s, Ve, av);
    double d = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) d += 2.0 * f[i] * xv[i] - xv[i] * av[i];
    hi = d;
  }
  dw_block<ACT_BT>(hi, lo);
  if (threadIdx.x == 0) {
    part[2ll * blockIdx.x] = hi;
    part[2ll * blockIdx.x + 1] = lo;
  }
}

// one block: the nb block sums in a fixed order -> *out = hi + lo
__global__ void __launch_bounds__(ACT_BT) k_action_sum(const double *part, int nb, double *out) {
  double hi = 0.0, lo = 0.0;
  for (int i = threadIdx.x; i < nb; i += ACT_BT) dw_add(hi, lo, part[2ll * i], part[2ll * i + 1]);
  dw_block<ACT_BT>(hi, lo);
  if (threadIdx.x == 0) *out = hi + lo;
}

// out = a x over n doubles (the source gradient 2 gS X of the action)
__global__ void k_scale_reals(const double *__restrict__ x, double a, double *__restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i];
}

int action_blocks(int Ve) { return (Ve + ACT_BT - 1) / ACT_BT; }

cudaError_t launch_action(VecArg phi, VecArg x, VecArg ax, int Ve, double *part, double *out, cudaStream_t st) {
  const int nb = action_blocks(Ve);
  k_action_part<<<nb, ACT_BT, 0, st>>>(phi, x, ax, Ve, part);
  k_action_sum<<<1, ACT_BT, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_scale_reals(const double *x, double a, double *out, long long n, cudaStream_t st) {
  k_scale_reals<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, a, out, n);
  return cudaGetLastError();
}

}  // namespace stag
