// npr.cu -- the one-colour-trace four-fermion contraction of the NPR workload
// (Sec. 4 of the paper, Eq. (ffop); FP64, its 97 % kernel):
//   O(z) = sum_{A,B,C,D} [chibar1(z_A) (g_S1 x x_F1)_AB chi2(z_B)]
//                        [chibar3(z_C) (g_S2 x x_F2)_CD chi4(z_D)]
//                        [U_AD(z)]_{c1 c4} [U_CB(z)]_{c3 c2}
// on every hypercube z (sites z_A = 2z + A, corners A in {0,1}^4), with
//   (g_S x x_F)_AB = (1/4) Tr(g_A^dag g_S g_B g_F^dag),  g_A = g_1^A1 ... g_4^A4,
//   U_AD(z) = the average over the shortest paths from z_A to z_D inside the
//   hypercube of the link products (U_mu for +mu, U_mu^dag for -mu).
// One block per hypercube, 256 threads:
//   * the path averages W(A, D) in shared memory, both orientations (W(D, A) =
//     W(A, D)^dag, so that no read conjugates), W(A, A) = 1: level n = 1 is
//     the hypercube's 32 internal links; levels n = |A xor D| = 2, 3, 4 (a
//     table of the pairs A < D per level), one thread per matrix element: a
//     path's last step is one of the differing directions mu, so
//     W(A, D) = (1/n) sum_mu W(A, D xor mu) W(D xor mu, D);
//   * the spin-taste entries from the Clifford algebra: g_X g_Y = e(X, Y)
//     g_{X xor Y} with e(X, Y) = (-1)^(sum_{mu > nu} X_mu Y_nu), g_A^dag =
//     (-1)^(n(n-1)/2) g_A (n set bits), so (g_S x x_F)_AB is nonzero only for
//     A xor S xor B xor F = 0, where it is the product of those signs;
//   * thread (A, C) evaluates its term (B = A xor S1 xor F1, D = C xor S2 xor
//     F2), the block sums the 256 terms in a fixed order.
#include <cuda_runtime.h>

#include "launch.h"

namespace stag {

namespace {

constexpr int NPR_BT = 256;

__device__ __forceinline__ double2 zm(double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); }
__device__ __forceinline__ double2 za(double2 x, double2 y) { return make_double2(x.x + y.x, x.y + y.y); }
// s + x y as two FMA chains per component (4 FP64 instructions for 8 flops)
__device__ __forceinline__ double2 zfma(double2 x, double2 y, double2 s) {
  return make_double2(__fma_rn(-x.y, y.y, __fma_rn(x.x, y.x, s.x)), __fma_rn(x.y, y.x, __fma_rn(x.x, y.y, s.y)));
}

// reversal sign of g_A^dag = (-1)^(n(n-1)/2) g_A
__device__ __forceinline__ int rev_sign(int A) {
  const int n = __popc(A);
  return ((n * (n - 1) / 2) & 1) ? -1 : 1;
}
// e(X, Y): g_X g_Y = e g_{X xor Y}
__device__ __forceinline__ int mul_sign(int X, int Y) {
  int cnt = 0;
#pragma unroll
  for (int nu = 0; nu < 4; ++nu)
    if ((Y >> nu) & 1) cnt += __popc(X >> (nu + 1));
  return (cnt & 1) ? -1 : 1;
}
// (g_S x x_F)_AB (real: 0 or +-1)
__device__ __forceinline__ double spin_taste(int S, int F, int A, int B) {
  if ((A ^ S ^ B ^ F) != 0) return 0.0;
  const int s = rev_sign(A) * rev_sign(F) * mul_sign(A, S) * mul_sign(A ^ S, B) * mul_sign(A ^ S ^ B, F);
  return (double)s;
}

// the 120 corner pairs A < D of a hypercube, ordered by n = |A xor D|
// (32, 48, 32, 8 pairs), and the offset of each level
struct PairTable {
  unsigned char a[120], d[120];
  int off[5];
};
constexpr int popc4(int x) { return (x & 1) + ((x >> 1) & 1) + ((x >> 2) & 1) + ((x >> 3) & 1); }
constexpr PairTable make_pairs() {
  PairTable p{};
  int k = 0;
  for (int n = 1; n <= 4; ++n) {
    p.off[n - 1] = k;
    for (int A = 0; A < 16; ++A)
      for (int D = A + 1; D < 16; ++D)
        if (popc4(A ^ D) == n) {
          p.a[k] = (unsigned char)A;
          p.d[k] = (unsigned char)D;
          ++k;
        }
  }
  p.off[4] = k;
  return p;
}
__constant__ PairTable c_pairs = make_pairs();

struct NprArgs {
  int L[4], H[4];
  long long V;
  const double2 *U;  // [4][V][9]
  const double2 *cb1, *c2, *cb3, *c4;  // [V][3]
  int S1, F1, S2, F2;
  double2 *out;      // [nhyp]
};

__global__ void __launch_bounds__(NPR_BT) k_npr(const NprArgs a) {
  __shared__ double2 W[256][9];      // W(A, D), index A * 16 + D, both orientations
  __shared__ double2 fld[4][16][3];  // chibar1, chi2, chibar3, chi4 at the corners
  __shared__ double2 red[NPR_BT / 32];
  __shared__ unsigned char pa[120], pd[120];
  const long long h = blockIdx.x;
  int zc[4];
  {
    long long r = h;
    zc[0] = (int)(r % a.H[0]);
    r /= a.H[0];
    zc[1] = (int)(r % a.H[1]);
    r /= a.H[1];
    zc[2] = (int)(r % a.H[2]);
    zc[3] = (int)(r / a.H[2]);
  }
  auto site = [&](int A) -> long long {
    const int x0 = 2 * zc[0] + (A & 1), x1 = 2 * zc[1] + ((A >> 1) & 1), x2 = 2 * zc[2] + ((A >> 2) & 1),
              x3 = 2 * zc[3] + ((A >> 3) & 1);
    return x0 + (long long)a.L[0] * (x1 + (long long)a.L[1] * (x2 + (long long)a.L[2] * x3));
  };
  const int t = threadIdx.x;
  // level n = 1, the hypercube's 32 internal links: W(A, D) = U_mu(z_A) for
  // D = A + mu (A_mu = 0), W(D, A) its adjoint; level 0: W(A, A) = 1
  for (int k = t; k < 32 * 9; k += NPR_BT) {
    const int l = k / 9, e = k % 9, mu = l / 8, y = l % 8;
    const int A = ((y >> mu) << (mu + 1)) | (y & ((1 << mu) - 1)), D = A | (1 << mu);
    const double2 u = a.U[((long long)mu * a.V + site(A)) * 9 + e];
    W[A * 16 + D][e] = u;
    W[D * 16 + A][(e % 3) * 3 + e / 3] = make_double2(u.x, -u.y);
  }
  for (int k = t; k < 4 * 16 * 3; k += NPR_BT) {
    const int f = k / 48, A = (k / 3) % 16, c = k % 3;
    const double2 *src = f == 0 ? a.cb1 : f == 1 ? a.c2 : f == 2 ? a.cb3 : a.c4;
    fld[f][A][c] = src[site(A) * 3 + c];
  }
  for (int k = t; k < 16 * 9; k += NPR_BT) {
    const int Y = k / 9, e = k % 9;
    W[Y * 17][e] = make_double2((e % 4 == 0) ? 1.0 : 0.0, 0.0);
  }
  if (t < 120) {
    pa[t] = c_pairs.a[t];
    pd[t] = c_pairs.d[t];
  }
  __syncthreads();
  // levels n = 2, 3, 4, the pairs A < D from the table: the last step of a
  // path is one of the differing directions mu, from P = D xor mu, so
  // W(A, D) = (1/n) sum_mu W(A, P) W(P, D) (W(P, D): a link or its adjoint);
  // one thread per matrix element, which also writes the adjoint entry
  for (int n = 2; n <= 4; ++n) {
    const int p0 = c_pairs.off[n - 1], nitem = (c_pairs.off[n] - p0) * 9;
    for (int item = t; item < nitem; item += NPR_BT) {
      const int pr = p0 + item / 9, e = item % 9;
      const int A = pa[pr], D = pd[pr];
      const int i = e / 3, j = e % 3;
      double2 s = make_double2(0.0, 0.0);
      for (int mu = 0; mu < 4; ++mu) {
        if (!(((A ^ D) >> mu) & 1)) continue;
        const int P = D ^ (1 << mu);
        const double2 *wa = W[A * 16 + P], *wb = W[P * 16 + D];
#pragma unroll
        for (int k = 0; k < 3; ++k) s = zfma(wa[i * 3 + k], wb[k * 3 + j], s);
      }
      const double inv = n == 2 ? 0.5 : n == 3 ? 1.0 / 3.0 : 0.25;  // constants: no FP64 division
      s = make_double2(s.x * inv, s.y * inv);
      W[A * 16 + D][e] = s;
      W[D * 16 + A][j * 3 + i] = make_double2(s.x, -s.y);
    }
    __syncthreads();
  }
  // thread (A, C): its term
  const int A = t >> 4, C = t & 15;
  const int B = A ^ a.S1 ^ a.F1, Dd = C ^ a.S2 ^ a.F2;
  const double s = spin_taste(a.S1, a.F1, A, B) * spin_taste(a.S2, a.F2, C, Dd);
  double2 t1 = make_double2(0.0, 0.0), t2 = make_double2(0.0, 0.0);
  {
    auto wget = [&](int X, int Y, int i, int j) -> double2 { return W[X * 16 + Y][i * 3 + j]; };
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double2 v1 = make_double2(0.0, 0.0), v2 = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v1 = zfma(wget(A, Dd, i, j), fld[3][Dd][j], v1);
        v2 = zfma(wget(C, B, i, j), fld[1][B][j], v2);
      }
      t1 = zfma(fld[0][A][i], v1, t1);
      t2 = zfma(fld[2][C][i], v2, t2);
    }
  }
  double2 term = zm(t1, t2);
  term.x *= s;
  term.y *= s;
  // fixed-order block sum
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    term.x += __shfl_xor_sync(0xffffffffu, term.x, o);
    term.y += __shfl_xor_sync(0xffffffffu, term.y, o);
  }
  if ((t & 31) == 0) red[t >> 5] = term;
  __syncthreads();
  if (t == 0) {
    double2 o = make_double2(0.0, 0.0);
    for (int w = 0; w < NPR_BT / 32; ++w) o = za(o, red[w]);
    a.out[h] = o;
  }
}

// out[0] = sum of the n values of in, fixed order (one block)
__global__ void __launch_bounds__(NPR_BT) k_npr_sum(const double2 *in, long long n, double2 *out) {
  __shared__ double2 red[NPR_BT / 32];
  double2 s = make_double2(0.0, 0.0);
  for (long long i = threadIdx.x; i < n; i += NPR_BT) s = za(s, in[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 o = make_double2(0.0, 0.0);
    for (int w = 0; w < NPR_BT / 32; ++w) o = za(o, red[w]);
    *out = o;
  }
}

}  // namespace

cudaError_t launch_npr(const int dims[4], const double2 *U, const int st[4], const double2 *cb1, const double2 *c2,
                       const double2 *cb3, const double2 *c4, double2 *out, double2 *sum, cudaStream_t s) {
  NprArgs a;
  long long nh = 1;
  for (int k = 0; k < 4; ++k) {
    a.L[k] = dims[k];
    a.H[k] = dims[k] / 2;
    nh *= a.H[k];
  }
  a.V = 16 * nh;
  a.U = U;
  a.cb1 = cb1;
  a.c2 = c2;
  a.cb3 = cb3;
  a.c4 = c4;
  a.S1 = st[0];
  a.F1 = st[1];
  a.S2 = st[2];
  a.F2 = st[3];
  a.out = out;
  k_npr<<<(unsigned)nh, NPR_BT, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !sum) return e;
  k_npr_sum<<<1, NPR_BT, 0, s>>>(out, nh, sum);
  return cudaGetLastError();
}

}  // namespace stag
