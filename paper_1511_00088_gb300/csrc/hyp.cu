// hyp.cu -- HYP smearing of the gauge field on the GPU (FP64): the one-link
// field of the "HYP-smeared staggered quarks" whose CG Sec. 3 benchmarks.
//
// Three levels of decorated links, each a projection to SU(3) of the thin link
// plus a weighted staple sum over the level below, staples kept inside the
// hypercubes of the link (parameters (a1, a2, a3), Hasenfratz-Knechtli's
// (0.75, 0.6, 0.3) by default):
//   Vb(x,mu;e)  = P[(1-a3) U_mu(x) + a3/2 sum_{+-e} U_e U_mu U_e^dag]              (e != mu)
//   Vt(x,mu;nu) = P[(1-a2) U_mu(x) + a2/4 sum_{+-r, r != mu,nu} Vb(r;s) Vb(mu;s) Vb(r;s)^dag]
//                 (s = the direction outside {mu, nu, r})
//   V(x,mu)     = P[(1-a1) U_mu(x) + a1/6 sum_{+-nu != mu} Vt(nu;mu) Vt(mu;nu) Vt(nu;mu)^dag]
// A positive staple in direction d at x is W_d(x) W_mu(x+d) W_d(x+mu)^dag,
// a negative one W_d(x-d)^dag W_mu(x-d) W_d(x-d+mu).
// P(X) = the unitary polar factor of X with the phase of its determinant
// removed by the principal cube root.  Here the polar factor comes from
// Newton's iteration with determinant scaling (Y <- (g Y + (g Y)^-dag) / 2,
// g = |det Y|^(-1/3); Higham, "Computing the polar decomposition", 1986),
// which reaches the same unique factor in fewer steps than the plain one, and
// the determinant's phase from Newton's iteration for a complex cube root.
// One thread per (decorated link, site); links in the ABI layout
// [direction][site][3][3] complex (decorated: [12 (mu, decoration) slots][site][3][3]).
#include <cuda_runtime.h>

#include "launch.h"

namespace stag {

namespace {

struct M3 {
  double2 a[9];
};

__device__ __forceinline__ double2 cm(double2 x, double2 y) { return make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x); }
__device__ __forceinline__ double2 ccj(double2 x) { return make_double2(x.x, -x.y); }
// s + x y as two FMA chains per component (4 FP64 instructions for 8 flops)
__device__ __forceinline__ double2 cfma(double2 x, double2 y, double2 s) {
  return make_double2(__fma_rn(-x.y, y.y, __fma_rn(x.x, y.x, s.x)), __fma_rn(x.y, y.x, __fma_rn(x.x, y.y, s.y)));
}

// a b - c e as FMA chains (4 FP64 instructions per component)
__device__ __forceinline__ double2 cdet2(double2 a, double2 b, double2 c, double2 e) {
  return make_double2(__fma_rn(a.x, b.x, __fma_rn(-a.y, b.y, __fma_rn(-c.x, e.x, c.y * e.y))),
                      __fma_rn(a.x, b.y, __fma_rn(a.y, b.x, __fma_rn(-c.x, e.y, (-c.y) * e.x))));
}

__device__ __forceinline__ M3 ld(const double2 *p) {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.a[k] = p[k];
  return m;
}

// c += a b, with either factor optionally daggered
template <bool DA, bool DB>
__device__ __forceinline__ void mul_add(const M3 &a, const M3 &b, M3 &c) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = c.a[i * 3 + j];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = DA ? ccj(a.a[k * 3 + i]) : a.a[i * 3 + k];
        const double2 y = DB ? ccj(b.a[j * 3 + k]) : b.a[k * 3 + j];
        s = cfma(x, y, s);
      }
      c.a[i * 3 + j] = s;
    }
}

template <bool DA, bool DB>
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int k = 0; k < 9; ++k) c.a[k] = make_double2(0.0, 0.0);
  mul_add<DA, DB>(a, b, c);
  return c;
}

__device__ __forceinline__ double2 det3(const M3 &m) {
  const double2 *a = m.a;
  const double2 t0 = cdet2(a[4], a[8], a[5], a[7]);
  const double2 t1 = cdet2(a[5], a[6], a[3], a[8]);
  const double2 t2 = cdet2(a[3], a[7], a[4], a[6]);
  return cfma(a[2], t2, cfma(a[1], t1, cm(a[0], t0)));
}

// P(X): scaled Newton polar iteration, then the determinant's phase removed.
// One step is N = (g Y + (g Y)^-dag) / 2 = h Y + conj(C e) with C the cofactor
// matrix of Y ((Y^-1)^dag = conj(C / det Y)), h = g / 2 and e = s conj(det Y),
// s = 1 / (2 g |det Y|^2).  For Y = Q H (polar form) any positive g and s give
// N = Q (g H + c H^-1) / 2, the same Q: the scaled steps take g ~ |det Y|^(-1/3)
// and s = g^5 / 2 from FP32 arithmetic; the unscaled steps (g = 1) need s to
// FP64 accuracy, since with c != 1 the iterates would converge to sqrt(c) Q.
// Scaling while a step still changes Y by more than 1 % (relative); the
// iteration stops after an unscaled step that changed it by less than 1e-8:
// near the fixed point such a step leaves an error of about half its square
// (~5e-17, FP64 rounding).  The singular values of every iterate are >= 1
// (those of (g H + c H^-1) / 2 are >= sqrt(g c), = 1 unscaled), so |N|_F^2 >= 3
// and testing the squared step against 3 x (relative bound)^2 is never looser.
__device__ M3 project_su3(const M3 &X) {
  M3 Y = X;
  bool scaled = true;
  for (int it = 0; it < 60; ++it) {
    double2 C[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int r0 = (i + 1) % 3, r1 = (i + 2) % 3, c0 = (j + 1) % 3, c1 = (j + 2) % 3;
        C[i * 3 + j] = cdet2(Y.a[r0 * 3 + c0], Y.a[r1 * 3 + c1], Y.a[r0 * 3 + c1], Y.a[r1 * 3 + c0]);
      }
    const double2 d = cfma(Y.a[2], C[2], cfma(Y.a[1], C[1], cm(Y.a[0], C[0])));
    const double dd = __fma_rn(d.x, d.x, d.y * d.y);
    double h, sc;
    if (scaled) {
      // g = |det Y|^(-1/3) = dd^(-1/6)
      const double g = (dd > 1e-30 && dd < 1e30) ? (double)sqrtf(rcbrtf((float)dd)) : sqrt(rcbrt(dd));
      const double g2 = g * g;
      h = 0.5 * g;
      sc = 0.5 * (g2 * g2 * g);
    } else {
      h = 0.5;
      sc = 0.5 / dd;
    }
    const double2 e = make_double2(sc * d.x, -sc * d.y);
    double diff = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double2 c = C[k], y = Y.a[k];
      const double2 n = make_double2(__fma_rn(c.x, e.x, __fma_rn(-c.y, e.y, h * y.x)),
                                     __fma_rn(-c.x, e.y, __fma_rn(-c.y, e.x, h * y.y)));
      const double ex = n.x - y.x, ey = n.y - y.y;
      diff = __fma_rn(ex, ex, __fma_rn(ey, ey, diff));
      Y.a[k] = n;
    }
    if (!scaled && diff <= 3e-16) break;
    if (diff <= 3e-4) scaled = false;
  }
  // z = exp(-i arg(det Y) / 3), principal branch: an FP32 estimate (the branch
  // follows the sign of Im det, kept by the conversion), then two Newton steps
  // on z^3 det Y = 1 in FP64, z <- z (4 - z^3 det Y) / 3 (the residual
  // w - 1 becomes -(2/3)(w - 1)^2 + O((w - 1)^3): 1e-7 -> 1e-14 -> rounding)
  const double2 d = det3(Y);
  float sf, cf;
  sincosf(atan2f((float)d.y, (float)d.x) / 3.0f, &sf, &cf);
  double2 z = make_double2((double)cf, -(double)sf);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const double2 w = cm(cm(cm(z, z), z), d);
    z = cm(z, make_double2((4.0 - w.x) * (1.0 / 3.0), -w.y * (1.0 / 3.0)));
  }
  M3 W;
#pragma unroll
  for (int k = 0; k < 9; ++k) W.a[k] = cm(Y.a[k], z);
  return W;
}

struct Lat {
  int L[4];
  long long V;
};

__device__ __forceinline__ void coords(const Lat &g, long long i, int (&x)[4]) {
  x[0] = (int)(i % g.L[0]);
  i /= g.L[0];
  x[1] = (int)(i % g.L[1]);
  i /= g.L[1];
  x[2] = (int)(i % g.L[2]);
  x[3] = (int)(i / g.L[2]);
}

__device__ __forceinline__ long long lexs(const Lat &g, const int (&x)[4], int d, int s, int d2 = -1, int s2 = 0) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[d] = (y[d] + s + g.L[d]) % g.L[d];
  if (d2 >= 0) y[d2] = (y[d2] + s2 + g.L[d2]) % g.L[d2];
  return y[0] + (long long)g.L[0] * (y[1] + (long long)g.L[1] * (y[2] + (long long)g.L[2] * y[3]));
}

// slot of the decorated link (dir, deco != dir) among the 12 stored: [dir][3]
__device__ __forceinline__ int dslot(int dir, int deco) { return dir * 3 + (deco < dir ? deco : deco - 1); }

// a field of links: thin (deco < 0: [dir][V]) or decorated ([12][V], slot dslot(dir, deco))
struct Fld {
  const double2 *p;
  long long V;
  __device__ __forceinline__ const double2 *at(int dir, int deco, long long site) const {
    return deco < 0 ? p + ((long long)dir * V + site) * 9 : p + ((long long)dslot(dir, deco) * V + site) * 9;
  }
};

// acc += the two staples in direction d of the link (x, mu): side links of
// field A with decoration da, middle link of field B with decoration db
__device__ __forceinline__ void staples(const Lat &g, const int (&x)[4], long long i, int mu, int d, const Fld &A,
                                        int da, const Fld &B, int db, M3 &acc) {
  // + d: A_d(x) B_mu(x+d) A_d(x+mu)^dag
  {
    const M3 a = ld(A.at(d, da, i));
    const M3 b = ld(B.at(mu, db, lexs(g, x, d, 1)));
    const M3 c = ld(A.at(d, da, lexs(g, x, mu, 1)));
    const M3 t = mul<false, false>(a, b);
    mul_add<false, true>(t, c, acc);
  }
  // - d: A_d(x-d)^dag B_mu(x-d) A_d(x-d+mu)
  {
    const long long xm = lexs(g, x, d, -1);
    const M3 a = ld(A.at(d, da, xm));
    const M3 b = ld(B.at(mu, db, xm));
    const M3 c = ld(A.at(d, da, lexs(g, x, d, -1, mu, 1)));
    const M3 t = mul<true, false>(a, b);
    mul_add<false, false>(t, c, acc);
  }
}

__device__ __forceinline__ void smear_store(const double2 *u, double a, double w, const M3 &acc, double2 *out) {
  M3 X;
#pragma unroll
  for (int k = 0; k < 9; ++k) X.a[k] = make_double2((1.0 - a) * u[k].x + w * acc.a[k].x, (1.0 - a) * u[k].y + w * acc.a[k].y);
  const M3 W = project_su3(X);
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = W.a[k];
}

// level 1: thread over (mu, e != mu, site); Vb stored [dslot(mu, e)][V]
__global__ void k_hyp1(Lat g, const double2 *U, double a3, double2 *Vb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 12 * g.V) return;
  const long long i = t % g.V;
  const int pr = (int)(t / g.V), mu = pr / 3, e = (pr % 3 >= mu) ? pr % 3 + 1 : pr % 3;
  int x[4];
  coords(g, i, x);
  const Fld thin{U, g.V};
  M3 acc;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc.a[k] = make_double2(0.0, 0.0);
  staples(g, x, i, mu, e, thin, -1, thin, -1, acc);
  smear_store(thin.at(mu, -1, i), a3, a3 / 2.0, acc, Vb + ((long long)dslot(mu, e) * g.V + i) * 9);
}

// level 2: thread over (mu, nu != mu, site); Vt stored [dslot(mu, nu)][V]
__global__ void k_hyp2(Lat g, const double2 *U, const double2 *Vb, double a2, double2 *Vt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 12 * g.V) return;
  const long long i = t % g.V;
  const int pr = (int)(t / g.V), mu = pr / 3, nu = (pr % 3 >= mu) ? pr % 3 + 1 : pr % 3;
  int x[4];
  coords(g, i, x);
  const Fld vb{Vb, g.V};
  M3 acc;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc.a[k] = make_double2(0.0, 0.0);
  for (int r = 0; r < 4; ++r) {
    if (r == mu || r == nu) continue;
    const int s = 6 - mu - nu - r;  // the direction outside {mu, nu, r}
    staples(g, x, i, mu, r, vb, s, vb, s, acc);
  }
  smear_store(U + ((long long)mu * g.V + i) * 9, a2, a2 / 4.0, acc, Vt + ((long long)dslot(mu, nu) * g.V + i) * 9);
}

// level 3: thread over (mu, site); out may alias U (each thread reads only its own thin link)
__global__ void k_hyp3(Lat g, const double2 *U, const double2 *Vt, double a1, double2 *out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * g.V) return;
  const long long i = t % g.V;
  const int mu = (int)(t / g.V);
  int x[4];
  coords(g, i, x);
  const Fld vt{Vt, g.V};
  M3 acc;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc.a[k] = make_double2(0.0, 0.0);
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    // sides Vt(., nu; mu), middle Vt(., mu; nu)
    // + nu
    {
      const M3 a = ld(vt.at(nu, mu, i));
      const M3 b = ld(vt.at(mu, nu, lexs(g, x, nu, 1)));
      const M3 c = ld(vt.at(nu, mu, lexs(g, x, mu, 1)));
      mul_add<false, true>(mul<false, false>(a, b), c, acc);
    }
    // - nu
    {
      const long long xm = lexs(g, x, nu, -1);
      const M3 a = ld(vt.at(nu, mu, xm));
      const M3 b = ld(vt.at(mu, nu, xm));
      const M3 c = ld(vt.at(nu, mu, lexs(g, x, nu, -1, mu, 1)));
      mul_add<false, false>(mul<true, false>(a, b), c, acc);
    }
  }
  double2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = U[((long long)mu * g.V + i) * 9 + k];
  smear_store(u, a1, a1 / 6.0, acc, out + ((long long)mu * g.V + i) * 9);
}

}  // namespace

cudaError_t launch_hyp(const int dims[4], const double2 *U, const double alpha[3], double2 *Vb, double2 *Vt,
                       double2 *out, cudaStream_t st) {
  Lat g;
  for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
  g.V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  const int bt = 128;
  k_hyp1<<<(unsigned)((12 * g.V + bt - 1) / bt), bt, 0, st>>>(g, U, alpha[2], Vb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hyp2<<<(unsigned)((12 * g.V + bt - 1) / bt), bt, 0, st>>>(g, U, Vb, alpha[1], Vt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_hyp3<<<(unsigned)((4 * g.V + bt - 1) / bt), bt, 0, st>>>(g, U, Vt, alpha[0], out);
  return cudaGetLastError();
}

}  // namespace stag
