// multishift.cu -- the shifted-system update of the multi-shift CG (several
// masses of one source on one Krylov space; Sec. 3's inverter run for the
// 12-source x 4-mass workload).  One kernel per base iteration, launched
// between the two CG kernels: it finishes the first kernel's reduction itself
// (the same fixed-order fold the second kernel runs, so its alpha_k is
// bit-identical to the base's), advances every active shift's zeta, alpha,
// beta (FP64 scalars, recurrence in ShiftState's comment), and updates
//   p_s = zeta_k r_k + beta_s p_s,   x_s += alpha_s p_s   (FP32 per site).
// The base system's reliable updates leave the shifts alone: shifted
// solutions reach the FP32 floor of their own systems (~eps_32 kappa_s) and are
// refined to the tolerance afterwards (api.cu).
#include "launch.h"

namespace stag {

constexpr int MS_BT = 128;

__global__ void __launch_bounds__(MS_BT) k_shift_update(const MsArgs a) {
  const int j = blockIdx.x / a.nbx, bx = blockIdx.x % a.nbx;
  const int Ve = a.d.g.Ve;
  grid_dep_trigger();
  grid_dep_wait();
  __shared__ SysState sst[1];
  if (a.d.fold != FIN_NONE) {
    fold_state<1, MS_BT>(a.d, j, 1, sst);  // bx0 = 1: compute, never store the base state
  } else {
    if (threadIdx.x == 0) sst[0] = a.d.ctl.st[j];
    __syncthreads();
  }
  const SysState S = sst[0];
  if (S.done != 0) return;  // the base system is gated off (uniform over the block)
  constexpr int QMAX = 16;
  float cr[QMAX], cp[QMAX], ca[QMAX];
  bool on[QMAX];
  const int nsh = a.nsh < QMAX ? a.nsh : QMAX;
  for (int q = 0; q < nsh; ++q) {
    const ShiftState h = a.sh[(long long)j * a.nsh + q];
    on[q] = h.active != 0;
    if (!on[q]) continue;
    const double z = h.zeta, zp = h.zeta_prev, ap = h.alpha_prev;
    const double al = S.alpha, bp = S.beta;
    const double zn = z * zp * ap / (al * bp * (zp - z) + zp * ap * (1.0 + h.dm4 * al));
    const double zr = z / zp;
    cr[q] = (float)z;
    cp[q] = (float)(bp * zr * zr);
    ca[q] = (float)(al * zn / z);
    if (bx == 0 && threadIdx.x == 0) {
      ShiftState n = h;
      n.zeta_prev = z;
      n.zeta = zn;
      n.alpha_prev = al;
      n.iter = h.iter + 1;
      n.active = (zn * zn * S.rho <= a.tol2 * S.bnorm2 || !isfinite(zn)) ? 0 : 1;
      a.sh[(long long)j * a.nsh + q] = n;
    }
  }
  for (int s = bx * MS_BT + (int)threadIdx.x; s < Ve; s += a.nbx * MS_BT) {
    float r[6];
    load_vec<P32>(a.r, j, s, Ve, r);
    for (int q = 0; q < nsh; ++q) {
      if (!on[q]) continue;
      const int k = j * a.nsh + q;
      float p[6], x[6];
      load_vec_rw<P32>(a.ps, k, s, Ve, p);
      load_vec_rw<P32>(a.xs, k, s, Ve, x);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        p[i] = cr[q] * r[i] + cp[q] * p[i];
        x[i] += ca[q] * p[i];
      }
      store_vec<P32>(a.ps, k, s, Ve, p);
      store_vec<P32>(a.xs, k, s, Ve, x);
    }
  }
}

cudaError_t launch_shift_update(const MsArgs &a, cudaStream_t st) {
  return launch_ex(k_shift_update, a.nbx * a.d.nsys, MS_BT, st, a.d.pdl != 0, a);
}

// every system still running gets a reliable update pending (the first step
// of a solve from an initial guess: r = b - A x0 recomputed in FP64)
__global__ void k_mark_update(SysState *st, int nsys) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nsys && st[j].done == 0) st[j].update = 1;
}

cudaError_t launch_mark_update(SysState *st, int nsys, cudaStream_t s) {
  k_mark_update<<<(nsys + 127) / 128, 128, 0, s>>>(st, nsys);
  return cudaGetLastError();
}

}  // namespace stag
